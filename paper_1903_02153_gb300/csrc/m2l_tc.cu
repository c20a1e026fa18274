// m2l_tc.cu -- far-field stage (Sec. 2.3 item 2) on the 5th-generation tensor
// cores:  F~^alpha = scale_l * sum_{beta in I(alpha)} C^(t) M~^beta  with the
// compressed operators C^(t) = U^T K^(t) V (Sec. 2.5 "Fast M2L translation").
//
// The stage is a dense contraction.  For a tile of N targets (a box of parent
// cells of one octant class; N = 256 for the 16-bit forms, 128 for TF32, less
// on the two coarsest levels) and each of the 189 offsets of the class:
//     D[k][n] += sum_j C^(t)[k][j] M~[source(n, t)][j],   k < r, n < N.
// The MMA's M side is the operator's r output coefficients (padded to 128
// lanes), its N side the targets: one instruction then carries 128 x N x K
// products, and the instruction count per target is a half (N = 256) of what
// a targets-by-coefficients orientation (N = r) needs.  Each level uses the
// rank of its own operators (r_l, the columns past it are zero); a level with
// r_l in (128, 256] runs every tile twice, once per half of the rows.  Source vectors come
// straight out of the parity-split M~ array: for one offset and one tile the
// sources are a box of consecutive parent cells of one source octant, one TMA
// box load; out-of-range cells read as zero.  K is walked in chunks of 32
// elements (a 128-byte row of TF32, a 64-byte row of FP16 / BF16).
//
// One persistent launch covers every level 2..D.  The (tile, offset) pairs of
// all levels are numbered tile by tile and every CTA takes an equal
// contiguous range of them (a load balance to one offset).  A range cuts a
// tile into at most G segments; a segment's partial sum goes to slice g of the
// level's F~ buffer (g = the number of range boundaries inside the tile before
// it), and the downward pass adds the G slices in a fixed order
// (deterministic).  Slices no segment writes were zeroed before the launch.
//
//   warp 0         TMA producer: one lane arms a stage barrier and issues the
//                  box loads of C (and its low part) and of the sources (and
//                  their low part)
//   warp 1         MMA issuer: one lane issues tcgen05.mma, M = 128 (rows of
//                  C), N = tile size, K = 16 (f16 kinds) or 8 (tf32)
//   warps 2..      epilogue: thread = one TMEM lane (coefficient k) and 128
//                  target columns; after every offset it drains that
//                  offset's partial accumulator into FP32 registers; at the
//                  end of an item it scales and stores (a warp's 32 lanes
//                  store 32 consecutive coefficients of one target)
//   (When no level's rank exceeds 96, TMEM lane quadrant 3 holds no
//   coefficients: the 256-target launch then has 8 warps, epilogue warps
//   0-2 and 4-6, the producer 3 and the MMA issuer 7.)
//
// Precision: kind::tf32 reads 10 explicit mantissa bits.  The 3-pass mode
// splits each operand into hi and lo and forms hi*hi + hi*lo + lo*hi (the
// split-TF32 scheme of Ootomo & Yokota, 2022; the same with FP16 pieces after
// a power-of-two scale, or BF16 pieces).  The tensor core's own accumulation
// truncates; long runs of it (189 offsets x r/8 steps into one accumulator)
// lost ~1e-5 relative on the 1M-point workload, so, as that scheme
// prescribes, a TMEM accumulator only ever holds one offset and the sum over
// offsets is taken in FP32 registers with round-to-nearest.  Within an
// offset the correction products either have their own accumulator (NACC =
// 2) or, when TMEM has room for one accumulator per buffer only, each chunk's
// corrections are issued before its hi*hi (CF), so they are summed while the
// accumulator is still small.
//
// Every mbarrier wait is bounded (about 2^31 cycles): on expiry the kernel
// sets the plan's status word, stops issuing work, waits (bounded) for its own
// copies and MMAs in flight, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <math.h>
#include <string.h>

#include "bbfmm_internal.h"
#include "tc_ptx.cuh"

namespace bbfmm {

// ---------------------------------------------------------------------------
// host side: operand splitting (operators are split once, at upload)
static inline float to_tf32_host(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) { // finite: round to nearest, ties to even
        uint32_t lsb = (b >> 13) & 1u;
        b += 0x0fffu + lsb;
        b &= 0xffffe000u;
    }
    float y;
    memcpy(&y, &b, 4);
    return y;
}

void split_tf32(const float *in, float *hi, float *lo, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        float h = to_tf32_host(in[i]);
        hi[i] = h;
        lo[i] = to_tf32_host(in[i] - h);
    }
}

// K elements per pipeline stage: 32 (one 128-byte TF32 row, or one 64-byte
// FP16 / BF16 row in the 64-byte swizzle)
constexpr int kKChunk = 32;
// K elements per stage of the 16-bit forms: 32 (64-byte rows, 64-byte
// swizzle) or 64 (128-byte rows, 128-byte swizzle: half the TMA rows per byte)
#ifndef BBFMM_TC_K16
#define BBFMM_TC_K16 32
#endif
constexpr int kKChunk16 = BBFMM_TC_K16;
static_assert(kKChunk16 == 32 || kKChunk16 == 64, "16-bit K chunk is 32 or 64 elements");
__host__ __device__ constexpr int kchunk_of(int fmt) { return fmt == 0 ? kKChunk : kKChunk16; }
#ifndef BBFMM_TC_MAX_STAGES
#define BBFMM_TC_MAX_STAGES 8
#endif
constexpr int kMaxStages = BBFMM_TC_MAX_STAGES; // pipeline stages (shared memory permitting)
// targets per tile on the fine levels: 256 for the 16-bit forms, 128 for TF32
#ifndef BBFMM_TC_TILE16
#define BBFMM_TC_TILE16 256
#endif
constexpr int kTile16 = BBFMM_TC_TILE16;
static_assert(kTile16 == 128 || kTile16 == 256, "16-bit tile is 128 or 256 targets");

// ---------------------------------------------------------------------------
// Work entries of an octant class: a group of offsets that share a source
// octant and (ux, uy) and differ in uz.  The entry's sources are one box load
// of bz + zspan slabs; offset j of the entry reads it from slab d_j, so one
// load serves up to kMaxOps operators.  Table 0: one offset per entry (189);
// table 1: grouped (72 entries).  Encoding: x = op0 | op1 << 10 | op2 << 20,
// y = source octant | nops << 3 | zspan << 5, z = (ux + 1) | (uy + 1) << 2 |
// (uz_min + 1) << 4, w = d0 | d1 << 2 | d2 << 4.
constexpr int kMaxOps = 3;
constexpr int kEntries16 = 72; // grouped entries per class
#ifndef BBFMM_TC_GROUP
#define BBFMM_TC_GROUP 1
#endif
constexpr bool kGroupEntries = BBFMM_TC_GROUP != 0; // 16-bit forms: group the offsets that share sources
__constant__ int4 c_ent_tc[2][8][kOffsetsPerClass];

constexpr int kMaxTcLevels = 8;
constexpr int kMaxBuf = 8;

struct TcLevel {
    float *Ft;                // partial slice g at Ft + g * slice
    int64_t slice;            // floats per slice
    int H, bx, by, bz, lbx, lby, n; // tile extent (log2 of bx, by) and N = bx by bz
    const int4 *tl;           // the level's active tiles {tx, ty, tz, octant} (device)
    int nact, ntiles, tile_base, opl, l; // active tiles; x right-hand sides x row halves; first tile number
    int r, nk, ktail, nh;     // rank of the level's operators, K chunks, K steps of the last chunk, row halves
    uint32_t idesc;           // instruction descriptor (N of this level)
    uint32_t a_load, b_load;  // bytes of the operator rows loaded / of the sources (one piece, one chunk)
    uint32_t b_load2;         // sources of a grouped entry: bz + 2 slabs
    uint32_t slab16;          // one slab of sources (bx by rows) in descriptor units (16 bytes)
    int E, grp;               // entries per class and entry table of this level
    int64_t pair_base;        // first (tile, entry) pair of the level
    float scale;
};

struct TcLaunch {
    CUtensorMap src[kMaxTcLevels], srclo[kMaxTcLevels]; // M~ (hi, lo) of each level
    CUtensorMap src2[kMaxTcLevels], srclo2[kMaxTcLevels]; // the same with bz + 2 slabs (grouped entries)
    CUtensorMap op[kMaxTcLevels], oplo[kMaxTcLevels];   // C (hi, lo) of each operator level
    TcLevel lev[kMaxTcLevels];
    float bscale_inv[kMaxTcLevels]; // 1 / (scale of the 16-bit operators), per operator level
    const float *ascale;            // 16-bit forms: scale of M~ per tree level (device)
    int nlev, ntiles;               // levels; tiles of all levels
    int64_t total, per_cta;         // (tile, entry) pairs; pairs per CTA
    int maxops;                     // operator tiles per stage
    int q3;                         // three epilogue quadrants (ranks <= 96): 256 threads, see the kernel
    int *status;
    int rp, nrhs, R, nstage;            // R: right-hand-side stride of M~ / F~ rows
    int nbuf, bcols, tcols;             // TMEM partial buffers, columns per accumulator, allocated
    uint32_t stage_bytes, a_bytes, b_bytes; // a: C tile (128 rows); b: sources
};

struct Item {
    int L, tx, ty, tz, ot, c, h, g, e0, e1; // h: the 128 operator rows [128 h, 128 h + 128)
};

// the segment of this CTA's range that starts at pair `pos`
__device__ __forceinline__ Item decode_segment(const TcLaunch &P, int64_t pos, int64_t end)
{
    Item it;
    int L = 0;
    while (L + 1 < P.nlev && pos >= P.lev[L + 1].pair_base)
        ++L;
    it.L = L;
    const TcLevel &lv = P.lev[L];
    const int64_t rel = pos - lv.pair_base;
    int u = (int)(rel / lv.E); // the level's tile: ((c nact) + tile) nh + h, the row halves back to back
    it.e0 = (int)(rel - (int64_t)u * lv.E);
    it.e1 = (int)min((int64_t)lv.E, it.e0 + (end - pos));
    it.g = (int)(pos / P.per_cta - (lv.pair_base + (int64_t)u * lv.E) / P.per_cta);
    it.h = 0;
    if (lv.nh > 1) {
        it.h = u & 1;
        u >>= 1;
    }
    it.c = u / lv.nact;
    const int4 e = lv.tl[u - it.c * lv.nact];
    it.tx = e.x;
    it.ty = e.y;
    it.tz = e.z;
    it.ot = e.w;
    return it;
}

// FMT: operand format, 0 = TF32 (kind::tf32, K = 8 per MMA, 128-byte rows),
// 1 = FP16, 2 = BF16 (kind::f16, K = 16 per MMA, 64-byte rows).
// NACC: accumulators per partial buffer (2: hi*hi and corrections apart).
// CH: target columns / 128 (epilogue warp groups).
template <int NPROD, int NACC, bool CF, int CH, int FMT>
__global__ void __launch_bounds__(64 + 128 * CH, 1) k_m2l_tc(const __grid_constant__ TcLaunch P)
{
    constexpr int KSTEP = FMT == 0 ? 8 : 16; // K elements per MMA (32 bytes)
    constexpr int KCH = kchunk_of(FMT);      // K elements per stage
    constexpr int KMAX = KCH / KSTEP;        // MMAs per piece product and chunk
    constexpr bool SW64 = FMT != 0 && KCH == 32; // 64-byte rows
    constexpr int MAXOPS = FMT != 0 && kGroupEntries ? kMaxOps : 1; // operators per entry
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = smem_raw + (base - raw);
    const int S = P.nstage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (size_t)S * P.stage_bytes);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
    const uint32_t pfull0 = empty0 + 8 * S, pempty0 = pfull0 + 8 * kMaxBuf, done_bar = pempty0 + 8 * kMaxBuf;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 2 * kMaxBuf + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int NB = P.nbuf;
    const uint32_t tcols = (uint32_t)P.tcols;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(pfull0 + 8 * b, 1);
            mbar_init(pempty0 + 8 * b, (P.q3 ? 3 : 4) * CH);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // warp roles: producer, MMA issuer and 4 CH epilogue warps (TMEM lane
    // quadrant q = warp & 3); with q3 (every level's rank <= 96, so lane
    // quadrant 3 holds no coefficients) the block is 8 warps: epilogue warps
    // 0-2 and 4-6 (quadrants 0-2 of the two column halves), producer 3, MMA 7.
    // The two dropped warps' registers let the near field keep more blocks on
    // the SM beside this one.
    const int wprod = P.q3 ? 3 : 0, wmma = P.q3 ? 7 : 1;
    if (warp == wmma) {
        tmem_alloc(smem_u32(tmem_slot), tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == wprod && lane == 0) {
        // ------------------------------------------------------------ producer
        int last_round[kMaxStages];
        for (int s = 0; s < kMaxStages; ++s)
            last_round[s] = -1;
        int s = 0, round = 0;
        const int64_t end = min(P.total, (int64_t)(blockIdx.x + 1) * P.per_cta);
        for (int64_t pos = (int64_t)blockIdx.x * P.per_cta; pos < end && !*abort_flag;) {
            const Item w = decode_segment(P, pos, end);
            pos += w.e1 - w.e0;
            const TcLevel &lv = P.lev[w.L];
            const int X0 = lv.bx * w.tx, Y0 = lv.by * w.ty, Z0 = lv.bz * w.tz;
            constexpr uint32_t npc = NPROD == 3 ? 2u : 1u; // pieces (hi, lo)
            const int row0 = 128 * w.h;
            for (int e = w.e0; e < w.e1 && !*abort_flag; ++e) {
                const int4 en = c_ent_tc[lv.grp][w.ot][e];
                const int nops = MAXOPS == 1 ? 1 : (en.y >> 3) & 3, zspan = en.y >> 5, soct = en.y & 7;
                const int ux = (en.z & 3) - 1, uy = ((en.z >> 2) & 3) - 1, uz = ((en.z >> 4) & 3) - 1;
                const int zq = soct * (lv.H + 2) + 1 + Z0 + uz;
                const uint32_t tx_bytes = npc * ((uint32_t)nops * lv.a_load + (zspan ? lv.b_load2 : lv.b_load));
                const CUtensorMap *bm = zspan ? &P.src2[w.L] : &P.src[w.L];
                const CUtensorMap *bml = zspan ? &P.srclo2[w.L] : &P.srclo[w.L];
                for (int kc = 0; kc < lv.nk; ++kc) {
                    if (!mbar_wait(empty0 + 8 * s, round ^ 1, abort_flag))
                        break;
                    const uint32_t sa = base + (uint32_t)s * P.stage_bytes;
                    const uint32_t fb = full0 + 8 * s;
                    mbar_arrive_expect_tx(fb, tx_bytes);
                    last_round[s] = round;
                    // stage: [op 0 hi, lo][op 1 hi, lo]... (maxops slots) [sources hi][lo]
                    const uint32_t sb = sa + npc * (uint32_t)P.maxops * P.a_bytes;
#pragma unroll
                    for (int j = 0; j < MAXOPS; ++j)
                        if (MAXOPS == 1 || j < nops) {
                            const int opi = (en.x >> (10 * j)) & 1023;
                            const uint32_t aj = sa + npc * (uint32_t)j * P.a_bytes;
                            tma_load_3d(aj, &P.op[lv.opl], fb, KCH * kc, row0, opi);
                            if (NPROD == 3)
                                tma_load_3d(aj + P.a_bytes, &P.oplo[lv.opl], fb, KCH * kc, row0, opi);
                        }
                    tma_load_5d(sb, bm, fb, KCH * kc, w.c, X0 + ux, Y0 + uy, zq);
                    if (NPROD == 3)
                        tma_load_5d(sb + P.b_bytes, bml, fb, KCH * kc, w.c, X0 + ux, Y0 + uy, zq);
                    if (++s == S) {
                        s = 0;
                        round ^= 1;
                    }
                }
            }
        }
        // teardown: every armed stage must have landed before the CTA exits
        for (int q = 0; q < S; ++q)
            if (last_round[q] >= 0) {
                long long t0 = clock64();
                while (!mbar_test(full0 + 8 * q, (uint32_t)last_round[q]) && clock64() - t0 < kWaitCycles) {
                }
            }
    } else if (warp == wmma && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        // One thread issues every MMA of the CTA, so this loop is kept short:
        // ring positions are counters (no division), the descriptors of a
        // stage are the stage-0 descriptors plus a constant, the K steps of a
        // chunk are unrolled.
        constexpr uint32_t npc = NPROD == 3 ? 2u : 1u;
        const uint32_t b_off = npc * (uint32_t)P.maxops * P.a_bytes;
        const uint64_t d0 = SW64 ? sw64_desc(base) : sw128_desc(base);
        const uint32_t d_al = P.a_bytes >> 4, d_aop = (npc * P.a_bytes) >> 4; // lo piece; next operator
        const uint32_t d_bh = b_off >> 4, d_bl = (b_off + P.b_bytes) >> 4;
        const uint32_t d_st = P.stage_bytes >> 4;
        int s = 0, sph = 0, pb = 0, pph = 0; // stage ring and partial-buffer ring (position, phase)
        bool ok = true;
        const int64_t end = min(P.total, (int64_t)(blockIdx.x + 1) * P.per_cta);
        for (int64_t pos = (int64_t)blockIdx.x * P.per_cta; pos < end && ok && !*abort_flag;) {
            const Item w = decode_segment(P, pos, end);
            pos += w.e1 - w.e0;
            const TcLevel &lv = P.lev[w.L];
            const uint32_t idesc = lv.idesc;
            const int nk = lv.nk, ktail = lv.ktail;
            for (int e = w.e0; e < w.e1 && ok; ++e) {
                const int4 en = c_ent_tc[lv.grp][w.ot][e];
                const int nops = MAXOPS == 1 ? 1 : (en.y >> 3) & 3;
                // source slab of operator j within the entry's box load
                uint32_t sh[MAXOPS];
#pragma unroll
                for (int j = 0; j < MAXOPS; ++j)
                    sh[j] = MAXOPS == 1 ? 0u : (uint32_t)((en.w >> (2 * j)) & 3) * lv.slab16;
                if (!mbar_wait(pempty0 + 8 * pb, pph ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dh = tmem_base + (uint32_t)(pb * NACC * P.bcols);
                const uint32_t dc = NACC == 2 ? dh + (uint32_t)P.bcols : dh;
                uint32_t acc_h = 0, acc_c = 0;
                for (int kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(full0 + 8 * s, sph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t sbase = d0 + (uint64_t)(s * d_st);
                    const uint64_t bh0 = sbase + d_bh, bl0 = sbase + d_bl; // sources (hi, lo)
                    const int ks = kc + 1 < nk ? KMAX : ktail;
                    auto issue = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
                        if (FMT == 0)
                            mma_tf32(d, a, b, idesc, acc);
                        else
                            mma_f16(d, a, b, idesc, acc);
                    };
                    // the entry's operators one after the other, all into the
                    // entry's partial accumulator; operator j reads the
                    // sources from its slab
                    if (NPROD == 3 && (NACC == 2 || CF)) {
#pragma unroll
                        for (int j = 0; j < MAXOPS; ++j)
                            if (MAXOPS == 1 || j < nops) {
                                const uint64_t ah = sbase + (uint64_t)(j * d_aop), al = ah + d_al;
                                const uint64_t bh = bh0 + sh[j], bl = bl0 + sh[j];
#pragma unroll
                                for (int k = 0; k < KMAX; ++k)
                                    if (k < ks) {
                                        const uint64_t dk = (uint64_t)(2 * k); // 32 bytes >> 4
                                        issue(dc, ah + dk, bl + dk, acc_c);
                                        issue(dc, al + dk, bh + dk, 1u);
                                        acc_c = 1u;
                                        if (NACC == 1)
                                            acc_h = 1u;
                                    }
                            }
                    }
#pragma unroll
                    for (int j = 0; j < MAXOPS; ++j)
                        if (MAXOPS == 1 || j < nops) {
                            const uint64_t ah = sbase + (uint64_t)(j * d_aop);
                            const uint64_t bh = bh0 + sh[j];
#pragma unroll
                            for (int k = 0; k < KMAX; ++k)
                                if (k < ks) {
                                    const uint64_t dk = (uint64_t)(2 * k);
                                    issue(dh, ah + dk, bh + dk, acc_h);
                                    acc_h = 1u;
                                }
                        }
                    if (NPROD == 3 && NACC == 1 && !CF) {
#pragma unroll
                        for (int j = 0; j < MAXOPS; ++j)
                            if (MAXOPS == 1 || j < nops) {
                                const uint64_t ah = sbase + (uint64_t)(j * d_aop), al = ah + d_al;
                                const uint64_t bh = bh0 + sh[j], bl = bl0 + sh[j];
#pragma unroll
                                for (int k = 0; k < KMAX; ++k)
                                    if (k < ks) {
                                        const uint64_t dk = (uint64_t)(2 * k);
                                        issue(dh, ah + dk, bl + dk, 1u);
                                        issue(dh, al + dk, bh + dk, 1u);
                                    }
                            }
                    }
                    mma_commit(empty0 + 8 * s); // frees the stage once these MMAs have read it
                    if (++s == S) {
                        s = 0;
                        sph ^= 1;
                    }
                }
                if (!ok)
                    break;
                mma_commit(pfull0 + 8 * pb); // the offset's partial sums are complete
                if (++pb == NB) {
                    pb = 0;
                    pph ^= 1;
                }
            }
        }
        // all MMAs issued by this thread have completed before TMEM is freed
        mma_commit(done_bar);
        long long t0 = clock64();
        while (!mbar_test(done_bar, 0) && clock64() - t0 < kWaitCycles) {
        }
    } else if (P.q3 ? (warp != wprod && warp != wmma) : warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int ew = P.q3 ? warp : warp - 2;
        const int q = warp & 3;   // TMEM lane quadrant this warp may access
        const int half = ew >> 2; // target columns [128 half, 128 half + 128)
        const uint32_t tlane = tmem_base + ((uint32_t)(32 * q) << 16);
        int pb = 0, pph = 0; // partial-buffer ring (position, phase)
        bool ok = true;
        const int64_t end = min(P.total, (int64_t)(blockIdx.x + 1) * P.per_cta);
        for (int64_t pos = (int64_t)blockIdx.x * P.per_cta; pos < end && ok;) {
            const Item w = decode_segment(P, pos, end);
            pos += w.e1 - w.e0;
            const TcLevel &lv = P.lev[w.L];
            const int ncol = min(128, lv.n - 128 * half); // target columns of this warp
            const int k = 128 * w.h + 32 * q + lane;     // output coefficient of this thread
            const bool rows = 128 * w.h + 32 * q < lv.r; // warp-uniform: the quadrant holds coefficients
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j)
                acc[j] = 0.0f;
            for (int e = w.e0; e < w.e1; ++e) {
                int got = 1;
                if (lane == 0)
                    got = mbar_wait(pfull0 + 8 * pb, pph, abort_flag) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0); // keep the warp converged for tcgen05.ld
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (rows) {
#pragma unroll
                    for (int a = 0; a < NACC; ++a) {
                        const uint32_t tb = tlane + (uint32_t)((pb * NACC + a) * P.bcols + 128 * half);
#pragma unroll
                        for (int c32 = 0; c32 < 4; ++c32) {
                            if (32 * c32 + 32 <= ncol) {
                                float v[32];
                                tmem_ld32(tb + (uint32_t)(32 * c32), v);
#pragma unroll
                                for (int j = 0; j < 32; ++j)
                                    acc[32 * c32 + j] += v[j];
                            } else if (32 * c32 < ncol) {
                                float v[16];
                                tmem_ld16(tb + (uint32_t)(32 * c32), v);
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    acc[32 * c32 + j] += v[j];
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(pempty0 + 8 * pb);
                if (++pb == NB) {
                    pb = 0;
                    pph ^= 1;
                }
            }
            if (!ok)
                break;
            if (!rows || k >= lv.r)
                continue;
            // level scale; 16-bit forms also undo the power-of-two operand scales
            float f = lv.scale;
            if (FMT != 0)
                f *= P.bscale_inv[lv.opl] / __ldg(P.ascale + lv.l);
            const int X0 = lv.bx * w.tx, Y0 = lv.by * w.ty, Z0 = lv.bz * w.tz;
            const int64_t rowstride = (int64_t)P.R * P.rp;
            float *out = lv.Ft + (int64_t)w.g * lv.slice + (int64_t)w.c * P.rp + k;
#pragma unroll
            for (int j = 0; j < 128; ++j) {
                const int t = 128 * half + j;
                const int X = X0 + (t & (lv.bx - 1)), Y = Y0 + ((t >> lv.lbx) & (lv.by - 1)),
                          Z = Z0 + (t >> (lv.lbx + lv.lby));
                if (j < ncol && X < lv.H && Y < lv.H && Z < lv.H)
                    out[((((int64_t)w.ot * lv.H + Z) * lv.H + Y) * lv.H + X) * rowstride] = f * acc[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_flag && threadIdx.x == 0)
        atomicOr(P.status, kStatusTimeout);
    if (warp == wmma) {
        __syncwarp();
        tmem_dealloc(tmem_base, tcols);
    }
}

// ---------------------------------------------------------------------------
// host: tensor maps, work split and launch
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_tc_mu;
static bool g_tab_tc_ready = false;
static int g_num_sms = 0;

static cudaError_t tc_init()
{
    std::lock_guard<std::mutex> g(g_tc_mu);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return cudaErrorNotSupported;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (!g_tab_tc_ready) {
        static int4 tab[8][kOffsetsPerClass];
        if (!fill_m2l_table(tab))
            return cudaErrorInvalidValue;
        static int4 ent[2][8][kOffsetsPerClass];
        memset(ent, 0, sizeof(ent));
        for (int o = 0; o < 8; ++o) {
            // table 0: one offset per entry
            for (int k = 0; k < kOffsetsPerClass; ++k) {
                const int4 t = tab[o][k];
                ent[0][o][k] = make_int4(t.x, t.y | (1 << 3), t.z, 0);
            }
            // table 1: offsets grouped by (source octant, ux, uy), uz ascending
            int n = 0, covered = 0;
            for (int q = 0; q < 8; ++q)
                for (int uy = -1; uy <= 1; ++uy)
                    for (int ux = -1; ux <= 1; ++ux) {
                        int ops[3], uzs[3], m = 0;
                        for (int uz = -1; uz <= 1; ++uz)
                            for (int k = 0; k < kOffsetsPerClass; ++k) {
                                const int4 t = tab[o][k];
                                if (t.y == q && (t.z & 3) - 1 == ux && ((t.z >> 2) & 3) - 1 == uy &&
                                    ((t.z >> 4) & 3) - 1 == uz) {
                                    if (m >= kMaxOps)
                                        return cudaErrorInvalidValue;
                                    ops[m] = t.x;
                                    uzs[m++] = uz;
                                }
                            }
                        if (m == 0)
                            continue;
                        const int uzmin = uzs[0], zspan = uzs[m - 1] - uzs[0];
                        if (zspan != 0 && zspan != 2 && !(zspan == 1 && m == 2))
                            return cudaErrorInvalidValue;
                        int x = 0, wv = 0;
                        for (int j = 0; j < m; ++j) {
                            x |= ops[j] << (10 * j);
                            wv |= (uzs[j] - uzmin) << (2 * j);
                        }
                        // the box load always covers bz + 2 slabs when the group spans z
                        const int span = zspan > 0 ? 2 : 0;
                        ent[1][o][n++] = make_int4(x, q | (m << 3) | (span << 5),
                                                   (ux + 1) | ((uy + 1) << 2) | ((uzmin + 1) << 4), wv);
                        covered += m;
                    }
            if (covered != kOffsetsPerClass || n != kEntries16)
                return cudaErrorInvalidValue;
        }
        cudaError_t e = cudaMemcpyToSymbol(c_ent_tc, ent, sizeof(ent));
        if (e != cudaSuccess)
            return e;
        g_tab_tc_ready = true;
    }
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return cudaSuccess;
}

static CUtensorMapDataType tm_type(int fmt)
{
    return fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                    : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
}

// M~ (parity split, padded in Z): dims (rp, R, H, H, 8 (H + 2)); box (32
// elements of K, 1, bx, by, bz): the sources of one tile for one offset
static cudaError_t encode_src(CUtensorMap *tm, const void *ptr, int H, int R, int rp, int fmt, int bx, int by,
                              int bz)
{
    const cuuint64_t es_b = fmt == 0 ? 4 : 2;
    cuuint64_t dims[5] = {(cuuint64_t)rp, (cuuint64_t)R, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)8 * (H + 2)};
    cuuint64_t strides[4] = {(cuuint64_t)rp * es_b, (cuuint64_t)R * rp * es_b, (cuuint64_t)H * R * rp * es_b,
                             (cuuint64_t)H * H * R * rp * es_b};
    const int kch = kchunk_of(fmt);
    cuuint32_t box[5] = {(cuuint32_t)kch, 1, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode(tm, tm_type(fmt), 5, (void *)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          kch * es_b == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// a 2D FP32 matrix (outer rows of inner elements, row pitch row_bytes), box
// of box_inner x box_outer with the 128-byte swizzle (box_inner = 32); shared
// with the leaf-box GEMMs (box_gemm.cu)
cudaError_t tc_encode_2d_f32(CUtensorMap *tm, const void *ptr, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                             uint32_t box_inner, uint32_t box_outer)
{
    cudaError_t e = tc_init();
    if (e != cudaSuccess)
        return e;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_sm_count()
{
    return tc_init() == cudaSuccess ? g_num_sms : 0;
}

// C (operators): dims (rp, rows64, 316); box (32 elements of K, nb rows, 1)
static cudaError_t encode_op(CUtensorMap *tm, const void *ptr, int rp, int rows64, int nb, int fmt)
{
    const cuuint64_t es_b = fmt == 0 ? 4 : 2;
    cuuint64_t dims[3] = {(cuuint64_t)rp, (cuuint64_t)rows64, (cuuint64_t)kNumOffsets};
    cuuint64_t strides[2] = {(cuuint64_t)rp * es_b, (cuuint64_t)rows64 * rp * es_b};
    const int kch = kchunk_of(fmt);
    cuuint32_t box[3] = {(cuuint32_t)kch, (cuuint32_t)nb, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(tm, tm_type(fmt), 3, (void *)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          kch * es_b == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// tile of a level with H parent cells per axis, for a largest tile of nt
// targets: (8, 4, nt / 32) on the fine levels, the whole class on the coarse
// ones (padded in y to 16 targets on level 2)
static void tile_of(int H, int nt, int &bx, int &by, int &bz)
{
    if (H >= 8) {
        bx = 8;
        by = 4;
        bz = nt / 32;
    } else if (H == 4) {
        bx = by = bz = 4;
    } else {
        // H = 2: 2 x 4 x 2 parent cells (y padded), 16 targets; a z slab is
        // 8 rows, one swizzle atom, so the level's offsets can be grouped
        bx = 2;
        by = 4;
        bz = 2;
    }
}

int m2l_tile_choices(int precision, int *nt)
{
    if (precision == BBFMM_PREC_FP16X3 || precision == BBFMM_PREC_BF16X3) {
        nt[0] = kTile16;
        nt[1] = kTile16 == 256 ? 128 : 256;
        return 2;
    }
    nt[0] = 128; // TF32: 128-byte rows leave room for 128 targets only
    return 1;
}

void m2l_active_tiles(int D, int nt, const std::vector<uint8_t> &leaf_occ, std::vector<int4> &tiles, int *count)
{
    tiles.clear();
    for (int l = 0; l <= kMaxDepth; ++l)
        count[l] = 0;
    if (D < 2)
        return;
    // occupancy of the boxes of every level, from the leaves (Morton order)
    std::vector<std::vector<uint8_t>> occ(D + 1);
    occ[D] = leaf_occ;
    for (int l = D - 1; l >= 2; --l) {
        occ[l].assign((size_t)1 << (3 * l), 0);
        for (size_t b = 0; b < occ[l + 1].size(); ++b)
            if (occ[l + 1][b])
                occ[l][b >> 3] = 1;
    }
    for (int l = D; l >= 2; --l) { // finest first, the order of the launch
        const int H = 1 << (l - 1);
        int bx, by, bz;
        tile_of(H, nt, bx, by, bz);
        const int size = 1 << l;
        for (int ot = 0; ot < 8; ++ot)
            for (int tz = 0; tz * bz < H; ++tz)
                for (int ty = 0; ty * by < H; ++ty)
                    for (int tx = 0; tx * bx < H; ++tx) {
                        bool any = false;
                        for (int Z = tz * bz; Z < std::min(H, (tz + 1) * bz) && !any; ++Z)
                            for (int Y = ty * by; Y < std::min(H, (ty + 1) * by) && !any; ++Y)
                                for (int X = tx * bx; X < std::min(H, (tx + 1) * bx) && !any; ++X) {
                                    const int x = 2 * X + (ot & 1), y = 2 * Y + ((ot >> 1) & 1),
                                              z = 2 * Z + (ot >> 2);
                                    if (x < size && y < size && z < size &&
                                        occ[l][morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)])
                                        any = true;
                                }
                        if (any) {
                            tiles.push_back(make_int4(tx, ty, tz, ot));
                            count[l]++;
                        }
                    }
    }
}

// slices of F~ per level: 2 when the (active) tiles outnumber the SMs (every
// CTA's range is then at least one tile long, so a tile meets at most one
// range boundary), else 4 (ranges of at least 63 offsets)
// grouped entries on a level: 16-bit forms, a slab of whole 8-row swizzle
// atoms, and sources of bz + 2 slabs within the stage's source buffer
static bool level_grouped(int H, int nt, int fmt)
{
    int bx, by, bz;
    tile_of(H, nt, bx, by, bz);
    return fmt != 0 && kGroupEntries && (bx * by) % 8 == 0 && bx * by * bz + 2 * bx * by <= nt + 64;
}

// slices of F~ per level: enough that, with equal ranges of (tile, entry)
// pairs over the SMs, a tile meets at most G - 1 range boundaries
int m2l_groups_for(int D, int nrhs, int precision, int nt, int r, const int *ntiles, const std::vector<int> &rl)
{
    if (precision == BBFMM_PREC_FP32 || D < 2 || r > 256)
        return 1;
    if (tc_init() != cudaSuccess)
        return 1;
    const int fmt = precision == BBFMM_PREC_FP16X3 ? 1 : precision == BBFMM_PREC_BF16X3 ? 2 : 0;
    int64_t pairs = 0;
    int emax = 1;
    for (int l = 2; l <= D; ++l) {
        const int E = level_grouped(1 << (l - 1), nt, fmt) ? kEntries16 : kOffsetsPerClass;
        const int rk = rl.empty() ? r : rl[rl.size() == 1 ? 0 : l - 2];
        pairs += (int64_t)ntiles[l] * nrhs * (rk > 128 ? 2 : 1) * E;
        emax = std::max(emax, E);
    }
    const int64_t per_cta = std::max<int64_t>(1, (pairs + g_num_sms - 1) / g_num_sms);
    const int64_t need = 1 + (emax + per_cta - 1) / per_cta;
    return (int)std::max<int64_t>(2, std::min<int64_t>(8, need));
}

// bytes of one pipeline stage: the operator tiles (kMaxOps of them with
// grouped entries) and the sources, high and low parts for three passes
static uint32_t tc_stage_bytes(int fmt, bool three, int nt)
{
    const int rowb = kchunk_of(fmt) * (fmt == 0 ? 4 : 2);
    const bool group = fmt != 0 && kGroupEntries;
    const uint32_t a = 128u * rowb, b = (uint32_t)(nt + (group ? 64 : 0)) * rowb;
    return (three ? 2u : 1u) * ((group ? kMaxOps : 1u) * a + b);
}

static constexpr size_t kTcSmemBudget = 220 * 1024;

int m2l_max_stages(int precision, int nt)
{
    const int fmt = precision == BBFMM_PREC_FP16X3 ? 1 : precision == BBFMM_PREC_BF16X3 ? 2 : 0;
    const int n = (int)((kTcSmemBudget - 1024 - 512) / tc_stage_bytes(fmt, precision != BBFMM_PREC_TF32, nt));
    return n > kMaxStages ? kMaxStages : n;
}

template <int NPROD, int NACC, bool CF, int CH, int FMT>
static cudaError_t launch_tc(const TcLaunch &P, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<NPROD, NACC, CF, CH, FMT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_m2l_tc<NPROD, NACC, CF, CH, FMT><<<grid, P.q3 ? 256 : 64 + 128 * CH, smem, s>>>(P);
    return cudaGetLastError();
}

template <int FMT, int CH>
static cudaError_t launch_three(const TcLaunch &L, int nacc, bool cf, int grid, size_t smem, cudaStream_t s)
{
    if (nacc == 2)
        return launch_tc<3, 2, true, CH, FMT>(L, grid, smem, s);
    return cf ? launch_tc<3, 1, true, CH, FMT>(L, grid, smem, s) : launch_tc<3, 1, false, CH, FMT>(L, grid, smem, s);
}

cudaError_t launch_m2l_all(bbfmm_plan_impl *P, int nrhs, cudaStream_t s)
{
    if (P->nodeset == BBFMM_INTERP_UNIFORM)
        return launch_m2l_fft(P, nrhs, s); // equally spaced nodes: Fourier-domain M2L
    const DevOps &O = *P->ops;
    auto scale_of = [&](int l) {
        // homogeneous kernels: operators made for the leaf box, scaled by (h_l / h_D)^m
        return O.host->hom_degree != 0 ? (float)pow(2.0, (double)O.host->hom_degree * (P->D - l)) : 1.0f;
    };
    // the M side of one MMA is 128 operator rows; a level whose rank is above
    // 128 runs each tile as two row halves.  Ranks above 256 (high p with a
    // small svd_eps) run on the FP32 CUDA-core form (with one offset group,
    // see m2l_groups_for)
    if (P->precision == BBFMM_PREC_FP32 || O.r > 256) {
        for (int l = 2; l <= P->D; ++l) {
            const int k = O.nlev == 1 ? 0 : l - 2;
            cudaError_t e = launch_m2l_fp32(P->lev[l].Mt, O.C[k], P->lev[l].Ft, l, O.r, O.rp, O.rows64, nrhs,
                                            P->max_nrhs, scale_of(l), s);
            if (e != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = tc_init();
    if (e != cudaSuccess)
        return e;
    // operand format: 0 = TF32 (1 or 3 passes), 1 = FP16 x3, 2 = BF16 x3
    const int fmt = P->precision == BBFMM_PREC_FP16X3 ? 1 : P->precision == BBFMM_PREC_BF16X3 ? 2 : 0;
    const bool three = P->precision != BBFMM_PREC_TF32;
    const int kch = kchunk_of(fmt);
    const int elem = fmt == 0 ? 4 : 2, rowb = kch * elem, kstep = fmt == 0 ? 8 : 16;
    const int nt = P->m2l_nt; // targets per tile: the plan's tuning
    if (nt != 128 && !(nt == 256 && fmt != 0))
        return cudaErrorInvalidValue;
    if (O.rp % 16 != 0 || P->D - 1 > kMaxTcLevels || (int)O.rl.size() != O.nlev)
        return cudaErrorInvalidValue;
    // operator rows loaded per tile of each operator level (the M side is
    // always 128): the rank rounded to 16, or 128 per half above 128
    int nbk[kMaxTcLevels];
    for (int k = 0; k < O.nlev; ++k) {
        if (O.rl[k] < 1 || O.rl[k] > O.r)
            return cudaErrorInvalidValue;
        nbk[k] = O.rl[k] > 128 ? 128 : (O.rl[k] + 15) / 16 * 16;
    }
    if (fmt != 0 && (int)O.C16hi[fmt - 1].size() != O.nlev)
        return cudaErrorInvalidValue;
    TcLaunch L;
    memset(&L, 0, sizeof(L));
    L.status = P->status;
    L.rp = O.rp;
    L.nrhs = nrhs;
    L.R = P->max_nrhs;

    // grouped entries (16-bit forms): a stage holds up to kMaxOps operator
    // tiles and sources of bz + 2 slabs (2 slabs = 64 rows on the fine levels)
    const bool group = fmt != 0 && kGroupEntries;
    L.maxops = group ? kMaxOps : 1;
    L.a_bytes = 128 * rowb; // C tile: 128 rows in shared memory, nbk of them loaded
    L.b_bytes = (uint32_t)(nt + (group ? 64 : 0)) * rowb; // sources
    L.stage_bytes = (three ? 2 : 1) * ((uint32_t)L.maxops * L.a_bytes + L.b_bytes);
    if (L.stage_bytes != tc_stage_bytes(fmt, three, nt))
        return cudaErrorInvalidValue;
    L.ascale = P->a16_scale;
    // TMEM: one accumulator of nt columns per partial buffer; two per buffer
    // (hi*hi and corrections apart) when two double-buffered pairs still fit
    L.bcols = nt;
    const int nacc = three && P->split_acc && 4 * nt <= 512 ? 2 : 1;
    L.nbuf = 512 / (nacc * nt) > kMaxBuf ? kMaxBuf : 512 / (nacc * nt);
    L.tcols = 32;
    while (L.tcols < L.nbuf * nacc * nt)
        L.tcols *= 2;
    // pipeline stages: as many as fit, or fewer when the plan's tuning asks
    int nstage = m2l_max_stages(P->precision, nt);
    if (P->m2l_stages > 0 && P->m2l_stages < nstage)
        nstage = P->m2l_stages;
    if (nstage < 2)
        return cudaErrorInvalidValue;
    L.nstage = nstage;
    const size_t smem = 1024 + (size_t)nstage * L.stage_bytes + 512; // + barriers and TMEM slot
    // levels, finest first
    int tiles = 0, emax = 0;
    int64_t pairs = 0;
    L.nlev = 0;
    for (int l = P->D; l >= 2; --l) {
        TcLevel &lv = L.lev[L.nlev];
        const int H = 1 << (l - 1);
        lv.Ft = P->lev[l].Ft;
        lv.slice = ((int64_t)1 << (3 * l)) * P->max_nrhs * O.rp;
        lv.H = H;
        tile_of(H, nt, lv.bx, lv.by, lv.bz);
        lv.lbx = __builtin_ctz((unsigned)lv.bx);
        lv.lby = __builtin_ctz((unsigned)lv.by);
        lv.n = lv.bx * lv.by * lv.bz;
        lv.tl = P->m2l_tiles + P->m2l_tile_off[l];
        lv.nact = P->m2l_ntiles[l];
        lv.opl = O.nlev == 1 ? 0 : l - 2;
        lv.r = O.rl[lv.opl];
        lv.nh = lv.r > 128 ? 2 : 1;
        lv.nk = (lv.r + kch - 1) / kch;
        lv.ktail = (lv.r - kch * (lv.nk - 1) + kstep - 1) / kstep;
        lv.a_load = (uint32_t)nbk[lv.opl] * rowb;
        lv.ntiles = lv.nact * nrhs * lv.nh;
        lv.tile_base = tiles;
        lv.l = l;
        lv.scale = scale_of(l);
        lv.idesc = fmt == 0 ? idesc_tf32(128, lv.n) : idesc_f16(128, lv.n, fmt == 2 ? 1 : 0);
        lv.b_load = (uint32_t)lv.n * rowb;
        // a slab shift must keep the swizzle phase: whole 8-row atoms
        const uint32_t slab_bytes = (uint32_t)(lv.bx * lv.by) * rowb;
        lv.grp = group && level_grouped(H, nt, fmt) ? 1 : 0;
        lv.E = lv.grp ? kEntries16 : kOffsetsPerClass;
        lv.slab16 = slab_bytes >> 4;
        lv.b_load2 = (uint32_t)(lv.n + 2 * lv.bx * lv.by) * rowb;
        lv.pair_base = pairs;
        pairs += (int64_t)lv.ntiles * lv.E;
        emax = std::max(emax, lv.E);
        tiles += lv.ntiles;
        const void *A, *Alo;
        if (fmt != 0) {
            A = P->lev[l].Mt16_hi;
            Alo = P->lev[l].Mt16_lo;
        } else {
            A = three ? (const void *)P->lev[l].Mt_hi : (const void *)P->lev[l].Mt;
            Alo = three ? (const void *)P->lev[l].Mt_lo : A;
        }
        e = encode_src(&L.src[L.nlev], A, H, P->max_nrhs, O.rp, fmt, lv.bx, lv.by, lv.bz);
        if (e == cudaSuccess)
            e = encode_src(&L.srclo[L.nlev], Alo, H, P->max_nrhs, O.rp, fmt, lv.bx, lv.by, lv.bz);
        if (e == cudaSuccess && lv.grp)
            e = encode_src(&L.src2[L.nlev], A, H, P->max_nrhs, O.rp, fmt, lv.bx, lv.by, lv.bz + 2);
        if (e == cudaSuccess && lv.grp)
            e = encode_src(&L.srclo2[L.nlev], Alo, H, P->max_nrhs, O.rp, fmt, lv.bx, lv.by, lv.bz + 2);
        if (e != cudaSuccess)
            return e;
        L.nlev++;
    }
    // equal ranges of (tile, entry) pairs; a range is long enough that no
    // tile meets more than G - 1 range boundaries (G = slices allocated)
    const int G = P->m2l_groups;
    L.ntiles = tiles;
    L.total = pairs;
    const int64_t min_len = G >= 2 ? (emax + G - 2) / (G - 1) : L.total;
    L.per_cta = (L.total + g_num_sms - 1) / g_num_sms;
    if (L.per_cta < min_len)
        L.per_cta = min_len;
    for (int k = 0; k < O.nlev; ++k) {
        const void *B, *Blo;
        if (fmt != 0) {
            B = O.C16hi[fmt - 1][k];
            Blo = O.C16lo[fmt - 1][k];
            L.bscale_inv[k] = 1.0f / O.c16_scale[fmt - 1][k];
        } else {
            B = three ? (const void *)O.Chi[k] : (const void *)O.C[k];
            Blo = three ? (const void *)O.Clo[k] : B;
            L.bscale_inv[k] = 1.0f;
        }
        e = encode_op(&L.op[k], B, O.rp, O.rows64, nbk[k], fmt);
        if (e == cudaSuccess)
            e = encode_op(&L.oplo[k], Blo, O.rp, O.rows64, nbk[k], fmt);
        if (e != cudaSuccess)
            return e;
    }
    const int grid = (int)((L.total + L.per_cta - 1) / L.per_cta);
    // slices 1..G-1 of tiles that no range boundary cuts are never written
    for (int l = 2; l <= P->D && G > 1; ++l) {
        const int64_t sl = ((int64_t)1 << (3 * l)) * P->max_nrhs * O.rp;
        e = cudaMemsetAsync(P->lev[l].Ft + sl, 0, sizeof(float) * sl * (G - 1), s);
        if (e != cudaSuccess)
            return e;
    }
    // three epilogue quadrants when no level's rank needs the fourth (256-target
    // tiles of the 16-bit forms): measured 0.817 -> 0.813 ms per matvec at
    // depth 5 and 3.367 -> 3.337 ms at depth 6 (1M points, 1/r, p = 5, r = 89)
    L.q3 = fmt != 0 && nt == 256 ? 1 : 0;
    for (int k = 0; k < O.nlev; ++k)
        if (O.rl[k] > 96)
            L.q3 = 0;
    const bool cf = P->split_acc;
    if (!three)
        return launch_tc<1, 1, false, 1, 0>(L, grid, smem, s);
    if (fmt == 0)
        return launch_three<0, 1>(L, nacc, cf, grid, smem, s);
    if (nt == 256)
        return fmt == 1 ? launch_three<1, 2>(L, nacc, cf, grid, smem, s) : launch_three<2, 2>(L, nacc, cf, grid, smem, s);
    return fmt == 1 ? launch_three<1, 1>(L, nacc, cf, grid, smem, s) : launch_three<2, 1>(L, nacc, cf, grid, smem, s);
}

} // namespace bbfmm
