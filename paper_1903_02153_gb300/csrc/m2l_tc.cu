// m2l_tc.cu -- far-field stage (Sec. 2.2 item 2) on the 5th-generation tensor
// cores:  F~^alpha = scale_l * sum_{beta in I(alpha)} C^(t) M~^beta  with the
// compressed operators C^(t) = U^T K^(t) V (Sec. 2.5 "Fast M2L translation").
//
// The stage is a dense contraction: for the 128 targets of a tile (an 8x4x4
// block of parent cells of one octant class) and each of the 189 offsets of
// the class, D[128 x r] += A_t[128 x r] * B_t[r x r]^T, where A_t gathers the
// source vectors M~ of the 128 targets (one TMA box of the parity-split M~
// array: consecutive parent cells of one source octant; out-of-range cells
// read as zero) and B_t = C^(t).  K is walked in chunks of 32 elements (a
// 128-byte row) for TF32, of kChunk16 elements for FP16 / BF16.
//
// One persistent launch covers every level 2..D.  A work item is (level,
// tile, group of offsets): the 189 offsets of a tile are split into G groups
// so that all SMs stay busy; each item writes its partial sum to slice g of
// the level's F~ buffer and the decompress GEMM adds the G slices in a fixed
// order (deterministic).
//
//   warp 0         TMA producer: one lane arms a stage barrier and issues the
//                  box loads of A (and its low part) and B (and its low part)
//   warp 1         MMA issuer: one lane issues tcgen05.mma kind::tf32, M = 128,
//                  N = r rounded to 16, K = 8 per instruction
//   warps 2..      epilogue: after every offset it drains the offset's partial
//                  accumulator from TMEM into FP32 registers; at the end of an
//                  item it scales and stores the sum.  As many partial
//                  buffers as fit in the 512 TMEM columns (5 for r <= 96) let
//                  the MMAs run several offsets ahead of the drains, so the
//                  round trip commit -> drain -> release stays off the tensor
//                  pipe's critical path
//
// Precision: kind::tf32 reads 10 explicit mantissa bits.  The 3-pass mode
// splits each operand into hi = tf32(x) and lo = tf32(x - hi) and forms
// hi*hi + hi*lo + lo*hi (the split-TF32 scheme of Ootomo & Yokota, 2022).
// The tensor core's own accumulation truncates; long runs of it (189 offsets
// x r/8 steps into one accumulator) lost ~1e-5 relative on the 1M-point
// workload, so, as that scheme prescribes, a TMEM accumulator only ever holds
// one offset and the sum over offsets is taken in FP32 registers with
// round-to-nearest.  Within an offset, with CF, each K chunk's correction
// products (hi*lo, lo*hi: 2^-11 of hi*hi) are issued before its hi*hi
// products, so they are summed while the accumulator is still small and
// only the hi*hi additions truncate at the scale of the result.
//
// Every mbarrier wait is bounded (about 2^31 cycles): on expiry the kernel
// sets the plan's status word, stops issuing work, waits (bounded) for its own
// copies and MMAs in flight, frees its TMEM and returns.
#include <cudaTypedefs.h>
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

// K elements per pipeline stage for the 16-bit forms: 32 (64-byte rows,
// 64-byte swizzle) or 64 (128-byte rows, 128-byte swizzle); TF32 always uses
// 32 (128-byte rows)
#ifndef BBFMM_TC_CHUNK16
#define BBFMM_TC_CHUNK16 64
#endif
constexpr int kChunk16 = BBFMM_TC_CHUNK16;
#ifndef BBFMM_TC_MAX_STAGES
#define BBFMM_TC_MAX_STAGES 8
#endif
constexpr int kMaxStages = BBFMM_TC_MAX_STAGES; // pipeline stages (shared memory permitting)
#ifndef BBFMM_TC_ACC_PER_BUF
#define BBFMM_TC_ACC_PER_BUF 2
#endif
constexpr int kAccPerBuf = BBFMM_TC_ACC_PER_BUF; // accumulators per offset (1 or 2)
static_assert(kChunk16 == 32 || kChunk16 == 64, "16-bit K chunk is 32 or 64 elements");

// ---------------------------------------------------------------------------
__constant__ int4 c_tab_tc[8][kOffsetsPerClass];

constexpr int kMaxTcLevels = 8;

struct TcLevel {
    float *Ft;     // partial slice g at Ft + g * slice
    int64_t slice; // floats per slice
    int H, tiles_x, tiles_y, tiles_z, ntiles, item_base, opl, l;
    float scale;
};

struct TcLaunch {
    CUtensorMap a[kMaxTcLevels], alo[kMaxTcLevels]; // M~ (hi, lo) of each level
    CUtensorMap b[kMaxTcLevels], blo[kMaxTcLevels]; // C (hi, lo) of each operator level
    TcLevel lev[kMaxTcLevels];
    float bscale_inv[kMaxTcLevels]; // 1 / (scale of the 16-bit operators), per operator level
    const float *ascale;            // 16-bit forms: scale of M~ per tree level (device)
    int nlev, nitems, groups, per_group;
    int *status;
    int r, rp, nb, ncols, nrhs, R, nk, nstage; // R: right-hand-side stride of M~ / F~ rows
    int nbuf, nacc, bcols, tcols; // TMEM partial buffers, accumulators per buffer, columns
                                  // per accumulator, columns allocated
    uint32_t stage_bytes, a_bytes, b_bytes;
};

struct Item {
    int L, tx, ty, tz, ot, c, g, e0, e1;
};

__device__ __forceinline__ Item decode_item(const TcLaunch &P, int item)
{
    Item it;
    int L = 0;
    while (L + 1 < P.nlev && item >= P.lev[L + 1].item_base)
        ++L;
    it.L = L;
    int local = item - P.lev[L].item_base;
    it.g = local % P.groups;
    int t = local / P.groups;
    const TcLevel &lv = P.lev[L];
    it.tx = t % lv.tiles_x;
    t /= lv.tiles_x;
    it.ty = t % lv.tiles_y;
    t /= lv.tiles_y;
    it.tz = t % lv.tiles_z;
    t /= lv.tiles_z;
    it.ot = t & 7;
    it.c = t >> 3;
    it.e0 = it.g * P.per_group;
    it.e1 = min(kOffsetsPerClass, it.e0 + P.per_group);
    return it;
}

// FMT: operand format, 0 = TF32 (kind::tf32, 32 elements per 128-byte row,
// K = 8 per MMA), 1 = FP16, 2 = BF16 (kind::f16, 64 elements per row, K = 16)
template <int NPROD, bool CF, int NACC, int CH, int FMT>
__global__ void __launch_bounds__(64 + 128 * CH, 1) k_m2l_tc(const __grid_constant__ TcLaunch P)
{
    // K is walked in chunks of 32 elements per stage: one 128-byte swizzled
    // row for TF32, one 64-byte swizzled row for the 16-bit forms (the smaller
    // stage keeps more offsets in flight for the same shared memory)
    constexpr int CHUNK = FMT == 0 ? 32 : kChunk16;
    constexpr bool SW64 = FMT != 0 && kChunk16 == 32; // 64-byte rows
    constexpr int KSTEP = FMT == 0 ? 8 : 16;         // K elements per MMA (32 bytes)
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = smem_raw + (base - raw);
    const int S = P.nstage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (size_t)S * P.stage_bytes);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
    constexpr int kMaxBuf = 8;
    const int NB = P.nbuf;
    const uint32_t pfull0 = empty0 + 8 * S, pempty0 = pfull0 + 8 * kMaxBuf, done_bar = pempty0 + 8 * kMaxBuf;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 2 * kMaxBuf + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t tcols = (uint32_t)P.tcols;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(pfull0 + 8 * b, 1);
            mbar_init(pempty0 + 8 * b, 4 * CH);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ producer
        int last_round[16];
        for (int s = 0; s < 16; ++s)
            last_round[s] = -1;
        int it = 0;
        for (int item = blockIdx.x; item < P.nitems && !*abort_flag; item += gridDim.x) {
            const Item w = decode_item(P, item);
            const TcLevel &lv = P.lev[w.L];
            const int X0 = 8 * w.tx, Y0 = 4 * w.ty, Z0 = 4 * w.tz;
            for (int e = w.e0; e < w.e1 && !*abort_flag; ++e) {
                const int4 en = c_tab_tc[w.ot][e];
                const int ux = (en.z & 3) - 1, uy = ((en.z >> 2) & 3) - 1, uz = ((en.z >> 4) & 3) - 1;
                const int zq = en.y * (lv.H + 2) + 1 + Z0 + uz;
                for (int kc = 0; kc < P.nk; ++kc, ++it) {
                    const int s = it % S, round = it / S;
                    if (!mbar_wait(empty0 + 8 * s, (round & 1) ^ 1, abort_flag))
                        break;
                    const uint32_t sa = base + (uint32_t)s * P.stage_bytes;
                    const uint32_t fb = full0 + 8 * s;
                    mbar_arrive_expect_tx(fb, P.stage_bytes);
                    last_round[s] = round;
                    tma_load_5d(sa, &P.a[w.L], fb, CHUNK * kc, w.c, X0 + ux, Y0 + uy, zq);
                    uint32_t off = P.a_bytes;
                    if (NPROD == 3) {
                        tma_load_5d(sa + off, &P.alo[w.L], fb, CHUNK * kc, w.c, X0 + ux, Y0 + uy, zq);
                        off += P.a_bytes;
                    }
                    tma_load_3d(sa + off, &P.b[lv.opl], fb, CHUNK * kc, 0, en.x);
                    off += P.b_bytes;
                    if (NPROD == 3)
                        tma_load_3d(sa + off, &P.blo[lv.opl], fb, CHUNK * kc, 0, en.x);
                }
            }
        }
        // teardown: every armed stage must have landed before the CTA exits
        for (int s = 0; s < S && s < 16; ++s)
            if (last_round[s] >= 0) {
                long long t0 = clock64();
                while (!mbar_test(full0 + 8 * s, last_round[s] & 1) && clock64() - t0 < kWaitCycles) {
                }
            }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        // One thread issues every MMA of the CTA, so this loop is kept short:
        // ring positions are counters (no division), the operand descriptors
        // of a stage are the stage-0 descriptors plus a constant, the K steps
        // of a chunk are unrolled.
        const uint32_t idesc = FMT == 0 ? idesc_tf32(128, P.nb) : idesc_f16(128, P.nb, FMT == 2 ? 1 : 0);
        const uint32_t b_off = NPROD == 3 ? 2 * P.a_bytes : P.a_bytes;
        const uint64_t d0 = SW64 ? sw64_desc(base) : sw128_desc(base);
        const uint32_t d_al = P.a_bytes >> 4, d_bh = b_off >> 4, d_bl = (b_off + P.b_bytes) >> 4;
        const uint32_t d_st = P.stage_bytes >> 4;
        constexpr int KMAX = CHUNK / KSTEP;
        const int ktail = (P.r - CHUNK * (P.nk - 1) + KSTEP - 1) / KSTEP; // K steps of the last chunk
        int s = 0, sph = 0, pb = 0, pph = 0; // stage ring and partial-buffer ring (position, phase)
        bool ok = true;
        for (int item = blockIdx.x; item < P.nitems && ok && !*abort_flag; item += gridDim.x) {
            const Item w = decode_item(P, item);
            for (int e = w.e0; e < w.e1 && ok; ++e) {
                if (!mbar_wait(pempty0 + 8 * pb, pph ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // NACC = 2: hi*hi into the first accumulator, the corrections
                // into the second; NACC = 1: one accumulator, corrections of
                // each chunk first (CF) or after its hi*hi
                const uint32_t dh = tmem_base + (uint32_t)(pb * NACC * P.bcols);
                const uint32_t dc = NACC == 2 ? dh + (uint32_t)P.bcols : dh;
                uint32_t acc_h = 0, acc_c = 0;
                for (int kc = 0; kc < P.nk; ++kc) {
                    if (!mbar_wait(full0 + 8 * s, sph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ah = d0 + (uint64_t)(s * d_st);
                    const uint64_t al = ah + d_al, bh = ah + d_bh, bl = ah + d_bl;
                    const int ks = kc + 1 < P.nk ? KMAX : ktail;
                    auto issue = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
                        if (FMT == 0)
                            mma_tf32(d, a, b, idesc, acc);
                        else
                            mma_f16(d, a, b, idesc, acc);
                    };
                    if (NPROD == 3 && (NACC == 2 || CF)) {
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
#pragma unroll
                    for (int k = 0; k < KMAX; ++k)
                        if (k < ks) {
                            const uint64_t dk = (uint64_t)(2 * k);
                            issue(dh, ah + dk, bh + dk, acc_h);
                            acc_h = 1u;
                        }
                    if (NPROD == 3 && NACC == 1 && !CF) {
#pragma unroll
                        for (int k = 0; k < KMAX; ++k)
                            if (k < ks) {
                                const uint64_t dk = (uint64_t)(2 * k);
                                issue(dh, ah + dk, bl + dk, 1u);
                                issue(dh, al + dk, bh + dk, 1u);
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
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const int half = ew >> 2; // column block [128 half, 128 half + 128)
        const int row = 32 * q + lane;
        const int bx = row & 7, by = (row >> 3) & 3, bz = row >> 5;
        const uint32_t tlane = tmem_base + ((uint32_t)(32 * q) << 16);
        int pb = 0, pph = 0; // partial-buffer ring (position, phase)
        bool ok = true;
        // add the columns [128 half, 128 half + nb) of TMEM buffer tb into acc,
        // 32 (or, for the last piece, 16) columns per load
        auto drain = [&](uint32_t tb, float *acc) {
#pragma unroll
            for (int c32 = 0; c32 < 4; ++c32) {
                const int col = 128 * half + 32 * c32;
                if (col + 32 <= P.nb) {
                    float v[32];
                    tmem_ld32(tb + (uint32_t)col, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        acc[32 * c32 + j] += v[j];
                } else if (col < P.nb) {
                    float v[16];
                    tmem_ld16(tb + (uint32_t)col, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[32 * c32 + j] += v[j];
                }
            }
        };
        for (int item = blockIdx.x; item < P.nitems && ok; item += gridDim.x) {
            const Item w = decode_item(P, item);
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
                drain(tlane + (uint32_t)(pb * NACC * P.bcols), acc);
                if (NACC == 2)
                    drain(tlane + (uint32_t)((pb * NACC + 1) * P.bcols), acc);
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
            const TcLevel &lv = P.lev[w.L];
            const int X = 8 * w.tx + bx, Y = 4 * w.ty + by, Z = 4 * w.tz + bz;
            if (X < lv.H && Y < lv.H && Z < lv.H) {
                float *out = lv.Ft + (int64_t)w.g * lv.slice +
                             ((((int64_t)w.ot * lv.H + Z) * lv.H + Y) * lv.H + X) * (int64_t)P.R * P.rp +
                             (int64_t)w.c * P.rp;
                // level scale; 16-bit forms also undo the power-of-two operand scales
                float f = lv.scale;
                if (FMT != 0)
                    f *= P.bscale_inv[lv.opl] / __ldg(P.ascale + lv.l);
#pragma unroll
                for (int j = 0; j < 128; j += 4) {
                    const int col = 128 * half + j;
                    if (col < P.r)
                        *reinterpret_cast<float4 *>(out + col) =
                            make_float4(f * acc[j], f * acc[j + 1], f * acc[j + 2], f * acc[j + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_flag && threadIdx.x == 0)
        atomicOr(P.status, kStatusTimeout);
    if (warp == 1) {
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
        int4 tab[8][kOffsetsPerClass];
        if (!fill_m2l_table(tab))
            return cudaErrorInvalidValue;
        cudaError_t e = cudaMemcpyToSymbol(c_tab_tc, tab, sizeof(tab));
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


// M~ (parity split, padded in Z): dims (rp, R, H, H, 8 (H + 2)); box (one
// K chunk, 1, 8, 4, 4); elem = 4 (FP32 / TF32: 32 per 128-byte row, 128-byte
// swizzle) or 2 (FP16 / BF16: kChunk16 per row, 64- or 128-byte swizzle)
static cudaError_t encode_a(CUtensorMap *tm, const void *ptr, int H, int R, int rp, int fmt)
{
    const cuuint64_t es_b = fmt == 0 ? 4 : 2;
    cuuint64_t dims[5] = {(cuuint64_t)rp, (cuuint64_t)R, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)8 * (H + 2)};
    cuuint64_t strides[4] = {(cuuint64_t)rp * es_b, (cuuint64_t)R * rp * es_b, (cuuint64_t)H * R * rp * es_b,
                             (cuuint64_t)H * H * R * rp * es_b};
    const bool sw64 = fmt != 0 && kChunk16 == 32;
    cuuint32_t box[5] = {(cuuint32_t)(fmt == 0 ? 32 : kChunk16), 1, 8, 4, 4};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUtensorMapDataType dt = fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUresult r = g_encode(tm, dt, 5, (void *)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// C (operators): dims (rp, rows64, 316); box (one K chunk, nb, 1), rows and
// swizzle as for M~
static cudaError_t encode_b(CUtensorMap *tm, const void *ptr, int rp, int rows64, int nb, int fmt)
{
    const cuuint64_t es_b = fmt == 0 ? 4 : 2;
    cuuint64_t dims[3] = {(cuuint64_t)rp, (cuuint64_t)rows64, (cuuint64_t)kNumOffsets};
    cuuint64_t strides[2] = {(cuuint64_t)rp * es_b, (cuuint64_t)rows64 * rp * es_b};
    const bool sw64 = fmt != 0 && kChunk16 == 32;
    cuuint32_t box[3] = {(cuuint32_t)(fmt == 0 ? 32 : kChunk16), (cuuint32_t)nb, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUtensorMapDataType dt = fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUresult r = g_encode(tm, dt, 3, (void *)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int tiles_of_level(int l, int nrhs)
{
    int H = 1 << (l - 1);
    return ((H + 7) / 8) * ((H + 3) / 4) * ((H + 3) / 4) * 8 * nrhs;
}

int m2l_groups_for(int D, int nrhs, int precision)
{
    if (precision == BBFMM_PREC_FP32 || D < 2)
        return 1;
    if (tc_init() != cudaSuccess)
        return 1;
    int64_t T = 0;
    for (int l = 2; l <= D; ++l)
        T += tiles_of_level(l, nrhs);
    // makespan in units of one offset: waves x offsets per item (+2 for the
    // fill / drain / store of an item)
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int G = 1; G <= 8; ++G) {
        int64_t waves = (T * G + g_num_sms - 1) / g_num_sms;
        int64_t cost = waves * ((kOffsetsPerClass + G - 1) / G + 2);
        if (cost < best_cost) {
            best_cost = cost;
            best = G;
        }
    }
    return best;
}

template <int NPROD, bool CF, int NACC, int CH, int FMT>
static cudaError_t launch_tc(const TcLaunch &P, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<NPROD, CF, NACC, CH, FMT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_m2l_tc<NPROD, CF, NACC, CH, FMT><<<grid, 64 + 128 * CH, smem, s>>>(P);
    return cudaGetLastError();
}

template <int FMT>
static cudaError_t launch_three(const TcLaunch &L, bool cf, int CH, int grid, size_t smem, cudaStream_t s)
{
    if (L.nacc == 2) // two accumulators fit only when nb <= 128, so CH = 1
        return launch_tc<3, true, 2, 1, FMT>(L, grid, smem, s);
    if (CH == 1)
        return cf ? launch_tc<3, true, 1, 1, FMT>(L, grid, smem, s) : launch_tc<3, false, 1, 1, FMT>(L, grid, smem, s);
    return cf ? launch_tc<3, true, 1, 2, FMT>(L, grid, smem, s) : launch_tc<3, false, 1, 2, FMT>(L, grid, smem, s);
}

cudaError_t launch_m2l_all(bbfmm_plan_impl *P, int nrhs, cudaStream_t s)
{
    const DevOps &O = *P->ops;
    auto scale_of = [&](int l) {
        // homogeneous kernels: operators made for the leaf box, scaled by (h_l / h_D)^m
        return O.host->hom_degree != 0 ? (float)pow(2.0, (double)O.host->hom_degree * (P->D - l)) : 1.0f;
    };
    if (P->precision == BBFMM_PREC_FP32) {
        for (int l = 2; l <= P->D; ++l) {
            const int k = O.nlev == 1 ? 0 : l - 2;
            cudaError_t e =
                launch_m2l_fp32(P->lev[l].Mt, O.C[k], P->lev[l].Ft, l, O.r, O.rp, O.rows64, nrhs, P->max_nrhs, scale_of(l), s);
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
    const int elem = fmt == 0 ? 4 : 2, chunk = fmt == 0 ? 32 : kChunk16, rowb = chunk * elem;
    const int nb = (O.r + 15) / 16 * 16;
    if (nb > 256 || O.rp % 16 != 0 || P->D - 1 > kMaxTcLevels)
        return cudaErrorInvalidValue;
    if (fmt != 0 && (int)O.C16hi[fmt - 1].size() != O.nlev)
        return cudaErrorInvalidValue;
    TcLaunch L;
    memset(&L, 0, sizeof(L));
    L.status = P->status;
    L.r = O.r;
    L.rp = O.rp;
    L.nb = nb;
    L.ncols = nb <= 32 ? 32 : nb <= 64 ? 64 : nb <= 128 ? 128 : 256;
    // accumulators of nb columns rounded to 32.  Three-product forms keep
    // hi*hi and the corrections in two accumulators per offset when two
    // double-buffered pairs fit in the 512 TMEM columns (nb <= 128), else one
    // accumulator with each chunk's corrections issued first.  As many partial
    // buffers as fit (at most 8); the allocation is a power of two.
    L.bcols = (nb + 31) / 32 * 32;
    L.nacc = three && P->split_acc && kAccPerBuf == 2 && 4 * L.bcols <= 512 ? 2 : 1;
    L.nbuf = 512 / (L.nacc * L.bcols) > 8 ? 8 : 512 / (L.nacc * L.bcols);
    L.tcols = 32;
    while (L.tcols < L.nbuf * L.nacc * L.bcols)
        L.tcols *= 2;
    L.nrhs = nrhs;
    L.R = P->max_nrhs;
    L.nk = (O.r + chunk - 1) / chunk;
    L.groups = P->m2l_groups;
    L.per_group = (kOffsetsPerClass + L.groups - 1) / L.groups;
    L.a_bytes = 128 * rowb;
    L.b_bytes = (uint32_t)nb * rowb;
    L.stage_bytes = (three ? 2 : 1) * (L.a_bytes + L.b_bytes);
    L.ascale = P->a16_scale;
    const size_t budget = 220 * 1024;
    int nstage = (int)((budget - 1024 - 512) / L.stage_bytes);
    nstage = nstage > kMaxStages ? kMaxStages : nstage;
    if (nstage < 2)
        return cudaErrorInvalidValue;
    L.nstage = nstage;
    const size_t smem = 1024 + (size_t)nstage * L.stage_bytes + 512; // + barriers and TMEM slot
    // levels, finest first
    int items = 0;
    L.nlev = 0;
    for (int l = P->D; l >= 2; --l) {
        TcLevel &lv = L.lev[L.nlev];
        const int H = 1 << (l - 1);
        lv.Ft = P->lev[l].Ft;
        lv.slice = ((int64_t)1 << (3 * l)) * P->max_nrhs * O.rp;
        lv.H = H;
        lv.tiles_x = (H + 7) / 8;
        lv.tiles_y = (H + 3) / 4;
        lv.tiles_z = (H + 3) / 4;
        lv.ntiles = tiles_of_level(l, nrhs);
        lv.item_base = items;
        lv.opl = O.nlev == 1 ? 0 : l - 2;
        lv.l = l;
        lv.scale = scale_of(l);
        items += lv.ntiles * L.groups;
        const void *A, *Alo;
        if (fmt != 0) {
            A = P->lev[l].Mt16_hi;
            Alo = P->lev[l].Mt16_lo;
        } else {
            A = three ? (const void *)P->lev[l].Mt_hi : (const void *)P->lev[l].Mt;
            Alo = three ? (const void *)P->lev[l].Mt_lo : A;
        }
        e = encode_a(&L.a[L.nlev], A, H, P->max_nrhs, O.rp, fmt);
        if (e == cudaSuccess)
            e = encode_a(&L.alo[L.nlev], Alo, H, P->max_nrhs, O.rp, fmt);
        if (e != cudaSuccess)
            return e;
        L.nlev++;
    }
    L.nitems = items;
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
        e = encode_b(&L.b[k], B, O.rp, O.rows64, nb, fmt);
        if (e == cudaSuccess)
            e = encode_b(&L.blo[k], Blo, O.rp, O.rows64, nb, fmt);
        if (e != cudaSuccess)
            return e;
    }
    const int grid = items < g_num_sms ? items : g_num_sms;
    const int CH = nb > 128 ? 2 : 1;
    const bool split = three && P->split_acc; // corrections first within each K chunk
    if (!three)
        return CH == 1 ? launch_tc<1, false, 1, 1, 0>(L, grid, smem, s) : launch_tc<1, false, 1, 2, 0>(L, grid, smem, s);
    if (fmt == 0)
        return launch_three<0>(L, split, CH, grid, smem, s);
    if (fmt == 1)
        return launch_three<1>(L, split, CH, grid, smem, s);
    return launch_three<2>(L, split, CH, grid, smem, s);
}

} // namespace bbfmm
