// box_gemm.cu -- the compression of the leaf multipole coefficients and the
// decompression of the leaf local coefficients (Sec. 2.5 "Fast M2L
// translation", applied to every leaf box by the upward and downward passes,
// Sec. 2.3 items 1 and 3) as GEMMs on the tensor cores.
//
// Compression (MODE 0): rows are (right-hand side c, leaf box), one row of M
// the p^3 coefficients of one box for one column, and the leaf level is
//     M~[row][k] = sum_i M[row][i] V[i][k],   rows = nrhs x 8^D, i < p^3, k < r,
// a tall GEMM with K = p^3 and N = r (p = 5: K = 125, N = 89).  The upward
// pass writes M of the leaves ([R][8^D][p3p], zero past p^3) instead of
// compressing them; this kernel stores M~ at the leaf's row of the
// parity-split layout (with the TF32 split and the level's max |M~| when the
// M2L needs them).
//
// Decompression (MODE 1): rows are the rows of the parity-split F~ (leaf
// cell x R + c), summed over the M2L's offset-group slices as part of K:
//     F[row][i] = sum_g sum_k F~_g[row][k] U[i][k],   K = r, N = p^3,
// written to [rows][p3p] for the downward pass, which adds it to the L2L
// part of each leaf's local coefficients.
//
// Arithmetic: kind::tf32 with FP32 accumulation, 3 products per K step
// (hi*hi + hi*lo + lo*hi, the split-TF32 scheme of Ootomo & Yokota, 2022).
// V^T's hi / lo parts are split once on the host; M's are split in shared
// memory after each TMA load (two warps), so the upward pass writes plain
// FP32.  The tensor core's FP32 accumulation truncates; with N <= 128 each
// K chunk of 32 goes to a fresh TMEM partial (two alternate) and the
// epilogue sums the partials with round-to-nearest FP32 adds, so a long K
// (decompression sums several slices of r) loses no more than one chunk.
//
//   warp 0      TMA producer: V^T (hi, lo; all of K) once, then per tile of
//               128 rows and K chunk of 32 the rows' chunk of M
//   warp 1      TMEM allocation; one lane issues the MMAs (M = 128 rows,
//               N = r rounded to 16, K = 8)
//   warps 2..3  split each landed chunk into hi (in place) and lo
//   warps 4..7  epilogue: thread = TMEM lane = row of the tile
//
// Every mbarrier wait is bounded; on expiry the kernel records it in the
// plan's status word, stops, waits (bounded) for its own copies and MMAs and
// frees its TMEM.
#include <math.h>

#include "bbfmm_internal.h"
#include "tc_ptx.cuh"

namespace bbfmm {

namespace {

constexpr int kGemmRows = 128;  // rows per tile (the MMA's M, TMEM lanes)
constexpr int kGemmK = 32;      // K elements per chunk: one 128-byte swizzled row
constexpr int kGemmStages = 3;  // A chunks in flight
constexpr int kGemmThreads = 256;
constexpr uint32_t kAChunkBytes = kGemmRows * kGemmK * 4; // 16 KB
constexpr int kStatusTimeoutBit = 2;

struct GemmLaunch {
    CUtensorMap a;        // A: [slices x slice_rows][K] FP32, box (32, 128)
    CUtensorMap bhi, blo; // B hi / lo: [N'][K] FP32, box (32, N)
    int ntiles;           // tiles of 128 rows
    int kchunks;          // K chunks of 32 per slice
    int slices;           // A slices summed into one product (decompression: F~'s offset groups)
    int64_t slice_rows;   // rows between slices
    int ldo;              // decompression: output row pitch (floats)
    int N;                // MMA N: r rounded up to 16 (<= 256)
    uint32_t idesc;
    uint32_t tcols;       // TMEM columns allocated (two accumulators)
    int64_t rows;         // rows with data: nrhs x nb
    int64_t nb;           // leaf boxes
    int H, R, rp, ncols;  // M~ layout: parity split, H = 2^(D-1); ncols = r of the leaf level
    float *out, *out_hi, *out_lo;
    unsigned *maxbits;    // the level's max |M~| (float bits), or null
    int *status;
    // a second segment (the boxes of level D-1 when they share the leaves'
    // operator): tiles tile2 .. ntiles-1, its own A, rows, output and max
    CUtensorMap a2;
    int tile2;            // ntiles when there is no second segment
    int drain;            // a fresh TMEM partial per K chunk, summed in FP32 by the epilogue (N <= 128)
    int64_t rows2, slice_rows2, nb2;
    int H2;
    float *out2, *out2_hi, *out2_lo;
    unsigned *maxbits2;
};

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int MODE>
__global__ void __launch_bounds__(kGemmThreads, 1) k_leaf_gemm(const __grid_constant__ GemmLaunch G)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = smem_raw + (base - raw);
    // [B hi: kchunks x N x 128 B][B lo: same][stages x (A hi 16 KB, A lo 16 KB)][barriers]
    const uint32_t bchunk = (uint32_t)G.N * 128u;
    const uint32_t bhi0 = base, blo0 = base + (uint32_t)G.kchunks * bchunk;
    const uint32_t a0 = blo0 + (uint32_t)G.kchunks * bchunk;
    uint8_t *const abase = gbase + (a0 - base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(abase + (size_t)kGemmStages * 2 * kAChunkBytes);
    const uint32_t bfull = smem_u32(bars), full0 = bfull + 8, split0 = full0 + 8 * kGemmStages,
                   empty0 = split0 + 8 * kGemmStages, afull0 = empty0 + 8 * kGemmStages, aempty0 = afull0 + 16,
                   done_bar = aempty0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 + 3 * kGemmStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(bfull, 1);
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(split0 + 8 * s, 64);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(afull0 + 8 * b, 1);
            mbar_init(aempty0 + 8 * b, 128);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), G.tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int nkc = G.kchunks, nk = G.kchunks * G.slices; // chunks per tile (over all slices)

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ producer
        mbar_arrive_expect_tx(bfull, 2u * (uint32_t)nkc * bchunk);
        for (int kc = 0; kc < nkc; ++kc) {
            tma_load_2d(bhi0 + (uint32_t)kc * bchunk, &G.bhi, bfull, kGemmK * kc, 0);
            tma_load_2d(blo0 + (uint32_t)kc * bchunk, &G.blo, bfull, kGemmK * kc, 0);
        }
        int s = 0, round = 0;
        int last_round[kGemmStages] = {-1, -1, -1};
        for (int tile = blockIdx.x; tile < G.ntiles && !*abort_flag; tile += gridDim.x)
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(empty0 + 8 * s, round ^ 1, abort_flag))
                    break;
                mbar_arrive_expect_tx(full0 + 8 * s, kAChunkBytes);
                last_round[s] = round;
                const int g = kc / nkc, kk = kc - g * nkc;
                const bool sec = tile >= G.tile2;
                const int lt = sec ? tile - G.tile2 : tile;
                tma_load_2d(a0 + (uint32_t)s * 2u * kAChunkBytes, sec ? &G.a2 : &G.a, full0 + 8 * s, kGemmK * kk,
                            (int)(g * (sec ? G.slice_rows2 : G.slice_rows) + (int64_t)kGemmRows * lt));
                if (++s == kGemmStages) {
                    s = 0;
                    round ^= 1;
                }
            }
        // teardown: every armed copy has landed before the CTA exits
        long long t0 = clock64();
        while (!mbar_test(bfull, 0) && clock64() - t0 < kWaitCycles) {
        }
        for (int q = 0; q < kGemmStages; ++q)
            if (last_round[q] >= 0) {
                t0 = clock64();
                while (!mbar_test(full0 + 8 * q, (uint32_t)last_round[q]) && clock64() - t0 < kWaitCycles) {
                }
            }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        bool ok = mbar_wait(bfull, 0, abort_flag);
        tc_fence_after();
        const uint64_t dbh = sw128_desc(bhi0), dbl = sw128_desc(blo0), da = sw128_desc(a0);
        const uint32_t d_bch = bchunk >> 4, d_st = (2u * kAChunkBytes) >> 4, d_lo = kAChunkBytes >> 4;
        int s = 0, sph = 0, buf = 0, bph = 0;
        for (int tile = blockIdx.x; ok && tile < G.ntiles; tile += gridDim.x) {
            uint32_t d = 0, acc = 0;
            for (int kc = 0; kc < nk; ++kc) {
                // a fresh accumulator per tile, or per chunk with drain
                if (G.drain || kc == 0) {
                    if (!mbar_wait(aempty0 + 8 * buf, bph ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    d = tmem_base + (uint32_t)(buf * G.N);
                    acc = 0;
                }
                if (!mbar_wait(split0 + 8 * s, sph, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ah = da + (uint64_t)(s * d_st), al = ah + d_lo;
                const int kk = kc % nkc; // the B chunk: K position within the slice
                const uint64_t bh = dbh + (uint64_t)(kk * d_bch), bl = dbl + (uint64_t)(kk * d_bch);
#pragma unroll
                for (int k = 0; k < kGemmK / 8; ++k) { // K = 8 per MMA: 32 bytes
                    const uint64_t dk = (uint64_t)(2 * k);
                    mma_tf32(d, ah + dk, bl + dk, G.idesc, acc); // corrections first: the sum is small then
                    mma_tf32(d, al + dk, bh + dk, G.idesc, 1u);
                    mma_tf32(d, ah + dk, bh + dk, G.idesc, 1u);
                    acc = 1u;
                }
                mma_commit(empty0 + 8 * s); // frees the stage once these MMAs have read it
                if (++s == kGemmStages) {
                    s = 0;
                    sph ^= 1;
                }
                if (G.drain || kc == nk - 1) {
                    mma_commit(afull0 + 8 * buf); // the chunk's (or the tile's) partial is complete
                    if (++buf == 2) {
                        buf = 0;
                        bph ^= 1;
                    }
                }
            }
            if (!ok)
                break;
        }
        mma_commit(done_bar); // every MMA of this thread has completed before TMEM is freed
        long long t0 = clock64();
        while (!mbar_test(done_bar, 0) && clock64() - t0 < kWaitCycles) {
        }
    } else if (warp == 2 || warp == 3) {
        // ------------------------------------------------------------ splitter
        const int t = threadIdx.x - 64;
        int s = 0, sph = 0;
        for (int tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x) {
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(full0 + 8 * s, sph, abort_flag)) {
                    ok = false;
                    break;
                }
                float4 *hi = reinterpret_cast<float4 *>(abase + (size_t)s * 2 * kAChunkBytes);
                float4 *lo = hi + kAChunkBytes / 16;
#pragma unroll 4
                for (int j = t; j < (int)(kAChunkBytes / 16); j += 64) {
                    const float4 x = hi[j];
                    const float4 h = make_float4(tf32_rna(x.x), tf32_rna(x.y), tf32_rna(x.z), tf32_rna(x.w));
                    hi[j] = h;
                    lo[j] = make_float4(tf32_rna(x.x - h.x), tf32_rna(x.y - h.y), tf32_rna(x.z - h.z),
                                        tf32_rna(x.w - h.w));
                }
                // the tensor core reads shared memory through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(split0 + 8 * s);
                if (++s == kGemmStages) {
                    s = 0;
                    sph ^= 1;
                }
            }
            if (!ok)
                break;
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ epilogue
        const int e = threadIdx.x - 128; // TMEM lane = row of the tile
        const uint32_t lane_base = (uint32_t)(32 * (warp - 4)) << 16;
        int buf = 0, bph = 0;
        float mx = 0.0f, mx2 = 0.0f; // the two segments' max |M~|
        for (int tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x) {
            const bool sec = tile >= G.tile2;
            const int64_t row = (int64_t)kGemmRows * (sec ? tile - G.tile2 : tile) + e;
            const int64_t nb = sec ? G.nb2 : G.nb;
            float *const out = sec ? G.out2 : G.out;
            float *const out_hi = sec ? G.out2_hi : G.out_hi;
            float *const out_lo = sec ? G.out2_lo : G.out_lo;
            float mt = 0.0f; // this tile's max |M~|
            int64_t off = -1;
            if (row < (sec ? G.rows2 : G.rows)) {
                if (MODE == 0) {
                    const int c = (int)(row / nb);
                    int x, y, z;
                    demorton3((uint32_t)(row % nb), x, y, z);
                    off = parity_row(x, y, z, c, sec ? G.H2 : G.H, 1, G.R) * G.rp;
                } else {
                    off = row * G.ldo;
                }
            }
            // columns n0 .. n0 + 15 of this thread's row
            auto emit = [&](int n0, float *v) {
                if (MODE == 1 && off >= 0) { // all N columns (zero past p^3): 16-byte stores
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(out + off + n0 + j) =
                            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                } else if (off >= 0) {
                    // columns past the level's rank stay as they are (zero)
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + j >= G.ncols)
                            v[j] = 0.0f;
                    const int nv = min(16, G.ncols - n0);
                    if (nv == 16) { // 16-byte stores (off and n0 are multiples of 16)
#pragma unroll
                        for (int j = 0; j < 16; j += 4) {
                            *reinterpret_cast<float4 *>(out + off + n0 + j) =
                                make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                            if (out_hi) {
                                float h[4], l[4];
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    h[q] = tf32_rna(v[j + q]);
                                    l[q] = tf32_rna(v[j + q] - h[q]);
                                }
                                *reinterpret_cast<float4 *>(out_hi + off + n0 + j) = make_float4(h[0], h[1], h[2], h[3]);
                                *reinterpret_cast<float4 *>(out_lo + off + n0 + j) = make_float4(l[0], l[1], l[2], l[3]);
                            }
                        }
                    } else {
                        for (int j = 0; j < nv; ++j) {
                            out[off + n0 + j] = v[j];
                            if (out_hi) {
                                const float h = tf32_rna(v[j]);
                                out_hi[off + n0 + j] = h;
                                out_lo[off + n0 + j] = tf32_rna(v[j] - h);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        mt = fmaxf(mt, fabsf(v[j]));
                }
            };
            bool ok = true;
            if (G.drain) {
                // the tile's K chunks arrive as separate partials: their FP32
                // sum (round to nearest, in chunk order) keeps the tensor
                // core's truncating accumulation to one chunk
                float sum[8][16];
#pragma unroll
                for (int b = 0; b < 8; ++b)
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        sum[b][j] = 0.0f;
                for (int kc = 0; kc < nk && ok; ++kc) {
                    if (!mbar_wait(afull0 + 8 * buf, bph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int b = 0; b < 8; ++b)
                        if (16 * b < G.N) {
                            float v[16];
                            tmem_ld16(tmem_base + lane_base + (uint32_t)(buf * G.N + 16 * b), v);
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                sum[b][j] += v[j];
                        }
                    tc_fence_before();
                    mbar_arrive(aempty0 + 8 * buf);
                    if (++buf == 2) {
                        buf = 0;
                        bph ^= 1;
                    }
                }
                if (!ok)
                    break;
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    if (16 * b < G.N)
                        emit(16 * b, sum[b]);
            } else {
                if (!mbar_wait(afull0 + 8 * buf, bph, abort_flag))
                    break;
                tc_fence_after();
                for (int n0 = 0; n0 < G.N; n0 += 16) {
                    float v[16];
                    tmem_ld16(tmem_base + lane_base + (uint32_t)(buf * G.N + n0), v);
                    emit(n0, v);
                }
                tc_fence_before();
                mbar_arrive(aempty0 + 8 * buf);
                if (++buf == 2) {
                    buf = 0;
                    bph ^= 1;
                }
            }
            if (sec)
                mx2 = fmaxf(mx2, mt);
            else
                mx = fmaxf(mx, mt);
        }
        if (MODE == 0) {
            for (int o = 16; o > 0; o >>= 1) {
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, o));
            }
            if (lane == 0 && mx > 0.0f && G.maxbits)
                atomicMax(G.maxbits, __float_as_uint(mx));
            if (lane == 0 && mx2 > 0.0f && G.maxbits2)
                atomicMax(G.maxbits2, __float_as_uint(mx2));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag)
        atomicOr(G.status, kStatusTimeoutBit);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, G.tcols);
    }
}

size_t gemm_smem_bytes(int N, int kchunks)
{
    return 1024 + 2 * (size_t)kchunks * N * 128 + (size_t)kGemmStages * 2 * kAChunkBytes + 256;
}

} // namespace

bool leaf_compress_fits(int r, int p3p)
{
    const int N = (r + 15) / 16 * 16, nk = (p3p + kGemmK - 1) / kGemmK;
    return r >= 1 && N <= 256 && gemm_smem_bytes(N, nk) <= 227 * 1024;
}

bool leaf_decompress_fits(int rp, int p3p)
{
    const int nk = (rp + kGemmK - 1) / kGemmK;
    return p3p % 16 == 0 && p3p <= 256 && gemm_smem_bytes(p3p, nk) <= 227 * 1024;
}

static cudaError_t run_gemm(GemmLaunch &G, int mode, cudaStream_t s)
{
    const size_t smem = gemm_smem_bytes(G.N, G.kchunks);
    const void *fn = mode == 0 ? (const void *)k_leaf_gemm<0> : (const void *)k_leaf_gemm<1>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const int sms = tc_sm_count();
    const int grid = std::max(1, std::min(G.ntiles, sms > 0 ? sms : 1));
    if (mode == 0)
        k_leaf_gemm<0><<<grid, kGemmThreads, smem, s>>>(G);
    else
        k_leaf_gemm<1><<<grid, kGemmThreads, smem, s>>>(G);
    return cudaGetLastError();
}

// the GEMM of one compression (rows = nrhs x nb boxes of one level)
static cudaError_t compress_setup(GemmLaunch &G, const LeafCompressArgs &L)
{
    if (!leaf_compress_fits(L.r, L.p3p) || L.nrhs < 1 || L.nb < 1 || L.p3p % 4 != 0 || L.rp % 4 != 0)
        return cudaErrorInvalidValue;
    memset(&G, 0, sizeof(G));
    G.N = (L.r + 15) / 16 * 16;
    G.kchunks = (L.p3p + kGemmK - 1) / kGemmK;
    G.slices = 1;
    G.rows = (int64_t)L.nrhs * L.nb;
    G.slice_rows = G.rows;
    G.ntiles = (int)((G.rows + kGemmRows - 1) / kGemmRows);
    G.tile2 = G.ntiles;
    G.drain = G.N <= 128 ? 1 : 0;
    G.idesc = idesc_tf32(kGemmRows, G.N);
    G.tcols = 32;
    while (G.tcols < (uint32_t)(2 * G.N))
        G.tcols *= 2;
    G.nb = L.nb;
    G.H = L.H;
    G.R = L.R;
    G.rp = L.rp;
    G.ncols = L.r;
    G.out = L.out;
    G.out_hi = L.out_hi;
    G.out_lo = L.out_lo;
    G.maxbits = L.maxbits;
    G.status = L.status;
    cudaError_t e = tc_encode_2d_f32(&G.a, L.M, (uint64_t)L.p3p, (uint64_t)G.rows, (uint64_t)L.p3p * 4, kGemmK,
                                     kGemmRows);
    if (e == cudaSuccess)
        e = tc_encode_2d_f32(&G.bhi, L.Vt_hi, (uint64_t)L.p3p, (uint64_t)L.rp, (uint64_t)L.p3p * 4, kGemmK,
                             (uint32_t)G.N);
    if (e == cudaSuccess)
        e = tc_encode_2d_f32(&G.blo, L.Vt_lo, (uint64_t)L.p3p, (uint64_t)L.rp, (uint64_t)L.p3p * 4, kGemmK,
                             (uint32_t)G.N);
    return e;
}

cudaError_t launch_leaf_compress(const LeafCompressArgs &L, cudaStream_t s)
{
    GemmLaunch G;
    cudaError_t e = compress_setup(G, L);
    if (e != cudaSuccess)
        return e;
    return run_gemm(G, 0, s);
}

// two levels in one launch when they share the operator (and the shapes):
// the second level's tiles follow the first's
cudaError_t launch_leaf_compress2(const LeafCompressArgs &L, const LeafCompressArgs &L2, cudaStream_t s)
{
    if (L.Vt_hi != L2.Vt_hi || L.Vt_lo != L2.Vt_lo || L.r != L2.r || L.rp != L2.rp || L.p3p != L2.p3p ||
        L.nrhs != L2.nrhs || L.R != L2.R || L.status != L2.status) {
        cudaError_t e = launch_leaf_compress(L, s);
        return e == cudaSuccess ? launch_leaf_compress(L2, s) : e;
    }
    GemmLaunch G;
    cudaError_t e = compress_setup(G, L);
    if (e != cudaSuccess || L2.nb < 1)
        return e == cudaSuccess ? cudaErrorInvalidValue : e;
    G.rows2 = (int64_t)L2.nrhs * L2.nb;
    G.slice_rows2 = G.rows2;
    G.tile2 = G.ntiles;
    G.ntiles += (int)((G.rows2 + kGemmRows - 1) / kGemmRows);
    G.nb2 = L2.nb;
    G.H2 = L2.H;
    G.out2 = L2.out;
    G.out2_hi = L2.out_hi;
    G.out2_lo = L2.out_lo;
    G.maxbits2 = L2.maxbits;
    e = tc_encode_2d_f32(&G.a2, L2.M, (uint64_t)L2.p3p, (uint64_t)G.rows2, (uint64_t)L2.p3p * 4, kGemmK,
                         kGemmRows);
    if (e != cudaSuccess)
        return e;
    return run_gemm(G, 0, s);
}

// the GEMM of one decompression (rows = the rows of one F~ slice)
static cudaError_t decompress_setup(GemmLaunch &G, const LeafDecompressArgs &L)
{
    if (!leaf_decompress_fits(L.rp, L.p3p) || L.rows < 1 || L.slices < 1 || L.rp % 4 != 0)
        return cudaErrorInvalidValue;
    memset(&G, 0, sizeof(G));
    G.N = L.p3p;
    G.kchunks = (L.rp + kGemmK - 1) / kGemmK;
    G.slices = L.slices;
    G.rows = L.rows;
    G.slice_rows = L.slice_rows;
    G.ntiles = (int)((G.rows + kGemmRows - 1) / kGemmRows);
    G.tile2 = G.ntiles;
    G.drain = G.N <= 128 ? 1 : 0;
    G.idesc = idesc_tf32(kGemmRows, G.N);
    G.tcols = 32;
    while (G.tcols < (uint32_t)(2 * G.N))
        G.tcols *= 2;
    G.ldo = L.p3p;
    G.ncols = L.p3p;
    G.out = L.out;
    G.status = L.status;
    // A: the slices of F~ as one 2D matrix of slices x slice_rows rows
    cudaError_t e = tc_encode_2d_f32(&G.a, L.Ft, (uint64_t)L.rp, (uint64_t)L.slices * L.slice_rows,
                                     (uint64_t)L.rp * 4, kGemmK, kGemmRows);
    if (e == cudaSuccess)
        e = tc_encode_2d_f32(&G.bhi, L.U_hi, (uint64_t)L.rp, (uint64_t)L.p3p, (uint64_t)L.rp * 4, kGemmK,
                             (uint32_t)G.N);
    if (e == cudaSuccess)
        e = tc_encode_2d_f32(&G.blo, L.U_lo, (uint64_t)L.rp, (uint64_t)L.p3p, (uint64_t)L.rp * 4, kGemmK,
                             (uint32_t)G.N);
    return e;
}

cudaError_t launch_leaf_decompress(const LeafDecompressArgs &L, cudaStream_t s)
{
    GemmLaunch G;
    cudaError_t e = decompress_setup(G, L);
    if (e != cudaSuccess)
        return e;
    return run_gemm(G, 1, s);
}

cudaError_t launch_leaf_decompress2(const LeafDecompressArgs &L, const LeafDecompressArgs &L2, cudaStream_t s)
{
    if (L.U_hi != L2.U_hi || L.U_lo != L2.U_lo || L.rp != L2.rp || L.p3p != L2.p3p || L.slices != L2.slices ||
        L.status != L2.status) {
        cudaError_t e = launch_leaf_decompress(L, s);
        return e == cudaSuccess ? launch_leaf_decompress(L2, s) : e;
    }
    GemmLaunch G;
    cudaError_t e = decompress_setup(G, L);
    if (e != cudaSuccess || L2.rows < 1)
        return e == cudaSuccess ? cudaErrorInvalidValue : e;
    G.rows2 = L2.rows;
    G.slice_rows2 = L2.slice_rows;
    G.tile2 = G.ntiles;
    G.ntiles += (int)((G.rows2 + kGemmRows - 1) / kGemmRows);
    G.out2 = L2.out;
    e = tc_encode_2d_f32(&G.a2, L2.Ft, (uint64_t)L2.rp, (uint64_t)L2.slices * L2.slice_rows, (uint64_t)L2.rp * 4,
                         kGemmK, kGemmRows);
    if (e != cudaSuccess)
        return e;
    return run_gemm(G, 1, s);
}

} // namespace bbfmm
