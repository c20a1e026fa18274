// m2l_tc.cu -- far-field stage (Sec. 2.2 item 2) on the 5th-generation tensor
// cores:  F~^alpha = scale_l * sum_{beta in I(alpha)} C^(t) M~^beta  with the
// compressed operators C^(t) = U^T K^(t) V (Sec. 2.5 "Fast M2L translation").
//
// The stage is a dense contraction: for the 128 targets of a tile (an 8x4x4
// block of parent cells of one octant class) and each of the 189 offsets of
// the class, D[128 x r] += A_t[128 x r] * B_t[r x r]^T, where A_t gathers the
// source vectors M~ of the 128 targets (one TMA box of the parity-split M~
// array: consecutive parent cells of one source octant; out-of-range cells
// read as zero) and B_t = C^(t).  K is walked in 32-float (128-byte) chunks.
//
//   warp 0      TMA producer: one elected lane arms a stage barrier and issues
//               the box loads of A (and its low part) and B (and its low part)
//   warp 1      MMA issuer: one lane issues tcgen05.mma kind::tf32, M = 128,
//               N = r rounded to 16, K = 8 per instruction, accumulating in
//               TMEM; tcgen05.commit frees the stage / publishes the tile
//   warps 2..5  epilogue: tcgen05.ld of the 128 x N accumulator (double
//               buffered in TMEM so the next tile's MMAs overlap), scale, store
//
// Precision: kind::tf32 reads 10 explicit mantissa bits.  The 3-pass mode
// splits each operand into hi = tf32(x) and lo = tf32(x - hi) and forms
// hi*hi + hi*lo + lo*hi (the split-TF32 scheme of Ootomo & Yokota, 2022),
// which carries ~21 bits; the 1-pass mode uses the operands as they are.
//
// Every mbarrier wait is bounded (about 2^31 cycles): on expiry the kernel
// sets the plan's status word, stops issuing work, waits (bounded) for its own
// copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "bbfmm_internal.h"

namespace bbfmm {

// ---------------------------------------------------------------------------
// host side: operand splitting
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

// ---------------------------------------------------------------------------
// device helpers (inline PTX)
__constant__ int4 c_tab_tc[8][kOffsetsPerClass];

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

constexpr long long kWaitCycles = 1LL << 31;

// bounded wait; false (and *abort set) when the limit or an abort is hit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort_flag)
            return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *tm, uint32_t bar, int c0, int c1,
                                            int c2, int c3, int c4)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
                 "l"((uint64_t)tm), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, uint32_t bar, int c0, int c1,
                                            int c2)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
                 "l"((uint64_t)tm), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32, FP32 accumulate
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// shared-memory matrix descriptor: K-major operand in the canonical 128-byte
// swizzled layout (rows of 128 bytes, 8-row groups 1024 bytes apart)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3fffu);  // start address >> 4
    d |= (uint64_t)1u << 16;                  // leading-dimension byte offset (unused here) = 16 B
    d |= (uint64_t)(1024u >> 4) << 32;        // stride-dimension byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                  // descriptor version for tcgen05
    d |= (uint64_t)2u << 61;                  // 128-byte swizzle
    return d;
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
struct TcParams {
    float *Ft;
    int *status;
    int l, H, r, rp, nb, ncols, nrhs, nk, nstage, op_base;
    int tiles_x, tiles_y, tiles_z, ntiles;
    float scale;
    uint32_t stage_bytes, a_bytes, b_bytes;
};

template <int NPROD>
__global__ void __launch_bounds__(192, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
             const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBlo,
             const __grid_constant__ TcParams prm)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = smem_raw + (base - raw);
    const int S = prm.nstage;
    // barriers after the stage buffers
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (size_t)S * prm.stage_bytes);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
    const uint32_t tfull0 = empty0 + 8 * S, tempty0 = tfull0 + 16, done_bar = tempty0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(tfull0, 1);
        mbar_init(tfull0 + 8, 1);
        mbar_init(tempty0, 4);
        mbar_init(tempty0 + 8, 4);
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 2 * prm.ncols);
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
        for (int tile = blockIdx.x; tile < prm.ntiles && !*abort_flag; tile += gridDim.x) {
            int t = tile;
            const int tx = t % prm.tiles_x;
            t /= prm.tiles_x;
            const int ty = t % prm.tiles_y;
            t /= prm.tiles_y;
            const int tz = t % prm.tiles_z;
            t /= prm.tiles_z;
            const int ot = t & 7, c = t >> 3;
            const int X0 = 8 * tx, Y0 = 4 * ty, Z0 = 4 * tz;
            for (int e = 0; e < kOffsetsPerClass && !*abort_flag; ++e) {
                const int4 en = c_tab_tc[ot][e];
                const int ux = (en.z & 3) - 1, uy = ((en.z >> 2) & 3) - 1, uz = ((en.z >> 4) & 3) - 1;
                const int zq = en.y * (prm.H + 2) + 1 + Z0 + uz;
                for (int kc = 0; kc < prm.nk; ++kc, ++it) {
                    const int s = it % S, round = it / S;
                    if (!mbar_wait(empty0 + 8 * s, (round & 1) ^ 1, abort_flag))
                        break;
                    const uint32_t sa = base + (uint32_t)s * prm.stage_bytes;
                    const uint32_t fb = full0 + 8 * s;
                    mbar_arrive_expect_tx(fb, prm.stage_bytes);
                    last_round[s] = round;
                    tma_load_5d(sa, &tmA, fb, 32 * kc, c, X0 + ux, Y0 + uy, zq);
                    uint32_t off = prm.a_bytes;
                    if (NPROD == 3) {
                        tma_load_5d(sa + off, &tmAlo, fb, 32 * kc, c, X0 + ux, Y0 + uy, zq);
                        off += prm.a_bytes;
                    }
                    tma_load_3d(sa + off, &tmB, fb, 32 * kc, 0, prm.op_base + en.x);
                    off += prm.b_bytes;
                    if (NPROD == 3)
                        tma_load_3d(sa + off, &tmBlo, fb, 32 * kc, 0, prm.op_base + en.x);
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
        const uint32_t idesc = idesc_tf32(128, prm.nb);
        int it = 0, tcount = 0;
        for (int tile = blockIdx.x; tile < prm.ntiles && !*abort_flag; tile += gridDim.x, ++tcount) {
            const int buf = tcount & 1, use = tcount >> 1;
            if (!mbar_wait(tempty0 + 8 * buf, (use & 1) ^ 1, abort_flag))
                break;
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(buf * prm.ncols);
            uint32_t acc = 0;
            bool ok = true;
            for (int e = 0; e < kOffsetsPerClass && ok; ++e) {
                for (int kc = 0; kc < prm.nk; ++kc, ++it) {
                    const int s = it % S, round = it / S;
                    if (!mbar_wait(full0 + 8 * s, round & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + (uint32_t)s * prm.stage_bytes;
                    const uint64_t a_hi = sw128_desc(sa);
                    const uint64_t a_lo = sw128_desc(sa + prm.a_bytes);
                    const uint32_t b_off = NPROD == 3 ? 2 * prm.a_bytes : prm.a_bytes;
                    const uint64_t b_hi = sw128_desc(sa + b_off);
                    const uint64_t b_lo = sw128_desc(sa + b_off + prm.b_bytes);
                    const int rem = prm.r - 32 * kc;
                    const int ksteps = rem >= 32 ? 4 : (rem + 7) / 8;
                    for (int k = 0; k < ksteps; ++k) {
                        const uint64_t dk = (uint64_t)(2 * k); // 32 bytes >> 4
                        mma_tf32(d, a_hi + dk, b_hi + dk, idesc, acc);
                        acc = 1;
                        if (NPROD == 3) {
                            mma_tf32(d, a_hi + dk, b_lo + dk, idesc, 1);
                            mma_tf32(d, a_lo + dk, b_hi + dk, idesc, 1);
                        }
                    }
                    mma_commit(empty0 + 8 * s); // frees the stage once these MMAs have read it
                }
            }
            if (!ok)
                break;
            mma_commit(tfull0 + 8 * buf);
        }
        // all MMAs issued by this thread have completed before TMEM is freed
        mma_commit(done_bar);
        long long t0 = clock64();
        while (!mbar_test(done_bar, 0) && clock64() - t0 < kWaitCycles) {
        }
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3; // TMEM lane quadrant this warp may access
        const int row = 32 * q + lane;
        const int bx = row & 7, by = (row >> 3) & 3, bz = row >> 5;
        int tcount = 0;
        for (int tile = blockIdx.x; tile < prm.ntiles; tile += gridDim.x, ++tcount) {
            const int buf = tcount & 1, use = tcount >> 1;
            int ok = 1;
            if (lane == 0)
                ok = mbar_wait(tfull0 + 8 * buf, use & 1, abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0); // keep the warp converged for tcgen05.ld
            if (!ok)
                break;
            tc_fence_after();
            int t = tile;
            const int tx = t % prm.tiles_x;
            t /= prm.tiles_x;
            const int ty = t % prm.tiles_y;
            t /= prm.tiles_y;
            const int tz = t % prm.tiles_z;
            t /= prm.tiles_z;
            const int ot = t & 7, c = t >> 3;
            const int X = 8 * tx + bx, Y = 4 * ty + by, Z = 4 * tz + bz;
            const bool valid = X < prm.H && Y < prm.H && Z < prm.H;
            float *out = prm.Ft + ((((int64_t)ot * prm.H + Z) * prm.H + Y) * prm.H + X) * (int64_t)prm.nrhs *
                                      prm.rp +
                         (int64_t)c * prm.rp;
            const uint32_t trow = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * prm.ncols);
            for (int col = 0; col < prm.nb; col += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)col, v);
                if (valid) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        if (col + j < prm.r) {
                            float4 w = make_float4(prm.scale * v[j], prm.scale * v[j + 1], prm.scale * v[j + 2],
                                                   prm.scale * v[j + 3]);
                            *reinterpret_cast<float4 *>(out + col + j) = w;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(tempty0 + 8 * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*abort_flag && threadIdx.x == 0)
        atomicOr(prm.status, kStatusTimeout);
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem_base, 2 * prm.ncols);
    }
}

// ---------------------------------------------------------------------------
// host: tensor maps and launch
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_tc_mu;
static bool g_tab_tc_ready = false;

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
    return cudaSuccess;
}

// M~ (parity split, padded in Z): dims (rp, R, H, H, 8 (H + 2)); box (32, 1, 8, 4, 4)
static cudaError_t encode_a(CUtensorMap *tm, const float *ptr, int H, int R, int rp)
{
    cuuint64_t dims[5] = {(cuuint64_t)rp, (cuuint64_t)R, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)8 * (H + 2)};
    cuuint64_t strides[4] = {(cuuint64_t)rp * 4, (cuuint64_t)R * rp * 4, (cuuint64_t)H * R * rp * 4,
                             (cuuint64_t)H * H * R * rp * 4};
    cuuint32_t box[5] = {32, 1, 8, 4, 4};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, (void *)ptr, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// C (operators): dims (rp, rows64, nops); box (32, nb, 1)
static cudaError_t encode_b(CUtensorMap *tm, const float *ptr, int rp, int rows64, int nops, int nb)
{
    cuuint64_t dims[3] = {(cuuint64_t)rp, (cuuint64_t)rows64, (cuuint64_t)nops};
    cuuint64_t strides[2] = {(cuuint64_t)rp * 4, (cuuint64_t)rows64 * rp * 4};
    cuuint32_t box[3] = {32, (cuuint32_t)nb, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)ptr, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int g_num_sms = 0;

cudaError_t launch_m2l(bbfmm_plan_impl *P, int l, int nrhs, cudaStream_t s)
{
    const DevOps &O = *P->ops;
    const int k = O.nlev == 1 ? 0 : l - 2;
    // homogeneous kernels: operators made for the leaf box, scaled by (h_l / h_D)^m
    float scale = 1.0f;
    if (O.host->hom_degree != 0)
        scale = (float)pow(2.0, (double)O.host->hom_degree * (P->D - l));
    if (P->precision == BBFMM_PREC_FP32)
        return launch_m2l_fp32(P->lev[l].Mt, O.C[k], P->lev[l].Ft, l, O.r, O.rp, O.rows64, nrhs, scale, s);

    cudaError_t e = tc_init();
    if (e != cudaSuccess)
        return e;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const bool three = P->precision == BBFMM_PREC_TF32X3;
    const int H = 1 << (l - 1);
    const int nb = (O.r + 15) / 16 * 16;
    if (nb > 256 || O.rp % 4 != 0)
        return cudaErrorInvalidValue;
    TcParams prm;
    prm.Ft = P->lev[l].Ft;
    prm.status = P->status;
    prm.l = l;
    prm.H = H;
    prm.r = O.r;
    prm.rp = O.rp;
    prm.nb = nb;
    prm.ncols = nb <= 32 ? 32 : nb <= 64 ? 64 : nb <= 128 ? 128 : 256;
    prm.nrhs = nrhs;
    prm.nk = (O.r + 31) / 32;
    prm.op_base = 0;
    prm.tiles_x = (H + 7) / 8;
    prm.tiles_y = (H + 3) / 4;
    prm.tiles_z = (H + 3) / 4;
    prm.ntiles = prm.tiles_x * prm.tiles_y * prm.tiles_z * 8 * nrhs;
    prm.scale = scale;
    prm.a_bytes = 128 * 128;
    prm.b_bytes = (uint32_t)nb * 128;
    prm.stage_bytes = (three ? 2 : 1) * (prm.a_bytes + prm.b_bytes);
    const size_t budget = 220 * 1024;
    int nstage = (int)((budget - 1024 - 256) / prm.stage_bytes);
    nstage = nstage > 8 ? 8 : nstage;
    if (nstage < 2)
        return cudaErrorInvalidValue;
    prm.nstage = nstage;
    const size_t smem = 1024 + (size_t)nstage * prm.stage_bytes + 256;

    const float *A = three ? P->lev[l].Mt_hi : P->lev[l].Mt;
    const float *B = three ? O.Chi[k] : O.C[k];
    CUtensorMap tA, tAlo, tB, tBlo;
    e = encode_a(&tA, A, H, P->max_nrhs, O.rp);
    if (e == cudaSuccess)
        e = encode_a(&tAlo, three ? P->lev[l].Mt_lo : A, H, P->max_nrhs, O.rp);
    if (e == cudaSuccess)
        e = encode_b(&tB, B, O.rp, O.rows64, kNumOffsets, nb);
    if (e == cudaSuccess)
        e = encode_b(&tBlo, three ? O.Clo[k] : B, O.rp, O.rows64, kNumOffsets, nb);
    if (e != cudaSuccess)
        return e;
    const int grid = prm.ntiles < g_num_sms ? prm.ntiles : g_num_sms;
    if (three) {
        e = cudaFuncSetAttribute(k_m2l_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_m2l_tc<3><<<grid, 192, smem, s>>>(tA, tAlo, tB, tBlo, prm);
    } else {
        e = cudaFuncSetAttribute(k_m2l_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_m2l_tc<1><<<grid, 192, smem, s>>>(tA, tAlo, tB, tBlo, prm);
    }
    return cudaGetLastError();
}

} // namespace bbfmm
