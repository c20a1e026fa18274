// transfers.cu -- the interpolation stages of the black-box FMM (Sec. 2.2):
// P2M (item 1), M2M (item 1), the SVD compress / decompress around M2L
// (Sec. 2.5 "Fast M2L translation"), L2L and L2P (item 3), plus the gather of
// the weights into tree order and the final combine / un-permute.
//
// Points carry leaf-local coordinates u in [-1/2, 1/2]^3 (cell units), so the
// reference coordinate of a point in its leaf (the [-1,1] frame of Def. 2.2)
// is s = 2u.  The 1D Lagrange basis is evaluated as
// l_i(s) = w_i prod_{k != i} (s - s_k) with w_i = 1 / prod_{k != i} (s_i - s_k).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bbfmm_internal.h"

namespace bbfmm {

InterpTables make_interp_tables(const HostOps &h)
{
    InterpTables T = {};
    for (int k = 0; k < h.p; ++k) {
        T.nodes[k] = (float)h.nodes[k];
        T.wbary[k] = (float)h.wbary[k];
    }
    for (int o = 0; o < 2; ++o)
        for (int i = 0; i < h.p; ++i)
            for (int j = 0; j < h.p; ++j)
                T.S[o][i][j] = (float)h.S[(size_t)o * h.p * h.p + (size_t)i * h.p + j];
    return T;
}

template <int P>
__device__ inline void lagrange_1d(const InterpTables &T, float s, float *out)
{
#pragma unroll
    for (int i = 0; i < P; ++i) {
        float v = T.wbary[i];
#pragma unroll
        for (int k = 0; k < P; ++k)
            if (k != i)
                v *= s - T.nodes[k];
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
__global__ void k_gather(const float *__restrict__ sigma, const int *__restrict__ perm, int64_t n, int nrhs,
                         float *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = perm[i];
    for (int c = 0; c < nrhs; ++c)
        out[(int64_t)c * n + i] = sigma[(int64_t)c * n + j];
}

const void *gather_kernel() { return (const void *)k_gather; }

cudaError_t launch_gather_sigma(const float *sigma, const int *perm, int64_t n, int nrhs, float *out,
                                cudaStream_t s)
{
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sigma, perm, n, nrhs, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// P2M: M^alpha_i = sum_{y_j in alpha} L_p(y*_i, y_j) sigma_j.  One warp per
// leaf; points in chunks of 32, lane j tabulates the 3p basis values of point
// j in shared memory, then every lane accumulates coefficients lane, lane+32...
constexpr int kP2MWarps = 4;

template <int P>
__global__ void __launch_bounds__(32 * kP2MWarps) k_p2m(const __grid_constant__ InterpTables T, const float4 *__restrict__ pts, const float *__restrict__ sig,
                                                       const int *__restrict__ off, int64_t n, int64_t nleaf,
                                                       int nrhs, float *__restrict__ M)
{
    constexpr int P3 = P * P * P, NC = (P3 + 31) / 32;
    __shared__ float sL[kP2MWarps][3][32][P];
    __shared__ float sSig[kP2MWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * kP2MWarps + w;
    if (m >= nleaf)
        return;
    const int s0 = off[m], s1 = off[m + 1];
    int ci[NC][3];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        int i = lane + 32 * q;
        ci[q][0] = i % P;
        ci[q][1] = (i / P) % P;
        ci[q][2] = i / (P * P);
    }
    for (int c0 = s0; c0 < s1 || c0 == s0; c0 += 32) {
        const int cnt = min(32, s1 - c0);
        if (lane < cnt) {
            float4 u = pts[c0 + lane];
            float L[P];
            lagrange_1d<P>(T, 2.0f * u.x, L);
#pragma unroll
            for (int i = 0; i < P; ++i)
                sL[w][0][lane][i] = L[i];
            lagrange_1d<P>(T, 2.0f * u.y, L);
#pragma unroll
            for (int i = 0; i < P; ++i)
                sL[w][1][lane][i] = L[i];
            lagrange_1d<P>(T, 2.0f * u.z, L);
#pragma unroll
            for (int i = 0; i < P; ++i)
                sL[w][2][lane][i] = L[i];
        }
        for (int c = 0; c < nrhs; ++c) {
            __syncwarp();
            if (lane < cnt)
                sSig[w][lane] = sig[(int64_t)c * n + c0 + lane];
            __syncwarp();
            float acc[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q)
                acc[q] = 0.0f;
            for (int j = 0; j < cnt; ++j) {
                float sg = sSig[w][j];
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    acc[q] += sL[w][0][j][ci[q][0]] * sL[w][1][j][ci[q][1]] * sL[w][2][j][ci[q][2]] * sg;
            }
            float *out = M + ((int64_t)m * nrhs + c) * P3;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                int i = lane + 32 * q;
                if (i < P3)
                    out[i] = c0 == s0 ? acc[q] : out[i] + acc[q];
            }
        }
        if (cnt <= 0)
            break;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// L2P: phi_i = sum_j F^alpha_j L_p(x*_j, x_i).  One warp per leaf, one lane
// per target point; the leaf's coefficients are broadcast from shared memory.
constexpr int kL2PWarps = 4;

template <int P>
__global__ void __launch_bounds__(32 * kL2PWarps) k_l2p(const __grid_constant__ InterpTables T, const float4 *__restrict__ pts, const float *__restrict__ F,
                                                       const int *__restrict__ off, int64_t n, int64_t nleaf,
                                                       int nrhs, float *__restrict__ phi)
{
    constexpr int P3 = P * P * P;
    __shared__ float sF[kL2PWarps][P3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * kL2PWarps + w;
    if (m >= nleaf)
        return;
    const int s0 = off[m], s1 = off[m + 1];
    if (s1 == s0)
        return;
    for (int c0 = s0; c0 < s1; c0 += 32) {
        // the lane's point and its basis values, reused for every right-hand side
        const int j = c0 + lane;
        const bool has = j < s1;
        float Lx[P], Ly[P], Lz[P];
        const float4 u = pts[has ? j : s0];
        lagrange_1d<P>(T, 2.0f * u.x, Lx);
        lagrange_1d<P>(T, 2.0f * u.y, Ly);
        lagrange_1d<P>(T, 2.0f * u.z, Lz);
        for (int c = 0; c < nrhs; ++c) {
            __syncwarp();
            const float *Fm = F + ((int64_t)m * nrhs + c) * P3;
            for (int i = lane; i < P3; i += 32)
                sF[w][i] = Fm[i];
            __syncwarp();
            float acc = 0.0f;
#pragma unroll
            for (int i3 = 0; i3 < P; ++i3) {
#pragma unroll
                for (int i2 = 0; i2 < P; ++i2) {
                    float yz = Ly[i2] * Lz[i3];
                    float part = 0.0f;
#pragma unroll
                    for (int i1 = 0; i1 < P; ++i1)
                        part += sF[w][i1 + P * (i2 + P * i3)] * Lx[i1];
                    acc += part * yz;
                }
            }
            if (has)
                phi[(int64_t)c * n + j] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// M2M: M^parent = sum_o (S_ox (x) S_oy (x) S_oz) M^child_o, done as three
// 1D passes (the O(8 p^4) tensor form of Thm. 2.1, item 1).  One block per
// parent; the 8 children of parent m are boxes 8m..8m+7 (Morton order).
template <int P>
__global__ void __launch_bounds__(128) k_m2m(const __grid_constant__ InterpTables T, const float *__restrict__ Mc, float *__restrict__ Mp, int64_t npar,
                                             int nrhs)
{
    constexpr int P3 = P * P * P;
    extern __shared__ float smem[];
    float *A = smem, *B = smem + 8 * P3;
    const int64_t m = blockIdx.x;
    for (int c = 0; c < nrhs; ++c) {
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, j = q % P3;
            A[q] = Mc[((8 * m + o) * nrhs + c) * P3 + j];
        }
        __syncthreads();
        // x pass: B[o][i1 + P j2 + P^2 j3] = sum_j1 S[ox][i1][j1] A[o][j1 + P j2 + P^2 j3]
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, r = q % P3, i1 = r % P, rest = r / P;
            const float *a = A + o * P3 + rest * P;
            float acc = 0.0f;
#pragma unroll
            for (int j1 = 0; j1 < P; ++j1)
                acc += T.S[o & 1][i1][j1] * a[j1];
            B[q] = acc;
        }
        __syncthreads();
        // y pass: A[o][i1 + P i2 + P^2 j3] = sum_j2 S[oy][i2][j2] B[o][i1 + P j2 + P^2 j3]
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, r = q % P3, i1 = r % P, i2 = (r / P) % P, j3 = r / (P * P);
            const float *b = B + o * P3 + i1 + P * P * j3;
            float acc = 0.0f;
#pragma unroll
            for (int j2 = 0; j2 < P; ++j2)
                acc += T.S[(o >> 1) & 1][i2][j2] * b[P * j2];
            A[q] = acc;
        }
        __syncthreads();
        // z pass and sum over the children
        for (int r = threadIdx.x; r < P3; r += blockDim.x) {
            int i12 = r % (P * P), i3 = r / (P * P);
            float acc = 0.0f;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const float *a = A + o * P3 + i12;
#pragma unroll
                for (int j3 = 0; j3 < P; ++j3)
                    acc += T.S[o >> 2][i3][j3] * a[P * P * j3];
            }
            Mp[(m * nrhs + c) * P3 + r] = acc;
        }
        __syncthreads();
    }
}

// L2L: F^child_o[i] = sum_j F^parent[j] S_ox[j1][i1] S_oy[j2][i2] S_oz[j3][i3]
// (Sec. 2.2 item 3, the transpose of M2M); writes (does not accumulate) the
// 8 children of each parent.
template <int P>
__global__ void __launch_bounds__(128) k_l2l(const __grid_constant__ InterpTables T, const float *__restrict__ Fp, float *__restrict__ Fc, int64_t npar,
                                             int nrhs)
{
    constexpr int P3 = P * P * P;
    extern __shared__ float smem[];
    float *Fs = smem, *A = smem + P3, *B = smem + P3 + 8 * P3;
    const int64_t m = blockIdx.x;
    for (int c = 0; c < nrhs; ++c) {
        for (int q = threadIdx.x; q < P3; q += blockDim.x)
            Fs[q] = Fp[(m * nrhs + c) * P3 + q];
        __syncthreads();
        // z pass: A[o][j1 + P j2 + P^2 i3] = sum_j3 S[oz][j3][i3] F[j1 + P j2 + P^2 j3]
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, r = q % P3, j12 = r % (P * P), i3 = r / (P * P);
            float acc = 0.0f;
#pragma unroll
            for (int j3 = 0; j3 < P; ++j3)
                acc += T.S[o >> 2][j3][i3] * Fs[j12 + P * P * j3];
            A[q] = acc;
        }
        __syncthreads();
        // y pass: B[o][j1 + P i2 + P^2 i3] = sum_j2 S[oy][j2][i2] A[o][j1 + P j2 + P^2 i3]
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, r = q % P3, j1 = r % P, i2 = (r / P) % P, i3 = r / (P * P);
            const float *a = A + o * P3 + j1 + P * P * i3;
            float acc = 0.0f;
#pragma unroll
            for (int j2 = 0; j2 < P; ++j2)
                acc += T.S[(o >> 1) & 1][j2][i2] * a[P * j2];
            B[q] = acc;
        }
        __syncthreads();
        // x pass: out[o][i1 + P i2 + P^2 i3] = sum_j1 S[ox][j1][i1] B[o][j1 + P i2 + P^2 i3]
        for (int q = threadIdx.x; q < 8 * P3; q += blockDim.x) {
            int o = q / P3, r = q % P3, i1 = r % P, rest = r / P;
            const float *b = B + o * P3 + rest * P;
            float acc = 0.0f;
#pragma unroll
            for (int j1 = 0; j1 < P; ++j1)
                acc += T.S[o & 1][j1][i1] * b[j1];
            Fc[((8 * m + o) * nrhs + c) * P3 + r] = acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// node GEMMs of the SVD compression: rows are (box, rhs) pairs.
//   compress   (MODE 0): Mt[row][k] = sum_i M[row][i] V[i][k]      (M~ = V^T M)
//   decompress (MODE 1): F[row][i] (+)= sum_k Ft[row][k] Ut[k][i]  (F = U F~)
// M and F rows are contiguous p3-vectors in Morton order; Mt / Ft rows sit at
// parity_row() of their box.
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_node_gemm(const float *__restrict__ A, const float *__restrict__ W,
                                                   float *__restrict__ Out, int64_t rows, int K, int N, int ldw,
                                                   int lda, int ldo, int level, int nrhs, int accumulate,
                                                   float *__restrict__ Out_hi, float *__restrict__ Out_lo,
                                                   int nslices, int64_t slice, unsigned *__restrict__ maxbits,
                                                   int R)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Ws[16][64 + 4];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t row0 = (int64_t)blockIdx.x * 64;
    const int col0 = blockIdx.y * 64;
    const int H = level >= 1 ? 1 << (level - 1) : 1;
    // address of a row of A (input) and of Out
    auto parity_addr = [&](int64_t row, int padZ, int ld) -> int64_t {
        int64_t m = row / nrhs;
        int c = (int)(row % nrhs);
        int x, y, z;
        demorton3((uint32_t)m, x, y, z);
        return parity_row(x, y, z, c, H, padZ, R) * ld;
    };
    const int lr = tid >> 2, lk = (tid & 3) * 4; // A loader: row lr, k lk..lk+3
    const int64_t arow = row0 + lr;
    int64_t abase = -1;
    if (arow < rows)
        abase = MODE == 0 ? arow * lda : parity_addr(arow, 0, lda);
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int k = k0 + lk + q;
            float a = 0.0f;
            if (abase >= 0 && k < K) {
                // partial M2L sums of the offset groups, added in a fixed order
                a = A[abase + k];
                for (int g = 1; g < nslices; ++g)
                    a += A[g * slice + abase + k];
            }
            As[lk + q][lr] = a;
        }
        {
            int wk = tid >> 4, wc = (tid & 15) * 4;
            int k = k0 + wk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int col = col0 + wc + q;
                Ws[wk][wc + q] = (k < K && col < N) ? W[(int64_t)k * ldw + col] : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Ws[kk][tx * 4 + q];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t row = row0 + ty * 4 + i;
        if (row >= rows)
            continue;
        int64_t obase = MODE == 0 ? parity_addr(row, 1, ldo) : row * ldo;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int col = col0 + tx * 4 + j;
            if (col >= N)
                continue;
            if (accumulate)
                Out[obase + col] += acc[i][j];
            else
                Out[obase + col] = acc[i][j];
            if (MODE == 0 && Out_hi) { // split for the 3-pass tensor-core M2L
                float hi = tf32_rna(acc[i][j]);
                Out_hi[obase + col] = hi;
                Out_lo[obase + col] = tf32_rna(acc[i][j] - hi);
            }
        }
    }
    if (MODE == 0 && maxbits) { // max |M~| of the level (order-independent)
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (row0 + ty * 4 + i < rows && col0 + tx * 4 + j < N)
                    m = fmaxf(m, fabsf(acc[i][j]));
        for (int o = 16; o > 0; o >>= 1)
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0)
            atomicMax(maxbits, __float_as_uint(m));
    }
}

// 16-bit split: x * s = hi + lo, hi = round16(x s), lo = round16(x s - hi);
// s = 2^(13 - e) with 2^(e-1) < max|x| <= 2^e for FP16 (keeps hi below the
// FP16 range limit and lo away from the subnormals), s = 1 for BF16
template <int FMT>
__global__ void k_split16(const float *__restrict__ x, int64_t n, const unsigned *__restrict__ maxbits,
                          float *__restrict__ scale, uint16_t *__restrict__ hi, uint16_t *__restrict__ lo)
{
    float s = 1.0f;
    if (FMT == 0) {
        float mx = __uint_as_float(*maxbits);
        int e = 0;
        if (mx > 0.0f)
            frexpf(mx, &e);
        s = ldexpf(1.0f, 13 - e);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *scale = s;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v = x[i] * s;
        if (FMT == 0) {
            __half h = __float2half_rn(v);
            __half l = __float2half_rn(v - __half2float(h));
            hi[i] = __half_as_ushort(h);
            lo[i] = __half_as_ushort(l);
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            hi[i] = __bfloat16_as_ushort(h);
            lo[i] = __bfloat16_as_ushort(l);
        }
    }
}

cudaError_t launch_split16(const float *Mt, int64_t n, int fmt, const unsigned *maxbits, float *scale, uint16_t *hi,
                           uint16_t *lo, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    blocks = blocks > 4096 ? 4096 : blocks;
    if (fmt == 0)
        k_split16<0><<<(unsigned)blocks, 256, 0, s>>>(Mt, n, maxbits, scale, hi, lo);
    else
        k_split16<1><<<(unsigned)blocks, 256, 0, s>>>(Mt, n, maxbits, scale, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_compress(const float *M, const float *V, float *Mt, float *Mt_hi, float *Mt_lo, unsigned *maxbits,
                            int l, int p3, int r, int rp, int nrhs, int R, cudaStream_t s)
{
    int64_t rows = ((int64_t)1 << (3 * l)) * nrhs;
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((r + 63) / 64));
    k_node_gemm<0><<<grid, 256, 0, s>>>(M, V, Mt, rows, p3, r, rp, p3, rp, l, nrhs, 0, Mt_hi, Mt_lo, 1, 0, maxbits, R);
    return cudaGetLastError();
}

cudaError_t launch_decompress(const float *Ft, int nslices, int64_t slice, const float *Ut, float *F, int l, int p3,
                              int p3p, int r, int rp, int nrhs, int R, bool accumulate, cudaStream_t s)
{
    int64_t rows = ((int64_t)1 << (3 * l)) * nrhs;
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((p3 + 63) / 64));
    k_node_gemm<1><<<grid, 256, 0, s>>>(Ft, Ut, F, rows, r, p3, p3p, rp, p3, l, nrhs, accumulate ? 1 : 0, nullptr,
                                        nullptr, nslices, slice, nullptr, R);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_combine(const float *__restrict__ far, const float *__restrict__ near,
                          const int *__restrict__ perm, int64_t n, int nrhs, float *__restrict__ phi)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = perm[i];
    for (int c = 0; c < nrhs; ++c) {
        float v = near[(int64_t)c * n + i];
        if (far)
            v += far[(int64_t)c * n + i];
        phi[(int64_t)c * n + j] = v;
    }
}

const void *combine_kernel() { return (const void *)k_combine; }

cudaError_t launch_combine(const float *phi_far, const float *phi_near, const int *perm, int64_t n, int nrhs,
                           float *phi, cudaStream_t s)
{
    k_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi_far, phi_near, perm, n, nrhs, phi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dispatch on p
#define BBFMM_DISPATCH_P(p, F)                                                                                  \
    switch (p) {                                                                                                \
    case 2: F(2); break;                                                                                        \
    case 3: F(3); break;                                                                                        \
    case 4: F(4); break;                                                                                        \
    case 5: F(5); break;                                                                                        \
    case 6: F(6); break;                                                                                        \
    case 7: F(7); break;                                                                                        \
    case 8: F(8); break;                                                                                        \
    case 9: F(9); break;                                                                                        \
    case 10: F(10); break;                                                                                      \
    default: return cudaErrorInvalidValue;                                                                      \
    }

cudaError_t launch_p2m(const InterpTables &T, const float4 *pts, const float *sig, const int *leaf_off, int64_t n, int D, int p, int nrhs,
                       float *M, cudaStream_t s)
{
    int64_t nleaf = (int64_t)1 << (3 * D);
    unsigned blocks = (unsigned)((nleaf + kP2MWarps - 1) / kP2MWarps);
#define L(P) k_p2m<P><<<blocks, 32 * kP2MWarps, 0, s>>>(T, pts, sig, leaf_off, n, nleaf, nrhs, M)
    BBFMM_DISPATCH_P(p, L)
#undef L
    return cudaGetLastError();
}

cudaError_t launch_l2p(const InterpTables &T, const float4 *pts, const float *F, const int *leaf_off, int64_t n, int D, int p, int nrhs,
                       float *phi_far, cudaStream_t s)
{
    int64_t nleaf = (int64_t)1 << (3 * D);
    unsigned blocks = (unsigned)((nleaf + kL2PWarps - 1) / kL2PWarps);
#define L(P) k_l2p<P><<<blocks, 32 * kL2PWarps, 0, s>>>(T, pts, F, leaf_off, n, nleaf, nrhs, phi_far)
    BBFMM_DISPATCH_P(p, L)
#undef L
    return cudaGetLastError();
}

template <int P>
static cudaError_t m2m_p(const InterpTables &T, const float *Mc, float *Mp, int64_t npar, int nrhs, cudaStream_t s)
{
    size_t smem = sizeof(float) * 16 * P * P * P;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_m2m<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    k_m2m<P><<<(unsigned)npar, 128, smem, s>>>(T, Mc, Mp, npar, nrhs);
    return cudaGetLastError();
}

template <int P>
static cudaError_t l2l_p(const InterpTables &T, const float *Fp, float *Fc, int64_t npar, int nrhs, cudaStream_t s)
{
    size_t smem = sizeof(float) * 17 * P * P * P;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_l2l<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    k_l2l<P><<<(unsigned)npar, 128, smem, s>>>(T, Fp, Fc, npar, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_m2m(const InterpTables &T, const float *Mchild, float *Mparent, int lparent, int p, int nrhs, cudaStream_t s)
{
    int64_t npar = (int64_t)1 << (3 * lparent);
#define L(P) return m2m_p<P>(T, Mchild, Mparent, npar, nrhs, s)
    BBFMM_DISPATCH_P(p, L)
#undef L
    return cudaSuccess;
}

cudaError_t launch_l2l(const InterpTables &T, const float *Fparent, float *Fchild, int lparent, int p, int nrhs, cudaStream_t s)
{
    int64_t npar = (int64_t)1 << (3 * lparent);
#define L(P) return l2l_p<P>(T, Fparent, Fchild, npar, nrhs, s)
    BBFMM_DISPATCH_P(p, L)
#undef L
    return cudaSuccess;
}

} // namespace bbfmm
