// eig.cu -- dense kernels of the randomized eigen-decomposition of a kernel
// matrix (the randomized PCA application of Sec. 4.3): tall-skinny Gram
// products A^T B of n x m blocks and right products Y T by small m x m'
// matrices.  The matvecs with the kernel matrix are the library's own
// bbfmm_matvec; the m x m eigenproblems are solved on the host.
#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int kGramTile = 32;    // output tile of one block
constexpr int kGramRows = 64;    // rows staged in shared memory per step
constexpr int kGramFlush = 1024; // rows summed in FP32 before adding to FP64

// partial[split][a][b] = sum over the split's rows i of A[i + a n] B[i + b n]
// (column-major n x m blocks).  Block = one 32 x 32 tile of (a, b) and one
// row split; thread = 2 x 2 outputs.  Products are summed in FP32 over
// kGramFlush rows, then added into FP64.
__global__ void __launch_bounds__(256) k_gram(const float *__restrict__ A, const float *__restrict__ B, int64_t n,
                                              int m, int64_t rows_per_split, double *__restrict__ partial)
{
    __shared__ float sA[kGramRows][kGramTile + 1], sB[kGramRows][kGramTile + 1];
    const int ntile = (m + kGramTile - 1) / kGramTile;
    const int ta = blockIdx.x % ntile, tb = blockIdx.x / ntile;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t r1 = r0 + rows_per_split < n ? r0 + rows_per_split : n;
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    double accd[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    int since = 0;
    for (int64_t base = r0; base < r1; base += kGramRows) {
        for (int q = t; q < kGramRows * kGramTile; q += 256) {
            const int rr = q % kGramRows, cc = q / kGramRows; // consecutive threads, consecutive rows
            const int64_t i = base + rr;
            const int a = ta * kGramTile + cc, b = tb * kGramTile + cc;
            sA[rr][cc] = (i < r1 && a < m) ? A[i + (int64_t)a * n] : 0.0f;
            sB[rr][cc] = (i < r1 && b < m) ? B[i + (int64_t)b * n] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < kGramRows; ++rr) {
            const float a0 = sA[rr][2 * ty], a1 = sA[rr][2 * ty + 1];
            const float b0 = sB[rr][2 * tx], b1 = sB[rr][2 * tx + 1];
            acc[0][0] += a0 * b0;
            acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0;
            acc[1][1] += a1 * b1;
        }
        __syncthreads();
        since += kGramRows;
        if (since >= kGramFlush) {
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    accd[u][v] += (double)acc[u][v];
                    acc[u][v] = 0.0f;
                }
            since = 0;
        }
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            accd[u][v] += (double)acc[u][v];
            const int a = ta * kGramTile + 2 * ty + u, b = tb * kGramTile + 2 * tx + v;
            if (a < m && b < m)
                partial[((int64_t)blockIdx.y * m + a) * m + b] = accd[u][v];
        }
}

// out[i + c n] = sum_a Y[i + a n] T[a + c m], c < mo (T column-major m x mo,
// held in shared memory); thread = one row, 16 output columns at a time
__global__ void __launch_bounds__(256) k_rmul(const float *__restrict__ Y, int64_t n, int m,
                                              const float *__restrict__ T, int mo, float *__restrict__ out)
{
    extern __shared__ float sT[];
    for (int q = threadIdx.x; q < m * mo; q += blockDim.x)
        sT[q] = T[q];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    for (int c0 = 0; c0 < mo; c0 += 16) {
        float acc[16];
#pragma unroll
        for (int cc = 0; cc < 16; ++cc)
            acc[cc] = 0.0f;
        for (int a = 0; a < m; ++a) {
            const float y = Y[i + (int64_t)a * n];
#pragma unroll
            for (int cc = 0; cc < 16; ++cc)
                if (c0 + cc < mo)
                    acc[cc] += y * sT[a + (c0 + cc) * m];
        }
#pragma unroll
        for (int cc = 0; cc < 16; ++cc)
            if (c0 + cc < mo)
                out[i + (int64_t)(c0 + cc) * n] = acc[cc];
    }
}

int gram_splits(int64_t n)
{
    int64_t s = (n + 4095) / 4096; // at least 4096 rows per split
    return (int)(s > 64 ? 64 : (s < 1 ? 1 : s));
}

cudaError_t launch_gram(const float *A, const float *B, int64_t n, int m, double *partial, int splits, cudaStream_t s)
{
    if (m < 1 || splits < 1)
        return cudaErrorInvalidValue;
    const int ntile = (m + kGramTile - 1) / kGramTile;
    const int64_t rows = (n + splits - 1) / splits;
    k_gram<<<dim3((unsigned)(ntile * ntile), (unsigned)splits), 256, 0, s>>>(A, B, n, m, rows, partial);
    return cudaGetLastError();
}

cudaError_t launch_rmul(const float *Y, int64_t n, int m, const float *T, int mo, float *out, cudaStream_t s)
{
    if (m < 1 || mo < 1 || Y == out)
        return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)m * mo;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_rmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    k_rmul<<<(unsigned)((n + 255) / 256), 256, smem, s>>>(Y, n, m, T, mo, out);
    return cudaGetLastError();
}

} // namespace bbfmm
