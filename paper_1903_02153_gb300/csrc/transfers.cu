// transfers.cu -- the element-wise stages around the black-box FMM passes:
// the gather of the weights into tree order, the 16-bit split of the
// compressed multipole coefficients for the tensor-core M2L (Sec. 2.5 "Fast
// M2L translation" run as split-precision products), and the final combine /
// un-permute of near and far fields.  The interpolation tables the passes use
// are made here from the host operators.
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

// ---------------------------------------------------------------------------
// out: tree order, column-major (n x nrhs); rows (if not null): the same
// values row-major (nrhs per point), the layout of the several-RHS near field
__global__ void k_gather(const float *__restrict__ sigma, const int *__restrict__ perm, int64_t n, int nrhs,
                         float *__restrict__ out, float *__restrict__ rows)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = perm[i];
    for (int c = 0; c < nrhs; ++c) {
        const float v = sigma[(int64_t)c * n + j];
        out[(int64_t)c * n + i] = v;
        if (rows)
            rows[i * nrhs + c] = v;
    }
}

const void *gather_kernel() { return (const void *)k_gather; }

cudaError_t launch_gather_sigma(const float *sigma, const int *perm, int64_t n, int nrhs, float *out, float *rows,
                                cudaStream_t s)
{
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sigma, perm, n, nrhs, out, rows);
    return cudaGetLastError();
}

// 16-bit split: x * s = hi + lo, hi = round16(x s), lo = round16(x s - hi);
// s = 2^(13 - e) with 2^(e-1) < max|x| <= 2^e for FP16 (keeps hi below the
// FP16 range limit and lo away from the subnormals), s = 1 for BF16.  One
// launch for all levels: blockIdx.y picks the level.
__global__ void k_split16_levels(const __grid_constant__ Split16Args A)
{
    const int l = A.lmin + blockIdx.y;
    const float *x = A.x[l];
    const int64_t n = A.n[l];
    float s = 1.0f;
    if (A.fmt == 0) {
        const float mx = __uint_as_float(A.maxbits[l]);
        int e = 0;
        if (mx > 0.0f)
            frexpf(mx, &e);
        s = ldexpf(1.0f, 13 - e);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        A.scale[l] = s;
    uint16_t *hi = A.hi[l], *lo = A.lo[l];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i] * s;
        if (A.fmt == 0) {
            const __half h = __float2half_rn(v);
            hi[i] = __half_as_ushort(h);
            lo[i] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[i] = __bfloat16_as_ushort(h);
            lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
        }
    }
}

cudaError_t launch_split16_levels(const Split16Args &A, cudaStream_t s)
{
    if (A.lmin < 0 || A.lmax > kMaxDepth || A.lmin > A.lmax || (A.fmt != 0 && A.fmt != 1))
        return cudaErrorInvalidValue;
    int64_t most = 0;
    for (int l = A.lmin; l <= A.lmax; ++l)
        most = A.n[l] > most ? A.n[l] : most;
    int64_t blocks = (most + 255) / 256;
    blocks = blocks > 2048 ? 2048 : (blocks < 1 ? 1 : blocks);
    k_split16_levels<<<dim3((unsigned)blocks, (unsigned)(A.lmax - A.lmin + 1)), 256, 0, s>>>(A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// slots (symmetric near field, one RHS): the 13 column sums a point receives
// from its backward neighbour leaves, added in slot order
__global__ void k_combine(const float *__restrict__ far, const float *__restrict__ near,
                          const float *__restrict__ slots, const int *__restrict__ perm, int64_t n, int nrhs,
                          float *__restrict__ phi)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = perm[i];
    for (int c = 0; c < nrhs; ++c) {
        float v = near[(int64_t)c * n + i];
        if (slots)
            for (int q = 0; q < 13; ++q)
                v += slots[q * n + i];
        if (far)
            v += far[(int64_t)c * n + i];
        phi[(int64_t)c * n + j] = v;
    }
}

const void *combine_kernel() { return (const void *)k_combine; }

cudaError_t launch_combine(const float *phi_far, const float *phi_near, const float *slots, const int *perm,
                           int64_t n, int nrhs, float *phi, cudaStream_t s)
{
    k_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi_far, phi_near, slots, perm, n, nrhs, phi);
    return cudaGetLastError();
}

} // namespace bbfmm
