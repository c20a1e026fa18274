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

// one right-hand side: four points per thread (one 16-byte load of perm,
// four independent loads of sigma in flight, one 16-byte store), the last
// n % 4 points one per thread.  Same parameters as k_gather (nrhs and rows
// unused), so a captured matvec graph patches either the same way.
__global__ void k_gather4(const float *__restrict__ sigma, const int *__restrict__ perm, int64_t n, int,
                          float *__restrict__ out, float *)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, n4 = n / 4;
    if (q < n4) {
        const int4 j = reinterpret_cast<const int4 *>(perm)[q];
        reinterpret_cast<float4 *>(out)[q] = make_float4(sigma[j.x], sigma[j.y], sigma[j.z], sigma[j.w]);
    } else if (q < n4 + (n & 3)) {
        const int64_t i = 4 * n4 + (q - n4);
        out[i] = sigma[perm[i]];
    }
}

const void *gather_kernel() { return (const void *)k_gather; }
const void *gather4_kernel() { return (const void *)k_gather4; }

cudaError_t launch_gather_sigma(const float *sigma, const int *perm, int64_t n, int nrhs, float *out, float *rows,
                                cudaStream_t s)
{
    if (nrhs == 1 && !rows && reinterpret_cast<uintptr_t>(perm) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(out) % 16 == 0) {
        const int64_t threads = n / 4 + (n & 3);
        k_gather4<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(sigma, perm, n, 1, out, nullptr);
        return cudaGetLastError();
    }
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sigma, perm, n, nrhs, out, rows);
    return cudaGetLastError();
}

// 16-bit split: x * s = hi + lo, hi = round16(x s), lo = round16(x s - hi);
// s = 2^(13 - e) with 2^(e-1) < max|x| <= 2^e for FP16 (keeps hi below the
// FP16 range limit and lo away from the subnormals), s = 1 for BF16.  One
// launch for all levels: blockIdx.y picks the level.  A thread splits four
// consecutive values (one 16-byte load, two 8-byte stores); the launcher
// checks that every level's length is a multiple of 4 and its arrays aligned.
template <int FMT>
__device__ __forceinline__ unsigned split16(float v, unsigned &lo)
{
    if (FMT == 0) {
        const __half h = __float2half_rn(v);
        lo = __half_as_ushort(__float2half_rn(v - __half2float(h)));
        return __half_as_ushort(h);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
    return __bfloat16_as_ushort(h);
}

template <int FMT>
__global__ void k_split16_levels(const __grid_constant__ Split16Args A)
{
    const int l = A.lmin + blockIdx.y;
    const float4 *x = reinterpret_cast<const float4 *>(A.x[l]);
    const int64_t n4 = A.n[l] / 4;
    float s = 1.0f;
    if (FMT == 0) {
        const float mx = __uint_as_float(A.maxbits[l]);
        int e = 0;
        if (mx > 0.0f)
            frexpf(mx, &e);
        s = ldexpf(1.0f, 13 - e);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        A.scale[l] = s;
    uint2 *hi = reinterpret_cast<uint2 *>(A.hi[l]), *lo = reinterpret_cast<uint2 *>(A.lo[l]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        unsigned l0, l1, l2, l3;
        const unsigned h0 = split16<FMT>(v.x * s, l0), h1 = split16<FMT>(v.y * s, l1);
        const unsigned h2 = split16<FMT>(v.z * s, l2), h3 = split16<FMT>(v.w * s, l3);
        hi[i] = make_uint2(h0 | (h1 << 16), h2 | (h3 << 16));
        lo[i] = make_uint2(l0 | (l1 << 16), l2 | (l3 << 16));
    }
}

cudaError_t launch_split16_levels(const Split16Args &A, cudaStream_t s)
{
    if (A.lmin < 0 || A.lmax > kMaxDepth || A.lmin > A.lmax || (A.fmt != 0 && A.fmt != 1))
        return cudaErrorInvalidValue;
    int64_t most = 0;
    for (int l = A.lmin; l <= A.lmax; ++l) {
        if (A.n[l] % 4 != 0 || reinterpret_cast<uintptr_t>(A.x[l]) % 16 != 0 ||
            reinterpret_cast<uintptr_t>(A.hi[l]) % 8 != 0 || reinterpret_cast<uintptr_t>(A.lo[l]) % 8 != 0)
            return cudaErrorInvalidValue;
        most = A.n[l] / 4 > most ? A.n[l] / 4 : most;
    }
    int64_t blocks = (most + 255) / 256;
    blocks = blocks > 2048 ? 2048 : (blocks < 1 ? 1 : blocks);
    const dim3 grid((unsigned)blocks, (unsigned)(A.lmax - A.lmin + 1));
    if (A.fmt == 0)
        k_split16_levels<0><<<grid, 256, 0, s>>>(A);
    else
        k_split16_levels<1><<<grid, 256, 0, s>>>(A);
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
