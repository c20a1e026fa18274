// p2p.cu -- near-field stage (Sec. 2.2 item 4):
//   phi_i += sum_{beta in N(alpha)} sum_{y_j in beta} K(x_i, y_j) sigma_j,
// N(alpha) = the up to 27 leaves adjacent to alpha, alpha included (Def. 2.1).
//
// Work item = up to kChunk consecutive targets of one leaf; one block of 128
// threads per item.  The block first gathers the neighbour leaves' sources
// into shared memory (all threads at once, coalesced, 2048 at a time) as
// float4 (x, y, z, sigma) with coordinates in the target leaf's cell units:
// y' = u_y + (cell_y - cell_x).  The offset is an exact small integer, so the
// FP32 difference u_x - y' only carries the rounding of u (|u| <= 1/2), not
// that of absolute coordinates.  Threads are (target, slice) pairs,
// thread = target + nt * slice: every slice walks a strided share of the
// staged sources for its target (all lanes of a warp read the same source, a
// shared-memory broadcast), and the slices of a target are summed in a fixed
// order at the end (deterministic).
// K at r = 0 follows the library's convention: 0 for 1/r and 1/r^2.
#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int kP2PThreads = 128;
constexpr int kStageSrc = 2048; // staged sources per pass (32 KB)

struct KInvR {
    float a; // unused
    __device__ float operator()(float dx, float dy, float dz) const
    {
        float r2 = dx * dx + dy * dy + dz * dz;
        return r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    }
};
struct KInvR2 {
    float a;
    __device__ float operator()(float dx, float dy, float dz) const
    {
        float r2 = dx * dx + dy * dy + dz * dz;
        return r2 > 0.0f ? 1.0f / r2 : 0.0f;
    }
};
struct KExp { // exp(-h r / ell) = 2^(-a r), a = h / (ell ln 2)
    float a;
    __device__ float operator()(float dx, float dy, float dz) const
    {
        float r2 = dx * dx + dy * dy + dz * dz;
        return exp2f(-a * sqrtf(r2));
    }
};
struct KGauss { // exp(-(h r / ell)^2) = 2^(-a r^2), a = h^2 / (ell^2 ln 2)
    float a;
    __device__ float operator()(float dx, float dy, float dz) const
    {
        float r2 = dx * dx + dy * dy + dz * dz;
        return exp2f(-a * r2);
    }
};
struct KPoly { // q(d) with d = h * (x - y) in physical units
    float a; // h
    __device__ float operator()(float dx, float dy, float dz) const
    {
        float d0 = a * dx, d1 = a * dy, d2 = a * dz;
        return 1.0f + d0 - 2.0f * d1 * d2 + 3.0f * d0 * d0 * d1;
    }
};
struct KConst {
    float a;
    __device__ float operator()(float, float, float) const { return 1.0f; }
};

template <class Kern>
__global__ void __launch_bounds__(kP2PThreads)
    k_p2p(const float4 *__restrict__ pts, const float *__restrict__ sig, const int *__restrict__ off,
          const int4 *__restrict__ chunks, int nchunks, int64_t n, int D, Kern kern, float scale, int nrhs,
          float *__restrict__ phi)
{
    __shared__ float4 stage[kStageSrc];
    __shared__ int nb_start[28], nb_pre[28];
    __shared__ float4 nb_delta[27];
    __shared__ float red[kP2PThreads];
    const int tid = threadIdx.x;
    const int4 ch = chunks[blockIdx.x];
    const int nt = ch.z;
    const int S = kP2PThreads / nt; // slices per target (>= 1)
    const int t = tid % nt, slice = tid / nt;
    const bool active = slice < S;
    int ax, ay, az;
    demorton3((uint32_t)ch.x, ax, ay, az);
    const int nside = 1 << D;

    // neighbour leaves: start, count (prefix) and cell offset
    if (tid < 32) {
        int cnt = 0, start = 0;
        if (tid < 27) {
            const int dx = tid % 3 - 1, dy = (tid / 3) % 3 - 1, dz = tid / 9 - 1;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < nside && by < nside && bz < nside) {
                const uint32_t nm = morton3((uint32_t)bx, (uint32_t)by, (uint32_t)bz);
                start = off[nm];
                cnt = off[nm + 1] - start;
            }
            nb_start[tid] = start;
            nb_delta[tid] = make_float4((float)dx, (float)dy, (float)dz, 0.0f);
        }
        int incl = cnt; // inclusive warp scan of the counts
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o)
                incl += v;
        }
        if (tid < 28)
            nb_pre[tid] = incl - cnt; // exclusive prefix; nb_pre[27] = total
    }
    __syncthreads();
    const int ns = nb_pre[27];
    const float4 xt = pts[ch.y + (active ? t : 0)];

    for (int c = 0; c < nrhs; ++c) {
        const float *sg = sig + (int64_t)c * n;
        float acc = 0.0f;
        for (int base = 0; base < ns; base += kStageSrc) {
            const int cnt = min(kStageSrc, ns - base);
            for (int g = tid; g < cnt; g += kP2PThreads) {
                const int gg = base + g;
                int k = 0; // neighbour holding source gg: largest k with nb_pre[k] <= gg
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (k + step < 27 && nb_pre[k + step] <= gg)
                        k += step;
                const int src = nb_start[k] + (gg - nb_pre[k]);
                const float4 u = pts[src];
                const float4 d = nb_delta[k];
                stage[g] = make_float4(u.x + d.x, u.y + d.y, u.z + d.z, sg[src]);
            }
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int j = slice; j < cnt; j += S) {
                    const float4 q = stage[j];
                    acc += kern(xt.x - q.x, xt.y - q.y, xt.z - q.z) * q.w;
                }
            }
            __syncthreads();
        }
        red[tid] = active ? acc : 0.0f;
        __syncthreads();
        if (tid < nt) {
            float sum = 0.0f;
            for (int q = 0; q < S; ++q)
                sum += red[tid + q * nt];
            phi[(int64_t)c * n + ch.y + tid] = scale * sum;
        }
        __syncthreads();
    }
}

template <class Kern>
static cudaError_t p2p_launch(const float4 *pts, const float *sig, const int *off, const int4 *chunks, int nchunks,
                              int64_t n, int D, Kern k, float scale, int nrhs, float *phi, cudaStream_t s)
{
    if (nchunks <= 0)
        return cudaSuccess;
    k_p2p<Kern><<<nchunks, kP2PThreads, 0, s>>>(pts, sig, off, chunks, nchunks, n, D, k, scale, nrhs, phi);
    return cudaGetLastError();
}

cudaError_t launch_p2p(const float4 *pts, const float *sig, const int *leaf_off, const int4 *chunks, int nchunks,
                       int64_t n, int D, int kernel, double ell, double h, int nrhs, float *phi_near,
                       cudaStream_t s)
{
    static_assert(kChunk <= kP2PThreads, "a work item holds at most one target per thread");
    const double ln2 = 0.69314718055994530942;
    switch (kernel) {
    case BBFMM_K_INV_R:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KInvR{0.f}, (float)(1.0 / h), nrhs,
                          phi_near, s);
    case BBFMM_K_INV_R2:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KInvR2{0.f}, (float)(1.0 / (h * h)), nrhs,
                          phi_near, s);
    case BBFMM_K_EXP:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KExp{(float)(h / (ell * ln2))}, 1.0f, nrhs,
                          phi_near, s);
    case BBFMM_K_GAUSS:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KGauss{(float)(h * h / (ell * ell * ln2))},
                          1.0f, nrhs, phi_near, s);
    case BBFMM_K_TEST_POLY:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KPoly{(float)h}, 1.0f, nrhs, phi_near, s);
    case BBFMM_K_TEST_CONST:
        return p2p_launch(pts, sig, leaf_off, chunks, nchunks, n, D, KConst{0.f}, 1.0f, nrhs, phi_near, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace bbfmm
