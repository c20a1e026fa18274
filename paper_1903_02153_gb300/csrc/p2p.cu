// p2p.cu -- near-field stage (Sec. 2.2 item 4):
//   phi_i += sum_{beta in N(alpha)} sum_{y_j in beta} K(x_i, y_j) sigma_j,
// N(alpha) = the up to 27 leaves adjacent to alpha, alpha included (Def. 2.1).
//
// Work item = a chunk of <= 32 consecutive targets of one leaf; one warp per
// chunk.  With nt targets in the chunk the warp's lanes form S = floor(32/nt)
// slices per target (lane = target + nt * slice), so small leaves still keep
// the lanes busy; the slices are summed through shared memory at the end.
// Sources of the 27 neighbour leaves are staged, 32 at a time per leaf, in a
// per-warp shared-memory ring as float4 (x, y, z, sigma) with coordinates in
// the target leaf's cell units: y' = u_y + (cell_y - cell_x).  The offset is an
// exact small integer, so the FP32 difference u_x - y' loses no more than the
// rounding of u (|u| <= 1/2) instead of that of absolute coordinates.
// K at r = 0 follows the library's convention: 0 for 1/r and 1/r^2.
#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int kP2PWarps = 4;
constexpr int kStage = 128; // staged sources per warp

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
__global__ void __launch_bounds__(32 * kP2PWarps)
    k_p2p(const float4 *__restrict__ pts, const float *__restrict__ sig, const int *__restrict__ off,
          const int4 *__restrict__ chunks, int nchunks, int64_t n, int D, Kern kern, float scale, int nrhs,
          float *__restrict__ phi)
{
    __shared__ float4 stage[kP2PWarps][kStage];
    __shared__ float red[kP2PWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kP2PWarps + w;
    if (item >= nchunks)
        return;
    const int4 ch = chunks[item];
    const int nt = ch.z;
    const int S = 32 / nt;
    const int t = lane % nt, slice = lane / nt;
    const bool active = slice < S;
    const float4 xt = pts[ch.y + t];
    int ax, ay, az;
    demorton3((uint32_t)ch.x, ax, ay, az);
    const int nside = 1 << D;

    for (int c = 0; c < nrhs; ++c) {
        const float *sg = sig + (int64_t)c * n;
        float acc = 0.0f;
        int fill = 0;
        for (int k = 0; k < 27; ++k) {
            const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx < 0 || by < 0 || bz < 0 || bx >= nside || by >= nside || bz >= nside)
                continue;
            const uint32_t nm = morton3((uint32_t)bx, (uint32_t)by, (uint32_t)bz);
            const int s0 = off[nm], s1 = off[nm + 1];
            for (int o = s0; o < s1; o += 32) {
                const int cnt = min(32, s1 - o);
                if (lane < cnt) {
                    float4 u = pts[o + lane];
                    stage[w][fill + lane] = make_float4(u.x + (float)dx, u.y + (float)dy, u.z + (float)dz,
                                                        sg[o + lane]);
                }
                fill += cnt;
                if (fill > kStage - 32) {
                    __syncwarp();
                    if (active)
                        for (int j = slice; j < fill; j += S) {
                            float4 q = stage[w][j];
                            acc += kern(xt.x - q.x, xt.y - q.y, xt.z - q.z) * q.w;
                        }
                    __syncwarp();
                    fill = 0;
                }
            }
        }
        __syncwarp();
        if (active)
            for (int j = slice; j < fill; j += S) {
                float4 q = stage[w][j];
                acc += kern(xt.x - q.x, xt.y - q.y, xt.z - q.z) * q.w;
            }
        red[w][lane] = active ? acc : 0.0f;
        __syncwarp();
        if (lane < nt) {
            float sum = 0.0f;
            for (int q = 0; q < S; ++q)
                sum += red[w][lane + q * nt];
            phi[(int64_t)c * n + ch.y + lane] = scale * sum;
        }
        __syncwarp();
    }
}

template <class Kern>
static cudaError_t p2p_launch(const float4 *pts, const float *sig, const int *off, const int4 *chunks, int nchunks,
                              int64_t n, int D, Kern k, float scale, int nrhs, float *phi, cudaStream_t s)
{
    if (nchunks <= 0)
        return cudaSuccess;
    unsigned blocks = (unsigned)((nchunks + kP2PWarps - 1) / kP2PWarps);
    k_p2p<Kern><<<blocks, 32 * kP2PWarps, 0, s>>>(pts, sig, off, chunks, nchunks, n, D, k, scale, nrhs, phi);
    return cudaGetLastError();
}

cudaError_t launch_p2p(const float4 *pts, const float *sig, const int *leaf_off, const int4 *chunks, int nchunks,
                       int64_t n, int D, int kernel, double ell, double h, int nrhs, float *phi_near,
                       cudaStream_t s)
{
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
