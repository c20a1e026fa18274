// p2p.cu -- near-field stage (Sec. 2.3 item 4): launches of the kernels in
// p2p_kernels.cuh for the built-in kernel functions; user-supplied kernels
// run the same templates compiled at run time (user_kernel.cu).
#include "bbfmm_internal.h"
#include "p2p_kernels.cuh"

namespace bbfmm {

static_assert(kP2PChunk == kChunk, "near-field work items");
static_assert(kSymSlots == kSymSlotsHost, "slots of the symmetric near field");

template <class Kern>
static cudaError_t p2p_launch(const P2PArgs &A, Kern k, float scale, int nrhs, float *phi, cudaStream_t s)
{
    if (A.nchunks <= 0)
        return cudaSuccess;
    if (nrhs == 1 && A.slots) {
        k_p2p_sym<Kern><<<A.nchunks, kP2PThreads, 0, s>>>(A.spts, A.chunks, A.ns, A.sig, A.soff, A.D, k, scale, phi,
                                                           A.slots);
    } else if (nrhs == 1 && A.boxes) {
        if (A.nboxes > 0)
            k_p2p_box<Kern><<<A.nboxes, kP2PThreads, 0, s>>>(A.tpts, A.toff, A.boxes, A.nt, A.spts, A.sig, A.soff,
                                                               A.D, k, scale, phi);
    } else if (nrhs > 1) {
        k_p2p_gemm<Kern, kGemmT><<<A.nchunks, gemm_threads(kGemmT), 0, s>>>(
            A.tpts, A.chunks, A.nt, A.spts, A.sig_rows, A.soff, A.ns, A.D, k, scale, nrhs, phi);
    } else {
        k_p2p<Kern><<<A.nchunks, kP2PThreads, 0, s>>>(A.tpts, A.chunks, A.nt, A.spts, A.sig, A.soff, A.ns, A.D, k,
                                                       scale, nrhs, phi);
    }
    return cudaGetLastError();
}

// the near-field functor of a built-in kernel and the scale its sums are
// multiplied by (distances are in cell units; h = leaf box side)
template <class F>
static cudaError_t with_kernel(int kernel, double ell, double h, F &&f)
{
    const double ln2 = 0.69314718055994530942;
    switch (kernel) {
    case BBFMM_K_INV_R:
        return f(KInvR{0.f}, (float)(1.0 / h));
    case BBFMM_K_INV_R2:
        return f(KInvR2{0.f}, (float)(1.0 / (h * h)));
    case BBFMM_K_EXP:
        return f(KExp{(float)(h / (ell * ln2))}, 1.0f);
    case BBFMM_K_GAUSS:
        return f(KGauss{(float)(h * h / (ell * ell * ln2))}, 1.0f);
    case BBFMM_K_TEST_POLY:
        return f(KPoly{(float)h}, 1.0f);
    case BBFMM_K_TEST_CONST:
        return f(KConst{0.f}, 1.0f);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_p2p(const P2PArgs &A, int kernel, double ell, double h, int nrhs, float *phi_near,
                       cudaStream_t s)
{
    static_assert(kChunk <= 2 * kP2PThreads, "a work item holds at most two targets per thread");
    static_assert(kChunk <= kTPT * kP2PThreads, "a work item holds at most kTPT targets per thread");
    if (kernel >= BBFMM_K_USER_FIRST)
        return launch_p2p_user(A, kernel, h, nrhs, phi_near, s);
    return with_kernel(kernel, ell, h, [&](auto k, float scale) { return p2p_launch(A, k, scale, nrhs, phi_near, s); });
}

// K(d) of a built-in kernel in FP64, d = x - y in the caller's units; the
// r = 0 convention of the singular kernels as in the near field
struct ExactBuiltin {
    int kernel;
    double ell;
    __device__ double operator()(double d0, double d1, double d2) const
    {
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        switch (kernel) {
        case BBFMM_K_INV_R:
            return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
        case BBFMM_K_INV_R2:
            return r2 > 0.0 ? 1.0 / r2 : 0.0;
        case BBFMM_K_EXP:
            return exp(-sqrt(r2) / ell);
        case BBFMM_K_GAUSS:
            return exp(-r2 / (ell * ell));
        case BBFMM_K_TEST_POLY:
            return 1.0 + d0 - 2.0 * d1 * d2 + 3.0 * d0 * d0 * d1;
        default:
            return 1.0;
        }
    }
};

cudaError_t launch_close_pairs(const CloseArgs &A, int kernel, double ell, double h, bool fill, cudaStream_t s)
{
    if (A.nchunks <= 0)
        return cudaSuccess;
    if (kernel >= BBFMM_K_USER_FIRST)
        return launch_close_pairs_user(A, kernel, h, fill, s);
    CloseArgs B = A;
    const ExactBuiltin ex{kernel, ell};
    return with_kernel(kernel, ell, h, [&](auto k, float scale) {
        B.scale = scale;
        if (fill)
            k_close_pairs<decltype(k), ExactBuiltin, true><<<A.nchunks, kP2PThreads, 0, s>>>(B, k, ex);
        else
            k_close_pairs<decltype(k), ExactBuiltin, false><<<A.nchunks, kP2PThreads, 0, s>>>(B, k, ex);
        return cudaGetLastError();
    });
}

// the listed close pairs' corrections: target m of the list (tree index
// tgt[m]) adds sum over its entries e of c[e] sigma[src[e]] to each column of
// its near field, entries in list order
__global__ void k_near_fix(const int *__restrict__ tgt, const int *__restrict__ start, int ntgt,
                           const int *__restrict__ src, const float *__restrict__ c, const float *__restrict__ sig,
                           long long ns, long long nt, int nrhs, float *__restrict__ phi)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= ntgt)
        return;
    const int t = tgt[m], a = start[m], b = start[m + 1];
    for (int col = 0; col < nrhs; ++col) {
        const float *sg = sig + (long long)col * ns;
        float acc = 0.0f;
        for (int e = a; e < b; ++e)
            acc = fmaf(c[e], sg[src[e]], acc);
        phi[(long long)col * nt + t] += acc;
    }
}

cudaError_t launch_near_fix(const CloseList &L, int form, const float *sig, int64_t ns, int64_t nt, int nrhs,
                            float *phi, cudaStream_t s)
{
    if (L.ntgt <= 0)
        return cudaSuccess;
    const float *c = nrhs > 1 ? L.cm : form == 1 ? L.c1s : form == 2 ? L.c1b : L.c1;
    if (!c)
        return cudaErrorInvalidValue;
    k_near_fix<<<(L.ntgt + 127) / 128, 128, 0, s>>>(L.tgt, L.start, L.ntgt, L.src, c, sig, ns, nt, nrhs, phi);
    return cudaGetLastError();
}

} // namespace bbfmm
