// p2p.cu -- near-field stage (Sec. 2.2 item 4): launches of the kernels in
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
    } else if (nrhs > 1) {
        k_p2p_gemm<Kern, kGemmT><<<A.nchunks, gemm_threads(kGemmT), 0, s>>>(
            A.tpts, A.chunks, A.nt, A.spts, A.sig_rows, A.soff, A.ns, A.D, k, scale, nrhs, phi);
    } else {
        k_p2p<Kern><<<A.nchunks, kP2PThreads, 0, s>>>(A.tpts, A.chunks, A.nt, A.spts, A.sig, A.soff, A.ns, A.D, k,
                                                       scale, nrhs, phi);
    }
    return cudaGetLastError();
}

cudaError_t launch_p2p(const P2PArgs &A, int kernel, double ell, double h, int nrhs, float *phi_near,
                       cudaStream_t s)
{
    static_assert(kChunk <= 2 * kP2PThreads, "a work item holds at most two targets per thread");
    static_assert(kChunk <= kTPT * kP2PThreads, "a work item holds at most kTPT targets per thread");
    const double ln2 = 0.69314718055994530942;
    switch (kernel) {
    case BBFMM_K_INV_R:
        return p2p_launch(A, KInvR{0.f}, (float)(1.0 / h), nrhs, phi_near, s);
    case BBFMM_K_INV_R2:
        return p2p_launch(A, KInvR2{0.f}, (float)(1.0 / (h * h)), nrhs, phi_near, s);
    case BBFMM_K_EXP:
        return p2p_launch(A, KExp{(float)(h / (ell * ln2))}, 1.0f, nrhs, phi_near, s);
    case BBFMM_K_GAUSS:
        return p2p_launch(A, KGauss{(float)(h * h / (ell * ell * ln2))}, 1.0f, nrhs, phi_near, s);
    case BBFMM_K_TEST_POLY:
        return p2p_launch(A, KPoly{(float)h}, 1.0f, nrhs, phi_near, s);
    case BBFMM_K_TEST_CONST:
        return p2p_launch(A, KConst{0.f}, 1.0f, nrhs, phi_near, s);
    }
    if (kernel >= BBFMM_K_USER_FIRST)
        return launch_p2p_user(A, kernel, h, nrhs, phi_near, s);
    return cudaErrorInvalidValue;
}

} // namespace bbfmm
