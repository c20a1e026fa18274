// m2l_tc.cu -- far-field stage (Sec. 2.2 item 2) dispatch, and the operand
// splitting used by the split-precision tensor-core form.
#include <math.h>
#include <string.h>

#include "bbfmm_internal.h"

namespace bbfmm {

// Round an FP32 value to TF32 (10 explicit mantissa bits), round to nearest
// even, returned in an FP32 container with the low 13 bits clear.
static inline float to_tf32_host(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) { // finite
        uint32_t lsb = (b >> 13) & 1u;
        b += 0x0fffu + lsb;
        b &= 0xffffe000u;
    }
    float y;
    memcpy(&y, &b, 4);
    return y;
}

// hi = tf32(x), lo = tf32(x - hi): x = hi + lo up to 2^-22 relative
void split_tf32(const float *in, float *hi, float *lo, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        float h = to_tf32_host(in[i]);
        hi[i] = h;
        lo[i] = to_tf32_host(in[i] - h);
    }
}

cudaError_t launch_m2l(bbfmm_plan_impl *P, int l, int nrhs, cudaStream_t s)
{
    const DevOps &O = *P->ops;
    const int k = O.nlev == 1 ? 0 : l - 2;
    // homogeneous kernels: operators made for the leaf box, scaled by (h_l / h_D)^m
    float scale = 1.0f;
    if (O.host->hom_degree != 0)
        scale = (float)pow(2.0, (double)O.host->hom_degree * (P->D - l));
    return launch_m2l_fp32(P->lev[l].Mt, O.C[k], P->lev[l].Ft, l, O.r, O.rp, O.rows64, nrhs, scale, s);
}

} // namespace bbfmm
