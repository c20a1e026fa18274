// morton.cuh -- Morton order of the boxes of one level (x in bit 0 of every
// 3-bit group).  Self-contained (no includes): it is also compiled at run
// time, with the near-field kernels, for user-supplied kernels.
#pragma once

namespace bbfmm {

__host__ __device__ inline unsigned spread3(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ inline unsigned compact3(unsigned v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}
__host__ __device__ inline unsigned morton3(unsigned x, unsigned y, unsigned z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}
__host__ __device__ inline void demorton3(unsigned m, int &x, int &y, int &z)
{
    x = (int)compact3(m);
    y = (int)compact3(m >> 1);
    z = (int)compact3(m >> 2);
}

} // namespace bbfmm
