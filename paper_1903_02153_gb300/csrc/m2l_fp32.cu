// m2l_fp32.cu -- far-field stage (Sec. 2.3 item 2) on the CUDA cores in FP32:
//   F~^alpha = scale_l * sum_{beta in I(alpha)} C^(t(alpha,beta)) M~^beta,
// with the compressed operators C^(t) = U^T K^(t) V (Sec. 2.5 "Fast M2L
// translation").  This is the plain-FP32 reference form of the stage; the
// tensor-core form lives in m2l_tc.cu.
//
// Structure: boxes of one level are split into the 8 octant classes o (the
// parity of the box coordinates).  For a target of class o the 189 members of
// I(alpha) sit at offsets t with t_d in [-2 - o_d, 3 - o_d] minus the 27
// neighbours, and the source of offset t is the box of octant (o + t) & 1 whose
// parent cell is the target's parent cell + u, u_d = floor((o_d + t_d) / 2) in
// {-1, 0, 1}.  A block computes a 64-row slice of F~ for a 4x4x4 block of parent
// cells (64 targets) of one class, looping over the 189 offsets; each offset is
// a 64 x r x 64 FP32 GEMM slice with the operator from L2 and the source
// vectors gathered from the parity-split M~ array.
#include "bbfmm_internal.h"

namespace bbfmm {

// per class: (operator index, source octant, packed u = (ux+1) | (uy+1)<<2 | (uz+1)<<4)
__constant__ int4 c_m2l_tab[8][kOffsetsPerClass];

static bool g_tab_ready = false;
static std::mutex g_tab_mu;

bool fill_m2l_table(int4 (*tab)[kOffsetsPerClass])
{
    for (int o = 0; o < 8; ++o) {
        int c[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
        int k = 0;
        for (int tz = -2 - c[2]; tz <= 3 - c[2]; ++tz)
            for (int ty = -2 - c[1]; ty <= 3 - c[1]; ++ty)
                for (int tx = -2 - c[0]; tx <= 3 - c[0]; ++tx) {
                    int idx = offset_index(tx, ty, tz);
                    if (idx < 0)
                        continue;
                    int t[3] = {tx, ty, tz}, q[3], u[3];
                    for (int d = 0; d < 3; ++d) {
                        q[d] = (c[d] + t[d]) & 1;
                        u[d] = (c[d] + t[d] - q[d]) / 2;
                    }
                    tab[o][k++] = make_int4(idx, q[0] | (q[1] << 1) | (q[2] << 2),
                                            (u[0] + 1) | ((u[1] + 1) << 2) | ((u[2] + 1) << 4), 0);
                }
        if (k != kOffsetsPerClass)
            return false;
    }
    return true;
}

static cudaError_t upload_m2l_table()
{
    std::lock_guard<std::mutex> g(g_tab_mu);
    if (g_tab_ready)
        return cudaSuccess;
    int4 tab[8][kOffsetsPerClass];
    if (!fill_m2l_table(tab))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_m2l_tab, tab, sizeof(tab));
    if (e == cudaSuccess)
        g_tab_ready = true;
    return e;
}

__global__ void __launch_bounds__(256) k_m2l_fp32(const float *__restrict__ Mt, const float *__restrict__ C,
                                                  float *__restrict__ Ft, int l, int r, int rp, int rows64,
                                                  int nrhs, int R, float scale)
{
    __shared__ __align__(16) float As[16][64]; // operator rows x k
    __shared__ __align__(16) float Bs[16][64]; // k x targets
    const int H = 1 << (l - 1);
    const int tpd = (H + 3) / 4; // tiles per dimension
    const int tile = blockIdx.x;
    const int X0 = 4 * (tile % tpd), Y0 = 4 * ((tile / tpd) % tpd), Z0 = 4 * (tile / (tpd * tpd));
    const int ot = blockIdx.y;
    const int nrt = rows64 / 64;
    const int row0 = 64 * (blockIdx.z % nrt);
    const int c = blockIdx.z / nrt;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int ld = tid >> 2, lk = (tid & 3) * 4; // loaders: row / target ld, k lk..lk+3
    const int bx = ld & 3, by = (ld >> 2) & 3, bz = ld >> 4;
    const int X = X0 + bx, Y = Y0 + by, Z = Z0 + bz;
    const bool tgt_ok = X < H && Y < H && Z < H;
    const int64_t zs = H + 2; // padded Z extent of M~

    float acc[4][4] = {};
    for (int e = 0; e < kOffsetsPerClass; ++e) {
        const int4 en = c_m2l_tab[ot][e];
        const int ux = (en.z & 3) - 1, uy = ((en.z >> 2) & 3) - 1, uz = ((en.z >> 4) & 3) - 1;
        const int sx = X + ux, sy = Y + uy, sz = Z + uz;
        const bool src_ok = tgt_ok && sx >= 0 && sx < H && sy >= 0 && sy < H && sz >= 0 && sz < H;
        const float *brow =
            Mt + ((((int64_t)en.y * zs + sz + 1) * H + sy) * H + sx) * (int64_t)R * rp + (int64_t)c * rp;
        const float *arow = C + ((int64_t)en.x * rows64 + row0 + ld) * rp;
        for (int k0 = 0; k0 < r; k0 += 16) {
            float4 a = *reinterpret_cast<const float4 *>(arow + k0 + lk);
            float4 b = src_ok ? *reinterpret_cast<const float4 *>(brow + k0 + lk) : make_float4(0, 0, 0, 0);
            As[lk + 0][ld] = a.x;
            As[lk + 1][ld] = a.y;
            As[lk + 2][ld] = a.z;
            As[lk + 3][ld] = a.w;
            Bs[lk + 0][ld] = b.x;
            Bs[lk + 1][ld] = b.y;
            Bs[lk + 2][ld] = b.z;
            Bs[lk + 3][ld] = b.w;
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                float aa[4] = {av.x, av.y, av.z, av.w}, bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        acc[i][j] += aa[i] * bb[j];
            }
            __syncthreads();
        }
    }
    // epilogue: thread (ty, tx) holds rows row0 + 4ty.. and targets 4tx..
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int b = tx * 4 + j;
        int Xb = X0 + (b & 3), Yb = Y0 + ((b >> 2) & 3), Zb = Z0 + (b >> 4);
        if (Xb >= H || Yb >= H || Zb >= H)
            continue;
        float *out = Ft + ((((int64_t)ot * H + Zb) * H + Yb) * H + Xb) * (int64_t)R * rp + (int64_t)c * rp;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int row = row0 + ty * 4 + i;
            if (row < r)
                out[row] = scale * acc[i][j];
        }
    }
}

cudaError_t m2l_fp32_init() { return upload_m2l_table(); }

cudaError_t launch_m2l_fp32(const float *Mt, const float *C, float *Ft, int l, int r, int rp, int rows64,
                            int nrhs, int R, float scale, cudaStream_t s)
{
    if (rp % 16 != 0 || rows64 % 64 != 0 || l < 2 || nrhs > R)
        return cudaErrorInvalidValue;
    cudaError_t e = upload_m2l_table();
    if (e != cudaSuccess)
        return e;
    int H = 1 << (l - 1);
    int tpd = (H + 3) / 4;
    dim3 grid((unsigned)(tpd * tpd * tpd), 8, (unsigned)((rows64 / 64) * nrhs));
    k_m2l_fp32<<<grid, 256, 0, s>>>(Mt, C, Ft, l, r, rp, rows64, nrhs, R, scale);
    return cudaGetLastError();
}

} // namespace bbfmm
