// m2l_fft.cu -- far-field stage (Sec. 2.2 item 2) with equally spaced nodes
// (Sec. 2.2 node sets): the M2L operator between two boxes is block-Toeplitz,
// K^(t)_ij = c_t(i - j) per axis, so (Sec. 2.5 "Fast M2L translation")
//     F^alpha = sum_{beta in I(alpha)} K^(t) M^beta
// becomes, with n = 2p - 1 point DFTs (n keeps the 2p - 1 index differences
// apart, so the circular convolution equals the Toeplitz product),
//     F^^alpha(w) = sum_{beta in I(alpha)} K^_t(w) M^^beta(w),
//     F^alpha     = the first p^3 entries of IDFT(F^^alpha).
// Three kernels per level:
//   k_fft_fwd   per box: real-to-complex DFT of its p^3 coefficients zero-
//               padded to n^3 (x, then y, then z; only w_x < p is kept, the
//               other half is the complex conjugate), written frequency-major
//               onto a box grid with a zero halo of 3 boxes.
//   k_fft_m2l   per frequency w and tile of 8^3 target boxes: the 189-term
//               sum over the interaction list, a stencil on the box grid.
//               Warp = one octant class (its 189 offsets are warp-uniform),
//               thread = two targets adjacent in x, packed two-lane FP32 FMA.
//   k_fft_inv   per box: the inverse DFT (z, y, then x with the conjugate
//               half restored), only the p^3 outputs that are kept.
// The kernel spectra K^_t (host, FP64 -> FP32) already carry the 1 / n^3 of
// the inverse transform.  FP32 throughout; the tensor cores have no use here
// (the Fourier-domain product is diagonal).
#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int kFftMaxN = 2 * kMaxP - 1;
constexpr int kFftTile = 8;        // target tile edge (boxes); 4 on level 2
constexpr int kFftThreads = 256;   // 8 warps = 8 octant classes
constexpr int kFftBoxes = 16;      // most boxes per block of the forward / inverse DFT
constexpr int kFftSmem = 96 * 1024; // shared memory budget of the DFT blocks
constexpr int kFftWPerBlock = 16;  // frequencies per block of the stencil

struct FftArgs {
    float2 tw[kFftMaxN]; // (cos, sin)(2 pi k / n)
    int p, n, nw, p3, rp, R, nrhs;
    int l, S, G, H;      // level, boxes per axis, M^ grid edge (S + 6), parent cells per axis (S / 2)
    int T, Ts, tsel;     // tile edge, halo edge per parity (T / 2 + 3), tap table (0: T = 8, 1: T = 4)
    int nbf, nbi;        // boxes per block of the forward / inverse DFT
    const float *Mt;     // M~ = M (no compression), parity-split rows of rp floats
    float *Ft;           // F~ = F, slice 0
    float2 *Mhat, *Fhat;
    const float2 *khat;  // [w][316]
    const int4 *tiles;   // the level's active tiles
    float scale;         // homogeneous kernels: (h_l / h_D)^m
    int *status;         // device status word (kStatusBounds on a tile outside the level)
};

// per tap table (2 tile sizes x 8 octant classes x 189 offsets): x = offset
// of the source from the target in the parity-split halo tile (in float4
// pairs), y = offset index 0..315 (the kernel spectrum's column)
__constant__ int2 c_fft_tap[2][8][kOffsetsPerClass];

// ---------------------------------------------------------------------------
// forward DFT: block = A.nbf consecutive boxes (lexicographic) x 1 RHS
__global__ void __launch_bounds__(128) k_fft_fwd(const __grid_constant__ FftArgs A)
{
    extern __shared__ float2 fsm[];
    const int p = A.p, n = A.n, p3 = A.p3;
    const int c = blockIdx.y;
    const int64_t nbox = (int64_t)A.S * A.S * A.S;
    const int NB = A.nbf;
    const int64_t b0 = (int64_t)blockIdx.x * NB;
    float *sM = reinterpret_cast<float *>(fsm); // [box][p3]
    float2 *sA = fsm + (NB * p3 + 1) / 2;       // [box][z][y][wx]
    float2 *sB = sA + NB * p3;                  // [box][z][wy][wx]
    __shared__ int sRow[kFftBoxes];
    const int t = threadIdx.x;
    if (t < NB) {
        const int64_t b = b0 + t;
        int row = -1;
        if (b < nbox) {
            const int x = (int)(b % A.S), y = (int)((b / A.S) % A.S), z = (int)(b / ((int64_t)A.S * A.S));
            row = (int)parity_row(x, y, z, c, A.H, 1, A.R);
        }
        sRow[t] = row;
    }
    __syncthreads();
    for (int q = t; q < NB * p3; q += blockDim.x) {
        const int bx = q / p3, k = q - bx * p3;
        const int row = sRow[bx];
        sM[q] = row >= 0 ? __ldg(A.Mt + (int64_t)row * A.rp + k) : 0.0f;
    }
    __syncthreads();
    // x: A(wx; y, z) = sum_x M(x, y, z) e^{-2 pi i wx x / n}, wx < p
    for (int q = t; q < NB * p3; q += blockDim.x) {
        const int bx = q / p3, r = q - bx * p3;
        const int wx = r % p, yz = r / p;
        const float *m = sM + bx * p3 + yz * p;
        float re = 0.0f, im = 0.0f;
        int k = 0;
        for (int x = 0; x < p; ++x) {
            const float2 w = A.tw[k];
            re += m[x] * w.x;
            im -= m[x] * w.y;
            k += wx;
            k -= k >= n ? n : 0;
        }
        sA[q] = make_float2(re, im);
    }
    __syncthreads();
    // y: B(wx, wy; z) = sum_y A(wx; y, z) e^{-2 pi i wy y / n}
    const int pnp = p * n * p;
    for (int q = t; q < NB * pnp; q += blockDim.x) {
        const int bx = q / pnp, r = q - bx * pnp;
        const int wx = r % p, wy = (r / p) % n, z = r / (p * n);
        const float2 *a = sA + bx * p3 + z * p * p + wx;
        float re = 0.0f, im = 0.0f;
        int k = 0;
        for (int y = 0; y < p; ++y) {
            const float2 v = a[y * p], w = A.tw[k];
            re += v.x * w.x + v.y * w.y;
            im += v.y * w.x - v.x * w.y;
            k += wy;
            k -= k >= n ? n : 0;
        }
        sB[q] = make_float2(re, im);
    }
    __syncthreads();
    // z, and the store: consecutive threads take consecutive boxes of one
    // frequency (coalesced rows of the M^ grid)
    const int64_t G = A.G, plane = G * G * G;
    for (int q = t; q < NB * A.nw; q += blockDim.x) {
        const int bx = q % NB, w = q / NB;
        const int64_t b = b0 + bx;
        if (b >= nbox)
            continue;
        const int wx = w % p, wy = (w / p) % n, wz = w / (p * n);
        const float2 *bb = sB + bx * pnp + wy * p + wx;
        float re = 0.0f, im = 0.0f;
        int k = 0;
        for (int z = 0; z < p; ++z) {
            const float2 v = bb[z * n * p], tw = A.tw[k];
            re += v.x * tw.x + v.y * tw.y;
            im += v.y * tw.x - v.x * tw.y;
            k += wz;
            k -= k >= n ? n : 0;
        }
        const int x = (int)(b % A.S), y = (int)((b / A.S) % A.S), z = (int)(b / ((int64_t)A.S * A.S));
        A.Mhat[((int64_t)w * A.R + c) * plane + ((z + 3) * G + (y + 3)) * G + (x + 3)] = make_float2(re, im);
    }
}

// ---------------------------------------------------------------------------
// Fourier-domain M2L: block = one active tile x kFftWPerBlock frequencies x 1 RHS
__global__ void __launch_bounds__(kFftThreads) k_fft_m2l(const __grid_constant__ FftArgs A)
{
    extern __shared__ float4 sC[]; // [8 parity planes][Ts^3]: (re[i], re[i+1], im[i], im[i+1])
    __shared__ float4 sK[kNumOffsets]; // (re, re, im, im) of K^_t(w)
    const int T = A.T, Ts = A.Ts, Ts3 = Ts * Ts * Ts, E = T + 6;
    const int c = blockIdx.z;
    const int4 tile = A.tiles[blockIdx.x];
    const int x0 = tile.x * T, y0 = tile.y * T, z0 = tile.z * T;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (tile.x < 0 || tile.y < 0 || tile.z < 0 || x0 + T > A.S || y0 + T > A.S || z0 + T > A.S) {
        if (t == 0)
            atomicOr(A.status, kStatusBounds);
        return; // block-uniform: no barrier is skipped by part of the block
    }
    // this thread's targets: class = warp, pair (X, X + 1) of class cells
    const int Tc = T / 2, npair = Tc / 2;
    const int xp = lane % npair, Y = (lane / npair) % Tc, Z = lane / (npair * Tc);
    const bool active = Z < Tc;
    const int X = 2 * xp;
    const int sbase = X + Ts * (Y + Ts * Z);
    const int2 *tap = c_fft_tap[A.tsel][warp];
    const int64_t G = A.G, plane = G * G * G;
    const int w0 = blockIdx.y * kFftWPerBlock, w1 = min(A.nw, w0 + kFftWPerBlock);
    // output: parity-split F^ [w][c][oct][H][H][H], the pair adjacent in x
    const int px = warp & 1, py = (warp >> 1) & 1, pz = warp >> 2;
    const int64_t H = A.H, nb = 8 * H * H * H;
    const int64_t orow = (((int64_t)warp * H + (z0 / 2 + Z)) * H + (y0 / 2 + Y)) * H + (x0 / 2 + X);
    (void)px;
    (void)py;
    (void)pz;
    float *sCf = reinterpret_cast<float *>(sC);
    for (int w = w0; w < w1; ++w) {
        __syncthreads(); // the previous frequency's reads are done
        for (int u = t; u < kNumOffsets; u += kFftThreads) {
            const float2 k = __ldg(A.khat + (int64_t)w * kNumOffsets + u);
            sK[u] = make_float4(k.x, k.x, k.y, k.y);
        }
        // halo tile of M^(w): box (x0 - 3 + hx, ...) sits at grid (x0 + hx, ...)
        const float2 *src = A.Mhat + ((int64_t)w * A.R + c) * plane;
        for (int q = t; q < E * E * E; q += kFftThreads) {
            const int hx = q % E, hy = (q / E) % E, hz = q / (E * E);
            const float2 v = __ldg(src + ((int64_t)(z0 + hz) * G + (y0 + hy)) * G + (x0 + hx));
            const int i = ((hx & 1) | ((hy & 1) << 1) | ((hz & 1) << 2)) * Ts3 + ((hz >> 1) * Ts + (hy >> 1)) * Ts +
                          (hx >> 1);
            sCf[4 * i] = v.x;     // first of the pair starting at i
            sCf[4 * i + 2] = v.y;
            if ((hx >> 1) > 0) {  // second of the pair starting at i - 1
                sCf[4 * (i - 1) + 1] = v.x;
                sCf[4 * (i - 1) + 3] = v.y;
            }
        }
        __syncthreads();
        if (active) {
            // re = sum m.re k.re - m.im k.im, im = sum m.re k.im + m.im k.re,
            // as four packed sums (P, Q, R, S) over the two targets
            float2 P2 = make_float2(0.0f, 0.0f), Q2 = P2, R2 = P2, S2 = P2;
#pragma unroll 7
            for (int j = 0; j < kOffsetsPerClass; ++j) {
                const int2 e = tap[j];
                const float4 m = sC[sbase + e.x];
                const float4 k = sK[e.y];
                const float2 mre = make_float2(m.x, m.y), mim = make_float2(m.z, m.w);
                const float2 kre = make_float2(k.x, k.y), kim = make_float2(k.z, k.w);
                P2 = __ffma2_rn(mre, kre, P2);
                Q2 = __ffma2_rn(mim, kim, Q2);
                R2 = __ffma2_rn(mre, kim, R2);
                S2 = __ffma2_rn(mim, kre, S2);
            }
            float4 o = make_float4(P2.x - Q2.x, R2.x + S2.x, P2.y - Q2.y, R2.y + S2.y);
            *reinterpret_cast<float4 *>(A.Fhat + ((int64_t)w * A.R + c) * nb + orow) = o;
        }
    }
}

// ---------------------------------------------------------------------------
// inverse DFT: block = A.nbi boxes of an active tile x 1 RHS
__global__ void __launch_bounds__(128) k_fft_inv(const __grid_constant__ FftArgs A)
{
    extern __shared__ float2 fsm[];
    const int p = A.p, n = A.n, p3 = A.p3, nw = A.nw, pnp = p * n * p;
    const int c = blockIdx.z;
    const int T = A.T, Tc = T / 2;
    const int per_tile = T * T * T;
    const int4 tile = A.tiles[blockIdx.x];
    const int t = threadIdx.x, NB = A.nbi;
    if (tile.x < 0 || tile.y < 0 || tile.z < 0 || (tile.x + 1) * T > A.S || (tile.y + 1) * T > A.S ||
        (tile.z + 1) * T > A.S) {
        if (t == 0)
            atomicOr(A.status, kStatusBounds);
        return;
    }
    float2 *sG = fsm;           // [box][w]
    float2 *sBz = sG + NB * nw; // [box][z][wy][wx]
    float2 *sAy = sG;           // [box][z][y][wx] (over sG once it is used)
    __shared__ int64_t sIdx[kFftBoxes];
    __shared__ int sRow[kFftBoxes];
    const int64_t H = A.H, nb = 8 * H * H * H;
    if (t < NB) {
        // box q of the tile in parity-split order: class, then Z, Y, X
        const int q = blockIdx.y * NB + t;
        const int Tc3 = Tc * Tc * Tc;
        const int oct = q / Tc3, r = q - oct * Tc3;
        const int X = r % Tc, Y = (r / Tc) % Tc, Z = r / (Tc * Tc);
        const int Xg = tile.x * Tc + X, Yg = tile.y * Tc + Y, Zg = tile.z * Tc + Z;
        const bool in = q < per_tile;
        sIdx[t] = in ? (((int64_t)oct * H + Zg) * H + Yg) * H + Xg : 0;
        const int x = 2 * Xg + (oct & 1), y = 2 * Yg + ((oct >> 1) & 1), z = 2 * Zg + (oct >> 2);
        sRow[t] = in ? (int)parity_row(x, y, z, c, A.H, 0, A.R) : -1;
    }
    __syncthreads();
    for (int q = t; q < NB * nw; q += blockDim.x) {
        const int bx = q % NB, w = q / NB;
        sG[bx * nw + w] = sRow[bx] >= 0 ? A.Fhat[((int64_t)w * A.R + c) * nb + sIdx[bx]] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    // z: Bz(wx, wy; z) = sum_wz G(wx, wy, wz) e^{+2 pi i wz z / n}, z < p
    for (int q = t; q < NB * pnp; q += blockDim.x) {
        const int bx = q / pnp, r = q - bx * pnp;
        const int wx = r % p, wy = (r / p) % n, z = r / (p * n);
        const float2 *g = sG + bx * nw + wy * p + wx;
        float re = 0.0f, im = 0.0f;
        int k = 0;
        for (int wz = 0; wz < n; ++wz) {
            const float2 v = g[wz * n * p], tw = A.tw[k];
            re += v.x * tw.x - v.y * tw.y;
            im += v.y * tw.x + v.x * tw.y;
            k += z;
            k -= k >= n ? n : 0;
        }
        sBz[q] = make_float2(re, im);
    }
    __syncthreads();
    // y: Ay(wx; y, z) = sum_wy Bz(wx, wy; z) e^{+2 pi i wy y / n}, y < p
    for (int q = t; q < NB * p3; q += blockDim.x) {
        const int bx = q / p3, r = q - bx * p3;
        const int wx = r % p, y = (r / p) % p, z = r / (p * p);
        const float2 *b = sBz + bx * pnp + z * n * p + wx;
        float re = 0.0f, im = 0.0f;
        int k = 0;
        for (int wy = 0; wy < n; ++wy) {
            const float2 v = b[wy * p], tw = A.tw[k];
            re += v.x * tw.x - v.y * tw.y;
            im += v.y * tw.x + v.x * tw.y;
            k += y;
            k -= k >= n ? n : 0;
        }
        sAy[q] = make_float2(re, im);
    }
    __syncthreads();
    // x (real output): f = Re Ay(0) + 2 sum_{wx >= 1} Re(Ay(wx) e^{+2 pi i wx x / n})
    for (int q = t; q < NB * p3; q += blockDim.x) {
        const int bx = q / p3, r = q - bx * p3;
        const int row = sRow[bx];
        if (row < 0)
            continue;
        const int x = r % p, yz = r / p;
        const float2 *a = sAy + bx * p3 + yz * p;
        float f = 0.0f;
        int k = x;
        for (int wx = 1; wx < p; ++wx) {
            const float2 v = a[wx], tw = A.tw[k];
            f += v.x * tw.x - v.y * tw.y;
            k += x;
            k -= k >= n ? n : 0;
        }
        f = a[0].x + 2.0f * f;
        A.Ft[(int64_t)row * A.rp + r] = A.scale * f;
    }
}

// ---------------------------------------------------------------------------
// host side
static std::mutex g_fft_mu;
static bool g_fft_ready = false;

// tap tables and kernel attributes; called when a plan is built (outside any
// stream capture: the constant upload is a synchronous copy)
cudaError_t m2l_fft_init()
{
    std::lock_guard<std::mutex> g(g_fft_mu);
    if (g_fft_ready)
        return cudaSuccess;
    static int2 tab[2][8][kOffsetsPerClass];
    for (int sel = 0; sel < 2; ++sel) {
        const int T = sel == 0 ? 8 : 4, Ts = T / 2 + 3, Ts3 = Ts * Ts * Ts;
        for (int cls = 0; cls < 8; ++cls) {
            const int pc[3] = {cls & 1, (cls >> 1) & 1, cls >> 2};
            int j = 0;
            // offsets t with parent(target + t) next to parent(target), minus the
            // target's own neighbours: per axis t in [-2 - p, 3 - p]
            for (int tz = -2 - pc[2]; tz <= 3 - pc[2]; ++tz)
                for (int ty = -2 - pc[1]; ty <= 3 - pc[1]; ++ty)
                    for (int tx = -2 - pc[0]; tx <= 3 - pc[0]; ++tx) {
                        const int u = offset_index(tx, ty, tz);
                        if (u < 0)
                            continue;
                        if (j >= kOffsetsPerClass)
                            return cudaErrorInvalidValue;
                        const int tt[3] = {tx, ty, tz};
                        int q[3], d[3];
                        for (int a = 0; a < 3; ++a) {
                            q[a] = (pc[a] + tt[a] + 3) & 1;
                            d[a] = (pc[a] + tt[a] + 3) >> 1;
                        }
                        const int planeq = q[0] | (q[1] << 1) | (q[2] << 2);
                        tab[sel][cls][j++] = make_int2(planeq * Ts3 + (d[2] * Ts + d[1]) * Ts + d[0], u);
                    }
            if (j != kOffsetsPerClass)
                return cudaErrorInvalidValue;
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(c_fft_tap, tab, sizeof(tab));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmem + 8);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_m2l, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float4) * 8 * 7 * 7 * 7));
    if (e != cudaSuccess)
        return e;
    g_fft_ready = true;
    return cudaSuccess;
}

int64_t fft_grid_boxes(int l)
{
    const int64_t g = (1LL << l) + 6;
    return g * g * g;
}

void fft_active_tiles(int D, const std::vector<uint8_t> &leaf_occ, std::vector<int4> &tiles, int *count)
{
    tiles.clear();
    for (int l = 0; l <= kMaxDepth; ++l)
        count[l] = 0;
    if (D < 2)
        return;
    std::vector<std::vector<uint8_t>> occ(D + 1);
    occ[D] = leaf_occ;
    for (int l = D - 1; l >= 2; --l) {
        occ[l].assign((size_t)1 << (3 * l), 0);
        for (size_t b = 0; b < occ[l + 1].size(); ++b)
            if (occ[l + 1][b])
                occ[l][b >> 3] = 1;
    }
    for (int l = D; l >= 2; --l) {
        const int S = 1 << l, T = std::min(kFftTile, S), nt = S / T;
        std::vector<uint8_t> any((size_t)nt * nt * nt, 0);
        for (size_t b = 0; b < occ[l].size(); ++b)
            if (occ[l][b]) {
                int x, y, z;
                demorton3((uint32_t)b, x, y, z);
                any[((size_t)(z / T) * nt + y / T) * nt + x / T] = 1;
            }
        for (int tz = 0; tz < nt; ++tz)
            for (int ty = 0; ty < nt; ++ty)
                for (int tx = 0; tx < nt; ++tx)
                    if (any[((size_t)tz * nt + ty) * nt + tx]) {
                        tiles.push_back(make_int4(tx, ty, tz, 0));
                        count[l]++;
                    }
    }
}

cudaError_t launch_m2l_fft(bbfmm_plan_impl *P, int nrhs, cudaStream_t s)
{
    const DevOps &O = *P->ops;
    const int p = P->p, n = O.nfft;
    if (n != 2 * p - 1 || n > kFftMaxN || (int)O.khat.size() != O.nlev || nrhs < 1 || nrhs > P->max_nrhs)
        return cudaErrorInvalidValue;
    if (!g_fft_ready)
        return cudaErrorNotReady; // m2l_fft_init runs when the plan is built
    cudaError_t e = cudaSuccess;
    FftArgs A;
    memset(&A, 0, sizeof(A));
    for (int k = 0; k < n; ++k)
        A.tw[k] = make_float2((float)cos(2.0 * M_PI * k / n), (float)sin(2.0 * M_PI * k / n));
    A.p = p;
    A.n = n;
    A.nw = O.nw;
    A.p3 = p * p * p;
    A.rp = O.rp;
    A.R = P->max_nrhs;
    A.nrhs = nrhs;
    A.status = P->status;
    // boxes per DFT block: as many as the shared-memory budget holds (<= 16)
    const int pnp = p * n * p;
    const size_t fwd_box = sizeof(float) * A.p3 + sizeof(float2) * (A.p3 + pnp);
    const size_t inv_box = sizeof(float2) * (A.nw + pnp);
    A.nbf = (int)std::max<size_t>(1, std::min<size_t>(kFftBoxes, (kFftSmem - 8) / fwd_box));
    A.nbi = (int)std::max<size_t>(1, std::min<size_t>(kFftBoxes, kFftSmem / inv_box));
    const size_t fwd_smem = sizeof(float) * (A.nbf * A.p3 + 1) + sizeof(float2) * A.nbf * (A.p3 + pnp);
    const size_t inv_smem = inv_box * A.nbi;
    if (fwd_smem > kFftSmem + 8 || inv_smem > kFftSmem)
        return cudaErrorInvalidValue; // p beyond what one box's transform fits in
    for (int l = 2; l <= P->D; ++l) {
        const int k = O.nlev == 1 ? 0 : l - 2;
        A.l = l;
        A.S = 1 << l;
        A.G = A.S + 6;
        A.H = A.S / 2;
        A.T = std::min(kFftTile, A.S);
        A.Ts = A.T / 2 + 3;
        A.tsel = A.T == 8 ? 0 : 1;
        A.Mt = P->lev[l].Mt;
        A.Ft = P->lev[l].Ft;
        A.Mhat = P->lev[l].Mhat;
        A.Fhat = P->lev[l].Fhat;
        A.khat = O.khat[k];
        A.tiles = P->fft_tiles + P->fft_tile_off[l];
        A.scale = O.host->hom_degree != 0 ? (float)pow(2.0, (double)O.host->hom_degree * (P->D - l)) : 1.0f;
        const int ntile = P->fft_ntiles[l];
        const int64_t nbox = (int64_t)A.S * A.S * A.S;
        k_fft_fwd<<<dim3((unsigned)((nbox + A.nbf - 1) / A.nbf), (unsigned)nrhs), 128, fwd_smem, s>>>(A);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        if (ntile == 0)
            continue;
        const size_t smem = sizeof(float4) * 8 * A.Ts * A.Ts * A.Ts;
        k_fft_m2l<<<dim3((unsigned)ntile, (unsigned)((A.nw + kFftWPerBlock - 1) / kFftWPerBlock), (unsigned)nrhs),
                    kFftThreads, smem, s>>>(A);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        const int groups = (A.T * A.T * A.T + A.nbi - 1) / A.nbi;
        k_fft_inv<<<dim3((unsigned)ntile, (unsigned)groups, (unsigned)nrhs), 128, inv_smem, s>>>(A);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

} // namespace bbfmm
