// m2l_fft.cu -- far-field stage (Sec. 2.3 item 2) with equally spaced nodes
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
//   k_fft_m2l_tiled  (levels with 16+ boxes per axis) per frequency w and
//               tile of 16 x 16 x 8 target boxes: the 189-term sum over the
//               interaction list, a stencil on the box grid.  Warp = one
//               octant class (its offsets are warp-uniform), thread = 4 x 2
//               targets of the class; per z offset and pair of x / y source
//               parities the thread loads a 6 x 4 window of sources once and
//               applies the 9 offsets that read it (register reuse: 24
//               complex loads per 72 complex multiply-adds).  The 27 offsets
//               of the own neighbourhood enter with a zero spectrum instead
//               of a branch.
//   k_fft_m2l   the same for the two coarsest levels (one tile each):
//               thread = two targets adjacent in x.
//   k_fft_inv   per box: the inverse DFT (z, y, then x with the conjugate
//               half restored), only the p^3 outputs that are kept.
// The kernel spectra K^_t (host, FP64 -> FP32) already carry the 1 / n^3 of
// the inverse transform.  FP32 throughout; the tensor cores have no use here
// (the Fourier-domain product is diagonal).
#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int kFftMaxN = 2 * kMaxP - 1;
// tiles of target boxes: 16 x 16 x 8 on levels with 16+ boxes per axis (the
// tiled stencil), the whole level on the two coarsest
constexpr int kTX = 16, kTY = 16, kTZ = 8;
// halo tile of the tiled stencil, per source parity: 11 x 11 x 7 boxes,
// stored with a row stride of 14 and a z stride of 155 (float2 units), so
// that the 16 lanes of a half-warp read 16 different bank pairs
constexpr int kHX = kTX / 2 + 3, kHY = kTY / 2 + 3, kHZ = kTZ / 2 + 3;
constexpr int kPY = 14, kPZ = 155, kPP = kHZ * kPZ;
static_assert(kPY >= kHX && kPZ >= kHY * kPY, "halo strides");
constexpr int kTaps = 216; // 6^3 offsets per class, the 27 neighbours among them
constexpr int kFftThreads = 256;   // 8 warps = 8 octant classes
constexpr int kFftBoxes = 16;      // most boxes per block of the forward / inverse DFT
constexpr int kFftSmem = 96 * 1024; // shared memory budget of the DFT blocks
constexpr int kFftWPerBlock = 16;  // frequencies per block of the stencil

struct FftArgs {
    float2 tw[kFftMaxN]; // (cos, sin)(2 pi k / n)
    int p, n, nw, p3, rp, R, nrhs;
    int l, S, G, H;      // level, boxes per axis, M^ grid edge (S + 6), parent cells per axis (S / 2)
    int TX, TY, TZ;      // tile (boxes)
    int T, Ts, tsel;     // coarse levels: tile edge, halo edge per parity (T / 2 + 3), tap table (0: T = 8, 1: T = 4)
    int wpb;             // frequencies per block of the stencil
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
// tiled stencil: spectrum column (0..315, or 316 = zero) of the tap
// (tz, y parity, x parity, ey, ex) of each class, [8][216]
static int16_t *g_kmap = nullptr;

// ---------------------------------------------------------------------------
// DFT sizes of order P: n = 2P - 1 points per axis, P^3 coefficients, the
// kept half of the spectrum N W = n n P, and the boxes one block transforms
// (as many as kFftSmem holds, at most kFftBoxes)
template <int P> struct Dft {
    static constexpr int N = 2 * P - 1, P3 = P * P * P, PNP = P * N * P, NW = N * N * P;
    static constexpr int FWD_BOX = 4 * P3 + 8 * (P3 + PNP), INV_BOX = 8 * (NW + PNP);
    static constexpr int NBF = FWD_BOX * kFftBoxes <= kFftSmem ? kFftBoxes : (kFftSmem / FWD_BOX > 0 ? kFftSmem / FWD_BOX : 1);
    static constexpr int NBI = INV_BOX * kFftBoxes <= kFftSmem ? kFftBoxes : (kFftSmem / INV_BOX > 0 ? kFftSmem / INV_BOX : 1);
    static constexpr size_t FWD_SMEM = (size_t)FWD_BOX * NBF + 16, INV_SMEM = (size_t)INV_BOX * NBI;
};

// twiddle table in shared memory: tw[w * P + x] = (cos, sin)(2 pi (w x mod n) / n), w < n, x < P
template <int P> __device__ __forceinline__ void load_twiddles(const FftArgs &A, float2 *tw)
{
    constexpr int N = 2 * P - 1;
    for (int q = threadIdx.x; q < N * P; q += blockDim.x) {
        const int w = q / P, x = q - w * P;
        tw[q] = A.tw[(w * x) % N];
    }
}

// forward DFT: block = NBF consecutive boxes (lexicographic) x 1 RHS
constexpr int kDftThreads = 256;

template <int P> __global__ void __launch_bounds__(kDftThreads) k_fft_fwd(const __grid_constant__ FftArgs A)
{
    using D = Dft<P>;
    constexpr int N = D::N, P3 = D::P3, PNP = D::PNP, NB = D::NBF;
    extern __shared__ float2 fsm[];
    __shared__ float2 tw[N * P];
    __shared__ int sRow[kFftBoxes];
    float2 *sA = fsm;                                  // [box][z][y][wx]
    float2 *sB = sA + NB * P3;                         // [box][z][wy][wx]
    float *sM = reinterpret_cast<float *>(sB + NB * PNP); // [box][P3]
    const int c = blockIdx.y, l = A.l;
    const int64_t nbox = (int64_t)1 << (3 * l);
    const int64_t b0 = (int64_t)blockIdx.x * NB;
    const int t = threadIdx.x, S1 = A.S - 1;
    load_twiddles<P>(A, tw);
    if (t < NB) {
        const int64_t b = b0 + t;
        sRow[t] = b < nbox ? (int)parity_row((int)(b & S1), (int)((b >> l) & S1), (int)(b >> (2 * l)), c, A.H, 1, A.R)
                           : -1;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = t; q < NB * P3; q += blockDim.x) {
        const int bx = q / P3, k = q - bx * P3;
        const int row = sRow[bx];
        sM[q] = row >= 0 ? __ldg(A.Mt + (int64_t)row * A.rp + k) : 0.0f;
    }
    __syncthreads();
    // x: A(wx; y, z) = sum_x M(x, y, z) e^{-2 pi i wx x / n}, wx < P
    for (int q = t; q < NB * P3; q += blockDim.x) {
        const int wx = q % P, byz = q / P; // byz = box * P^2 + z P + y
        const float *m = sM + byz * P;
        const float2 *e = tw + wx * P;
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int x = 0; x < P; ++x) {
            re = fmaf(m[x], e[x].x, re);
            im = fmaf(-m[x], e[x].y, im);
        }
        sA[q] = make_float2(re, im);
    }
    __syncthreads();
    // y: B(wx, wy; z) = sum_y A(wx; y, z) e^{-2 pi i wy y / n}
    for (int q = t; q < NB * PNP; q += blockDim.x) {
        const int wx = q % P, r = q / P, wy = r % N, bz = r / N; // bz = box * P + z
        const float2 *a = sA + bz * P * P + wx;
        const float2 *e = tw + wy * P;
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int y = 0; y < P; ++y) {
            const float2 v = a[y * P];
            re = fmaf(v.x, e[y].x, fmaf(v.y, e[y].y, re));
            im = fmaf(v.y, e[y].x, fmaf(-v.x, e[y].y, im));
        }
        sB[q] = make_float2(re, im);
    }
    __syncthreads();
    // z, and the store: consecutive threads take consecutive boxes of one
    // frequency (coalesced rows of the M^ grid)
    const int64_t G = A.G, plane = G * G * G;
#pragma unroll 4
    for (int q = t; q < NB * D::NW; q += blockDim.x) {
        const int bx = q % NB, f = q / NB; // box, frequency
        const int64_t b = b0 + bx;
        if (b >= nbox)
            continue;
        const int wx = f % P, wy = (f / P) % N, wz = f / (P * N);
        const float2 *bb = sB + bx * PNP + wy * P + wx;
        const float2 *e = tw + wz * P;
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int z = 0; z < P; ++z) {
            const float2 v = bb[z * N * P];
            re = fmaf(v.x, e[z].x, fmaf(v.y, e[z].y, re));
            im = fmaf(v.y, e[z].x, fmaf(-v.x, e[z].y, im));
        }
        const int x = (int)(b & S1), y = (int)((b >> l) & S1), z = (int)(b >> (2 * l));
        A.Mhat[((int64_t)f * A.R + c) * plane + ((z + 3) * G + (y + 3)) * G + (x + 3)] = make_float2(re, im);
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
    const int w0 = blockIdx.y * A.wpb, w1 = min(A.nw, w0 + A.wpb);
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
// Fourier-domain M2L, tiled: block = one active 16 x 16 x 8 tile x A.wpb
// frequencies x 1 RHS; warp = octant class, lane = 4 x 2 targets of it
__global__ void __launch_bounds__(kFftThreads, 2) k_fft_m2l_tiled(const __grid_constant__ FftArgs A,
                                                                   const int16_t *__restrict__ kmap)
{
    extern __shared__ float2 sH[];        // [8 parities][kHZ][kHY][kHX], strides kPP, kPZ, kPY
    float2 *sKc = sH + 8 * kPP;           // [8 classes][216 taps]: the spectrum of each tap
    constexpr int EX = kTX + 6, EY = kTY + 6, EZ = kTZ + 6;
    const int c = blockIdx.z;
    const int4 tile = A.tiles[blockIdx.x];
    const int x0 = tile.x * kTX, y0 = tile.y * kTY, z0 = tile.z * kTZ;
    const int t = threadIdx.x, cls = t >> 5, lane = t & 31;
    if (tile.x < 0 || tile.y < 0 || tile.z < 0 || x0 + kTX > A.S || y0 + kTY > A.S || z0 + kTZ > A.S) {
        if (t == 0)
            atomicOr(A.status, kStatusBounds);
        return; // block-uniform
    }
    // the lane's targets: class cells (X0 + ix, Y0 + iy, Z), ix < 4, iy < 2;
    // the 16 lanes of a half-warp differ in y and z (conflict-free rows)
    const int X0 = 4 * (lane >> 4), Y0 = 2 * (lane & 3), Z = (lane >> 2) & 3;
    const int64_t G = A.G, plane = G * G * G;
    const int64_t H = A.H, nb = 8 * H * H * H;
    const int w0 = blockIdx.y * A.wpb, w1 = min(A.nw, w0 + A.wpb);
    for (int w = w0; w < w1; ++w) {
        __syncthreads(); // the previous frequency's reads are done
        const float2 *kh = A.khat + (int64_t)w * kNumOffsets;
        for (int q = t; q < 8 * kTaps; q += kFftThreads) {
            const int m = __ldg(kmap + q);
            sKc[q] = m < kNumOffsets ? __ldg(kh + m) : make_float2(0.0f, 0.0f);
        }
        const float2 *src = A.Mhat + ((int64_t)w * A.R + c) * plane;
#pragma unroll 4
        for (int q = t; q < EX * EY * EZ; q += kFftThreads) {
            const int hx = q % EX, hy = (q / EX) % EY, hz = q / (EX * EY);
            const float2 v = __ldg(src + ((int64_t)(z0 + hz) * G + (y0 + hy)) * G + (x0 + hx));
            const int par = (hx & 1) | ((hy & 1) << 1) | ((hz & 1) << 2);
            sH[par * kPP + (hz >> 1) * kPZ + (hy >> 1) * kPY + (hx >> 1)] = v;
        }
        __syncthreads();
        float ar[2][4], ai[2][4];
#pragma unroll
        for (int iy = 0; iy < 2; ++iy)
#pragma unroll
            for (int ix = 0; ix < 4; ++ix)
                ar[iy][ix] = ai[iy][ix] = 0.0f;
        const float2 *kc = sKc + cls * kTaps;
#pragma unroll 1
        for (int tzi = 0; tzi < 6; ++tzi) {
            // z offset tz = tzi - 2 - pz: source z parity and cell shift do
            // not depend on the class
            const int qz = (tzi + 1) & 1, dz = (tzi + 1) >> 1;
#pragma unroll
            for (int qy = 0; qy < 2; ++qy)
#pragma unroll
                for (int qx = 0; qx < 2; ++qx) {
                    // sources of the 9 offsets with these x / y parities:
                    // cells (X0 + d0x + rx, Y0 + d0y + ry), d0 = 1 - parity
                    const float2 *sp = sH + (qx | (qy << 1) | (qz << 2)) * kPP + (Z + dz) * kPZ +
                                       (Y0 + 1 - qy) * kPY + (X0 + 1 - qx);
                    float2 sv[4][6];
#pragma unroll
                    for (int ry = 0; ry < 4; ++ry)
#pragma unroll
                        for (int rx = 0; rx < 6; ++rx)
                            sv[ry][rx] = sp[ry * kPY + rx];
                    const float2 *kk = kc + ((tzi * 2 + qy) * 2 + qx) * 9;
#pragma unroll
                    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
                        for (int ex = 0; ex < 3; ++ex) {
                            const float2 k = kk[ey * 3 + ex];
#pragma unroll
                            for (int iy = 0; iy < 2; ++iy)
#pragma unroll
                                for (int ix = 0; ix < 4; ++ix) {
                                    const float2 m = sv[iy + ey][ix + ex];
                                    ar[iy][ix] = fmaf(m.x, k.x, ar[iy][ix]);
                                    ar[iy][ix] = fmaf(-m.y, k.y, ar[iy][ix]);
                                    ai[iy][ix] = fmaf(m.x, k.y, ai[iy][ix]);
                                    ai[iy][ix] = fmaf(m.y, k.x, ai[iy][ix]);
                                }
                        }
                }
        }
        // F^ [w][c][class][H][H][H]: four consecutive x cells per row
        float2 *out = A.Fhat + ((int64_t)w * A.R + c) * nb;
#pragma unroll
        for (int iy = 0; iy < 2; ++iy) {
            const int64_t row = (((int64_t)cls * H + (z0 / 2 + Z)) * H + (y0 / 2 + Y0 + iy)) * H + (x0 / 2 + X0);
            float4 *o = reinterpret_cast<float4 *>(out + row);
            o[0] = make_float4(ar[iy][0], ai[iy][0], ar[iy][1], ai[iy][1]);
            o[1] = make_float4(ar[iy][2], ai[iy][2], ar[iy][3], ai[iy][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// inverse DFT: block = NBI boxes of an active tile x 1 RHS
template <int P> __global__ void __launch_bounds__(kDftThreads) k_fft_inv(const __grid_constant__ FftArgs A)
{
    using D = Dft<P>;
    constexpr int N = D::N, P3 = D::P3, PNP = D::PNP, NW = D::NW, NB = D::NBI;
    extern __shared__ float2 fsm[];
    __shared__ float2 tw[N * P];
    __shared__ int64_t sIdx[kFftBoxes];
    __shared__ int sRow[kFftBoxes];
    const int c = blockIdx.z;
    const int Cx = A.TX / 2, Cy = A.TY / 2, Cz = A.TZ / 2; // class cells of the tile per axis
    const int per_tile = A.TX * A.TY * A.TZ;
    const int4 tile = A.tiles[blockIdx.x];
    const int t = threadIdx.x;
    if (tile.x < 0 || tile.y < 0 || tile.z < 0 || (tile.x + 1) * A.TX > A.S || (tile.y + 1) * A.TY > A.S ||
        (tile.z + 1) * A.TZ > A.S) {
        if (t == 0)
            atomicOr(A.status, kStatusBounds);
        return;
    }
    float2 *sG = fsm;           // [box][w]
    float2 *sBz = sG + NB * NW; // [box][z][wy][wx]
    float2 *sAy = sG;           // [box][z][y][wx] (over sG once it is used)
    const int64_t H = A.H, nb = 8 * H * H * H;
    load_twiddles<P>(A, tw);
    if (t < NB) {
        // box q of the tile in parity-split order: class, then Z, Y, X
        const int q = blockIdx.y * NB + t;
        const int C3 = Cx * Cy * Cz;
        const int oct = q / C3, r = q - oct * C3;
        const int X = r % Cx, Y = (r / Cx) % Cy, Z = r / (Cx * Cy);
        const int Xg = tile.x * Cx + X, Yg = tile.y * Cy + Y, Zg = tile.z * Cz + Z;
        const bool in = q < per_tile;
        sIdx[t] = in ? (((int64_t)oct * H + Zg) * H + Yg) * H + Xg : 0;
        const int x = 2 * Xg + (oct & 1), y = 2 * Yg + ((oct >> 1) & 1), z = 2 * Zg + (oct >> 2);
        sRow[t] = in ? (int)parity_row(x, y, z, c, A.H, 0, A.R) : -1;
    }
    __syncthreads();
    const float2 *fh = A.Fhat + (int64_t)c * nb;
    const int64_t fstride = (int64_t)A.R * nb;
#pragma unroll 8
    for (int q = t; q < NB * NW; q += blockDim.x) {
        const int bx = q % NB, w = q / NB;
        sG[bx * NW + w] = sRow[bx] >= 0 ? __ldg(fh + w * fstride + sIdx[bx]) : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    // z: Bz(wx, wy; z) = sum_wz G(wx, wy, wz) e^{+2 pi i wz z / n}, z < P
    for (int q = t; q < NB * PNP; q += blockDim.x) {
        const int wx = q % P, r = q / P, wy = r % N, r2 = r / N, z = r2 % P, bx = r2 / P;
        const float2 *g = sG + bx * NW + wy * P + wx;
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int wz = 0; wz < N; ++wz) {
            const float2 v = g[wz * N * P], e = tw[wz * P + z];
            re = fmaf(v.x, e.x, fmaf(-v.y, e.y, re));
            im = fmaf(v.y, e.x, fmaf(v.x, e.y, im));
        }
        sBz[q] = make_float2(re, im); // [box][z][wy][wx]
    }
    __syncthreads();
    // y: Ay(wx; y, z) = sum_wy Bz(wx, wy; z) e^{+2 pi i wy y / n}, y < P
    for (int q = t; q < NB * P3; q += blockDim.x) {
        const int wx = q % P, r = q / P, y = r % P, bz = r / P; // bz = box * P + z
        const float2 *b = sBz + bz * N * P + wx;
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int wy = 0; wy < N; ++wy) {
            const float2 v = b[wy * P], e = tw[wy * P + y];
            re = fmaf(v.x, e.x, fmaf(-v.y, e.y, re));
            im = fmaf(v.y, e.x, fmaf(v.x, e.y, im));
        }
        sAy[q] = make_float2(re, im); // [box][z][y][wx]
    }
    __syncthreads();
    // x (real output): f = Re Ay(0) + 2 sum_{wx >= 1} Re(Ay(wx) e^{+2 pi i wx x / n})
    for (int q = t; q < NB * P3; q += blockDim.x) {
        const int bx = q / P3, r = q - bx * P3;
        const int row = sRow[bx];
        if (row < 0)
            continue;
        const int x = r % P, yz = r / P;
        const float2 *a = sAy + bx * P3 + yz * P;
        float f = 0.0f;
#pragma unroll
        for (int wx = 1; wx < P; ++wx) {
            const float2 v = a[wx], e = tw[wx * P + x];
            f = fmaf(v.x, e.x, fmaf(-v.y, e.y, f));
        }
        f = a[0].x + 2.0f * f;
        A.Ft[(int64_t)row * A.rp + r] = A.scale * f;
    }
}

// ---------------------------------------------------------------------------
// host side
template <int P> static cudaError_t dft_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_fft_fwd<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Dft<P>::FWD_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_inv<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Dft<P>::INV_SMEM);
    if (e != cudaSuccess || P == kMaxP)
        return e;
    return dft_attrs<(P < kMaxP ? P + 1 : P)>();
}

template <int P> static cudaError_t launch_fwd(const FftArgs &A, int nrhs, cudaStream_t s)
{
    const int64_t nbox = (int64_t)A.S * A.S * A.S;
    k_fft_fwd<P><<<dim3((unsigned)((nbox + Dft<P>::NBF - 1) / Dft<P>::NBF), (unsigned)nrhs), kDftThreads,
                   Dft<P>::FWD_SMEM, s>>>(A);
    return cudaGetLastError();
}

template <int P> static cudaError_t launch_inv(const FftArgs &A, int ntile, int nrhs, cudaStream_t s)
{
    const int groups = (A.TX * A.TY * A.TZ + Dft<P>::NBI - 1) / Dft<P>::NBI;
    k_fft_inv<P><<<dim3((unsigned)ntile, (unsigned)groups, (unsigned)nrhs), kDftThreads, Dft<P>::INV_SMEM, s>>>(A);
    return cudaGetLastError();
}

#define BBFMM_DFT_DISPATCH(p, fn, args)                                                                         \
    switch (p) {                                                                                                \
    case 2: e = fn<2> args; break;                                                                              \
    case 3: e = fn<3> args; break;                                                                              \
    case 4: e = fn<4> args; break;                                                                              \
    case 5: e = fn<5> args; break;                                                                              \
    case 6: e = fn<6> args; break;                                                                              \
    case 7: e = fn<7> args; break;                                                                              \
    case 8: e = fn<8> args; break;                                                                              \
    case 9: e = fn<9> args; break;                                                                              \
    case 10: e = fn<10> args; break;                                                                            \
    default: e = cudaErrorInvalidValue;                                                                         \
    }
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
    // tiled stencil: the spectrum column of every (class, tap)
    std::vector<int16_t> km(8 * kTaps);
    for (int cls = 0; cls < 8; ++cls) {
        const int px = cls & 1, py = (cls >> 1) & 1, pz = cls >> 2;
        for (int tzi = 0; tzi < 6; ++tzi)
            for (int qy = 0; qy < 2; ++qy)
                for (int qx = 0; qx < 2; ++qx)
                    for (int ey = 0; ey < 3; ++ey)
                        for (int ex = 0; ex < 3; ++ex) {
                            // parity q, shift d = (1 - q) + e: t = 2 d + q - 3 - p
                            const int tz = tzi - 2 - pz;
                            const int ty = 2 * (1 - qy + ey) + qy - 3 - py;
                            const int tx = 2 * (1 - qx + ex) + qx - 3 - px;
                            const int u = offset_index(tx, ty, tz); // -1 for the 27 neighbours
                            km[cls * kTaps + (((tzi * 2 + qy) * 2 + qx) * 3 + ey) * 3 + ex] =
                                (int16_t)(u < 0 ? kNumOffsets : u);
                        }
    }
    int used = 0;
    for (int16_t v : km)
        used += v < kNumOffsets;
    if (used != 8 * kOffsetsPerClass)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMalloc(&g_kmap, km.size() * sizeof(int16_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(g_kmap, km.data(), km.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_fft_tap, tab, sizeof(tab));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_m2l_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float2) * (8 * kPP + 8 * kTaps)));
    if (e == cudaSuccess)
        e = dft_attrs<2>();
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
        const int S = 1 << l;
        const int TX = S >= 16 ? kTX : S, TY = S >= 16 ? kTY : S, TZ = S >= 16 ? kTZ : S;
        const int nx = S / TX, ny = S / TY, nz = S / TZ;
        std::vector<uint8_t> any((size_t)nx * ny * nz, 0);
        for (size_t b = 0; b < occ[l].size(); ++b)
            if (occ[l][b]) {
                int x, y, z;
                demorton3((uint32_t)b, x, y, z);
                any[((size_t)(z / TZ) * ny + y / TY) * nx + x / TX] = 1;
            }
        for (int tz = 0; tz < nz; ++tz)
            for (int ty = 0; ty < ny; ++ty)
                for (int tx = 0; tx < nx; ++tx)
                    if (any[((size_t)tz * ny + ty) * nx + tx]) {
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
    for (int l = 2; l <= P->D; ++l) {
        const int k = O.nlev == 1 ? 0 : l - 2;
        A.l = l;
        A.S = 1 << l;
        A.G = A.S + 6;
        A.H = A.S / 2;
        const bool tiled = A.S >= 16;
        A.TX = tiled ? kTX : A.S;
        A.TY = tiled ? kTY : A.S;
        A.TZ = tiled ? kTZ : A.S;
        A.T = A.S; // coarse levels: one tile of the whole level
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
        BBFMM_DFT_DISPATCH(p, launch_fwd, (A, nrhs, s))
        if (e != cudaSuccess)
            return e;
        if (ntile == 0)
            continue;
        // frequencies per block: enough blocks to fill the GPU several times
        A.wpb = (int)std::max<int64_t>(1, std::min<int64_t>(kFftWPerBlock, (int64_t)ntile * nrhs * A.nw / 1200));
        const unsigned nwb = (unsigned)((A.nw + A.wpb - 1) / A.wpb);
        if (tiled) {
            const size_t smem = sizeof(float2) * (8 * kPP + 8 * kTaps);
            k_fft_m2l_tiled<<<dim3((unsigned)ntile, nwb, (unsigned)nrhs), kFftThreads, smem, s>>>(A, g_kmap);
        } else {
            const size_t smem = sizeof(float4) * 8 * A.Ts * A.Ts * A.Ts;
            k_fft_m2l<<<dim3((unsigned)ntile, nwb, (unsigned)nrhs), kFftThreads, smem, s>>>(A);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        BBFMM_DFT_DISPATCH(p, launch_inv, (A, ntile, nrhs, s))
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

} // namespace bbfmm
