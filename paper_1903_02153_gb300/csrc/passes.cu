// passes.cu -- the upward and downward passes of the black-box FMM, each as
// ONE launch over the boxes of level D-1 (one block per box and right-hand
// side).
//
// Upward (Sec. 2.3 item 1, with the compression of Sec. 2.5 "Fast M2L
// translation"): a block makes the multipole coefficients of its 8 leaves
// (P2M, Def. 2.2 applied to the sources), compresses them (M~ = V^T M),
// combines them into its own box (M2M, the nested interpolation of Thm. 2.1
// item 1) and compresses that.  The upper levels follow without another
// launch: after its box is written, a block counts itself in at the parent;
// the eighth of the siblings to arrive (the others return) reads the 8
// sibling coefficient sets, makes and compresses the parent's, and counts
// itself in one level up, down to level 2.  No block waits for another.
//
// Downward (Sec. 2.3 item 3): a block makes the local coefficients of its
// box (decompress F = U F~, plus the L2L of its parent's), spreads them to
// its 8 leaves (L2L), adds the leaves' decompressed far fields and evaluates
// them at the leaves' points (L2P).  The levels above come from a first,
// small launch with a block per box of level D-2: it recomputes that box's
// ancestors from level 2 down (repeated once per level-(D-2) box, small) and
// stores the box's F, which the main launch reads as its parent.  Below depth
// 4 the main launch recomputes its ancestors itself.
//
// Coefficient layouts: M and F are Morton-ordered [box][nrhs][p^3]; M~ / F~
// rows sit at parity_row() of their box with the plan's max_nrhs as stride.
// Inside a block the coefficient sets of 8 sibling boxes are kept as
// [p^3][8] so that one 16-byte shared load gives 4 boxes.
#include "bbfmm_internal.h"

namespace bbfmm {

namespace {

constexpr int kThreads = 256;
// the wide upward pass (a block per box of level D-2) pays off once its
// 8^(D-2) blocks fill the GPU several times over, and only while the pass
// compresses the leaves itself (it shares each operator load among 8 of
// them); below that depth, or when a GEMM compresses the leaves, the narrow
// one (a block per box of level D-1) keeps more blocks in flight (depth 6,
// leaves compressed by the GEMM: 0.542 -> 0.450 ms for the upward stage)
constexpr int kWideMaxP = 7;     // largest p whose 64 leaf sets fit in shared memory
constexpr int kWideMinDepth = 6; // 4096 blocks

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int P>
__device__ __forceinline__ void basis_1d(const InterpTables &T, float s, float *out)
{
#pragma unroll
    for (int i = 0; i < P; ++i) {
        float v = T.wbary[i];
#pragma unroll
        for (int k = 0; k < P; ++k)
            if (k != i)
                v *= s - T.nodes[k];
        out[i] = v;
    }
}

template <int P> struct Smem {
    static constexpr int P3 = P * P * P;
    // upward: sMT [P3][8] | scratch: max(basis table 8 warps x 3 x 32 x P + sigma 8 x 32, two [P3][8])
    //         | sPar [P3]
    static constexpr int kScratch = (768 * P + 256) > 16 * P3 ? (768 * P + 256) : 16 * P3;
    static constexpr int kUpFloats = 8 * P3 + kScratch + P3;
    // downward: sMT [P3][8] | two [P3][8] | sPar [P3] | sOne [P3] | sFt [r][8] (r <= P3);
    // sFt is read as float4, so its offset is a multiple of 4 floats
    static constexpr int kDownFt = (26 * P3 + 3) & ~3;
    static constexpr int kDownFloats = kDownFt + 8 * P3;
};

// The child-to-parent transfers are tensor products of 1D matrices
// (Thm. 2.1 item 1): M^parent = sum_o (S_oz (x) S_oy (x) S_ox) M^child_o,
// with child o = (x, y, z parity) = (o & 1, (o >> 1) & 1, o >> 2), its
// position in Morton order.  They are applied one axis at a time, and the
// children that share the remaining axes' matrices are summed as soon as the
// axis that tells them apart is done (x pass on 8, y pass on 4 pairs, z pass
// on 2 quadruples: 14 p^4 products instead of 24 p^4).  A thread owns one
// line of p values along the current axis: it loads the p inputs once and
// writes the p outputs, so index arithmetic is paid once per line.

// M2M of 8 children X ([P3][8], row stride XS) into one parent out[r * OS];
// scratch Y [P3][8], Z [P3][4]
template <int P, int XS = 8, int OS = 1>
__device__ void m2m8(const InterpTables &T, const float *X, float *Y, float *Z, float *out)
{
    constexpr int P2 = P * P;
    const int t = threadIdx.x;
    for (int q = t; q < 8 * P2; q += kThreads) { // x pass: line (child o, j2 + P j3)
        const int o = q & 7, rest = q >> 3;
        float x[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            x[j] = X[(j + P * rest) * XS + o];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][i][j] * x[j];
            Y[(i + P * rest) * 8 + o] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < 4 * P2; q += kThreads) { // y pass: line (oy + 2 oz, i1, j3), x pairs summed
        const int yz = q & 3, u = q >> 2, i1 = u % P, j3 = u / P;
        float y[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float *src = Y + (i1 + P * j + P2 * j3) * 8 + 2 * yz;
            y[j] = src[0] + src[1];
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[yz & 1][i][j] * y[j];
            Z[(i1 + P * i + P2 * j3) * 4 + yz] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < P2; q += kThreads) { // z pass: line i1 + P i2, y pairs summed
        float z0[P], z1[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float *src = Z + (q + P2 * j) * 4;
            z0[j] = src[0] + src[1];
            z1[j] = src[2] + src[3];
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[0][i][j] * z0[j] + T.S[1][i][j] * z1[j];
            out[(q + P2 * i) * OS] = a;
        }
    }
    __syncthreads();
}

// L2L of one parent F (P3) into its 8 children (out[r * OS + o]), the
// transpose of m2m8, the children sharing a z (then y) matrix sharing the
// pass: z pass for 2, y pass for 4, x pass for 8; scratch Y, Z (>= 4 P3 each)
template <int P, int OS = 8>
__device__ void l2l8(const InterpTables &T, const float *F, float *Y, float *Z, float *out)
{
    constexpr int P2 = P * P, P3 = P2 * P;
    const int t = threadIdx.x;
    for (int q = t; q < 2 * P2; q += kThreads) { // z pass: line (oz, j1 + P j2)
        const int oz = q & 1, j12 = q >> 1;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = F[j12 + P2 * j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[oz][j][i] * f[j];
            Y[oz * P3 + j12 + P2 * i] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < 4 * P2; q += kThreads) { // y pass: line (oy + 2 oz, j1, i3)
        const int yz = q & 3, u = q >> 2, j1 = u % P, i3 = u / P;
        const float *src = Y + (yz >> 1) * P3 + j1 + P2 * i3;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = src[P * j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[yz & 1][j][i] * f[j];
            Z[yz * P3 + j1 + P * i + P2 * i3] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < 8 * P2; q += kThreads) { // x pass: line (child o, i2 + P i3)
        const int o = q & 7, rest = q >> 3;
        const float *src = Z + (o >> 1) * P3 + P * rest;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = src[j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][j][i] * f[j];
            out[(i + P * rest) * OS + o] = a;
        }
    }
    __syncthreads();
}

// L2L of a parent F into its child o only; scratch Y (P3); result in out
// (which may be F)
template <int P>
__device__ void l2l1(const InterpTables &T, const float *F, int o, float *Y, float *out)
{
    constexpr int P2 = P * P;
    const int t = threadIdx.x;
    for (int q = t; q < P2; q += kThreads) { // z pass: line j1 + P j2
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = F[q + P2 * j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o >> 2][j][i] * f[j];
            Y[q + P2 * i] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < P2; q += kThreads) { // y pass: line (j1, i3), into out
        const int j1 = q % P, i3 = q / P;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = Y[j1 + P * j + P2 * i3];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[(o >> 1) & 1][j][i] * f[j];
            out[j1 + P * i + P2 * i3] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < P2; q += kThreads) { // x pass: line i2 + P i3, in place
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = out[P * q + j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][j][i] * f[j];
            out[P * q + i] = a;
        }
    }
    __syncthreads();
}

// store one M~ value: FP32 row, optional TF32 hi/lo split, running max |M~|
__device__ __forceinline__ void put_mt(const PassArgs &A, int l, int64_t at, float v, float &mx)
{
    A.Mt[l][at] = v;
    if (A.Mt_hi[l]) {
        const float hi = tf32_round(v);
        A.Mt_hi[l][at] = hi;
        A.Mt_lo[l][at] = tf32_round(v - hi);
    }
    mx = fmaxf(mx, fabsf(v));
}

__device__ __forceinline__ void flush_max(const PassArgs &A, int l, float mx)
{
    if (!A.maxbits)
        return;
    for (int o = 16; o > 0; o >>= 1)
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0f)
        atomicMax(A.maxbits + l, __float_as_uint(mx));
}

// compress 8 sibling boxes box0..box0+7 at level l: M~[k] = sum_i V[i][k] M[i];
// X is [P3][8], or [8][P3] with XT
template <int P, bool XT = false>
__device__ void compress8(const PassArgs &A, int l, const float *X, int64_t box0, int c, bool zero)
{
    constexpr int P3 = P * P * P;
    const int t = threadIdx.x, h = t >> 7;
    const int H = 1 << (l - 1);
    const float *V = A.V[l];
    float mx = 0.0f;
    for (int k0 = 0; k0 < A.rl[l]; k0 += 128) { // uniform trip count: the warp shuffles below need all lanes
        const int k = k0 + (t & 127);
        const bool on = k < A.rl[l];
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (on && !zero) {
#pragma unroll 5
            for (int i = 0; i < P3; ++i) {
                const float v = __ldg(V + (int64_t)i * A.rp + k);
                const float4 m = XT ? make_float4(X[4 * h * P3 + i], X[(4 * h + 1) * P3 + i],
                                                  X[(4 * h + 2) * P3 + i], X[(4 * h + 3) * P3 + i])
                                    : *reinterpret_cast<const float4 *>(X + i * 8 + 4 * h);
                acc[0] += m.x * v;
                acc[1] += m.y * v;
                acc[2] += m.z * v;
                acc[3] += m.w * v;
            }
        }
        if (on) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int x, y, z;
                demorton3((uint32_t)(box0 + 4 * h + q), x, y, z);
                put_mt(A, l, parity_row(x, y, z, c, H, 1, A.R) * A.rp + k, acc[q], mx);
            }
        }
    }
    flush_max(A, l, mx);
}

// leaf multipoles for the compression GEMM: columns box0 .. box0 + ncol - 1
// of X ([P3][XS]) into rows (c, box) of A.Mleaf ([R][8^D][p3p])
template <int P, int XS>
__device__ void store_leaves(const PassArgs &A, const float *X, int64_t box0, int ncol, int c)
{
    constexpr int P3 = P * P * P;
    const int64_t nb = 1LL << (3 * A.D);
    for (int q = threadIdx.x; q < ncol * P3; q += kThreads) {
        const int o = q / P3, i = q - o * P3;
        A.Mleaf[((int64_t)c * nb + box0 + o) * A.p3p + i] = X[i * XS + o];
    }
}

// compress one box at level l from F32 coefficients X[P3]
template <int P>
__device__ void compress1(const PassArgs &A, int l, const float *X, int64_t box, int c)
{
    constexpr int P3 = P * P * P;
    const int t = threadIdx.x;
    const int H = 1 << (l - 1);
    const float *V = A.V[l];
    int x, y, z;
    demorton3((uint32_t)box, x, y, z);
    const int64_t row = parity_row(x, y, z, c, H, 1, A.R) * A.rp;
    float mx = 0.0f;
    for (int k0 = 0; k0 < A.rl[l]; k0 += kThreads) {
        const int k = k0 + t;
        if (k < A.rl[l]) {
            float a0 = 0.0f, a1 = 0.0f;
            int i = 0;
            for (; i + 1 < P3; i += 2) {
                a0 += X[i] * __ldg(V + (int64_t)i * A.rp + k);
                a1 += X[i + 1] * __ldg(V + (int64_t)(i + 1) * A.rp + k);
            }
            if (i < P3)
                a0 += X[i] * __ldg(V + (int64_t)i * A.rp + k);
            put_mt(A, l, row + k, a0 + a1, mx);
        }
    }
    flush_max(A, l, mx);
}

// ---------------------------------------------------------------------------
// five blocks per SM (<= 51 registers) up to p = 5: more blocks hide the
// pass's barriers and loads (148 -> 134 us at p = 5, depth 5; six blocks were
// slower, and p = 6 spills at five)
template <int P> constexpr int kUpMinBlocks = P <= 5 ? 5 : 1;

template <int P>
__global__ void __launch_bounds__(kThreads, kUpMinBlocks<P>) k_upward(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P;
    constexpr int NQ = (P * P + 31) / 32; // (i2, i3) pairs per lane in P2M
    extern __shared__ __align__(16) float sm[];
    float *sMT = sm;                       // [P3][8]
    float *sScr = sm + 8 * P3;             // scratch
    float *sPar = sScr + Smem<P>::kScratch; // [P3]
    float *sL = sScr;                      // [8][3][32][P] basis values (x row premultiplied by sigma)
    __shared__ int sLast;

    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int D = A.D;
    const int64_t b = blockIdx.x; // box at level D-1
    const int c = blockIdx.y;     // right-hand side
    const int64_t leaf = 8 * b + w;
    const int s0 = A.off[leaf], s1 = A.off[leaf + 1];

    // ---- P2M: warp w makes M of leaf 8b + w (Sec. 2.3 item 1, Def. 2.2)
    {
        float acc[NQ][P];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < P; ++i)
                acc[q][i] = 0.0f;
        float *L = sL + w * 3 * 32 * P;
        for (int c0 = s0; c0 < s1; c0 += 32) {
            const int cnt = min(32, s1 - c0);
            __syncwarp();
            if (lane < cnt) {
                const float4 u = A.pts[c0 + lane];
                const float sg = A.sig[(int64_t)c * A.n + c0 + lane];
                float v[P];
                basis_1d<P>(A.T, 2.0f * u.x, v);
#pragma unroll
                for (int i = 0; i < P; ++i)
                    L[lane * P + i] = v[i] * sg;
                basis_1d<P>(A.T, 2.0f * u.y, v);
#pragma unroll
                for (int i = 0; i < P; ++i)
                    L[(32 + lane) * P + i] = v[i];
                basis_1d<P>(A.T, 2.0f * u.z, v);
#pragma unroll
                for (int i = 0; i < P; ++i)
                    L[(64 + lane) * P + i] = v[i];
            }
            __syncwarp();
            for (int j = 0; j < cnt; ++j) {
                float lx[P];
#pragma unroll
                for (int i = 0; i < P; ++i)
                    lx[i] = L[j * P + i];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int pq = lane + 32 * q;
                    if (pq < P * P) {
                        const float yz = L[(32 + j) * P + pq % P] * L[(64 + j) * P + pq / P];
#pragma unroll
                        for (int i = 0; i < P; ++i)
                            acc[q][i] += lx[i] * yz;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int pq = lane + 32 * q;
            if (pq < P * P) {
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const int idx = i + P * pq;
                    sMT[idx * 8 + w] = acc[q][i];
                    if (A.keep)
                        A.M[D][(leaf * A.nrhs + c) * P3 + idx] = acc[q][i];
                }
            }
        }
    }
    // the barrier after P2M also tells whether the box holds points
    const bool zero = __syncthreads_count(s1 > s0) == 0;

    // ---- compress the leaves (or leave them to the compression GEMM; a box
    // without points keeps the zeros its rows were given at plan time)
    if (!A.Mleaf)
        compress8<P>(A, D, sMT, 8 * b, c, zero);
    else if (!zero)
        store_leaves<P, 8>(A, sMT, 8 * b, 8, c);
    if (D - 1 < 2)
        return;

    // ---- own box at level D-1: M2M of the 8 leaves, store, compress
    if (zero) {
        for (int r = t; r < P3; r += kThreads)
            sPar[r] = 0.0f;
        __syncthreads();
    } else {
        m2m8<P>(A.T, sMT, sScr, sScr + 8 * P3, sPar);
    }
    for (int r = t; r < P3; r += kThreads)
        A.M[D - 1][(b * A.nrhs + c) * P3 + r] = sPar[r];
    if (A.Mlev1) // compressed by the GEMM after this launch
        for (int r = t; r < P3; r += kThreads)
            A.Mlev1[((int64_t)c * (1LL << (3 * (D - 1))) + b) * A.p3p + r] = sPar[r];
    else
        compress1<P>(A, D - 1, sPar, b, c);

    // ---- upper levels: the last of 8 siblings to arrive makes the parent
    int64_t box = b;
    for (int l = D - 2; l >= 2; --l) {
        const int64_t par = box >> 3;
        // the barrier orders every thread's stores of the level-(l+1) box
        // before thread 0's fence, which makes them visible device-wide
        // before its arrival is counted
        __syncthreads();
        if (t == 0) {
            __threadfence();
            int *cnt = A.count[l] + par * A.R + c;
            const int before = atomicAdd(cnt, 1);
            sLast = before == 7;
            if (before == 7) {
                atomicExch(cnt, 0); // ready for the next matvec
                __threadfence();
            }
        }
        __syncthreads();
        if (!sLast)
            return;
        const float *Mc = A.M[l + 1] + (8 * par * A.nrhs + c) * (int64_t)P3;
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q & 7, r = q >> 3;
            sMT[q] = __ldcg(Mc + (int64_t)o * A.nrhs * P3 + r);
        }
        __syncthreads();
        m2m8<P>(A.T, sMT, sScr, sScr + 8 * P3, sPar);
        for (int r = t; r < P3; r += kThreads)
            A.M[l][(par * A.nrhs + c) * P3 + r] = sPar[r];
        compress1<P>(A, l, sPar, par, c);
        box = par;
    }
}

// ---------------------------------------------------------------------------
// F~ row of box at level l, column c, summed over the M2L offset-group slices
// in a fixed order, into dst[k * stride] for k < r
__device__ __forceinline__ void load_ft(const PassArgs &A, int l, int64_t box, int c, float *dst, int stride,
                                        int k)
{
    const int H = 1 << (l - 1);
    int x, y, z;
    demorton3((uint32_t)box, x, y, z);
    const float *src = A.Ft[l] + parity_row(x, y, z, c, H, 0, A.R) * A.rp + k;
    float v = __ldg(src);
    for (int g = 1; g < A.nslices; ++g)
        v += __ldg(src + g * A.slice[l]);
    dst[k * stride] = v;
}

// L2P of a leaf with few points (Sec. 2.3 item 3): a warp takes 32 / P
// points at a time, lane = (point, i3); the lane sums the z slice i3 of the
// leaf's coefficients at its point, times the z basis value, and the P lanes
// of a point are added in order of i3 by shuffles.  Per point this costs P^2
// products on each of P lanes instead of P^3 on one lane (most of a warp is
// idle when a leaf holds a handful of points).  F: the leaf's coefficients,
// element i at F[8 i].  Used up to p = 6: above it the extra path would cost
// the kernel registers, i.e. blocks per SM.
template <int P> __host__ __device__ constexpr int l2p_round() { return 32 / P; }
template <int P> constexpr bool kL2PSmall = P <= 6;

template <int P>
__device__ void l2p_small(const PassArgs &A, const float *F, int s0, int s1, int c)
{
    constexpr int R = l2p_round<P>();
    const int lane = threadIdx.x & 31;
    const int pl = lane / P, i3 = lane - pl * P;
    const float *Fz = F + (P * P * i3) * 8;
    for (int c0 = s0; c0 < s1; c0 += R) {
        const int j = c0 + pl;
        const bool has = pl < R && j < s1;
        const float4 u = A.tpts[has ? j : s0];
        float Lx[P], Ly[P];
        basis_1d<P>(A.T, 2.0f * u.x, Lx);
        basis_1d<P>(A.T, 2.0f * u.y, Ly);
        const float sz = 2.0f * u.z;
        float lz = A.T.wbary[i3];
#pragma unroll
        for (int k = 0; k < P; ++k)
            lz *= k != i3 ? sz - A.T.nodes[k] : 1.0f;
        // one row of P coefficients live at a time (the kernel's other
        // phases fit in 32 registers; so must this one)
        float slice = 0.0f;
#pragma unroll 1
        for (int i2 = 0; i2 < P; ++i2) {
            float part = 0.0f;
#pragma unroll
            for (int i1 = 0; i1 < P; ++i1)
                part += Fz[(i1 + P * i2) * 8] * Lx[i1];
            slice += part * Ly[i2];
        }
        const float v = slice * lz;
        // the point's P slices in order of i3 (lanes pl P .. pl P + P - 1)
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < P; ++k)
            acc += __shfl_sync(0xffffffffu, v, pl * P + k);
        if (has && i3 == 0)
            A.phi[(int64_t)c * A.nt + j] = acc;
    }
}

// 4-byte asynchronous copies global -> shared (the block waits for its own
// groups, then a barrier makes every thread's copies visible)
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int P>
__global__ void __launch_bounds__(kThreads) k_downward(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P;
    extern __shared__ __align__(16) float sm[];
    float *sMT = sm;              // [P3][8] leaf local coefficients
    float *sY = sm + 8 * P3;      // [P3][8] scratch
    float *sZ = sY + 8 * P3;      // [P3][8] scratch
    float *sPar = sZ + 8 * P3;    // [P3] local coefficients of the current ancestor
    float *sOne = sPar + P3;      // [P3] scratch
    float *sFt = sm + Smem<P>::kDownFt; // [r][8] far-field coefficients (compressed)

    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int D = A.D;
    const int64_t b = blockIdx.x; // box at level D-1
    const int c = blockIdx.y;
    if (!A.keep && A.toff[8 * b] == A.toff[8 * b + 8])
        return; // no targets below this box

    if (A.Ftop && A.Fdec1 && A.Fdec) {
        // everything this block reads from the earlier launches, copied in at
        // once: the parent's F (first launch), then the own box's and the 8
        // leaves' decompressed far fields (GEMM), which land while the
        // parent's F is carried down to the own box
        float *sOwnF = sY;  // [P3]: sY is free until the 8-child L2L
        float *sDec = sFt;  // [8][P3]: sFt is not used on this path
        __shared__ int64_t sRows[9];
        const float *Fp = A.Ftop + ((b >> 3) * A.nrhs + c) * (int64_t)P3;
        for (int i = t; i < P3; i += kThreads)
            cp_async4(sPar + i, Fp + i);
        cp_async_commit();
        if (t < 9) {
            const int64_t box = t < 8 ? 8 * b + t : b;
            int x, y, z;
            demorton3((uint32_t)box, x, y, z);
            sRows[t] = parity_row(x, y, z, c, 1 << (t < 8 ? D - 1 : D - 2), 0, A.R) * A.p3p;
        }
        __syncthreads();
        for (int i = t; i < P3; i += kThreads)
            cp_async4(sOwnF + i, A.Fdec1 + sRows[8] + i);
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q / P3;
            cp_async4(sDec + q, A.Fdec + sRows[o] + (q - o * P3));
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        l2l1<P>(A.T, sPar, (int)(b & 7), sOne, sPar); // parent -> own box (level D-1 >= 3)
        cp_async_wait<0>();
        __syncthreads();
        for (int i = t; i < P3; i += kThreads) {
            const float f = sPar[i] + sOwnF[i];
            sPar[i] = f;
            if (A.keep)
                A.F[D - 1][(b * A.nrhs + c) * P3 + i] = f;
        }
        __syncthreads();
        l2l8<P>(A.T, sPar, sY, sZ, sMT);
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q / P3, i = q - o * P3;
            sMT[i * 8 + o] += sDec[q];
        }
    } else {
    // ---- ancestors at levels 2 .. D-1 (the last one is the block's own box);
    // with Ftop the parent's F comes from the first launch
    int l0 = 2;
    if (A.Ftop) {
        const float *Fp = A.Ftop + ((b >> 3) * A.nrhs + c) * (int64_t)P3;
        for (int i = t; i < P3; i += kThreads)
            sPar[i] = __ldcg(Fp + i);
        __syncthreads();
        l0 = D - 1;
    }
    for (int l = l0; l <= D - 1; ++l) {
        const int64_t anc = b >> (3 * (D - 1 - l));
        if (l > 2)
            l2l1<P>(A.T, sPar, (int)(anc & 7), sOne, sPar);
        if (l == D - 1 && A.Fdec1) {
            // the block's own box, decompressed by the GEMM before this launch
            int x, y, z;
            demorton3((uint32_t)anc, x, y, z);
            const float *src = A.Fdec1 + parity_row(x, y, z, c, 1 << (l - 1), 0, A.R) * A.p3p;
            for (int i = t; i < P3; i += kThreads) {
                const float f = (l > 2 ? sPar[i] : 0.0f) + __ldg(src + i);
                sPar[i] = f;
                if (A.keep)
                    A.F[l][(anc * A.nrhs + c) * P3 + i] = f;
            }
            __syncthreads();
            continue;
        }
        const int rl = A.rl[l];
        for (int k = t; k < rl; k += kThreads)
            load_ft(A, l, anc, c, sFt, 1, k);
        __syncthreads();
        const float *Ut = A.Ut[l];
        for (int i = t; i < P3; i += kThreads) {
            float a0 = 0.0f, a1 = 0.0f;
            int k = 0;
            for (; k + 1 < rl; k += 2) {
                a0 += sFt[k] * __ldg(Ut + (int64_t)k * A.p3p + i);
                a1 += sFt[k + 1] * __ldg(Ut + (int64_t)(k + 1) * A.p3p + i);
            }
            if (k < rl)
                a0 += sFt[k] * __ldg(Ut + (int64_t)k * A.p3p + i);
            const float f = (l > 2 ? sPar[i] : 0.0f) + (a0 + a1);
            sPar[i] = f;
            if (A.keep && (b & ((1LL << (3 * (D - 1 - l))) - 1)) == 0)
                A.F[l][(anc * A.nrhs + c) * P3 + i] = f;
        }
        __syncthreads();
    }

    // ---- the 8 leaves: L2L from the block's box (none when it is at level 1)
    // plus their own decompressed far field
    if (D - 1 >= 2) {
        l2l8<P>(A.T, sPar, sY, sZ, sMT);
    } else {
        for (int q = t; q < 8 * P3; q += kThreads)
            sMT[q] = 0.0f;
    }
    if (A.Fdec) {
        // the leaves' far fields, decompressed by the GEMM before this launch
        __shared__ int64_t sDec[8];
        if (t < 8) {
            int x, y, z;
            demorton3((uint32_t)(8 * b + t), x, y, z);
            sDec[t] = parity_row(x, y, z, c, 1 << (D - 1), 0, A.R) * A.p3p;
        }
        __syncthreads();
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q / P3, i = q - o * P3;
            sMT[i * 8 + o] += __ldg(A.Fdec + sDec[o] + i);
        }
    } else {
        __shared__ int64_t sRow[8]; // F~ row offsets of the 8 leaves
        if (t < 8) {
            int x, y, z;
            demorton3((uint32_t)(8 * b + t), x, y, z);
            sRow[t] = parity_row(x, y, z, c, 1 << (D - 1), 0, A.R) * A.rp;
        }
        __syncthreads();
        for (int q = t; q < 8 * A.rl[D]; q += kThreads) {
            const int o = q & 7, k = q >> 3;
            const float *src = A.Ft[D] + sRow[o] + k;
            float v = __ldg(src);
            for (int g = 1; g < A.nslices; ++g)
                v += __ldg(src + g * A.slice[D]);
            sFt[k * 8 + o] = v;
        }
        __syncthreads();
        const float *Ut = A.Ut[D];
        const int h = t >> 7;
        for (int i0 = 0; i0 < P3; i0 += 128) {
            const int i = i0 + (t & 127);
            if (i < P3) {
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
                for (int k = 0; k < A.rl[D]; ++k) {
                    const float u = __ldg(Ut + (int64_t)k * A.p3p + i);
                    const float4 f = *reinterpret_cast<const float4 *>(sFt + k * 8 + 4 * h);
                    acc[0] += f.x * u;
                    acc[1] += f.y * u;
                    acc[2] += f.z * u;
                    acc[3] += f.w * u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sMT[i * 8 + 4 * h + q] += acc[q];
            }
        }
    }
    }
    __syncthreads();
    if (A.keep)
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q & 7, r = q >> 3;
            A.F[D][((8 * b + o) * A.nrhs + c) * P3 + r] = sMT[q];
        }

    // ---- L2P: warp w evaluates leaf 8b + w at its targets (Sec. 2.3 item 3)
    const int64_t leaf = 8 * b + w;
    const int s0 = A.toff[leaf], s1 = A.toff[leaf + 1];
    if (kL2PSmall<P> && s1 - s0 <= 2 * l2p_round<P>()) {
        l2p_small<P>(A, sMT + w, s0, s1, c);
        return;
    }
    for (int c0 = s0; c0 < s1; c0 += 32) {
        const int j = c0 + lane;
        const bool has = j < s1;
        const float4 u = A.tpts[has ? j : s0];
        float Lx[P], Ly[P];
        basis_1d<P>(A.T, 2.0f * u.x, Lx);
        basis_1d<P>(A.T, 2.0f * u.y, Ly);
        const float sz = 2.0f * u.z;
        float acc = 0.0f;
        // the z slices one at a time (the z basis value made on the spot), so
        // that the P^3 coefficient loads are not all kept in registers
#pragma unroll 1
        for (int i3 = 0; i3 < P; ++i3) {
            float lz = A.T.wbary[i3];
#pragma unroll
            for (int k = 0; k < P; ++k)
                lz *= k != i3 ? sz - A.T.nodes[k] : 1.0f;
            const float *Fz = sMT + (P * P * i3) * 8 + w;
            float slice = 0.0f;
#pragma unroll
            for (int i2 = 0; i2 < P; ++i2) {
                float part = 0.0f;
#pragma unroll
                for (int i1 = 0; i1 < P; ++i1)
                    part += Fz[(i1 + P * i2) * 8] * Lx[i1];
                slice += part * Ly[i2];
            }
            acc += slice * lz;
        }
        if (has)
            A.phi[(int64_t)c * A.nt + j] = acc;
    }
}

// ---------------------------------------------------------------------------
// First downward launch (depth >= 4): block = (box of level D-2, RHS); the
// box's F from level 2 down, as the main launch would recompute it, into Ftop
template <int P>
__global__ void __launch_bounds__(kThreads) k_down_top(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P;
    extern __shared__ __align__(16) float sm[];
    float *sPar = sm;         // [P3] local coefficients of the current ancestor
    float *sOne = sm + P3;    // [P3] scratch
    float *sFt = sm + 2 * P3; // [r] far-field coefficients (compressed)
    const int t = threadIdx.x;
    const int D = A.D, lt = D - 2;
    const int64_t b = blockIdx.x; // box at level D-2
    const int c = blockIdx.y;
    if (!A.keep && A.toff[64 * b] == A.toff[64 * b + 64])
        return; // no targets below this box: the main launch skips its children too
    for (int l = 2; l <= lt; ++l) {
        const int64_t anc = b >> (3 * (lt - l));
        if (l > 2)
            l2l1<P>(A.T, sPar, (int)(anc & 7), sOne, sPar);
        const int rl = A.rl[l];
        for (int k = t; k < rl; k += kThreads)
            load_ft(A, l, anc, c, sFt, 1, k);
        __syncthreads();
        const float *Ut = A.Ut[l];
        for (int i = t; i < P3; i += kThreads) {
            float a0 = 0.0f, a1 = 0.0f;
            int k = 0;
            for (; k + 1 < rl; k += 2) {
                a0 += sFt[k] * __ldg(Ut + (int64_t)k * A.p3p + i);
                a1 += sFt[k + 1] * __ldg(Ut + (int64_t)(k + 1) * A.p3p + i);
            }
            if (k < rl)
                a0 += sFt[k] * __ldg(Ut + (int64_t)k * A.p3p + i);
            const float f = (l > 2 ? sPar[i] : 0.0f) + (a0 + a1);
            sPar[i] = f;
            if (A.keep && (b & ((1LL << (3 * (lt - l))) - 1)) == 0)
                A.F[l][(anc * A.nrhs + c) * P3 + i] = f;
            if (l == lt)
                A.Ftop[(b * A.nrhs + c) * P3 + i] = f;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Wide upward pass: one block per (box of level D-2, right-hand side), i.e.
// 64 leaves and their 8 parents; used for depth >= kWideMinDepth and p <=
// kWideMaxP.  The 64 leaf coefficient sets sit as [p^3][64] in shared
// memory, so the compression GEMM reuses every operator element it loads for
// 8 boxes per thread and every coefficient load (two float4) for 3 columns.
template <int P> struct SmemW {
    static constexpr int P3 = P * P * P;
    // leaves [P3][64] | mids [P3][8] | top [P3] | scratch: max(basis 8 x 96 P, two [P3][8])
    static constexpr int kMid = 64 * P3;
    static constexpr int kTop = kMid + 8 * P3;
    static constexpr int kScr = (kTop + P3 + 3) & ~3;
    static constexpr int kScrN = 768 * P > 16 * P3 ? 768 * P : 16 * P3;
    static constexpr int kUpFloats = kScr + kScrN;
};

// P2M of leaf `leaf` (column `col` of X, row stride XS) by one warp
template <int P, int XS>
__device__ __forceinline__ void p2m_leaf(const PassArgs &A, int64_t leaf, int c, float *L, float *X, int col)
{
    constexpr int P3 = P * P * P;
    constexpr int NQ = (P * P + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int s0 = A.off[leaf], s1 = A.off[leaf + 1];
    float acc[NQ][P];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < P; ++i)
            acc[q][i] = 0.0f;
    for (int c0 = s0; c0 < s1; c0 += 32) {
        const int cnt = min(32, s1 - c0);
        __syncwarp();
        if (lane < cnt) {
            const float4 u = A.pts[c0 + lane];
            const float sg = A.sig[(int64_t)c * A.n + c0 + lane];
            float v[P];
            basis_1d<P>(A.T, 2.0f * u.x, v);
#pragma unroll
            for (int i = 0; i < P; ++i)
                L[lane * P + i] = v[i] * sg;
            basis_1d<P>(A.T, 2.0f * u.y, v);
#pragma unroll
            for (int i = 0; i < P; ++i)
                L[(32 + lane) * P + i] = v[i];
            basis_1d<P>(A.T, 2.0f * u.z, v);
#pragma unroll
            for (int i = 0; i < P; ++i)
                L[(64 + lane) * P + i] = v[i];
        }
        __syncwarp();
        for (int j = 0; j < cnt; ++j) {
            float lx[P];
#pragma unroll
            for (int i = 0; i < P; ++i)
                lx[i] = L[j * P + i];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int pq = lane + 32 * q;
                if (pq < P * P) {
                    const float yz = L[(32 + j) * P + pq % P] * L[(64 + j) * P + pq / P];
#pragma unroll
                    for (int i = 0; i < P; ++i)
                        acc[q][i] += lx[i] * yz;
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int pq = lane + 32 * q;
        if (pq < P * P) {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int idx = i + P * pq;
                X[idx * XS + col] = acc[q][i];
                if (A.keep)
                    A.M[A.D][(leaf * A.nrhs + c) * P3 + idx] = acc[q][i];
            }
        }
    }
}

// compress the 64 leaves (columns of X [P3][64]) of box B at level D: thread
// (kg = t % 32, bg = t / 32) makes coefficients k = k0 + 3 kg + {0, 1, 2} of
// boxes 8 bg .. 8 bg + 7
template <int P>
__device__ void compress64(const PassArgs &A, const float *X, int64_t B, int c, bool zero)
{
    constexpr int P3 = P * P * P;
    const int t = threadIdx.x, kg = t & 31, bg = t >> 5;
    const int l = A.D, H = 1 << (l - 1);
    const float *V = A.V[l];
    float mx = 0.0f;
    for (int k0 = 0; k0 < A.rl[l]; k0 += 96) {
        const int kb = k0 + 3 * kg;
        float acc[3][8];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                acc[j][b] = 0.0f;
        if (!zero) {
#pragma unroll 2
            for (int i = 0; i < P3; ++i) {
                const float *vr = V + (int64_t)i * A.rp;
                const float v0 = kb < A.rl[l] ? __ldg(vr + kb) : 0.0f;
                const float v1 = kb + 1 < A.rl[l] ? __ldg(vr + kb + 1) : 0.0f;
                const float v2 = kb + 2 < A.rl[l] ? __ldg(vr + kb + 2) : 0.0f;
                const float4 m0 = *reinterpret_cast<const float4 *>(X + i * 64 + 8 * bg);
                const float4 m1 = *reinterpret_cast<const float4 *>(X + i * 64 + 8 * bg + 4);
                const float m[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    acc[0][b] += m[b] * v0;
                    acc[1][b] += m[b] * v1;
                    acc[2][b] += m[b] * v2;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            int x, y, z;
            demorton3((uint32_t)(64 * B + 8 * bg + b), x, y, z);
            const int64_t row = parity_row(x, y, z, c, H, 1, A.R) * A.rp;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (kb + j < A.rl[l])
                    put_mt(A, l, row + kb + j, acc[j][b], mx);
        }
    }
    flush_max(A, l, mx);
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_upward_wide(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P;
    extern __shared__ __align__(16) float sm[];
    float *sLeaf = sm;
    float *sMid = sm + SmemW<P>::kMid;
    float *sTop = sm + SmemW<P>::kTop;
    float *sScr = sm + SmemW<P>::kScr;
    __shared__ int sLast;
    const int t = threadIdx.x, w = t >> 5;
    const int D = A.D;
    const int64_t B = blockIdx.x; // box at level D-2
    const int c = blockIdx.y;
    const bool zero = A.off[64 * B] == A.off[64 * B + 64];

    // P2M: warp w makes leaves 64 B + 8 j + w, j = 0..7 (column 8 j + w)
    for (int j = 0; j < 8; ++j)
        p2m_leaf<P, 64>(A, 64 * B + 8 * j + w, c, sScr + w * 96 * P, sLeaf, 8 * j + w);
    __syncthreads();
    if (!A.Mleaf)
        compress64<P>(A, sLeaf, B, c, zero);
    else if (!zero)
        store_leaves<P, 64>(A, sLeaf, 64 * B, 64, c);
    // the 8 boxes of level D-1: M2M of their leaves, compression
    for (int m = 0; m < 8; ++m)
        m2m8<P, 64, 8>(A.T, sLeaf + 8 * m, sScr, sScr + 8 * P3, sMid + m);
    if (A.keep)
        for (int q = t; q < 8 * P3; q += kThreads)
            A.M[D - 1][((8 * B + (q & 7)) * A.nrhs + c) * P3 + (q >> 3)] = sMid[q];
    if (!A.Mlev1)
        compress8<P>(A, D - 1, sMid, 8 * B, c, zero);
    else if (!zero) // compressed by the GEMM after this launch
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q / P3, i = q - o * P3;
            A.Mlev1[((int64_t)c * (1LL << (3 * (D - 1))) + 8 * B + o) * A.p3p + i] = sMid[i * 8 + o];
        }
    if (D - 2 < 2)
        return;
    // the block's own box (level D-2)
    m2m8<P>(A.T, sMid, sScr, sScr + 8 * P3, sTop);
    for (int r = t; r < P3; r += kThreads)
        A.M[D - 2][(B * A.nrhs + c) * P3 + r] = sTop[r];
    compress1<P>(A, D - 2, sTop, B, c);

    // upper levels: the last of 8 siblings to arrive makes the parent
    int64_t box = B;
    for (int l = D - 3; l >= 2; --l) {
        const int64_t par = box >> 3;
        // the barrier orders every thread's stores of the level-(l+1) box
        // before thread 0's fence, which makes them visible device-wide
        // before its arrival is counted
        __syncthreads();
        if (t == 0) {
            __threadfence();
            int *cnt = A.count[l] + par * A.R + c;
            const int before = atomicAdd(cnt, 1);
            sLast = before == 7;
            if (before == 7) {
                atomicExch(cnt, 0); // ready for the next matvec
                __threadfence();
            }
        }
        __syncthreads();
        if (!sLast)
            return;
        const float *Mc = A.M[l + 1] + (8 * par * A.nrhs + c) * (int64_t)P3;
        for (int q = t; q < 8 * P3; q += kThreads) {
            const int o = q & 7, r = q >> 3;
            sMid[q] = __ldcg(Mc + (int64_t)o * A.nrhs * P3 + r);
        }
        __syncthreads();
        m2m8<P>(A.T, sMid, sScr, sScr + 8 * P3, sTop);
        for (int r = t; r < P3; r += kThreads)
            A.M[l][(par * A.nrhs + c) * P3 + r] = sTop[r];
        compress1<P>(A, l, sTop, par, c);
        box = par;
    }
}

// ---------------------------------------------------------------------------
// Several right-hand sides (Sec. 2.5 "Multiple right-hand-sides"): the same
// passes with a block per (box, chunk of RC columns).  The basis values of a
// leaf's points, every operator element a compression or decompression loads
// and every transfer matrix are shared by RC columns, and each phase between
// two barriers has RC times the lines of the one-column kernels.  With a block
// per (box, column) the passes were bound by the latency of their short
// phases (3.4 ms each way for 500k points x 64 columns at depth 5).
//
// Shared-memory layouts (floats): X [RC][8][P3] (8 sibling boxes of each
// column, a box's coefficients contiguous: P2M's lanes, 5 coefficients
// apart, and the rows stored for the compression GEMM meet distinct banks);
// P [P3][RC] (one box, the
// columns side by side, so one vector load gives a thread its columns);
// the leaves' local coefficients in the downward pass [8][P3][RC] (L2P reads
// a leaf's RC columns of one coefficient with one vector load; the far-field
// rows are added by lanes that run over (column, coefficient), 32 banks apart).
template <int P> constexpr int kRC = P <= 5 ? 8 : (P <= 7 ? 4 : 2);

template <int P> struct SmemRC {
    static constexpr int P3 = P * P * P, RC = kRC<P>;
    // upward: X | Y (the P2M basis scratch 256 x (3P + RC) aliases it) | P
    static constexpr int kUpY = 8 * P3 * RC;
    static constexpr int kUpYN = 8 * P3 * RC > 256 * (3 * P + RC) ? 8 * P3 * RC : 256 * (3 * P + RC);
    static constexpr int kUpPar = kUpY + kUpYN;
    static constexpr int kUpFloats = kUpPar + P3 * RC;
    // downward: leaves [8][P3][RC] (the L2L's Y [RC][2][P3] aliases them: Y
    // is dead before the L2L's last pass writes the leaves) | Z [RC][4][P3]
    // (the ancestors' scratch P and F~ [r][RC] alias it) | P
    static constexpr int kDnY = 0, kDnZ = 8 * P3 * RC, kDnOne = 8 * P3 * RC, kDnFt = 9 * P3 * RC,
                         kDnPar = 12 * P3 * RC, kDnFloats = 13 * P3 * RC;
    static_assert(kDnPar % 2 == 0 && kUpPar % 2 == 0, "vector loads of the column sets");
};

// N consecutive floats of shared memory (N = 1, 2, 4, 8; aligned to N)
template <int N>
__device__ __forceinline__ void ldv(const float *p, float (&v)[N])
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 f = reinterpret_cast<const float4 *>(p)[q];
            v[4 * q] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
    } else if constexpr (N == 2) {
        const float2 f = *reinterpret_cast<const float2 *>(p);
        v[0] = f.x;
        v[1] = f.y;
    } else {
        v[0] = p[0];
    }
}

// P2M of leaf `leaf` for columns c0 .. c0 + RC - 1 (nc of them real) by one
// warp, into box leaf & 7 of X [RC][8][P3]; L: the warp's 32 x (3P + RC)
// scratch (basis values of 32 points, then their RC weights)
template <int P, int RC>
__device__ __forceinline__ void p2m_leaf_rc(const PassArgs &A, int64_t leaf, int c0, int nc, float *L, float *X)
{
    constexpr int P3 = P * P * P, NQ = (P * P + 31) / 32, LS = 3 * P + RC;
    const int lane = threadIdx.x & 31, o = (int)(leaf & 7);
    const int s0 = A.off[leaf], s1 = A.off[leaf + 1];
    float acc[NQ][RC][P];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < RC; ++c)
#pragma unroll
            for (int i = 0; i < P; ++i)
                acc[q][c][i] = 0.0f;
    for (int j0 = s0; j0 < s1; j0 += 32) {
        const int cnt = min(32, s1 - j0);
        __syncwarp();
        if (lane < cnt) {
            const float4 u = A.pts[j0 + lane];
            float *Lr = L + lane * LS;
            basis_1d<P>(A.T, 2.0f * u.x, Lr);
            basis_1d<P>(A.T, 2.0f * u.y, Lr + P);
            basis_1d<P>(A.T, 2.0f * u.z, Lr + 2 * P);
#pragma unroll
            for (int c = 0; c < RC; ++c)
                Lr[3 * P + c] = c < nc ? A.sig[(int64_t)(c0 + c) * A.n + j0 + lane] : 0.0f;
        }
        __syncwarp();
        for (int j = 0; j < cnt; ++j) {
            const float *Lr = L + j * LS;
            float lx[P], sg[RC];
#pragma unroll
            for (int i = 0; i < P; ++i)
                lx[i] = Lr[i];
#pragma unroll
            for (int c = 0; c < RC; ++c)
                sg[c] = Lr[3 * P + c];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int pq = lane + 32 * q;
                if (pq < P * P) {
                    const float yz = Lr[P + pq % P] * Lr[2 * P + pq / P];
#pragma unroll
                    for (int c = 0; c < RC; ++c) {
                        const float s = sg[c] * yz;
#pragma unroll
                        for (int i = 0; i < P; ++i)
                            acc[q][c][i] += lx[i] * s;
                    }
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int pq = lane + 32 * q;
        if (pq < P * P) {
#pragma unroll
            for (int c = 0; c < RC; ++c)
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const int idx = i + P * pq;
                    X[(c * 8 + o) * P3 + idx] = acc[q][c][i];
                    if (A.keep && c < nc)
                        A.M[A.D][(leaf * A.nrhs + c0 + c) * P3 + idx] = acc[q][c][i];
                }
        }
    }
}

// M2M of 8 children, RC columns: X [RC][8][P3] -> out [P3][RC]; scratch Y
// [RC][P3][8] and Z [RC][P3][4] (Z may alias X: X is read by the first pass only)
template <int P, int RC>
__device__ void m2m8_rc(const InterpTables &T, const float *X, float *Y, float *Z, float *out)
{
    constexpr int P2 = P * P, P3 = P2 * P;
    const int t = threadIdx.x;
    for (int q = t; q < RC * 8 * P2; q += kThreads) { // x pass: line (child o, j2 + P j3, column)
        const int o = q & 7, u = q >> 3, rest = u % P2, c = u / P2;
        const float *Xc = X + (c * 8 + o) * P3 + P * rest;
        float x[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            x[j] = Xc[j];
        float *Yc = Y + c * 8 * P3;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][i][j] * x[j];
            Yc[(i + P * rest) * 8 + o] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * 4 * P2; q += kThreads) { // y pass: x pairs summed
        const int yz = q & 3, u = q >> 2, v = u % P2, c = u / P2, i1 = v % P, j3 = v / P;
        const float *Yc = Y + c * 8 * P3;
        float y[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float *src = Yc + (i1 + P * j + P2 * j3) * 8 + 2 * yz;
            y[j] = src[0] + src[1];
        }
        float *Zc = Z + c * 4 * P3;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[yz & 1][i][j] * y[j];
            Zc[(i1 + P * i + P2 * j3) * 4 + yz] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * P2; q += kThreads) { // z pass: y pairs summed
        const int v = q % P2, c = q / P2;
        const float *Zc = Z + c * 4 * P3;
        float z0[P], z1[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float *src = Zc + (v + P2 * j) * 4;
            z0[j] = src[0] + src[1];
            z1[j] = src[2] + src[3];
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[0][i][j] * z0[j] + T.S[1][i][j] * z1[j];
            out[(v + P2 * i) * RC + c] = a;
        }
    }
    __syncthreads();
}

// L2L of a parent F [P3][RC] into its child o only, in place allowed (out may
// be F); scratch Y [P3][RC]
template <int P, int RC>
__device__ void l2l1_rc(const InterpTables &T, const float *F, int o, float *Y, float *out)
{
    constexpr int P2 = P * P;
    const int t = threadIdx.x;
    for (int q = t; q < RC * P2; q += kThreads) { // z pass: line (j1 + P j2, column)
        const int c = q % RC, v = q / RC;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = F[(v + P2 * j) * RC + c];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o >> 2][j][i] * f[j];
            Y[(v + P2 * i) * RC + c] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * P2; q += kThreads) { // y pass: line (j1, i3, column), into out
        const int c = q % RC, v = q / RC, j1 = v % P, i3 = v / P;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = Y[(j1 + P * j + P2 * i3) * RC + c];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[(o >> 1) & 1][j][i] * f[j];
            out[(j1 + P * i + P2 * i3) * RC + c] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * P2; q += kThreads) { // x pass: line (i2 + P i3, column), in place
        const int c = q % RC, v = q / RC;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = out[(P * v + j) * RC + c];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][j][i] * f[j];
            out[(P * v + i) * RC + c] = a;
        }
    }
    __syncthreads();
}

// L2L of one parent F [P3][RC] into its 8 children out [8][P3][RC]; scratch
// Y [RC][2][P3], Z [RC][4][P3]
template <int P, int RC>
__device__ void l2l8_rc(const InterpTables &T, const float *F, float *Y, float *Z, float *out)
{
    constexpr int P2 = P * P, P3 = P2 * P;
    const int t = threadIdx.x;
    for (int q = t; q < RC * 2 * P2; q += kThreads) { // z pass: line (oz, j1 + P j2, column)
        const int c = q % RC, u = q / RC, oz = u & 1, j12 = u >> 1;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = F[(j12 + P2 * j) * RC + c];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[oz][j][i] * f[j];
            Y[(c * 2 + oz) * P3 + j12 + P2 * i] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * 4 * P2; q += kThreads) { // y pass: line (oy + 2 oz, j1, i3, column)
        const int c = q % RC, u = q / RC, yz = u & 3, v = u >> 2, j1 = v % P, i3 = v / P;
        const float *src = Y + (c * 2 + (yz >> 1)) * P3 + j1 + P2 * i3;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = src[P * j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[yz & 1][j][i] * f[j];
            Z[(c * 4 + yz) * P3 + j1 + P * i + P2 * i3] = a;
        }
    }
    __syncthreads();
    for (int q = t; q < RC * 8 * P2; q += kThreads) { // x pass: line (child o, i2 + P i3, column)
        const int c = q % RC, u = q / RC, o = u & 7, rest = u >> 3;
        const float *src = Z + (c * 4 + (o >> 1)) * P3 + P * rest;
        float f[P];
#pragma unroll
        for (int j = 0; j < P; ++j)
            f[j] = src[j];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j)
                a += T.S[o & 1][j][i] * f[j];
            out[(o * P3 + i + P * rest) * RC + c] = a;
        }
    }
    __syncthreads();
}

// compress one box at level l, RC columns of X [P3][RC]: thread (k, half h)
// makes columns RC/2 h .. RC/2 h + RC/2 - 1 of coefficient k
template <int P, int RC>
__device__ void compress1_rc(const PassArgs &A, int l, const float *X, int64_t box, int c0, int nc)
{
    constexpr int P3 = P * P * P, CPT = RC / 2;
    const int t = threadIdx.x, kk = t & 127, h = t >> 7;
    const int H = 1 << (l - 1);
    const float *V = A.V[l];
    int x, y, z;
    demorton3((uint32_t)box, x, y, z);
    float mx = 0.0f;
    for (int k0 = 0; k0 < A.rl[l]; k0 += 128) { // uniform trip count (warp shuffles in flush_max)
        const int k = k0 + kk;
        if (k < A.rl[l]) {
            float acc[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                acc[j] = 0.0f;
#pragma unroll 5
            for (int i = 0; i < P3; ++i) {
                const float v = __ldg(V + (int64_t)i * A.rp + k);
                float m[CPT];
                ldv<CPT>(X + i * RC + h * CPT, m);
#pragma unroll
                for (int j = 0; j < CPT; ++j)
                    acc[j] += m[j] * v;
            }
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int c = h * CPT + j;
                if (c < nc)
                    put_mt(A, l, parity_row(x, y, z, c0 + c, H, 1, A.R) * A.rp + k, acc[j], mx);
            }
        }
    }
    flush_max(A, l, mx);
}

// local coefficients of one box at level l, RC columns: sPar [P3][RC] (the
// L2L part when add, else 0) + U F~ with F~ [r][RC] in sFt; with keep also
// stored to F[l] (when `store`)
template <int P, int RC>
__device__ void decompress1_rc(const PassArgs &A, int l, const float *sFt, float *sPar, bool add, int64_t box,
                               int c0, int nc, bool store)
{
    constexpr int P3 = P * P * P, CPT = RC / 2;
    const int t = threadIdx.x, h = t >> 7;
    const int rl = A.rl[l];
    const float *Ut = A.Ut[l];
    for (int i0 = 0; i0 < P3; i0 += 128) {
        const int i = i0 + (t & 127);
        if (i < P3) {
            float acc[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                acc[j] = 0.0f;
#pragma unroll 4
            for (int k = 0; k < rl; ++k) {
                const float u = __ldg(Ut + (int64_t)k * A.p3p + i);
                float f[CPT];
                ldv<CPT>(sFt + k * RC + h * CPT, f);
#pragma unroll
                for (int j = 0; j < CPT; ++j)
                    acc[j] += f[j] * u;
            }
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int c = h * CPT + j;
                const float f = (add ? sPar[i * RC + c] : 0.0f) + acc[j];
                sPar[i * RC + c] = f;
                if (store && c < nc)
                    A.F[l][(box * A.nrhs + c0 + c) * P3 + i] = f;
            }
        }
    }
}

// F~ of one box at level l, RC columns (slices summed), into sFt [r][RC]
template <int RC>
__device__ __forceinline__ void load_ft_rc(const PassArgs &A, int l, int64_t box, int c0, int nc, float *sFt)
{
    const int rl = A.rl[l];
    for (int q = threadIdx.x; q < rl * RC; q += kThreads) {
        const int c = q % RC, k = q / RC;
        if (c < nc)
            load_ft(A, l, box, c0 + c, sFt + c, RC, k);
        else
            sFt[q] = 0.0f;
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_upward_rc(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P, RC = kRC<P>;
    extern __shared__ __align__(16) float sm[];
    float *sX = sm, *sY = sm + SmemRC<P>::kUpY, *sPar = sm + SmemRC<P>::kUpPar;
    __shared__ int sLast;
    const int t = threadIdx.x, w = t >> 5;
    const int D = A.D;
    const int64_t b = blockIdx.x; // box at level D-1
    const int c0 = blockIdx.y * RC, nc = min(RC, A.nrhs - c0);
    const int64_t leaf = 8 * b + w, nb = 1LL << (3 * D);
    const bool zero = __syncthreads_count(A.off[leaf + 1] > A.off[leaf]) == 0;

    // ---- P2M: warp w makes M of leaf 8b + w for the chunk's columns
    p2m_leaf_rc<P, RC>(A, leaf, c0, nc, sY + w * 32 * (3 * P + RC), sX);
    __syncthreads();
    // ---- the leaves' compression, or their rows for the compression GEMM
    if (!A.Mleaf) {
        for (int c = 0; c < nc; ++c)
            compress8<P, true>(A, D, sX + c * 8 * P3, 8 * b, c0 + c, zero);
    } else if (!zero) {
        for (int q = t; q < nc * 8 * P3; q += kThreads) {
            const int i = q % P3, u = q / P3; // u = 8 c + o
            A.Mleaf[((int64_t)(c0 + (u >> 3)) * nb + 8 * b + (u & 7)) * A.p3p + i] = sX[q];
        }
    }
    if (D - 1 < 2)
        return;

    // ---- own box at level D-1 (the M2M's third pass overwrites X: the
    // compression above read it before the M2M's first barrier)
    if (zero) {
        for (int r = t; r < P3 * RC; r += kThreads)
            sPar[r] = 0.0f;
        __syncthreads();
    } else {
        m2m8_rc<P, RC>(A.T, sX, sY, sX, sPar);
    }
    for (int q = t; q < nc * P3; q += kThreads) {
        const int r = q % P3, c = q / P3;
        A.M[D - 1][(b * A.nrhs + c0 + c) * P3 + r] = sPar[r * RC + c];
    }
    if (A.Mlev1) // compressed by the GEMM after this launch
        for (int q = t; q < nc * P3; q += kThreads) {
            const int r = q % P3, c = q / P3;
            A.Mlev1[((int64_t)(c0 + c) * (1LL << (3 * (D - 1))) + b) * A.p3p + r] = sPar[r * RC + c];
        }
    else
        compress1_rc<P, RC>(A, D - 1, sPar, b, c0, nc);

    // ---- upper levels: the last of 8 siblings to arrive makes the parent
    int64_t box = b;
    for (int l = D - 2; l >= 2; --l) {
        const int64_t par = box >> 3;
        // the barrier orders every thread's stores of the level-(l+1) box
        // before thread 0's fence, which makes them visible device-wide
        // before its arrival is counted
        __syncthreads();
        if (t == 0) {
            __threadfence();
            int *cnt = A.count[l] + par * A.R + c0; // one counter per (box, chunk)
            const int before = atomicAdd(cnt, 1);
            sLast = before == 7;
            if (before == 7) {
                atomicExch(cnt, 0); // ready for the next matvec
                __threadfence();
            }
        }
        __syncthreads();
        if (!sLast)
            return;
        for (int q = t; q < RC * 8 * P3; q += kThreads) {
            const int r = q % P3, o = (q / P3) & 7, c = q / (8 * P3);
            sX[q] = c < nc ? __ldcg(A.M[l + 1] + ((8 * par + o) * A.nrhs + c0 + c) * (int64_t)P3 + r) : 0.0f;
        }
        __syncthreads();
        m2m8_rc<P, RC>(A.T, sX, sY, sX, sPar);
        for (int q = t; q < nc * P3; q += kThreads) {
            const int r = q % P3, c = q / P3;
            A.M[l][(par * A.nrhs + c0 + c) * P3 + r] = sPar[r * RC + c];
        }
        compress1_rc<P, RC>(A, l, sPar, par, c0, nc);
        box = par;
    }
}

// first downward launch (depth >= 4), several columns: block = (box of level
// D-2, chunk of RC columns)
template <int P>
__global__ void __launch_bounds__(kThreads) k_down_top_rc(const __grid_constant__ PassArgs A)
{
    constexpr int P3 = P * P * P, RC = kRC<P>;
    extern __shared__ __align__(16) float sm[];
    float *sPar = sm, *sOne = sm + P3 * RC, *sFt = sm + 2 * P3 * RC;
    const int t = threadIdx.x;
    const int D = A.D, lt = D - 2;
    const int64_t b = blockIdx.x; // box at level D-2
    const int c0 = blockIdx.y * RC, nc = min(RC, A.nrhs - c0);
    if (!A.keep && A.toff[64 * b] == A.toff[64 * b + 64])
        return; // no targets below this box: the main launch skips its children too
    for (int l = 2; l <= lt; ++l) {
        const int64_t anc = b >> (3 * (lt - l));
        if (l > 2)
            l2l1_rc<P, RC>(A.T, sPar, (int)(anc & 7), sOne, sPar);
        load_ft_rc<RC>(A, l, anc, c0, nc, sFt);
        __syncthreads();
        const bool store = A.keep && (b & ((1LL << (3 * (lt - l))) - 1)) == 0;
        decompress1_rc<P, RC>(A, l, sFt, sPar, l > 2, anc, c0, nc, store);
        __syncthreads();
    }
    for (int q = t; q < nc * P3; q += kThreads) {
        const int i = q % P3, c = q / P3;
        A.Ftop[(b * A.nrhs + c0 + c) * P3 + i] = sPar[i * RC + c];
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_downward_rc(const __grid_constant__ PassArgs A)
{
    constexpr int P2 = P * P, P3 = P2 * P, RC = kRC<P>;
    extern __shared__ __align__(16) float sm[];
    float *sMT = sm;                        // [8][P3][RC] the leaves' local coefficients
    float *sY = sm + SmemRC<P>::kDnY;       // [RC][2][P3] L2L scratch (aliases the leaves)
    float *sZ = sm + SmemRC<P>::kDnZ;       // [RC][4][P3] L2L scratch
    float *sPar = sm + SmemRC<P>::kDnPar;   // [P3][RC] the current ancestor
    float *sOne = sm + SmemRC<P>::kDnOne;   // [P3][RC] ancestors' scratch (aliases Z)
    float *sFt = sm + SmemRC<P>::kDnFt;     // [r][RC] compressed far field of the current ancestor (aliases Z)
    __shared__ int64_t sRow[8 * RC];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int D = A.D;
    const int64_t b = blockIdx.x; // box at level D-1
    const int c0 = blockIdx.y * RC, nc = min(RC, A.nrhs - c0);
    if (!A.keep && A.toff[8 * b] == A.toff[8 * b + 8])
        return; // no targets below this box

    // ---- ancestors at levels 2 .. D-1 (with Ftop: the parent from the first launch)
    int l0 = 2;
    if (A.Ftop) {
        for (int q = t; q < P3 * RC; q += kThreads) {
            const int i = q / RC, c = q % RC;
            sPar[q] = c < nc ? __ldcg(A.Ftop + ((b >> 3) * A.nrhs + c0 + c) * (int64_t)P3 + i) : 0.0f;
        }
        __syncthreads();
        l0 = D - 1;
    }
    for (int l = l0; l <= D - 1; ++l) {
        const int64_t anc = b >> (3 * (D - 1 - l));
        if (l > 2)
            l2l1_rc<P, RC>(A.T, sPar, (int)(anc & 7), sOne, sPar);
        if (l == D - 1 && A.Fdec1) {
            // the block's own box, decompressed by the GEMM before this launch
            if (t < RC) {
                int x, y, z;
                demorton3((uint32_t)anc, x, y, z);
                sRow[t] = t < nc ? parity_row(x, y, z, c0 + t, 1 << (l - 1), 0, A.R) : -1;
            }
            __syncthreads();
            for (int q = t; q < nc * P3; q += kThreads) {
                const int i = q % P3, c = q / P3;
                const float f = (l > 2 ? sPar[i * RC + c] : 0.0f) + __ldg(A.Fdec1 + sRow[c] * A.p3p + i);
                sPar[i * RC + c] = f;
                if (A.keep)
                    A.F[l][(anc * A.nrhs + c0 + c) * P3 + i] = f;
            }
            __syncthreads();
            continue;
        }
        load_ft_rc<RC>(A, l, anc, c0, nc, sFt);
        __syncthreads();
        const bool store = A.keep && (b & ((1LL << (3 * (D - 1 - l))) - 1)) == 0;
        decompress1_rc<P, RC>(A, l, sFt, sPar, l > 2, anc, c0, nc, store);
        __syncthreads();
    }

    // ---- the 8 leaves: L2L from the block's box plus their own far field
    if (D - 1 >= 2) {
        l2l8_rc<P, RC>(A.T, sPar, sY, sZ, sMT);
    } else {
        for (int q = t; q < 8 * P3 * RC; q += kThreads)
            sMT[q] = 0.0f;
        __syncthreads();
    }
    if (t < 8 * RC) {
        const int o = t & 7, c = t >> 3;
        int x, y, z;
        demorton3((uint32_t)(8 * b + o), x, y, z);
        sRow[t] = c < nc ? parity_row(x, y, z, c0 + c, 1 << (D - 1), 0, A.R) : -1;
    }
    __syncthreads();
    if (A.Fdec) {
        // decompressed by the GEMM before this launch
#pragma unroll 4
        for (int q = t; q < 8 * P3 * RC; q += kThreads) {
            const int c = q % RC, u = q / RC, i = u % P3, o = u / P3;
            if (c < nc)
                sMT[q] += __ldg(A.Fdec + sRow[8 * c + o] * A.p3p + i);
        }
    } else {
        // per column: the 8 leaves' F~ [r][8] (in Z, free after the L2L)
        // decompressed on the CUDA cores, 4 leaves per thread
        float *sF8 = sZ;
        const float *Ut = A.Ut[D];
        const int h = t >> 7, rl = A.rl[D];
        for (int c = 0; c < nc; ++c) {
            for (int q = t; q < 8 * rl; q += kThreads) {
                const int o = q & 7, k = q >> 3;
                const float *src = A.Ft[D] + sRow[8 * c + o] * A.rp + k;
                float v = __ldg(src);
                for (int g = 1; g < A.nslices; ++g)
                    v += __ldg(src + g * A.slice[D]);
                sF8[k * 8 + o] = v;
            }
            __syncthreads();
            for (int i0 = 0; i0 < P3; i0 += 128) {
                const int i = i0 + (t & 127);
                if (i < P3) {
                    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
                    for (int k = 0; k < rl; ++k) {
                        const float u = __ldg(Ut + (int64_t)k * A.p3p + i);
                        const float4 f = *reinterpret_cast<const float4 *>(sF8 + k * 8 + 4 * h);
                        acc[0] += f.x * u;
                        acc[1] += f.y * u;
                        acc[2] += f.z * u;
                        acc[3] += f.w * u;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        sMT[((4 * h + q) * P3 + i) * RC + c] += acc[q];
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (A.keep)
        for (int q = t; q < 8 * P3 * nc; q += kThreads) {
            const int r = q % P3, u = q / P3, o = u & 7, c = u >> 3;
            A.F[D][((8 * b + o) * A.nrhs + c0 + c) * P3 + r] = sMT[(o * P3 + r) * RC + c];
        }

    // ---- L2P: warp w evaluates leaf 8b + w at its targets, RC columns
    const int64_t leaf = 8 * b + w;
    const int s0 = A.toff[leaf], s1 = A.toff[leaf + 1];
    for (int j0 = s0; j0 < s1; j0 += 32) {
        const int j = j0 + lane;
        const bool has = j < s1;
        const float4 u = A.tpts[has ? j : s0];
        float Lx[P], Ly[P];
        basis_1d<P>(A.T, 2.0f * u.x, Lx);
        basis_1d<P>(A.T, 2.0f * u.y, Ly);
        const float sz = 2.0f * u.z;
        float acc[RC];
#pragma unroll
        for (int c = 0; c < RC; ++c)
            acc[c] = 0.0f;
#pragma unroll 1
        for (int i3 = 0; i3 < P; ++i3) {
            float lz = A.T.wbary[i3];
#pragma unroll
            for (int k = 0; k < P; ++k)
                lz *= k != i3 ? sz - A.T.nodes[k] : 1.0f;
            const float *Fz = sMT + (w * P3 + P2 * i3) * RC;
            float slice[RC];
#pragma unroll
            for (int c = 0; c < RC; ++c)
                slice[c] = 0.0f;
#pragma unroll
            for (int i2 = 0; i2 < P; ++i2) {
                float part[RC];
#pragma unroll
                for (int c = 0; c < RC; ++c)
                    part[c] = 0.0f;
#pragma unroll
                for (int i1 = 0; i1 < P; ++i1) {
                    float f[RC];
                    ldv<RC>(Fz + (i1 + P * i2) * RC, f);
#pragma unroll
                    for (int c = 0; c < RC; ++c)
                        part[c] += f[c] * Lx[i1];
                }
#pragma unroll
                for (int c = 0; c < RC; ++c)
                    slice[c] += part[c] * Ly[i2];
            }
#pragma unroll
            for (int c = 0; c < RC; ++c)
                acc[c] += slice[c] * lz;
        }
        if (has)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (c < nc)
                    A.phi[(int64_t)(c0 + c) * A.nt + j] = acc[c];
    }
}

template <int P>
cudaError_t upward_p(const PassArgs &A, cudaStream_t s)
{
    if (A.nrhs > 1) {
        const size_t smem = sizeof(float) * SmemRC<P>::kUpFloats;
        cudaError_t e =
            cudaFuncSetAttribute(k_upward_rc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        dim3 grid((unsigned)(1LL << (3 * (A.D - 1))), (unsigned)((A.nrhs + kRC<P> - 1) / kRC<P>));
        k_upward_rc<P><<<grid, kThreads, smem, s>>>(A);
        return cudaGetLastError();
    }
    if (P <= kWideMaxP && A.D >= kWideMinDepth && !A.Mleaf) {
        const size_t smem = sizeof(float) * SmemW<P>::kUpFloats;
        cudaError_t e =
            cudaFuncSetAttribute(k_upward_wide<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        dim3 grid((unsigned)(1LL << (3 * (A.D - 2))), (unsigned)A.nrhs);
        k_upward_wide<P><<<grid, kThreads, smem, s>>>(A);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(float) * Smem<P>::kUpFloats;
    cudaError_t e = cudaFuncSetAttribute(k_upward<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)(1LL << (3 * (A.D - 1))), (unsigned)A.nrhs);
    k_upward<P><<<grid, kThreads, smem, s>>>(A);
    return cudaGetLastError();
}

template <int P>
cudaError_t downward_p(const PassArgs &A, cudaStream_t s)
{
    if (A.nrhs > 1) {
        const unsigned chunks = (unsigned)((A.nrhs + kRC<P> - 1) / kRC<P>);
        if (A.Ftop) {
            if (A.D < 4)
                return cudaErrorInvalidValue;
            const size_t smem = sizeof(float) * 3 * P * P * P * kRC<P>;
            cudaError_t e =
                cudaFuncSetAttribute(k_down_top_rc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return e;
            dim3 grid((unsigned)(1LL << (3 * (A.D - 2))), chunks);
            k_down_top_rc<P><<<grid, kThreads, smem, s>>>(A);
            e = cudaGetLastError();
            if (e != cudaSuccess)
                return e;
        }
        const size_t smem = sizeof(float) * SmemRC<P>::kDnFloats;
        cudaError_t e =
            cudaFuncSetAttribute(k_downward_rc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        dim3 grid((unsigned)(1LL << (3 * (A.D - 1))), chunks);
        k_downward_rc<P><<<grid, kThreads, smem, s>>>(A);
        return cudaGetLastError();
    }
    if (A.Ftop) {
        if (A.D < 4)
            return cudaErrorInvalidValue;
        dim3 grid((unsigned)(1LL << (3 * (A.D - 2))), (unsigned)A.nrhs);
        k_down_top<P><<<grid, kThreads, sizeof(float) * 3 * P * P * P, s>>>(A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    const size_t smem = sizeof(float) * Smem<P>::kDownFloats;
    cudaError_t e = cudaFuncSetAttribute(k_downward<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)(1LL << (3 * (A.D - 1))), (unsigned)A.nrhs);
    k_downward<P><<<grid, kThreads, smem, s>>>(A);
    return cudaGetLastError();
}

} // namespace

#define BBFMM_PASS_DISPATCH(p, F)                                                                               \
    switch (p) {                                                                                                \
    case 2: return F<2>(A, s);                                                                                  \
    case 3: return F<3>(A, s);                                                                                  \
    case 4: return F<4>(A, s);                                                                                  \
    case 5: return F<5>(A, s);                                                                                  \
    case 6: return F<6>(A, s);                                                                                  \
    case 7: return F<7>(A, s);                                                                                  \
    case 8: return F<8>(A, s);                                                                                  \
    case 9: return F<9>(A, s);                                                                                  \
    case 10: return F<10>(A, s);                                                                                \
    default: return cudaErrorInvalidValue;                                                                      \
    }

cudaError_t launch_upward(const PassArgs &A, int p, cudaStream_t s)
{
    if (A.D < 2 || A.r > p * p * p || A.nrhs < 1 || A.nrhs > A.R)
        return cudaErrorInvalidValue;
    BBFMM_PASS_DISPATCH(p, upward_p)
}

cudaError_t launch_downward(const PassArgs &A, int p, cudaStream_t s)
{
    if (A.D < 2 || A.r > p * p * p || A.nrhs < 1 || A.nrhs > A.R)
        return cudaErrorInvalidValue;
    BBFMM_PASS_DISPATCH(p, downward_p)
}

#undef BBFMM_PASS_DISPATCH

} // namespace bbfmm
