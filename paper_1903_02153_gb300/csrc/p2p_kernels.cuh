// p2p_kernels.cuh -- the near-field kernels (Sec. 2.3 item 4), templated on
// the kernel function.  Self-contained apart from morton.cuh: the library
// compiles it with nvcc for the built-in kernels, and at run time with NVRTC
// (its text is embedded at build time) for a user-supplied kernel.
//
//   phi_i += sum_{beta in N(alpha)} sum_{y_j in beta} K(x_i, y_j) sigma_j,
// N(alpha) = the up to 27 leaves adjacent to alpha, alpha included (Def. 2.1).
//
// Targets and sources are two point sets binned into the same leaves (the
// same arrays when the targets are the sources).  Work item = up to
// kP2PChunk consecutive targets of one leaf; one block of 128 threads per
// item.  The block first gathers the neighbour leaves' sources into shared
// memory (all threads at once, coalesced, kStageSrc at a time),
// with coordinates in the target leaf's cell units: y' = u_y + (cell_y -
// cell_x).  The offset is an exact small integer, so the FP32 difference
// u_x - y' only carries the rounding of u (|u| <= 1/2), not that of absolute
// coordinates.
//
// Each thread owns kTPT targets (two packed pairs by default) and evaluates
// them against every source it visits with the packed two-lane FP32
// instructions of sm_100+ (FADD2 / FMUL2 / FFMA2); a source is staged as
// (x, x, y, y), (z, z, s, s) so both halves of a packed operand come from one
// shared-memory broadcast.
// Threads are (target group, slice): slice s walks sources s, s + S, ...; the
// slices of a target are added in a fixed order at the end (deterministic).
// K at r = 0 follows the library's convention: 0 for 1/r and 1/r^2.
#pragma once

#include "morton.cuh"

namespace bbfmm {

constexpr int kP2PChunk = 128; // targets per work item (one block)
constexpr int kP2PThreads = 128;
constexpr int kStageSrc = 512; // staged sources per pass (16 KB): 8+ blocks per SM

// single hardware approximations (MUFU); distinct points never give a
// subnormal squared distance here (|u| <= 1.5, so r2 >= 2^-48 or r2 = 0)
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// each kernel maps the squared distance r2 (cell units) and the offsets to
// K; the packed form applies it to both lanes.  one() follows the r = 0
// convention (0 for the singular kernels) and serves the target's own leaf,
// the only place where a point meets itself or an exact duplicate; far()
// serves the other 26 leaves.  There r2 = 0 could only come from FP32
// rounding of two distinct points closer than ~1e-7 cells, so the kernel
// adds kR2Floor = 2^-48 (cell units squared) to r2 instead of testing it:
// 1/r stays below 2^24 / h, and the shift is 1e-14 of any r2 that can occur.
constexpr float kR2Floor = 3.5527136788005009e-15f; // 2^-48
struct KInvR {
    float a; // unused
    __device__ float one(float r2, float, float, float) const { return r2 > 0.0f ? rsqrt_approx(r2) : 0.0f; }
    __device__ float far(float r2, float, float, float) const { return rsqrt_approx(r2); }
};
struct KInvR2 {
    float a;
    __device__ float one(float r2, float, float, float) const { return r2 > 0.0f ? rcp_approx(r2) : 0.0f; }
    __device__ float far(float r2, float, float, float) const { return rcp_approx(r2); }
};
struct KExp { // exp(-h r / ell) = 2^(-a r), a = h / (ell ln 2)
    float a;
    __device__ float one(float r2, float, float, float) const
    {
        return ex2_approx(-a * (r2 > 0.0f ? r2 * rsqrt_approx(r2) : 0.0f));
    }
    __device__ float far(float r2, float, float, float) const { return ex2_approx(-a * (r2 * rsqrt_approx(r2))); }
};
struct KGauss { // exp(-(h r / ell)^2) = 2^(-a r^2), a = h^2 / (ell^2 ln 2)
    float a;
    __device__ float one(float r2, float, float, float) const { return ex2_approx(-a * r2); }
    __device__ float far(float r2, float dx, float dy, float dz) const { return one(r2, dx, dy, dz); }
};
struct KPoly { // q(d) with d = h * (x - y) in physical units
    float a;   // h
    __device__ float one(float, float dx, float dy, float dz) const
    {
        float d0 = a * dx, d1 = a * dy, d2 = a * dz;
        return 1.0f + d0 - 2.0f * d1 * d2 + 3.0f * d0 * d0 * d1;
    }
    __device__ float far(float r2, float dx, float dy, float dz) const { return one(r2, dx, dy, dz); }
};
struct KConst {
    float a;
    __device__ float one(float, float, float, float) const { return 1.0f; }
    __device__ float far(float, float, float, float) const { return 1.0f; }
};

// tags: the target's own leaf (r = 0 possible) or one of the other 26
struct OwnLeaf {
    static constexpr bool value = true;
};
struct FarLeaf {
    static constexpr bool value = false;
};

template <bool OWN, class Kern>
__device__ __forceinline__ float2 kern2(const Kern &k, float2 r2, float2 dx, float2 dy, float2 dz)
{
    if (OWN)
        return make_float2(k.one(r2.x, dx.x, dy.x, dz.x), k.one(r2.y, dx.y, dy.y, dz.y));
    return make_float2(k.far(r2.x, dx.x, dy.x, dz.x), k.far(r2.y, dx.y, dy.y, dz.y));
}

// targets per thread (2 or 4): each thread runs 1 or 2 packed target pairs
// against every source it visits, so a source's two shared-memory loads serve
// that many targets
#ifndef BBFMM_P2P_TPT
#define BBFMM_P2P_TPT 4
#endif
constexpr int kTPT = BBFMM_P2P_TPT;
static_assert(kTPT == 2 || kTPT == 4, "2 or 4 targets per thread");

template <class Kern>
__global__ void __launch_bounds__(kP2PThreads, 8)
    k_p2p(const float4 *__restrict__ tpts, const int4 *__restrict__ chunks, long long n_tgt,
          const float4 *__restrict__ spts, const float *__restrict__ sig, const int *__restrict__ off, long long n_src,
          int D, Kern kern, float scale, int nrhs, float *__restrict__ phi)
{
    constexpr int NPK = kTPT / 2; // packed target pairs per thread
    // staged sources: [j] = (x, x, y, y), [kStageSrc + j] = (z, z, sigma, sigma)
    __shared__ float4 stage[2 * kStageSrc];
    __shared__ int nb_start[28], nb_pre[28];
    __shared__ float4 nb_delta[27];
    __shared__ float2 red[NPK][kP2PThreads];
    const int tid = threadIdx.x;
    const int4 ch = chunks[blockIdx.x];
    const int nt = ch.z;
    const int nq = (nt + kTPT - 1) / kTPT; // target groups (one per thread and slice)
    const int S = kP2PThreads / nq;        // slices per group (>= 1)
    const int t = tid % nq, slice = tid / nq;
    const bool active = slice < S;
    int ax, ay, az;
    demorton3((unsigned)ch.x, ax, ay, az);
    const int nside = 1 << D;
    // the group's targets t + q nq (a missing one duplicates target t),
    // loaded while warp 0 looks up the neighbours
    float2 X[NPK], Y[NPK], Z[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk) {
        const int i0 = t + 2 * pk * nq, i1 = i0 + nq;
        const float4 xa = tpts[ch.y + (active && i0 < nt ? i0 : 0)];
        const float4 xb = tpts[ch.y + (active && i1 < nt ? i1 : 0)];
        X[pk] = make_float2(xa.x, xb.x);
        Y[pk] = make_float2(xa.y, xb.y);
        Z[pk] = make_float2(xa.z, xb.z);
    }

    // neighbour leaves: start, count (prefix) and cell offset; the target's
    // own leaf comes first, so its sources are staged ahead of the others
    if (tid < 32) {
        int cnt = 0, start = 0;
        if (tid < 27) {
            const int nid = tid == 0 ? 13 : (tid <= 13 ? tid - 1 : tid);
            const int dx = nid % 3 - 1, dy = (nid / 3) % 3 - 1, dz = nid / 9 - 1;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < nside && by < nside && bz < nside) {
                const unsigned nm = morton3((unsigned)bx, (unsigned)by, (unsigned)bz);
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
    const int ns = nb_pre[27], nown = nb_pre[1]; // all sources; those of the own leaf
    const float2 floor2 = make_float2(kR2Floor, kR2Floor);

    for (int c = 0; c < nrhs; ++c) {
        const float *sg = sig + (long long)c * n_src;
        float2 acc[NPK], acc2[NPK];
#pragma unroll
        for (int pk = 0; pk < NPK; ++pk)
            acc[pk] = acc2[pk] = make_float2(0.0f, 0.0f);
        for (int base = 0; base < ns; base += kStageSrc) {
            const int cnt = min(kStageSrc, ns - base);
            int k = 0; // neighbour holding source gg: it only moves forward as gg grows
            for (int g = tid; g < cnt; g += kP2PThreads) {
                const int gg = base + g;
                while (nb_pre[k + 1] <= gg)
                    ++k;
                const int src = nb_start[k] + (gg - nb_pre[k]);
                const float4 u = spts[src];
                const float4 d = nb_delta[k];
                const float s = sg[src];
                // staged negated so that x_target - y' is one packed add
                const float x = -__fadd_rn(u.x, d.x), y = -__fadd_rn(u.y, d.y), z = -__fadd_rn(u.z, d.z);
                stage[g] = make_float4(x, x, y, y);
                stage[kStageSrc + g] = make_float4(z, z, s, s);
            }
            __syncthreads();
            if (active) {
                // one source (at p) against the thread's NPK target pairs
                auto visit = [&](auto own, const float4 *p, float2 *a) {
                    const float4 qa = p[0];
                    const float4 qb = p[kStageSrc];
#pragma unroll
                    for (int pk = 0; pk < NPK; ++pk) {
                        const float2 dx = __fadd2_rn(X[pk], make_float2(qa.x, qa.y));
                        const float2 dy = __fadd2_rn(Y[pk], make_float2(qa.z, qa.w));
                        const float2 dz = __fadd2_rn(Z[pk], make_float2(qb.x, qb.y));
                        float2 r2 = decltype(own)::value ? __fmul2_rn(dx, dx) : __ffma2_rn(dx, dx, floor2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        const float2 K = kern2<decltype(own)::value>(kern, r2, dx, dy, dz);
                        a[pk] = __ffma2_rn(K, make_float2(qb.z, qb.w), a[pk]);
                    }
                };
                // the own leaf's sources (staged first) with the r = 0 test;
                // the thread walks its sources with one pointer
                const float4 *p = stage + slice;
                const float4 *const pown = stage + min(cnt, max(0, nown - base)), *const pend = stage + cnt;
                for (; p < pown; p += S)
                    visit(OwnLeaf{}, p, acc);
                // two sources per iteration into two accumulator sets (shorter
                // dependency chains), added in a fixed order at the end
#pragma unroll 2
                for (; p + S < pend; p += 2 * S) {
                    visit(FarLeaf{}, p, acc);
                    visit(FarLeaf{}, p + S, acc2);
                }
                if (p < pend)
                    visit(FarLeaf{}, p, acc);
            }
            __syncthreads();
        }
#pragma unroll
        for (int pk = 0; pk < NPK; ++pk)
            red[pk][tid] = active ? make_float2(acc[pk].x + acc2[pk].x, acc[pk].y + acc2[pk].y)
                                  : make_float2(0.0f, 0.0f);
        __syncthreads();
        if (tid < nq) {
#pragma unroll
            for (int pk = 0; pk < NPK; ++pk) {
                float sa = 0.0f, sb = 0.0f;
                for (int q = 0; q < S; ++q) {
                    const float2 v = red[pk][tid + q * nq];
                    sa += v.x;
                    sb += v.y;
                }
                const int i0 = tid + 2 * pk * nq, i1 = i0 + nq;
                if (i0 < nt)
                    phi[(long long)c * n_tgt + ch.y + i0] = scale * sa;
                if (i1 < nt)
                    phi[(long long)c * n_tgt + ch.y + i1] = scale * sb;
            }
        }
        __syncthreads();
    }
}

// Small leaves (a few points each): a work item is up to kP2PChunk targets
// of one level-(D-1) box, i.e. of its 8 child leaves, and the sources of the
// 4x4x4 block of leaves around that box are staged once for all of them (a
// per-leaf item would stage its 27 leaves for a handful of targets).  The
// union's leaves are staged in (z, y, x) order, so the 27 neighbours of a
// child are 9 rows of 3 consecutive leaves, i.e. 9 runs of the stage (the
// row through the child itself split at its own leaf, which takes the r = 0
// test).  Coordinates are in the frame of child (0, 0, 0): a point of leaf L
// sits at u + (L - 2P) with |L - 2P| <= 2 per axis (targets: 0 or 1).
// Threads are (group of <= kTPT targets of one child, slice), as in k_p2p.
constexpr int kBoxStage = 512; // staged sources per pass (16 KB)

template <class Kern>
__global__ void __launch_bounds__(kP2PThreads, 8)
    k_p2p_box(const float4 *__restrict__ tpts, const int *__restrict__ toff, const int4 *__restrict__ items,
              long long n_tgt, const float4 *__restrict__ spts, const float *__restrict__ sig,
              const int *__restrict__ soff, int D, Kern kern, float scale, float *__restrict__ phi)
{
    constexpr int NPK = kTPT / 2;
    __shared__ float4 stage[2 * kBoxStage];
    __shared__ int lpre[65];      // prefix of the source counts of the 64 union leaves
    __shared__ int lfirst[64];    // first source (tree order) of each union leaf
    __shared__ int cfirst[9];     // the item's targets by child: [cfirst[c], cfirst[c + 1])
    __shared__ int gpre[9];       // target groups by child (prefix)
    __shared__ float2 red[NPK][kP2PThreads];
    const int tid = threadIdx.x;
    const int4 it = items[blockIdx.x];
    int px, py, pz;
    demorton3((unsigned)it.x, px, py, pz);
    const int nside = 1 << D;
    if (tid < 64) { // union leaves: counts, then a scan over the two warps
        const int lx = 2 * px - 1 + (tid & 3), ly = 2 * py - 1 + ((tid >> 2) & 3), lz = 2 * pz - 1 + (tid >> 4);
        int cnt = 0, start = 0;
        if (lx >= 0 && ly >= 0 && lz >= 0 && lx < nside && ly < nside && lz < nside) {
            const unsigned m = morton3((unsigned)lx, (unsigned)ly, (unsigned)lz);
            start = soff[m];
            cnt = soff[m + 1] - start;
        }
        lfirst[tid] = start;
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o)
                incl += v;
        }
        lpre[tid + 1] = incl; // warp-local inclusive prefix; warp 1 adds warp 0's total below
    }
    if (tid >= 64 && tid < 64 + 9) { // the item's targets by child leaf, clipped to the item
        const int c = tid - 64;
        const int a = c < 8 ? toff[8 * it.x + c] : toff[8 * it.x + 8];
        cfirst[c] = min(max(a, it.y), it.y + it.z);
    }
    __syncthreads();
    if (tid >= 32 && tid < 64)
        lpre[tid + 1] += lpre[32];
    if (tid == 0) {
        lpre[0] = 0;
        int q = 0;
        for (int c = 0; c < 8; ++c) {
            gpre[c] = q;
            q += (cfirst[c + 1] - cfirst[c] + kTPT - 1) / kTPT;
        }
        gpre[8] = q;
    }
    __syncthreads();
    const int Q = gpre[8];
    const int S = kP2PThreads / Q;
    const int q = tid % Q, slice = tid / Q;
    const bool active = slice < S;
    int c = 0;
    while (c < 7 && gpre[c + 1] <= q)
        ++c;
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    const int t0 = cfirst[c] + kTPT * (q - gpre[c]), tend = cfirst[c + 1];
    float2 X[NPK], Y[NPK], Z[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk) {
        const int i0 = t0 + 2 * pk, i1 = i0 + 1;
        const float4 xa = tpts[active && i0 < tend ? i0 : t0];
        const float4 xb = tpts[active && i1 < tend ? i1 : t0];
        X[pk] = make_float2(__fadd_rn(xa.x, (float)cx), __fadd_rn(xb.x, (float)cx));
        Y[pk] = make_float2(__fadd_rn(xa.y, (float)cy), __fadd_rn(xb.y, (float)cy));
        Z[pk] = make_float2(__fadd_rn(xa.z, (float)cz), __fadd_rn(xb.z, (float)cz));
    }
    const float2 floor2 = make_float2(kR2Floor, kR2Floor);
    float2 acc[NPK], acc2[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk)
        acc[pk] = acc2[pk] = make_float2(0.0f, 0.0f);
    const int ns = lpre[64];
    for (int base = 0; base < ns; base += kBoxStage) {
        const int cnt = min(kBoxStage, ns - base);
        for (int g = tid; g < cnt; g += kP2PThreads) {
            const int gg = base + g;
            int lo = 0, hi = 63; // the union leaf holding source gg: lpre[lo] <= gg < lpre[lo + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (lpre[mid] <= gg)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int src = lfirst[lo] + (gg - lpre[lo]);
            const float4 u = spts[src];
            const float s = sig[src];
            // staged negated, in the frame of child (0, 0, 0): union leaf x index - 1
            const float x = -__fadd_rn(u.x, (float)((lo & 3) - 1)), y = -__fadd_rn(u.y, (float)(((lo >> 2) & 3) - 1)),
                        z = -__fadd_rn(u.z, (float)((lo >> 4) - 1));
            stage[g] = make_float4(x, x, y, y);
            stage[kBoxStage + g] = make_float4(z, z, s, s);
        }
        __syncthreads();
        if (active) {
            auto visit = [&](auto own, const float4 *p, float2 *a) {
                const float4 qa = p[0];
                const float4 qb = p[kBoxStage];
#pragma unroll
                for (int pk = 0; pk < NPK; ++pk) {
                    const float2 dx = __fadd2_rn(X[pk], make_float2(qa.x, qa.y));
                    const float2 dy = __fadd2_rn(Y[pk], make_float2(qa.z, qa.w));
                    const float2 dz = __fadd2_rn(Z[pk], make_float2(qb.x, qb.y));
                    float2 r2 = decltype(own)::value ? __fmul2_rn(dx, dx) : __ffma2_rn(dx, dx, floor2);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    const float2 K = kern2<decltype(own)::value>(kern, r2, dx, dy, dz);
                    a[pk] = __ffma2_rn(K, make_float2(qb.z, qb.w), a[pk]);
                }
            };
            // the child's neighbours: 9 rows of 3 union leaves (x = cx .. cx + 2)
            for (int row = 0; row < 9; ++row) {
                const int u0 = cx + 4 * (cy + row % 3) + 16 * (cz + row / 3);
                const int A = lpre[u0], B = lpre[u0 + 1], C = lpre[u0 + 2], E = lpre[u0 + 3];
                // runs of this row: [A, E) far, or, on the child's own row,
                // [A, B) far, [B, C) own, [C, E) far
                const bool ownrow = row == 4;
                for (int part = 0; part < (ownrow ? 3 : 1); ++part) {
                    const int r0 = ownrow ? (part == 0 ? A : part == 1 ? B : C) : A;
                    const int r1 = ownrow ? (part == 0 ? B : part == 1 ? C : E) : E;
                    const int lo = max(r0, base) - base, hi = min(r1, base + cnt) - base;
                    const float4 *p = stage + lo + slice;
                    const float4 *const pend = stage + max(hi, lo);
                    if (ownrow && part == 1) {
                        for (; p < pend; p += S)
                            visit(OwnLeaf{}, p, acc);
                    } else {
#pragma unroll 2
                        for (; p + S < pend; p += 2 * S) {
                            visit(FarLeaf{}, p, acc);
                            visit(FarLeaf{}, p + S, acc2);
                        }
                        if (p < pend)
                            visit(FarLeaf{}, p, acc);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk)
        red[pk][tid] = active ? make_float2(acc[pk].x + acc2[pk].x, acc[pk].y + acc2[pk].y) : make_float2(0.0f, 0.0f);
    __syncthreads();
    if (tid < Q) {
#pragma unroll
        for (int pk = 0; pk < NPK; ++pk) {
            float sa = 0.0f, sb = 0.0f;
            for (int k = 0; k < S; ++k) {
                const float2 v = red[pk][tid + k * Q];
                sa += v.x;
                sb += v.y;
            }
            const int i0 = t0 + 2 * pk, i1 = i0 + 1;
            if (i0 < tend)
                phi[i0] = scale * sa;
            if (i1 < tend)
                phi[i1] = scale * sb;
        }
    }
}

// Symmetric near field (K(d) = K(-d), the targets are the sources, one
// right-hand side).  K(x_i, y_j) = K(x_j, y_i), so a pair of neighbour leaves
// needs its kernel values once (the paper's remark on symmetry, Sec. 2.5):
// the work item of leaf alpha takes
//   - its own leaf, one way (rows of alpha only, r = 0 test);
//   - the 13 "forward" neighbours beta = alpha + d (nid > 13 in the 3x3x3
//     numbering): both ways when alpha holds at most kSymMaxPoints points --
//     rows of alpha in registers, and for every source of beta the column
//     sum sum_t K(x_t, y_j) sigma_t over alpha's targets, which goes to slot
//     26 - nid of that point (the nid under which beta sees alpha); one way
//     otherwise;
//   - a backward neighbour (nid < 13) only when that leaf holds more than
//     kSymMaxPoints points: such a leaf writes no slots, so both sides then
//     take their own rows of the pair.
// Each (slot, point) is written by one work item and never by two, and the
// combine adds the 13 slots in a fixed order after the point's own rows:
// the result does not depend on scheduling.  Slots no work item writes (the
// backward neighbour is absent, empty or above kSymMaxPoints) stay at the
// zero they were given when the plan was made.
//
// Column sums: the thread of target group q visiting source j stores its
// partial sum over its kTPT targets in colpart[j][q] (row stride nq rounded
// up to 4, the padding zero); after the pass one thread per source adds its
// row in order and stores the sum through the slot pointer staged with the
// source.
constexpr int kSymSlots = 13;
struct OneWay {
    static constexpr bool value = false;
};
struct TwoWay {
    static constexpr bool value = true;
};
constexpr int kSymStage = 256; // staged sources per pass
constexpr int kColBuf = 2048;  // column partials per pass (nq x pass length)
// leaves of more points take their pairs one way: their column rows would
// cut the passes short (the rule is the same on both sides of a pair)
#ifndef BBFMM_SYM_MAX_POINTS
#define BBFMM_SYM_MAX_POINTS 64
#endif
constexpr int kSymMaxPoints = BBFMM_SYM_MAX_POINTS;
static_assert(kSymMaxPoints <= kP2PChunk, "a two-way leaf is one work item");

template <class Kern>
__global__ void __launch_bounds__(kP2PThreads, 8)
    k_p2p_sym(const float4 *__restrict__ pts, const int4 *__restrict__ chunks, long long n,
              const float *__restrict__ sig, const int *__restrict__ off, int D, Kern kern, float scale,
              float *__restrict__ phi, float *__restrict__ slots)
{
    constexpr int NPK = kTPT / 2;
    // staged sources: [j] = (x, x, y, y), [kSymStage + j] = (z, z, sigma, sigma)
    __shared__ float4 stage[2 * kSymStage];
    __shared__ __align__(16) float colpart[kColBuf];
    __shared__ float *sDst[kSymStage];         // slot entry of a staged two-way source
    __shared__ int nb_start[28], nb_pre[28], nb_cnt[28], nb_slot[28];
    __shared__ float4 nb_delta[27];
    __shared__ float2 red[NPK][kP2PThreads];
    __shared__ int s_nsym0;
    const int tid = threadIdx.x;
    const int4 ch = chunks[blockIdx.x];
    const int nt = ch.z;
    const int nq = (nt + kTPT - 1) / kTPT;
    const int S = kP2PThreads / nq;
    const int t = tid % nq, slice = tid / nq;
    const bool active = slice < S;
    const bool whole = off[ch.x + 1] - off[ch.x] <= kSymMaxPoints; // alpha takes its pairs both ways
    int ax, ay, az;
    demorton3((unsigned)ch.x, ax, ay, az);
    const int nside = 1 << D;
    // the thread's targets, loaded while warp 0 looks up the neighbours
    float2 X[NPK], Y[NPK], Z[NPK], SG[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk) {
        const int i0 = t + 2 * pk * nq, i1 = i0 + nq;
        const bool h0 = active && i0 < nt, h1 = active && i1 < nt;
        const float4 xa = pts[ch.y + (h0 ? i0 : 0)];
        const float4 xb = pts[ch.y + (h1 ? i1 : 0)];
        X[pk] = make_float2(xa.x, xb.x);
        Y[pk] = make_float2(xa.y, xb.y);
        Z[pk] = make_float2(xa.z, xb.z);
        // a missing target (a duplicate of target t) adds nothing to the columns
        SG[pk] = make_float2(h0 ? sig[ch.y + i0] : 0.0f, h1 ? sig[ch.y + i1] : 0.0f);
    }

    // neighbour leaves in staging order: own (key 0), one way (key 1), both
    // ways (key 2); key 3 is not visited
    if (tid < 32) {
        int cnt = 0, start = 0, key = 3;
        float4 dl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (tid < 27) {
            const int dx = tid % 3 - 1, dy = (tid / 3) % 3 - 1, dz = tid / 9 - 1;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < nside && by < nside && bz < nside) {
                const unsigned nm = morton3((unsigned)bx, (unsigned)by, (unsigned)bz);
                start = off[nm];
                cnt = off[nm + 1] - start;
            }
            if (cnt > 0)
                key = tid == 13 ? 0 : tid > 13 ? (whole ? 2 : 1) : (cnt > kSymMaxPoints ? 1 : 3);
            dl = make_float4((float)dx, (float)dy, (float)dz, 0.0f);
        }
        const unsigned lt = (1u << tid) - 1u;
        const unsigned m0 = __ballot_sync(0xffffffffu, key == 0), m1 = __ballot_sync(0xffffffffu, key == 1),
                       m2 = __ballot_sync(0xffffffffu, key == 2);
        const int n0 = __popc(m0), n1 = __popc(m1), nst = n0 + n1 + __popc(m2);
        const int rank = key == 0   ? __popc(m0 & lt)
                         : key == 1 ? n0 + __popc(m1 & lt)
                         : key == 2 ? n0 + n1 + __popc(m2 & lt)
                                    : -1;
        if (rank >= 0) {
            nb_start[rank] = start;
            nb_cnt[rank] = cnt;
            nb_delta[rank] = dl;
            nb_slot[rank] = 26 - tid;
        }
        __syncwarp();
        const int c = tid < nst ? nb_cnt[tid] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o)
                incl += v;
        }
        if (tid < 28)
            nb_pre[tid] = incl - c;
        const int sym0 = __shfl_sync(0xffffffffu, incl - c, n0 + n1); // first position of key 2
        if (tid == 0)
            s_nsym0 = sym0;
    }
    __syncthreads();
    const int ns = nb_pre[27], nown = nb_pre[1], nsym0 = s_nsym0;
    const float2 floor2 = make_float2(kR2Floor, kR2Floor);
    const int NQP = (nq + 3) & ~3; // colpart row stride
    // pass length: with two-way sources PL rows of NQP partials must fit
    // colpart (PL * NQP <= kColBuf); without, colpart is not used
    const bool two_way = nsym0 < ns;
    const int PL = two_way ? min(kSymStage, kColBuf / NQP) : kSymStage;
    if (two_way && NQP > nq) // the row padding (groups nq .. NQP-1) is never written: zero it once
        for (int r = tid; r < PL; r += kP2PThreads)
            for (int q = nq; q < NQP; ++q)
                colpart[r * NQP + q] = 0.0f;

    float2 acc[NPK], acc2[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk)
        acc[pk] = acc2[pk] = make_float2(0.0f, 0.0f);
    for (int base = 0; base < ns; base += PL) {
        const int cnt = min(PL, ns - base);
        int k = 0;
        for (int g = tid; g < cnt; g += kP2PThreads) {
            const int gg = base + g;
            while (nb_pre[k + 1] <= gg)
                ++k;
            const int src = nb_start[k] + (gg - nb_pre[k]);
            const float4 u = pts[src];
            const float4 d = nb_delta[k];
            const float s = sig[src];
            const float x = -__fadd_rn(u.x, d.x), y = -__fadd_rn(u.y, d.y), z = -__fadd_rn(u.z, d.z);
            stage[g] = make_float4(x, x, y, y);
            stage[kSymStage + g] = make_float4(z, z, s, s);
            if (gg >= nsym0) {
                sDst[g] = slots + (long long)nb_slot[k] * n + src;
            }
        }
        __syncthreads();
        if (active) {
            // one source (at p) against the thread's targets: rows into a;
            // two ways, also the source's column partial over those targets
            auto visit = [&](auto own, auto two, const float4 *p, float2 *a, float *col) {
                const float4 qa = p[0];
                const float4 qb = p[kSymStage];
                float2 cs = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int pk = 0; pk < NPK; ++pk) {
                    const float2 dx = __fadd2_rn(X[pk], make_float2(qa.x, qa.y));
                    const float2 dy = __fadd2_rn(Y[pk], make_float2(qa.z, qa.w));
                    const float2 dz = __fadd2_rn(Z[pk], make_float2(qb.x, qb.y));
                    float2 r2 = decltype(own)::value ? __fmul2_rn(dx, dx) : __ffma2_rn(dx, dx, floor2);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    const float2 K = kern2<decltype(own)::value>(kern, r2, dx, dy, dz);
                    a[pk] = __ffma2_rn(K, make_float2(qb.z, qb.w), a[pk]);
                    if (decltype(two)::value)
                        cs = __ffma2_rn(K, SG[pk], cs);
                }
                if (decltype(two)::value)
                    *col = cs.x + cs.y;
            };
            const float4 *p = stage + slice;
            const float4 *const pown = stage + min(cnt, max(0, nown - base));
            const float4 *const psym = stage + min(cnt, max(0, nsym0 - base)), *const pend = stage + cnt;
            for (; p < pown; p += S)
                visit(OwnLeaf{}, OneWay{}, p, acc, nullptr);
#pragma unroll 2
            for (; p + S < psym; p += 2 * S) {
                visit(FarLeaf{}, OneWay{}, p, acc, nullptr);
                visit(FarLeaf{}, OneWay{}, p + S, acc2, nullptr);
            }
            if (p < psym) {
                visit(FarLeaf{}, OneWay{}, p, acc, nullptr);
                p += S;
            }
            float *col = colpart + (p - stage) * NQP + t;
            const int cstep = S * NQP;
#pragma unroll 2
            for (; p + S < pend; p += 2 * S, col += 2 * cstep) {
                visit(FarLeaf{}, TwoWay{}, p, acc, col);
                visit(FarLeaf{}, TwoWay{}, p + S, acc2, col + cstep);
            }
            if (p < pend)
                visit(FarLeaf{}, TwoWay{}, p, acc, col);
        }
        __syncthreads();
        // column sums of this pass's two-way sources, in target-group order
        for (int g = max(0, nsym0 - base) + tid; g < cnt; g += kP2PThreads) {
            const float4 *row = reinterpret_cast<const float4 *>(colpart + g * NQP);
            float v = 0.0f;
            for (int q = 0; q < NQP / 4; ++q) {
                const float4 c4 = row[q];
                v += c4.x;
                v += c4.y;
                v += c4.z;
                v += c4.w;
            }
            *sDst[g] = scale * v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk)
        red[pk][tid] = active ? make_float2(acc[pk].x + acc2[pk].x, acc[pk].y + acc2[pk].y) : make_float2(0.0f, 0.0f);
    __syncthreads();
    if (tid < nq) {
#pragma unroll
        for (int pk = 0; pk < NPK; ++pk) {
            float sa = 0.0f, sb = 0.0f;
            for (int q = 0; q < S; ++q) {
                const float2 v = red[pk][tid + q * nq];
                sa += v.x;
                sb += v.y;
            }
            const int i0 = tid + 2 * pk * nq, i1 = i0 + nq;
            if (i0 < nt)
                phi[ch.y + i0] = scale * sa;
            if (i1 < nt)
                phi[ch.y + i1] = scale * sb;
        }
    }
}

// Several right-hand sides (Sec. 2.5 "Multiple right-hand-sides"): the near
// field of a work item is a product of its kernel matrix (targets x
// neighbourhood sources) with the weights (sources x nrhs, read row-major).  The block walks
// the item's targets in sub-tiles of TT; per chunk of kGemmS sources it
// evaluates the K tile once (TT x kGemmS, shared memory), stages the
// weights (kGemmS x kGemmC) and adds K . sigma into registers: thread = 4
// targets x 8 columns, 32 FMAs per source for three shared-memory loads.
// Columns run in passes of kGemmC.  Leaves hold tens of points, so the tile
// is narrow and the block small (two warps, many blocks per SM).
constexpr int kGemmT = 32;  // targets per sub-tile (measured: 16 was slower on ~15-point leaves)
constexpr int kGemmS = 32;  // sources per chunk
constexpr int kGemmC = 64;  // right-hand sides per pass
__host__ __device__ constexpr int gemm_threads(int TT) { return (TT / 4) * (kGemmC / 8); }

// TT: targets per sub-tile (kGemmT), gemm_threads(TT) threads
template <class Kern, int TT>
__global__ void __launch_bounds__(gemm_threads(TT))
    k_p2p_gemm(const float4 *__restrict__ tpts, const int4 *__restrict__ chunks, long long n_tgt,
               const float4 *__restrict__ spts, const float *__restrict__ sig_rows, const int *__restrict__ off,
               long long n_src, int D, Kern kern, float scale, int nrhs, float *__restrict__ phi)
{
    __shared__ float4 sTgt[TT];
    __shared__ float4 sPos[kGemmS];                     // (x, y, z) in the target leaf's frame, w = own leaf
    __shared__ int sSrc[kGemmS];
    __shared__ __align__(16) float sK[kGemmS][TT];
    __shared__ __align__(16) float sSig[kGemmS][kGemmC];
    __shared__ int nb_start[28], nb_pre[28];
    __shared__ float4 nb_delta[27];
    const int tid = threadIdx.x;
    const int4 ch = chunks[blockIdx.x];
    int ax, ay, az;
    demorton3((unsigned)ch.x, ax, ay, az);
    const int nside = 1 << D;
    // neighbour leaves, the target's own first (as in k_p2p)
    if (tid < 32) {
        int cnt = 0, start = 0;
        if (tid < 27) {
            const int nid = tid == 0 ? 13 : (tid <= 13 ? tid - 1 : tid);
            const int dx = nid % 3 - 1, dy = (nid / 3) % 3 - 1, dz = nid / 9 - 1;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < nside && by < nside && bz < nside) {
                const unsigned nm = morton3((unsigned)bx, (unsigned)by, (unsigned)bz);
                start = off[nm];
                cnt = off[nm + 1] - start;
            }
            nb_start[tid] = start;
            nb_delta[tid] = make_float4((float)dx, (float)dy, (float)dz, 0.0f);
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o)
                incl += v;
        }
        if (tid < 28)
            nb_pre[tid] = incl - cnt;
    }
    __syncthreads();
    const int ns = nb_pre[27], nown = nb_pre[1];
    const int tg = tid % (TT / 4), cg = tid / (TT / 4);
    const bool vec4 = (nrhs & 3) == 0; // rows of sig_rows start on 16-byte boundaries
    const int t0 = 4 * tg, c8 = 8 * cg; // this thread's targets (in the sub-tile) and columns (in the pass)
    for (int tt = 0; tt < ch.z; tt += TT) {
        const int nt = min(TT, ch.z - tt); // targets of this sub-tile
        for (int c0 = 0; c0 < nrhs; c0 += kGemmC) {
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[i][j] = 0.0f;
            for (int base = 0; base < ns; base += kGemmS) {
                const int cnt = min(kGemmS, ns - base);
                __syncthreads(); // the previous chunk's tiles are consumed
                if (tid < TT)
                    sTgt[tid] = tpts[ch.y + tt + (tid < nt ? tid : 0)];
                if (tid < kGemmS) {
                    const int gg = base + tid;
                    float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    int src = -1;
                    if (tid < cnt) {
                        int k = 0;
                        while (nb_pre[k + 1] <= gg)
                            ++k;
                        src = nb_start[k] + (gg - nb_pre[k]);
                        const float4 u = spts[src];
                        const float4 d = nb_delta[k];
                        p = make_float4(__fadd_rn(u.x, d.x), __fadd_rn(u.y, d.y), __fadd_rn(u.z, d.z),
                                        gg < nown ? 1.0f : 0.0f);
                    }
                    sPos[tid] = p;
                    sSrc[tid] = src;
                }
                __syncthreads();
                // weights, row-major (nrhs per source): consecutive threads take
                // consecutive columns of one source, four at a time when the
                // rows are 16-byte aligned
                if (vec4) {
#pragma unroll 8
                    for (int q = tid; q < kGemmS * kGemmC / 4; q += gemm_threads(TT)) {
                        const int c = 4 * (q % (kGemmC / 4)), sidx = q / (kGemmC / 4);
                        const int src = sSrc[sidx];
                        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (src >= 0 && c0 + c < nrhs) // nrhs % 4 == 0: the whole quad is in range
                            v = __ldg(reinterpret_cast<const float4 *>(sig_rows + (long long)src * nrhs + c0 + c));
                        *reinterpret_cast<float4 *>(&sSig[sidx][c]) = v;
                    }
                } else {
#pragma unroll 8
                    for (int q = tid; q < kGemmS * kGemmC; q += gemm_threads(TT)) {
                        const int c = q % kGemmC, sidx = q / kGemmC;
                        const int src = sSrc[sidx];
                        sSig[sidx][c] =
                            (src >= 0 && c0 + c < nrhs) ? __ldg(sig_rows + (long long)src * nrhs + c0 + c) : 0.0f;
                    }
                }
                // K tile: thread = one target (coordinates in registers) and
                // a stride of sources; a source's position is one broadcast
                {
                    constexpr int SPLIT = gemm_threads(TT) / TT; // threads per target
                    const int t = tid % TT;
                    const float4 x = sTgt[t];
                    const bool tv = t < nt;
#pragma unroll 4
                    for (int sidx = tid / TT; sidx < kGemmS; sidx += SPLIT) {
                        const float4 y = sPos[sidx];
                        const float dx = __fsub_rn(x.x, y.x), dy = __fsub_rn(x.y, y.y), dz = __fsub_rn(x.z, y.z);
                        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
                        float K = 0.0f;
                        if (sidx < cnt && tv)
                            K = y.w != 0.0f ? kern.one(r2, dx, dy, dz)
                                            : kern.far(__fadd_rn(r2, kR2Floor), dx, dy, dz);
                        sK[sidx][t] = K;
                    }
                }
                __syncthreads();
#pragma unroll 4
                for (int sidx = 0; sidx < cnt; ++sidx) {
                    const float4 k4 = *reinterpret_cast<const float4 *>(&sK[sidx][t0]);
                    const float4 sa = *reinterpret_cast<const float4 *>(&sSig[sidx][c8]);
                    const float4 sb = *reinterpret_cast<const float4 *>(&sSig[sidx][c8 + 4]);
                    const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
                    const float sv[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            acc[i][j] = fmaf(kv[i], sv[j], acc[i][j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + c8 + j;
                if (c >= nrhs)
                    continue;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (t0 + i < nt)
                        phi[(long long)c * n_tgt + ch.y + tt + t0 + i] = scale * acc[i][j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Close pairs (plan time).  The near-field kernels take x - y from FP32
// leaf-local coordinates; each coordinate carries a rounding of up to
// ~2^-25 cells, so a pair at distance r (cells) gets a relative error of
// about 1e-7 / r in K.  For the singular kernels the few closest pairs of a
// point set dominate the error of the whole near field (on clustered points
// it exceeds 1e-5).  Pairs closer than 1/64 cell are therefore listed when
// the plan is made, each with the coefficient
//     c = K(x_i - y_j)  [FP64, from the caller's FP64 coordinates]
//         - scale * K32(i, j)  [the FP32 value the near-field kernel adds],
// and every matvec adds sum_j c sigma_j to the near field of target i
// (k_near_fix), so the listed pairs enter the result as if evaluated in
// FP64.  K32 is recomputed here with the same rounded operations as the
// kernel that adds it (same frame, same operation order).  A point's pair
// with itself and exact duplicates (c = 0 in both forms) are not listed.
//
// Frames: every near-field kernel evaluates a pair in the target leaf's
// frame, except the symmetric one, where the value for target i in leaf A
// and source j in leaf B != A comes from B's work item (B's frame, column
// sums) when B precedes A in the 3x3x3 order and holds at most kSymMaxPoints
// points.
constexpr float kCloseR2 = 2.44140625e-4f; // (1/64 cell)^2

struct CloseArgs {
    const float4 *tpts;   // targets: leaf-local coordinates, tree order
    const int4 *chunks;   // near-field work items over the target leaves
    int nchunks;
    const float4 *spts;   // sources: leaf-local coordinates, tree order
    const int *soff;      // sources: leaf offsets
    const double *tx;     // targets: FP64 coordinates, caller order (n x 3)
    const int *tperm;     // target tree order -> caller order
    const double *sx;     // sources: FP64 coordinates, caller order
    const int *sperm;     // source tree order -> caller order
    int D;
    int same;             // the targets are the sources (skip i == j)
    int sym;              // also the coefficients of the symmetric one-RHS form
    float scale;          // the near-field kernels write scale * sum K sigma
    int *count;           // count pass: listed pairs per target (tree order)
    const int *first;     // fill pass: first entry of each target
    int *e_src;           // fill pass: source (tree order) of each entry
    float *e_c1, *e_c1s, *e_c1b, *e_cm; // fill pass: c for one RHS (ordered by leaf, symmetric,
                                        // ordered by box) and several RHS
};

// FP32 squared distances as the near-field kernels form them
__device__ __forceinline__ float r2_rows(float dx, float dy, float dz, bool own)
{ // k_p2p / k_p2p_sym: x first, the floor on the other 26 leaves
    const float r2 = own ? __fmul_rn(dx, dx) : __fmaf_rn(dx, dx, kR2Floor);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, r2));
}
__device__ __forceinline__ float r2_gemm(float dx, float dy, float dz, bool own)
{ // k_p2p_gemm: z first, the floor added after
    const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
    return own ? r2 : __fadd_rn(r2, kR2Floor);
}

// one block (kP2PThreads) per work item, a thread per target; the 27
// neighbour leaves' sources are staged kStageSrc at a time.  FILL = false
// counts the listed pairs of each target, FILL = true writes them from
// first[target] on, in staging order (deterministic).
template <class Kern, class Exact, bool FILL>
__global__ void __launch_bounds__(kP2PThreads) k_close_pairs(const CloseArgs A, Kern kern, Exact exact)
{
    __shared__ float4 stage[kStageSrc]; // u + d of the source; w = its neighbour number (bits)
    __shared__ int ssrc[kStageSrc];
    __shared__ int nb_start[27], nb_cnt[27], nb_pre[28];
    const int tid = threadIdx.x;
    const int4 ch = A.chunks[blockIdx.x];
    int ax, ay, az;
    demorton3((unsigned)ch.x, ax, ay, az);
    const int nside = 1 << A.D;
    if (tid < 32) {
        int cnt = 0, start = 0;
        if (tid < 27) {
            const int bx = ax + tid % 3 - 1, by = ay + (tid / 3) % 3 - 1, bz = az + tid / 9 - 1;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < nside && by < nside && bz < nside) {
                const unsigned nm = morton3((unsigned)bx, (unsigned)by, (unsigned)bz);
                start = A.soff[nm];
                cnt = A.soff[nm + 1] - start;
            }
            nb_start[tid] = start;
            nb_cnt[tid] = cnt;
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o)
                incl += v;
        }
        if (tid < 28)
            nb_pre[tid] = incl - cnt;
    }
    __syncthreads();
    const int ns = nb_pre[27];
    const bool act = tid < ch.z;
    const int ti = ch.y + (act ? tid : 0);
    const float4 X = A.tpts[ti];
    const long long tc = A.tperm[ti];
    const double x0 = A.tx[3 * tc], x1 = A.tx[3 * tc + 1], x2 = A.tx[3 * tc + 2];
    int listed = 0, pos = FILL && act ? A.first[ti] : 0;
    for (int base = 0; base < ns; base += kStageSrc) {
        const int cnt = min(kStageSrc, ns - base);
        int k = 0;
        for (int g = tid; g < cnt; g += kP2PThreads) {
            const int gg = base + g;
            while (nb_pre[k + 1] <= gg)
                ++k;
            const int src = nb_start[k] + (gg - nb_pre[k]);
            const float4 u = A.spts[src];
            const float ox = (float)(k % 3 - 1), oy = (float)((k / 3) % 3 - 1), oz = (float)(k / 9 - 1);
            stage[g] = make_float4(__fadd_rn(u.x, ox), __fadd_rn(u.y, oy), __fadd_rn(u.z, oz), __int_as_float(k));
            ssrc[g] = src;
        }
        __syncthreads();
        if (act) {
            for (int j = 0; j < cnt; ++j) {
                const float4 q = stage[j];
                const int nid = __float_as_int(q.w);
                const bool own = nid == 13;
                const float dx = __fsub_rn(X.x, q.x), dy = __fsub_rn(X.y, q.y), dz = __fsub_rn(X.z, q.z);
                const float r2 = r2_rows(dx, dy, dz, own);
                if (!(r2 < kCloseR2))
                    continue;
                const int src = ssrc[j];
                if (A.same && src == ti)
                    continue;
                // one RHS: the rows form, in the frame of the leaf that
                // evaluates the pair (ordered: the target's; symmetric: the
                // source's when that leaf takes the pair both ways)
                const float K1 = own ? kern.one(r2, dx, dy, dz) : kern.far(r2, dx, dy, dz);
                float K1s = K1;
                if (A.sym && nid < 13 && nb_cnt[nid] <= kSymMaxPoints) {
                    const float4 us = A.spts[src]; // the target seen from the source's leaf
                    const float ox = (float)(1 - nid % 3), oy = (float)(1 - (nid / 3) % 3), oz = (float)(1 - nid / 9);
                    const float ex = __fsub_rn(us.x, __fadd_rn(X.x, ox)), ey = __fsub_rn(us.y, __fadd_rn(X.y, oy)),
                                ez = __fsub_rn(us.z, __fadd_rn(X.z, oz));
                    K1s = kern.far(r2_rows(ex, ey, ez, false), ex, ey, ez);
                }
                // one RHS by level-(D-1) box (k_p2p_box): the frame of the
                // box's first child, target at u + (cell & 1), source at
                // u + (cell & 1) + neighbour offset
                float K1b;
                {
                    const float4 us = A.spts[src];
                    const int tx = ax & 1, ty = ay & 1, tz = az & 1;
                    const float bx = __fsub_rn(__fadd_rn(X.x, (float)tx), __fadd_rn(us.x, (float)(tx + nid % 3 - 1)));
                    const float by = __fsub_rn(__fadd_rn(X.y, (float)ty), __fadd_rn(us.y, (float)(ty + (nid / 3) % 3 - 1)));
                    const float bz = __fsub_rn(__fadd_rn(X.z, (float)tz), __fadd_rn(us.z, (float)(tz + nid / 9 - 1)));
                    const float rb = r2_rows(bx, by, bz, own);
                    K1b = own ? kern.one(rb, bx, by, bz) : kern.far(rb, bx, by, bz);
                }
                // several RHS: k_p2p_gemm's form, the target's frame
                const float rg = r2_gemm(dx, dy, dz, own);
                const float Km = own ? kern.one(rg, dx, dy, dz) : kern.far(rg, dx, dy, dz);
                const long long sc = A.sperm[src];
                const double Kx = exact(x0 - A.sx[3 * sc], x1 - A.sx[3 * sc + 1], x2 - A.sx[3 * sc + 2]);
                const float c1 = (float)(Kx - (double)A.scale * (double)K1);
                const float c1s = (float)(Kx - (double)A.scale * (double)K1s);
                const float c1b = (float)(Kx - (double)A.scale * (double)K1b);
                const float cm = (float)(Kx - (double)A.scale * (double)Km);
                if (c1 == 0.0f && c1s == 0.0f && c1b == 0.0f && cm == 0.0f)
                    continue;
                if (FILL) {
                    A.e_src[pos] = src;
                    A.e_c1[pos] = c1;
                    A.e_c1b[pos] = c1b;
                    if (A.sym)
                        A.e_c1s[pos] = c1s;
                    A.e_cm[pos] = cm;
                    ++pos;
                } else {
                    ++listed;
                }
            }
        }
        __syncthreads();
    }
    if (!FILL && act)
        A.count[ti] = listed;
}

} // namespace bbfmm
