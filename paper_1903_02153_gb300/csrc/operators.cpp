// operators.cpp -- host FP64 precomputation of the interpolation and M2L
// operators (the PrecomputeM2L step of Sec. 3).
//
//  * Chebyshev nodes S = {cos((2k-1) pi / (2p))} on [-1, 1] (Sec. 2.2).
//  * 1D Lagrange basis l_i(x) = prod_{k != i} (x - s_k)/(s_i - s_k) (Def. 2.2),
//    evaluated on the device as w_i * prod_{k != i} (x - s_k) with the
//    denominators w_i tabulated here.
//  * Child-transfer matrices S_o[i][j] = l_i((s_j + 2o - 1)/2), o = 0 (lower
//    half) or 1 (upper half): the node j of a child box, seen from its parent
//    box, sits at (s_j + 2o - 1)/2.  M2M is M^parent = sum_children
//    (S_ox (x) S_oy (x) S_oz) M^child, L2L its transpose (Sec. 2.3 items 1, 3).
//  * M2L operators K^(t)_ij = K(x*_i, y*_j) for the 316 offsets t between a box
//    and the members of its interaction list (Thm. 2.1 discussion), with the
//    target box centred at 0 and the source box at t*h.
//  * SVD compression (Sec. 2.5 "Fast M2L translation"): U spans the columns of
//    the fat matrix [K^(1) ... K^(316)], V the rows of the tall matrix
//    [K^(1); ...; K^(316)]; each is truncated at singular values below
//    eps * sigma_max, r = max of the two ranks, and C^(t) = U^T K^(t) V, so
//    K^(t) ~ U C^(t) V^T.  The singular vectors are the eigenvectors of the
//    Gram matrices sum_t K K^T and sum_t K^T K, found by cyclic Jacobi.
//  * Homogeneous kernels (Sec. 2.5 "Homogeneous kernel"): K(a x, a y) =
//    a^m K(x, y), so one operator set made for the leaf box size serves every
//    level, scaled by (h_l / h_D)^m.
//  * Equally spaced nodes s_k = -1 + 2k/(p-1) (Sec. 2.2; the paper prints them
//    on [0, 1]): no compression (U = V = I); instead, per offset t, the
//    (2p-1)^3 distinct values of the block-Toeplitz operator (Sec. 2.5 "Fast
//    M2L translation"): x*_i - y*_j = h (-t + (i - j) / (p - 1)) per axis, so
//    K^(t)_ij = c_t(i - j), and K^(t) M is the circular convolution of c_t
//    (stored at index d mod n, n = 2p - 1, which keeps the 2p - 1 differences
//    apart) with M zero-padded to n^3, i.e. a pointwise product of DFTs.  The
//    DFTs of the c_t are tabulated here in FP64.
#include <math.h>

#include <algorithm>
#include <numeric>

#include "bbfmm_internal.h"

namespace bbfmm {

double kernel_value_host(int kernel, double ell, double d0, double d1, double d2)
{
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
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
    case BBFMM_K_TEST_CONST:
        return 1.0;
    }
    return 0.0;
}

int kernel_homogeneity(int kernel)
{
    if (kernel == BBFMM_K_INV_R)
        return -1;
    if (kernel == BBFMM_K_INV_R2)
        return -2;
    int h = 0, sym = 0;
    if (kernel >= BBFMM_K_USER_FIRST && user_kernel_traits(kernel, &h, &sym))
        return h;
    return 0;
}

bool kernel_symmetric(int kernel)
{
    int h = 0, sym = 0;
    if (kernel >= BBFMM_K_USER_FIRST && user_kernel_traits(kernel, &h, &sym))
        return sym != 0;
    return kernel == BBFMM_K_INV_R || kernel == BBFMM_K_INV_R2 || kernel == BBFMM_K_EXP ||
           kernel == BBFMM_K_GAUSS || kernel == BBFMM_K_TEST_CONST;
}

// K at n difference vectors d (n x 3, physical units): built-in kernels on
// the host, user kernels on the device in batches
static bool eval_kernel(const HostOps &o, const double *d, int64_t n, double *out)
{
    if (o.kernel < BBFMM_K_USER_FIRST) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            out[i] = kernel_value_host(o.kernel, o.ell, d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        return true;
    }
    const int64_t batch = 1 << 22;
    for (int64_t i0 = 0; i0 < n; i0 += batch)
        if (user_kernel_eval(o.kernel, d + 3 * i0, std::min(batch, n - i0), out + i0) != cudaSuccess)
            return false;
    return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (row-major,
// destroyed).  On return w holds the eigenvalues in decreasing order and the
// columns of Q (row-major n x n) the matching orthonormal eigenvectors.
void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &Q)
{
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        Q[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double v : A)
        fro += v * v;
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (sqrt(2.0 * off) <= 1e-15 * fro || fro == 0.0)
            break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (fabs(apq) <= 1e-300)
                    continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                // A <- J^T A J with J the rotation in the (p, q) plane
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
                    Q[(size_t)k * n + p] = c * qkp - s * qkq;
                    Q[(size_t)k * n + q] = s * qkp + c * qkq;
                }
            }
        }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
    std::vector<double> Qs((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)idx[j] * n + idx[j]];
        for (int i = 0; i < n; ++i)
            Qs[(size_t)i * n + j] = Q[(size_t)i * n + idx[j]];
    }
    Q.swap(Qs);
}

static int rank_at(const std::vector<double> &w, double eps)
{
    double lmax = std::max(w.empty() ? 0.0 : w[0], 0.0);
    int r = 0;
    for (double v : w)
        if (v > 0.0 && v >= eps * eps * lmax)
            ++r;
    return std::max(r, 1);
}

// operators of one level with box side h
static bool build_level(HostOps &o, double h, std::vector<double> &U, std::vector<double> &V,
                        std::vector<double> &C, std::vector<double> &sv, int &ru, int &rv)
{
    const int p = o.p, p3 = o.p3;
    // K^(t) for all 316 offsets, row = target node i, column = source node j;
    // evaluated in groups of offsets (the difference vectors of one group at
    // a time)
    std::vector<double> K((size_t)kNumOffsets * p3 * p3);
    const int group = (int)std::max<int64_t>(1, std::min<int64_t>(kNumOffsets, (1 << 22) / ((int64_t)p3 * p3)));
    std::vector<double> dv((size_t)group * p3 * p3 * 3);
    for (int u0 = 0; u0 < kNumOffsets; u0 += group) {
        const int u1 = std::min(kNumOffsets, u0 + group);
#pragma omp parallel for schedule(dynamic)
        for (int t = 0; t < 343; ++t) {
            int tx = t % 7 - 3, ty = (t / 7) % 7 - 3, tz = t / 49 - 3;
            int idx = offset_index(tx, ty, tz);
            if (idx < u0 || idx >= u1)
                continue;
            double *dt = &dv[(size_t)(idx - u0) * p3 * p3 * 3];
            for (int i = 0; i < p3; ++i) {
                double x0 = 0.5 * h * o.nodes[i % p], x1 = 0.5 * h * o.nodes[(i / p) % p],
                       x2 = 0.5 * h * o.nodes[i / (p * p)];
                for (int j = 0; j < p3; ++j) {
                    double y0 = tx * h + 0.5 * h * o.nodes[j % p];
                    double y1 = ty * h + 0.5 * h * o.nodes[(j / p) % p];
                    double y2 = tz * h + 0.5 * h * o.nodes[j / (p * p)];
                    double *e = dt + ((size_t)i * p3 + j) * 3;
                    e[0] = x0 - y0;
                    e[1] = x1 - y1;
                    e[2] = x2 - y2;
                }
            }
        }
        if (!eval_kernel(o, dv.data(), (int64_t)(u1 - u0) * p3 * p3, &K[(size_t)u0 * p3 * p3]))
            return false;
    }
    if (o.eps <= 0.0) { // no compression: U = V = I, C = K
        o.r = p3;
        ru = rv = p3;
        U.assign((size_t)p3 * p3, 0.0);
        for (int i = 0; i < p3; ++i)
            U[(size_t)i * p3 + i] = 1.0;
        V = U;
        C = K;
        sv.assign(p3, 0.0);
        return true;
    }
    // Gram matrices of the fat and the tall operator matrices
    std::vector<double> GU((size_t)p3 * p3, 0.0), GV;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < p3; ++i)
        for (int t = 0; t < kNumOffsets; ++t) {
            const double *Kt = &K[(size_t)t * p3 * p3];
            for (int j = 0; j <= i; ++j) {
                double acc = 0.0;
                for (int k = 0; k < p3; ++k)
                    acc += Kt[(size_t)i * p3 + k] * Kt[(size_t)j * p3 + k];
                GU[(size_t)i * p3 + j] += acc;
            }
        }
    for (int i = 0; i < p3; ++i)
        for (int j = 0; j < i; ++j)
            GU[(size_t)j * p3 + i] = GU[(size_t)i * p3 + j];
    bool sym = kernel_symmetric(o.kernel);
    if (!sym) {
        GV.assign((size_t)p3 * p3, 0.0);
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < p3; ++i)
            for (int t = 0; t < kNumOffsets; ++t) {
                const double *Kt = &K[(size_t)t * p3 * p3];
                for (int j = 0; j <= i; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < p3; ++k)
                        acc += Kt[(size_t)k * p3 + i] * Kt[(size_t)k * p3 + j];
                    GV[(size_t)i * p3 + j] += acc;
                }
            }
        for (int i = 0; i < p3; ++i)
            for (int j = 0; j < i; ++j)
                GV[(size_t)j * p3 + i] = GV[(size_t)i * p3 + j];
    }
    std::vector<double> wu, Qu, wv, Qv;
    jacobi_eigen(p3, GU, wu, Qu);
    ru = rank_at(wu, o.eps);
    if (sym) {
        // K^(-t) = K^(t)^T for a symmetric kernel, so both Gram matrices agree
        wv = wu;
        Qv = Qu;
        rv = ru;
    } else {
        jacobi_eigen(p3, GV, wv, Qv);
        rv = rank_at(wv, o.eps);
    }
    int r = std::max(ru, rv);
    o.r = r;
    sv.resize(p3);
    for (int i = 0; i < p3; ++i)
        sv[i] = sqrt(std::max(wu[i], 0.0));
    U.assign((size_t)p3 * r, 0.0);
    V.assign((size_t)p3 * r, 0.0);
    for (int i = 0; i < p3; ++i)
        for (int k = 0; k < r; ++k) {
            U[(size_t)i * r + k] = Qu[(size_t)i * p3 + k];
            V[(size_t)i * r + k] = Qv[(size_t)i * p3 + k];
        }
    C.assign((size_t)kNumOffsets * r * r, 0.0);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < kNumOffsets; ++t) {
        const double *Kt = &K[(size_t)t * p3 * p3];
        std::vector<double> KV((size_t)p3 * r, 0.0); // K^(t) V
        for (int i = 0; i < p3; ++i)
            for (int j = 0; j < p3; ++j) {
                double kij = Kt[(size_t)i * p3 + j];
                for (int k = 0; k < r; ++k)
                    KV[(size_t)i * r + k] += kij * V[(size_t)j * r + k];
            }
        double *Ct = &C[(size_t)t * r * r];
        for (int i = 0; i < p3; ++i)
            for (int a = 0; a < r; ++a) {
                double u = U[(size_t)i * r + a];
                for (int k = 0; k < r; ++k)
                    Ct[(size_t)a * r + k] += u * KV[(size_t)i * r + k];
            }
    }
    return true;
}

// spectra of the 316 kernel tables c_t of one level (box side h), equally
// spaced nodes: out[(w * 316 + u) * 2 + {0, 1}] = DFT(c_t)(w) / n^3 with
// DFT(c)(w) = sum_j c[j] exp(-2 pi i (w . j) / n), j, w in [0, n)^3, w =
// (wz n + wy) p + wx, wx < p
static bool build_khat(const HostOps &o, double h, std::vector<double> &out)
{
    const int p = o.p, n = 2 * p - 1, nw = n * n * p, n3 = n * n * n;
    out.assign((size_t)nw * kNumOffsets * 2, 0.0);
    std::vector<double> cs(n), sn(n);
    for (int k = 0; k < n; ++k) {
        cs[k] = cos(2.0 * M_PI * k / n);
        sn[k] = sin(2.0 * M_PI * k / n);
    }
    const double norm = 1.0 / ((double)n * n * n);
    // the kernel tables c_t[jz][jy][jx], j = d mod n for d in [-(p-1), p-1]
    std::vector<double> dv((size_t)kNumOffsets * n3 * 3), cv((size_t)kNumOffsets * n3);
    for (int t = 0; t < 343; ++t) {
        const int tx = t % 7 - 3, ty = (t / 7) % 7 - 3, tz = t / 49 - 3;
        const int u = offset_index(tx, ty, tz);
        if (u < 0)
            continue;
        for (int dz = 1 - p; dz < p; ++dz)
            for (int dy = 1 - p; dy < p; ++dy)
                for (int dx = 1 - p; dx < p; ++dx) {
                    const int jx = (dx + n) % n, jy = (dy + n) % n, jz = (dz + n) % n;
                    double *e = &dv[((size_t)u * n3 + ((size_t)jz * n + jy) * n + jx) * 3];
                    e[0] = h * (-tx + dx / (p - 1.0));
                    e[1] = h * (-ty + dy / (p - 1.0));
                    e[2] = h * (-tz + dz / (p - 1.0));
                }
    }
    if (!eval_kernel(o, dv.data(), (int64_t)kNumOffsets * n3, cv.data()))
        return false;
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < 343; ++t) {
        const int tx = t % 7 - 3, ty = (t / 7) % 7 - 3, tz = t / 49 - 3;
        const int u = offset_index(tx, ty, tz);
        if (u < 0)
            continue;
        const double *c = &cv[(size_t)u * n3];
        // x: real -> complex, wx < p; then y and z complex, all n frequencies
        std::vector<double> A((size_t)n * n * p * 2), B((size_t)n * n * p * 2);
        for (int jz = 0; jz < n; ++jz)
            for (int jy = 0; jy < n; ++jy)
                for (int wx = 0; wx < p; ++wx) {
                    double re = 0.0, im = 0.0;
                    for (int jx = 0; jx < n; ++jx) {
                        const double v = c[((size_t)jz * n + jy) * n + jx];
                        const int k = (wx * jx) % n;
                        re += v * cs[k];
                        im -= v * sn[k];
                    }
                    const size_t q = (((size_t)jz * n + jy) * p + wx) * 2;
                    A[q] = re;
                    A[q + 1] = im;
                }
        for (int jz = 0; jz < n; ++jz)
            for (int wy = 0; wy < n; ++wy)
                for (int wx = 0; wx < p; ++wx) {
                    double re = 0.0, im = 0.0;
                    for (int jy = 0; jy < n; ++jy) {
                        const size_t q = (((size_t)jz * n + jy) * p + wx) * 2;
                        const int k = (wy * jy) % n;
                        re += A[q] * cs[k] + A[q + 1] * sn[k];
                        im += A[q + 1] * cs[k] - A[q] * sn[k];
                    }
                    const size_t q = (((size_t)jz * n + wy) * p + wx) * 2;
                    B[q] = re;
                    B[q + 1] = im;
                }
        for (int wz = 0; wz < n; ++wz)
            for (int wy = 0; wy < n; ++wy)
                for (int wx = 0; wx < p; ++wx) {
                    double re = 0.0, im = 0.0;
                    for (int jz = 0; jz < n; ++jz) {
                        const size_t q = (((size_t)jz * n + wy) * p + wx) * 2;
                        const int k = (wz * jz) % n;
                        re += B[q] * cs[k] + B[q + 1] * sn[k];
                        im += B[q + 1] * cs[k] - B[q] * sn[k];
                    }
                    const size_t w = ((size_t)wz * n + wy) * p + wx;
                    out[(w * kNumOffsets + u) * 2] = re * norm;
                    out[(w * kNumOffsets + u) * 2 + 1] = im * norm;
                }
    }
    return true;
}

std::shared_ptr<HostOps> build_host_ops(int kernel, double ell, int p, double eps, int depth, double side,
                                        int interp, std::string &err)
{
    auto o = std::make_shared<HostOps>();
    o->kernel = kernel;
    o->ell = ell;
    o->p = p;
    o->p3 = p * p * p;
    o->eps = eps;
    o->hom_degree = kernel_homogeneity(kernel);
    o->interp = interp;
    o->nodes.resize(p);
    for (int k = 1; k <= p; ++k)
        o->nodes[k - 1] = interp == BBFMM_INTERP_UNIFORM ? -1.0 + 2.0 * (k - 1) / (p - 1.0)
                                                         : cos((2.0 * k - 1.0) * M_PI / (2.0 * p));
    o->wbary.resize(p);
    for (int i = 0; i < p; ++i) {
        double d = 1.0;
        for (int k = 0; k < p; ++k)
            if (k != i)
                d *= o->nodes[i] - o->nodes[k];
        o->wbary[i] = 1.0 / d;
    }
    o->S.assign(2 * p * p, 0.0);
    for (int oc = 0; oc < 2; ++oc)
        for (int j = 0; j < p; ++j) {
            double x = 0.5 * (o->nodes[j] + 2.0 * oc - 1.0);
            for (int i = 0; i < p; ++i) {
                double v = o->wbary[i];
                for (int k = 0; k < p; ++k)
                    if (k != i)
                        v *= x - o->nodes[k];
                o->S[(size_t)oc * p * p + (size_t)i * p + j] = v;
            }
        }
    if (depth < 2)
        return o; // no far field
    int nlev = o->hom_degree != 0 ? 1 : depth - 1;
    if (interp == BBFMM_INTERP_UNIFORM) {
        // no compression; the M2L works on the spectra of the kernel tables
        const int p3 = o->p3;
        o->nfft = 2 * p - 1;
        o->nw = o->nfft * o->nfft * p;
        o->r = o->rank_u = o->rank_v = p3;
        std::vector<double> I((size_t)p3 * p3, 0.0);
        for (int i = 0; i < p3; ++i)
            I[(size_t)i * p3 + i] = 1.0;
        for (int k = 0; k < nlev; ++k) {
            int level = o->hom_degree != 0 ? depth : k + 2;
            double h = side / (double)(1LL << level);
            o->h.push_back(h);
            o->rl.push_back(p3);
            o->U.push_back(I);
            o->V.push_back(I);
            o->khat.emplace_back();
            if (!build_khat(*o, h, o->khat.back())) {
                err = "evaluating the kernel tables failed";
                return nullptr;
            }
        }
        return o;
    }
    o->U.resize(nlev);
    o->V.resize(nlev);
    o->C.resize(nlev);
    o->sv.resize(nlev);
    o->h.resize(nlev);
    int rmax = 0;
    for (int k = 0; k < nlev; ++k) {
        int level = o->hom_degree != 0 ? depth : k + 2;
        double h = side / (double)(1LL << level);
        o->h[k] = h;
        int ru = 0, rv = 0;
        if (!build_level(*o, h, o->U[k], o->V[k], o->C[k], o->sv[k], ru, rv)) {
            err = "evaluating the M2L operators failed";
            return nullptr;
        }
        o->rl.push_back(o->r);
        o->rank_u = std::max(o->rank_u, ru);
        o->rank_v = std::max(o->rank_v, rv);
        rmax = std::max(rmax, o->r);
    }
    if (nlev > 1) {
        // levels may truncate at different ranks; pad every level to the largest
        for (int k = 0; k < nlev; ++k) {
            int r = (int)(o->U[k].size() / o->p3);
            if (r == rmax)
                continue;
            std::vector<double> U2((size_t)o->p3 * rmax, 0.0), V2((size_t)o->p3 * rmax, 0.0),
                C2((size_t)kNumOffsets * rmax * rmax, 0.0);
            for (int i = 0; i < o->p3; ++i)
                for (int a = 0; a < r; ++a) {
                    U2[(size_t)i * rmax + a] = o->U[k][(size_t)i * r + a];
                    V2[(size_t)i * rmax + a] = o->V[k][(size_t)i * r + a];
                }
            for (int t = 0; t < kNumOffsets; ++t)
                for (int a = 0; a < r; ++a)
                    for (int b = 0; b < r; ++b)
                        C2[((size_t)t * rmax + a) * rmax + b] = o->C[k][((size_t)t * r + a) * r + b];
            o->U[k].swap(U2);
            o->V[k].swap(V2);
            o->C[k].swap(C2);
        }
    }
    o->r = rmax;
    (void)err;
    return o;
}

} // namespace bbfmm
