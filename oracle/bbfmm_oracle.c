/*
 * bbfmm_oracle.c -- plain, slow FP64 CPU oracle for the black-box FMM of
 * "PBBFMM3D: a parallel black-box algorithm for kernel matrix-vector
 * multiplication" (Wang, Chen, Lee, Darve; arXiv 1903.02153).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code, header, table or constant with the CUDA library under
 * paper_1903_02153_gb300/csrc, and the CUDA library never calls it.
 *
 * What it computes, in the paper's order and notation:
 *   - the direct sum phi_i = sum_j K(x_i, y_j) sigma_j           (Sec. 1, Eq. summation)
 *   - the black-box FMM approximation of the same sum            (Sec. 2.3, four stages)
 *       upward pass:  P2M on leaves, M2M on non-leaves            (Sec. 2.3 item 1)
 *       far field:    M2L over the interaction list I(alpha)      (Sec. 2.3 item 2, Def. 2.1)
 *       downward:     L2L, then L2P on leaves                     (Sec. 2.3 item 3)
 *       near field:   P2P over the neighbours N(alpha)            (Sec. 2.3 item 4, Def. 2.1)
 *     with Chebyshev nodes or equally spaced nodes (the two node sets of
 *     Sec. 2.2), the 1D/3D Lagrange basis (Def. 2.2) and the M2L operator
 *     K(x*_i, y*_j) evaluated at the nodes of the two boxes, uncompressed
 *     (Eq. low-rank-form).  With equally spaced nodes that dense operator is
 *     the block-Toeplitz matrix the paper applies by FFT (Sec. 2.5 "Fast M2L
 *     translation"); the oracle applies it as the plain matrix product.  The 316 distinct
 *     translation operators of a level are tabulated once per level, as the
 *     memory discussion after Thm. 2.1 states.
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *   - domain: the caller gives the cube (lo, side); leaf cell of a point is
 *     min(floor((x - lo) / h_D), 2^D - 1) per axis, computed in FP64.
 *   - 3D index of a node: i = i1 + p*i2 + p*p*i3, 0-based, x fastest (the
 *     printed 1D/3D map in Sec. 2.2 is garbled).
 *   - levels: root = level 0, leaves = level D, 8^D leaves; M2L runs on
 *     levels 2..D (levels 0 and 1 have empty interaction lists).
 *   - K at r == 0: 0 for the singular kernels (1/r, 1/r^2), the natural value
 *     for the smooth ones.
 *   - the traversal is the level-by-level form Sec. 2.4 names as the
 *     alternative to the task-based one; results do not depend on it.
 *   - equally spaced nodes: the paper prints them on [0, 1] as (k-1)/(p-1);
 *     on the reference interval [-1, 1] of a box (where the Chebyshev nodes
 *     live) they are -1 + 2 (k-1)/(p-1), k = 1..p, end points included.
 *
 * Parity pins: tests/test_oracle_pins.py checks this file against numpy brute
 * force, closed forms, depth-0/1 identity with the direct sum, exact
 * reproduction of a low-degree polynomial kernel, the interaction-list
 * partition, symmetry, invariances and error decay in p, for both node sets;
 * the equally spaced nodes also against their closed form, and their M2L
 * operator against its block-Toeplitz structure applied by numpy's FFT.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* kernel ids (same numbers as the public header, restated here on purpose) */
#define ORK_INV_R 1
#define ORK_INV_R2 2
#define ORK_EXP 3
#define ORK_GAUSS 4
#define ORK_POLY 100
#define ORK_CONST 101
#define ORK_USER 1000 /* the function set by oracle_set_user_kernel */

static const double OR_PI = 3.14159265358979323846264338327950288;

/* K(x, y) for a translation-invariant kernel, as a function of d = x - y.
 * 1/r and 1/r^2: 0 at r == 0 (reading of "K can be singular at x = y", Sec. 1).
 * exp(-r/ell), exp(-(r/ell)^2): covariance kernels named in Sec. 4 (ell = 1 is
 * the paper's exp(-r)).
 * poly: q(d) = 1 + d1 - 2 d2 d3 + 3 d1^2 d2, degree <= 2 in every coordinate,
 * reproduced exactly by interpolation with p >= 3 nodes (Def. 2.2).
 * const: 1.
 * user: a caller-supplied function of d (the black-box interface: the method
 * needs only evaluations of K, Sec. 1). */
static double (*or_user_kernel)(double, double, double) = NULL;

void oracle_set_user_kernel(double (*k)(double, double, double)) { or_user_kernel = k; }

static double or_kernel(int kid, double ell, double d1, double d2, double d3)
{
    double r2 = d1 * d1 + d2 * d2 + d3 * d3;
    if (kid == ORK_USER)
        return or_user_kernel ? or_user_kernel(d1, d2, d3) : NAN;
    switch (kid) {
    case ORK_INV_R:
        return r2 == 0.0 ? 0.0 : 1.0 / sqrt(r2);
    case ORK_INV_R2:
        return r2 == 0.0 ? 0.0 : 1.0 / r2;
    case ORK_EXP:
        return exp(-sqrt(r2) / ell);
    case ORK_GAUSS:
        return exp(-r2 / (ell * ell));
    case ORK_POLY:
        return 1.0 + d1 - 2.0 * d2 * d3 + 3.0 * d1 * d1 * d2;
    case ORK_CONST:
        return 1.0;
    default:
        return NAN;
    }
}

double oracle_kernel(int kid, double ell, const double *x, const double *y)
{
    return or_kernel(kid, ell, x[0] - y[0], x[1] - y[1], x[2] - y[2]);
}

static double or_now(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* The dense kernel matrix K[i][j] = K(x_i, x_j) (n x n, row-major), whose
 * leading eigenvalues the randomized PCA of Sec. 4.3 approximates; the same
 * K(0) convention as everywhere else. */
void oracle_kernel_matrix(int64_t n, const double *x, int kid, double ell, double *K)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            K[i * n + j] = or_kernel(kid, ell, x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                                     x[3 * i + 2] - x[3 * j + 2]);
}

/* ------------------------------------------------------------------------- */
/* Direct sum, Sec. 1 Eq. summation: phi_i = sum_j K(x_i, y_j) sigma_j.
 * x: nt x 3 row-major targets, y: ns x 3 row-major sources,
 * sigma: ns x nrhs column-major, phi: nt x nrhs column-major (overwritten). */
void oracle_direct(int64_t nt, const double *x, int64_t ns, const double *y,
                   const double *sigma, int nrhs, int kid, double ell, double *phi)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < nt; ++i) {
        for (int c = 0; c < nrhs; ++c) {
            double acc = 0.0;
            for (int64_t j = 0; j < ns; ++j)
                acc += or_kernel(kid, ell, x[3 * i] - y[3 * j], x[3 * i + 1] - y[3 * j + 1],
                                 x[3 * i + 2] - y[3 * j + 2]) *
                       sigma[(int64_t)c * ns + j];
            phi[(int64_t)c * nt + i] = acc;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Interpolation: Chebyshev nodes (Sec. 2.2) and the Lagrange basis (Def. 2.2). */

/* S = { cos((2k - 1) pi / (2p)), k = 1..p }, stored 0-based. */
void oracle_cheb_nodes(int p, double *s)
{
    for (int k = 1; k <= p; ++k)
        s[k - 1] = cos((2.0 * k - 1.0) * OR_PI / (2.0 * p));
}

/* Equally spaced nodes (Sec. 2.2): (k-1)/(p-1) on [0, 1], i.e.
 * -1 + 2 (k-1)/(p-1) on [-1, 1], k = 1..p, stored 0-based. */
void oracle_uniform_nodes(int p, double *s)
{
    for (int k = 1; k <= p; ++k)
        s[k - 1] = -1.0 + 2.0 * (k - 1.0) / (p - 1.0);
}

/* ell_p(x*_i, x) = prod_{k != i} (x - x*_k) / (x*_i - x*_k), for i = 0..p-1. */
void oracle_lagrange_1d(int p, const double *s, double x, double *out)
{
    for (int i = 0; i < p; ++i) {
        double v = 1.0;
        for (int k = 0; k < p; ++k)
            if (k != i)
                v *= (x - s[k]) / (s[i] - s[k]);
        out[i] = v;
    }
}

/* L_p(x*_i, x) for all p^3 nodes i = i1 + p i2 + p^2 i3, where x is already
 * mapped to the reference cube [-1,1]^3 of the box. */
static void or_lagrange_3d(int p, const double *s, const double *xs, double *out)
{
    double l1[16], l2[16], l3[16];
    oracle_lagrange_1d(p, s, xs[0], l1);
    oracle_lagrange_1d(p, s, xs[1], l2);
    oracle_lagrange_1d(p, s, xs[2], l3);
    for (int i3 = 0; i3 < p; ++i3)
        for (int i2 = 0; i2 < p; ++i2)
            for (int i1 = 0; i1 < p; ++i1)
                out[i1 + p * i2 + p * p * i3] = l1[i1] * l2[i2] * l3[i3];
}

/* ------------------------------------------------------------------------- */
/* The uniform tree (Sec. 2.1): level l has 2^l boxes per axis of side
 * h_l = side / 2^l; box (a, b, c) has lexicographic index a + n (b + n c). */

typedef struct {
    int D, p, nrhs, kid;
    double ell, lo[3], side;
    int64_t n;
    const double *pts;
    const double *sigma;
    double *s;          /* p interpolation nodes on [-1, 1] */
    int64_t *leaf_of;   /* leaf index of each point */
    int64_t *lstart;    /* CSR over leaves: points of leaf b are order[lstart[b] .. lstart[b+1]) */
    int64_t *order;     /* point ids, increasing inside a leaf */
    double **M;         /* M[l]: 8^l boxes x nrhs x p^3 multipole coefficients */
    double **F;         /* F[l]: 8^l boxes x nrhs x p^3 local coefficients */
    unsigned char **nonempty; /* nonempty[l][box]: the box holds at least one point */
    unsigned char **needed;   /* needed[l][box]: the box is an ancestor of a sampled target */
} or_tree;

static int64_t or_nbox(int l) { return (int64_t)1 << (3 * l); }

static int64_t or_lex(int l, int64_t a, int64_t b, int64_t c)
{
    int64_t n = (int64_t)1 << l;
    return a + n * (b + n * c);
}

static void or_unlex(int l, int64_t idx, int64_t *a, int64_t *b, int64_t *c)
{
    int64_t n = (int64_t)1 << l;
    *a = idx % n;
    *b = (idx / n) % n;
    *c = idx / (n * n);
}

/* center of box (a, b, c) at level l */
static void or_center(const or_tree *t, int l, int64_t a, int64_t b, int64_t c, double *ctr)
{
    double h = t->side / (double)((int64_t)1 << l);
    ctr[0] = t->lo[0] + ((double)a + 0.5) * h;
    ctr[1] = t->lo[1] + ((double)b + 0.5) * h;
    ctr[2] = t->lo[2] + ((double)c + 0.5) * h;
}

/* leaf cell of coordinate x along one axis: min(floor((x - lo)/h_D), 2^D - 1) */
static int64_t or_cell(double x, double lo, double h, int D)
{
    double u = floor((x - lo) / h);
    int64_t nmax = ((int64_t)1 << D) - 1;
    if (u < 0.0)
        return 0;
    if (u > (double)nmax)
        return nmax;
    return (int64_t)u;
}

void oracle_leaf_cells(int64_t n, const double *pts, const double *lo, double side, int D,
                       int64_t *cells /* n x 3 */)
{
    double h = side / (double)((int64_t)1 << D);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            cells[3 * i + d] = or_cell(pts[3 * i + d], lo[d], h, D);
}

/* Def. 2.1: N(alpha) = same-level boxes adjacent to alpha, alpha included.
 * Writes (a, b, c) triples; returns the count (27 for an interior box). */
int oracle_neighbors(int l, int64_t a, int64_t b, int64_t c, int64_t *out)
{
    int64_t n = (int64_t)1 << l;
    int cnt = 0;
    for (int64_t dc = -1; dc <= 1; ++dc)
        for (int64_t db = -1; db <= 1; ++db)
            for (int64_t da = -1; da <= 1; ++da) {
                int64_t x = a + da, y = b + db, z = c + dc;
                if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n)
                    continue;
                out[3 * cnt] = x;
                out[3 * cnt + 1] = y;
                out[3 * cnt + 2] = z;
                ++cnt;
            }
    return cnt;
}

/* Def. 2.1: I(alpha) = C(N(P(alpha))) \ N(alpha): children of the parent's
 * neighbours that are not neighbours of alpha.  Enumerated literally.
 * Returns the count (189 for an interior box), 0 on levels 0 and 1. */
int oracle_interaction_list(int l, int64_t a, int64_t b, int64_t c, int64_t *out)
{
    if (l < 1)
        return 0;
    int64_t pn[27 * 3];
    int np = oracle_neighbors(l - 1, a >> 1, b >> 1, c >> 1, pn);
    int cnt = 0;
    for (int k = 0; k < np; ++k)
        for (int oc = 0; oc < 2; ++oc)
            for (int ob = 0; ob < 2; ++ob)
                for (int oa = 0; oa < 2; ++oa) {
                    int64_t x = 2 * pn[3 * k] + oa, y = 2 * pn[3 * k + 1] + ob, z = 2 * pn[3 * k + 2] + oc;
                    int64_t dx = x - a, dy = y - b, dz = z - c;
                    int adjacent = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
                    if (adjacent)
                        continue;
                    out[3 * cnt] = x;
                    out[3 * cnt + 1] = y;
                    out[3 * cnt + 2] = z;
                    ++cnt;
                }
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Stage 1, upward pass (Sec. 2.3 item 1). */

/* P2M: M^alpha_i = sum_{y_j in alpha} L_p(y*_i, y_j) sigma_j */
static void or_p2m(or_tree *t)
{
    int D = t->D, p = t->p, p3 = p * p * p;
    int64_t nb = or_nbox(D);
    double h = t->side / (double)((int64_t)1 << D);
    int64_t bi;
#pragma omp parallel for schedule(dynamic, 64)
    for (bi = 0; bi < nb; ++bi) {
        if (t->lstart[bi] == t->lstart[bi + 1])
            continue;
        int64_t a, b, c;
        or_unlex(D, bi, &a, &b, &c);
        double ctr[3], xs[3], L[1000];
        or_center(t, D, a, b, c, ctr);
        double *M = t->M[D] + bi * (int64_t)t->nrhs * p3;
        for (int64_t q = t->lstart[bi]; q < t->lstart[bi + 1]; ++q) {
            int64_t j = t->order[q];
            for (int d = 0; d < 3; ++d)
                xs[d] = 2.0 * (t->pts[3 * j + d] - ctr[d]) / h;
            or_lagrange_3d(p, t->s, xs, L);
            for (int r = 0; r < t->nrhs; ++r) {
                double sg = t->sigma[(int64_t)r * t->n + j];
                for (int i = 0; i < p3; ++i)
                    M[(int64_t)r * p3 + i] += L[i] * sg;
            }
        }
    }
}

/* M2M: M^alpha_i = sum_{beta in C(alpha)} sum_j L_p(y*_i, y*_j) M^beta_j, where
 * y*_i are the nodes of alpha and y*_j those of the child beta. */
static void or_m2m(or_tree *t, int l /* parent level */)
{
    int p = t->p, p3 = p * p * p, nr = t->nrhs;
    int64_t nb = or_nbox(l);
    double hp = t->side / (double)((int64_t)1 << l);
    double hc = hp * 0.5;
    int64_t bi;
#pragma omp parallel for schedule(dynamic, 16)
    for (bi = 0; bi < nb; ++bi) {
        if (!t->nonempty[l][bi])
            continue;
        int64_t a, b, c;
        or_unlex(l, bi, &a, &b, &c);
        double cp[3], cc[3], xs[3];
        double *Lrow = (double *)malloc(sizeof(double) * p3);
        or_center(t, l, a, b, c, cp);
        double *Mp = t->M[l] + bi * (int64_t)nr * p3;
        for (int oc = 0; oc < 2; ++oc)
            for (int ob = 0; ob < 2; ++ob)
                for (int oa = 0; oa < 2; ++oa) {
                    int64_t ch = or_lex(l + 1, 2 * a + oa, 2 * b + ob, 2 * c + oc);
                    if (!t->nonempty[l + 1][ch])
                        continue;
                    or_center(t, l + 1, 2 * a + oa, 2 * b + ob, 2 * c + oc, cc);
                    const double *Mc = t->M[l + 1] + ch * (int64_t)nr * p3;
                    for (int j3 = 0; j3 < p; ++j3)
                        for (int j2 = 0; j2 < p; ++j2)
                            for (int j1 = 0; j1 < p; ++j1) {
                                int j = j1 + p * j2 + p * p * j3;
                                /* child node y*_j, mapped into the parent's [-1,1]^3 */
                                double y0 = cc[0] + 0.5 * hc * t->s[j1];
                                double y1 = cc[1] + 0.5 * hc * t->s[j2];
                                double y2 = cc[2] + 0.5 * hc * t->s[j3];
                                xs[0] = 2.0 * (y0 - cp[0]) / hp;
                                xs[1] = 2.0 * (y1 - cp[1]) / hp;
                                xs[2] = 2.0 * (y2 - cp[2]) / hp;
                                or_lagrange_3d(p, t->s, xs, Lrow); /* Lrow[i] = L_p(y*_i, y*_j) */
                                for (int r = 0; r < nr; ++r) {
                                    double m = Mc[(int64_t)r * p3 + j];
                                    for (int i = 0; i < p3; ++i)
                                        Mp[(int64_t)r * p3 + i] += Lrow[i] * m;
                                }
                            }
                }
        free(Lrow);
    }
}

/* ------------------------------------------------------------------------- */
/* Stage 2, far field (Sec. 2.3 item 2):
 *   F^alpha_i = sum_{beta in I(alpha)} sum_j K(x*_i, y*_j) M^beta_j.
 * K(x*_i, y*_j) depends only on the offset t = beta - alpha (translation
 * invariance), so the operator of each of the 7^3 - 3^3 = 316 offsets is
 * tabulated once per level (discussion after Thm. 2.1). */
static void or_m2l(or_tree *t, int l)
{
    int p = t->p, p3 = p * p * p, nr = t->nrhs;
    int64_t nb = or_nbox(l);
    double h = t->side / (double)((int64_t)1 << l);
    /* Kt[(tx+3) + 7 (ty+3) + 49 (tz+3)]: p3 x p3 row-major, row i = target node */
    double **Kt = (double **)calloc(343, sizeof(double *));
    for (int tz = -3; tz <= 3; ++tz)
        for (int ty = -3; ty <= 3; ++ty)
            for (int tx = -3; tx <= 3; ++tx) {
                if (tx >= -1 && tx <= 1 && ty >= -1 && ty <= 1 && tz >= -1 && tz <= 1)
                    continue;
                double *K = (double *)malloc(sizeof(double) * p3 * p3);
                for (int i = 0; i < p3; ++i) {
                    int i1 = i % p, i2 = (i / p) % p, i3 = i / (p * p);
                    /* target box centred at the origin, source box centred at t h */
                    double x0 = 0.5 * h * t->s[i1], x1 = 0.5 * h * t->s[i2], x2 = 0.5 * h * t->s[i3];
                    for (int j = 0; j < p3; ++j) {
                        int j1 = j % p, j2 = (j / p) % p, j3 = j / (p * p);
                        double y0 = tx * h + 0.5 * h * t->s[j1];
                        double y1 = ty * h + 0.5 * h * t->s[j2];
                        double y2 = tz * h + 0.5 * h * t->s[j3];
                        K[(int64_t)i * p3 + j] = or_kernel(t->kid, t->ell, x0 - y0, x1 - y1, x2 - y2);
                    }
                }
                Kt[(tx + 3) + 7 * (ty + 3) + 49 * (tz + 3)] = K;
            }
    int64_t bi;
#pragma omp parallel for schedule(dynamic, 8)
    for (bi = 0; bi < nb; ++bi) {
        if (!t->needed[l][bi])
            continue;
        int64_t a, b, c, il[189 * 3];
        or_unlex(l, bi, &a, &b, &c);
        int ni = oracle_interaction_list(l, a, b, c, il);
        double *Fa = t->F[l] + bi * (int64_t)nr * p3;
        for (int k = 0; k < ni; ++k) {
            int64_t bb = or_lex(l, il[3 * k], il[3 * k + 1], il[3 * k + 2]);
            if (!t->nonempty[l][bb])
                continue;
            int tx = (int)(il[3 * k] - a), ty = (int)(il[3 * k + 1] - b), tz = (int)(il[3 * k + 2] - c);
            const double *K = Kt[(tx + 3) + 7 * (ty + 3) + 49 * (tz + 3)];
            const double *Mb = t->M[l] + bb * (int64_t)nr * p3;
            for (int r = 0; r < nr; ++r)
                for (int i = 0; i < p3; ++i) {
                    double acc = 0.0;
                    for (int j = 0; j < p3; ++j)
                        acc += K[(int64_t)i * p3 + j] * Mb[(int64_t)r * p3 + j];
                    Fa[(int64_t)r * p3 + i] += acc;
                }
        }
    }
    for (int k = 0; k < 343; ++k)
        free(Kt[k]);
    free(Kt);
}

/* ------------------------------------------------------------------------- */
/* Stage 3, downward pass (Sec. 2.3 item 3). */

/* L2L: F^alpha_i += sum_j F^beta_j L_p(x*_j, x*_i), beta = P(alpha); x*_j are the
 * nodes of the parent beta, x*_i those of alpha. */
static void or_l2l(or_tree *t, int l /* child level */)
{
    int p = t->p, p3 = p * p * p, nr = t->nrhs;
    int64_t nb = or_nbox(l);
    double hc = t->side / (double)((int64_t)1 << l);
    double hp = 2.0 * hc;
    int64_t bi;
#pragma omp parallel for schedule(dynamic, 16)
    for (bi = 0; bi < nb; ++bi) {
        if (!t->needed[l][bi])
            continue;
        int64_t a, b, c;
        or_unlex(l, bi, &a, &b, &c);
        int64_t par = or_lex(l - 1, a >> 1, b >> 1, c >> 1);
        double cc[3], cp[3], xs[3];
        double *Lcol = (double *)malloc(sizeof(double) * p3);
        or_center(t, l, a, b, c, cc);
        or_center(t, l - 1, a >> 1, b >> 1, c >> 1, cp);
        const double *Fp = t->F[l - 1] + par * (int64_t)nr * p3;
        double *Fc = t->F[l] + bi * (int64_t)nr * p3;
        for (int i3 = 0; i3 < p; ++i3)
            for (int i2 = 0; i2 < p; ++i2)
                for (int i1 = 0; i1 < p; ++i1) {
                    int i = i1 + p * i2 + p * p * i3;
                    double x0 = cc[0] + 0.5 * hc * t->s[i1];
                    double x1 = cc[1] + 0.5 * hc * t->s[i2];
                    double x2 = cc[2] + 0.5 * hc * t->s[i3];
                    xs[0] = 2.0 * (x0 - cp[0]) / hp;
                    xs[1] = 2.0 * (x1 - cp[1]) / hp;
                    xs[2] = 2.0 * (x2 - cp[2]) / hp;
                    or_lagrange_3d(p, t->s, xs, Lcol); /* Lcol[j] = L_p(x*_j, x*_i) */
                    for (int r = 0; r < nr; ++r) {
                        double acc = 0.0;
                        for (int j = 0; j < p3; ++j)
                            acc += Fp[(int64_t)r * p3 + j] * Lcol[j];
                        Fc[(int64_t)r * p3 + i] += acc;
                    }
                }
        free(Lcol);
    }
}

/* L2P: phi_i = sum_j F^alpha_j L_p(x*_j, x_i) for a target x_i in leaf alpha. */
static void or_l2p(const or_tree *t, const double *x, int64_t bi, double *out /* nrhs */)
{
    int D = t->D, p = t->p, p3 = p * p * p;
    double h = t->side / (double)((int64_t)1 << D);
    int64_t a, b, c;
    or_unlex(D, bi, &a, &b, &c);
    double ctr[3], xs[3], L[1000];
    or_center(t, D, a, b, c, ctr);
    for (int d = 0; d < 3; ++d)
        xs[d] = 2.0 * (x[d] - ctr[d]) / h;
    or_lagrange_3d(p, t->s, xs, L);
    const double *F = t->F[D] + bi * (int64_t)t->nrhs * p3;
    for (int r = 0; r < t->nrhs; ++r) {
        double acc = 0.0;
        for (int j = 0; j < p3; ++j)
            acc += F[(int64_t)r * p3 + j] * L[j];
        out[r] = acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Stage 4, near field (Sec. 2.3 item 4):
 *   phi_i += sum_{beta in N(alpha)} sum_{y_j in beta} K(x_i, y_j) sigma_j. */
static void or_p2p(const or_tree *t, const double *x, int64_t bi, double *out /* nrhs */)
{
    int D = t->D;
    int64_t a, b, c, nb[27 * 3];
    or_unlex(D, bi, &a, &b, &c);
    int nn = oracle_neighbors(D, a, b, c, nb);
    for (int k = 0; k < nn; ++k) {
        int64_t bj = or_lex(D, nb[3 * k], nb[3 * k + 1], nb[3 * k + 2]);
        for (int64_t q = t->lstart[bj]; q < t->lstart[bj + 1]; ++q) {
            int64_t j = t->order[q];
            double K = or_kernel(t->kid, t->ell, x[0] - t->pts[3 * j], x[1] - t->pts[3 * j + 1],
                                 x[2] - t->pts[3 * j + 2]);
            for (int r = 0; r < t->nrhs; ++r)
                out[r] += K * t->sigma[(int64_t)r * t->n + j];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* The whole FMM (Alg. 1 without the OpenMP task structure), for targets
 * tx[q] (ntgt x 3 row-major) lying in leaves tleaf[q] of the source tree. */
static int or_run(or_tree *t, int64_t ntgt, const double *tx, const int64_t *tleaf, double *phi,
                  double *M_dump, double *F_dump, double *times);

/* Bin the sources of t into leaves (FMMDistribute, Sec. 3): a counting sort
 * keeps increasing point ids inside each leaf. */
static void or_bin_sources(or_tree *t)
{
    int D = t->D;
    int64_t n = t->n, nleaf = or_nbox(D);
    double hD = t->side / (double)((int64_t)1 << D);
    t->leaf_of = (int64_t *)malloc(sizeof(int64_t) * n);
    t->lstart = (int64_t *)calloc(nleaf + 1, sizeof(int64_t));
    t->order = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = or_cell(t->pts[3 * i], t->lo[0], hD, D);
        int64_t b = or_cell(t->pts[3 * i + 1], t->lo[1], hD, D);
        int64_t c = or_cell(t->pts[3 * i + 2], t->lo[2], hD, D);
        t->leaf_of[i] = or_lex(D, a, b, c);
        t->lstart[t->leaf_of[i] + 1]++;
    }
    for (int64_t k = 0; k < nleaf; ++k)
        t->lstart[k + 1] += t->lstart[k];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nleaf);
    memcpy(fill, t->lstart, sizeof(int64_t) * nleaf);
    for (int64_t i = 0; i < n; ++i)
        t->order[fill[t->leaf_of[i]]++] = i;
    free(fill);
}

static int or_setup(or_tree *t, int64_t n, const double *pts, const double *sigma, int nrhs, int kid, double ell,
                    int p, int D, const double *lo, double side, int nodes)
{
    if (n < 1 || nrhs < 1 || nrhs > 256 || p < 2 || p > 10 || D < 0 || D > 8 || !(side > 0.0) ||
        (nodes != 0 && nodes != 1))
        return -1;
    memset(t, 0, sizeof(*t));
    t->D = D;
    t->p = p;
    t->nrhs = nrhs;
    t->kid = kid;
    t->ell = ell;
    t->lo[0] = lo[0];
    t->lo[1] = lo[1];
    t->lo[2] = lo[2];
    t->side = side;
    t->n = n;
    t->pts = pts;
    t->sigma = sigma;
    t->s = (double *)malloc(sizeof(double) * p);
    if (nodes == 0)
        oracle_cheb_nodes(p, t->s);
    else
        oracle_uniform_nodes(p, t->s);
    or_bin_sources(t);
    return 0;
}

/* pts: n x 3 row-major (targets = sources), sigma: n x nrhs column-major.
 * lo[3], side: the cubical domain.  nodes: 0 = Chebyshev, 1 = equally spaced.
 * p: nodes per axis (2..10).
 * D: depth, 8^D leaves.  nsample >= 0 with sample != NULL: phi is produced only
 * for those targets (phi: nsample x nrhs column-major); the far field is then
 * computed only for the boxes on their ancestor chains, which gives the same
 * values for those targets.  nsample < 0: all targets (phi: n x nrhs).
 * M_dump / F_dump (optional): levels 0..D concatenated, each 8^l x nrhs x p^3
 * in lexicographic box order.  times (optional, 4 doubles): seconds spent in
 * upward pass, far field, downward pass, near field.
 * Returns 0, or -1 on invalid arguments. */
int oracle_bbfmm(int64_t n, const double *pts, const double *sigma, int nrhs, int kid, double ell,
                 int p, int D, const double *lo, double side, int nodes, int64_t nsample, const int64_t *sample,
                 double *phi, double *M_dump, double *F_dump, double *times)
{
    or_tree t;
    if (or_setup(&t, n, pts, sigma, nrhs, kid, ell, p, D, lo, side, nodes) != 0)
        return -1;
    int64_t ntgt = nsample >= 0 && sample ? nsample : n;
    double *tx = (double *)malloc(sizeof(double) * 3 * ntgt);
    int64_t *tleaf = (int64_t *)malloc(sizeof(int64_t) * ntgt);
    for (int64_t q = 0; q < ntgt; ++q) {
        int64_t i = nsample >= 0 && sample ? sample[q] : q;
        memcpy(tx + 3 * q, pts + 3 * i, sizeof(double) * 3);
        tleaf[q] = t.leaf_of[i];
    }
    int rc = or_run(&t, ntgt, tx, tleaf, phi, M_dump, F_dump, times);
    free(tx);
    free(tleaf);
    return rc;
}

/* Separate targets (Sec. 1: the target and source sets may differ; here
 * they share the domain, which must contain both): sources src (ns x 3) with
 * weights sigma (ns x nrhs column-major), targets tgt (nt x 3); phi: nt x nrhs
 * column-major.  Every other argument as in oracle_bbfmm.  Returns 0, or -1
 * on invalid arguments. */
int oracle_bbfmm_targets(int64_t ns, const double *src, const double *sigma, int nrhs, int kid, double ell,
                         int p, int D, const double *lo, double side, int nodes, int64_t nt, const double *tgt,
                         double *phi, double *times)
{
    or_tree t;
    if (nt < 1 || or_setup(&t, ns, src, sigma, nrhs, kid, ell, p, D, lo, side, nodes) != 0)
        return -1;
    double hD = side / (double)((int64_t)1 << D);
    int64_t *tleaf = (int64_t *)malloc(sizeof(int64_t) * nt);
    for (int64_t q = 0; q < nt; ++q)
        tleaf[q] = or_lex(D, or_cell(tgt[3 * q], lo[0], hD, D), or_cell(tgt[3 * q + 1], lo[1], hD, D),
                          or_cell(tgt[3 * q + 2], lo[2], hD, D));
    int rc = or_run(&t, nt, tgt, tleaf, phi, NULL, NULL, times);
    free(tleaf);
    return rc;
}

static int or_run(or_tree *tp, int64_t ntgt, const double *tx, const int64_t *tleaf, double *phi,
                  double *M_dump, double *F_dump, double *times)
{
    or_tree t = *tp;
    int D = t.D, p = t.p, nrhs = t.nrhs;
    int p3 = p * p * p;
    int64_t nleaf = or_nbox(D);
    double tm[4] = {0, 0, 0, 0}, t0;

    t.M = (double **)calloc(D + 1, sizeof(double *));
    t.F = (double **)calloc(D + 1, sizeof(double *));
    t.nonempty = (unsigned char **)calloc(D + 1, sizeof(unsigned char *));
    t.needed = (unsigned char **)calloc(D + 1, sizeof(unsigned char *));
    for (int l = 0; l <= D; ++l) {
        t.M[l] = (double *)calloc(or_nbox(l) * nrhs * p3, sizeof(double));
        t.F[l] = (double *)calloc(or_nbox(l) * nrhs * p3, sizeof(double));
        t.nonempty[l] = (unsigned char *)calloc(or_nbox(l), 1);
        t.needed[l] = (unsigned char *)calloc(or_nbox(l), 1);
    }
    for (int64_t k = 0; k < nleaf; ++k)
        t.nonempty[D][k] = t.lstart[k + 1] > t.lstart[k];
    for (int l = D - 1; l >= 0; --l)
        for (int64_t k = 0; k < or_nbox(l + 1); ++k)
            if (t.nonempty[l + 1][k]) {
                int64_t a, b, c;
                or_unlex(l + 1, k, &a, &b, &c);
                t.nonempty[l][or_lex(l, a >> 1, b >> 1, c >> 1)] = 1;
            }
    for (int64_t q = 0; q < ntgt; ++q) {
        int64_t a, b, c;
        or_unlex(D, tleaf[q], &a, &b, &c);
        for (int l = D; l >= 0; --l)
            t.needed[l][or_lex(l, a >> (D - l), b >> (D - l), c >> (D - l))] = 1;
    }

    /* 1. upward pass */
    t0 = or_now();
    or_p2m(&t);
    for (int l = D - 1; l >= 2; --l)
        or_m2m(&t, l);
    tm[0] = or_now() - t0;

    /* 2. far field: levels 2..D (I(alpha) is empty on levels 0 and 1) */
    t0 = or_now();
    for (int l = 2; l <= D; ++l)
        or_m2l(&t, l);
    tm[1] = or_now() - t0;

    /* 3. downward pass: L2L from level 3 on (F vanishes above level 2), then L2P */
    t0 = or_now();
    for (int l = 3; l <= D; ++l)
        or_l2l(&t, l);
    int64_t q;
#pragma omp parallel for schedule(dynamic, 256)
    for (q = 0; q < ntgt; ++q) {
        double out[256];
        if (D >= 2) {
            or_l2p(&t, tx + 3 * q, tleaf[q], out);
        } else {
            for (int r = 0; r < nrhs; ++r)
                out[r] = 0.0;
        }
        for (int r = 0; r < nrhs; ++r)
            phi[(int64_t)r * ntgt + q] = out[r];
    }
    tm[2] = or_now() - t0;

    /* 4. near field */
    t0 = or_now();
#pragma omp parallel for schedule(dynamic, 256)
    for (q = 0; q < ntgt; ++q) {
        double out[256];
        for (int r = 0; r < nrhs; ++r)
            out[r] = 0.0;
        or_p2p(&t, tx + 3 * q, tleaf[q], out);
        for (int r = 0; r < nrhs; ++r)
            phi[(int64_t)r * ntgt + q] += out[r];
    }
    tm[3] = or_now() - t0;

    if (M_dump || F_dump) {
        int64_t off = 0;
        for (int l = 0; l <= D; ++l) {
            int64_t cnt = or_nbox(l) * nrhs * p3;
            if (M_dump)
                memcpy(M_dump + off, t.M[l], sizeof(double) * cnt);
            if (F_dump)
                memcpy(F_dump + off, t.F[l], sizeof(double) * cnt);
            off += cnt;
        }
    }
    if (times)
        memcpy(times, tm, sizeof(tm));

    for (int l = 0; l <= D; ++l) {
        free(t.M[l]);
        free(t.F[l]);
        free(t.nonempty[l]);
        free(t.needed[l]);
    }
    free(t.M);
    free(t.F);
    free(t.nonempty);
    free(t.needed);
    free(t.leaf_of);
    free(t.lstart);
    free(t.order);
    free(t.s);
    return 0;
}
