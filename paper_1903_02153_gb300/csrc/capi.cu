// capi.cu -- the C ABI of include/bbfmm.h: plan construction (tree build on
// the device, FP64 operators on the host, buffer layout), the matvec driver
// that enqueues the four stages of Sec. 2.3 (Alg. 1 as level-synchronous
// kernels, near field on a forked stream), and introspection helpers.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <map>
#include <tuple>

#include "bbfmm_internal.h"
#include "p2p_kernels.cuh" // CloseArgs

namespace bbfmm {

static thread_local std::string g_last_error;

static int fail(int status, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

#define CUDA_TRY(call)                                                                                         \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess)                                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? BBFMM_ENOMEM : BBFMM_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                           \
    } while (0)

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------------------
// operator cache: one device copy per (kernel, ell, p, eps, depth, side)
DevOps::~DevOps()
{
    for (auto *v : {&V, &Ut, &C, &Chi, &Clo, &Vt_hi, &Vt_lo, &U_hi, &U_lo})
        for (float *ptr : *v)
            if (ptr)
                cudaFree(ptr);
    for (int f = 0; f < 2; ++f)
        for (auto *v : {&C16hi[f], &C16lo[f]})
            for (uint16_t *ptr : *v)
                if (ptr)
                    cudaFree(ptr);
    for (float2 *ptr : khat)
        if (ptr)
            cudaFree(ptr);
}

// 16-bit split copies of the M2L operators (fmt 0 = FP16 scaled by a power of
// two per operator level so that max |C| s lies in (2^12, 2^13]; 1 = BF16)
int ensure_ops16(DevOps &O, int fmt)
{
    std::lock_guard<std::mutex> g(O.mu16);
    if ((int)O.C16hi[fmt].size() == O.nlev)
        return BBFMM_OK;
    const HostOps &h = *O.host;
    const int r = O.r, rp = O.rp, rows64 = O.rows64;
    for (int k = 0; k < O.nlev; ++k) {
        double mx = 0.0;
        for (double v : h.C[k])
            mx = std::max(mx, fabs(v));
        int e = 0;
        if (mx > 0.0)
            frexp(mx, &e);
        const float s = fmt == 0 ? (float)ldexp(1.0, 13 - e) : 1.0f;
        const size_t cnt = (size_t)kNumOffsets * rows64 * rp;
        std::vector<uint16_t> hi(cnt, 0), lo(cnt, 0);
        for (int t = 0; t < kNumOffsets; ++t)
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) {
                    const float x = (float)h.C[k][((size_t)t * r + a) * r + b] * s;
                    const size_t i = ((size_t)t * rows64 + a) * rp + b;
                    if (fmt == 0) {
                        __half hh = __float2half_rn(x);
                        hi[i] = __half_as_ushort(hh);
                        lo[i] = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
                    } else {
                        __nv_bfloat16 hh = __float2bfloat16_rn(x);
                        hi[i] = __bfloat16_as_ushort(hh);
                        lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hh)));
                    }
                }
        uint16_t *dhi = nullptr, *dlo = nullptr;
        CUDA_TRY(cudaMalloc(&dhi, cnt * 2));
        O.C16hi[fmt].push_back(dhi);
        CUDA_TRY(cudaMalloc(&dlo, cnt * 2));
        O.C16lo[fmt].push_back(dlo);
        CUDA_TRY(cudaMemcpy(dhi, hi.data(), cnt * 2, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(dlo, lo.data(), cnt * 2, cudaMemcpyHostToDevice));
        O.c16_scale[fmt].push_back(s);
        O.bytes += (int64_t)cnt * 4;
    }
    return BBFMM_OK;
}

typedef std::tuple<int, double, int, double, int, double, int, int> OpsKey;
static std::mutex g_ops_mu;
static std::map<OpsKey, std::weak_ptr<DevOps>> g_ops_cache;

void split_tf32(const float *in, float *hi, float *lo, int64_t n); // m2l_tc.cu (host helper)

static int get_ops(int kernel, double ell, int p, double eps, int depth, double side, int device, int interp,
                   std::shared_ptr<DevOps> &out)
{
    // homogeneous kernels depend on the domain only through h_D
    double key_side = side;
    int key_depth = depth;
    if (kernel_homogeneity(kernel) != 0) {
        key_side = side / (double)(1LL << depth);
        key_depth = 0;
    }
    if (interp == BBFMM_INTERP_UNIFORM)
        eps = 0.0; // no compression
    OpsKey key(kernel, ell, p, eps, key_depth, key_side, device, interp);
    std::lock_guard<std::mutex> g(g_ops_mu);
    auto it = g_ops_cache.find(key);
    if (it != g_ops_cache.end()) {
        if (auto sp = it->second.lock()) {
            out = sp;
            return BBFMM_OK;
        }
    }
    std::string err;
    auto host = build_host_ops(kernel, ell, p, eps, depth, side, interp, err);
    if (!host)
        return fail(BBFMM_EINTERNAL, "operator precompute failed: %s", err.c_str());
    auto d = std::make_shared<DevOps>();
    d->host = host;
    d->nlev = (int)host->U.size(); // operator levels (both node sets)
    d->r = host->r;
    d->rl = host->rl;
    d->rp = (int)round_up(std::max(host->r, 1), 16);
    d->rows64 = (int)round_up(std::max(host->r, 1), 64);
    d->p3p = (int)round_up(host->p3, 16);
    const int p3 = host->p3, r = host->r, rp = d->rp, rows64 = d->rows64, p3p = d->p3p;
    d->nfft = host->nfft;
    d->nw = host->nw;
    for (int k = 0; k < d->nlev; ++k) {
        std::vector<float> V((size_t)p3 * rp, 0.f), Ut((size_t)r * p3p, 0.f);
        for (int i = 0; i < p3; ++i)
            for (int a = 0; a < r; ++a) {
                V[(size_t)i * rp + a] = (float)host->V[k][(size_t)i * r + a];
                Ut[(size_t)a * p3p + i] = (float)host->U[k][(size_t)i * r + a];
            }
        float *dV = nullptr, *dUt = nullptr;
        CUDA_TRY(cudaMalloc(&dV, V.size() * 4));
        d->V.push_back(dV);
        CUDA_TRY(cudaMalloc(&dUt, Ut.size() * 4));
        d->Ut.push_back(dUt);
        CUDA_TRY(cudaMemcpy(dV, V.data(), V.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(dUt, Ut.data(), Ut.size() * 4, cudaMemcpyHostToDevice));
        d->bytes += (int64_t)(V.size() + Ut.size()) * 4;
        if (host->interp == BBFMM_INTERP_CHEBYSHEV) {
            // V transposed ([rp][p3p], K = p3 contiguous), split into TF32 hi / lo
            // for the leaf compression GEMM; columns past the level's rank zero
            std::vector<float> Vt((size_t)rp * p3p, 0.f), Vh(Vt.size()), Vl(Vt.size());
            const int rk = host->rl[k];
            for (int a = 0; a < rk; ++a)
                for (int i = 0; i < p3; ++i)
                    Vt[(size_t)a * p3p + i] = (float)host->V[k][(size_t)i * r + a];
            split_tf32(Vt.data(), Vh.data(), Vl.data(), (int64_t)Vt.size());
            float *dh = nullptr, *dl = nullptr;
            CUDA_TRY(cudaMalloc(&dh, Vt.size() * 4));
            d->Vt_hi.push_back(dh);
            CUDA_TRY(cudaMalloc(&dl, Vt.size() * 4));
            d->Vt_lo.push_back(dl);
            CUDA_TRY(cudaMemcpy(dh, Vh.data(), Vt.size() * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(dl, Vl.data(), Vt.size() * 4, cudaMemcpyHostToDevice));
            d->bytes += (int64_t)(2 * Vt.size()) * 4;
            // U ([p3p][rp], K = r contiguous) for the leaf decompression GEMM
            std::vector<float> Um((size_t)p3p * rp, 0.f), Uh(Um.size()), Ul(Um.size());
            for (int i = 0; i < p3; ++i)
                for (int a = 0; a < rk; ++a)
                    Um[(size_t)i * rp + a] = (float)host->U[k][(size_t)i * r + a];
            split_tf32(Um.data(), Uh.data(), Ul.data(), (int64_t)Um.size());
            float *uh = nullptr, *ul = nullptr;
            CUDA_TRY(cudaMalloc(&uh, Um.size() * 4));
            d->U_hi.push_back(uh);
            CUDA_TRY(cudaMalloc(&ul, Um.size() * 4));
            d->U_lo.push_back(ul);
            CUDA_TRY(cudaMemcpy(uh, Uh.data(), Um.size() * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(ul, Ul.data(), Um.size() * 4, cudaMemcpyHostToDevice));
            d->bytes += (int64_t)(2 * Um.size()) * 4;
        }
        if (host->interp == BBFMM_INTERP_UNIFORM) {
            // kernel spectra for the Fourier-domain M2L
            const std::vector<double> &kh = host->khat[k];
            std::vector<float2> hk(kh.size() / 2);
            for (size_t q = 0; q < hk.size(); ++q)
                hk[q] = make_float2((float)kh[2 * q], (float)kh[2 * q + 1]);
            float2 *dk = nullptr;
            CUDA_TRY(cudaMalloc(&dk, hk.size() * sizeof(float2)));
            d->khat.push_back(dk);
            CUDA_TRY(cudaMemcpy(dk, hk.data(), hk.size() * sizeof(float2), cudaMemcpyHostToDevice));
            d->bytes += (int64_t)hk.size() * 8;
            continue;
        }
        std::vector<float> C((size_t)kNumOffsets * rows64 * rp, 0.f);
        for (int t = 0; t < kNumOffsets; ++t)
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b)
                    C[((size_t)t * rows64 + a) * rp + b] = (float)host->C[k][((size_t)t * r + a) * r + b];
        std::vector<float> Chi(C.size()), Clo(C.size());
        split_tf32(C.data(), Chi.data(), Clo.data(), (int64_t)C.size());
        float *dC = nullptr, *dChi = nullptr, *dClo = nullptr;
        CUDA_TRY(cudaMalloc(&dC, C.size() * 4));
        d->C.push_back(dC);
        CUDA_TRY(cudaMalloc(&dChi, C.size() * 4));
        d->Chi.push_back(dChi);
        CUDA_TRY(cudaMalloc(&dClo, C.size() * 4));
        d->Clo.push_back(dClo);
        CUDA_TRY(cudaMemcpy(dC, C.data(), C.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(dChi, Chi.data(), C.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(dClo, Clo.data(), C.size() * 4, cudaMemcpyHostToDevice));
        d->bytes += (int64_t)(3 * C.size()) * 4;
    }
    g_ops_cache[key] = d;
    out = d;
    return BBFMM_OK;
}

// ---------------------------------------------------------------------------
static int plan_alloc(bbfmm_plan_impl *P, void **ptr, int64_t bytes, bool zero, cudaStream_t s)
{
    *ptr = nullptr;
    if (bytes <= 0)
        return BBFMM_OK;
    cudaError_t e = cudaMalloc(ptr, (size_t)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BBFMM_ENOMEM, "cudaMalloc(%lld bytes) failed: %s", (long long)bytes, cudaGetErrorString(e));
    }
    P->allocations.push_back(*ptr);
    P->bytes += bytes;
    if (zero) {
        e = cudaMemsetAsync(*ptr, 0, (size_t)bytes, s);
        if (e != cudaSuccess)
            return fail(BBFMM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    return BBFMM_OK;
}

#define PTRY(x)                                                                                                \
    do {                                                                                                       \
        int st_ = (x);                                                                                         \
        if (st_ != BBFMM_OK)                                                                                   \
            return st_;                                                                                        \
    } while (0)

static void plan_free(bbfmm_plan_impl *P)
{
    if (!P)
        return;
    cudaDeviceSynchronize();
    for (void *ptr : P->allocations)
        cudaFree(ptr);
    P->allocations.clear();
    if (P->chunks)
        cudaFree(P->chunks);
    for (auto &g : P->graphs) {
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
        if (g.graph)
            cudaGraphDestroy(g.graph);
    }
    if (P->side_stream)
        cudaStreamDestroy(P->side_stream);
    if (P->far_stream)
        cudaStreamDestroy(P->far_stream);
    if (P->cap_stream)
        cudaStreamDestroy(P->cap_stream);
    if (P->ev_fork)
        cudaEventDestroy(P->ev_fork);
    if (P->ev_join)
        cudaEventDestroy(P->ev_join);
    if (P->ev_far)
        cudaEventDestroy(P->ev_far);
    for (auto &e : P->ev)
        if (e)
            cudaEventDestroy(e);
    if (P->ev_p2p0)
        cudaEventDestroy(P->ev_p2p0);
    if (P->ev_p2p1)
        cudaEventDestroy(P->ev_p2p1);
    cudaGetLastError();
}

// number of (target, source) box pairs over the interaction lists of one
// level of the dense grid: |I(alpha)| = |A_x||A_y||A_z| - |B_x||B_y||B_z| with
// A = children of the parent's neighbours, B = neighbours, per axis
static int64_t m2l_pairs_level(int l)
{
    int64_t n = 1LL << l, np = n / 2, sa = 0, sb = 0;
    for (int64_t a = 0; a < n; ++a) {
        int64_t P = a / 2, lo = std::max<int64_t>(P - 1, 0), hi = std::min<int64_t>(P + 1, np - 1);
        sa += 2 * (hi - lo + 1);
        sb += std::min<int64_t>(a + 1, n - 1) - std::max<int64_t>(a - 1, 0) + 1;
    }
    return sa * sa * sa - sb * sb * sb;
}

// ---------------------------------------------------------------------------
// launch choices (bbfmm_tuning): the near-field order of one-RHS matvecs and
// the tensor-core M2L's tile size and pipeline depth
static Tuning default_tuning(const bbfmm_plan_impl *P, int nrhs = 1)
{
    Tuning t;
    t.near_sym = P->near_sym_default && nrhs == 1;
    t.m2l_nt = P->m2l_nsets > 0 ? P->m2l_set[0].nt : 128;
    t.m2l_stages = 0;
    t.leaf_gemm = P->Mleaf != nullptr;
    return t;
}

static void apply_tuning(bbfmm_plan_impl *P, const Tuning &t)
{
    P->near_sym = t.near_sym && P->near_slots != nullptr;
    P->near_box = t.near_box && !P->near_sym && P->box_items != nullptr;
    P->leaf_gemm = t.leaf_gemm && P->Mleaf != nullptr;
    for (int k = 0; k < P->m2l_nsets; ++k) {
        const bbfmm_plan_impl::TileSet &T = P->m2l_set[k];
        if (T.nt != t.m2l_nt)
            continue;
        P->m2l_nt = T.nt;
        P->m2l_tiles = T.tiles;
        P->m2l_groups = T.groups;
        for (int l = 0; l <= kMaxDepth; ++l) {
            P->m2l_ntiles[l] = T.ntiles[l];
            P->m2l_tile_off[l] = T.off[l];
        }
    }
    P->m2l_stages = t.m2l_stages;
}

static bool tensor_m2l(const bbfmm_plan_impl *P)
{
    return P->precision != BBFMM_PREC_FP32 && P->nodeset == BBFMM_INTERP_CHEBYSHEV && P->ops && P->ops->r <= 256 &&
           P->D >= 2;
}

// is t a choice this plan can run?
static bool tuning_valid(const bbfmm_plan_impl *P, const Tuning &t)
{
    if (t.near_sym && !P->near_slots)
        return false;
    if (t.near_box && (t.near_sym || !P->box_items))
        return false;
    if (t.leaf_gemm && !P->Mleaf)
        return false;
    bool tile = false;
    for (int k = 0; k < P->m2l_nsets; ++k)
        tile = tile || P->m2l_set[k].nt == t.m2l_nt;
    if (!tile)
        return false;
    if (t.m2l_stages != 0 && (t.m2l_stages < 2 || t.m2l_stages > m2l_max_stages(P->precision, t.m2l_nt)))
        return false;
    return true;
}

static int plan_build(bbfmm_plan_impl *P, const double *points, const double *targets, cudaStream_t s)
{
    const int64_t n = P->n, nt = P->nt;
    const int D = P->D;
    const int64_t nleaf = 1LL << (3 * D);
    CUDA_TRY(cudaGetDevice(&P->device));
    struct Tmp {
        std::vector<void *> v;
        ~Tmp()
        {
            for (void *p : v)
                cudaFree(p);
        }
    } tmp;
    auto talloc = [&](void **ptr, int64_t bytes) -> int {
        cudaError_t e = cudaMalloc(ptr, (size_t)std::max<int64_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BBFMM_ENOMEM, "cudaMalloc(%lld bytes) failed", (long long)bytes);
        }
        tmp.v.push_back(*ptr);
        return BBFMM_OK;
    };
    // point sets on the device (FP64)
    auto upload = [&](const double *h, int64_t cnt, double **d) -> int {
        if (is_device_ptr(h)) {
            *d = const_cast<double *>(h);
            return BBFMM_OK;
        }
        PTRY(talloc((void **)d, sizeof(double) * 3 * cnt));
        CUDA_TRY(cudaMemcpyAsync(*d, h, sizeof(double) * 3 * cnt, cudaMemcpyHostToDevice, s));
        return BBFMM_OK;
    };
    double *dpts = nullptr, *dtgt = nullptr;
    PTRY(upload(points, n, &dpts));
    if (P->separate)
        PTRY(upload(targets, nt, &dtgt));

    // domain: the given cube, or the bounding cube of all points
    unsigned long long *mm = nullptr;
    int *bad = nullptr;
    PTRY(talloc((void **)&mm, 6 * 8));
    PTRY(talloc((void **)&bad, 16));
    if (P->side <= 0.0) {
        double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int set = 0; set < (P->separate ? 2 : 1); ++set) {
            CUDA_TRY(launch_domain_minmax(set ? dtgt : dpts, set ? nt : n, reinterpret_cast<double *>(mm), s));
            unsigned long long h[6];
            CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            for (int k = 0; k < 6; ++k) {
                unsigned long long e = h[k];
                unsigned long long b = (e >> 63) ? (e & ~0x8000000000000000ull) : ~e;
                double x;
                memcpy(&x, &b, 8);
                v[k] = k < 3 ? std::min(v[k], x) : std::max(v[k], x);
            }
        }
        double side = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (!isfinite(v[d]) || !isfinite(v[3 + d]))
                return fail(BBFMM_EINVAL, "points contain NaN or infinite coordinates");
            P->lo[d] = v[d];
            side = std::max(side, v[3 + d] - v[d]);
        }
        P->side = side > 0.0 ? side : 1.0;
    }

    // leaf binning and Morton sort of one point set
    const int64_t nmax = std::max(n, nt);
    uint32_t *keys = nullptr, *keys2 = nullptr;
    int *vals = nullptr, *vals2 = nullptr, *scratch = nullptr;
    PTRY(talloc((void **)&keys, 4 * nmax));
    PTRY(talloc((void **)&keys2, 4 * nmax));
    PTRY(talloc((void **)&vals, 4 * nmax));
    PTRY(talloc((void **)&vals2, 4 * nmax));
    int64_t sc = std::max(radix_sort_scratch_ints(nmax), 2 * (nleaf + 1) + scan_scratch_ints(nleaf + 1));
    PTRY(talloc((void **)&scratch, 4 * sc));
    auto build_set = [&](const double *dp, int64_t cnt, float4 **pts, int **perm, int **off) -> int {
        CUDA_TRY(cudaMemsetAsync(bad, 0, 16, s));
        CUDA_TRY(launch_bin_points(dp, cnt, P->lo, P->side, D, keys, vals, bad, s));
        int hbad = 0;
        CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad)
            return fail(BBFMM_EINVAL, "points contain NaN/inf coordinates or lie outside the domain");
        CUDA_TRY(radix_sort_pairs(keys, vals, keys2, vals2, cnt, 3 * D, scratch, sc, s));
        PTRY(plan_alloc(P, (void **)off, 4 * (nleaf + 1), false, s));
        CUDA_TRY(launch_leaf_offsets(keys, cnt, nleaf, *off, s));
        PTRY(plan_alloc(P, (void **)pts, 16 * cnt, false, s));
        PTRY(plan_alloc(P, (void **)perm, 4 * cnt, false, s));
        CUDA_TRY(launch_local_coords(dp, vals, cnt, P->lo, P->side, D, *pts, *perm, s));
        return BBFMM_OK;
    };
    PTRY(build_set(dpts, n, &P->pts, &P->perm, &P->leaf_off));
    if (P->separate) {
        PTRY(build_set(dtgt, nt, &P->tpts, &P->tperm, &P->tleaf_off));
    } else {
        P->tpts = P->pts;
        P->tperm = P->perm;
        P->tleaf_off = P->leaf_off;
    }
    // near-field work items: chunks of the target leaves
    int64_t chunk_bytes = 0;
    CUDA_TRY(build_chunks(P->tleaf_off, nleaf, scratch, &P->chunks, &P->nchunks, &chunk_bytes, s));
    P->bytes += chunk_bytes;

    // statistics of the tree (host copies of the leaf offsets)
    std::vector<uint8_t> leaf_occ; // leaves holding targets
    std::vector<int4> box_items;   // read by an asynchronous copy until the final synchronize
    {
        std::vector<int> off(nleaf + 1), toff;
        CUDA_TRY(cudaMemcpyAsync(off.data(), P->leaf_off, 4 * (nleaf + 1), cudaMemcpyDeviceToHost, s));
        if (P->separate) {
            toff.resize(nleaf + 1);
            CUDA_TRY(cudaMemcpyAsync(toff.data(), P->tleaf_off, 4 * (nleaf + 1), cudaMemcpyDeviceToHost, s));
        }
        CUDA_TRY(cudaStreamSynchronize(s));
        const std::vector<int> &to = P->separate ? toff : off;
        if (off[nleaf] != n || to[nleaf] != nt)
            return fail(BBFMM_EINTERNAL, "leaf offsets do not cover all points");
        leaf_occ.resize(nleaf);
        for (int64_t m = 0; m < nleaf; ++m)
            leaf_occ[m] = to[m + 1] > to[m] ? 1 : 0;
        int side_cells = 1 << D;
        int64_t pairs = 0, sym_evals = 0;
        for (int64_t m = 0; m < nleaf; ++m) {
            const int64_t cs = off[m + 1] - off[m], ct = to[m + 1] - to[m];
            if (cs > 0) {
                P->nonempty_leaves++;
                P->max_leaf = std::max(P->max_leaf, cs);
            }
            if (ct == 0)
                continue;
            int x, y, z;
            demorton3((uint32_t)m, x, y, z);
            int64_t src = 0, fwd = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int a = x + dx, b = y + dy, cc = z + dz;
                        if (a < 0 || b < 0 || cc < 0 || a >= side_cells || b >= side_cells || cc >= side_cells)
                            continue;
                        uint32_t nm = morton3(a, b, cc);
                        src += off[nm + 1] - off[nm];
                        if ((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1) > 13)
                            fwd += off[nm + 1] - off[nm];
                    }
            pairs += ct * src;
            // the symmetric near field's evaluations: own leaf one way, each
            // forward neighbour once (twice when alpha is too full to take it
            // both ways, then both sides take their own rows)
            sym_evals += cs * cs + cs * fwd * (cs <= kSymMaxPoints ? 1 : 2);
        }
        P->p2p_pairs = pairs;
        P->p2p_sym_evals = sym_evals;
        // near-field work items of one level-(D-1) box (its 8 leaves' targets,
        // at most kChunk per item), for small leaves
        if (D >= 1) {
            const int64_t npar = nleaf / 8;
            for (int64_t b = 0; b < npar; ++b)
                for (int a = to[8 * b]; a < to[8 * b + 8]; a += kChunk)
                    box_items.push_back(make_int4((int)b, a, std::min(kChunk, to[8 * b + 8] - a), 0));
        }
        for (int l = 2; l <= D; ++l)
            P->m2l_pairs += m2l_pairs_level(l);
    }

    if (!box_items.empty()) {
        P->nbox_items = (int)box_items.size();
        PTRY(plan_alloc(P, (void **)&P->box_items, sizeof(int4) * box_items.size(), false, s));
        CUDA_TRY(cudaMemcpyAsync(P->box_items, box_items.data(), sizeof(int4) * box_items.size(),
                                 cudaMemcpyHostToDevice, s));
    }

    // operators
    PTRY(get_ops(P->kernel, P->ell, P->p, P->eps, D, P->side, P->device, P->nodeset, P->ops));
    P->interp = make_interp_tables(*P->ops->host);

    // per-level coefficient buffers
    const int R = P->max_nrhs, p3 = P->p3;
    const int rp = P->ops->rp;
    // the tensor-core M2L visits only tiles with occupied targets: one tile
    // list per tile size the precision allows (the first is the default)
    std::vector<int4> tiles[2]; // read by the asynchronous copies below until the final synchronize
    {
        int nts[2];
        P->m2l_nsets = m2l_tile_choices(P->precision, nts);
        for (int k = 0; k < P->m2l_nsets; ++k) {
            bbfmm_plan_impl::TileSet &T = P->m2l_set[k];
            T.nt = nts[k];
            m2l_active_tiles(D, T.nt, leaf_occ, tiles[k], T.ntiles);
            for (int l = D, o = 0; l >= 2; --l) {
                T.off[l] = o;
                o += T.ntiles[l];
            }
            if (!tiles[k].empty()) {
                PTRY(plan_alloc(P, (void **)&T.tiles, sizeof(int4) * tiles[k].size(), false, s));
                CUDA_TRY(cudaMemcpyAsync(T.tiles, tiles[k].data(), sizeof(int4) * tiles[k].size(),
                                         cudaMemcpyHostToDevice, s));
            }
            T.groups = m2l_groups_for(D, R, P->precision, T.nt, P->ops->r, T.ntiles, P->ops->rl);
            P->m2l_groups = std::max(P->m2l_groups, T.groups); // slices allocated below
        }
    }
    for (int l = 2; l <= D; ++l) {
        Level &L = P->lev[l];
        int64_t nb = 1LL << (3 * l), H = 1LL << (l - 1);
        // M of levels below the leaves feeds the M2M chain of the upward pass;
        // leaf M and every F stay in the passes' shared memory unless kept
        if (l < D || P->keep_coeffs)
            PTRY(plan_alloc(P, (void **)&L.M, 4 * nb * R * p3, false, s));
        if (P->keep_coeffs)
            PTRY(plan_alloc(P, (void **)&L.F, 4 * nb * R * p3, false, s));
        if (l <= D - 2)
            PTRY(plan_alloc(P, (void **)&P->up_count[l], 4 * nb * R, true, s));
        PTRY(plan_alloc(P, (void **)&L.Mt, 4 * 8 * (H + 2) * H * H * R * rp, true, s));
        PTRY(plan_alloc(P, (void **)&L.Ft, 4 * nb * R * rp * P->m2l_groups, true, s)); // most slices of any tile size
        if (P->precision == BBFMM_PREC_TF32X3) {
            PTRY(plan_alloc(P, (void **)&L.Mt_hi, 4 * 8 * (H + 2) * H * H * R * rp, true, s));
            PTRY(plan_alloc(P, (void **)&L.Mt_lo, 4 * 8 * (H + 2) * H * H * R * rp, true, s));
        }
        if (P->precision == BBFMM_PREC_FP16X3 || P->precision == BBFMM_PREC_BF16X3) {
            PTRY(plan_alloc(P, (void **)&L.Mt16_hi, 2 * 8 * (H + 2) * H * H * R * rp, true, s));
            PTRY(plan_alloc(P, (void **)&L.Mt16_lo, 2 * 8 * (H + 2) * H * H * R * rp, true, s));
        }
        if (P->nodeset == BBFMM_INTERP_UNIFORM) {
            // spectra: M^ on the grid with a zero halo of 3 boxes, F^ per box
            const int64_t nw = P->ops->nw;
            PTRY(plan_alloc(P, (void **)&L.Mhat, 8 * nw * R * fft_grid_boxes(l), true, s));
            PTRY(plan_alloc(P, (void **)&L.Fhat, 8 * nw * R * nb, false, s));
        }
    }
    std::vector<int4> ft; // read by the asynchronous copy below until the final synchronize
    if (P->nodeset == BBFMM_INTERP_UNIFORM) {
        fft_active_tiles(D, leaf_occ, ft, P->fft_ntiles);
        for (int l = D, o = 0; l >= 2; --l) {
            P->fft_tile_off[l] = o;
            o += P->fft_ntiles[l];
        }
        if (!ft.empty()) {
            PTRY(plan_alloc(P, (void **)&P->fft_tiles, sizeof(int4) * ft.size(), false, s));
            CUDA_TRY(cudaMemcpyAsync(P->fft_tiles, ft.data(), sizeof(int4) * ft.size(), cudaMemcpyHostToDevice, s));
        }
    }
    if (P->precision == BBFMM_PREC_FP16X3 || P->precision == BBFMM_PREC_BF16X3) {
        PTRY(ensure_ops16(*P->ops, P->precision == BBFMM_PREC_FP16X3 ? 0 : 1));
        PTRY(plan_alloc(P, (void **)&P->a16_max, 4 * (kMaxDepth + 1), true, s));
        PTRY(plan_alloc(P, (void **)&P->a16_scale, 4 * (kMaxDepth + 1), true, s));
    }
    PTRY(plan_alloc(P, (void **)&P->sigma_s, 4 * n * R, false, s));
    if (R > 1)
        PTRY(plan_alloc(P, (void **)&P->sigma_rows, 4 * n * R, false, s));
    PTRY(plan_alloc(P, (void **)&P->phi_far, 4 * nt * R, false, s));
    PTRY(plan_alloc(P, (void **)&P->phi_near, 4 * nt * R, false, s));
    if (D >= 4)
        PTRY(plan_alloc(P, (void **)&P->Ftop, 4 * (1LL << (3 * (D - 2))) * R * P->p3, false, s));
    // leaf multipoles for the compression GEMM, zero past p^3 and for empty
    // leaves; the TMA setup is made here, outside any stream capture
    if (P->nodeset == BBFMM_INTERP_CHEBYSHEV && D >= 2 && !P->ops->Vt_hi.empty() &&
        leaf_compress_fits(P->ops->rl[P->ops->nlev == 1 ? 0 : D - 2], P->ops->p3p) && tc_sm_count() > 0)
        PTRY(plan_alloc(P, (void **)&P->Mleaf, 4 * (int64_t)R * (1LL << (3 * D)) * P->ops->p3p, true, s));
    // the leaves' decompressed far fields (the downward GEMM's output)
    if (P->Mleaf && leaf_decompress_fits(P->ops->rp, P->ops->p3p))
        PTRY(plan_alloc(P, (void **)&P->Fdec, 4 * (int64_t)R * (1LL << (3 * D)) * P->ops->p3p, false, s));
    // and for the boxes of level D-1 (the passes then neither compress nor
    // decompress on the CUDA cores below level D-2)
    if (P->Fdec && D >= 3 && leaf_compress_fits(P->ops->rl[P->ops->nlev == 1 ? 0 : D - 3], P->ops->p3p)) {
        PTRY(plan_alloc(P, (void **)&P->Mlev1, 4 * (int64_t)R * (1LL << (3 * (D - 1))) * P->ops->p3p, true, s));
        PTRY(plan_alloc(P, (void **)&P->Fdec1, 4 * (int64_t)R * (1LL << (3 * (D - 1))) * P->ops->p3p, false, s));
    }
    if (P->near_sym && P->near_auto) {
        // occupancy of the leaves the near-field work meets: pairs per point
        // over the 27 neighbours.  Measured at 1M / 2M points: faster at ~30,
        // slower at ~4 (per-item work dominates) and on the clustered set
        // (~170, where the pairs sit in dense leaves).  The autotuner, when
        // on, measures both orders instead
        const double occ = (double)P->p2p_pairs / (27.0 * (double)n);
        P->near_sym = occ >= 16.0 && occ <= 48.0;
    }
    // slots nobody writes stay zero for the plan's lifetime; allocated when
    // the symmetric order is used or may be chosen by the autotuner
    if (P->near_sym || (P->near_sym_ok && P->near_auto && P->autotune))
        PTRY(plan_alloc(P, (void **)&P->near_slots, 4 * (int64_t)kSymSlotsHost * n, true, s));
    P->near_sym_default = P->near_sym;
    apply_tuning(P, default_tuning(P));
    if (P->close_refine && P->nchunks > 0) {
        // near-field pairs closer than 1/64 cell, with FP64 corrections of
        // the FP32 values the near-field kernels add (k_close_pairs): count
        // per target, lay the entries out on the host, fill
        int *cnt = nullptr, *first = nullptr;
        PTRY(talloc((void **)&cnt, 4 * nt));
        CloseArgs C = {};
        C.tpts = P->tpts;
        C.chunks = P->chunks;
        C.nchunks = P->nchunks;
        C.spts = P->pts;
        C.soff = P->leaf_off;
        C.tx = P->separate ? dtgt : dpts;
        C.tperm = P->tperm;
        C.sx = dpts;
        C.sperm = P->perm;
        C.D = D;
        C.same = P->separate ? 0 : 1;
        C.sym = P->near_slots ? 1 : 0; // coefficients for the symmetric order too
        C.count = cnt;
        const double h = P->side / (double)(1LL << D);
        CUDA_TRY(launch_close_pairs(C, P->kernel, P->ell, h, false, s));
        std::vector<int> hc(nt), hfirst(nt), tg, st;
        CUDA_TRY(cudaMemcpyAsync(hc.data(), cnt, 4 * nt, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        int64_t E = 0;
        for (int64_t t = 0; t < nt; ++t) {
            hfirst[t] = (int)std::min<int64_t>(E, INT32_MAX);
            if (hc[t] > 0) {
                tg.push_back((int)t);
                st.push_back((int)std::min<int64_t>(E, INT32_MAX));
                E += hc[t];
            }
        }
        if (E >= INT32_MAX)
            return fail(BBFMM_ENOMEM, "%lld close near-field pairs: too many for the correction list", (long long)E);
        st.push_back((int)E);
        if (E > 0) {
            CloseList &L = P->close;
            L.ntgt = (int)tg.size();
            L.nentries = E;
            PTRY(talloc((void **)&first, 4 * nt));
            PTRY(plan_alloc(P, (void **)&L.tgt, 4 * (int64_t)tg.size(), false, s));
            PTRY(plan_alloc(P, (void **)&L.start, 4 * (int64_t)st.size(), false, s));
            PTRY(plan_alloc(P, (void **)&L.src, 4 * E, false, s));
            PTRY(plan_alloc(P, (void **)&L.c1, 4 * E, false, s));
            PTRY(plan_alloc(P, (void **)&L.c1b, 4 * E, false, s));
            if (C.sym)
                PTRY(plan_alloc(P, (void **)&L.c1s, 4 * E, false, s));
            PTRY(plan_alloc(P, (void **)&L.cm, 4 * E, false, s));
            CUDA_TRY(cudaMemcpyAsync(first, hfirst.data(), 4 * nt, cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(L.tgt, tg.data(), 4 * tg.size(), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(L.start, st.data(), 4 * st.size(), cudaMemcpyHostToDevice, s));
            C.first = first;
            C.e_src = L.src;
            C.e_c1 = L.c1;
            C.e_c1b = L.c1b;
            C.e_c1s = L.c1s;
            C.e_cm = L.cm;
            CUDA_TRY(launch_close_pairs(C, P->kernel, P->ell, h, true, s));
            CUDA_TRY(cudaStreamSynchronize(s)); // the host vectors above are read until here
        }
    }
    PTRY(plan_alloc(P, (void **)&P->status, 16, true, s));

    // constant tables the matvec kernels read, uploaded before any capture
    CUDA_TRY(m2l_fp32_init());
    if (P->nodeset == BBFMM_INTERP_UNIFORM)
        CUDA_TRY(m2l_fft_init());
    CUDA_TRY(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
    int prio_low = 0, prio_high = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    CUDA_TRY(cudaStreamCreateWithPriority(&P->far_stream, cudaStreamNonBlocking, prio_high));
    CUDA_TRY(cudaStreamCreateWithPriority(&P->side_stream, cudaStreamNonBlocking, prio_low));
    CUDA_TRY(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&P->ev_far, cudaEventDisableTiming));
    for (auto &e : P->ev)
        CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventCreate(&P->ev_p2p0));
    CUDA_TRY(cudaEventCreate(&P->ev_p2p1));
    CUDA_TRY(cudaStreamSynchronize(s));
    return BBFMM_OK;
}

// ---------------------------------------------------------------------------
static PassArgs pass_args(const bbfmm_plan_impl *P, int nrhs, bool split16)
{
    const DevOps &O = *P->ops;
    PassArgs A;
    memset(&A, 0, sizeof(A));
    A.T = P->interp;
    A.pts = P->pts;
    A.off = P->leaf_off;
    A.n = P->n;
    A.tpts = P->tpts;
    A.toff = P->tleaf_off;
    A.nt = P->nt;
    A.D = P->D;
    A.nrhs = nrhs;
    A.R = P->max_nrhs;
    A.r = O.r;
    A.rp = O.rp;
    A.p3p = O.p3p;
    A.sig = P->sigma_s;
    A.phi = P->phi_far;
    A.nslices = P->m2l_groups;
    A.maxbits = split16 ? P->a16_max : nullptr;
    A.keep = P->keep_coeffs ? 1 : 0;
    A.Ftop = P->Ftop;
    A.Mleaf = P->leaf_gemm ? P->Mleaf : nullptr;
    A.Fdec = P->leaf_gemm ? P->Fdec : nullptr;
    A.Mlev1 = P->leaf_gemm ? P->Mlev1 : nullptr;
    A.Fdec1 = P->leaf_gemm ? P->Fdec1 : nullptr;
    for (int l = 2; l <= P->D; ++l) {
        const Level &L = P->lev[l];
        A.M[l] = L.M;
        A.Mt[l] = L.Mt;
        A.Mt_hi[l] = L.Mt_hi;
        A.Mt_lo[l] = L.Mt_lo;
        A.Ft[l] = L.Ft;
        A.slice[l] = (1LL << (3 * l)) * P->max_nrhs * O.rp;
        A.F[l] = L.F;
        A.V[l] = O.V[O.nlev == 1 ? 0 : l - 2];
        A.Ut[l] = O.Ut[O.nlev == 1 ? 0 : l - 2];
        A.rl[l] = O.rl[O.nlev == 1 ? 0 : l - 2];
        A.count[l] = P->up_count[l];
    }
    return A;
}

static int matvec_device(bbfmm_plan_impl *P, const float *sigma, float *phi, int nrhs, cudaStream_t s)
{
    const int64_t n = P->n, nt = P->nt;
    const int D = P->D, p = P->p;
    const DevOps &O = *P->ops;
    const bool tm = P->timing;
    if (tm)
        CUDA_TRY(cudaEventRecord(P->ev[Stage::Start], s));
    float *rows = nrhs > 1 ? P->sigma_rows : nullptr;
    float *slots = nrhs == 1 && P->near_sym ? P->near_slots : nullptr;
    CUDA_TRY(launch_gather_sigma(sigma, P->perm, n, nrhs, P->sigma_s, rows, s));
    if (tm)
        CUDA_TRY(cudaEventRecord(P->ev[Stage::Gather], s));

    CUDA_TRY(cudaEventRecord(P->ev_fork, s));
    // near field on the low-priority side stream, started once `after` has
    // fired: the gather, unless stage timing is on (then the far field, so
    // each stage is timed alone).  Its blocks fill whatever the high-priority
    // far field leaves of the SMs, from the upward pass on (measured 0.850 ->
    // 0.817 ms on 1M points at depth 5, against starting after the upward
    // pass; in a graph only with node priorities in force)
    auto near_field = [&](cudaEvent_t after) -> int {
        CUDA_TRY(cudaStreamWaitEvent(P->side_stream, after, 0));
        if (tm)
            CUDA_TRY(cudaEventRecord(P->ev_p2p0, P->side_stream));
        const bool box = nrhs == 1 && !slots && P->near_box;
        const P2PArgs pa = {P->tpts, P->chunks,   P->nchunks, nt, P->pts, P->sigma_s,
                            rows,    P->leaf_off, n,          D,  slots,
                            box ? P->box_items : nullptr, box ? P->nbox_items : 0, P->tleaf_off};
        CUDA_TRY(launch_p2p(pa, P->kernel, P->ell, P->side / (double)(1LL << D), nrhs, P->phi_near,
                            P->side_stream));
        CUDA_TRY(launch_near_fix(P->close, slots ? 1 : box ? 2 : 0, P->sigma_s, n, nt, nrhs, P->phi_near,
                                 P->side_stream));
        if (tm)
            CUDA_TRY(cudaEventRecord(P->ev_p2p1, P->side_stream));
        CUDA_TRY(cudaEventRecord(P->ev_join, P->side_stream));
        return BBFMM_OK;
    };
    if (D < 2 || !tm)
        PTRY(near_field(P->ev_fork));

    if (D >= 2) {
        // far field on the high-priority plan stream
        cudaStream_t fs = P->far_stream;
        CUDA_TRY(cudaStreamWaitEvent(fs, P->ev_fork, 0));
        const bool split16 = P->precision == BBFMM_PREC_FP16X3 || P->precision == BBFMM_PREC_BF16X3;
        const PassArgs A = pass_args(P, nrhs, split16);
        // upward pass: P2M, M2M and compression of every level in one launch
        if (split16)
            CUDA_TRY(cudaMemsetAsync(P->a16_max, 0, 4 * (kMaxDepth + 1), fs));
        CUDA_TRY(launch_upward(A, p, fs));
        // the compression of level l (the leaves, and level D-1) as a
        // tensor-core GEMM over the multipoles the pass stored in M
        auto compress_args = [&](int l, const float *M) {
            const int opl = O.nlev == 1 ? 0 : l - 2;
            LeafCompressArgs L = {};
            L.M = M;
            L.Vt_hi = O.Vt_hi[opl];
            L.Vt_lo = O.Vt_lo[opl];
            L.nb = 1LL << (3 * l);
            L.nrhs = nrhs;
            L.R = P->max_nrhs;
            L.r = O.rl[opl];
            L.rp = O.rp;
            L.p3p = O.p3p;
            L.H = 1 << (l - 1);
            L.out = P->lev[l].Mt;
            L.out_hi = P->lev[l].Mt_hi;
            L.out_lo = P->lev[l].Mt_lo;
            L.maxbits = split16 ? P->a16_max + l : nullptr;
            L.status = P->status;
            return L;
        };
        // both levels in one launch when they share the operator
        if (A.Mleaf && A.Mlev1)
            CUDA_TRY(launch_leaf_compress2(compress_args(D, A.Mleaf), compress_args(D - 1, A.Mlev1), fs));
        else if (A.Mleaf)
            CUDA_TRY(launch_leaf_compress(compress_args(D, A.Mleaf), fs));
        else if (A.Mlev1)
            CUDA_TRY(launch_leaf_compress(compress_args(D - 1, A.Mlev1), fs));
        if (split16) {
            Split16Args S = {};
            S.fmt = P->precision == BBFMM_PREC_FP16X3 ? 0 : 1;
            S.lmin = 2;
            S.lmax = D;
            S.maxbits = P->a16_max;
            S.scale = P->a16_scale;
            for (int l = 2; l <= D; ++l) {
                const int64_t H = 1LL << (l - 1);
                S.x[l] = P->lev[l].Mt;
                S.n[l] = 8 * (H + 2) * H * H * P->max_nrhs * O.rp;
                S.hi[l] = P->lev[l].Mt16_hi;
                S.lo[l] = P->lev[l].Mt16_lo;
            }
            CUDA_TRY(launch_split16_levels(S, fs));
        }
        if (tm)
            CUDA_TRY(cudaEventRecord(P->ev[Stage::Up], fs));
        // far field, all levels
        CUDA_TRY(launch_m2l_all(P, nrhs, fs));
        if (tm)
            CUDA_TRY(cudaEventRecord(P->ev[Stage::M2L], fs));
        // downward pass: decompression, L2L and L2P in one launch (the
        // leaves' decompression before it, as a GEMM, when the plan has it)
        auto decompress_args = [&](int l, float *out) {
            const int opl = O.nlev == 1 ? 0 : l - 2;
            LeafDecompressArgs L = {};
            L.Ft = P->lev[l].Ft;
            L.U_hi = O.U_hi[opl];
            L.U_lo = O.U_lo[opl];
            L.rows = (1LL << (3 * l)) * P->max_nrhs;
            L.slice_rows = L.rows;
            L.slices = P->m2l_groups;
            L.rp = O.rp;
            L.p3p = O.p3p;
            L.out = out;
            L.status = P->status;
            return L;
        };
        if (A.Fdec && A.Fdec1)
            CUDA_TRY(launch_leaf_decompress2(decompress_args(D, P->Fdec), decompress_args(D - 1, P->Fdec1), fs));
        else if (A.Fdec)
            CUDA_TRY(launch_leaf_decompress(decompress_args(D, P->Fdec), fs));
        else if (A.Fdec1)
            CUDA_TRY(launch_leaf_decompress(decompress_args(D - 1, P->Fdec1), fs));
        CUDA_TRY(launch_downward(A, p, fs));
        if (tm) {
            CUDA_TRY(cudaEventRecord(P->ev[Stage::Down], fs));
            CUDA_TRY(cudaEventRecord(P->ev[Stage::L2P], fs));
        }
        CUDA_TRY(cudaEventRecord(P->ev_far, fs));
        // with stage timing on, the near field waits for the far field, so
        // every stage's events bracket that stage alone
        if (tm)
            PTRY(near_field(P->ev_far));
        CUDA_TRY(cudaStreamWaitEvent(s, P->ev_far, 0));
    } else if (tm) {
        for (int k = Stage::Up; k <= Stage::L2P; ++k)
            CUDA_TRY(cudaEventRecord(P->ev[k], s));
    }
    CUDA_TRY(cudaStreamWaitEvent(s, P->ev_join, 0));
    if (tm)
        CUDA_TRY(cudaEventRecord(P->ev[Stage::P2P], s));
    CUDA_TRY(launch_combine(D >= 2 ? P->phi_far : nullptr, P->phi_near, slots, P->tperm, nt, nrhs, phi, s));
    if (tm)
        CUDA_TRY(cudaEventRecord(P->ev[Stage::Combine], s));
    P->last_nrhs = nrhs;
    return BBFMM_OK;
}

// The matvec as one CUDA graph: captured on the plan's capture stream the
// first time a given nrhs is used, then replayed on the caller's stream.  The
// caller's sigma / phi enter only the gather and the combine kernels; their
// graph nodes get the pointers of each call before the launch.
static int matvec_graph(bbfmm_plan_impl *P, const float *sigma, float *phi, int nrhs, cudaStream_t s)
{
    auto &g = P->graphs[nrhs];
    if (!g.exec) {
        cudaStream_t cs = P->cap_stream;
        CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int st = matvec_device(P, sigma, phi, nrhs, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st != BBFMM_OK || e != cudaSuccess) {
            if (graph)
                cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != BBFMM_OK ? st : fail(BBFMM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        size_t nn = 0;
        CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nn));
        for (cudaGraphNode_t node : nodes) {
            cudaGraphNodeType type;
            CUDA_TRY(cudaGraphNodeGetType(node, &type));
            if (type != cudaGraphNodeTypeKernel)
                continue;
            ++g.nkernels;
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess) {
                // kernels of a run-time compiled library (user kernels) do not
                // report their parameters here; they are not gather / combine
                cudaGetLastError();
                continue;
            }
            if (kp.func == gather_kernel() || kp.func == gather4_kernel()) {
                g.gather = node;
                g.gp = kp;
            } else if (kp.func == combine_kernel()) {
                g.combine = node;
                g.cp = kp;
            }
        }
        if (!g.gather || !g.combine) {
            cudaGraphDestroy(graph);
            return fail(BBFMM_EINTERNAL, "captured matvec graph lacks its gather / combine node");
        }
        // the captured kernels keep their streams' priorities (far field
        // high, near field low) when the graph runs
        cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(graph);
            g.exec = nullptr;
            return fail(BBFMM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        }
        g.graph = graph;
    }
    // this call's pointers into the two boundary kernels
    const int64_t n = P->n, nt = P->nt;
    const float *far = P->D >= 2 ? P->phi_far : nullptr;
    float *rows = nrhs > 1 ? P->sigma_rows : nullptr;
    void *gargs[] = {(void *)&sigma, (void *)&P->perm, (void *)&n, (void *)&nrhs, (void *)&P->sigma_s,
                     (void *)&rows};
    const float *slots = nrhs == 1 && P->near_sym ? P->near_slots : nullptr;
    void *cargs[] = {(void *)&far,  (void *)&P->phi_near, (void *)&slots, (void *)&P->tperm,
                     (void *)&nt,   (void *)&nrhs,        (void *)&phi};
    cudaKernelNodeParams gp = g.gp, cp = g.cp;
    gp.kernelParams = gargs;
    gp.extra = nullptr;
    cp.kernelParams = cargs;
    cp.extra = nullptr;
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(g.exec, g.gather, &gp));
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(g.exec, g.combine, &cp));
    CUDA_TRY(cudaGraphLaunch(g.exec, s));
    P->last_nrhs = nrhs;
    return BBFMM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: a measured sweep over the launch choices of one nrhs (Sec. 2.5
// "Multiple right-hand-sides": the work per launch grows with nrhs, and the
// best tile and near-field order with it).  Candidates: both near-field
// orders (one RHS, AUTO mode, symmetric kernel and one point set) x every
// tensor-core M2L tile size of the precision x every pipeline depth that fits.
// Each candidate runs one untimed and kTuneReps timed matvecs (zero weights,
// the plan's own buffers, eager launches); the fastest mean wins.  Results are
// cached per process by what sets the work: kernel, p, rank, depth, nrhs,
// precision, node set, point count, near-field occupancy and tile count (as
// binary logarithms).
static constexpr int kTuneReps = 3;
typedef std::tuple<int, int, int, int, int, int, int, int, int, int, int> TuneKey;
static std::mutex g_tune_mu;
static std::map<TuneKey, Tuning> g_tune_cache;

static TuneKey tune_key(const bbfmm_plan_impl *P, int nrhs)
{
    auto lg = [](double x) { return (int)floor(2.0 * log2(1.0 + x)); };
    const double occ = (double)P->p2p_pairs / (27.0 * (double)P->nt);
    const int leaf_tiles = P->m2l_nsets > 0 ? P->m2l_set[0].ntiles[P->D] : 0;
    return TuneKey(P->kernel, P->p, P->ops ? P->ops->r : 0, P->D, nrhs, P->precision, P->nodeset,
                   lg((double)P->n), lg(occ), lg((double)leaf_tiles),
                   (P->separate ? 1 : 0) | (P->near_slots && P->near_auto ? 2 : 0) | (P->near_sym_default ? 4 : 0));
}

static void drop_graph(bbfmm_plan_impl *P, int nrhs)
{
    auto &g = P->graphs[nrhs];
    if (g.exec)
        cudaGraphExecDestroy(g.exec);
    if (g.graph)
        cudaGraphDestroy(g.graph);
    g = bbfmm_plan_impl::Graph();
}

static int autotune_sweep(bbfmm_plan_impl *P, int nrhs, bool use_cache, cudaStream_t s)
{
    const TuneKey key = tune_key(P, nrhs);
    if (use_cache) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && tuning_valid(P, it->second)) {
            P->tuning[nrhs] = it->second;
            drop_graph(P, nrhs);
            return BBFMM_OK;
        }
    }
    const Tuning base = default_tuning(P, nrhs);
    if (!P->io_sigma) {
        PTRY(plan_alloc(P, (void **)&P->io_sigma, 4 * P->n * P->max_nrhs, false, s));
        PTRY(plan_alloc(P, (void **)&P->io_phi, 4 * P->nt * P->max_nrhs, false, s));
    }
    CUDA_TRY(cudaMemsetAsync(P->io_sigma, 0, 4 * P->n * nrhs, s));
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaEventCreate(&a));
    cudaError_t ce = cudaEventCreate(&b);
    if (ce != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(BBFMM_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(ce));
    }
    const bool tm = P->timing;
    P->timing = false;
    int st = BBFMM_OK;
    float best = INFINITY;
    Tuning chosen = base;
    std::vector<Tuning> seen;
    // one candidate: an untimed matvec, then kTuneReps timed ones
    auto measure = [&](const Tuning &t) {
        for (const Tuning &u : seen)
            if (u.near_sym == t.near_sym && u.near_box == t.near_box && u.m2l_nt == t.m2l_nt &&
                u.m2l_stages == t.m2l_stages && u.leaf_gemm == t.leaf_gemm)
                return;
        seen.push_back(t);
        if (st != BBFMM_OK || !tuning_valid(P, t))
            return;
        apply_tuning(P, t);
        st = matvec_device(P, P->io_sigma, P->io_phi, nrhs, s);
        if (st == BBFMM_OK && cudaEventRecord(a, s) != cudaSuccess)
            st = fail(BBFMM_ECUDA, "cudaEventRecord failed");
        for (int r = 0; r < kTuneReps && st == BBFMM_OK; ++r)
            st = matvec_device(P, P->io_sigma, P->io_phi, nrhs, s);
        if (st == BBFMM_OK && (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess))
            st = fail(BBFMM_ECUDA, "timing a tuning candidate failed");
        if (st != BBFMM_OK)
            return;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            chosen = t;
        }
    };
    // the choices are nearly independent (different stages of the matvec), so
    // they are measured one group at a time, each against the best so far:
    // 1. the tensor-core M2L's tile size and pipeline depth
    if (tensor_m2l(P))
        for (int k = 0; k < P->m2l_nsets; ++k) {
            const int mx = m2l_max_stages(P->precision, P->m2l_set[k].nt);
            for (int sg = 2; sg <= mx; ++sg) {
                Tuning t = base;
                t.m2l_nt = P->m2l_set[k].nt;
                t.m2l_stages = sg == mx ? 0 : sg;
                measure(t);
            }
        }
    else
        measure(base);
    // 2. the near-field form of one-RHS matvecs: ordered by leaf, symmetric
    // (AUTO mode, symmetric kernel, one point set), ordered by box
    if (nrhs == 1) {
        // forms: 0 ordered by leaf, 1 symmetric, 2 ordered by box
        const Tuning m = chosen;
        const bool sym_ok = P->near_slots != nullptr, forced_sym = sym_ok && !P->near_auto;
        for (int nf = 0; nf < 3; ++nf) {
            const bool sym = nf == 1;
            if (sym && !sym_ok)
                continue;
            if (!sym && forced_sym)
                continue; // near_mode SYMMETRIC: the caller's order stands
            Tuning t = m;
            t.near_sym = sym;
            t.near_box = nf == 2;
            measure(t);
        }
    }
    // 3. the leaf compression: tensor-core GEMM or inside the upward pass
    if (P->Mleaf) {
        Tuning t = chosen;
        t.leaf_gemm = !t.leaf_gemm;
        measure(t);
    }
    P->timing = tm;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != BBFMM_OK)
        return st;
    chosen.measured = true;
    P->tuning[nrhs] = chosen;
    drop_graph(P, nrhs);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = chosen;
    return BBFMM_OK;
}

// the launch choices of this nrhs.  Counts of right-hand sides share the
// choice of their power-of-two bucket (nrhs in [b, 2b) uses b's), so a
// stream of uneven batch widths measures at most one sweep per bucket; with
// opts.autotune the bucket is measured on first use (or taken from the cache)
static int tune_bucket(int nrhs)
{
    int b = 1;
    while (2 * b <= nrhs)
        b *= 2;
    return b;
}

static int ensure_tuning(bbfmm_plan_impl *P, int nrhs, cudaStream_t s)
{
    if (!P->tuning.count(nrhs)) {
        const int b = tune_bucket(nrhs);
        if (!P->tuning.count(b)) {
            if (P->autotune)
                PTRY(autotune_sweep(P, b, true, s));
            else
                P->tuning[b] = default_tuning(P, b);
        }
        Tuning t = P->tuning[b];
        t.near_sym = t.near_sym && nrhs == 1;
        P->tuning[nrhs] = t;
    }
    apply_tuning(P, P->tuning[nrhs]);
    return BBFMM_OK;
}

} // namespace bbfmm

using namespace bbfmm;

extern "C" {

void bbfmm_default_opts(bbfmm_opts *o)
{
    if (!o)
        return;
    memset(o, 0, sizeof(*o));
    o->ell = 1.0;
    o->svd_eps = 1e-7;
    o->precision = BBFMM_PREC_FP32;
    o->domain_given = 0;
    o->side = 1.0;
    o->max_nrhs = 1;
    o->split_accumulate = 1;
    o->use_graph = 1;
    o->close_refine = 1;
    o->autotune = 1;
}

const char *bbfmm_last_error(void) { return g_last_error.c_str(); }

int bbfmm_kernel_register(const char *source, int homogeneity, int symmetric, int *kernel_id)
{
    g_last_error.clear();
    if (!source || !kernel_id)
        return fail(BBFMM_EINVAL, "NULL argument");
    *kernel_id = 0;
    if (homogeneity < -8 || homogeneity > 8)
        return fail(BBFMM_EINVAL, "homogeneity %d out of range [-8, 8]", homogeneity);
    std::string err;
    int st = user_kernel_register(source, homogeneity, symmetric, kernel_id, err);
    if (st != BBFMM_OK)
        return fail(st, "%s", err.c_str());
    return BBFMM_OK;
}

static int plan_create(const double *points, int64_t n, const double *targets, int64_t nt, int kernel_id,
                       int cheb_order, int depth, const bbfmm_opts *opts_in, void *stream, bbfmm_plan_t *out)
{
    g_last_error.clear();
    if (!out)
        return fail(BBFMM_EINVAL, "out is NULL");
    *out = nullptr;
    bbfmm_opts opts;
    bbfmm_default_opts(&opts);
    if (opts_in)
        opts = *opts_in;
    if (!points)
        return fail(BBFMM_EINVAL, "points is NULL");
    if (n < 1 || n >= (1LL << 31))
        return fail(BBFMM_EINVAL, "n = %lld out of range [1, 2^31)", (long long)n);
    if (targets && (nt < 1 || nt >= (1LL << 31)))
        return fail(BBFMM_EINVAL, "number of targets %lld out of range [1, 2^31)", (long long)nt);
    if (!(kernel_id == BBFMM_K_INV_R || kernel_id == BBFMM_K_INV_R2 || kernel_id == BBFMM_K_EXP ||
          kernel_id == BBFMM_K_GAUSS || kernel_id == BBFMM_K_TEST_POLY || kernel_id == BBFMM_K_TEST_CONST ||
          (kernel_id >= BBFMM_K_USER_FIRST && user_kernel_known(kernel_id))))
        return fail(BBFMM_EINVAL, "unknown kernel id %d", kernel_id);
    if (cheb_order < 2 || cheb_order > kMaxP)
        return fail(BBFMM_EINVAL, "cheb_order %d out of range [2, %d]", cheb_order, kMaxP);
    if (depth < 0 || depth > kMaxDepth)
        return fail(BBFMM_EINVAL, "depth %d out of range [0, %d]", depth, kMaxDepth);
    if (!(opts.ell > 0.0) || !(opts.svd_eps >= 0.0) || opts.max_nrhs < 1 || opts.max_nrhs > 1024)
        return fail(BBFMM_EINVAL, "invalid options (ell > 0, svd_eps >= 0, 1 <= max_nrhs <= 1024)");
    if (opts.precision < BBFMM_PREC_FP32 || opts.precision > BBFMM_PREC_FP16X3)
        return fail(BBFMM_EINVAL, "unknown precision %d", opts.precision);
    if (opts.interp != BBFMM_INTERP_CHEBYSHEV && opts.interp != BBFMM_INTERP_UNIFORM)
        return fail(BBFMM_EINVAL, "unknown interp %d", opts.interp);
    if (opts.near_mode != BBFMM_NEAR_AUTO && opts.near_mode != BBFMM_NEAR_ORDERED &&
        opts.near_mode != BBFMM_NEAR_SYMMETRIC)
        return fail(BBFMM_EINVAL, "unknown near_mode %d", opts.near_mode);
    if (opts.interp == BBFMM_INTERP_UNIFORM && opts.precision != BBFMM_PREC_FP32)
        return fail(BBFMM_EINVAL, "equally spaced nodes run the Fourier-domain M2L in FP32 (precision must be "
                                  "BBFMM_PREC_FP32)");
    if (opts.domain_given && !(opts.side > 0.0 && isfinite(opts.side) && isfinite(opts.lo[0]) &&
                               isfinite(opts.lo[1]) && isfinite(opts.lo[2])))
        return fail(BBFMM_EINVAL, "invalid domain");
    // memory estimate: coefficient grids + points
    {
        int64_t p3 = (int64_t)cheb_order * cheb_order * cheb_order, grid = 0;
        for (int l = 2; l <= depth; ++l)
            grid += (1LL << (3 * l)) * opts.max_nrhs * (4 * p3 + 8 * p3);
        const int64_t ntg = targets ? nt : 0;
        int64_t need = grid * 4 + n * (16 + 4 + 12LL * opts.max_nrhs) + ntg * (16 + 4 + 8LL * opts.max_nrhs) +
                       (1LL << (3 * depth)) * 8;
        if (opts.interp == BBFMM_INTERP_UNIFORM) {
            const int64_t nf = 2LL * cheb_order - 1, nw = nf * nf * cheb_order;
            for (int l = 2; l <= depth; ++l) {
                const int64_t g = (1LL << l) + 6;
                need += 8 * nw * opts.max_nrhs * (g * g * g + (1LL << (3 * l)));
            }
        }
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return fail(BBFMM_ECUDA, "no usable CUDA device");
        }
        if ((double)need > 0.9 * (double)fr)
            return fail(BBFMM_ENOMEM, "plan needs ~%.1f GB, %.1f GB free", need / 1e9, fr / 1e9);
    }
    auto *P = new (std::nothrow) bbfmm_plan_s();
    if (!P)
        return fail(BBFMM_ENOMEM, "host allocation failed");
    P->n = n;
    P->separate = targets != nullptr;
    P->nt = targets ? nt : n;
    P->D = depth;
    P->p = cheb_order;
    P->p3 = cheb_order * cheb_order * cheb_order;
    P->kernel = kernel_id;
    P->precision = opts.precision;
    P->max_nrhs = opts.max_nrhs;
    P->ell = opts.ell;
    P->eps = opts.svd_eps;
    P->split_acc = opts.split_accumulate != 0;
    P->use_graph = opts.use_graph != 0;
    P->keep_coeffs = opts.keep_coefficients != 0;
    P->nodeset = opts.interp;
    P->close_refine = opts.close_refine != 0;
    // the symmetric near field needs K(x, y) = K(y, x) (for a user kernel, as
    // registered) and one point set
    P->near_sym_ok = !targets && kernel_symmetric(kernel_id);
    P->near_sym = opts.near_mode != BBFMM_NEAR_ORDERED && P->near_sym_ok;
    P->near_auto = opts.near_mode == BBFMM_NEAR_AUTO;
    P->autotune = opts.autotune != 0;
    if (opts.domain_given) {
        for (int d = 0; d < 3; ++d)
            P->lo[d] = opts.lo[d];
        P->side = opts.side;
    } else {
        P->side = -1.0;
    }
    int st = plan_build(P, points, targets, (cudaStream_t)stream);
    if (st != BBFMM_OK) {
        std::string msg = g_last_error;
        plan_free(P);
        delete P;
        g_last_error = msg;
        return st;
    }
    *out = P;
    return BBFMM_OK;
}

int bbfmm_plan(const double *points, int64_t n, int kernel_id, int cheb_order, int depth, const bbfmm_opts *opts,
               void *stream, bbfmm_plan_t *out)
{
    return plan_create(points, n, nullptr, 0, kernel_id, cheb_order, depth, opts, stream, out);
}

int bbfmm_plan_targets(const double *sources, int64_t ns, const double *targets, int64_t nt, int kernel_id,
                       int cheb_order, int depth, const bbfmm_opts *opts, void *stream, bbfmm_plan_t *out)
{
    if (!targets) {
        g_last_error.clear();
        if (out)
            *out = nullptr;
        return fail(BBFMM_EINVAL, "targets is NULL");
    }
    return plan_create(sources, ns, targets, nt, kernel_id, cheb_order, depth, opts, stream, out);
}

int bbfmm_matvec(bbfmm_plan_t plan, const float *sigma, float *phi, int nrhs, void *stream)
{
    g_last_error.clear();
    if (!plan)
        return fail(BBFMM_EINVAL, "plan is NULL");
    if (!sigma || !phi)
        return fail(BBFMM_EINVAL, "sigma / phi is NULL");
    if (nrhs < 1 || nrhs > plan->max_nrhs)
        return fail(BBFMM_EINVAL, "nrhs = %d out of range [1, %d]", nrhs, plan->max_nrhs);
    int expected = 0;
    if (!plan->busy.compare_exchange_strong(expected, 1))
        return fail(BBFMM_EBUSY, "plan is in use by another thread");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dsig = is_device_ptr(sigma), dphi = is_device_ptr(phi);
    const int64_t bytes_in = 4 * plan->n * nrhs, bytes_out = 4 * plan->nt * nrhs;
    // launch choices first: a tuning sweep runs matvecs in the plan's staging
    // buffers, which the host copies below then fill
    int st = ensure_tuning(plan, nrhs, s);
    const float *sg = sigma;
    float *ph = phi;
    if (st == BBFMM_OK && (!dsig || !dphi)) {
        if (!plan->io_sigma) {
            st = plan_alloc(plan, (void **)&plan->io_sigma, 4 * plan->n * plan->max_nrhs, false, s);
            if (st == BBFMM_OK)
                st = plan_alloc(plan, (void **)&plan->io_phi, 4 * plan->nt * plan->max_nrhs, false, s);
        }
        if (st == BBFMM_OK && !dsig) {
            cudaError_t e = cudaMemcpyAsync(plan->io_sigma, sigma, bytes_in, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess)
                st = fail(BBFMM_ECUDA, "copy of sigma: %s", cudaGetErrorString(e));
            sg = plan->io_sigma;
        }
        if (!dphi)
            ph = plan->io_phi;
    }
    if (st == BBFMM_OK)
        st = plan->use_graph && !plan->timing ? matvec_graph(plan, sg, ph, nrhs, s)
                                              : matvec_device(plan, sg, ph, nrhs, s);
    if (st == BBFMM_OK && !dphi) {
        cudaError_t e = cudaMemcpyAsync(phi, plan->io_phi, bytes_out, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            st = fail(BBFMM_ECUDA, "copy of phi: %s", cudaGetErrorString(e));
    }
    plan->busy.store(0);
    return st;
}

// ---------------------------------------------------------------------------
// randomized eigen-decomposition of the kernel matrix (Sec. 4.3)
namespace {
struct DevBuffer {
    void *p = nullptr;
    ~DevBuffer()
    {
        if (p)
            cudaFree(p);
    }
};
} // namespace

// G (m x m, FP64, row-major) = A^T B, partial sums added in split order
static int gram_host(const float *A, const float *B, int64_t n, int m, double *dpartial, int splits,
                     cudaStream_t s, std::vector<double> &G)
{
    CUDA_TRY(launch_gram(A, B, n, m, dpartial, splits, s));
    std::vector<double> h((size_t)splits * m * m);
    CUDA_TRY(cudaMemcpyAsync(h.data(), dpartial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    G.assign((size_t)m * m, 0.0);
    for (int sp = 0; sp < splits; ++sp)
        for (size_t q = 0; q < (size_t)m * m; ++q)
            G[q] += h[(size_t)sp * m * m + q];
    return BBFMM_OK;
}

// Q (n x mq) = an orthonormal basis of the columns of Y (n x m): with
// Y^T Y = W L W^T, Q = Y W_k L_k^(-1/2) over the eigenvalues above 1e-10 of
// the largest (directions below that are lost to FP32 rounding of Y)
static int orthonormalize(const float *Y, int64_t n, int m, float *Q, int &mq, double *dpartial, int splits,
                          float *dT, cudaStream_t s)
{
    std::vector<double> G, w, W;
    PTRY(gram_host(Y, Y, n, m, dpartial, splits, s, G));
    jacobi_eigen(m, G, w, W);
    int k = 0;
    while (k < m && w[k] > 0.0 && w[k] > 1e-10 * w[0])
        ++k;
    if (k == 0)
        return fail(BBFMM_EINVAL, "the block K Omega is zero");
    std::vector<float> T((size_t)m * k); // column-major m x k
    for (int c = 0; c < k; ++c)
        for (int a = 0; a < m; ++a)
            T[a + (size_t)c * m] = (float)(W[(size_t)a * m + c] / sqrt(w[c]));
    CUDA_TRY(cudaMemcpyAsync(dT, T.data(), sizeof(float) * T.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s)); // T is a local vector
    CUDA_TRY(launch_rmul(Y, n, m, dT, k, Q, s));
    mq = k;
    return BBFMM_OK;
}

int bbfmm_rand_eig(bbfmm_plan_t plan, const float *omega, int m, int k, int power, double *evals, float *evecs,
                   void *stream)
{
    g_last_error.clear();
    if (!plan || !omega || !evals)
        return fail(BBFMM_EINVAL, "NULL argument");
    if (m < 1 || m > plan->max_nrhs || k < 1 || k > m || power < 0 || power > 8)
        return fail(BBFMM_EINVAL, "need 1 <= k <= m <= max_nrhs (%d) and 0 <= power <= 8", plan->max_nrhs);
    if (!is_device_ptr(omega) || (evecs && !is_device_ptr(evecs)))
        return fail(BBFMM_EINVAL, "omega and evecs must be device memory");
    if (plan->separate)
        return fail(BBFMM_EINVAL, "the plan's targets are not its sources (the kernel matrix is not square)");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = plan->n;
    const int splits = gram_splits(n);
    DevBuffer b1, b2, bp, bt;
    CUDA_TRY(cudaMalloc(&b1.p, sizeof(float) * n * m));
    CUDA_TRY(cudaMalloc(&b2.p, sizeof(float) * n * m));
    CUDA_TRY(cudaMalloc(&bp.p, sizeof(double) * (size_t)splits * m * m));
    CUDA_TRY(cudaMalloc(&bt.p, sizeof(float) * (size_t)m * m));
    float *Y = (float *)b1.p, *Q = (float *)b2.p, *dT = (float *)bt.p;
    double *dpartial = (double *)bp.p;
    // range finder: Y = K Omega, then `power` rounds of Y = K orth(Y)
    PTRY(bbfmm_matvec(plan, omega, Y, m, stream));
    int mq = m;
    for (int it = 0; it < power; ++it) {
        PTRY(orthonormalize(Y, n, mq, Q, mq, dpartial, splits, dT, s));
        PTRY(bbfmm_matvec(plan, Q, Y, mq, stream));
    }
    // Q = orth(Y), twice: the second pass restores the orthogonality that
    // the first loses to rounding
    PTRY(orthonormalize(Y, n, mq, Q, mq, dpartial, splits, dT, s));
    PTRY(orthonormalize(Q, n, mq, Y, mq, dpartial, splits, dT, s));
    float *basis = Y, *Z = Q;
    // Rayleigh-Ritz: B = Q^T K Q, B = V L V^T; eigenvectors U = Q V
    PTRY(bbfmm_matvec(plan, basis, Z, mq, stream));
    std::vector<double> Bm, w, V;
    PTRY(gram_host(basis, Z, n, mq, dpartial, splits, s, Bm));
    for (int a = 0; a < mq; ++a)
        for (int b = a + 1; b < mq; ++b) {
            const double v = 0.5 * (Bm[(size_t)a * mq + b] + Bm[(size_t)b * mq + a]);
            Bm[(size_t)a * mq + b] = Bm[(size_t)b * mq + a] = v;
        }
    jacobi_eigen(mq, Bm, w, V);
    const int kk = k < mq ? k : mq;
    for (int j = 0; j < k; ++j)
        evals[j] = j < kk ? w[j] : 0.0;
    if (evecs) {
        std::vector<float> T((size_t)mq * kk);
        for (int c = 0; c < kk; ++c)
            for (int a = 0; a < mq; ++a)
                T[a + (size_t)c * mq] = (float)V[(size_t)a * mq + c];
        CUDA_TRY(cudaMemcpyAsync(dT, T.data(), sizeof(float) * T.size(), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s)); // T is a local vector
        CUDA_TRY(launch_rmul(basis, n, mq, dT, kk, evecs, s));
        if (kk < k)
            CUDA_TRY(cudaMemsetAsync(evecs + (size_t)kk * n, 0, sizeof(float) * n * (k - kk), s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    return BBFMM_OK;
}

int bbfmm_destroy(bbfmm_plan_t plan)
{
    if (!plan)
        return BBFMM_OK;
    plan_free(plan);
    delete plan;
    return BBFMM_OK;
}

int bbfmm_plan_info(bbfmm_plan_t plan, bbfmm_info *info)
{
    if (!plan || !info)
        return fail(BBFMM_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = plan->n;
    info->n_targets = plan->nt;
    auto t1 = plan->tuning.find(1);
    const bool sym1 = plan->near_slots && (t1 != plan->tuning.end() ? t1->second.near_sym : plan->near_sym_default);
    info->near_symmetric = sym1 ? 1 : 0;
    info->depth = plan->D;
    info->order = plan->p;
    info->rank = plan->ops ? plan->ops->r : 0;
    info->kernel = plan->kernel;
    info->precision = plan->precision;
    info->max_nrhs = plan->max_nrhs;
    for (int d = 0; d < 3; ++d)
        info->lo[d] = plan->lo[d];
    info->side = plan->side;
    info->device_bytes = plan->bytes + (plan->ops ? plan->ops->bytes : 0);
    info->nonempty_leaves = plan->nonempty_leaves;
    info->max_leaf_points = plan->max_leaf;
    info->p2p_pairs = plan->p2p_pairs;
    info->m2l_pairs = plan->m2l_pairs;
    info->close_pairs = (int)plan->close.nentries;
    info->p2p_evals = sym1 ? plan->p2p_sym_evals : plan->p2p_pairs;
    return BBFMM_OK;
}

int bbfmm_get_coefficients(bbfmm_plan_t plan, int which, int level, int nrhs, float *out)
{
    if (!plan || !out)
        return fail(BBFMM_EINVAL, "NULL argument");
    if (level < 2 || level > plan->D || (which != 0 && which != 1) || nrhs < 1 || nrhs > plan->max_nrhs)
        return fail(BBFMM_EINVAL, "bad which / level / nrhs");
    if (!plan->keep_coeffs)
        return fail(BBFMM_EINVAL, "the plan was built without opts.keep_coefficients");
    const float *src = which == 0 ? plan->lev[level].M : plan->lev[level].F;
    int64_t nb = 1LL << (3 * level), p3 = plan->p3;
    std::vector<float> tmp(nb * nrhs * p3);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(tmp.data(), src, tmp.size() * 4, cudaMemcpyDeviceToHost));
    int64_t ns = 1LL << level;
    for (int64_t m = 0; m < nb; ++m) {
        int x, y, z;
        demorton3((uint32_t)m, x, y, z);
        int64_t lex = x + ns * (y + ns * z);
        memcpy(out + lex * nrhs * p3, tmp.data() + m * nrhs * p3, 4 * nrhs * p3);
    }
    return BBFMM_OK;
}

int bbfmm_get_leaf_cells(bbfmm_plan_t plan, int32_t *out)
{
    if (!plan || !out)
        return fail(BBFMM_EINVAL, "NULL argument");
    int64_t nleaf = 1LL << (3 * plan->D), n = plan->n;
    std::vector<int> off(nleaf + 1), perm(n);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(off.data(), plan->leaf_off, 4 * (nleaf + 1), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(perm.data(), plan->perm, 4 * n, cudaMemcpyDeviceToHost));
    for (int64_t m = 0; m < nleaf; ++m) {
        int x, y, z;
        demorton3((uint32_t)m, x, y, z);
        for (int i = off[m]; i < off[m + 1]; ++i) {
            out[3 * (int64_t)perm[i]] = x;
            out[3 * (int64_t)perm[i] + 1] = y;
            out[3 * (int64_t)perm[i] + 2] = z;
        }
    }
    return BBFMM_OK;
}

int bbfmm_status(bbfmm_plan_t plan, int *word)
{
    if (!plan)
        return fail(BBFMM_EINVAL, "plan is NULL");
    int w = 0;
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(&w, plan->status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(plan->status, 0, sizeof(int)));
    if (word)
        *word = w;
    if (w & kStatusTimeout)
        return fail(BBFMM_ETIMEOUT, "a device-side wait timed out (status word %d)", w);
    if (w & kStatusBounds)
        return fail(BBFMM_EINTERNAL, "a device-side bounds check failed (status word %d)", w);
    return BBFMM_OK;
}

int bbfmm_set_timing(bbfmm_plan_t plan, int on)
{
    if (!plan)
        return fail(BBFMM_EINVAL, "plan is NULL");
    plan->timing = on != 0;
    return BBFMM_OK;
}

static int tuning_args(bbfmm_plan_t plan, int nrhs)
{
    if (!plan)
        return fail(BBFMM_EINVAL, "plan is NULL");
    if (nrhs < 1 || nrhs > plan->max_nrhs)
        return fail(BBFMM_EINVAL, "nrhs = %d out of range [1, %d]", nrhs, plan->max_nrhs);
    return BBFMM_OK;
}

int bbfmm_get_tuning(bbfmm_plan_t plan, int nrhs, bbfmm_tuning *out)
{
    g_last_error.clear();
    PTRY(tuning_args(plan, nrhs));
    if (!out)
        return fail(BBFMM_EINVAL, "out is NULL");
    auto it = plan->tuning.find(nrhs);
    const Tuning t = it != plan->tuning.end() ? it->second : default_tuning(plan, nrhs);
    memset(out, 0, sizeof(*out));
    out->near_mode = t.near_sym && plan->near_slots ? BBFMM_NEAR_SYMMETRIC : BBFMM_NEAR_ORDERED;
    out->m2l_tile = t.m2l_nt;
    out->m2l_stages = t.m2l_stages;
    out->measured = t.measured ? 1 : 0;
    out->near_box = t.near_box && !t.near_sym && plan->box_items && nrhs == 1 ? 1 : 0;
    out->leaf_gemm = t.leaf_gemm && plan->Mleaf ? 1 : 0;
    return BBFMM_OK;
}

int bbfmm_matvec_launches(bbfmm_plan_t plan, int nrhs, int *launches)
{
    g_last_error.clear();
    PTRY(tuning_args(plan, nrhs));
    if (!launches)
        return fail(BBFMM_EINVAL, "launches is NULL");
    const auto &g = plan->graphs[nrhs];
    if (!g.exec)
        return fail(BBFMM_EINVAL, "no matvec graph for nrhs = %d yet", nrhs);
    *launches = g.nkernels;
    return BBFMM_OK;
}

int bbfmm_set_tuning(bbfmm_plan_t plan, int nrhs, const bbfmm_tuning *in)
{
    g_last_error.clear();
    PTRY(tuning_args(plan, nrhs));
    if (!in)
        return fail(BBFMM_EINVAL, "tuning is NULL");
    if (in->near_mode != BBFMM_NEAR_ORDERED && in->near_mode != BBFMM_NEAR_SYMMETRIC)
        return fail(BBFMM_EINVAL, "near_mode must be BBFMM_NEAR_ORDERED or BBFMM_NEAR_SYMMETRIC");
    Tuning t;
    t.near_sym = in->near_mode == BBFMM_NEAR_SYMMETRIC;
    t.m2l_nt = in->m2l_tile;
    t.m2l_stages = in->m2l_stages;
    t.near_box = in->near_box != 0;
    t.leaf_gemm = in->leaf_gemm != 0;
    if ((t.near_sym || t.near_box) && nrhs != 1)
        return fail(BBFMM_EINVAL, "the symmetric and box near-field forms run one right-hand side only");
    if (t.near_sym && nrhs != 1)
        return fail(BBFMM_EINVAL, "the symmetric near field runs one right-hand side only");
    if (!tuning_valid(plan, t))
        return fail(BBFMM_EINVAL,
                    "this plan cannot run near_mode %d, near_box %d, m2l_tile %d, m2l_stages %d, leaf_gemm %d",
                    in->near_mode, in->near_box, in->m2l_tile, in->m2l_stages, in->leaf_gemm);
    int expected = 0;
    if (!plan->busy.compare_exchange_strong(expected, 1))
        return fail(BBFMM_EBUSY, "plan is in use by another thread");
    cudaDeviceSynchronize(); // a captured graph of this nrhs may still run
    plan->tuning[nrhs] = t;
    drop_graph(plan, nrhs);
    plan->busy.store(0);
    return BBFMM_OK;
}

int bbfmm_autotune(bbfmm_plan_t plan, int nrhs, void *stream)
{
    g_last_error.clear();
    PTRY(tuning_args(plan, nrhs));
    int expected = 0;
    if (!plan->busy.compare_exchange_strong(expected, 1))
        return fail(BBFMM_EBUSY, "plan is in use by another thread");
    cudaDeviceSynchronize(); // a captured graph of this nrhs may still run
    int st = autotune_sweep(plan, nrhs, false, (cudaStream_t)stream);
    if (st == BBFMM_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        st = fail(BBFMM_ECUDA, "autotune: stream synchronize failed");
    plan->busy.store(0);
    return st;
}

int bbfmm_stage_times(bbfmm_plan_t plan, float *out)
{
    if (!plan || !out)
        return fail(BBFMM_EINVAL, "NULL argument");
    if (!plan->timing)
        return fail(BBFMM_EINVAL, "timing is off for this plan");
    CUDA_TRY(cudaDeviceSynchronize());
    auto el = [&](cudaEvent_t a, cudaEvent_t b) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.f;
        }
        return ms;
    };
    out[0] = el(plan->ev[Stage::Start], plan->ev[Stage::Gather]);
    out[1] = el(plan->ev[Stage::Gather], plan->ev[Stage::Up]);
    out[2] = el(plan->ev[Stage::Up], plan->ev[Stage::M2L]);
    out[3] = el(plan->ev[Stage::M2L], plan->ev[Stage::Down]);
    out[4] = el(plan->ev[Stage::Down], plan->ev[Stage::L2P]);
    out[5] = el(plan->ev_p2p0, plan->ev_p2p1);
    out[6] = el(plan->ev[Stage::P2P], plan->ev[Stage::Combine]);
    out[7] = el(plan->ev[Stage::Start], plan->ev[Stage::Combine]);
    return BBFMM_OK;
}

} // extern "C"
