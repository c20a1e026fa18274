// tree.cu -- uniform octree of Sec. 2.1 on the device: domain, leaf binning
// (FMMDistribute, Sec. 3), a stable LSD radix sort of the points by the Morton
// index of their leaf, leaf offsets, leaf-local coordinates and the list of
// near-field work items.
//
// Binning rule: cell = min(floor((x - lo) / h_D), 2^D - 1) per axis, in FP64,
// so a point on the upper face of the domain falls into the last cell.
#include <math.h>

#include "bbfmm_internal.h"

namespace bbfmm {

// ---------------------------------------------------------------------------
// order-preserving encoding of doubles as unsigned 64-bit integers
__host__ __device__ inline unsigned long long enc_double(double x)
{
#ifdef __CUDA_ARCH__
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, 8);
#endif
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_minmax_init(unsigned long long *mm)
{
    int t = threadIdx.x;
    if (t < 3)
        mm[t] = ~0ull;
    else if (t < 6)
        mm[t] = 0ull;
}

__global__ void k_minmax(const double *pts, int64_t n, unsigned long long *mm)
{
    __shared__ unsigned long long smin[3][32], smax[3][32];
    unsigned long long lmin[3] = {~0ull, ~0ull, ~0ull}, lmax[3] = {0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double x = pts[3 * i + d];
            if (!isfinite(x))
                continue;
            unsigned long long e = enc_double(x);
            lmin[d] = e < lmin[d] ? e : lmin[d];
            lmax[d] = e > lmax[d] ? e : lmax[d];
        }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, lmin[d], o);
            unsigned long long b = __shfl_xor_sync(0xffffffffu, lmax[d], o);
            lmin[d] = a < lmin[d] ? a : lmin[d];
            lmax[d] = b > lmax[d] ? b : lmax[d];
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            smin[d][w] = lmin[d];
            smax[d][w] = lmax[d];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        int d = threadIdx.x;
        unsigned long long a = ~0ull, b = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a = smin[d][k] < a ? smin[d][k] : a;
            b = smax[d][k] > b ? smax[d][k] : b;
        }
        atomicMin(&mm[d], a);
        atomicMax(&mm[3 + d], b);
    }
}

cudaError_t launch_domain_minmax(const double *pts, int64_t n, double *d_minmax, cudaStream_t s)
{
    // d_minmax receives 6 encoded values; the caller decodes them
    unsigned long long *mm = reinterpret_cast<unsigned long long *>(d_minmax);
    k_minmax_init<<<1, 32, 0, s>>>(mm);
    int blocks = (int)((n + 255) / 256);
    blocks = blocks > 1216 ? 1216 : (blocks < 1 ? 1 : blocks);
    k_minmax<<<blocks, 256, 0, s>>>(pts, n, mm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__device__ inline int cell_of(double x, double lo, double h, int D)
{
    double u = floor((x - lo) / h);
    double nmax = (double)((1 << D) - 1);
    if (u < 0.0)
        return 0;
    if (u > nmax)
        return (1 << D) - 1;
    return (int)u;
}

__global__ void k_bin(const double *pts, int64_t n, double lo0, double lo1, double lo2, double side, int D,
                      uint32_t *keys, int *vals, int *bad)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double h = side / (double)(1 << D);
    double lo[3] = {lo0, lo1, lo2};
    int c[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
        double x = pts[3 * i + d];
        double rel = x - lo[d];
        if (!isfinite(x) || rel < -1e-12 * side || rel > side * (1.0 + 1e-12))
            ok = false;
        c[d] = ok ? cell_of(x, lo[d], h, D) : 0;
    }
    if (!ok)
        atomicOr(bad, 1);
    keys[i] = morton3((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]);
    vals[i] = (int)i;
}

cudaError_t launch_bin_points(const double *pts, int64_t n, const double *lo, double side, int D,
                              uint32_t *keys, int *vals, int *bad, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    k_bin<<<blocks, 256, 0, s>>>(pts, n, lo[0], lo[1], lo[2], side, D, keys, vals, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan of int32 (reduce-then-scan, recursive on the
// block sums)
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ inline int block_exclusive_scan(int v, int *total)
{
    __shared__ int warp_sums[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o)
                s += y;
        }
        warp_sums[lane] = s; // inclusive
    }
    __syncthreads();
    int before = w > 0 ? warp_sums[w - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_tiles(const int *in, int *out, int64_t n, int *block_sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems], sum = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int ex = block_exclusive_scan(sum, &total);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n)
            out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0 && block_sums)
        block_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int *out, int64_t n, const int *block_offsets)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int add = block_offsets[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n)
            out[base + k] += add;
}

int64_t scan_scratch_ints(int64_t n)
{
    // each level with more than one tile keeps its block sums and their scan
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1)
        return 16;
    return 2 * nb + 16 + scan_scratch_ints(nb);
}

cudaError_t exclusive_scan_int(const int *in, int *out, int64_t n, int *scratch, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int *sums = scratch, *sums_scan = scratch + nb;
    k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = exclusive_scan_int(sums, sums_scan, nb, scratch + 2 * nb + 16, s);
    if (e != cudaSuccess)
        return e;
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, sums_scan);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, value) pairs, 8-bit digits
constexpr int kSortThreads = 256, kSortItems = 8, kSortTile = kSortThreads * kSortItems;

__global__ void k_radix_hist(const uint32_t *keys, int64_t n, int shift, int *counts, int nblocks)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (i < n)
            atomicAdd(&h[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t *keys, const int *vals, int64_t n, int shift,
                                const int *offsets, int nblocks, uint32_t *okeys, int *ovals)
{
    __shared__ int s_run[256];
    __shared__ int s_w[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    s_run[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int k = 0; k < kSortItems; ++k) {
        for (int q = tid; q < (kSortThreads / 32) * 256; q += kSortThreads)
            (&s_w[0][0])[q] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)k * kSortThreads + tid;
        bool valid = i < n;
        uint32_t key = valid ? keys[i] : 0u;
        int d = valid ? (int)((key >> shift) & 0xff) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader)
            s_w[w][d] = __popc(peers);
        __syncthreads();
        {
            int run = s_run[tid];
            for (int q = 0; q < kSortThreads / 32; ++q) {
                int c = s_w[q][tid];
                s_w[q][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = s_w[w][d] + rank;
            okeys[pos] = key;
            ovals[pos] = vals[i];
        }
        __syncthreads();
    }
}

int64_t radix_sort_scratch_ints(int64_t n)
{
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    return 2 * 256 * nb + scan_scratch_ints(256 * nb) + 64;
}

cudaError_t radix_sort_pairs(uint32_t *keys, int *vals, uint32_t *keys_tmp, int *vals_tmp, int64_t n,
                             int key_bits, int *scratch, int64_t scratch_ints, cudaStream_t s)
{
    if (n <= 1 || key_bits <= 0)
        return cudaSuccess;
    int nb = (int)((n + kSortTile - 1) / kSortTile);
    if (scratch_ints < radix_sort_scratch_ints(n))
        return cudaErrorInvalidValue;
    int *counts = scratch, *offsets = scratch + 256 * (int64_t)nb, *scan_tmp = offsets + 256 * (int64_t)nb;
    uint32_t *ka = keys, *kb = keys_tmp;
    int *va = vals, *vb = vals_tmp;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8, ++passes) {
        k_radix_hist<<<nb, kSortThreads, 0, s>>>(ka, n, shift, counts, nb);
        cudaError_t e = exclusive_scan_int(counts, offsets, 256 * (int64_t)nb, scan_tmp, s);
        if (e != cudaSuccess)
            return e;
        k_radix_scatter<<<nb, kSortThreads, 0, s>>>(ka, va, n, shift, offsets, nb, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, n * sizeof(int), cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_leaf_offsets(const uint32_t *keys, int64_t n, int64_t nleaf, int *off)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int64_t k = keys[i];
    int64_t kp = i == 0 ? -1 : (int64_t)keys[i - 1];
    for (int64_t m = kp + 1; m <= k; ++m)
        off[m] = (int)i;
    if (i == n - 1)
        for (int64_t m = k + 1; m <= nleaf; ++m)
            off[m] = (int)n;
}

cudaError_t launch_leaf_offsets(const uint32_t *keys, int64_t n, int64_t nleaf, int *leaf_off, cudaStream_t s)
{
    k_leaf_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, nleaf, leaf_off);
    return cudaGetLastError();
}

__global__ void k_local(const double *pts, const int *vals, int64_t n, double lo0, double lo1, double lo2,
                        double side, int D, float4 *local, int *perm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = vals[i];
    double h = side / (double)(1 << D);
    double lo[3] = {lo0, lo1, lo2};
    float u[3];
    for (int d = 0; d < 3; ++d) {
        double x = pts[3 * (int64_t)j + d];
        int c = cell_of(x, lo[d], h, D);
        u[d] = (float)((x - lo[d]) / h - ((double)c + 0.5));
    }
    local[i] = make_float4(u[0], u[1], u[2], 0.0f);
    perm[i] = j;
}

cudaError_t launch_local_coords(const double *pts, const int *sorted_vals, int64_t n, const double *lo,
                                double side, int D, float4 *local, int *perm, cudaStream_t s)
{
    k_local<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, sorted_vals, n, lo[0], lo[1], lo[2], side, D,
                                                        local, perm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// near-field work items: every leaf with c points gets ceil(c/32) chunks of at
// most 32 consecutive targets: (leaf Morton index, first point, count, 0)
__global__ void k_chunk_counts(const int *off, int64_t nleaf, int *cnt)
{
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= nleaf)
        return;
    int c = off[m + 1] - off[m];
    cnt[m] = (c + kChunk - 1) / kChunk;
}

__global__ void k_chunk_fill(const int *off, const int *cstart, int64_t nleaf, int4 *chunks)
{
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= nleaf)
        return;
    int c = off[m + 1] - off[m];
    int s = cstart[m];
    for (int q = 0; q * kChunk < c; ++q) {
        int cnt = c - q * kChunk < kChunk ? c - q * kChunk : kChunk;
        chunks[s + q] = make_int4((int)m, off[m] + q * kChunk, cnt, 0);
    }
}

cudaError_t build_chunks(const int *leaf_off, int64_t nleaf, int *scratch, int4 **chunks_out, int *nchunks_out,
                         int64_t *bytes_out, cudaStream_t s)
{
    // scratch: 2 * (nleaf + 1) + scan_scratch_ints(nleaf + 1) ints
    int *cnt = scratch, *cstart = scratch + (nleaf + 1);
    int *scan_tmp = cstart + (nleaf + 1);
    unsigned blocks = (unsigned)((nleaf + 255) / 256);
    k_chunk_counts<<<blocks, 256, 0, s>>>(leaf_off, nleaf, cnt);
    cudaMemsetAsync(cnt + nleaf, 0, sizeof(int), s);
    cudaError_t e = exclusive_scan_int(cnt, cstart, nleaf + 1, scan_tmp, s);
    if (e != cudaSuccess)
        return e;
    int total = 0;
    e = cudaMemcpyAsync(&total, cstart + nleaf, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return e;
    int4 *ch = nullptr;
    if (total > 0) {
        e = cudaMalloc(&ch, sizeof(int4) * (size_t)total);
        if (e != cudaSuccess)
            return e;
        k_chunk_fill<<<blocks, 256, 0, s>>>(leaf_off, cstart, nleaf, ch);
    }
    *chunks_out = ch;
    *nchunks_out = total;
    *bytes_out = sizeof(int4) * (int64_t)total;
    return cudaGetLastError();
}

} // namespace bbfmm
