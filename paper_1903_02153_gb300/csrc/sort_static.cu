// sort_static.cu -- bbfmm_sort_points_static: the tree build of bbfmm_plan
// (leaf binning, stable Morton sort, leaf offsets) into caller buffers,
// without allocating anything.
//
// Who needs it: callers that must not call cudaMalloc at the time they build
// a tree -- for example code running under a device-memory budget owned by
// another runtime (a serving engine or framework that reserved the GPU's
// memory up front), or code on a path where a synchronous allocation would
// stall other work on the device.  They pass the points and the two outputs;
// the temporary buffers of the sort (key / value ping-pong arrays, digit
// histograms, scan block sums, an error flag) live in one file-scope device
// array of fixed size instead of being allocated per call.
//
// The array, g_sort_scratch, holds kStaticSortMaxPoints points' worth of
// scratch (about 13.6 MB) and stays resident on every GPU that loads this
// library until the process exits.  Its device address is looked up once per
// device, with that device current, on the first call made on that device,
// and kept (a cudaDeviceReset would invalidate it: calls after a reset of the
// device are not supported).  Pointers must be memory of the current device
// (or managed): the kernels read and write them from that device.
#include <mutex>

#include "bbfmm_internal.h"

namespace bbfmm {

constexpr int64_t kStaticSortMaxPoints = 1 << 20;
constexpr int64_t kStaticSortTile = 2048; // items per block of the radix sort
constexpr int64_t kStaticRadixInts = 2 * 256 * (kStaticSortMaxPoints / kStaticSortTile) + 4096;
constexpr int64_t kStaticSortBytes = 3 * 4 * kStaticSortMaxPoints + 4 * kStaticRadixInts + 256;

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticSortBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[64] = {};

// device address of g_sort_scratch on the current device (looked up once)
static cudaError_t static_scratch(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess)
            return e;
        g_static_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_ptr[dev]);
    return cudaSuccess;
}

} // namespace bbfmm

using namespace bbfmm;

extern "C" int bbfmm_sort_points_static(const double *points, int64_t n, int depth, const double *lo, double side,
                                        int32_t *perm, int32_t *leaf_off, void *stream)
{
    if (!points || !lo || !perm || !leaf_off)
        return BBFMM_EINVAL;
    if (n < 1 || n > kStaticSortMaxPoints || depth < 0 || depth > kMaxDepth || !(side > 0.0))
        return BBFMM_EINVAL;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess)
        return BBFMM_ECUDA;
    for (const void *p : {(const void *)points, (const void *)perm, (const void *)leaf_off}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return BBFMM_EINVAL;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return BBFMM_EINVAL; // no host staging: that would need an allocation
        if (a.type == cudaMemoryTypeDevice && a.device != cur)
            return BBFMM_EINVAL; // another GPU's memory: the kernels run on the current device
    }
    if (radix_sort_scratch_ints(n) > kStaticRadixInts)
        return BBFMM_EINTERNAL;
    unsigned char *base = nullptr;
    if (static_scratch(&base) != cudaSuccess)
        return BBFMM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *keys = reinterpret_cast<uint32_t *>(base);
    uint32_t *keys2 = keys + kStaticSortMaxPoints;
    int *vals2 = reinterpret_cast<int *>(keys2 + kStaticSortMaxPoints);
    int *radix = vals2 + kStaticSortMaxPoints;
    int *bad = radix + kStaticRadixInts;
    // the array keeps the previous call's contents: clear the error flag
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess)
        return BBFMM_ECUDA;
    const int64_t nleaf = 1LL << (3 * depth);
    if (launch_bin_points(points, n, lo, side, depth, keys, perm, bad, s) != cudaSuccess)
        return BBFMM_ECUDA;
    if (radix_sort_pairs(keys, perm, keys2, vals2, n, 3 * depth, radix, kStaticRadixInts, s) != cudaSuccess)
        return BBFMM_ECUDA;
    if (launch_leaf_offsets(keys, n, nleaf, leaf_off, s) != cudaSuccess)
        return BBFMM_ECUDA;
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return BBFMM_ECUDA;
    return hbad ? BBFMM_EINVAL : BBFMM_OK;
}
