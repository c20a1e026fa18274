// user_kernel.cu -- kernel functions supplied by the caller (the black-box
// promise of Sec. 1 and the kernel interface of Sec. 3: the method needs only
// evaluations of K).  The caller gives CUDA C source that defines
//     __device__ double bbfmm_kernel_f64(double d0, double d1, double d2);
//     __device__ float  bbfmm_kernel_f32(float d0, float d1, float d2);
// the kernel as a function of d = x - y in physical units (the operators of a
// level are shared by all box pairs with the same offset, so K must depend
// on x - y only).  NVRTC compiles it once, for sm_103a, together with the
// near-field kernels of p2p_kernels.cuh (their text is embedded at build
// time) and an evaluation kernel: the FP64 function fills the operator tables
// (on the device, batched), the FP32 one runs in the near field.
#include <dlfcn.h>
#include <nvrtc.h>

#include <map>

#include "bbfmm_internal.h"
#include "nvrtc_headers.inc" // kNvrtcHeaders: {name, text} of morton.cuh and p2p_kernels.cuh
#include "p2p_kernels.cuh"

namespace bbfmm {

static_assert(kGemmT == 32, "the run-time instantiation below names k_p2p_gemm<KUser, 32>");

namespace {

// NVRTC, opened on first use (the library does not link it)
struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcAddNameExpression) add_name = nullptr;
    decltype(&nvrtcGetLoweredName) lowered = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) error_string = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr)
                break;
        if (!h)
            return;
        auto sym = [&](auto &fn, const char *name) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
            return fn != nullptr;
        };
        n.ok = sym(n.create, "nvrtcCreateProgram") && sym(n.compile, "nvrtcCompileProgram") &&
               sym(n.log_size, "nvrtcGetProgramLogSize") && sym(n.log, "nvrtcGetProgramLog") &&
               sym(n.cubin_size, "nvrtcGetCUBINSize") && sym(n.cubin, "nvrtcGetCUBIN") &&
               sym(n.add_name, "nvrtcAddNameExpression") && sym(n.lowered, "nvrtcGetLoweredName") &&
               sym(n.destroy, "nvrtcDestroyProgram") && sym(n.error_string, "nvrtcGetErrorString");
    });
    return n;
}

struct UserKernel {
    int homogeneity = 0, symmetric = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t eval = nullptr, p2p = nullptr, p2p_multi = nullptr, p2p_sym = nullptr;
    cudaKernel_t close_count = nullptr, close_fill = nullptr; // k_close_pairs, both passes
    cudaKernel_t p2p_box = nullptr;
};

std::mutex g_mu;
std::map<int, UserKernel> g_kernels;
int g_next = BBFMM_K_USER_FIRST;

// glue compiled after the caller's source: the near-field functor and the
// evaluation kernel
const char *kGlue = R"(
namespace bbfmm {
struct KUser { // d in cell units; h = leaf box side
    float h;
    __device__ float one(float, float dx, float dy, float dz) const { return bbfmm_kernel_f32(h * dx, h * dy, h * dz); }
    __device__ float far(float, float dx, float dy, float dz) const { return bbfmm_kernel_f32(h * dx, h * dy, h * dz); }
};
struct KUserExact { // d in the caller's units
    __device__ double operator()(double d0, double d1, double d2) const { return bbfmm_kernel_f64(d0, d1, d2); }
};
} // namespace bbfmm
extern "C" __global__ void bbfmm_user_eval(const double *d, long long n, double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = bbfmm_kernel_f64(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
}
)";

} // namespace

int user_kernel_register(const char *source, int homogeneity, int symmetric, int *id, std::string &err)
{
    const Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        err = "NVRTC (libnvrtc.so.13) could not be loaded";
        return BBFMM_ECUDA;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        err = "no usable CUDA device";
        return BBFMM_ECUDA;
    }
    if (major * 10 + minor != 103) {
        err = "user kernels are compiled for sm_103a only";
        return BBFMM_ECUDA;
    }
    std::string src = "#include \"p2p_kernels.cuh\"\n";
    src += source;
    src += "\n";
    src += kGlue;
    const char *hdr_text[2] = {kNvrtcHeaders[0].text, kNvrtcHeaders[1].text};
    const char *hdr_name[2] = {kNvrtcHeaders[0].name, kNvrtcHeaders[1].name};
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, src.c_str(), "bbfmm_user_kernel.cu", 2, hdr_text, hdr_name) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        return BBFMM_ECUDA;
    }
    const char *p2p_name = "bbfmm::k_p2p<bbfmm::KUser>", *multi_name = "bbfmm::k_p2p_gemm<bbfmm::KUser, 32>",
               *sym_name = "bbfmm::k_p2p_sym<bbfmm::KUser>";
    const char *count_name = "bbfmm::k_close_pairs<bbfmm::KUser, bbfmm::KUserExact, false>",
               *fill_name = "bbfmm::k_close_pairs<bbfmm::KUser, bbfmm::KUserExact, true>";
    nv.add_name(prog, p2p_name);
    nv.add_name(prog, multi_name);
    nv.add_name(prog, sym_name);
    nv.add_name(prog, count_name);
    nv.add_name(prog, fill_name);
    const char *box_name = "bbfmm::k_p2p_box<bbfmm::KUser>";
    nv.add_name(prog, box_name);
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
    const nvrtcResult rc = nv.compile(prog, 3, opts);
    size_t log_size = 0;
    nv.log_size(prog, &log_size);
    std::string log(log_size, '\0');
    if (log_size)
        nv.log(prog, &log[0]);
    if (rc != NVRTC_SUCCESS) {
        err = std::string("the kernel source does not compile: ") + nv.error_string(rc) + "\n" + log;
        nv.destroy(&prog);
        return BBFMM_EINVAL;
    }
    size_t cubin_size = 0;
    nv.cubin_size(prog, &cubin_size);
    std::vector<char> cubin(cubin_size);
    nv.cubin(prog, cubin.data());
    const char *p2p_low = nullptr, *multi_low = nullptr, *sym_low = nullptr, *count_low = nullptr,
               *fill_low = nullptr;
    nv.lowered(prog, p2p_name, &p2p_low);
    nv.lowered(prog, multi_name, &multi_low);
    nv.lowered(prog, sym_name, &sym_low);
    nv.lowered(prog, count_name, &count_low);
    nv.lowered(prog, fill_name, &fill_low);
    const char *box_low = nullptr;
    nv.lowered(prog, box_name, &box_low);
    const std::string box_sym = box_low ? box_low : "";
    const std::string p2p_sym = p2p_low ? p2p_low : "", multi_sym = multi_low ? multi_low : "",
                      pair_sym = sym_low ? sym_low : "", count_sym = count_low ? count_low : "",
                      fill_sym = fill_low ? fill_low : "";
    nv.destroy(&prog);
    UserKernel k;
    k.homogeneity = homogeneity;
    k.symmetric = symmetric ? 1 : 0;
    cudaError_t e = cudaLibraryLoadData(&k.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.eval, k.lib, "bbfmm_user_eval");
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.p2p, k.lib, p2p_sym.c_str());
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.p2p_multi, k.lib, multi_sym.c_str());
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.p2p_sym, k.lib, pair_sym.c_str());
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.close_count, k.lib, count_sym.c_str());
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.close_fill, k.lib, fill_sym.c_str());
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&k.p2p_box, k.lib, box_sym.c_str());

    if (e != cudaSuccess) {
        cudaGetLastError();
        if (k.lib)
            cudaLibraryUnload(k.lib);
        err = std::string("loading the compiled kernel: ") + cudaGetErrorString(e);
        return BBFMM_ECUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    *id = g_next++;
    g_kernels[*id] = k;
    return BBFMM_OK;
}

bool user_kernel_known(int id)
{
    std::lock_guard<std::mutex> g(g_mu);
    return g_kernels.count(id) != 0;
}

bool user_kernel_traits(int id, int *homogeneity, int *symmetric)
{
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_kernels.find(id);
    if (it == g_kernels.end())
        return false;
    *homogeneity = it->second.homogeneity;
    *symmetric = it->second.symmetric;
    return true;
}

static bool user_kernel_get(int id, UserKernel &out)
{
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_kernels.find(id);
    if (it == g_kernels.end())
        return false;
    out = it->second;
    return true;
}

cudaError_t user_kernel_eval(int id, const double *d, int64_t n, double *out)
{
    UserKernel k;
    if (!user_kernel_get(id, k))
        return cudaErrorInvalidValue;
    if (n <= 0)
        return cudaSuccess;
    double *dd = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dd, sizeof(double) * 3 * n);
    if (e == cudaSuccess)
        e = cudaMalloc(&dout, sizeof(double) * n);
    if (e == cudaSuccess)
        e = cudaMemcpy(dd, d, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        long long nn = n;
        void *args[] = {(void *)&dd, (void *)&nn, (void *)&dout};
        e = cudaLaunchKernel((const void *)k.eval, dim3((unsigned)((n + 255) / 256)), dim3(256), args, 0, nullptr);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (dd)
        cudaFree(dd);
    if (dout)
        cudaFree(dout);
    return e;
}

cudaError_t launch_p2p_user(const P2PArgs &A, int id, double h, int nrhs, float *phi, cudaStream_t s)
{
    UserKernel k;
    if (!user_kernel_get(id, k))
        return cudaErrorInvalidValue;
    if (A.nchunks <= 0)
        return cudaSuccess;
    struct {
        float h;
    } kern = {(float)h};
    float scale = 1.0f;
    long long nt = A.nt, ns = A.ns;
    int D = A.D, nr = nrhs;
    if (nrhs == 1 && A.slots) { // symmetric near field (the kernel was registered as symmetric)
        void *sargs[] = {(void *)&A.spts, (void *)&A.chunks, (void *)&ns, (void *)&A.sig, (void *)&A.soff,
                         (void *)&D,      (void *)&kern,     (void *)&scale, (void *)&phi, (void *)&A.slots};
        return cudaLaunchKernel((const void *)k.p2p_sym, dim3((unsigned)A.nchunks), dim3(kP2PThreads), sargs, 0,
                                s);
    }
    if (nrhs == 1 && A.boxes) { // ordered, work items of one level-(D-1) box
        if (A.nboxes <= 0)
            return cudaSuccess;
        void *bargs[] = {(void *)&A.tpts, (void *)&A.toff, (void *)&A.boxes, (void *)&nt,   (void *)&A.spts,
                         (void *)&A.sig,  (void *)&A.soff, (void *)&D,       (void *)&kern, (void *)&scale,
                         (void *)&phi};
        return cudaLaunchKernel((const void *)k.p2p_box, dim3((unsigned)A.nboxes), dim3(kP2PThreads), bargs, 0, s);
    }
    void *args[] = {(void *)&A.tpts, (void *)&A.chunks,  (void *)&nt,    (void *)&A.spts,
                    (void *)(nrhs > 1 ? &A.sig_rows : &A.sig), (void *)&A.soff,
                    (void *)&ns,     (void *)&D,        (void *)&kern,  (void *)&scale,
                    (void *)&nr,     (void *)&phi};
    if (nrhs == 1)
        return cudaLaunchKernel((const void *)k.p2p, dim3((unsigned)A.nchunks), dim3(kP2PThreads), args, 0, s);
    return cudaLaunchKernel((const void *)k.p2p_multi, dim3((unsigned)A.nchunks), dim3(gemm_threads(kGemmT)), args, 0,
                            s);
}

cudaError_t launch_close_pairs_user(const CloseArgs &A, int id, double h, bool fill, cudaStream_t s)
{
    UserKernel k;
    if (!user_kernel_get(id, k))
        return cudaErrorInvalidValue;
    CloseArgs B = A;
    B.scale = 1.0f; // KUser returns K in the caller's units
    struct {
        float h;
    } kern = {(float)h};
    struct {
    } exact;
    void *args[] = {(void *)&B, (void *)&kern, (void *)&exact};
    return cudaLaunchKernel((const void *)(fill ? k.close_fill : k.close_count), dim3((unsigned)A.nchunks),
                            dim3(kP2PThreads), args, 0, s);
}

} // namespace bbfmm
