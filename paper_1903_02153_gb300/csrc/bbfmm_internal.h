// bbfmm_internal.h -- data layout, plan structure and kernel entry points of
// the GB300 black-box FMM library.  Host code and device code both include it.
//
// Layout of one plan in device memory (N points, depth D, p nodes per axis,
// p3 = p^3 coefficients per box, r = rank of the compressed M2L operators,
// R = number of right-hand sides):
//
//   pts      [N] float4   leaf-local coordinates (x-lo)/h_D - (cell + 1/2),
//                          points sorted by the Morton index of their leaf
//   perm     [N] int      original index of the sorted point
//   leaf_off [8^D + 1]    first sorted point of each leaf (Morton order)
//   chunks   [nchunks]    near-field work items (leaf, first point, count <= 128)
//   M_l, F_l [8^l][R][p3] multipole / local coefficients, boxes in Morton order
//   Mt_l     [8][H+2][H][H][R][rp]  compressed multipoles, H = 2^(l-1):
//                          split by box parity (octant o = x&1 | (y&1)<<1 | (z&1)<<2)
//                          and indexed by the parent cell (X, Y, Z) = (x, y, z) >> 1,
//                          with one zero slab below and above in Z
//   Ft_l     [8][H][H][H][R][rp]    compressed local coefficients (M2L output)
//
// The parity split makes the sources of one M2L offset, for a block of targets
// of one octant, a block of consecutive parent cells of one source octant.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bbfmm.h"
#include "morton.cuh"

namespace bbfmm {

constexpr int kMaxP = 10;
constexpr int kMaxDepth = 8;
constexpr int kNumOffsets = 316;      // 7^3 - 3^3 distinct M2L offsets (Sec. 2.3)
constexpr int kOffsetsPerClass = 189; // 6^3 - 3^3 interaction-list boxes (Def. 2.1)
constexpr int kChunk = 128;           // near-field targets per work item (one block)
constexpr int kSymSlotsHost = 13;     // two-way column sums per point (symmetric near field)

// status word bits written by device-side checks
constexpr int kStatusBounds = 1;
constexpr int kStatusTimeout = 2;

// row offset (in floats) of box (x, y, z), right-hand side c, in the
// parity-split layouts at level l (H = 2^(l-1), padZ = 1 for Mt, 0 for Ft)
__host__ __device__ inline int64_t parity_row(int x, int y, int z, int c, int H, int padZ, int R)
{
    int o = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    int64_t Zs = H + 2 * padZ;
    int64_t cell = (((int64_t)o * Zs + (z >> 1) + padZ) * H + (y >> 1)) * H + (x >> 1);
    return cell * R + c;
}

// ---------------------------------------------------------------------------
// Host FP64 operators (operators.cpp)
struct HostOps {
    int kernel = 0, p = 0, p3 = 0, r = 0, rank_u = 0, rank_v = 0;
    double ell = 1.0, eps = 0.0;
    int hom_degree = 0;         // m of K(a x, a y) = a^m K(x, y); 0 = not homogeneous
    int interp = 0;             // BBFMM_INTERP_*: node set, and SVD (0) or Fourier (1) M2L
    std::vector<double> nodes;  // interpolation nodes s_k on [-1, 1], k = 0..p-1
    std::vector<double> wbary;  // 1 / prod_{m != k} (s_k - s_m)
    std::vector<double> S;      // S[o][i][j] = l_i((s_j + 2o - 1) / 2), o = 0, 1
    // per operator level: (one level if homogeneous, else one per tree level 2..D)
    std::vector<double> h;               // box side of the level the operators were made for
    std::vector<int> rl;                 // rank of each operator level before padding to r
    std::vector<std::vector<double>> U;  // p3 x r row-major
    std::vector<std::vector<double>> V;  // p3 x r row-major
    std::vector<std::vector<double>> C;  // 316 x r x r: C[t] = U^T K^(t) V
    std::vector<std::vector<double>> sv; // singular values of the fat operator matrix
    // equally spaced nodes: n = 2p - 1 point DFTs; per operator level the
    // spectra of the 316 offsets' kernel tables, [w][316] complex (re, im
    // interleaved), w = (wz n + wy) p + wx with wx < p (real input), divided
    // by n^3 (the inverse transform's normalisation)
    int nfft = 0, nw = 0;
    std::vector<std::vector<double>> khat;
};

// offset index 0..315 of t = (tx, ty, tz) in [-3,3]^3 \ [-1,1]^3, or -1
__host__ __device__ inline int offset_index(int tx, int ty, int tz)
{
    if (tx >= -1 && tx <= 1 && ty >= -1 && ty <= 1 && tz >= -1 && tz <= 1)
        return -1;
    int idx = 0;
    for (int c = -3; c <= 3; ++c)
        for (int b = -3; b <= 3; ++b)
            for (int a = -3; a <= 3; ++a) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1 && c >= -1 && c <= 1)
                    continue;
                if (a == tx && b == ty && c == tz)
                    return idx;
                ++idx;
            }
    return -1;
}

std::shared_ptr<HostOps> build_host_ops(int kernel, double ell, int p, double eps, int depth,
                                        double side, int interp, std::string &err);
double kernel_value_host(int kernel, double ell, double d0, double d1, double d2);
int kernel_homogeneity(int kernel); // m of K(a x, a y) = a^m K(x, y), 0 if none
bool kernel_symmetric(int kernel);  // K(x, y) = K(y, x)

// user_kernel.cu: kernels registered through bbfmm_kernel_register
int user_kernel_register(const char *source, int homogeneity, int symmetric, int *id, std::string &err);
bool user_kernel_known(int id);
bool user_kernel_traits(int id, int *homogeneity, int *symmetric);
// K(d) in FP64 on the device for n difference vectors (host arrays n x 3 -> n)
cudaError_t user_kernel_eval(int id, const double *d, int64_t n, double *out);

// interpolation tables passed by value to the transfer kernels
struct InterpTables {
    float nodes[kMaxP];
    float wbary[kMaxP];
    float S[2][kMaxP][kMaxP]; // S[o][i][j] = l_i((s_j + 2o - 1)/2)
};
InterpTables make_interp_tables(const HostOps &h);
// cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (row-major,
// destroyed): eigenvalues w in decreasing order, eigenvectors in the columns
// of Q (row-major n x n); operators.cpp
void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &Q);

// ---------------------------------------------------------------------------
// Device operator set, uploaded once per host operator set
struct DevOps {
    std::shared_ptr<HostOps> host;
    int nlev = 0;            // operator levels
    int r = 0, rp = 0;       // rank (largest over the levels), row pitch (floats) of r-vectors
    std::vector<int> rl;     // rank of each operator level (columns past it are zero)
    int rows64 = 0;          // r rounded up to 64 (FP32 M2L tile rows)
    int p3p = 0;             // p3 rounded up to 16
    std::vector<float *> V;  // [p3][rp]    compress weights
    std::vector<float *> Ut; // [r][p3p]    decompress weights (U transposed)
    std::vector<float *> C;  // [316][rows64][rp]
    std::vector<float *> Chi, Clo; // split copies for the tensor-core M2L (hi/lo)
    std::vector<float *> Vt_hi, Vt_lo; // [rp][p3p] V transposed, TF32 hi / lo (leaf compression GEMM)
    std::vector<float *> U_hi, U_lo;   // [p3p][rp] U, TF32 hi / lo (leaf decompression GEMM)
    // 16-bit split copies, made on first use: [0] = FP16 (scaled by c16_scale),
    // [1] = BF16; same [316][rows64][rp] layout
    std::vector<uint16_t *> C16hi[2], C16lo[2];
    std::vector<float> c16_scale[2];
    int nfft = 0, nw = 0;           // equally spaced nodes: DFT size, frequencies kept
    std::vector<float2 *> khat;     // [w][316] kernel spectra per operator level
    std::mutex mu16;
    int64_t bytes = 0;
    ~DevOps();
};
int ensure_ops16(DevOps &O, int fmt); // capi.cu; fmt 0 = FP16, 1 = BF16

// ---------------------------------------------------------------------------
// Plan
struct Level {
    float *M = nullptr, *Mt = nullptr, *Ft = nullptr, *F = nullptr;
    float2 *Mhat = nullptr, *Fhat = nullptr; // equally spaced nodes: spectra [w][R][boxes]
    float *Mt_hi = nullptr, *Mt_lo = nullptr;        // split TF32 copies of Mt
    uint16_t *Mt16_hi = nullptr, *Mt16_lo = nullptr; // split 16-bit copies of Mt
};

// near-field pairs closer than 1/64 cell with their FP64 corrections, listed
// per target when the plan is made (k_close_pairs), added by k_near_fix
struct CloseList {
    int ntgt = 0;                   // targets with listed pairs
    int64_t nentries = 0;           // listed (target, source) pairs
    int *tgt = nullptr;             // [ntgt] target (tree order)
    int *start = nullptr;           // [ntgt + 1] first entry of each
    int *src = nullptr;             // [nentries] source (tree order)
    float *c1 = nullptr;            // [nentries] coefficient, one RHS, ordered near field
    float *c1s = nullptr;           // [nentries] coefficient, one RHS, symmetric near field (or null)
    float *c1b = nullptr;           // [nentries] coefficient, one RHS, ordered by level-(D-1) box
    float *cm = nullptr;            // [nentries] coefficient, several RHS
};

// the launch choices the autotuner measures (bbfmm_tuning in the header)
struct Tuning {
    bool near_sym = false; // one-RHS near field in symmetric order
    bool near_box = false; // one-RHS ordered near field in work items of one level-(D-1) box
    bool leaf_gemm = false; // leaf compression as a tensor-core GEMM after the upward pass
    int m2l_nt = 128;      // targets per tensor-core M2L tile
    int m2l_stages = 0;    // tensor-core M2L pipeline stages (0 = as many as fit)
    bool measured = false; // chosen by a measured sweep (or its cache)
};

struct Stage { // indices into Plan::ev
    enum { Start = 0, Gather, Up, M2L, Down, L2P, P2P, Combine, NumEv };
};

struct bbfmm_plan_impl {
    int64_t n = 0;         // sources
    int64_t nt = 0;        // targets (= n when the targets are the sources)
    bool separate = false; // targets are a point set of their own
    int D = 0, p = 0, p3 = 0, kernel = 0, precision = 0, max_nrhs = 1;
    double ell = 1.0, lo[3] = {0, 0, 0}, side = 1.0, eps = 1e-7;
    int device = 0;
    bool split_acc = true; // 3-pass tensor-core M2L: separate correction accumulator
    int nodeset = 0;       // BBFMM_INTERP_*: interpolation nodes and M2L form
    int m2l_groups = 1;    // offset groups per M2L tile (partial slices of F~)

    // tree: sources, and the targets (the same arrays unless separate)
    float4 *pts = nullptr;
    int *perm = nullptr;
    int *leaf_off = nullptr;
    float4 *tpts = nullptr;
    int *tperm = nullptr;
    int *tleaf_off = nullptr;
    int4 *chunks = nullptr; // near-field work items over the target leaves
    int nchunks = 0;
    float *Mleaf = nullptr;    // [R][8^D][p3p] leaf multipoles for the compression GEMM (or null)
    float *Fdec = nullptr;     // [8^D R][p3p] decompressed leaf far fields (parity-split rows), or null
    // the same two GEMMs for the boxes of level D-1 (D >= 3): their multipoles
    // [R][8^(D-1)][p3p] and decompressed far fields [8^(D-1) R][p3p], or null
    float *Mlev1 = nullptr;
    float *Fdec1 = nullptr;
    bool leaf_gemm = false;    // leaf compression by the GEMM (tuning)
    int4 *box_items = nullptr; // near-field work items of one level-(D-1) box (D >= 1)
    int nbox_items = 0;
    bool near_box = false;     // one-RHS ordered near field by box items (tuning)
    int64_t nonempty_leaves = 0, max_leaf = 0, p2p_pairs = 0, m2l_pairs = 0;
    int64_t p2p_sym_evals = 0; // kernel evaluations of the symmetric near field (one RHS)

    // operators
    std::shared_ptr<DevOps> ops;
    InterpTables interp;

    // work buffers
    Level lev[kMaxDepth + 1];
    float *sigma_s = nullptr, *phi_far = nullptr, *phi_near = nullptr;
    float *sigma_rows = nullptr;                  // max_nrhs > 1: sigma_s row-major, for the near field
    bool near_sym = false;                        // near field evaluated pairwise both ways (one RHS)
    bool near_auto = false;                       // near_sym chosen (occupancy band, or the autotuner)
    bool near_sym_ok = false;                     // the symmetric form applies (kernel, one point set)
    bool near_sym_default = false;                // near_sym before any tuning (mode, occupancy band)
    float *near_slots = nullptr;                  // symmetric near field: 13 x n column sums (zeroed at plan time)
    bool close_refine = true; // list the near field's close pairs with FP64 corrections
    CloseList close;
    float *Ftop = nullptr;                        // depth >= 4: F of the level-(D-2) boxes (downward pass)
    float *io_sigma = nullptr, *io_phi = nullptr; // staging for host sigma / phi
    int *status = nullptr;                        // device status word
    // 16-bit split M2L: per level max |M~| (float bits) and the power-of-two
    // scale applied before splitting, both written on the device each matvec
    unsigned *a16_max = nullptr;
    float *a16_scale = nullptr;
    // upward pass: arrival counters of the boxes of levels 2..D-2 (x max_nrhs),
    // zero between matvecs
    int *up_count[kMaxDepth + 1] = {};
    // tensor-core M2L: the tiles with occupied targets (device), per level,
    // for the tile size in use (m2l_nt) ...
    int4 *m2l_tiles = nullptr;
    int m2l_ntiles[kMaxDepth + 1] = {}, m2l_tile_off[kMaxDepth + 1] = {};
    int m2l_nt = 128, m2l_stages = 0;
    // ... and for every tile size the precision allows (the tuner's choices)
    struct TileSet {
        int nt = 0, groups = 1;
        int4 *tiles = nullptr;
        int ntiles[kMaxDepth + 1] = {}, off[kMaxDepth + 1] = {};
    };
    TileSet m2l_set[2];
    int m2l_nsets = 0;
    // launch choices per nrhs: set by bbfmm_set_tuning or the autotuner
    bool autotune = false;
    std::map<int, Tuning> tuning;
    bool keep_coeffs = false; // also store leaf M and every level's F
    // Fourier-domain M2L: the 8^3-box tiles holding targets, per level
    int4 *fft_tiles = nullptr;
    int fft_ntiles[kMaxDepth + 1] = {}, fft_tile_off[kMaxDepth + 1] = {};

    std::vector<void *> allocations;
    int64_t bytes = 0;

    // the far field runs on a high-priority stream, the near field on a
    // low-priority one, so near-field blocks fill what the far field leaves
    cudaStream_t far_stream = nullptr, side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr;
    bool timing = false;
    cudaEvent_t ev[Stage::NumEv] = {};
    cudaEvent_t ev_p2p0 = nullptr, ev_p2p1 = nullptr;
    int last_nrhs = 0;
    std::atomic<int> busy{0};

    // captured CUDA graphs of the whole matvec, one per nrhs
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    struct Graph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t gather = nullptr, combine = nullptr;
        cudaKernelNodeParams gp{}, cp{};
        int nkernels = 0; // kernel nodes: the launches of one matvec
    };
    Graph graphs[1025];
};

// ---------------------------------------------------------------------------
// Arguments of the fused upward / downward passes (passes.cu); arrays are
// indexed by level
struct PassArgs {
    InterpTables T;
    const float4 *pts;          // sources: leaf-local coordinates, tree order
    const int *off;             // sources: leaf start offsets, 8^D + 1
    int64_t n;
    const float4 *tpts;         // targets: leaf-local coordinates, tree order
    const int *toff;            // targets: leaf start offsets
    int64_t nt;
    int D, nrhs, R, r, rp, p3p; // R = max_nrhs (row stride of M~ / F~)
    int rl[kMaxDepth + 1];      // rank of each level's operators (<= r; coefficients past it stay 0)
    const float *sig;           // upward: n x nrhs weights in tree order
    float *phi;                 // downward: nt x nrhs far field in target tree order
    float *M[kMaxDepth + 1];    // Morton [box][nrhs][p^3]; leaf level used only with keep
    float *Mt[kMaxDepth + 1], *Mt_hi[kMaxDepth + 1], *Mt_lo[kMaxDepth + 1];
    const float *Ft[kMaxDepth + 1];
    int64_t slice[kMaxDepth + 1]; // floats between the offset-group slices of F~
    int nslices;
    float *F[kMaxDepth + 1];    // written only with keep
    const float *V[kMaxDepth + 1], *Ut[kMaxDepth + 1];
    unsigned *maxbits;          // per level max |M~| (float bits), or null
    int *count[kMaxDepth + 1];  // upward arrival counters, levels 2..D-2
    int keep;
    float *Ftop;                // D >= 4: local coefficients of the level-(D-2) boxes, [box][nrhs][p^3]
    float *Mleaf;               // non-null: store leaf M here ([R][8^D][p3p]) instead of compressing it
    const float *Fdec;          // non-null: the leaves' decompressed far fields, [parity row][p3p]
    float *Mlev1;               // non-null: store level-(D-1) M here ([R][8^(D-1)][p3p]) instead of compressing it
    const float *Fdec1;         // non-null: level D-1's decompressed far fields, [parity row][p3p]
};
cudaError_t launch_upward(const PassArgs &A, int p, cudaStream_t s);
// box_gemm.cu: the leaf compression M~ = V^T M as a tensor-core GEMM (3 x TF32)
struct LeafCompressArgs {
    const float *M;              // [R][nb][p3p] leaf multipoles, zero past p^3
    const float *Vt_hi, *Vt_lo;  // [rp][p3p] V transposed, TF32 split
    int64_t nb;                  // leaf boxes (8^D)
    int nrhs, R, r, rp, p3p, H;  // r = rank of the leaf level; H = 2^(D-1)
    float *out, *out_hi, *out_lo; // M~ of the leaf level (and its TF32 split, or null)
    unsigned *maxbits;           // the level's max |M~| slot, or null
    int *status;
};
bool leaf_compress_fits(int r, int p3p);
cudaError_t launch_leaf_compress(const LeafCompressArgs &L, cudaStream_t s);
// two levels in one launch when they share the operator (else two launches)
cudaError_t launch_leaf_compress2(const LeafCompressArgs &L, const LeafCompressArgs &L2, cudaStream_t s);
// the leaf decompression F = U F~ (summed over F~'s offset-group slices) as
// the same kind of GEMM, into [rows][p3p] for the downward pass
struct LeafDecompressArgs {
    const float *Ft;             // F~ of the leaf level: slices x slice_rows rows of rp floats
    const float *U_hi, *U_lo;    // [p3p][rp] U, TF32 split
    int64_t rows, slice_rows;    // rows of one slice (8 H^3 R), rows between slices
    int slices, rp, p3p;
    float *out;                  // [rows][p3p]
    int *status;
};
bool leaf_decompress_fits(int rp, int p3p);
cudaError_t launch_leaf_decompress(const LeafDecompressArgs &L, cudaStream_t s);
cudaError_t launch_leaf_decompress2(const LeafDecompressArgs &L, const LeafDecompressArgs &L2, cudaStream_t s);
cudaError_t launch_downward(const PassArgs &A, int p, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (each checks its arguments and returns a cudaError_t)
// tree.cu
cudaError_t launch_domain_minmax(const double *pts, int64_t n, double *d_minmax, cudaStream_t s);
cudaError_t launch_bin_points(const double *pts, int64_t n, const double *lo, double side, int D,
                              uint32_t *keys, int *vals, int *bad, cudaStream_t s);
cudaError_t radix_sort_pairs(uint32_t *keys, int *vals, uint32_t *keys_tmp, int *vals_tmp, int64_t n,
                             int key_bits, int *scratch, int64_t scratch_ints, cudaStream_t s);
int64_t radix_sort_scratch_ints(int64_t n);
cudaError_t launch_leaf_offsets(const uint32_t *keys, int64_t n, int64_t nleaf, int *leaf_off,
                                cudaStream_t s);
cudaError_t launch_local_coords(const double *pts, const int *sorted_vals, int64_t n, const double *lo,
                                double side, int D, float4 *local, int *perm, cudaStream_t s);
cudaError_t build_chunks(const int *leaf_off, int64_t nleaf, int *scratch_counts, int4 **chunks_out,
                         int *nchunks_out, int64_t *bytes_out, cudaStream_t s);
cudaError_t exclusive_scan_int(const int *in, int *out, int64_t n, int *block_sums, cudaStream_t s);
int64_t scan_scratch_ints(int64_t n);

// transfers.cu
cudaError_t launch_gather_sigma(const float *sigma, const int *perm, int64_t n, int nrhs, float *out, float *rows,
                                cudaStream_t s);
// split the FP32 M~ of levels lmin..lmax (x[l], n[l] floats) into 16-bit
// hi / lo after scaling by a power of two chosen from maxbits[l] (FP16, fmt 0)
// or 1 (BF16, fmt 1); the scale is written to scale[l]
struct Split16Args {
    const float *x[kMaxDepth + 1];
    int64_t n[kMaxDepth + 1];
    uint16_t *hi[kMaxDepth + 1], *lo[kMaxDepth + 1];
    const unsigned *maxbits;
    float *scale;
    int lmin, lmax, fmt;
};
cudaError_t launch_split16_levels(const Split16Args &A, cudaStream_t s);

// eig.cu: tall-skinny products for the randomized eigen-decomposition
int gram_splits(int64_t n);
// partial[split][a][b] (FP64) = rows of the split of A^T B, A and B column-major n x m
cudaError_t launch_gram(const float *A, const float *B, int64_t n, int m, double *partial, int splits,
                        cudaStream_t s);
// out (n x mo) = Y (n x m) T (m x mo), all column-major; out must not alias Y
cudaError_t launch_rmul(const float *Y, int64_t n, int m, const float *T, int mo, float *out, cudaStream_t s);
cudaError_t launch_combine(const float *phi_far, const float *phi_near, const float *slots, const int *perm, int64_t n,
                           int nrhs, float *phi, cudaStream_t s);
// entry points of the kernels whose pointer arguments (the caller's sigma and
// phi) change from call to call of a captured matvec graph: the gather (either
// form; both take the same parameters) and the combine
const void *gather_kernel();
const void *gather4_kernel();
const void *combine_kernel();
cudaError_t m2l_fp32_init(); // uploads the offset table (outside any stream capture)
// m2l_fp32.cu
// per octant class o: the 189 interaction-list offsets as (operator index,
// source octant, packed parent-cell shift (ux+1) | (uy+1)<<2 | (uz+1)<<4)
bool fill_m2l_table(int4 (*tab)[kOffsetsPerClass]);
cudaError_t launch_m2l_fp32(const float *Mt, const float *C, float *Ft, int l, int r, int rp, int rows64,
                            int nrhs, int R, float scale, cudaStream_t s);
// m2l_fft.cu: the far field with equally spaced nodes (Fourier-domain M2L)
cudaError_t launch_m2l_fft(bbfmm_plan_impl *P, int nrhs, cudaStream_t s);
cudaError_t m2l_fft_init(); // tap tables and kernel attributes (outside any capture)
// target tiles (T^3 boxes, T = min(8, 2^l)) holding targets, levels D..2, as
// {tx, ty, tz, 0}; count[l] per level
void fft_active_tiles(int D, const std::vector<uint8_t> &leaf_occ, std::vector<int4> &tiles, int *count);
int64_t fft_grid_boxes(int l); // boxes of the zero-padded M^ grid of level l
// m2l_tc.cu: every level of the far field in one go (FP32 or tensor cores)
cudaError_t launch_m2l_all(bbfmm_plan_impl *P, int nrhs, cudaStream_t s);
int m2l_groups_for(int D, int nrhs, int precision, int nt, int r, const int *ntiles, const std::vector<int> &rl);
// the tensor-core M2L tiles of nt targets that hold at least one occupied
// target box, level by level from D down to 2, as {tx, ty, tz, octant};
// count[l] per level
void m2l_active_tiles(int D, int nt, const std::vector<uint8_t> &leaf_occ, std::vector<int4> &tiles, int *count);
// tile sizes (targets per tile) the tensor-core M2L runs for a precision,
// the default first; returns how many
int m2l_tile_choices(int precision, int *nt);
// pipeline stages that fit in shared memory for a precision and tile size
int m2l_max_stages(int precision, int nt);
// m2l_tc.cu: a 2D FP32 TMA map (box_inner x box_outer, 128-byte swizzle) and
// the SM count, for the leaf-box GEMMs
cudaError_t tc_encode_2d_f32(CUtensorMap *tm, const void *ptr, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                             uint32_t box_inner, uint32_t box_outer);
int tc_sm_count();
// p2p.cu
// targets: tree-order coordinates and the work items over their leaves;
// sources: tree-order coordinates, weights (ns x nrhs) and leaf offsets
struct P2PArgs {
    const float4 *tpts;
    const int4 *chunks;
    int nchunks;
    int64_t nt;
    const float4 *spts;
    const float *sig;      // ns x nrhs column-major
    const float *sig_rows; // the same row-major (nrhs per source); used with several RHS
    const int *soff;
    int64_t ns;
    int D;
    float *slots; // non-null: symmetric near field (one RHS), 13 x ns two-way column sums
    // non-null (one RHS, ordered): work items of one level-(D-1) box each
    // (k_p2p_box) instead of the leaf chunks; toff = target leaf offsets
    const int4 *boxes;
    int nboxes;
    const int *toff;
};
cudaError_t launch_p2p(const P2PArgs &A, int kernel, double ell, double h, int nrhs, float *phi_near,
                       cudaStream_t s);
cudaError_t launch_p2p_user(const P2PArgs &A, int id, double h, int nrhs, float *phi_near, cudaStream_t s);
// close pairs of the near field (p2p_kernels.cuh, k_close_pairs): the plan
// lists the pairs closer than 1/64 cell with FP64 correction coefficients;
// a matvec adds them after the near-field kernel (k_near_fix)
struct CloseArgs;
cudaError_t launch_close_pairs(const CloseArgs &A, int kernel, double ell, double h, bool fill, cudaStream_t s);
cudaError_t launch_close_pairs_user(const CloseArgs &A, int id, double h, bool fill, cudaStream_t s);
// form of the one-RHS near field that ran (its coefficients): 0 ordered by
// leaf, 1 symmetric, 2 ordered by box
cudaError_t launch_near_fix(const CloseList &L, int form, const float *sig, int64_t ns, int64_t nt, int nrhs,
                            float *phi, cudaStream_t s);

} // namespace bbfmm

struct bbfmm_plan_s : bbfmm::bbfmm_plan_impl {};
