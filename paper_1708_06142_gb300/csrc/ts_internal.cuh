// Internal declarations of the GB300 tree solver (not part of the C ABI).
//
// Device data layout (one context = one mesh):
//   internal nodes  nid in [0, nint): amr blocks first (breadth-first, so the 8 children of a
//                   block are contiguous), then 72 block-tree nodes per leaf-block n at
//                   nb + 72 n: 8 level-1 nodes, then 8 x 8 level-2 nodes (children contiguous).
//   cells           Morton order inside each leaf-block: cell id = 512 n + 64 q + 8 o + o2
//                   (q: level-1 octant, o: level-2 octant, o2: cell octant), so the 8 cells of a
//                   level-2 node are contiguous too.
//   records         ncom[nid] = (centre of mass xyz, M), ncen[nid] = (geometric centre xyz,
//                   child word); cell[id] = (cell centre xyz, m).  FP32 and FP64 copies.
//   child word      bits 0..25 first child id, bit 26 set if the children are cells,
//                   bits 27..31 tree depth of the children (root depth 0).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "treesolver.h"

#define TS_NB 8
#define TS_NCB 512
#define TS_MAX_DEPTH 31
#define TS_CW_INDEX_MASK 0x03ffffffu
#define TS_CW_CELLS (1u << 26)
#define TS_CW_DEPTH_SHIFT 27
#define TS_MAX_CELLS (1ll << 26)
#define TS_WALK_STACK 128          // per-warp stack entries of the walk kernels
#define TS_WALK_WARPS 4            // warps per CTA of the walk kernels

// device status word bits
#define TS_DEV_STACK_OVERFLOW 1
#define TS_DEV_NONFINITE 2

struct __align__(32) dbl4 {
    double x, y, z, w;
};

enum { TS_EW_NONE = 0, TS_EW_3P = 1, TS_EW_2P1I = 2, TS_EW_1P2I = 3 };

// Everything a walk kernel reads besides the node arrays.
struct WalkGeom {
    float half32[TS_MAX_DEPTH + 1][3];   // half edge per axis at each tree depth
    float hmax2_32[TS_MAX_DEPTH + 1];    // (longest edge)^2 at each depth
    double half64[TS_MAX_DEPTH + 1][3];
    double hmax2_64[TS_MAX_DEPTH + 1];
    int pbc[3];                          // 1 on periodic axes
    double L[3], invL[3];                // domain edge and its inverse
};

struct EwaldDev {
    int kind;                  // TS_EW_*
    int n;                     // table points per axis
    double ext[3], inv_dx[3];  // folded extent and (n-1)/ext
    double far;                // separation beyond which the far-field form is used
    double far_slope;          // 2P1I: 2 pi / (b Lx^2)
    double far_const;          // 2P1I: 2 sqrt(pi zeta)/(pi b Lx);  1P2I: -(gamma_E - ln 4 zeta)/Lx
    double far_lx;             // Lx
    const float4* tab32;
    const dbl4* tab64;
    // first-order Taylor table (Sec. 2.2.5, approach 2), J = dA_c/dd.  FP64: per grid point 4
    // records of 4 values, (C, A_cx, A_cy, A_cz), (Jxx, Jyy, Jzz, Jxy), (Jxz, Jyz, 0, 0), (0, 0, 0, 0).
    // FP32: per grid point 2 records, (C, A_c) and the FP16 pairs (Jxx, Jyy), (Jzz, Jxy), (Jxz, Jyz)
    // of J / s with s = max |J| as the fourth word
    int taylor;                // 1: the walk expands about the nearest grid point instead of trilinear
    double h[3];               // grid spacing ext / (n - 1)
    const float4* tay32;
    const dbl4* tay64;
};

struct ts_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // mesh
    bool have_mesh = false, have_tree = false;
    bool rec64 = true;                // tree builds write the FP64 cell and in-block node records
    bool rec64_valid = false;         // the current tree has them
    int nb = 0, nleaf = 0, nint = 0, depth_max = 0;
    int64_t ncell = 0;
    int bc[3] = {0, 0, 0};
    double L[3] = {1, 1, 1}, dlo[3] = {0, 0, 0};
    std::vector<int> blk_nid;        // node id of each block
    std::vector<int> leaf_blk;       // block of each leaf
    std::vector<int> amr_order;      // non-leaf node ids, deepest first
    std::vector<int> amr_level_off;  // offsets into amr_order per reduction round
    WalkGeom geom;
    uint32_t root_cw = 0;
    int walk_T[2] = {1, 1};           // targets per lane of the walk kernels (FP32, FP64)

    // device topology and records
    int* d_leaf_nid = nullptr;       // [nleaf]
    double* d_leaf_lo = nullptr;     // [nleaf*3]
    double* d_leaf_size = nullptr;   // [nleaf*3]
    int* d_amr_order = nullptr;      // [nb - nleaf]
    float4 *d_ncom32 = nullptr, *d_ncen32 = nullptr, *d_cell32 = nullptr;
    // FP32 positions and masses of every group of 8 siblings, structure of arrays (x[8], y[8],
    // z[8], m[8]: 8 float4 per group) for the paired walk: cells 8 g .. 8 g + 7 are cell group g,
    // nodes 1 + 8 g .. 8 + 8 g node group g (every child group of the breadth-first node ids)
    float4 *d_cellsoa = nullptr, *d_ncomsoa = nullptr;
    dbl4 *d_ncom64 = nullptr, *d_ncen64 = nullptr, *d_cell64 = nullptr;
    // MPE MAC moments (B2, B3) per internal node, computed on demand after each tree build
    std::vector<int> leaf_anc;       // [nleaf][anc_max] amr ancestors of each leaf-block (-1 padded)
    int anc_max = 0;
    int* d_leaf_anc = nullptr;
    double2* d_bmom64 = nullptr;     // [nint]
    float2* d_bmom32 = nullptr;      // [nint]
    int bmom_prec = 0;               // moments of the current tree: 0 none, 1 FP32 terms, 2 FP64 terms
    // Adaptive Block Update scratch (sized by the mesh)
    int64_t* d_abu_targets = nullptr;    // [abu_ntp] Morton ids of the corner cells, padded to 32
    int* d_abu_slot = nullptr;           // [nleaf * 8] list position of corner k of leaf-block n
    int64_t abu_ntp = 0;
    void* d_abu_out = nullptr;           // [abu_ntp][4] corner results (float or double)
    int* d_abu_warps = nullptr;          // [nleaf * 16] warps of the blocks to update
    int* d_abu_count = nullptr;          // [2] warps listed, blocks updated
    unsigned long long* d_blk_counts = nullptr;   // [nleaf] interactions per leaf-block
    double* d_workload = nullptr;        // [nleaf] block workload weights
    // numerical differentiation of the potential (ts_numdiff.cu), uploaded on first use
    std::vector<int2> nd_blk_host;       // [nb] by node id: (first child node id or -1, leaf index or -1)
    std::vector<int4> nd_leaf_host;      // [nleaf] integer position of the first cell at its depth, depth
    int2* d_nd_blk = nullptr;
    int4* d_nd_leaf = nullptr;
    bool have_nd = false;
    // partitioned walks (ts_partition.cu): interactions per leaf-block of the range walks, and the
    // per-block partial sums of the zero mean
    unsigned long long* d_range_counts = nullptr;   // [nleaf]
    bool range_counts_valid = false;
    double* d_range_part = nullptr;
    int range_part_cap = 0;
    // extra column quantities (ts_column_quantities): masses per cell (Morton) and per node
    int q_n = 0;                      // quantities of the current tree (0: total column only)
    float2* d_qcell32 = nullptr;      // [ncell]
    float2* d_qnode32 = nullptr;      // [nint]
    double2* d_qnode64 = nullptr;     // [nint] FP64 sums for the amr reduction
    float* d_shield_tab = nullptr;    // CO shielding table of the last ts_column_shielding
    size_t shield_cap = 0;
    void* d_sq = nullptr;             // SumSquare walk: per-thread priority queues
    size_t sq_bytes = 0;

    // Ewald correction table
    bool have_ewald = false;
    EwaldDev ew{};
    float4* d_ew32 = nullptr;
    dbl4* d_ew64 = nullptr;
    std::vector<double> ew_host;     // FP64 master copy [n^3 * 4]
    bool have_taylor = false;
    float4* d_tay32 = nullptr;       // [n^3][2] float4: 32-byte records (FP16 Jacobian, see ensure_taylor)
    dbl4* d_tay64 = nullptr;         // [n^3][4] dbl4 records
    std::vector<double> tay_host;    // [n^3][10] (C, A_c, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz)

    // node-ray table for the column walk
    bool have_noderay = false;
    int nr_nside = 0, nr_dims[4] = {0, 0, 0, 0}, nr_nsub = 0, nr_kmax = 0;   // nr_kmax: pairs in all
    double nr_psi[2] = {0, 0};
    double* d_nr_dense = nullptr;    // FP64 [ntheta][nphi][npsi][npix]
    uint4* d_nr_rec = nullptr;       // [entry] up to 4 (sub-cube count << 8) | pixel pairs (npix <= 192)
    uint32_t* d_nr_more = nullptr;   // continuation of the rows longer than 4 pairs

    // learned Ewald-correction surrogate (2P1I)
    bool have_mlp = false;
    double mlp_b[2] = {0.5, 2.0};       // aspect range b = Ly/Lx the network covers
    float* d_mlp_master = nullptr;       // FP32 parameters [8900]
    float* d_mlp_m = nullptr;            // Adam moments
    float* d_mlp_v = nullptr;
    float* d_mlp_grad = nullptr;         // gradient accumulator [8900]
    float* d_mlp_loss = nullptr;         // [1]
    void* d_mlp_img = nullptr;           // bf16 weight image + biases + de-normalisation (MLP_BYTES)
    float mlp_norm[8] = {1, 1, 1, 1, 0, 0, 0, 0};   // output scale[4], offset[4]

    // scratch, status and counters
    WalkGeom* d_geom = nullptr;                 // depth geometry read by the walk kernels
    int* d_status = nullptr;
    unsigned long long* d_counters = nullptr;   // [0] interactions, [1] MAC tests
    double* d_reduce = nullptr;                 // FP64 reduction scratch [4]
    double* d_err = nullptr;                    // error-metric values [2][err_cap]
    int64_t err_cap = 0;
    unsigned char* d_err_aux = nullptr;         // error-metric sums, maxima and selection state
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
};

// Makes `dev` the current device for the lifetime of the guard and restores the previous one.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Host-side fault injection for tests of the error paths (nothing is ever made to fail on the GPU).
// With the environment variable TS_FAULT=<site> (or <site>:<k>), every device or pinned-host
// allocation made while the entry point <site> runs (or only its k-th allocation, counted from 1
// per call) fails with cudaErrorMemoryAllocation without reaching the CUDA allocator.  Sites:
// create, tree_build, bmoments, ewald_field, taylor, noderay, walk, column, surrogate,
// batch_create, error_metrics, abu, probe.  The innermost FaultSite of a call is the active one.
struct FaultSite {
    const char* prev_site;
    int prev_count;
    explicit FaultSite(const char* site);
    ~FaultSite();
};
cudaError_t ts_malloc(void** p, size_t bytes);
cudaError_t ts_malloc_host(void** p, size_t bytes);

// 64-bit FNV-1a hash of a byte range (content check of the files the library writes), continuing
// from h (start with TS_FNV_INIT).
#define TS_FNV_INIT 0xcbf29ce484222325ull
uint64_t ts_fnv1a(const void* data, size_t bytes, uint64_t h);

// error helpers (ts_api.cu)
ts_status ts_fail(ts_status s, const std::string& msg);
ts_status ts_cuda_fail(cudaError_t e, const char* what);
#define TS_CUDA(call)                                          \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ts_cuda_fail(_e, #call); \
    } while (0)

// launchers (implemented next to their kernels)
cudaError_t launch_tree_build(ts_ctx* c, const double* density);
cudaError_t launch_bmoments(ts_ctx* c, bool fp64);
void free_abu(ts_ctx* c);
ts_status ensure_bmoments(ts_ctx* c, bool fp64);
cudaError_t launch_gravity_walk(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc);
ts_status validate_gravity(ts_ctx* c, const ts_gravity_params* p);
int ew_kind(const int bc[3]);
cudaError_t launch_zero_mean(ts_ctx* c, int precision, void* pot);
cudaError_t launch_num_diff(ts_ctx* c, int precision, const void* pot, void* acc);
ts_status ensure_numdiff(ts_ctx* c);
cudaError_t launch_ewald_table(ts_ctx* c, int n, double* d_out64);
cudaError_t launch_ewald_taylor(ts_ctx* c, int n, double eps, dbl4* d_out);
ts_status ensure_taylor(ts_ctx* c);
cudaError_t launch_noderay_dense(ts_ctx* c, int nside, const int dims[3], double psi_min,
                                 double psi_max, int nsub, double* d_out);
cudaError_t launch_column_walk(ts_ctx* c, const ts_column_params* p, float* cols);
cudaError_t launch_column_av(ts_ctx* c, int64_t n, int npix, const float* cols, double k, float* av);
cudaError_t launch_qsums(ts_ctx* c, int nq, const double* q);
cudaError_t launch_shielding(ts_ctx* c, int64_t n, int npix, const float* cols, const ts_shield_params* p,
                             const float* d_tab, float* out);
cudaError_t launch_ewald_samples_2p1i(cudaStream_t st, int64_t n, double bmin, double bmax, uint64_t seed,
                                      double zpow, float* feat, double* targ);
void free_mlp(ts_ctx* c);
ts_status ensure_noderay(ts_ctx* c, int nside, const int dims[3], double pmin, double pmax, int nsub);
ts_status column_table_params(const ts_column_params* p, int dims[3], double* pmin, double* pmax, int* nsub);
