/*
 * treesolver.h - C ABI of the GB300 tree solver for gravity and optical depths on block-structured
 * AMR meshes (Wünsch et al. 2018, "Tree-based solvers for adaptive mesh refinement code FLASH - I:
 * gravity and optical depths").
 *
 * General conventions
 * -------------------
 * - Every call returns a ts_status; nothing throws across the ABI.  ts_last_error() returns a
 *   thread-local message for the last failing call on this thread.
 * - Arguments are validated before any kernel launch.  A call that fails validation changes nothing.
 * - "_dev" pointers are CUDA device pointers on the context's device (for example a torch tensor's
 *   data_ptr()); all other pointers are host pointers that are only read during the call.  The
 *   caller owns every buffer it passes; the context owns all internal device memory.
 * - Calls are asynchronous on the context's stream; outputs are ready after ts_sync() or after
 *   any later synchronising operation on that stream.
 * - Device-side failures (walk stack overflow, non-finite output) are latched in a device status
 *   word and reported by ts_sync(); the outputs of the failing call are then undefined.
 * - A context is not thread-safe; use one context per host thread.
 * - Fault injection for tests of the error paths (host side only): with the environment variable
 *   TS_FAULT=<site> or TS_FAULT=<site>:<k>, the device and pinned-host allocations of the entry
 *   point <site> (all of them, or only the k-th of each call, counted from 1) fail as if the device
 *   were out of memory, without reaching the CUDA allocator; the call then returns
 *   TS_ERR_OUT_OF_MEMORY and leaves the context usable.  Sites: create, tree_build, bmoments,
 *   ewald_field, taylor, noderay, walk, column, surrogate, batch_create, batch_run, error_metrics,
 *   abu, probe.
 *
 * Mesh layout (Sec. 2): the domain is one root block (level 1) refined recursively into 8 equal
 * children; each leaf-block holds 8x8x8 cells (l_bt = 3).  Cells are addressed by the flat index
 *   cell = leaf * 512 + k * 64 + j * 8 + i        (x fastest),
 * where leaf counts leaf-blocks in the order they appear in the block list.  All per-cell inputs
 * and outputs (density, potential, acceleration, columns) use this order.
 */
#ifndef TREESOLVER_H
#define TREESOLVER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TS_API __attribute__((visibility("default")))
#else
#define TS_API
#endif

typedef enum {
    TS_OK = 0,
    TS_ERR_INVALID_ARG = 1,    /* a parameter or the mesh failed validation */
    TS_ERR_UNSUPPORTED = 2,    /* a valid request this build does not implement */
    TS_ERR_OUT_OF_MEMORY = 3,  /* device or host allocation failed */
    TS_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
    TS_ERR_NOT_BUILT = 5,      /* walk before tree build, or periodic walk before ts_ewald_field */
    TS_ERR_STACK_OVERFLOW = 6, /* a walk needed more stack than the kernel holds */
    TS_ERR_TIMEOUT = 7,        /* a bounded device wait gave up (reserved: no kernel of this
                                  build waits on another, so no call returns it) */
    TS_ERR_NUMERIC = 8         /* non-finite value detected */
} ts_status;

enum { TS_BC_ISOLATED = 0, TS_BC_PERIODIC = 1 };
enum { TS_MAC_BH = 0, TS_MAC_APE = 1, TS_MAC_MPE = 2, TS_MAC_SUMSQ = 3 };
enum { TS_PREC_FP64 = 0, TS_PREC_FP32_KAHAN = 1 };
enum { TS_EWALD_TABLE = 0, TS_EWALD_MLP = 1, TS_EWALD_TAYLOR = 2 };
enum { TS_ACCEL_DIRECT = 0, TS_ACCEL_NUMDIFF = 1 };

typedef struct ts_ctx ts_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to run on, or NULL
 * for a stream the context creates and owns.  *out receives the context (NULL on failure). */
TS_API ts_status ts_create(ts_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the context and the context itself.  NULL is accepted. */
TS_API ts_status ts_destroy(ts_ctx* ctx);

/* Message of the last failing call on this host thread ("" if none).  Valid until the next call. */
TS_API const char* ts_last_error(void);

/* Block octree of the mesh (Sec. 2): host arrays, copied during ts_tree_build.
 *   level[nblocks]     refinement level, root = 1, each child one deeper
 *   child[nblocks*8]   child block of octant c = ix + 2 iy + 4 iz, or -1 in all 8 for a leaf-block
 *   lo[nblocks*3]      lower corner; size[nblocks*3] edge lengths (cuboid blocks allowed, Sec. 2)
 *   bc[3]              gravity / column boundary condition per axis (TS_BC_*), Sec. 2.2
 * Block 0 must be the root; every child must lie exactly in its parent's octant. */
typedef struct {
    int32_t nblocks;
    const int32_t* level;
    const int32_t* child;
    const double* lo;
    const double* size;
    int32_t bc[3];
} ts_mesh;

/* Tree build (Sec. 2.1, "tree-build"): cell masses m = rho dV, then node masses and centres of mass
 * summed bottom-up in FP64 through the block-trees (8, 64, 512 nodes per leaf-block) and the
 * amr-tree to the root.  `mesh` may be NULL to keep the mesh of the previous call (only the
 * density changed); otherwise it is validated and ingested (a1).  density_dev: device FP64
 * [ncell] in the cell order above.  Errors: INVALID_ARG (mesh malformed, NULL density),
 * OUT_OF_MEMORY, CUDA. */
TS_API ts_status ts_tree_build(ts_ctx* ctx, const ts_mesh* mesh, const double* density_dev);

/* Whether the following tree builds write the FP64 records (default 1).  The FP32 walks read only
 * the FP32 records; the FP64 cell records and the FP64 records of the nodes inside leaf-blocks are
 * 45 % of a build's stores and serve only FP64 walks (and the FP64 MPE moments).  With 0, a build
 * skips them (the leaf-block and amr-tree nodes keep their FP64 records: ts_block_moments and the
 * amr sums read them), and an FP64 walk on that tree fails with NOT_BUILT until a build with 1.
 * Errors: INVALID_ARG (NULL ctx). */
TS_API ts_status ts_tree_fp64_records(ts_ctx* ctx, int32_t enabled);

/* Number of cells and leaf-blocks of the ingested mesh (0 before the first build). */
TS_API ts_status ts_mesh_info(ts_ctx* ctx, int64_t* ncell, int32_t* nleaf, int32_t* nblocks);

/* Copy the FP64 moments of every block (mass [nblocks], centre of mass [nblocks*3]) to host
 * memory, synchronising the stream.  For inspection and parity tests. */
TS_API ts_status ts_block_moments(ts_ctx* ctx, double* mass, double* com);

/* Ewald correction field (Secs. 2.2.3-2.2.5, App. A): tabulates C(d) = phi(d) - 1/|d| and
 * A_c(d) = A(d) - d/|d|^3 from the FP64 Ewald series on an n x n x n grid over the folded
 * separation domain [0, ex] x [0, ey] x [0, ez] (ex = Lx/2 on a periodic axis, the box edge on an
 * isolated axis, capped at the far distance where the far-field form takes over: 2 max(Lx, Ly) for
 * 2P1I, 2 Lx for 1P2I).  BCs and box aspect (b = Ly/Lx, c = Lz/Lx) come from the ingested mesh;
 * alpha = 2/Lx; real-space images i1^2 + (b i2)^2 + (c i3)^2 <= 15, Fourier terms
 * l1^2 + (l2/b)^2 + (l3/c)^2 <= 10.  Supported: fully periodic (3P), x,y periodic + z isolated
 * (2P1I), x periodic + y,z isolated (1P2I).  n_table in [8, 256] (0 selects 64).
 * cache_path: NULL, or a file to read the table from if it matches (BC, aspect, n) and its body
 * matches the 64-bit FNV-1a content hash stored in its header; otherwise (no file, another
 * configuration, or a damaged body) the table is generated and the file (re)written.
 * Errors: NOT_BUILT (no mesh), UNSUPPORTED (other BC combination), INVALID_ARG. */
TS_API ts_status ts_ewald_field(ts_ctx* ctx, int32_t n_table, const char* cache_path);

/* Copy the FP64 correction table [n][n][n][4] = (C, A_cx, A_cy, A_cz) with x slowest and its
 * extent[3] to host memory.  table may be NULL to query n only. */
TS_API ts_status ts_ewald_table_get(ts_ctx* ctx, int32_t* n, double* extent, double* table);

/* First-order Taylor table of the same field (Sec. 2.2.5, approach 2: the correction and its
 * gradient on one uniform grid, expanded to first order about the nearest grid point).  At every
 * point of the ts_ewald_field grid: C, A_c and the Jacobian J_ij = dA_c,i/dd_j (the gradient of C
 * is -A_c), J by central differences of the FP64 series with step 1e-5 Lx, symmetrised.  Built on
 * the device on first use (this call, or a walk with ewald = TS_EWALD_TAYLOR) and kept with the
 * correction table.  Copies [n][n][n][10] = (C, A_cx, A_cy, A_cz, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz) to
 * host memory (table may be NULL).  Synchronous.  Errors: NOT_BUILT (no ts_ewald_field), NUMERIC. */
TS_API ts_status ts_ewald_taylor_get(ts_ctx* ctx, int32_t* n, double* table);

/* Learned Ewald correction (an addition to the paper's table, Sec. 2.2.5 approach 2): a
 * 4-64-64-64-4 SiLU network maps the folded separation and the box aspect of x,y-periodic /
 * z-isolated (2P1I) domains,
 *   (|dx|/(Lx/2), |dy|/(Ly/2), |dz|/F_net, (b - b_min)/(b_max - b_min)) mapped to [-1, 1],
 *   F_net = 2 Lx max(1, b_max), b = Ly/Lx,
 * to the smooth correction (C, A_cx, A_cy, A_cz) in units Lx = 1 (C scales as 1/Lx, A as 1/Lx^2),
 * for |dz| <= F = 2 max(Lx, Ly) (the far-field form of Sec. 2.2.5 is used beyond).  |dz| is scaled
 * by one constant over the aspect range: scaled by F itself it would bend at b = 1.  The first
 * layer takes every feature as a BF16 value plus its BF16 remainder (16 significant bits).  Training data are samples of
 * the FP64 Ewald series (eqs. potential2p1i, intijscaled, int00; App. A) generated on the device;
 * forward and backward passes run on BF16 tensor cores with FP32 accumulation; Adam keeps FP32
 * master weights.  The table (ts_ewald_field) stays available as fallback and reference. */
typedef struct {
    double b_min, b_max;     /* aspect range covered, 0 < b_min < b_max */
    int64_t n_samples;       /* training samples (>= 1024) */
    int32_t steps;           /* optimiser steps */
    int32_t batch;           /* samples per step, a multiple of 128 */
    double lr;               /* peak learning rate (cosine decay to lr/100) */
    uint64_t seed;
    double z_power;          /* training separations have |dz|/F = t^z_power, t uniform (<= 0: 1) */
} ts_surrogate_params;

/* Train the surrogate (replaces any previous one).  final_loss: mean squared error of the last
 * batch in normalised output units (may be NULL).  Synchronous.  Errors: INVALID_ARG. */
TS_API ts_status ts_surrogate_train(ts_ctx* ctx, const ts_surrogate_params* p, double* final_loss);

/* Parameter export/import: params[8900] FP32 packed as W1[64][4], b1[64], W2[64][64], b2[64],
 * W3[64][64], b3[64], W4[4][64], b4[4] (W[out][in]); norm[8] = output scale[4], offset[4];
 * b_range[2] = (b_min, b_max).  get: NOT_BUILT without a surrogate. */
TS_API ts_status ts_surrogate_get(ts_ctx* ctx, float* params, float* norm, double* b_range);
TS_API ts_status ts_surrogate_set(ts_ctx* ctx, const float* params, const float* norm, const double* b_range);

/* Surrogate file (the trained network of ts_surrogate_train kept across runs, like the paper's
 * precomputed Ewald table file, App. B grv_bhEwaldFName): a header (magic "TSMLPNET", format
 * version, parameter count, b_range[2], norm[8], and a 64-bit FNV-1a hash of b_range, norm and the
 * parameters), then the FP32 parameters [8900] in the packing of ts_surrogate_get, little-endian.
 * save: NOT_BUILT without a surrogate, INVALID_ARG if the file cannot be written.
 * load: replaces the context's surrogate; INVALID_ARG for a missing, truncated, oversized or damaged
 * file (content hash mismatch; the context is then unchanged), UNSUPPORTED for another format
 * version or network shape.  Synchronous. */
TS_API ts_status ts_surrogate_save(ts_ctx* ctx, const char* path);
TS_API ts_status ts_surrogate_load(ts_ctx* ctx, const char* path);

/* Network outputs for n feature rows: feat_dev [n][4] (features as above, in [-1,1]) -> out_dev
 * [n][4] de-normalised corrections.  Asynchronous on the context stream. */
TS_API ts_status ts_surrogate_eval(ts_ctx* ctx, int64_t n, const float* feat_dev, float* out_dev);

/* Gradient of the mean squared error (normalised outputs) over n rows (a multiple of 128) with
 * respect to the packed parameters, computed by the training kernel without updating them:
 * grad[8900] host, loss host (may be NULL); targ_dev [n][4] normalised targets.  Synchronous. */
TS_API ts_status ts_surrogate_grad(ts_ctx* ctx, int64_t n, const float* feat_dev, const float* targ_dev,
                                   float* grad, double* loss);

/* Gravity walk parameters.
 *   mac        TS_MAC_BH (eq. bhmac: accept if h/|r - r_a| < theta), TS_MAC_APE (eq. ape with
 *              p = 1: accept if G M h^2 / d^4 < a_lim) or TS_MAC_MPE (eq. mpe with p = 1: accept if
 *              d > b_max and G/d^2 (1 - b_max/d)^-2 (3 B2/d^2 - 2 B3/d^3) < a_lim, with
 *              B_p = sum_i m_i |r_i - r_a|^p over the node's cells, computed on the device after
 *              each tree build on first use (from FP64 terms for the FP64 walk, from FP32 terms
 *              summed in FP64 across leaf-blocks for the FP32 walk), and b_max the distance from r_a to the node's
 *              furthest corner; one target per lane; not with the learned correction)
 *   theta      BH opening angle (paper default 0.5)
 *   safe_box   eta_SB: a node is accepted only if the target lies outside the cuboid eta_SB times
 *              the node around its geometric centre (Sec. 2.1; default 1.2); applied with both MACs
 *   a_lim      APE / MPE absolute limit (eq. abs_err); used when a_old_dev is NULL
 *   a_old_dev  NULL, or device float [ncell]: |a| of the previous step, so that the limit is
 *              eps_rel * a_old per cell (eq. rel_err)
 *   G          gravitational constant
 *   precision  TS_PREC_FP32_KAHAN: FP32 interactions with compensated per-cell sums; outputs
 *              float.  TS_PREC_FP64: FP64 throughout; outputs double.
 *   ewald      periodic and mixed BCs: TS_EWALD_TABLE trilinear interpolation of the correction
 *              table; TS_EWALD_TAYLOR the paper's first-order Taylor expansion about the nearest
 *              grid point (Sec. 2.2.5, approach 2; table built on first use, see
 *              ts_ewald_taylor_get); TS_EWALD_MLP the learned correction (2P1I, FP32 only).
 *              Ignored for isolated BCs.
 *   zero_mean  1: subtract the volume-weighted mean potential, accumulated in FP64 (meant for
 *              periodic and mixed BCs, whose potential is defined up to a constant; applied to
 *              any BC when requested)
 *   accel      TS_ACCEL_DIRECT: the walk sums eq. accel.  TS_ACCEL_NUMDIFF (Sec. 2.2.2, the
 *              alternative): the walk forms the potential alone (eq. pot; BH and absolute-limit APE
 *              have potential-only kernels, other MACs run the full walk) and the acceleration is
 *              the second-order central difference a_k = -(g(+1) - g(-1)) / (2 dx_k) of the
 *              potential, g(m) being the potential of the cube of the cell's own size m cells away
 *              along axis k: the containing leaf cell's value when that cell is as large or larger
 *              (injection), the volume-weighted mean of the leaf cells inside the cube when they
 *              are smaller (restriction); periodic axes wrap, and at an isolated domain edge the
 *              one-sided form -(-3 phi_0 + 4 g(1) - g(2)) / (2 dx_k) (mirrored) is used.  Not with
 *              the batched run, the adaptive block update or the autotuner (UNSUPPORTED).
 *   queue_max  TS_MAC_SUMSQ only: the most frontier nodes a target's priority queue holds (0: 4096).
 *
 * TS_MAC_SUMSQ, the SumSquare MAC (Sec. 2.2.1, experimental in the paper): per target, the frontier
 * of nodes waiting for evaluation is refined, node with the largest MPE bound (eq. mpe, p = 1)
 * first, until the sum of the squared bounds of the frontier is <= a_lim^2; the frontier is then
 * accepted.  A node whose bound does not apply (target within b_max of its centre of mass) or whose
 * safe box holds the target is always opened; cells are accepted when reached.  Equal bounds are
 * ordered by the node's depth and integer position.  The summed squares are kept exactly in integer
 * units of 2^-20 a_lim^2 (each bound rounded up).  If opening a node would need more than queue_max
 * queue entries the target's refinement stops there (counted, see ts_walk_counters).  One thread per
 * target with its queue in context-owned device scratch of (threads) x queue_max x (4 + 4 or 8) bytes
 * (threads: up to 2048 per SM, fewer if the queues would take more than half the free memory);
 * absolute a_lim only; any BC with the table or Taylor correction; not with the learned
 * correction, the batched run, ranges, the block update or the autotuner (UNSUPPORTED). */
typedef struct {
    int32_t mac;
    double theta;
    double safe_box;
    double a_lim;
    const float* a_old_dev;
    double eps_rel;
    double G;
    int32_t precision;
    int32_t ewald;
    int32_t zero_mean;
    int32_t accel;
    int32_t queue_max;
} ts_gravity_params;

/* Fill p with the paper's defaults: BH, theta 0.5, eta_SB 1.2, G 1, FP32+Kahan, table Ewald. */
TS_API void ts_gravity_params_default(ts_gravity_params* p);

/* Gravity walk (Sec. 2.1 tree-walk; Sec. 2.2.2 eqs. pot/accel; Secs. 2.2.3-2.2.5 with the
 * correction table for periodic and mixed BCs): for every cell, a depth-first walk from the root;
 * accepted nodes add Phi -= G M phi(d), a -= G M A(d) (d = r - r_a, minimum image on periodic
 * axes); cells are always accepted except the target itself.
 * pot_dev: device [ncell], acc_dev: device [ncell][3]; float for FP32_KAHAN, double for FP64.
 * Errors: NOT_BUILT (no tree, or periodic BCs without ts_ewald_field), INVALID_ARG (theta <= 0
 * with BH, a_lim <= 0 with APE and no a_old, NULL outputs).  Device errors via ts_sync. */
TS_API ts_status ts_gravity_walk(ts_ctx* ctx, const ts_gravity_params* p, void* pot_dev, void* acc_dev);

/* Column-density walk parameters (Sec. 2.3, OpticalDepth module).
 *   n_side     HEALPix resolution, N_PIX = 12 n_side^2 (the paper's tr_nSide = log2(n_side) + 1)
 *   theta      BH opening angle (Sec. 2.3 recommends theta ~ sqrt(4 pi / N_PIX))
 *   safe_box   eta_SB as for gravity
 *   max_dist   nodes farther than this are skipped (tr_bhMaxDist); <= 0 means unlimited
 *   table_*    node-ray table bins: theta, phi, psi counts (0: 25, 50, 25 as tr_ilNTheta,
 *              tr_ilNPhi, tr_ilNNS), psi range (0: [1e-3, 1]) and sub-cubes per edge (0: 8) */
typedef struct {
    int32_t n_side;
    double theta;
    double safe_box;
    double max_dist;
    int32_t table_ntheta, table_nphi, table_npsi, table_nsub;
    double table_psi_min, table_psi_max;
} ts_column_params;

TS_API void ts_column_params_default(ts_column_params* p);

/* Column-density walk (Sec. 2.3): per cell, the same walk with the BH MAC; each accepted node of
 * mass M at distance d adds M w_i / (Omega_pix d^2) to pixel i (Omega_pix = 4 pi / N_PIX), with
 * w_i the node-ray weights of the node's direction and angular size psi = h/d (nearest table
 * bin); the target's own cell adds rho dx / 2 to every pixel.  columns_dev: device float
 * [ncell][l_q][N_PIX], pixels in HEALPix RING order, l_q = 1 unless extra quantities are registered
 * (ts_column_quantities).  n_side in [1, 4].  The node-ray table is built on the device at the first
 * call for given table parameters.  Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED (l_q N_PIX > 432). */
TS_API ts_status ts_column_walk(ts_ctx* ctx, const ts_column_params* p, float* columns_dev);

/* Mean visual extinction per cell (Sec. 2.3, eq. av) from a column map:
 *   A_V = -(1/2.5) ln[(1/npix) sum_i exp(-2.5 k N_i)],
 * with k the conversion of the map's column unit into units of 1.87e21 cm^-2 of hydrogen (k = 1
 * for a map already in those units).  cols_dev: device float [n][npix] (the layout
 * ts_column_walk writes), read only; av_dev: device float [n], written; both caller-owned.  The sum
 * is formed about the smallest optical depth, so opaque cells give finite A_V.  Runs on the
 * context's stream (asynchronous); no tree is needed.  Errors: INVALID_ARG for a NULL ctx, n < 0,
 * npix < 1, k < 0 or not finite, or NULL pointers with n > 0. */
TS_API ts_status ts_column_av(ts_ctx* ctx, int64_t n, int32_t npix, const float* cols_dev, double k, float* av_dev);

/* Extra column quantities (Sec. 2.3: the paper maps l_q = 3 quantities, the total, H2 and CO
 * columns, with the same walk).  Registers nq in {0, 1, 2} extra per-cell densities q_dev (device
 * FP64 [nq][ncell], flat cell order, the density's units) for the current tree: their masses are
 * summed per node in FP64 (the node's position and MAC stay those of the total mass), and every
 * following ts_column_walk writes l_q = 1 + nq maps per cell, columns_dev [ncell][l_q][N_PIX] (total
 * first), each accepted node adding its mass of each quantity with the same node-ray weights.
 * A new ts_tree_build drops the quantities (l_q = 1 again); nq = 0 drops them explicitly.  The maps
 * live in shared memory during the walk: l_q N_PIX <= 432 (else the walk returns UNSUPPORTED).
 * Errors: NOT_BUILT (no tree), INVALID_ARG. */
TS_API ts_status ts_column_quantities(ts_ctx* ctx, int32_t nq, const double* q_dev);

/* Shielding averages per cell from l_q = 3 maps (Sec. 2.3: A_V by eq. av and the shielding
 * coefficients "computed by averaging over the Healpix maps in a similar way"):
 *   out[c][0] = A_V     = -(1/2.5) ln[(1/N_PIX) sum_i exp(-2.5 k_av N_i)]            (map 0)
 *   out[c][1] = <f_H2>  = (1/N_PIX) sum_i f(k_h2 N_H2,i), the H2 self-shielding factor
 *               f(N) = 0.965 / (1 + x / b5)^2 + 0.035 / sqrt(1 + x) exp(-8.5e-4 sqrt(1 + x)),
 *               x = N / 5e14 cm^-2 (Draine & Bertoldi 1996, eq. 37)                   (map 1)
 *   out[c][2] = <f_CO>  = (1/N_PIX) sum_i T(log10 k_co N_CO,i, log10 k_h2 N_H2,i), T the caller's
 *               table bilinearly interpolated and clamped at its edges; 1 without a table (map 2)
 * cols_dev: device float [n][3][npix] (the layout ts_column_walk writes with two quantities);
 * out_dev: device float [n][3].  FP32 arithmetic; asynchronous on the context's stream (the table
 * is copied before the call returns).  Errors: INVALID_ARG. */
typedef struct {
    double k_av;              /* map-0 column unit -> units of 1.87e21 cm^-2 of hydrogen (eq. av) */
    double k_h2;              /* map-1 column unit -> H2 molecules per cm^2 */
    double b5;                /* Doppler parameter of H2 in km/s (> 0) */
    double k_co;              /* map-2 column unit -> CO molecules per cm^2 */
    int32_t co_n_co, co_n_h2; /* CO table points per axis (>= 2 each), or both 0: no CO table */
    const double* co_table;   /* host [co_n_co][co_n_h2] shielding factors */
    double co_lg_co[2];       /* log10 N_CO of the first and last table rows */
    double co_lg_h2[2];       /* log10 N_H2 of the first and last table columns */
} ts_shield_params;
TS_API ts_status ts_column_shielding(ts_ctx* ctx, int64_t n, int32_t npix, const float* cols_dev,
                                     const ts_shield_params* p, float* out_dev);

/* Copy the node-ray table of the last column walk (dense FP64 [ntheta][nphi][npsi][N_PIX]) to host
 * memory; table may be NULL to query the sizes. */
TS_API ts_status ts_noderay_table_get(ts_ctx* ctx, int32_t* dims4, double* table);

/* ---- Batched execution of many independent grids (an addition beyond the paper, whose FLASH
 * runs walk one mesh per MPI rank).  A batch groups n contexts on one device, each holding its own
 * mesh (ts_tree_build called once with the mesh; ts_ewald_field for periodic/mixed BCs).  One run
 * rebuilds the trees (if densities are given) and walks every cell of every grid in ONE persistent
 * kernel: each warp takes the next chunk of 32-cell work items from a device queue (an atomic
 * counter) ordered by estimated cost (column items, then periodic, then isolated gravity items).
 * With use_graph the whole run (tree builds, queue reset, persistent kernel, zero-mean passes) is
 * captured once as a CUDA graph and replayed while the buffers and modes stay the same.  Runs on
 * the stream of ctxs[0]; the contexts must not be used elsewhere during a run.  FP32 + Kahan
 * gravity with the correction table only (no learned correction, no FP64) in batched mode. */
typedef struct ts_batch ts_batch;

TS_API ts_status ts_batch_create(ts_batch** out, ts_ctx* const* ctxs, int32_t n);
TS_API ts_status ts_batch_destroy(ts_batch* b);

/* gp: gravity parameters for all grids (or NULL: no gravity); pot_dev[i] / acc_dev[i]: float
 * outputs of grid i.  cp: column parameters (or NULL: no columns); cols_dev[i]: float
 * [ncell_i][N_PIX].  density_dev: NULL (keep the trees) or n device pointers (FP64 densities).
 * Errors: INVALID_ARG, NOT_BUILT (a context without mesh or Ewald table), UNSUPPORTED. */
TS_API ts_status ts_batch_run(ts_batch* b, const ts_gravity_params* gp, void* const* pot_dev, void* const* acc_dev,
                              const ts_column_params* cp, float* const* cols_dev, const double* const* density_dev,
                              int32_t use_graph);

/* Tuning of the persistent kernel: work items taken per queue access (1..64) and resident CTAs
 * per SM (1..16; 0 = as many as fit). */
TS_API ts_status ts_batch_set_tuning(ts_batch* b, int32_t items_per_dequeue, int32_t ctas_per_sm);

/* Execution form of ts_batch_run.  mode 0 (default): the persistent per-class kernels above.
 * mode 1: each grid's own single-grid kernels (tree build, walk specialised to its BCs and lookup,
 * column walk, zero mean), the grids spread largest first over `nstreams` streams (1..16) that
 * fork from and join into the batch stream, so small grids run beside large ones; with
 * use_graph the whole run is one captured graph, recaptured when any descriptor changes.  Both
 * forms give the same results; which is faster depends on the mix of grids (measure). */
TS_API ts_status ts_batch_set_mode(ts_batch* b, int32_t mode, int32_t nstreams);

/* Wait for the batch stream; report latched device status; counters of the last run:
 * out[0] gravity interactions, out[1] gravity MAC tests, out[2] column interactions, out[3] work
 * items, out[4] cells; last_ms: CUDA-event time of the last run (tree builds + walks). */
TS_API ts_status ts_batch_sync(ts_batch* b, int64_t* out5, double* last_ms);

/* Autotuner for the single-grid walk: times the given walk with 1, 2 and 4 targets per lane
 * (ts_set_walk_grouping) and keeps the fastest.  Outputs receive the walk's results.  ms[3]
 * (nullable) receives the three times.  Synchronous. */
TS_API ts_status ts_autotune_walk(ts_ctx* ctx, const ts_gravity_params* p, void* pot_dev, void* acc_dev,
                                  int32_t* best_targets_per_lane, double* ms);

/* Allocation-free zero-mean pass (no counterpart in the paper; a service for callers that may not
 * allocate device memory: host codes whose own allocator owns the device's memory budget, plugins
 * restricted to the memory they are handed, or time steps that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree).  It subtracts from pot_dev[0..n) the mean weighted by
 * weight_dev (device FP64 [n], NULL for equal weights), accumulated in FP64, like the zero_mean
 * option of ts_gravity_walk, but needs no context and allocates nothing: its scratch space is a
 * fixed file-scope device array of 4096 partial sums that every GPU loading the library keeps
 * until the process exits, so n may be at most 16,777,216 (larger n: TS_ERR_INVALID_ARG).
 * The first call on a device looks up the array's device address with that device current; make
 * that first call before any stream capture.  Asynchronous on cuda_stream (NULL: the legacy default
 * stream; pass the stream that wrote pot_dev and weight_dev).  pot_dev and weight_dev must be
 * device memory of `device` (or managed memory); any other pointer gives TS_ERR_INVALID_ARG.
 * All calls share the scratch array: calls that overlap on the GPU race. */
TS_API ts_status ts_zero_mean_noalloc(int32_t device, float* pot_dev, const double* weight_dev, int64_t n,
                                      void* cuda_stream);

/* Accuracy of a walk against a reference solution (Sec. 3, eq. ea, and its potential analogue).
 * For i in [0, n):
 *   e_a(i)   = |a(i) - a_ref(i)| / max_j |a_ref(j)|
 *   e_phi(i) = |phi(i) - phi_ref(i)| / max_j |phi_ref(j)|
 * where, with pot_mod_const != 0, phi and phi_ref are each first reduced by their own mean over
 * the n entries (potentials of periodic and mixed boundaries are defined up to a constant).
 * Statistics: median and 99th percentile by linear interpolation between order statistics
 * (position q (n - 1) in the sorted values), and the maximum.  Order statistics are selected
 * exactly on the device (radix selection on the FP64 bit patterns); sums and maxima are FP64.
 * Non-finite e values are counted in n_nonfinite and order above +inf.
 *   precision: TS_PREC_FP32_KAHAN (pot, acc are float) or TS_PREC_FP64 (double)
 *   pot_dev [n], acc_dev [n][3]: the walk's output; pot_ref_dev [n], acc_ref_dev [n][3]: FP64
 *   reference, all device pointers.  Either pair may be NULL (its statistics are then 0).
 *   e_dev: optional device FP64 [2][n] receiving e_a then e_phi per entry.
 * Scratch (16 n bytes + 33 KB) is owned by the context.  Runs on the context's stream and
 * synchronises it before returning the statistics.  n must be in [1, 2^31). */
typedef struct {
    int64_t n, n_nonfinite;
    double a_ref_max, phi_ref_max;
    double e_a_median, e_a_p99, e_a_max;
    double e_phi_median, e_phi_p99, e_phi_max;
} ts_error_stats;
TS_API ts_status ts_error_metrics(ts_ctx* ctx, int32_t precision, int64_t n, const void* pot_dev, const void* acc_dev,
                                  const double* pot_ref_dev, const double* acc_ref_dev, int32_t pot_mod_const,
                                  double* e_dev, ts_error_stats* out);

/* Adaptive Block Update (Sec. 2.2.6): pot_dev and acc_dev hold the previous potential and
 * acceleration of every cell on input (the result of an earlier walk of the same mesh) and the new
 * ones on output.  The walk first runs for the 8 corner cells (i, j, k in {0, 7}) of every
 * leaf-block; a block keeps its previous values in all its cells if at each corner
 * |a_new - a_old| < a_tol and, when phi_tol > 0, |phi_new - phi_old| < phi_tol; every other block
 * is walked in full.  Parameters as ts_gravity_walk (any MAC, BC, precision, Ewald mode; one target
 * per lane).  The workload weight of every leaf-block is then updated from the interactions of its
 * full walk N (0 if kept): W = W e^(-1/10) + (1 - e^(-1/10)) (2 + 8 N / N_max), starting at 2
 * (the paper's tau_wl = 10, omega_wl = 8).  n_updated (nullable): number of leaf-blocks walked in
 * full; giving it synchronises the stream.  Scratch (~80 B per leaf-block) is owned by the
 * context.  Errors as ts_gravity_walk; INVALID_ARG for a_tol < 0 or NaN. */
TS_API ts_status ts_gravity_walk_abu(ts_ctx* ctx, const ts_gravity_params* p, double a_tol, double phi_tol,
                                     void* pot_dev, void* acc_dev, int32_t* n_updated);

/* Workload weights [nleaf] of the leaf-blocks after the last ts_gravity_walk_abu (host copy,
 * synchronous).  NOT_BUILT before the first such call. */
TS_API ts_status ts_block_workload(ts_ctx* ctx, double* weights);

/* ---- One mesh partitioned over several GPUs (one process and one context per GPU).  The walk of a
 * cell reads only the tree (Sec. 2.1), so a rank walks the cells of its own contiguous range of
 * leaf-blocks [leaf_begin, leaf_end) (block order, the Morton order of the meshes of Sec. 2), ranges
 * of equal cost coming from each block's interactions in the previous walk (the per-block work the
 * paper balances its domains on, Sec. 2.2.6).  Every rank builds the whole tree (ts_tree_build from
 * all blocks' densities, gathered by the caller); the periodic zero mean sums the ranges' FP64 sums
 * over ranks (ts_potential_sums, caller's all-reduce, ts_potential_shift).
 *
 * ts_gravity_walk_range: as ts_gravity_walk for the cells of the range only; pot_dev / acc_dev are
 * the full-size [ncell] / [ncell][3] arrays, other cells are not written.  zero_mean must be 0
 * (INVALID_ARG) and accel TS_ACCEL_DIRECT (UNSUPPORTED).  The interactions of each leaf-block of the
 * range are recorded for ts_walk_block_counts.  An empty range is valid and launches nothing. */
TS_API ts_status ts_gravity_walk_range(ts_ctx* ctx, const ts_gravity_params* p, int32_t leaf_begin, int32_t leaf_end,
                                       void* pot_dev, void* acc_dev);

/* Interactions of every leaf-block in the latest range walk that covered it (0 for blocks no range
 * walk has covered since the mesh was ingested); counts[nleaf] host, synchronous.  NOT_BUILT before
 * the first ts_gravity_walk_range. */
TS_API ts_status ts_walk_block_counts(ts_ctx* ctx, int64_t* counts);

/* FP64 sums over the cells of leaf-blocks [leaf_begin, leaf_end): sums[0] = sum dV phi,
 * sums[1] = sum dV (host [2]; synchronous; per-block partial sums added in block order).  pot_dev:
 * float (TS_PREC_FP32_KAHAN) or double (TS_PREC_FP64) [ncell]. */
TS_API ts_status ts_potential_sums(ts_ctx* ctx, int32_t precision, const void* pot_dev, int32_t leaf_begin,
                                   int32_t leaf_end, double* sums);

/* pot_dev[i] -= shift (in FP64, stored in the array's precision) for the cells of the range;
 * asynchronous on the context's stream.  INVALID_ARG for a non-finite shift. */
TS_API ts_status ts_potential_shift(ts_ctx* ctx, int32_t precision, void* pot_dev, int32_t leaf_begin, int32_t leaf_end,
                                    double shift);

/* Wait for the context's stream and report any latched device status. */
TS_API ts_status ts_sync(ts_ctx* ctx);

/* Counters of the last walk: accepted interactions and MAC tests summed over cells, and the
 * CUDA-event time of the last walk kernel in milliseconds (after ts_sync). */
TS_API ts_status ts_stats(ts_ctx* ctx, int64_t* interactions, int64_t* mac_tests, double* last_walk_ms);

/* Walk-kernel grouping: each warp walks the tree for 32 * targets_per_lane target cells (1, 2 or 4
 * stacked 4x4x2 bricks of one leaf-block, sharing one stack and one staged node group per pop).
 * precision selects the FP32 or FP64 kernels.  Defaults: 1 (FP32), 1 (FP64).  Results do not
 * depend on the grouping (each target keeps its own MAC decisions); only the speed does. */
TS_API ts_status ts_set_walk_grouping(ts_ctx* ctx, int32_t precision, int32_t targets_per_lane);

/* Raw counters of the last walk kernel: out[0] accepted interactions, out[1] MAC tests (both summed
 * over cells), out[2] stack entries popped (summed over warps), out[3] lanes active in those
 * entries (summed), so out[3] / (32 out[2]) is the lane utilisation of the shared walk.  After a
 * SumSquare walk: out[1] bounds evaluated, out[2] queue pops, out[3] targets whose queue filled. */
TS_API ts_status ts_walk_counters(ts_ctx* ctx, int64_t* out);

/* Arithmetic peak probe (a measurement utility; no counterpart in the paper): the FMA throughput of
 * device `device` in TFLOP/s (2 flop per FMA), measured with 16 independent dependency chains per
 * thread on 8 CTAs of 256 threads per SM, timed with CUDA events after one warm-up launch.
 * kind: 0 FP32 scalar FMA, 1 FP32 packed f32x2 FMA, 2 FP64 FMA.  Synchronous; creates and destroys
 * its own stream, events and a 4-byte buffer. */
TS_API ts_status ts_peak_probe(int32_t device, int32_t kind, double* tflops);

/* Library version string. */
TS_API const char* ts_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TREESOLVER_H */
