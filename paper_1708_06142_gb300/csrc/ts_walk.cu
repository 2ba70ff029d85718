// Gravity tree walk (Sec. 2.1 tree-walk; BH MAC eq. bhmac with the safe box; APE MAC eq. ape with
// p = 1 and eqs. abs_err / rel_err; interactions eqs. pot / accel; periodic and mixed BCs through
// the Ewald correction table of Sec. 2.2.5, approach 2, with trilinear interpolation).
//
// Work decomposition: one warp walks the tree for 32 target cells that are consecutive in Morton
// order (a 4x4x2 brick of one leaf-block).  The warp shares one depth-first stack in shared
// memory; an entry is (child word of an opened node, mask of the lanes that opened it).  Popping
// an entry brings in the node's 8 children (the generic kernels stage them in shared memory with
// coalesced 16-byte loads, 128-256 B per group; the paired FP32 kernel reads the structure-of-
// arrays copy of the sibling group that the tree build writes, with broadcast 16-byte loads and no
// staging), then every lane of the mask tests each child against its own MAC:
// accepted children are summed, and a child opened by any lane is pushed with the ballot of the
// lanes that opened it.  Each lane therefore sees exactly the interaction list of its own
// depth-first walk, and lanes outside a mask idle.
//
// Precision: FP32 interactions; each popped group's <= 8 contributions are summed in FP32 and the
// group sum is added to the per-cell potential and acceleration with Kahan compensation (the
// FP64 variant sums plainly in FP64).  The isolated FP32 kernel with one target per lane takes the
// 8 children as 4 pairs and evaluates separations, MAC products and interactions of a pair with
// one packed f32x2 instruction each (sm_100+), which cuts the issue slots of the arithmetic by
// almost half; the kernel is issue bound, so this is its main lever after lane utilisation, and
// its bookkeeping is kept per warp (interaction counts from the pushed masks) or per pop (the
// compensated sums, in f32x2 pairs).
//
// Roofline: FP32-pipe (ALU) bound.  Algorithmic work: 20 flops + 1 rsqrt per accepted interaction
// (isolated), 9 + 6 flops per MAC test; node records come from L1/L2 (the tree of a 2M-cell mesh
// is ~43 MB of FP32 records and fits the 126 MB L2).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ts_walk_dev.cuh"

// Launchers of the kernel instantiations (ts_walk_f32_iso.cu, ts_walk_f32_corr.cu, ts_walk_f64.cu).
cudaError_t walk_launch_f32_iso(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T);
cudaError_t walk_launch_f32_table(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T);
cudaError_t walk_launch_f32_mlp(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T);
cudaError_t walk_launch_f64(ts_ctx* c, const WalkParams& P, int bck, int mac, bool rel, int T);
cudaError_t launch_walk_params(ts_ctx* c, const ts_gravity_params* p, const WalkParams& P, int bck, int T);
cudaError_t walk_launch_pot(ts_ctx* c, const WalkParams& P, bool fp64, int bck, int mac, bool rel);
cudaError_t launch_sumsq(ts_ctx* c, const ts_gravity_params* p, const WalkParams& W, void* pot, void* acc);

// per-context copy of the depth geometry in device memory (~2 KB, read once per CTA)
static cudaError_t upload_geom(ts_ctx* c, WalkGeom** out) {
    if (!c->d_geom) {
        cudaError_t e = ts_malloc((void**)&c->d_geom, sizeof(WalkGeom));
        if (e != cudaSuccess) return e;
    }
    *out = c->d_geom;
    return cudaMemcpyAsync(c->d_geom, &c->geom, sizeof(WalkGeom), cudaMemcpyHostToDevice, c->stream);
}

// Kernel parameters of one context's walk (also used for the batched persistent kernel).
// bck: 0 isolated, 1 correction table, 2 learned correction.
cudaError_t make_walk_params(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc, WalkParams* out, int* bck_out) {
    WalkGeom* dg = nullptr;
    cudaError_t e = upload_geom(c, &dg);
    if (e != cudaSuccess) return e;
    WalkParams& P = *out;
    memset(&P, 0, sizeof(P));
    const bool fp64 = p->precision == TS_PREC_FP64;
    P.ncom = fp64 ? (const void*)c->d_ncom64 : (const void*)c->d_ncom32;
    P.ncen = fp64 ? (const void*)c->d_ncen64 : (const void*)c->d_ncen32;
    P.cell = fp64 ? (const void*)c->d_cell64 : (const void*)c->d_cell32;
    P.cell_soa = c->d_cellsoa;
    P.ncom_soa = c->d_ncomsoa;
    P.ncell = c->ncell;
    P.leaf_begin = 0;
    P.leaf_end = c->nleaf;
    P.root_cw = c->root_cw;
    P.theta2 = p->theta * p->theta;
    P.eta = p->safe_box;
    P.a_lim = p->a_lim;
    P.G = p->G;
    P.eps_rel = p->eps_rel;
    P.a_old = p->a_old_dev;
    P.geom = dg;
    // The safe box (Sec. 2.1) only matters where a target inside it could pass the MAC.  A target
    // in the eta box of a node and the node's centre of mass are at most ext = |(eta + 1) half| apart,
    // so with BH (accept iff h^2 < theta^2 d^2) and theta^2 ext^2 < h^2 an accepted node always has
    // the target outside its box: the test is skipped at such depths (2 % margin for FP32 rounding).
    // The APE and MPE MACs can accept light nodes at any distance: always tested.
    P.bmom = fp64 ? (const void*)c->d_bmom64 : (const void*)c->d_bmom32;
    P.sb_depths = 0xffffffffu;
    if (p->mac == TS_MAC_BH) {
        P.sb_depths = 0;
        for (int d = 0; d <= TS_MAX_DEPTH; ++d) {
            const double e = p->safe_box + 1.0, *hf = c->geom.half64[d];
            const double ext2 = e * e * (hf[0] * hf[0] + hf[1] * hf[1] + hf[2] * hf[2]);
            if (!(p->theta * p->theta * ext2 < 0.98 * c->geom.hmax2_64[d])) P.sb_depths |= 1u << d;
        }
    }
    int bck = (c->bc[0] || c->bc[1] || c->bc[2]) ? 1 : 0;
    if (bck && p->ewald == TS_EWALD_MLP) {
        // far-field constants of 2P1I (Sec. 2.2.5) and the network's feature and output scales
        bck = 2;
        const double Lx = c->L[0], Ly = c->L[1], b = Ly / Lx, zeta = M_PI * M_PI / 4.0;
        const double F = 2.0 * Lx * std::max(1.0, b);
        memset(&P.ew, 0, sizeof(P.ew));
        P.ew.kind = TS_EW_2P1I;
        P.ew.far = F;
        P.ew.far_slope = 2 * M_PI / (b * Lx * Lx);
        P.ew.far_const = 2 * sqrt(M_PI * zeta) / (M_PI * b * Lx);
        P.ew.far_lx = Lx;
        P.mlp_img = c->d_mlp_img;
        P.mlp_sx = (float)(4.0 / Lx);
        P.mlp_sy = (float)(4.0 / Ly);
        // |dz| is scaled by the far distance of the widest box the network covers, one constant for
        // the whole aspect range (the walk's own far distance F = 2 max(Lx, Ly) bends at b = 1)
        P.mlp_sz = (float)(2.0 / (2.0 * Lx * std::max(1.0, c->mlp_b[1])));
        P.mlp_f3 = (float)(2.0 * (b - c->mlp_b[0]) / (c->mlp_b[1] - c->mlp_b[0]) - 1.0);
        P.mlp_c = (float)(1.0 / Lx);
        P.mlp_a = (float)(1.0 / (Lx * Lx));
    } else if (bck) {
        P.ew = c->ew;
        P.ew.taylor = p->ewald == TS_EWALD_TAYLOR ? 1 : 0;
    }
    P.pot = pot;
    P.acc = acc;
    P.status = c->d_status;
    P.counters = c->d_counters;
    *bck_out = bck;
    return cudaSuccess;
}

cudaError_t launch_gravity_walk(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc) {
    WalkParams P;
    int bck = 0;
    cudaError_t e = make_walk_params(c, p, pot, acc, &P, &bck);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, 4 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    cudaEventRecord(c->ev0, c->stream);
    if (p->mac == TS_MAC_SUMSQ) {   // priority-queue walk, one thread per target (ts_sumsq.cu)
        e = launch_sumsq(c, p, P, pot, acc);
        if (e == cudaSuccess && p->accel == TS_ACCEL_NUMDIFF) e = launch_num_diff(c, p->precision, pot, acc);
    } else if (p->accel == TS_ACCEL_NUMDIFF) {
        // potential-only walk (full walk where no potential-only kernel exists), then the
        // acceleration by numerical differentiation of the potential (Sec. 2.2.2)
        const bool rel = p->mac != TS_MAC_BH && p->a_old_dev != nullptr;
        e = walk_launch_pot(c, P, p->precision == TS_PREC_FP64, bck, p->mac, rel);
        if (e == cudaErrorNotSupported) e = launch_walk_params(c, p, P, bck, 1);
        if (e == cudaSuccess) e = launch_num_diff(c, p->precision, pot, acc);
    } else {
        e = launch_walk_params(c, p, P, bck, c->walk_T[p->precision == TS_PREC_FP64 ? 1 : 0]);
    }
    cudaEventRecord(c->ev1, c->stream);
    c->timed = true;
    return e;
}

// Launch of prepared parameters (T targets per lane; subsets of targets need T = 1).
cudaError_t launch_walk_params(ts_ctx* c, const ts_gravity_params* p, const WalkParams& P, int bck, int T) {
    const bool rel = p->mac != TS_MAC_BH && p->a_old_dev != nullptr;
    if (p->precision == TS_PREC_FP64) return walk_launch_f64(c, P, bck, p->mac, rel, T);
    if (bck == 0) return walk_launch_f32_iso(c, P, p->mac, rel, T);
    if (bck == 1) return walk_launch_f32_table(c, P, p->mac, rel, T);
    return walk_launch_f32_mlp(c, P, p->mac, rel, T);
}

// ------------------------------------------------------------------------------ zero mean
// Fully periodic BCs: the potential is defined up to a constant; subtract the volume-weighted
// mean over all cells, accumulated in FP64.
template <typename R>
__global__ void k_pot_mean(const R* __restrict__ pot, const double* __restrict__ leaf_size, int64_t ncell,
                           double* __restrict__ out) {
    double s = 0, v = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = i >> 9;
        const double dv = leaf_size[3 * n] * leaf_size[3 * n + 1] * leaf_size[3 * n + 2];
        s += dv * (double)pot[i];
        v += dv;
    }
    for (int off = 16; off; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    __shared__ double ss[32], sv[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { ss[w] = s; sv[w] = v; }
    __syncthreads();
    if (w == 0) {
        s = l < (int)(blockDim.x >> 5) ? ss[l] : 0;
        v = l < (int)(blockDim.x >> 5) ? sv[l] : 0;
        for (int off = 16; off; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            v += __shfl_xor_sync(0xffffffffu, v, off);
        }
        if (l == 0) { atomicAdd(&out[0], s); atomicAdd(&out[1], v); }
    }
}

template <typename R>
__global__ void k_pot_sub(R* __restrict__ pot, int64_t ncell, const double* __restrict__ sums) {
    const double mean = sums[0] / sums[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell; i += (int64_t)gridDim.x * blockDim.x)
        pot[i] = (R)((double)pot[i] - mean);
}

cudaError_t launch_zero_mean(ts_ctx* c, int precision, void* pot) {
    cudaError_t e = cudaMemsetAsync(c->d_reduce, 0, 2 * sizeof(double), c->stream);
    if (e != cudaSuccess) return e;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const int grid = nsm * 4;
    if (precision == TS_PREC_FP64) {
        k_pot_mean<double><<<grid, 256, 0, c->stream>>>((const double*)pot, c->d_leaf_size, c->ncell, c->d_reduce);
        k_pot_sub<double><<<grid, 256, 0, c->stream>>>((double*)pot, c->ncell, c->d_reduce);
    } else {
        k_pot_mean<float><<<grid, 256, 0, c->stream>>>((const float*)pot, c->d_leaf_size, c->ncell, c->d_reduce);
        k_pot_sub<float><<<grid, 256, 0, c->stream>>>((float*)pot, c->ncell, c->d_reduce);
    }
    return cudaGetLastError();
}
