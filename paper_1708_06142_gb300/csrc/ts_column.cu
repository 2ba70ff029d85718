// Column-density (OpticalDepth) walk, Sec. 2.3, and its node-ray weight table.
//
// k_noderay_dense: one thread per table entry (theta bin, phi bin, psi bin).  The node is an
// axis-aligned uniform cube of edge psi at unit distance in the bin-centre direction, split into
// nsub^3 sub-cubes; w_i is the fraction of sub-cube centres whose direction falls in HEALPix pixel
// i (RING scheme, Gorski et al. 2005).  theta bins are uniform in [0, pi], phi bins in [0, 2 pi),
// psi bins log-uniform in [psi_min, psi_max].  The host compacts each entry to its non-zero
// (pixel, weight) pairs.
//
// k_column_walk: the gravity walk's traversal (warp-shared stack, per-lane masks, BH MAC with the
// safe box); an accepted node of mass M at distance d adds M w_i / (Omega_pix d^2) to pixel i of
// its target's map, w from the nearest table bin of (theta, phi, psi = h/d) of the direction from
// the target to the node.  Each lane's map lives in shared memory as [pixel][lane] (conflict-free
// scatter).  The own cell adds rho dx / 2 to every pixel.
//
// Roofline: the scatter is FP32/shared-memory bound; the output ([ncell][N_PIX] floats, 403 MB for
// 128^3 cells at N_PIX = 48) is an HBM write.
#include <math.h>
#include <string.h>

#include "ts_internal.cuh"

// HEALPix RING pixel of a direction with z = cos(theta), azimuth phi.
__device__ int hp_ring_pixel(int ns, double z, double phi) {
    const double twopi = 2.0 * M_PI;
    z = fmin(1.0, fmax(-1.0, z));
    double t = fmod(phi, twopi);
    if (t < 0) t += twopi;
    t *= 2.0 / M_PI;                       // t in [0, 4)
    const double za = fabs(z);
    if (za <= 2.0 / 3.0) {
        // equatorial zone: pixel boundaries are the lines ns (t + 1/2) +- (3/4) ns z = integer
        const double u = ns * (0.5 + t), v = 0.75 * ns * z;
        const int asc = (int)floor(u - v), dsc = (int)floor(u + v);
        const int ring = ns + 1 + asc - dsc;             // 1 .. 2 ns + 1 below the z = 2/3 ring
        const int odd = (ring & 1) ? 0 : 1;
        int ip = (asc + dsc - ns + odd + 1) / 2;
        ip %= 4 * ns;
        if (ip < 0) ip += 4 * ns;
        return 2 * ns * (ns - 1) + (ring - 1) * 4 * ns + ip;
    }
    // polar caps: rings of 4 r pixels, r counted from the pole
    const double frac = t - floor(t);
    const double s = ns * sqrt(3.0 * (1.0 - za));
    const int asc = (int)floor(frac * s), dsc = (int)floor((1.0 - frac) * s);
    const int r = asc + dsc + 1;
    int ip = (int)floor(t * r);
    ip %= 4 * r;
    return z > 0 ? 2 * r * (r - 1) + ip : 12 * ns * ns - 2 * r * (r + 1) + ip;
}

__global__ void k_noderay_dense(int ns, int nth, int nph, int nps, double pmin, double pmax, int nsub,
                                double* __restrict__ out) {
    const int npix = 12 * ns * ns;
    const int nent = nth * nph * nps;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
        const int is = e % nps, ip = (e / nps) % nph, it = e / (nps * nph);
        const double th = (it + 0.5) * M_PI / nth, ph = (ip + 0.5) * 2.0 * M_PI / nph;
        const double psi = pmin * pow(pmax / pmin, (is + 0.5) / nps);
        double st, ct, sp, cp;
        sincos(th, &st, &ct);
        sincos(ph, &sp, &cp);
        const double cx = st * cp, cy = st * sp, cz = ct;
        double* w = out + (size_t)e * npix;
        for (int i = 0; i < npix; ++i) w[i] = 0;
        const double inv = 1.0 / ((double)nsub * nsub * nsub);
        for (int a = 0; a < nsub; ++a)
            for (int b = 0; b < nsub; ++b)
                for (int c = 0; c < nsub; ++c) {
                    const double x = cx + psi * ((a + 0.5) / nsub - 0.5);
                    const double y = cy + psi * ((b + 0.5) / nsub - 0.5);
                    const double z = cz + psi * ((c + 0.5) / nsub - 0.5);
                    const double r = sqrt(x * x + y * y + z * z);
                    const int p = hp_ring_pixel(ns, z / r, atan2(y, x));
                    if (p >= 0 && p < npix) w[p] += inv;
                }
    }
}

cudaError_t launch_noderay_dense(ts_ctx* c, int nside, const int dims[3], double pmin, double pmax, int nsub,
                                 double* d_out) {
    const int nent = dims[0] * dims[1] * dims[2];
    k_noderay_dense<<<(nent + 127) / 128, 128, 0, c->stream>>>(nside, dims[0], dims[1], dims[2], pmin, pmax, nsub,
                                                                d_out);
    return cudaGetLastError();
}

#include "ts_column_dev.cuh"

template <int NQ>
__global__ void __launch_bounds__(32 * TS_WALK_WARPS) k_column_walk(const __grid_constant__ ColParams P) {
    extern __shared__ float s_map[];   // [TS_WALK_WARPS][1 + NQ][npix][32]
    __shared__ __align__(16) float4 s_com[TS_WALK_WARPS][8];
    __shared__ __align__(16) float4 s_cen[TS_WALK_WARPS][8];
    __shared__ __align__(8) float2 s_q[TS_WALK_WARPS][8];
    __shared__ uint2 s_stack[TS_WALK_WARPS][TS_WALK_STACK];
    __shared__ float s_half[TS_MAX_DEPTH + 1][3];
    __shared__ float s_h2[TS_MAX_DEPTH + 1];
    for (int t = threadIdx.x; t <= TS_MAX_DEPTH; t += blockDim.x) {
        s_half[t][0] = P.geom->half32[t][0]; s_half[t][1] = P.geom->half32[t][1];
        s_half[t][2] = P.geom->half32[t][2]; s_h2[t] = P.geom->hmax2_32[t];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * TS_WALK_WARPS + warp;
    if (gw * 32 >= P.ncell) return;
    col_walk_warp<NQ>(P, gw, lane, s_map + (size_t)warp * (1 + NQ) * P.npix * 32, s_com[warp], s_cen[warp],
                      s_stack[warp], s_half, s_h2, s_q[warp]);
}

static size_t col_smem(const ColParams& P, int nq) { return sizeof(float) * (size_t)(1 + nq) * P.npix * 32 * TS_WALK_WARPS; }

static cudaError_t col_launch(ts_ctx* c, const ColParams& P, int nq) {
    const size_t smem = col_smem(P, nq);
    const int64_t nwarps = c->ncell / 32;
    const int grid = (int)((nwarps + TS_WALK_WARPS - 1) / TS_WALK_WARPS);
    cudaError_t e = cudaSuccess;
    if (nq == 0) {
        e = cudaFuncSetAttribute(k_column_walk<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_column_walk<0><<<grid, 32 * TS_WALK_WARPS, smem, c->stream>>>(P);
    } else if (nq == 1) {
        e = cudaFuncSetAttribute(k_column_walk<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_column_walk<1><<<grid, 32 * TS_WALK_WARPS, smem, c->stream>>>(P);
    } else {
        e = cudaFuncSetAttribute(k_column_walk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_column_walk<2><<<grid, 32 * TS_WALK_WARPS, smem, c->stream>>>(P);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Kernel parameters of one context's column walk; the node-ray table comes from `tab` (a context
// whose table matches the parameters; the batch shares one table between its grids).
cudaError_t make_col_params(ts_ctx* c, const ts_ctx* tab, const ts_column_params* p, float* cols, ColParams* out) {
    if (!c->d_geom) {
        cudaError_t e = ts_malloc((void**)&c->d_geom, sizeof(WalkGeom));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(c->d_geom, &c->geom, sizeof(WalkGeom), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    ColParams& P = *out;
    memset(&P, 0, sizeof(P));
    P.ncom = c->d_ncom32;
    P.ncen = c->d_ncen32;
    P.cell = c->d_cell32;
    P.ncell = c->ncell;
    P.theta2 = (float)(p->theta * p->theta);
    P.eta = (float)p->safe_box;
    P.max_dist2 = p->max_dist > 0 ? (float)(p->max_dist * p->max_dist) : 0.f;
    P.geom = c->d_geom;
    P.npix = tab->nr_dims[3];
    P.nth = tab->nr_dims[0];
    P.nph = tab->nr_dims[1];
    P.nps = tab->nr_dims[2];
    P.psi_lmin = (float)log2(tab->nr_psi[0]);
    P.psi_lscale = (float)(tab->nr_dims[2] / log2(tab->nr_psi[1] / tab->nr_psi[0]));
    // safe-box test only at depths where a target inside the box could pass the BH MAC (the same
    // bound as the gravity walk: |r - r_a| <= |(eta + 1) half| inside the box)
    P.sb_depths = 0;
    for (int d = 0; d <= TS_MAX_DEPTH; ++d) {
        const double e = p->safe_box + 1.0, *hf = c->geom.half64[d];
        const double ext2 = e * e * (hf[0] * hf[0] + hf[1] * hf[1] + hf[2] * hf[2]);
        if (!(p->theta * p->theta * ext2 < 0.98 * c->geom.hmax2_64[d])) P.sb_depths |= 1u << d;
    }
    // the pairs store sub-cube counts: their weight is count / nsub^3, folded into 1 / Omega_pix
    P.inv_omega = (float)(P.npix / (4.0 * M_PI) / ((double)tab->nr_nsub * tab->nr_nsub * tab->nr_nsub));
    P.leaf_size = c->d_leaf_size;
    P.nr_rec = tab->d_nr_rec;
    P.nr_more = tab->d_nr_more;
    P.out = cols;
    P.status = c->d_status;
    P.counters = c->d_counters;
    return cudaSuccess;
}

// Launch of prepared parameters on the context's stream (no counter reset, no timing events; the
// batch maps the total column only).
cudaError_t launch_col_params(ts_ctx* c, const ColParams& P) { return col_launch(c, P, 0); }

cudaError_t launch_column_walk(ts_ctx* c, const ts_column_params* p, float* cols) {
    ColParams P;
    cudaError_t e = make_col_params(c, c, p, cols, &P);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    const int nq = c->q_n;
    if (nq > 0) {
        P.qcell = c->d_qcell32;
        P.qnode = c->d_qnode32;
    }
    cudaEventRecord(c->ev0, c->stream);
    e = col_launch(c, P, nq);
    cudaEventRecord(c->ev1, c->stream);
    c->timed = true;
    return e;
}

// ------------------------------------------------------------------------------ extra quantities
// Masses of the extra mapped quantities (Sec. 2.3: the paper maps the H2 and CO columns beside the
// total one): per cell m_q = rho_q dV, per node the sum over its cells, in FP64 with the tree
// build's summation order (children in octant order), stored as FP32 pairs.  One CTA of 512
// threads per leaf-block, then one CTA for the amr-tree rounds (deepest first).
__device__ __forceinline__ int q_morton(int i, int j, int k) {
    const int q = (i >> 2) | ((j >> 2) << 1) | ((k >> 2) << 2);
    const int o = ((i >> 1) & 1) | (((j >> 1) & 1) << 1) | (((k >> 1) & 1) << 2);
    const int o2 = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return 64 * q + 8 * o + o2;
}

__global__ void __launch_bounds__(512) k_qsums(const double* __restrict__ q, int nq, int64_t ncell,
                                               const double* __restrict__ leaf_size, const int* __restrict__ leaf_nid,
                                               int nb, float2* __restrict__ qcell, float2* __restrict__ qnode32,
                                               double2* __restrict__ qnode64) {
    __shared__ double2 sm[512];
    __shared__ double2 l2[64], l1[8];
    const int n = blockIdx.x, t = threadIdx.x;
    const int i = t & 7, j = (t >> 3) & 7, k = t >> 6;
    const double dv = __dmul_rn(__dmul_rn(__dmul_rn(leaf_size[3 * n], 0.125), __dmul_rn(leaf_size[3 * n + 1], 0.125)),
                                __dmul_rn(leaf_size[3 * n + 2], 0.125));
    const size_t id = (size_t)n * TS_NCB + t;
    const double a = __dmul_rn(q[id], dv), b = nq > 1 ? __dmul_rn(q[ncell + id], dv) : 0.0;
    sm[q_morton(i, j, k)] = make_double2(a, b);
    __syncthreads();
    qcell[id] = make_float2((float)sm[t].x, (float)sm[t].y);   // Morton order, like the cell records
    const int base = nb + 72 * n;
    if (t < 64) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < 8; ++c) { s.x = __dadd_rn(s.x, sm[8 * t + c].x); s.y = __dadd_rn(s.y, sm[8 * t + c].y); }
        l2[t] = s;
        qnode64[base + 8 + t] = s;
        qnode32[base + 8 + t] = make_float2((float)s.x, (float)s.y);
    }
    __syncthreads();
    if (t < 8) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < 8; ++c) { s.x = __dadd_rn(s.x, l2[8 * t + c].x); s.y = __dadd_rn(s.y, l2[8 * t + c].y); }
        l1[t] = s;
        qnode64[base + t] = s;
        qnode32[base + t] = make_float2((float)s.x, (float)s.y);
    }
    __syncthreads();
    if (t == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < 8; ++c) { s.x = __dadd_rn(s.x, l1[c].x); s.y = __dadd_rn(s.y, l1[c].y); }
        qnode64[leaf_nid[n]] = s;
        qnode32[leaf_nid[n]] = make_float2((float)s.x, (float)s.y);
    }
}

__global__ void __launch_bounds__(256) k_qsums_amr(const int* __restrict__ order, const int* __restrict__ level_off,
                                                   int nrounds, const float4* __restrict__ ncen32,
                                                   float2* __restrict__ qnode32, double2* __restrict__ qnode64) {
    for (int r = 0; r < nrounds; ++r) {
        for (int idx = level_off[r] + threadIdx.x; idx < level_off[r + 1]; idx += blockDim.x) {
            const int nid = order[idx];
            const int first = (int)(__float_as_uint(ncen32[nid].w) & TS_CW_INDEX_MASK);
            double2 s = make_double2(0.0, 0.0);
            for (int c = 0; c < 8; ++c) {
                const double2 v = qnode64[first + c];
                s.x = __dadd_rn(s.x, v.x);
                s.y = __dadd_rn(s.y, v.y);
            }
            qnode64[nid] = s;
            qnode32[nid] = make_float2((float)s.x, (float)s.y);
        }
        __syncthreads();
        __threadfence_block();
    }
}

cudaError_t launch_qsums(ts_ctx* c, int nq, const double* q) {
    k_qsums<<<c->nleaf, 512, 0, c->stream>>>(q, nq, c->ncell, c->d_leaf_size, c->d_leaf_nid, c->nb, c->d_qcell32,
                                             c->d_qnode32, c->d_qnode64);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nrounds = (int)c->amr_level_off.size() - 1;
    if (nrounds > 0 && !c->amr_order.empty()) {
        k_qsums_amr<<<1, 256, 0, c->stream>>>(c->d_amr_order, c->d_amr_order + c->amr_order.size(), nrounds,
                                              c->d_ncen32, c->d_qnode32, c->d_qnode64);
        e = cudaGetLastError();
    }
    return e;
}

// ------------------------------------------------------------------------------ shielding averages
// Per cell, from its l_q = 3 maps (total, H2, CO; Sec. 2.3): A_V of eq. av (log-sum-exp about the
// smallest optical depth, as k_column_av), the mean over pixels of the H2 self-shielding factor
// f(N_H2) = 0.965 / (1 + x / b5)^2 + 0.035 / sqrt(1 + x) exp(-8.5e-4 sqrt(1 + x)), x = N_H2 / 5e14
// (Draine & Bertoldi 1996, eq. 37), and the mean over pixels of a CO shielding factor
// interpolated bilinearly in a caller's table over (log10 N_CO, log10 N_H2), clamped at its
// edges.  One thread per cell; HBM-bound (12 N_PIX + 12 bytes per cell).
__device__ __forceinline__ void lse_step(float t, float& tm, float& s);   // (mean extinction, below)

struct ShieldDev {
    float k25, ln_npix, k_h2, inv_b5, k_co;
    int nco, nh2;                 // table dims (0: no CO table)
    float lco0, sco, lh0, sh2;    // log10 origin and (n - 1) / range of each table axis
    const float* tab;             // [nco][nh2]
};

__device__ __forceinline__ float shield_h2(float n, float inv_b5) {
    const float x = n * (float)(1.0 / 5e14);
    const float a = 1.f + x * inv_b5;
    const float s = sqrtf(1.f + x);
    return 0.965f / (a * a) + 0.035f / s * expf(-8.5e-4f * s);
}

__device__ __forceinline__ float shield_co(const ShieldDev& S, float nco, float nh2) {
    const float uc = fminf(fmaxf((log10f(fmaxf(nco, 1e-30f)) - S.lco0) * S.sco, 0.f), (float)(S.nco - 1));
    const float uh = fminf(fmaxf((log10f(fmaxf(nh2, 1e-30f)) - S.lh0) * S.sh2, 0.f), (float)(S.nh2 - 1));
    const int ic = min((int)uc, S.nco - 2), ih = min((int)uh, S.nh2 - 2);
    const float fc = uc - ic, fh = uh - ih;
    const float* r0 = S.tab + ic * S.nh2 + ih;
    const float* r1 = r0 + S.nh2;
    return (r0[0] * (1.f - fh) + r0[1] * fh) * (1.f - fc) + (r1[0] * (1.f - fh) + r1[1] * fh) * fc;
}

__global__ void __launch_bounds__(256) k_shielding(int64_t n, int npix, const float* __restrict__ cols, ShieldDev S,
                                                   float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const float* tot = cols + c * 3 * npix;
        const float* h2 = tot + npix;
        const float* co = h2 + npix;
        float tm = S.k25 * __ldg(tot), s = 1.f, fh = 0.f, fc = 0.f;
        for (int p = 0; p < npix; ++p) {
            if (p) lse_step(S.k25 * __ldg(tot + p), tm, s);
            const float nh = S.k_h2 * __ldg(h2 + p);
            fh += shield_h2(nh, S.inv_b5);
            fc += S.nco ? shield_co(S, S.k_co * __ldg(co + p), nh) : 1.f;
        }
        out[3 * c] = (tm - logf(s) + S.ln_npix) / 2.5f;
        out[3 * c + 1] = fh / (float)npix;
        out[3 * c + 2] = fc / (float)npix;
    }
}

cudaError_t launch_shielding(ts_ctx* c, int64_t n, int npix, const float* cols, const ts_shield_params* p,
                             const float* d_tab, float* out) {
    if (n == 0) return cudaSuccess;
    ShieldDev S;
    S.k25 = (float)(2.5 * p->k_av);
    S.ln_npix = (float)log((double)npix);
    S.k_h2 = (float)p->k_h2;
    S.inv_b5 = (float)(1.0 / p->b5);
    S.k_co = (float)p->k_co;
    S.nco = d_tab ? p->co_n_co : 0;
    S.nh2 = d_tab ? p->co_n_h2 : 0;
    S.lco0 = (float)p->co_lg_co[0];
    S.sco = d_tab ? (float)((p->co_n_co - 1) / (p->co_lg_co[1] - p->co_lg_co[0])) : 0.f;
    S.lh0 = (float)p->co_lg_h2[0];
    S.sh2 = d_tab ? (float)((p->co_n_h2 - 1) / (p->co_lg_h2[1] - p->co_lg_h2[0])) : 0.f;
    S.tab = d_tab;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_shielding<<<(int)blocks, 256, 0, c->stream>>>(n, npix, cols, S, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ mean extinction
// A_V = -(1/2.5) ln[(1/N_PIX) sum_i exp(-2.5 k N_i)] per cell (Sec. 2.3, eq. av), from the cell's
// column map.  One thread per cell reads its row once (16-byte loads when the rows allow it, all
// independent, so many are in flight) and keeps a running log-sum-exp about the smallest optical
// depth seen so far: with t_i = 2.5 k N_i, t_m = min t_i and s = sum_i exp(t_m - t_i) >= 1,
// A_V = (t_m - ln s + ln N_PIX) / 2.5, finite however opaque the cell.  HBM-bound: 4 N_PIX + 4
// bytes per cell.
__device__ __forceinline__ void lse_step(float t, float& tm, float& s) {
    const float d = t - tm;
    const float e = expf(-fabsf(d));
    if (d >= 0.f) {
        s += e;                 // exp(t_m - t)
    } else {
        s = fmaf(s, e, 1.f);    // rescale to the new minimum t
        tm = t;
    }
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_column_av(int64_t n, int npix, const float* __restrict__ cols, float k25,
                                                   float ln_npix, float* __restrict__ av) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const float* row = cols + c * npix;
        float tm = k25 * row[0], s = 1.f;
        if constexpr (VEC) {   // npix % 4 == 0 and 16-byte aligned rows
            const float4* r4 = (const float4*)row;
            const float4 v0 = __ldg(r4);
            lse_step(k25 * v0.y, tm, s); lse_step(k25 * v0.z, tm, s); lse_step(k25 * v0.w, tm, s);
#pragma unroll 4
            for (int q = 1; q < npix / 4; ++q) {
                const float4 v = __ldg(r4 + q);
                lse_step(k25 * v.x, tm, s); lse_step(k25 * v.y, tm, s);
                lse_step(k25 * v.z, tm, s); lse_step(k25 * v.w, tm, s);
            }
        } else {
            for (int p = 1; p < npix; ++p) lse_step(k25 * __ldg(row + p), tm, s);
        }
        av[c] = (tm - logf(s) + ln_npix) / 2.5f;
    }
}

cudaError_t launch_column_av(ts_ctx* c, int64_t n, int npix, const float* cols, double k, float* av) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    const float k25 = (float)(2.5 * k), lnp = (float)log((double)npix);
    if (npix % 4 == 0 && ((uintptr_t)cols & 15) == 0)
        k_column_av<true><<<(int)blocks, 256, 0, c->stream>>>(n, npix, cols, k25, lnp, av);
    else
        k_column_av<false><<<(int)blocks, 256, 0, c->stream>>>(n, npix, cols, k25, lnp, av);
    return cudaGetLastError();
}
