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

struct ColParams {
    const float4* ncom;
    const float4* ncen;
    const float4* cell;
    int64_t ncell;
    float theta2, eta, max_dist2;
    const WalkGeom* geom;
    int npix, nth, nph, nps, kmax;
    float psi_lmin, psi_lscale;      // log(psi_min), nps / log(psi_max / psi_min)
    float inv_omega;                 // 1 / Omega_pix = N_PIX / (4 pi)
    const double* leaf_size;
    const float* nr_w;
    const uint8_t* nr_pix;
    const int* nr_cnt;
    float* out;
    int* status;
    unsigned long long* counters;
};

// Scatter one accepted node (mass m, separation d = r - r_a) into this lane's pixel map.
__device__ __forceinline__ void col_add(const ColParams& P, float* map, int lane, float m, float dx, float dy,
                                        float dz, float d2, float h) {
    if (P.max_dist2 > 0.f && d2 > P.max_dist2) return;
    const float inv = rsqrtf(d2);
    // direction from the target to the node is -d
    const float uz = fminf(1.f, fmaxf(-1.f, -dz * inv));
    const float th = acosf(uz);
    float ph = atan2f(-dy, -dx);
    if (ph < 0.f) ph += (float)(2.0 * M_PI);
    const float psi = h * inv;
    int it = (int)floorf(th * (float)(1.0 / M_PI) * P.nth);
    int ip = (int)floorf(ph * (float)(0.5 / M_PI) * P.nph);
    int is = (int)floorf((logf(psi) - P.psi_lmin) * P.psi_lscale);
    it = min(max(it, 0), P.nth - 1);
    ip = min(max(ip, 0), P.nph - 1);
    is = min(max(is, 0), P.nps - 1);
    const int ent = (it * P.nph + ip) * P.nps + is;
    const float f = m * P.inv_omega / d2;
    const int cnt = P.nr_cnt[ent];
    const float* wr = P.nr_w + (size_t)ent * P.kmax;
    const uint8_t* pr = P.nr_pix + (size_t)ent * P.kmax;
    for (int k = 0; k < cnt; ++k) map[(int)pr[k] * 32 + lane] += f * wr[k];
}

__global__ void __launch_bounds__(32 * TS_WALK_WARPS) k_column_walk(const __grid_constant__ ColParams P) {
    extern __shared__ float s_map[];   // [TS_WALK_WARPS][npix][32]
    __shared__ __align__(16) float4 s_com[TS_WALK_WARPS][8];
    __shared__ __align__(16) float4 s_cen[TS_WALK_WARPS][8];
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
    const int npix = P.npix;
    float* map = s_map + (size_t)warp * npix * 32;
    for (int p = 0; p < npix; ++p) map[p * 32 + lane] = 0.f;
    const int64_t me = gw * 32 + lane;
    const float4 mine = P.cell[me];
    const float rx = mine.x, ry = mine.y, rz = mine.z;
    const int ml = (int)(me & 511);
    const int q = ml >> 6, o = (ml >> 3) & 7, o2 = ml & 7;
    const int ci = 4 * (q & 1) + 2 * (o & 1) + (o2 & 1);
    const int cj = 4 * ((q >> 1) & 1) + 2 * ((o >> 1) & 1) + ((o2 >> 1) & 1);
    const int ck = 4 * (q >> 2) + 2 * (o >> 2) + (o2 >> 2);
    const int64_t nat = (me >> 9) * 512 + ck * 64 + cj * 8 + ci;
    const int px = P.geom->pbc[0], py = P.geom->pbc[1], pz = P.geom->pbc[2];
    const float Lx = (float)P.geom->L[0], Ly = (float)P.geom->L[1], Lz = (float)P.geom->L[2];
    const float iLx = (float)P.geom->invL[0], iLy = (float)P.geom->invL[1], iLz = (float)P.geom->invL[2];
    unsigned n_int = 0, n_mac = 0;

    int sp = 0;
    bool overflow = false;
    const float hroot = sqrtf(s_h2[0]);
    {   // the root is tested like any node (opened unless the target sees the whole domain small)
        const float4 c0 = P.ncom[0];
        const float4 g0 = P.ncen[0];
        float dx = rx - c0.x, dy = ry - c0.y, dz = rz - c0.z;
        if (px) dx -= Lx * rintf(dx * iLx);
        if (py) dy -= Ly * rintf(dy * iLy);
        if (pz) dz -= Lz * rintf(dz * iLz);
        float gx = rx - g0.x, gy = ry - g0.y, gz = rz - g0.z;
        if (px) gx -= Lx * rintf(gx * iLx);
        if (py) gy -= Ly * rintf(gy * iLy);
        if (pz) gz -= Lz * rintf(gz * iLz);
        const float d2 = dx * dx + dy * dy + dz * dz;
        const bool outside = fabsf(gx) > P.eta * s_half[0][0] || fabsf(gy) > P.eta * s_half[0][1] ||
                             fabsf(gz) > P.eta * s_half[0][2];
        const bool accept = outside && s_h2[0] < P.theta2 * d2;
        n_mac = 1;
        if (accept) {
            col_add(P, map, lane, c0.w, dx, dy, dz, d2, hroot);
            ++n_int;
        }
        const unsigned om = __ballot_sync(0xffffffffu, !accept);
        if (om) {
            if (lane == 0) s_stack[warp][0] = make_uint2(__float_as_uint(g0.w), om);
            sp = 1;
        }
    }
    __syncwarp();
    while (sp > 0 && !overflow) {
        const uint2 e = s_stack[warp][--sp];
        const uint32_t cw = e.x, mask = e.y;
        const int first = (int)(cw & TS_CW_INDEX_MASK);
        const bool cells = (cw & TS_CW_CELLS) != 0;
        const int dep = (int)(cw >> TS_CW_DEPTH_SHIFT);
        const bool active = (mask >> lane) & 1u;
        __syncwarp();
        if (cells) {
            if (lane < 8) s_com[warp][lane] = P.cell[first + lane];
        } else {
            if (lane < 8) s_com[warp][lane] = P.ncom[first + lane];
            else if (lane < 16) s_cen[warp][lane - 8] = P.ncen[first + lane - 8];
        }
        __syncwarp();
        const float hx = s_half[dep][0] * P.eta, hy = s_half[dep][1] * P.eta, hz = s_half[dep][2] * P.eta;
        const float h2 = s_h2[dep], h = sqrtf(h2);
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            const float4 c = s_com[warp][j];
            float dx = rx - c.x, dy = ry - c.y, dz = rz - c.z;
            if (px) dx -= Lx * rintf(dx * iLx);
            if (py) dy -= Ly * rintf(dy * iLy);
            if (pz) dz -= Lz * rintf(dz * iLz);
            const float d2 = dx * dx + dy * dy + dz * dz;
            bool accept, open = false;
            if (cells) {
                accept = active && (first + j != me);
            } else {
                const float4 g = s_cen[warp][j];
                float gx = rx - g.x, gy = ry - g.y, gz = rz - g.z;
                if (px) gx -= Lx * rintf(gx * iLx);
                if (py) gy -= Ly * rintf(gy * iLy);
                if (pz) gz -= Lz * rintf(gz * iLz);
                const bool outside = fabsf(gx) > hx || fabsf(gy) > hy || fabsf(gz) > hz;
                const bool mac = h2 < P.theta2 * d2;
                accept = active && outside && mac;
                open = active && !(outside && mac);
                n_mac += active;
            }
            if (accept) {
                col_add(P, map, lane, c.w, dx, dy, dz, d2, h);
                ++n_int;
            }
            if (!cells) {
                const unsigned om = __ballot_sync(0xffffffffu, open);
                if (om) {
                    if (sp >= TS_WALK_STACK) {
                        overflow = true;
                    } else {
                        if (lane == 0) s_stack[warp][sp] = make_uint2(__float_as_uint(s_cen[warp][j].w), om);
                        ++sp;
                    }
                }
            }
        }
        __syncwarp();
    }
    if (overflow && lane == 0) atomicOr(P.status, TS_DEV_STACK_OVERFLOW);
    // own cell: rho dx / 2 = m / (2 dy dz), cell edges dy = Ly_block / 8, dz = Lz_block / 8
    __syncwarp();
    const int64_t leaf = me >> 9;
    const float own = (float)((double)mine.w * 32.0 / (P.leaf_size[3 * leaf + 1] * P.leaf_size[3 * leaf + 2]));
    float* out = P.out + nat * npix;
    for (int p = 0; p < npix; ++p) out[p] = map[p * 32 + lane] + own;
    const unsigned wi = __reduce_add_sync(0xffffffffu, n_int), wm = __reduce_add_sync(0xffffffffu, n_mac);
    if (lane == 0) {
        atomicAdd(&P.counters[0], (unsigned long long)wi);
        atomicAdd(&P.counters[1], (unsigned long long)wm);
    }
}

cudaError_t launch_column_walk(ts_ctx* c, const ts_column_params* p, float* cols) {
    if (!c->d_geom) {
        cudaError_t e = cudaMalloc((void**)&c->d_geom, sizeof(WalkGeom));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(c->d_geom, &c->geom, sizeof(WalkGeom), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    ColParams P;
    memset(&P, 0, sizeof(P));
    P.ncom = c->d_ncom32;
    P.ncen = c->d_ncen32;
    P.cell = c->d_cell32;
    P.ncell = c->ncell;
    P.theta2 = (float)(p->theta * p->theta);
    P.eta = (float)p->safe_box;
    P.max_dist2 = p->max_dist > 0 ? (float)(p->max_dist * p->max_dist) : 0.f;
    P.geom = c->d_geom;
    P.npix = c->nr_dims[3];
    P.nth = c->nr_dims[0];
    P.nph = c->nr_dims[1];
    P.nps = c->nr_dims[2];
    P.kmax = c->nr_kmax;
    P.psi_lmin = (float)log(c->nr_psi[0]);
    P.psi_lscale = (float)(c->nr_dims[2] / log(c->nr_psi[1] / c->nr_psi[0]));
    P.inv_omega = (float)(P.npix / (4.0 * M_PI));
    P.leaf_size = c->d_leaf_size;
    P.nr_w = c->d_nr_w;
    P.nr_pix = c->d_nr_pix;
    P.nr_cnt = c->d_nr_cnt;
    P.out = cols;
    P.status = c->d_status;
    P.counters = c->d_counters;
    const size_t smem = sizeof(float) * (size_t)P.npix * 32 * TS_WALK_WARPS;
    e = cudaFuncSetAttribute(k_column_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nwarps = c->ncell / 32;
    const int grid = (int)((nwarps + TS_WALK_WARPS - 1) / TS_WALK_WARPS);
    cudaEventRecord(c->ev0, c->stream);
    k_column_walk<<<grid, 32 * TS_WALK_WARPS, smem, c->stream>>>(P);
    e = cudaGetLastError();
    cudaEventRecord(c->ev1, c->stream);
    c->timed = true;
    return e;
}
