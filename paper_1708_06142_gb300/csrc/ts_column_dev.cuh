// Device code of the column-density walk shared by k_column_walk (ts_column.cu) and the batched
// persistent kernel (ts_batch.cu).  See ts_column.cu for the design.
#pragma once
#include <math.h>

#include "ts_internal.cuh"

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

// One warp's column walk: warp gw of the grid described by P (32 Morton-consecutive targets).
// map: this warp's [npix][32] pixel maps in shared memory.
__device__ __forceinline__ void col_walk_warp(const ColParams& P, int64_t gw, int lane, float* map, float4* s_com_w,
                                              float4* s_cen_w, uint2* s_stack_w, const float (*s_half)[3],
                                              const float* s_h2) {
    const int npix = P.npix;
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
            if (lane == 0) s_stack_w[0] = make_uint2(__float_as_uint(g0.w), om);
            sp = 1;
        }
    }
    __syncwarp();
    while (sp > 0 && !overflow) {
        const uint2 e = s_stack_w[--sp];
        const uint32_t cw = e.x, mask = e.y;
        const int first = (int)(cw & TS_CW_INDEX_MASK);
        const bool cells = (cw & TS_CW_CELLS) != 0;
        const int dep = (int)(cw >> TS_CW_DEPTH_SHIFT);
        const bool active = (mask >> lane) & 1u;
        __syncwarp();
        if (cells) {
            if (lane < 8) s_com_w[lane] = P.cell[first + lane];
        } else {
            if (lane < 8) s_com_w[lane] = P.ncom[first + lane];
            else if (lane < 16) s_cen_w[lane - 8] = P.ncen[first + lane - 8];
        }
        __syncwarp();
        const float hx = s_half[dep][0] * P.eta, hy = s_half[dep][1] * P.eta, hz = s_half[dep][2] * P.eta;
        const float h2 = s_h2[dep], h = sqrtf(h2);
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            const float4 c = s_com_w[j];
            float dx = rx - c.x, dy = ry - c.y, dz = rz - c.z;
            if (px) dx -= Lx * rintf(dx * iLx);
            if (py) dy -= Ly * rintf(dy * iLy);
            if (pz) dz -= Lz * rintf(dz * iLz);
            const float d2 = dx * dx + dy * dy + dz * dz;
            bool accept, open = false;
            if (cells) {
                accept = active && (first + j != me);
            } else {
                const float4 g = s_cen_w[j];
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
                        if (lane == 0) s_stack_w[sp] = make_uint2(__float_as_uint(s_cen_w[j].w), om);
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

