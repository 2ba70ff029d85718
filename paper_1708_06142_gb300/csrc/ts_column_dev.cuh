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
    int npix, nth, nph, nps;
    uint32_t sb_depths;              // bit d: the safe-box test can change a MAC decision at depth d
    float psi_lmin, psi_lscale;      // log2(psi_min), nps / log2(psi_max / psi_min)
    float inv_omega;                 // 1 / Omega_pix = N_PIX / (4 pi), times 1 / nsub^3 (see nr_pairs)
    const double* leaf_size;
    // node-ray table: per entry one 16-byte record of up to 4 pairs (sub-cubes in the pixel << 8) |
    // pixel, the weight being that count over nsub^3; 0 marks an unused slot.  An entry with more
    // than 4 pairs keeps 3 in its record and, in slot 3, (offset << 8) | 255 into nr_more, which
    // holds the number of remaining pairs followed by them.
    const uint4* nr_rec;
    const uint32_t* nr_more;
    float* out;
    int* status;
    unsigned long long* counters;
    // extra mapped quantities (Sec. 2.3, l_q = 1 + nq maps): masses of up to 2 quantities per cell
    // (Morton order) and per internal node; maps and output rows are [l_q][npix]
    const float2* qcell;
    const float2* qnode;
};

// One accepted node (mass m and quantity masses mq, separation d = r - r_a, inv = 1/|d|): its bins
// and weight factors, and the load of its node-ray record, issued without waiting for it (a pop
// issues the loads of all its accepted children before the first scatter, so their L2 latencies
// overlap).  The table entry is one 16-byte record of up to four 4-byte (count, pixel) pairs (the
// N_PIX = 48 table is 0.5 MB; the rare longer rows continue in a second array).
#define COL_BATCH 2        // children whose record loads are in flight together (measured: 2 < 1, 4, 8)
#define COL_BATCH_CELLS 4  // the same for the cells of a leaf group, binned on every lane (4 < 2, 8)

// Direction angles of the bins.  theta = acos u_z and phi = atan2(y, x) come from polynomials, not
// from acosf / atan2f (which cost a quarter of the walk): least-squares fits at Chebyshev nodes on
// [0, 1] of acos x = sqrt(1 - x) Q(x) (Q of degree 6, |error| < 4.1e-7 rad evaluated in FP32) and of
// atan a = a R(a^2) (R of degree 7, |error| < 1.4e-7 rad), extended to [-1, 1] and to the four
// quadrants by the angle identities (pi - acos|u|; pi/2 - atan, pi - phi, 2 pi - phi), each adding
// one FP32 rounding (at most 6.2e-7 rad in all).  These errors are of the order of the FP32 library
// functions' own, and so is the rate of bin decisions that differ from those of the FP64 angles (a
// few per 10^6 directions).  Zero components follow the signed-zero conventions of atan2: phi = pi
// for x = -0, y = +-0 (the direction straight along z from a node, where phi is undefined), 0 for
// x = +0.
__device__ __forceinline__ float col_acos(float u) {
    const float x = fabsf(u), om = 1.f - x;
    const float q = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.0025606194976717234f, x, -0.01186282653361559f), x,
                                             0.027619101107120514f), x, -0.04913029447197914f), x,
                                   0.0888218879699707f), x, -0.21459004282951355f), x, 1.570796251296997f);
    const float a = q * (om * rsqrtf(fmaxf(om, 1e-30f)));   // sqrt(1 - x), 0 at x = 1
    return u < 0.f ? (float)M_PI - a : a;
}

__device__ __forceinline__ float col_phi(float y, float x) {   // atan2(y, x) wrapped to [0, 2 pi)
    const float ax = fabsf(x), ay = fabsf(y), mx = fmaxf(ax, ay);
    const float a = mx > 0.f ? __fdividef(fminf(ax, ay), mx) : 0.f;
    const float s = a * a;
    float p = a * fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-0.004073309246450663f, s, 0.021946610882878304f), s,
                                                -0.056063175201416016f), s, 0.09656256437301636f), s,
                                      -0.13915802538394928f), s, 0.19948509335517883f), s,
                            -0.3333010673522949f), s, 0.999999463558197f);
    if (ay > ax) p = (float)(0.5 * M_PI) - p;
    if (signbit(x)) p = (float)M_PI - p;
    if (y < 0.f) p = (float)(2.0 * M_PI) - p;
    return p;
}

template <int NQ>
struct ColHit {
    uint4 rec;
    float f, f1, f2;
};

// Bins and weight factors of one node for this lane; a lane that does not take the node (acc false:
// outside the popped entry's mask, its own cell, or beyond max_dist) gets weight factors 0, so its
// scatter adds zeros and leaves its map unchanged.  Leaf-cell groups are binned and scattered by
// every lane of the warp that way, with no per-lane branch (measured 4.7 % faster than branching).
// The bin indices stay in range for any separation (a zero one gives u_z = -1 and an infinite psi,
// both clamped).
template <int NQ>
__device__ __forceinline__ void col_bin(const ColParams& P, bool acc, float m, float2 mq, float dx, float dy, float dz,
                                        float d2, float inv, float h, ColHit<NQ>& hit) {
    acc = acc && !(P.max_dist2 > 0.f && d2 > P.max_dist2);
    // direction from the target to the node is -d
    const float uz = fminf(1.f, fmaxf(-1.f, -dz * inv));
    const float th = col_acos(uz);
    const float ph = col_phi(-dy, -dx);
    const float psi = h * inv;
    int it = (int)floorf(th * (float)(1.0 / M_PI) * P.nth);
    int ip = (int)floorf(ph * (float)(0.5 / M_PI) * P.nph);
    int is = (int)floorf((__log2f(psi) - P.psi_lmin) * P.psi_lscale);
    it = min(max(it, 0), P.nth - 1);
    ip = min(max(ip, 0), P.nph - 1);
    is = min(max(is, 0), P.nps - 1);
    const int ent = (it * P.nph + ip) * P.nps + is;
    const float g = P.inv_omega * inv * inv;
    hit.f = acc ? m * g : 0.f;
    if constexpr (NQ >= 1) hit.f1 = acc ? mq.x * g : 0.f;
    if constexpr (NQ >= 2) hit.f2 = acc ? mq.y * g : 0.f;
    hit.rec = __ldg(P.nr_rec + ent);
}

// Scatter of one node into this lane's pixel map and its quantity masses into the following maps
// (map stride npix * 32).  The four slots of the record are added without a test: an unused slot
// adds 0 to pixel 0, which leaves the sums unchanged and keeps the lanes of a warp on one path
// (measured 6 % faster than skipping the empty slots).
template <int NQ>
__device__ __forceinline__ void col_scatter(const ColParams& P, float* map, int lane, const ColHit<NQ>& hit) {
    const int ms = P.npix * 32;
    auto add = [&](uint32_t v) {
        const int p = (int)(v & 255u) * 32 + lane;
        const float w = (float)(v >> 8);
        map[p] += hit.f * w;
        if constexpr (NQ >= 1) map[ms + p] += hit.f1 * w;
        if constexpr (NQ >= 2) map[2 * ms + p] += hit.f2 * w;
    };
    const uint4 rec = hit.rec;
    add(rec.x);   // every entry has at least one pixel; an unused slot (0) adds 0 to pixel 0
    add(rec.y);
    add(rec.z);
    if ((rec.w & 255u) == 255u) {   // a longer row continues in nr_more
        const uint32_t* more = P.nr_more + (rec.w >> 8);
        const int n = (int)__ldg(more);
        for (int k = 1; k <= n; ++k) add(__ldg(more + k));
    } else {
        add(rec.w);
    }
}

// One warp's column walk: warp gw of the grid described by P (32 Morton-consecutive targets), the
// same shared depth-first traversal as the gravity walk: a stack entry is the child word of an
// opened node and the mask of the lanes that opened it; a pop stages the 8 children in shared
// memory, each lane applies the BH MAC (with the safe box, evaluated once per group as an 8-bit
// mask) to each child, and the children opened by any lane are pushed in one compacted write.
// map: this warp's [1 + NQ][npix][32] pixel maps in shared memory; s_q_w: staging of the children's
// quantity masses (NQ > 0).
template <int NQ = 0>
__device__ __forceinline__ void col_walk_warp(const ColParams& P, int64_t gw, int lane, float* map, float4* s_com_w,
                                              float4* s_cen_w, uint2* s_stack_w, const float (*s_half)[3],
                                              const float* s_h2, float2* s_q_w = nullptr) {
    const int npix = P.npix;
    for (int p = 0; p < (1 + NQ) * npix; ++p) map[p * 32 + lane] = 0.f;
    const float2 zq = make_float2(0.f, 0.f);
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
    auto mi = [](float d, int per, float L, float iL) { return per ? d - L * rintf(d * iL) : d; };

    int sp = 0;
    bool overflow = false;
    {   // the root is tested like any node (opened unless the target sees the whole domain small)
        const float4 c0 = P.ncom[0];
        const float4 g0 = P.ncen[0];
        const float dx = mi(rx - c0.x, px, Lx, iLx), dy = mi(ry - c0.y, py, Ly, iLy), dz = mi(rz - c0.z, pz, Lz, iLz);
        const float gx = mi(rx - g0.x, px, Lx, iLx), gy = mi(ry - g0.y, py, Ly, iLy), gz = mi(rz - g0.z, pz, Lz, iLz);
        const float d2 = dx * dx + dy * dy + dz * dz;
        const bool outside = fabsf(gx) > P.eta * s_half[0][0] || fabsf(gy) > P.eta * s_half[0][1] ||
                             fabsf(gz) > P.eta * s_half[0][2];
        const bool accept = outside && s_h2[0] < P.theta2 * d2;
        n_mac = 1;
        if (accept) {
            ColHit<NQ> hit;
            col_bin<NQ>(P, true, c0.w, NQ ? P.qnode[0] : zq, dx, dy, dz, d2, rsqrtf(d2), sqrtf(s_h2[0]), hit);
            col_scatter<NQ>(P, map, lane, hit);
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
        const int dep = (int)(cw >> TS_CW_DEPTH_SHIFT);
        const bool active = (mask >> lane) & 1u;
        __syncwarp();
        if (cw & TS_CW_CELLS) {
            // ---- 8 leaf cells: every active target accepts all of them except its own cell
            if (lane < 8) s_com_w[lane] = P.cell[first + lane];
            if constexpr (NQ > 0) if (lane >= 16 && lane < 24) s_q_w[lane - 16] = P.qcell[first + lane - 16];
            __syncwarp();
            const float h = sqrtf(s_h2[dep]);
            // per half of the group: bins and record loads of its 4 cells first, then the scatters
#pragma unroll 1
            for (int j0 = 0; j0 < 8; j0 += COL_BATCH_CELLS) {
                ColHit<NQ> hit[COL_BATCH_CELLS];
#pragma unroll
                for (int u = 0; u < COL_BATCH_CELLS; ++u) {
                    const int j = j0 + u;
                    const float4 c = s_com_w[j];
                    const float dx = mi(rx - c.x, px, Lx, iLx), dy = mi(ry - c.y, py, Ly, iLy),
                                dz = mi(rz - c.z, pz, Lz, iLz);
                    const bool acc = active && first + j != me;
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    col_bin<NQ>(P, acc, c.w, NQ ? s_q_w[j] : zq, dx, dy, dz, d2, rsqrtf(d2), h, hit[u]);
                    n_int += acc ? 1u : 0u;
                }
#pragma unroll
                for (int u = 0; u < COL_BATCH_CELLS; ++u) col_scatter<NQ>(P, map, lane, hit[u]);
            }
        } else {
            // ---- 8 internal nodes
            if (lane < 8) s_com_w[lane] = P.ncom[first + lane];
            else if (lane < 16) s_cen_w[lane - 8] = P.ncen[first + lane - 8];
            else if (NQ > 0 && lane < 24) s_q_w[lane - 16] = P.qnode[first + lane - 16];
            __syncwarp();
            const float hx = s_half[dep][0], hy = s_half[dep][1], hz = s_half[dep][2];
            const float h2 = s_h2[dep], h = sqrtf(h2);
            // safe box once per group (children centres at c0 + 2 h (ox, oy, oz)); skipped where no
            // target inside it can pass the MAC
            unsigned inside = 0u;
            if ((P.sb_depths >> dep) & 1u) {
                const float4 g0 = s_cen_w[0];
                const float qx = rx - g0.x, qy = ry - g0.y, qz = rz - g0.z;
                const float ex = P.eta * hx, ey = P.eta * hy, ez = P.eta * hz;
                const bool x0 = fabsf(mi(qx, px, Lx, iLx)) <= ex, x1 = fabsf(mi(qx - 2 * hx, px, Lx, iLx)) <= ex;
                const bool y0 = fabsf(mi(qy, py, Ly, iLy)) <= ey, y1 = fabsf(mi(qy - 2 * hy, py, Ly, iLy)) <= ey;
                const bool z0 = fabsf(mi(qz, pz, Lz, iLz)) <= ez, z1 = fabsf(mi(qz - 2 * hz, pz, Lz, iLz)) <= ez;
                inside = ((x0 ? 0x55u : 0u) | (x1 ? 0xAAu : 0u)) & ((y0 ? 0x33u : 0u) | (y1 ? 0xCCu : 0u)) &
                         ((z0 ? 0x0Fu : 0u) | (z1 ? 0xF0u : 0u));
            }
            n_mac += active ? 8u : 0u;
            // per COL_BATCH children: MAC, bins and record loads first, then the scatters
#pragma unroll 1
            for (int j0 = 0; j0 < 8; j0 += COL_BATCH) {
                ColHit<NQ> hit[COL_BATCH];
                uint32_t am = 0u;
#pragma unroll
                for (int u = 0; u < COL_BATCH; ++u) {
                    const int j = j0 + u;
                    const float4 c = s_com_w[j];
                    const float dx = mi(rx - c.x, px, Lx, iLx), dy = mi(ry - c.y, py, Ly, iLy),
                                dz = mi(rz - c.z, pz, Lz, iLz);
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    const bool ok = h2 < P.theta2 * d2 && !((inside >> j) & 1u);
                    const unsigned om = __ballot_sync(0xffffffffu, active && !ok);
                    if (lane == 0) s_stack_w[TS_WALK_STACK - 8 + j].y = om;   // parked above the stack top
                    if (active && ok) {
                        col_bin<NQ>(P, true, c.w, NQ ? s_q_w[j] : zq, dx, dy, dz, d2, rsqrtf(d2), h, hit[u]);
                        am |= 1u << u;
                        ++n_int;
                    }
                }
#pragma unroll
                for (int u = 0; u < COL_BATCH; ++u)
                    if ((am >> u) & 1u) col_scatter<NQ>(P, map, lane, hit[u]);
            }
            __syncwarp();
            // push the opened children in one compacted write: lane j < 8 owns child j
            const uint32_t my_om = lane < 8 ? s_stack_w[TS_WALK_STACK - 8 + lane].y : 0u;
            const unsigned nz = __ballot_sync(0xffffffffu, my_om != 0u);
            const int npush = __popc(nz);
            if (sp + npush > TS_WALK_STACK - 8) {   // the top 8 slots park the open masks
                overflow = true;
            } else {
                if (my_om) s_stack_w[sp + __popc(nz & ((1u << lane) - 1u))] =
                    make_uint2(__float_as_uint(s_cen_w[lane].w), my_om);
                sp += npush;
            }
        }
        __syncwarp();
    }
    if (overflow && lane == 0) atomicOr(P.status, TS_DEV_STACK_OVERFLOW);
    // own cell: rho dx / 2 = m / (2 dy dz), cell edges dy = Ly_block / 8, dz = Lz_block / 8
    __syncwarp();
    const int64_t leaf = me >> 9;
    const double own_f = 32.0 / (P.leaf_size[3 * leaf + 1] * P.leaf_size[3 * leaf + 2]);
    float* out = P.out + nat * (1 + NQ) * npix;
#pragma unroll
    for (int k = 0; k <= NQ; ++k) {
        const float mk = k == 0 ? mine.w : (k == 1 ? P.qcell[me].x : P.qcell[me].y);
        const float own = (float)((double)mk * own_f);
        for (int p = 0; p < npix; ++p) out[k * npix + p] = map[(k * npix + p) * 32 + lane] + own;
    }
    const unsigned wi = __reduce_add_sync(0xffffffffu, n_int), wm = __reduce_add_sync(0xffffffffu, n_mac);
    if (lane == 0) {
        atomicAdd(&P.counters[0], (unsigned long long)wi);
        atomicAdd(&P.counters[1], (unsigned long long)wm);
    }
}
