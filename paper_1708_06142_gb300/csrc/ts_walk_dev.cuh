// Device code of the gravity walk shared by the single-grid kernels (ts_walk.cu) and the batched
// persistent kernel (ts_batch.cu).  See ts_walk.cu for the design.
#pragma once
#include <math.h>
#include <string.h>

#include <algorithm>

#include <cuda_fp16.h>

#include "ts_internal.cuh"
#include "ts_mlp.cuh"

// Per-warp row buffers of the learned-correction mode (one pop: up to 8 children x 32 lanes).
#define MLP_ROWS 256
#define MLP_FWD_BF16 MLP_OFF_W2T            // forward weights W1p..W4p are the image's prefix
#define MLP_SMEM_WEIGHTS (MLP_FWD_BF16 * 2 + MLP_NF32 * 4)
#define MLP_SMEM_WARP (MLP_ROWS * (16 + 16 + 16))

template <typename R>
struct RT;
template <>
struct RT<float> {
    typedef float4 V4;
};
template <>
struct RT<double> {
    typedef dbl4 V4;
};

struct WalkParams {
    const void* ncom;
    const void* ncen;
    const void* cell;
    const float4* cell_soa;   // FP32 walk: sibling groups, structure of arrays (see ts_ctx)
    const float4* ncom_soa;
    int64_t ncell;
    uint32_t root_cw;
    uint32_t sb_depths;   // bit d: the safe-box test can change a MAC decision for nodes at depth d
    double theta2, eta, a_lim, G, eps_rel;
    const float* a_old;
    const WalkGeom* geom;
    const void* bmom;     // MPE MAC: (B2, B3) per internal node, float2 or double2 by precision
    // subsets of targets (Adaptive Block Update, one target per lane):
    //   targets != NULL: lane l of warp w walks for Morton cell targets[32 w + l] and writes its
    //                    results at index 32 w + l of pot/acc (ntargets a multiple of 32)
    //   warp_list != NULL: warp w walks the 32 cells of warp_list[w] and writes them in place;
    //                    *nwarp_dev warps are valid (the grid may be larger)
    const int64_t* targets;
    int64_t ntargets;
    const int* warp_list;
    const int* nwarp_dev;
    // full walks: the leaf-blocks [leaf_begin, leaf_end) whose cells are walked (all of them, or one
    // rank's range of a partitioned mesh)
    int64_t leaf_begin, leaf_end;
    unsigned long long* blk_counts;   // nullable: interactions per leaf-block (warp-list and full walks)
    EwaldDev ew;
    void* pot;
    void* acc;
    int* status;
    unsigned long long* counters;
    // learned-correction mode (2P1I): feature scales 4/Lx, 4/Ly, 2/F_net, the constant aspect feature,
    // and the unit conversion of the network outputs (1/Lx for C, 1/Lx^2 for A_c)
    const void* mlp_img;
    float mlp_sx, mlp_sy, mlp_sz, mlp_f3, mlp_c, mlp_a;
};

__device__ __forceinline__ float rint_t(float x) { return rintf(x); }
__device__ __forceinline__ double rint_t(double x) { return rint(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// ---- paired FP32 arithmetic (isolated FP32 walk, one target per lane): two children per
// instruction with the packed f32x2 add/mul/fma of sm_100+, halving the issue slots of the
// interaction arithmetic.  Children come as a sibling group stored structure-of-arrays (x[8],
// y[8], z[8], m[8]: 8 float4 that every lane of the warp reads at the same address).  Separations
// are taken as c - r (the negated d of eqs. pot and accel, exact), so accelerations accumulate
// with a plus sign.

// children j0 = 4 q + 2 h and j0 + 1 from the quads of the group
__device__ __forceinline__ void pk_pair(const float4& X, const float4& Y, const float4& Z, const float4& M, int h,
                                        float2& cx, float2& cy, float2& cz, float2& m) {
    cx = h ? make_float2(X.z, X.w) : make_float2(X.x, X.y);
    cy = h ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y);
    cz = h ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y);
    m = h ? make_float2(M.z, M.w) : make_float2(M.x, M.y);
}

__device__ __forceinline__ void pk_sep(float2 cx, float2 cy, float2 cz, float2 nrx, float2 nry, float2 nrz, float2& dx,
                                       float2& dy, float2& dz, float2& d2) {
    dx = __fadd2_rn(cx, nrx);
    dy = __fadd2_rn(cy, nry);
    dz = __fadd2_rn(cz, nrz);
    d2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
}

// sums of m/|d| and m (c - r)/|d|^3 over the accepted children of the pair
__device__ __forceinline__ void pk_interact(float2 dx, float2 dy, float2 dz, float2 d2, float2 m, bool a0, bool a1,
                                            float2& sp, float2& sx, float2& sy, float2& sz) {
    d2.x = a0 ? d2.x : 1.f;
    d2.y = a1 ? d2.y : 1.f;
    m.x = a0 ? m.x : 0.f;
    m.y = a1 ? m.y : 0.f;
    const float2 inv = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
    const float2 mi = __fmul2_rn(m, inv);
    sp = __fadd2_rn(sp, mi);
    const float2 g3 = __fmul2_rn(mi, __fmul2_rn(inv, inv));
    sx = __ffma2_rn(g3, dx, sx);
    sy = __ffma2_rn(g3, dy, sy);
    sz = __ffma2_rn(g3, dz, sz);
}

// the same sums with a rejected child's d2 replaced by +inf: rsqrt(+inf) = 0, so it adds exactly 0
// (its d2 may be 0: the target's own cell, or a node centred on the target)
__device__ __forceinline__ void pk_interact_m(float2 dx, float2 dy, float2 dz, float2 d2, float2 m, bool a0, bool a1,
                                              float2& sp, float2& sx, float2& sy, float2& sz) {
    d2.x = a0 ? d2.x : __int_as_float(0x7f800000);   // +inf: rsqrt gives 0, the child adds nothing
    d2.y = a1 ? d2.y : __int_as_float(0x7f800000);
    const float2 inv = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
    const float2 mi = __fmul2_rn(m, inv);
    sp = __fadd2_rn(sp, mi);
    const float2 g3 = __fmul2_rn(mi, __fmul2_rn(inv, inv));
    sx = __ffma2_rn(g3, dx, sx);
    sy = __ffma2_rn(g3, dy, sy);
    sz = __ffma2_rn(g3, dz, sz);
}

// the same with 1/|d| already formed (MPE: the MAC needs it); a rejected child's inv may be
// infinite (d2 = 0), so its mass is masked and its inv replaced
__device__ __forceinline__ void pk_interact_inv(float2 dx, float2 dy, float2 dz, float2 inv, float2 m, bool a0, bool a1,
                                                float2& sp, float2& sx, float2& sy, float2& sz) {
    m.x = a0 ? m.x : 0.f;
    m.y = a1 ? m.y : 0.f;
    inv.x = a0 ? inv.x : 0.f;
    inv.y = a1 ? inv.y : 0.f;
    const float2 mi = __fmul2_rn(m, inv);
    sp = __fadd2_rn(sp, mi);
    const float2 g3 = __fmul2_rn(mi, __fmul2_rn(inv, inv));
    sx = __ffma2_rn(g3, dx, sx);
    sy = __ffma2_rn(g3, dy, sy);
    sz = __ffma2_rn(g3, dz, sz);
}

// compensated (Kahan) addition of two sums at once; a - b is formed as fma(b, -1, a), which rounds
// once like the subtraction
__device__ __forceinline__ void kahan_add2(float2& s, float2& c, float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 y = __ffma2_rn(c, m1, x);
    const float2 t = __fadd2_rn(s, y);
    c = __ffma2_rn(y, m1, __ffma2_rn(s, m1, t));
    s = t;
}

// phi(d) and A(d) = -grad phi of one unit mass under periodic/mixed BCs: 1/|d| + C(d) and
// d/|d|^3 + A_c(d) from the folded correction table, or the far-field form beyond E.far.
// EWM: 0 trilinear only, 1 Taylor only, 2 chosen at run time by E.taylor (kernels serving both).
template <typename R, int EWM>
__device__ __forceinline__ void ewald_pair(const EwaldDev& E, R dx, R dy, R dz, R inv, R& phi, R& Ax, R& Ay, R& Az) {
    typedef typename RT<R>::V4 V4;
    const R ax = fabs(dx), ay = fabs(dy), az = fabs(dz);
    if (E.kind == TS_EW_2P1I && az > (R)E.far) {
        phi = (R)E.far_const - (R)E.far_slope * az;
        Ax = 0; Ay = 0; Az = copysign((R)E.far_slope, dz);
        return;
    }
    if (E.kind == TS_EW_1P2I) {
        const R r2 = dy * dy + dz * dz;
        if (r2 > (R)(E.far * E.far)) {
            const R lx = (R)E.far_lx;
            phi = (R)E.far_const - (R)(2.0 / E.far_lx) * log_t((R)(2.0 * M_PI) * sqrt(r2) / lx);
            Ax = 0; Ay = (R)2 * dy / (lx * r2); Az = (R)2 * dz / (lx * r2);
            return;
        }
    }
    const int n = E.n;
    if (EWM == 1 || (EWM == 2 && E.taylor)) {
        // first-order Taylor expansion about the nearest grid point g (Sec. 2.2.5, approach 2):
        // C(u) = C(g) - A_c(g).(u - g),  A_c(u) = A_c(g) + J(g) (u - g).  The FP64 kernels pick g
        // by dividing by the spacing (the same rounding as a host computation); FP32 multiplies.
        R gi[3];
        if constexpr (sizeof(R) == 8) {
            gi[0] = floor(ax / E.h[0] + 0.5); gi[1] = floor(ay / E.h[1] + 0.5); gi[2] = floor(az / E.h[2] + 0.5);
        } else {
            gi[0] = floorf(ax * (float)E.inv_dx[0] + 0.5f); gi[1] = floorf(ay * (float)E.inv_dx[1] + 0.5f);
            gi[2] = floorf(az * (float)E.inv_dx[2] + 0.5f);
        }
        const int g0 = min((int)gi[0], n - 1), g1 = min((int)gi[1], n - 1), g2 = min((int)gi[2], n - 1);
        const R ux = ax - (R)g0 * (R)E.h[0], uy = ay - (R)g1 * (R)E.h[1], uz = az - (R)g2 * (R)E.h[2];
        R c, tx, ty, tz;
        if constexpr (sizeof(R) == 4) {
            // one 32-byte record (one L1 sector): (C, A_c), then the Jacobian as FP16 pairs of J / s
            // (Jxx, Jyy), (Jzz, Jxy), (Jxz, Jyz) and s; the displacement is scaled by s instead
            const float4* rec = (const float4*)E.tay32 + 2 * (((size_t)g0 * n + g1) * n + g2);
            const float4 v = __ldg(rec);
            const uint4 q = __ldg((const uint4*)rec + 1);
            const float s = __uint_as_float(q.w);
            const float2 a = __half22float2(*(const __half2*)&q.x), b = __half22float2(*(const __half2*)&q.y),
                         d = __half22float2(*(const __half2*)&q.z);
            const float sx = s * ux, sy = s * uy, sz = s * uz;
            c = v.x - (v.y * ux + v.z * uy + v.w * uz);
            tx = v.y + a.x * sx + b.y * sy + d.x * sz;
            ty = v.z + b.y * sx + a.y * sy + d.y * sz;
            tz = v.w + d.x * sx + d.y * sy + b.x * sz;
        } else {   // (C, A_c), (Jxx, Jyy, Jzz, Jxy), (Jxz, Jyz, -, -) in FP64
            const V4* rec = (const V4*)E.tay64 + 4 * (((size_t)g0 * n + g1) * n + g2);
            const V4 v = rec[0], j1 = rec[1], j2 = rec[2];
            c = v.x - (v.y * ux + v.z * uy + v.w * uz);
            tx = v.y + j1.x * ux + j1.w * uy + j2.x * uz;
            ty = v.z + j1.w * ux + j1.y * uy + j2.y * uz;
            tz = v.w + j2.x * ux + j2.y * uy + j1.z * uz;
        }
        const R inv3 = inv * inv * inv;
        phi = inv + c;
        Ax = dx * inv3 + (dx < (R)0 ? -tx : tx);
        Ay = dy * inv3 + (dy < (R)0 ? -ty : ty);
        Az = dz * inv3 + (dz < (R)0 ? -tz : tz);
        return;
    }
    R u[3] = {ax * (R)E.inv_dx[0], ay * (R)E.inv_dx[1], az * (R)E.inv_dx[2]};
    int i0[3];
    R f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R v = fmin(u[a], (R)(n - 1));
        int i = min((int)v, n - 2);
        i0[a] = i;
        f[a] = v - (R)i;
    }
    const V4* tab;
    if constexpr (sizeof(R) == 4) tab = (const V4*)E.tab32; else tab = (const V4*)E.tab64;
    R c = 0, cx = 0, cy = 0, cz = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
        const R w = (ox ? f[0] : (R)1 - f[0]) * (oy ? f[1] : (R)1 - f[1]) * (oz ? f[2] : (R)1 - f[2]);
        const V4 v = tab[((size_t)(i0[0] + ox) * n + (i0[1] + oy)) * n + (i0[2] + oz)];
        c += w * v.x; cx += w * v.y; cy += w * v.z; cz += w * v.w;
    }
    const R inv3 = inv * inv * inv;
    phi = inv + c;
    // A_c is odd in its own axis and even in the others: restore the sign of the folded value
    Ax = dx * inv3 + (dx < (R)0 ? -cx : cx);
    Ay = dy * inv3 + (dy < (R)0 ? -cy : cy);
    Az = dz * inv3 + (dz < (R)0 ? -cz : cz);
}

// Minimum image along one axis (periodic axes only).
template <typename R, int BCK>
__device__ __forceinline__ R mimg(R d, int per, R L, R iL) {
    if (BCK && per) d -= L * rint_t(d * iL);
    return d;
}

// One warp's walk: warp gw of the grid described by P (T targets per lane: lane l holds the cells
// 32 T gw + 32 t + l, t < T, Morton order, i.e. T stacked 4x4x2 bricks of one leaf-block).  A stack
// entry is the child word of an opened node and T lane masks (bit l of mask t: target t of lane l
// opened it).  Shared memory: this warp's staging slots (generic kernels; the paired FP32 kernel
// stages only MPE moments), stack and masks, the depth geometry, and (learned-correction mode) the
// network weights and this warp's row buffers.  POT: potential only (Sec. 2.2.2, eq. pot; the
// acceleration is then obtained by numerical differentiation of the potential): the acceleration
// sums are not formed and acc is not written.
template <typename R, int BCK, int MAC, bool REL, int T, int EWM = 2, bool POT = false>
__device__ __forceinline__ void walk_warp(const WalkParams& P, int64_t gw, int warp, int lane,
                                          typename RT<R>::V4* s_com_w, typename RT<R>::V4* s_cen_w,
                                          uint32_t* s_cw_w, uint32_t (*s_mask_w)[T], const R (*s_half)[3],
                                          const R* s_h2, unsigned char* s_dyn,
                                          typename RT<R>::V4* s_bm_w = nullptr) {
    typedef typename RT<R>::V4 V4;
    const V4* ncom = (const V4*)P.ncom;
    const bool ewk = P.ew.kind != TS_EW_NONE;   // periodic or mixed BCs (runtime, per grid)
    const V4* ncen = (const V4*)P.ncen;
    const V4* cell = (const V4*)P.cell;
    const int64_t base = gw * 32 * T;             // first Morton cell id of this warp
    // the paired FP32 path: isolated FP32 walk with one target per lane (see below)
    constexpr bool PK = sizeof(R) == 4 && BCK == 0 && T == 1;
    // unrolling of the per-child loops of the scalar path: with the correction-table lookup inlined
    // into both, a 4-way unroll keeps the kernel body small enough for the instruction cache
    // (measured on the 3P 128^3 box: Taylor 28.6 -> 24.6 ms, trilinear 67.0 -> 58.4 ms)
    constexpr int CHILD_UNROLL = BCK == 1 ? 4 : 8;

    R rx[T], ry[T], rz[T], alim[T];
    int64_t nat[T], mcell[T];
    R phi[T], ax[T], ay[T], az[T], cphi[T], cax[T], cay[T], caz[T];
    const R theta2 = (R)P.theta2, eta = (R)P.eta, G = (R)P.G;
    const int px = P.geom->pbc[0], py = P.geom->pbc[1], pz = P.geom->pbc[2];
    const R Lx = (R)P.geom->L[0], Ly = (R)P.geom->L[1], Lz = (R)P.geom->L[2];
    const R iLx = (R)P.geom->invL[0], iLy = (R)P.geom->invL[1], iLz = (R)P.geom->invL[2];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t me = P.targets ? P.targets[gw * 32 + lane] : base + 32 * t + lane;
        mcell[t] = me;
        if constexpr (PK) {   // the paired walk reads only the sibling-group copy of the cells
            const float* g = (const float*)(P.cell_soa + 8 * (me >> 3));
            const int j = (int)(me & 7);
            rx[t] = g[j]; ry[t] = g[8 + j]; rz[t] = g[16 + j];
        } else {
            const V4 mine = cell[me];
            rx[t] = mine.x; ry[t] = mine.y; rz[t] = mine.z;
        }
        const int ml = (int)(me & 511);
        const int q = ml >> 6, o = (ml >> 3) & 7, o2 = ml & 7;
        const int ci = 4 * (q & 1) + 2 * (o & 1) + (o2 & 1);
        const int cj = 4 * ((q >> 1) & 1) + 2 * ((o >> 1) & 1) + ((o2 >> 1) & 1);
        const int ck = 4 * (q >> 2) + 2 * (o >> 2) + (o2 >> 2);
        nat[t] = (me >> 9) * 512 + ck * 64 + cj * 8 + ci;
        alim[t] = REL ? (R)P.eps_rel * (R)P.a_old[nat[t]] : (R)P.a_lim;
        phi[t] = ax[t] = ay[t] = az[t] = 0;
        cphi[t] = cax[t] = cay[t] = caz[t] = 0;
    }
    unsigned n_int = 0, n_mac = 0, n_pop = 0, n_lanes = 0;   // n_pop, n_lanes: warp-uniform
    unsigned n_int_w = 0, n_mac_w = 0;                        // warp-uniform counts (paired path)
    unsigned root_lanes = 0;                                  // lanes of the root's stack entry
    // The paired path's sums run without G and with the sign of c - r: (sum m/|d|, sum m (c - r)_x/|d|^3) and the y, z pair, compensated in
    // pairs; phi and a are formed from them once at the end.
    float2 k01 = make_float2(0.f, 0.f), k23 = k01, c01 = k01, c23 = k01;
    float2 nrx = make_float2(0.f, 0.f), nry = nrx, nrz = nrx;
    const float ith2 = PK ? (float)(1.0 / P.theta2) : 0.f;
    if constexpr (PK) {
        nrx = make_float2(-(float)rx[0], -(float)rx[0]);
        nry = make_float2(-(float)ry[0], -(float)ry[0]);
        nrz = make_float2(-(float)rz[0], -(float)rz[0]);
    }

    // the root is tested like any node (it is opened unless a target accepts the whole domain)
    int sp = 0;
    bool overflow = false;
    {
        const V4 c0 = ncom[0];
        const V4 g0 = ncen[0];
        bool any_open = false;
        uint32_t rm[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const R dx = mimg<R, BCK>(rx[t] - c0.x, px, Lx, iLx), dy = mimg<R, BCK>(ry[t] - c0.y, py, Ly, iLy),
                    dz = mimg<R, BCK>(rz[t] - c0.z, pz, Lz, iLz);
            const R gx = mimg<R, BCK>(rx[t] - g0.x, px, Lx, iLx), gy = mimg<R, BCK>(ry[t] - g0.y, py, Ly, iLy),
                    gz = mimg<R, BCK>(rz[t] - g0.z, pz, Lz, iLz);
            const R d2 = dx * dx + dy * dy + dz * dz;
            const bool outside = fabs(gx) > eta * s_half[0][0] || fabs(gy) > eta * s_half[0][1] ||
                                 fabs(gz) > eta * s_half[0][2];
            // (MPE: the target lies inside the root, closer than its furthest point: always opened)
            const bool mac = MAC == TS_MAC_BH    ? s_h2[0] < theta2 * d2
                             : MAC == TS_MAC_APE ? G * c0.w * s_h2[0] < alim[t] * d2 * d2
                                                 : false;
            // learned-correction mode: the root is always opened (the target lies inside it)
            const bool accept = BCK != 2 && outside && mac;
            ++n_mac;
            if (accept) {
                const R inv = rsqrt_t(d2);
                R pf = inv, Axx = dx * inv * inv * inv, Ayy = dy * inv * inv * inv, Azz = dz * inv * inv * inv;
                if (BCK == 1 && ewk) ewald_pair<R, EWM>(P.ew, dx, dy, dz, inv, pf, Axx, Ayy, Azz);
                phi[t] -= G * c0.w * pf; ax[t] -= G * c0.w * Axx; ay[t] -= G * c0.w * Ayy; az[t] -= G * c0.w * Azz;
                ++n_int;
            }
            rm[t] = __ballot_sync(0xffffffffu, !accept);
            any_open |= rm[t] != 0u;
            if (t == 0) root_lanes = (unsigned)__popc(rm[0]);
        }
        if (any_open) {
            if (lane == 0) {
                uint32_t cw;
                if constexpr (sizeof(R) == 4) cw = __float_as_uint(g0.w); else cw = (uint32_t)g0.w;
                s_cw_w[0] = cw;
#pragma unroll
                for (int t = 0; t < T; ++t) s_mask_w[0][t] = rm[t];
            }
            sp = 1;
        }
    }
    __syncwarp();

    while (sp > 0 && !overflow) {
        --sp;
        const uint32_t cw = s_cw_w[sp];
        bool act[T];
        unsigned lanes = 0;
        uint32_t m0 = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t m = s_mask_w[sp][t];
            if (t == 0) m0 = m;
            act[t] = (m >> lane) & 1u;
            lanes += __popc(m);
        }
        const int first = (int)(cw & TS_CW_INDEX_MASK);
        const int dep = (int)(cw >> TS_CW_DEPTH_SHIFT);
        ++n_pop;
        n_lanes += lanes;
        R gphi[T], gax[T], gay[T], gaz[T];
        uint32_t mlp_acc = 0;   // learned-correction mode: children accepted by this lane's target
#pragma unroll
        for (int t = 0; t < T; ++t) gphi[t] = gax[t] = gay[t] = gaz[t] = 0;
        // (no warp barrier here: the staging buffers written next were last read before the
        // barrier that ends the previous pop, and the stack slot just read is rewritten only after
        // the barrier that follows the staging)
        if (cw & TS_CW_CELLS) {
            // ---- 8 leaf cells: every active target accepts all of them except its own cell
            if constexpr (PK) {
                // the group's x[8], y[8], z[8], m[8], read by every lane (broadcast loads)
                const float4* sx = P.cell_soa + 8 * (first >> 3);
                // (cell ids fit the 26-bit index field of the child words)
                const unsigned sd = (unsigned)mcell[0] - (unsigned)first;
                const bool selfin = sd < 8u;
                const int self0 = selfin ? (int)sd : 8;
                const uint32_t sm = __ballot_sync(0xffffffffu, selfin);
                n_int_w += 8u * lanes - (unsigned)__popc(sm & m0);
                float2 sp = make_float2(0.f, 0.f), sax = sp, say = sp, saz = sp;
                // every lane sums all 8 cells (inactive lanes discard theirs below); only a group
                // holding some lane's own cell needs the per-cell mask
                if (sm == 0u) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 X = __ldg(sx + q), Y = __ldg(sx + 2 + q);
                        const float4 Z = __ldg(sx + 4 + q), M = __ldg(sx + 6 + q);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float2 cx, cy, cz, m, dx, dy, dz, d2;
                            pk_pair(X, Y, Z, M, h, cx, cy, cz, m);
                            pk_sep(cx, cy, cz, nrx, nry, nrz, dx, dy, dz, d2);
                            pk_interact(dx, dy, dz, d2, m, true, true, sp, sax, say, saz);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 X = __ldg(sx + q), Y = __ldg(sx + 2 + q);
                        const float4 Z = __ldg(sx + 4 + q), M = __ldg(sx + 6 + q);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int j0 = 4 * q + 2 * h;
                            float2 cx, cy, cz, m, dx, dy, dz, d2;
                            pk_pair(X, Y, Z, M, h, cx, cy, cz, m);
                            pk_sep(cx, cy, cz, nrx, nry, nrz, dx, dy, dz, d2);
                            pk_interact_m(dx, dy, dz, d2, m, j0 != self0, j0 + 1 != self0, sp, sax, say, saz);
                        }
                    }
                }
                if (act[0]) {
                    kahan_add2(k01, c01, make_float2(sp.x + sp.y, POT ? 0.f : sax.x + sax.y));
                    if constexpr (!POT) kahan_add2(k23, c23, make_float2(say.x + say.y, saz.x + saz.y));
                }
            } else {
            if (lane < 8) s_com_w[lane] = cell[first + lane];
            __syncwarp();
            int self[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                self[t] = (int)(mcell[t] - first);   // in [0, 8) if this group holds target t
                if (act[t]) n_int += (self[t] >= 0 && self[t] < 8) ? 7u : 8u;
            }
            if constexpr (BCK == 2) {
                mlp_acc = act[0] ? (0xFFu & ~((self[0] >= 0 && self[0] < 8) ? (1u << self[0]) : 0u)) : 0u;
            } else
#pragma unroll(CHILD_UNROLL)
            for (int j = 0; j < 8; ++j) {
                const V4 c = s_com_w[j];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const R dx = mimg<R, BCK>(rx[t] - c.x, px, Lx, iLx), dy = mimg<R, BCK>(ry[t] - c.y, py, Ly, iLy),
                            dz = mimg<R, BCK>(rz[t] - c.z, pz, Lz, iLz);
                    const bool acc = act[t] && j != self[t];
                    const R d2 = acc ? dx * dx + dy * dy + dz * dz : (R)1;
                    const R gm = acc ? G * c.w : (R)0;
                    const R inv = rsqrt_t(d2);
                    if (BCK == 1 && ewk) {
                        R pf, Axx, Ayy, Azz;
                        ewald_pair<R, EWM>(P.ew, dx, dy, dz, inv, pf, Axx, Ayy, Azz);
                        gphi[t] -= gm * pf; gax[t] -= gm * Axx; gay[t] -= gm * Ayy; gaz[t] -= gm * Azz;
                    } else {
                        const R gi3 = gm * inv * inv * inv;
                        gphi[t] -= gm * inv; gax[t] -= gi3 * dx; gay[t] -= gi3 * dy; gaz[t] -= gi3 * dz;
                    }
                }
            }
            }
        } else {
            // ---- 8 internal nodes: per-target MAC, accepted nodes summed, opened ones pushed
            // (the paired walk reads the children's moments from their sibling group instead)
            if constexpr (!PK) if (lane < 8) s_com_w[lane] = ncom[first + lane];
            if constexpr (!PK) if (lane >= 8 && lane < 16) s_cen_w[lane - 8] = ncen[first + lane - 8];
            if constexpr (MAC == TS_MAC_MPE) {
                // lanes 16..23: (B2, B3) of child j and b_max, the distance from its centre of mass to
                // its furthest corner, sqrt(sum_k (half_k + |com_k - centre_k|)^2)
                if (lane >= 16 && lane < 24) {
                    const int j = lane - 16;
                    const V4 cm = ncom[first + j], gc = ncen[first + j];
                    R bx, by;
                    if constexpr (sizeof(R) == 4) {
                        const float2 b = ((const float2*)P.bmom)[first + j];
                        bx = b.x; by = b.y;
                    } else {
                        const double2 b = ((const double2*)P.bmom)[first + j];
                        bx = b.x; by = b.y;
                    }
                    const R ex = s_half[dep][0] + fabs(cm.x - gc.x), ey = s_half[dep][1] + fabs(cm.y - gc.y),
                            ez = s_half[dep][2] + fabs(cm.z - gc.z);
                    const R bmax = sqrt(ex * ex + ey * ey + ez * ez);
                    if constexpr (PK) {   // structure of arrays: B2[8], B3[8], b_max[8]
                        float* q = (float*)s_bm_w;
                        q[j] = bx; q[8 + j] = by; q[16 + j] = bmax;
                    } else {
                        s_bm_w[j] = V4{bx, by, bmax, (R)0};
                    }
                }
            }
            // (the paired walk stages only the MPE moments: for BH and APE its first barrier is the
            // one before the open masks are read back)
            if constexpr (!PK || MAC == TS_MAC_MPE) __syncwarp();
            const R hx = s_half[dep][0], hy = s_half[dep][1], hz = s_half[dep][2];
            const R h2 = s_h2[dep];
            uint32_t my_om[T];   // lane j < 8 keeps the open masks of child j
#pragma unroll
            for (int t = 0; t < T; ++t) my_om[t] = 0;
            // bits of the children whose eta_SB box holds target t (bit j: child j); the children's
            // geometric centres are c0 + (ox, oy, oz) 2 h with c0 the centre of child 0
            auto box_bits = [&](int t) -> unsigned {
                const V4 g0 = PK ? ncen[first] : s_cen_w[0];   // centre of child 0
                const R qx = rx[t] - g0.x, qy = ry[t] - g0.y, qz = rz[t] - g0.z;
                const R ex = eta * hx, ey = eta * hy, ez = eta * hz;
                const bool x0 = fabs(mimg<R, BCK>(qx, px, Lx, iLx)) <= ex;
                const bool x1 = fabs(mimg<R, BCK>(qx - 2 * hx, px, Lx, iLx)) <= ex;
                const bool y0 = fabs(mimg<R, BCK>(qy, py, Ly, iLy)) <= ey;
                const bool y1 = fabs(mimg<R, BCK>(qy - 2 * hy, py, Ly, iLy)) <= ey;
                const bool z0 = fabs(mimg<R, BCK>(qz, pz, Lz, iLz)) <= ez;
                const bool z1 = fabs(mimg<R, BCK>(qz - 2 * hz, pz, Lz, iLz)) <= ez;
                const unsigned X = (x0 ? 0x55u : 0u) | (x1 ? 0xAAu : 0u);
                const unsigned Y = (y0 ? 0x33u : 0u) | (y1 ? 0xCCu : 0u);
                const unsigned Z = (z0 ? 0x0Fu : 0u) | (z1 ? 0xF0u : 0u);
                return X & Y & Z;
            };
            // (the box test is skipped at depths where no target inside the box can pass the MAC,
            // see make_walk_params)
            const bool sbd = (P.sb_depths >> dep) & 1u;
            if constexpr (PK) {
                n_mac_w += 8u * lanes;
                const float4* sx = P.ncom_soa + 8 * ((first - 1) >> 3);
                float2 sp = make_float2(0.f, 0.f), sax = sp, say = sp, saz = sp;
                // BH: accept iff d^2 > h^2 / theta^2, the threshold formed once per pop
                const float hb = (float)h2 * ith2;
                const float2 hh = make_float2((float)h2, (float)h2);
                const float2 gg = make_float2((float)G, (float)G), al = make_float2((float)alim[0], (float)alim[0]);
                const bool a_act = act[0];
                auto pairs = [&](unsigned ins) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 X = __ldg(sx + q), Y = __ldg(sx + 2 + q);
                        const float4 Z = __ldg(sx + 4 + q), M = __ldg(sx + 6 + q);
                        uint32_t om[4];   // open masks of children 4 q .. 4 q + 3, parked by one store
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int j0 = 4 * q + 2 * h;
                            float2 cx, cy, cz, m, dx, dy, dz, d2, inv;
                            pk_pair(X, Y, Z, M, h, cx, cy, cz, m);
                            pk_sep(cx, cy, cz, nrx, nry, nrz, dx, dy, dz, d2);
                            bool mac0, mac1;
                            if constexpr (MAC == TS_MAC_MPE) {
                                // eq. mpe, p = 1, as in the scalar path: G/d^2 (1 - b/d)^-2
                                // (3 B2/d^2 - 2 B3/d^3) < a_lim for d > b; the rsqrt is reused by
                                // the interaction
                                const float4* bq = (const float4*)s_bm_w;
                                float2 b2, b3, bm, unused;
                                pk_pair(bq[q], bq[2 + q], bq[4 + q], bq[4 + q], h, b2, b3, bm, unused);
                                inv = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
                                const float2 qq = __ffma2_rn(make_float2(-bm.x, -bm.y), inv, make_float2(1.f, 1.f));
                                const float2 i2 = __fmul2_rn(inv, inv);
                                const float2 br = __ffma2_rn(__fmul2_rn(make_float2(3.f, 3.f), b2), i2,
                                                             __fmul2_rn(__fmul2_rn(make_float2(-2.f, -2.f), b3),
                                                                        __fmul2_rn(i2, inv)));
                                const float2 lhs = __fmul2_rn(__fmul2_rn(gg, i2), br);
                                const float2 rhs = __fmul2_rn(__fmul2_rn(al, qq), qq);
                                mac0 = qq.x > 0.f && lhs.x < rhs.x; mac1 = qq.y > 0.f && lhs.y < rhs.y;
                            } else if constexpr (MAC == TS_MAC_BH) {
                                mac0 = d2.x > hb; mac1 = d2.y > hb;
                            } else {
                                const float2 lhs = __fmul2_rn(__fmul2_rn(gg, m), hh);
                                const float2 rhs = __fmul2_rn(__fmul2_rn(al, d2), d2);
                                mac0 = lhs.x < rhs.x; mac1 = lhs.y < rhs.y;
                            }
                            const bool a0 = a_act && mac0 && !((ins >> j0) & 1u);
                            const bool a1 = a_act && mac1 && !((ins >> (j0 + 1)) & 1u);
                            om[2 * h] = __ballot_sync(0xffffffffu, a_act && !a0);
                            om[2 * h + 1] = __ballot_sync(0xffffffffu, a_act && !a1);
                            // (no warp vote to skip pairs nobody accepts: most children are
                            // accepted, and the vote costs more than it saves)
                            if constexpr (MAC == TS_MAC_MPE)
                                pk_interact_inv(dx, dy, dz, inv, m, a0, a1, sp, sax, say, saz);
                            else
                                pk_interact_m(dx, dy, dz, d2, m, a0, a1, sp, sax, say, saz);
                        }
                        if (lane == 0)
                            *(uint4*)&s_mask_w[TS_WALK_STACK - 8 + 4 * q][0] = make_uint4(om[0], om[1], om[2], om[3]);
                    }
                };
                if (sbd) pairs(box_bits(0)); else pairs(0u);
                if (a_act) {
                    kahan_add2(k01, c01, make_float2(sp.x + sp.y, POT ? 0.f : sax.x + sax.y));
                    if constexpr (!POT) kahan_add2(k23, c23, make_float2(say.x + say.y, saz.x + saz.y));
                }
            } else {
            unsigned inside[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                inside[t] = sbd ? box_bits(t) : 0u;
                if (act[t]) n_mac += 8;
            }
#pragma unroll(CHILD_UNROLL)
            for (int j = 0; j < 8; ++j) {
                const V4 c = s_com_w[j];
                bool acc[T];
                bool anyacc = false;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const R dx = mimg<R, BCK>(rx[t] - c.x, px, Lx, iLx), dy = mimg<R, BCK>(ry[t] - c.y, py, Ly, iLy),
                            dz = mimg<R, BCK>(rz[t] - c.z, pz, Lz, iLz);
                    const R d2 = dx * dx + dy * dy + dz * dz;
                    bool mac;
                    if constexpr (MAC == TS_MAC_BH) {
                        mac = h2 < theta2 * d2;                              // eq. bhmac
                    } else if constexpr (MAC == TS_MAC_APE) {
                        mac = G * c.w * h2 < alim[t] * d2 * d2;              // eq. ape, p = 1
                    } else {
                        // eq. mpe, p = 1: G/d^2 (1 - b/d)^-2 (3 B2/d^2 - 2 B3/d^3) < a_lim, for d > b
                        const V4 bm = s_bm_w[j];
                        const R inv = rsqrt_t(d2), q = (R)1 - bm.z * inv;
                        mac = q > (R)0 &&
                              G * inv * inv * (3 * bm.x * inv * inv - 2 * bm.y * inv * inv * inv) < alim[t] * q * q;
                    }
                    const bool ok = mac && !((inside[t] >> j) & 1u);
                    acc[t] = act[t] && ok;
                    const uint32_t om = __ballot_sync(0xffffffffu, act[t] && !ok);
                    if (lane == 0) s_mask_w[TS_WALK_STACK - 8 + j][t] = om;   // parked above the stack top
                    anyacc |= acc[t];
                }
                if constexpr (BCK == 2) {
                    mlp_acc |= (acc[0] ? 1u : 0u) << j;
                    n_int += acc[0];
                } else if (__any_sync(0xffffffffu, anyacc)) {
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const R dx = mimg<R, BCK>(rx[t] - c.x, px, Lx, iLx),
                                dy = mimg<R, BCK>(ry[t] - c.y, py, Ly, iLy),
                                dz = mimg<R, BCK>(rz[t] - c.z, pz, Lz, iLz);
                        n_int += acc[t];
                        const R gm = acc[t] ? G * c.w : (R)0;
                        const R inv = rsqrt_t(acc[t] ? dx * dx + dy * dy + dz * dz : (R)1);
                        if (BCK == 1 && ewk) {
                            R pf, Axx, Ayy, Azz;
                            ewald_pair<R, EWM>(P.ew, dx, dy, dz, inv, pf, Axx, Ayy, Azz);
                            gphi[t] -= gm * pf; gax[t] -= gm * Axx; gay[t] -= gm * Ayy; gaz[t] -= gm * Azz;
                        } else {
                            const R gi3 = gm * inv * inv * inv;
                            gphi[t] -= gm * inv; gax[t] -= gi3 * dx; gay[t] -= gi3 * dy; gaz[t] -= gi3 * dz;
                        }
                    }
                }
            }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < T; ++t) my_om[t] = lane < 8 ? s_mask_w[TS_WALK_STACK - 8 + lane][t] : 0u;
            // (the paired path counts its accepted pairs at the end, from the pops' lane counts)
            // push the opened children in one compacted write: lane j < 8 owns child j
            bool mine = false;
#pragma unroll
            for (int t = 0; t < T; ++t) mine |= my_om[t] != 0u;
            const unsigned nz = __ballot_sync(0xffffffffu, mine);
            const int npush = __popc(nz);
            if (sp + npush > TS_WALK_STACK - 8) {   // the top 8 slots park the open masks
                overflow = true;
            } else {
                if (mine) {
                    const V4 g = PK ? ncen[first + lane] : s_cen_w[lane];
                    uint32_t ccw;
                    if constexpr (sizeof(R) == 4) ccw = __float_as_uint(g.w); else ccw = (uint32_t)g.w;
                    const int slot = sp + __popc(nz & ((1u << lane) - 1u));
                    s_cw_w[slot] = ccw;
#pragma unroll
                    for (int t = 0; t < T; ++t) s_mask_w[slot][t] = my_om[t];
                }
                sp += npush;
            }
        }
        if constexpr (BCK == 2) {
            // learned correction: the lanes' accepted children become compacted rows (warp scan),
            // the network evaluates them in 16-row tensor-core tiles, each lane sums its own rows
            uint4* rf = (uint4*)(s_dyn + MLP_SMEM_WEIGHTS + warp * MLP_SMEM_WARP);
            float4* ro = (float4*)(rf + MLP_ROWS);
            float4* rd = ro + MLP_ROWS;
            const int cnt = __popc(mlp_acc);
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int k0 = incl - cnt;
            int k = k0;
            const float far = (float)P.ew.far, slope = (float)P.ew.far_slope, fconst = (float)P.ew.far_const;
            for (int j = 0; j < 8; ++j) {
                if ((mlp_acc >> j) & 1u) {
                    const V4 c = s_com_w[j];
                    const float dx = mimg<R, BCK>(rx[0] - c.x, px, Lx, iLx), dy = mimg<R, BCK>(ry[0] - c.y, py, Ly, iLy),
                                dz = mimg<R, BCK>(rz[0] - c.z, pz, Lz, iLz);
                    const float adz = fabsf(dz);
                    if (adz > far) {   // far field of Sec. 2.2.5 (no network)
                        const float gm = G * c.w;
                        gphi[0] -= gm * (fconst - slope * adz);
                        gaz[0] -= gm * copysignf(slope, dz);
                        rf[k] = make_uint4(0u, 0u, 0u, 0u);
                        rd[k] = make_float4(dx, dy, dz, 0.f);
                    } else {
                        rf[k] = mlp_feat_pack(fabsf(dx) * P.mlp_sx - 1.f, fabsf(dy) * P.mlp_sy - 1.f,
                                              adz * P.mlp_sz - 1.f, P.mlp_f3);
                        rd[k] = make_float4(dx, dy, dz, G * c.w);
                    }
                    ++k;
                }
            }
            __syncwarp();
            MlpView M;
            M.w = (const __nv_bfloat16*)s_dyn;
            M.f = (const float*)(s_dyn + MLP_FWD_BF16 * 2);
            for (int m0 = 0; m0 < total; m0 += 16) mlp_eval_tile(M, rf, ro, m0, total, lane);
            __syncwarp();
            for (int q = k0; q < k0 + cnt; ++q) {
                const float4 dm = rd[q];
                if (dm.w != 0.f) {
                    const float4 o = ro[q];
                    const float inv = rsqrtf(dm.x * dm.x + dm.y * dm.y + dm.z * dm.z), inv3 = inv * inv * inv;
                    gphi[0] -= dm.w * (inv + o.x * P.mlp_c);
                    gax[0] -= dm.w * (dm.x * inv3 + (dm.x < 0.f ? -o.y : o.y) * P.mlp_a);
                    gay[0] -= dm.w * (dm.y * inv3 + (dm.y < 0.f ? -o.z : o.z) * P.mlp_a);
                    gaz[0] -= dm.w * (dm.z * inv3 + (dm.z < 0.f ? -o.w : o.w) * P.mlp_a);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if constexpr (PK) {
            } else if constexpr (sizeof(R) == 4) {
                kahan_add(phi[t], cphi[t], gphi[t]); kahan_add(ax[t], cax[t], gax[t]);
                kahan_add(ay[t], cay[t], gay[t]); kahan_add(az[t], caz[t], gaz[t]);
            } else {
                phi[t] += gphi[t]; ax[t] += gax[t]; ay[t] += gay[t]; az[t] += gaz[t];
            }
        }
        __syncwarp();
    }
    if (overflow && lane == 0) atomicOr(P.status, TS_DEV_STACK_OVERFLOW);
    R* pot = (R*)P.pot;
    R* acc = (R*)P.acc;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if constexpr (sizeof(R) == 4) {
            phi[t] -= cphi[t]; ax[t] -= cax[t]; ay[t] -= cay[t]; az[t] -= caz[t];
        }
        if constexpr (PK) {
            phi[t] -= G * (k01.x - c01.x); ax[t] += G * (k01.y - c01.y);
            ay[t] += G * (k23.x - c23.x); az[t] += G * (k23.y - c23.y);
        }
        const int64_t o = P.targets ? gw * 32 + lane : nat[t];
        pot[o] = phi[t];
        if constexpr (POT) {
            bad |= !isfinite(phi[t]);
        } else {
            acc[3 * o] = ax[t]; acc[3 * o + 1] = ay[t]; acc[3 * o + 2] = az[t];
            bad |= !isfinite(phi[t]) || !isfinite(ax[t]) || !isfinite(ay[t]) || !isfinite(az[t]);
        }
    }
    if (bad) atomicOr(P.status, TS_DEV_NONFINITE);
    // paired path: every opened (lane, child) pair of an internal pop is pushed and later popped
    // for that lane, so the opened pairs are the lanes of every pop but the root's, and the accepted
    // ones 8 per lane and internal pop less those (the counts are exact unless the stack overflowed,
    // which fails the walk)
    if constexpr (PK) n_int_w += n_mac_w - (n_lanes - root_lanes);
    const unsigned wi = __reduce_add_sync(0xffffffffu, n_int) + n_int_w,
                   wm = __reduce_add_sync(0xffffffffu, n_mac) + n_mac_w;
    if (lane == 0) {
        atomicAdd(&P.counters[0], (unsigned long long)wi);
        atomicAdd(&P.counters[1], (unsigned long long)wm);
        atomicAdd(&P.counters[2], (unsigned long long)n_pop);
        atomicAdd(&P.counters[3], (unsigned long long)n_lanes);
        if (P.blk_counts && !P.targets) atomicAdd(&P.blk_counts[base >> 9], (unsigned long long)wi);
    }
}
