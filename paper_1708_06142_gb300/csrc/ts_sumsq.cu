// SumSquare MAC walk (Sec. 2.2.1): the error of the total acceleration is limited instead of each
// node's.  Per target, the frontier of nodes waiting for evaluation is a priority queue ordered by
// the node's MPE bound (eq. mpe, p = 1); the node with the largest bound is replaced by its
// children until the summed squared bounds of the frontier are at most a_lim^2, then the whole
// frontier is accepted.  Bounds are infinite where they do not apply (target within b_max of the
// centre of mass) or where the target lies in the node's safe box; cells are exact and accepted
// when reached (the target's own cell excluded).  Equal bounds are ordered by the node's depth and
// integer position.  The summed squares are kept exactly, in integer units of 2^-20 a_lim^2 (a
// floating-point running sum loses small terms when large ones leave it, and the walk would then
// refine far past the limit).  A queue that would exceed queue_max nodes stops refining and its
// frontier is accepted.
//
// GPU form: the decisions of one target depend on the order of its own queue, so the walk is one
// thread per target (a persistent grid striding over the targets) with a binary max-heap in a
// per-thread slice of context-owned device scratch: keys (the squared bound, in the walk's
// precision) and node words (node id and depth).  Memory-latency bound; the paper calls this MAC
// experimental and finds it less efficient than the others, and it is not a hot path here.
#include <math.h>

#include <algorithm>

#include "ts_walk_dev.cuh"

struct SqParams {
    const void* ncom;      // RT<R>::V4 per internal node: (centre of mass, M)
    const dbl4* ncen64;    // geometric centre and child word (also the tie-break key)
    const void* cell;      // RT<R>::V4 per cell (Morton): (centre, m)
    const void* bmom;      // (B2, B3) per internal node, double2 / float2
    const WalkGeom* geom;
    int64_t ncell;
    uint32_t root_cw;
    double eta, a_lim2, G, dlo[3];
    int qmax;
    void* keys;            // [nthreads][qmax] R
    uint32_t* words;       // [nthreads][qmax] node id | depth << 26
    EwaldDev ew;
    void* pot;
    void* acc;
    int* status;
    unsigned long long* counters;   // [0] interactions, [1] bounds, [2] queue pops, [3] overflows
};

// canonical order of equal bounds: depth, then integer position x, y, z of the node at its depth
__device__ __forceinline__ long long sq_canon(const SqParams& P, uint32_t word) {
    const int nid = (int)(word & TS_CW_INDEX_MASK), dep = (int)(word >> TS_CW_DEPTH_SHIFT);
    const dbl4 c = P.ncen64[nid];
    const double cc[3] = {c.x, c.y, c.z};
    long long k = (long long)dep << 57;
    for (int a = 0; a < 3; ++a) {
        const long long i = llrint((cc[a] - P.dlo[a]) / P.geom->L[a] * ldexp(1.0, dep) - 0.5);
        k |= i << (38 - 19 * a);
    }
    return k;
}

template <typename R>
__device__ __forceinline__ bool sq_before(const SqParams& P, R ka, uint32_t wa, R kb, uint32_t wb) {
    if (ka != kb) return ka > kb;
    return sq_canon(P, wa) < sq_canon(P, wb);
}

template <typename R>
__device__ void sq_push(const SqParams& P, R* hk, uint32_t* hw, int& n, R k, uint32_t w) {
    int i = n++;
    while (i > 0) {
        const int p = (i - 1) >> 1;
        if (!sq_before<R>(P, k, w, hk[p], hw[p])) break;
        hk[i] = hk[p];
        hw[i] = hw[p];
        i = p;
    }
    hk[i] = k;
    hw[i] = w;
}

template <typename R>
__device__ void sq_pop(const SqParams& P, R* hk, uint32_t* hw, int& n, R& k, uint32_t& w) {
    k = hk[0];
    w = hw[0];
    --n;
    const R lk = hk[n];
    const uint32_t lw = hw[n];
    int i = 0;
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && sq_before<R>(P, hk[c + 1], hw[c + 1], hk[c], hw[c])) ++c;
        if (!sq_before<R>(P, hk[c], hw[c], lk, lw)) break;
        hk[i] = hk[c];
        hw[i] = hw[c];
        i = c;
    }
    if (n > 0) {
        hk[i] = lk;
        hw[i] = lw;
    }
}

template <typename R>
__device__ __forceinline__ R mimg_p(R d, int per, R L, R iL) {
    if (per) d -= L * rint_t(d * iL);
    return d;
}

// squared MPE bound of internal node nid at depth dep (infinite: the node must be opened); the
// FP64 form follows the oracle's operation order with explicitly rounded operations
template <typename R>
__device__ R sq_bound2(const SqParams& P, const R r[3], int nid, int dep) {
    typedef typename RT<R>::V4 V4;
    const V4 cm = ((const V4*)P.ncom)[nid];
    const dbl4 gc = P.ncen64[nid];
    const WalkGeom& Gm = *P.geom;
    const R com[3] = {cm.x, cm.y, cm.z}, cen[3] = {(R)gc.x, (R)gc.y, (R)gc.z};
    R dv[3], rc[3], half[3];
    bool outside = false;
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(R) == 8) half[a] = Gm.half64[dep][a]; else half[a] = Gm.half32[dep][a];
        dv[a] = mimg_p<R>(r[a] - com[a], Gm.pbc[a], (R)Gm.L[a], (R)Gm.invL[a]);
        rc[a] = mimg_p<R>(r[a] - cen[a], Gm.pbc[a], (R)Gm.L[a], (R)Gm.invL[a]);
        outside |= fabs(rc[a]) > (R)P.eta * half[a];
    }
    R B2, B3;
    if constexpr (sizeof(R) == 8) {
        const double2 b = ((const double2*)P.bmom)[nid];
        B2 = b.x; B3 = b.y;
    } else {
        const float2 b = ((const float2*)P.bmom)[nid];
        B2 = b.x; B3 = b.y;
    }
    if constexpr (sizeof(R) == 8) {
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dv[0], dv[0]), __dmul_rn(dv[1], dv[1])), __dmul_rn(dv[2], dv[2]));
        const double d = sqrt(d2);
        double bmax2 = 0;
        for (int a = 0; a < 3; ++a) {
            const double t = __dadd_rn(half[a], fabs(__dsub_rn(com[a], cen[a])));
            bmax2 = __dadd_rn(bmax2, __dmul_rn(t, t));
        }
        const double bmax = sqrt(bmax2);
        if (!outside || !(d > bmax)) return (double)INFINITY;
        const double q = __dsub_rn(1.0, __ddiv_rn(bmax, d));
        const double f = __ddiv_rn(__ddiv_rn(P.G, d2), __dmul_rn(q, q));
        const double g = __dsub_rn(__ddiv_rn(__dmul_rn(3.0, B2), d2), __ddiv_rn(__dmul_rn(2.0, B3), __dmul_rn(d2, d)));
        const double da = __dmul_rn(f, g);
        return __dmul_rn(da, da);
    } else {
        const float d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        const float d = sqrtf(d2);
        float bmax2 = 0;
        for (int a = 0; a < 3; ++a) {
            const float t = half[a] + fabsf(com[a] - cen[a]);
            bmax2 += t * t;
        }
        const float bmax = sqrtf(bmax2);
        if (!outside || !(d > bmax)) return INFINITY;
        const float q = 1.f - bmax / d;
        const float da = (float)P.G / d2 / (q * q) * (3.f * B2 / d2 - 2.f * B3 / (d2 * d));
        return da * da;
    }
}

// The frontier's summed squares kept exactly: a bound counts as ceil(2^20 e2 / a_lim^2) in an integer
// sum (order-independent: large and small terms cannot absorb one another), bounds of 2^30 a_lim^2
// or more are counted apart as large; the limit holds when nothing is large and the sum is at most
// 2^20.  The same function of the same (FP64-converted) key as the oracle's.
__device__ __forceinline__ long long sq_units(double e2, double lim2, int& large) {
    const double t = e2 / lim2;
    if (!(t < 1073741824.0)) {
        large = 1;
        return 0;
    }
    large = 0;
    return (long long)ceil(t * 1048576.0);
}

template <typename R>
struct SqAcc {
    R phi, ax, ay, az, cphi, cax, cay, caz;
};

// FP32 sums are compensated (Kahan), FP64 sums plain, as in the other walks
template <typename R>
__device__ __forceinline__ void sq_add(R v, R& s, R& c) {
    if constexpr (sizeof(R) == 4) {
        kahan_add(s, c, v);
    } else {
        s += v;
    }
}

template <typename R>
__device__ __forceinline__ void sq_interact(const SqParams& P, const R r[3], const typename RT<R>::V4& m, SqAcc<R>& A) {
    const WalkGeom& Gm = *P.geom;
    const R dx = mimg_p<R>(r[0] - m.x, Gm.pbc[0], (R)Gm.L[0], (R)Gm.invL[0]);
    const R dy = mimg_p<R>(r[1] - m.y, Gm.pbc[1], (R)Gm.L[1], (R)Gm.invL[1]);
    const R dz = mimg_p<R>(r[2] - m.z, Gm.pbc[2], (R)Gm.L[2], (R)Gm.invL[2]);
    const R inv = rsqrt_t(dx * dx + dy * dy + dz * dz);
    R pf = inv, Ax, Ay, Az;
    if (P.ew.kind != TS_EW_NONE) {
        ewald_pair<R, 2>(P.ew, dx, dy, dz, inv, pf, Ax, Ay, Az);
    } else {
        const R i3 = inv * inv * inv;
        Ax = dx * i3; Ay = dy * i3; Az = dz * i3;
    }
    const R gm = (R)P.G * m.w;
    sq_add<R>(-gm * pf, A.phi, A.cphi);
    sq_add<R>(-gm * Ax, A.ax, A.cax);
    sq_add<R>(-gm * Ay, A.ay, A.cay);
    sq_add<R>(-gm * Az, A.az, A.caz);
}

template <typename R>
__global__ void __launch_bounds__(64) k_sumsq_walk(const __grid_constant__ SqParams P) {
    typedef typename RT<R>::V4 V4;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    R* hk = (R*)P.keys + tid * P.qmax;
    uint32_t* hw = P.words + tid * P.qmax;
    const V4* cells = (const V4*)P.cell;
    const V4* nodes = (const V4*)P.ncom;
    unsigned long long n_int = 0, n_b = 0, n_pop = 0, n_ovf = 0;
    const double lim2 = P.a_lim2;
    for (int64_t me = tid; me < P.ncell; me += nthr) {
        const V4 mine = cells[me];
        const R r[3] = {mine.x, mine.y, mine.z};
        SqAcc<R> A = {0, 0, 0, 0, 0, 0, 0, 0};
        int n = 0, n_large = 0, lg;
        long long E = 0;
        {
            const uint32_t w = 0u;   // the root: node 0 at depth 0
            const R k = sq_bound2<R>(P, r, 0, 0);
            ++n_b;
            E += sq_units((double)k, lim2, lg);
            n_large += lg;
            sq_push<R>(P, hk, hw, n, k, w);
        }
        while (n > 0 && (n_large > 0 || E > 1048576ll)) {
            if (n - 1 + 8 > P.qmax) {
                ++n_ovf;
                break;
            }
            R k;
            uint32_t w;
            sq_pop<R>(P, hk, hw, n, k, w);
            ++n_pop;
            E -= sq_units((double)k, lim2, lg);
            n_large -= lg;
            const int nid = (int)(w & TS_CW_INDEX_MASK);
            const uint32_t cw = (uint32_t)P.ncen64[nid].w;
            const int first = (int)(cw & TS_CW_INDEX_MASK), cdep = (int)(cw >> TS_CW_DEPTH_SHIFT);
            if (cw & TS_CW_CELLS) {
                for (int j = 0; j < 8; ++j) {
                    if (first + j == me) continue;
                    sq_interact<R>(P, r, cells[first + j], A);
                    ++n_int;
                }
            } else {
                for (int j = 0; j < 8; ++j) {
                    const R kc = sq_bound2<R>(P, r, first + j, cdep);
                    ++n_b;
                    E += sq_units((double)kc, lim2, lg);
                    n_large += lg;
                    sq_push<R>(P, hk, hw, n, kc, (uint32_t)(first + j) | ((uint32_t)cdep << TS_CW_DEPTH_SHIFT));
                }
            }
        }
        for (int i = 0; i < n; ++i) {
            sq_interact<R>(P, r, nodes[hw[i] & TS_CW_INDEX_MASK], A);
            ++n_int;
        }
        R phi = A.phi, ax = A.ax, ay = A.ay, az = A.az;
        if constexpr (sizeof(R) == 4) {
            phi -= A.cphi; ax -= A.cax; ay -= A.cay; az -= A.caz;
        }
        // Morton id -> the caller's flat order
        const int ml = (int)(me & 511);
        const int q = ml >> 6, o = (ml >> 3) & 7, o2 = ml & 7;
        const int ci = 4 * (q & 1) + 2 * (o & 1) + (o2 & 1);
        const int cj = 4 * ((q >> 1) & 1) + 2 * ((o >> 1) & 1) + ((o2 >> 1) & 1);
        const int ck = 4 * (q >> 2) + 2 * (o >> 2) + (o2 >> 2);
        const int64_t nat = (me >> 9) * 512 + ck * 64 + cj * 8 + ci;
        ((R*)P.pot)[nat] = phi;
        R* a = (R*)P.acc + 3 * nat;
        a[0] = ax; a[1] = ay; a[2] = az;
        if (!isfinite(phi) || !isfinite(ax) || !isfinite(ay) || !isfinite(az)) atomicOr(P.status, TS_DEV_NONFINITE);
    }
    atomicAdd(&P.counters[0], n_int);
    atomicAdd(&P.counters[1], n_b);
    atomicAdd(&P.counters[2], n_pop);
    atomicAdd(&P.counters[3], n_ovf);
}

cudaError_t launch_sumsq(ts_ctx* c, const ts_gravity_params* p, const WalkParams& W, void* pot, void* acc) {
    const bool fp64 = p->precision == TS_PREC_FP64;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const int threads = 64;
    const int qmax = p->queue_max > 0 ? p->queue_max : 4096;
    const size_t per_thr = (size_t)qmax * ((fp64 ? 8 : 4) + 4);
    // one thread per target at a time; the heap operations are latency bound, so as many threads
    // as 32 CTAs of 64 per SM (measured on the 2M-cell Plummer mesh: 4 CTAs per SM 201 ms, 16 186 ms,
    // 32 165 ms), fewer if their queues would take more than half the free device memory
    int64_t nblk = std::min<int64_t>((c->ncell + threads - 1) / threads, (int64_t)nsm * 32);
    if (c->sq_bytes < (size_t)nblk * threads * per_thr) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const int64_t fit = (int64_t)(((fr + c->sq_bytes) / 2) / (per_thr * threads));
            nblk = std::max<int64_t>(std::min<int64_t>(nblk, fit), std::min<int64_t>(nblk, (int64_t)nsm * 4));
        }
    }
    const int64_t nthr = nblk * threads;
    const size_t need = (size_t)nthr * per_thr;
    if (c->sq_bytes < need) {
        if (c->d_sq) cudaFree(c->d_sq);
        c->d_sq = nullptr;
        c->sq_bytes = 0;
        cudaError_t e = ts_malloc(&c->d_sq, need);
        if (e != cudaSuccess) return e;
        c->sq_bytes = need;
    }
    SqParams P;
    memset(&P, 0, sizeof(P));
    P.ncom = W.ncom;
    P.ncen64 = c->d_ncen64;
    P.cell = W.cell;
    P.bmom = W.bmom;
    P.geom = W.geom;
    P.ncell = c->ncell;
    P.root_cw = c->root_cw;
    P.eta = p->safe_box;
    P.a_lim2 = p->a_lim * p->a_lim;
    P.G = p->G;
    for (int a = 0; a < 3; ++a) P.dlo[a] = c->dlo[a];
    P.qmax = qmax;
    P.keys = c->d_sq;
    P.words = (uint32_t*)((char*)c->d_sq + (size_t)nthr * qmax * (fp64 ? 8 : 4));
    P.ew = W.ew;
    P.pot = pot;
    P.acc = acc;
    P.status = c->d_status;
    P.counters = c->d_counters;
    if (fp64) k_sumsq_walk<double><<<(int)nblk, threads, 0, c->stream>>>(P);
    else k_sumsq_walk<float><<<(int)nblk, threads, 0, c->stream>>>(P);
    return cudaGetLastError();
}
