// Acceleration by numerical differentiation of the cell-centred potential (Sec. 2.2.2: the
// alternative to summing eq. accel during the walk; the walk then forms the potential of eq. pot
// alone), and the potential-only walk kernels that feed it.
//
// Definition (reading of the paper, which names the method but not its stencil): second-order
// central differences, a_k = -(g(+1) - g(-1)) / (2 dx_k), where g(m) is the potential of the
// guard cube D(m): the cube of the target cell's own size displaced by m cells along axis k.  On
// an AMR mesh D(m) is a dyadic cube of the target's depth, and g(m) is
//   - the value of the leaf cell that contains D(m) (same or coarser level: injection), or
//   - the volume-weighted mean over the leaf cells inside D(m) (finer level: restriction),
// the two guard-cell rules of a block-structured AMR code without interpolation.  Periodic axes
// wrap D(m); on isolated axes a cube outside the domain is missing and the one-sided second-order
// formula is used instead, a_k = -(-3 phi_0 + 4 g(+1) - g(+2)) / (2 dx_k) (mirrored at the upper
// edge).  Differences are formed in FP64 from the stored potential values.
//
// Data: the integer position of every cell at its own depth (the domain has 2^d cells per axis at
// depth d), a per-block table (first child node id or -1, leaf index or -1) for the descent from
// the root, and the potential in the caller's flat cell order.  One thread per cell, six guard
// lookups each (one descent of <= depth block levels per lookup); HBM-bound (a read of the
// potential, L2-served neighbour reads, a 12/24-byte write per cell).
#include <math.h>

#include <algorithm>

#include "ts_walk_kernels.cuh"

struct NdGeom {
    const int2* blk;          // [nb] (first child node id or -1, leaf index or -1), node ids of blocks
    const int4* leaf;         // [nleaf] (x0, y0, z0, cell depth): first cell of the block at its depth
    const double* leaf_size;  // [nleaf][3]
    int pbc[3];
    int64_t ncell;
};

__device__ __forceinline__ int64_t nd_flat(int leaf, int i, int j, int k) {
    return (int64_t)leaf * 512 + k * 64 + j * 8 + i;
}

// Potential of the guard cube at depth d, integer position (X, Y, Z) (already wrapped / checked).
template <typename R>
__device__ double nd_guard(const NdGeom& G, const R* __restrict__ pot, int d, int64_t X, int64_t Y, int64_t Z) {
    int node = 0, b = 0;
    int2 e = G.blk[0];
    while (e.x >= 0 && b < d) {
        const int s = d - b - 1;
        const int oct = (int)((X >> s) & 1) | (int)(((Y >> s) & 1) << 1) | (int)(((Z >> s) & 1) << 2);
        node = e.x + oct;
        e = G.blk[node];
        ++b;
    }
    if (e.x < 0) {                        // a leaf-block at depth b <= d
        const int4 L = G.leaf[e.y];
        const int dl = L.w;               // its cells' depth, b + 3
        if (dl <= d) {                    // same or coarser cell: injection
            const int sh = d - dl;
            return (double)pot[nd_flat(e.y, (int)((X >> sh) - L.x), (int)((Y >> sh) - L.y), (int)((Z >> sh) - L.z))];
        }
        const int sh = dl - d, w = 1 << sh;   // finer cells: the w^3 cells inside D, equal volumes
        const int i0 = (int)((X << sh) - L.x), j0 = (int)((Y << sh) - L.y), k0 = (int)((Z << sh) - L.z);
        double s = 0;
        for (int k = 0; k < w; ++k)
            for (int j = 0; j < w; ++j)
                for (int i = 0; i < w; ++i) s += (double)pot[nd_flat(e.y, i0 + i, j0 + j, k0 + k)];
        return s / (double)(w * w * w);
    }
    // a non-leaf block equal to D (level jump of 3 or more): volume-weighted mean over its subtree
    int stack[256];
    int sp = 0;
    stack[sp++] = node;
    double s = 0, v = 0;
    while (sp > 0) {
        const int n = stack[--sp];
        const int2 f = G.blk[n];
        if (f.x >= 0) {
            if (sp + 8 > 256) return nan("");   // deeper than any mesh the ingest accepts
            for (int o = 0; o < 8; ++o) stack[sp++] = f.x + o;
            continue;
        }
        const double wv = ldexp(1.0, -3 * (G.leaf[f.y].w - d));   // cell volume relative to D
        double ls = 0;
        for (int q = 0; q < 512; ++q) ls += (double)pot[(int64_t)f.y * 512 + q];
        s += wv * ls;
        v += wv * 512.0;
    }
    return s / v;
}

// Guard value at offset m cells along axis a; false if it lies outside the domain on an isolated axis.
template <typename R>
__device__ __forceinline__ bool nd_at(const NdGeom& G, const R* __restrict__ pot, int d, const int64_t P[3], int a, int m,
                                      int64_t N, double& out) {
    int64_t Q[3] = {P[0], P[1], P[2]};
    Q[a] += m;
    if (Q[a] < 0 || Q[a] >= N) {
        if (!G.pbc[a]) return false;
        Q[a] = ((Q[a] % N) + N) % N;
    }
    out = nd_guard<R>(G, pot, d, Q[0], Q[1], Q[2]);
    return true;
}

template <typename R>
__global__ void __launch_bounds__(256) k_num_diff(const NdGeom G, const R* __restrict__ pot, R* __restrict__ acc) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= G.ncell) return;
    const int leaf = (int)(c >> 9), l = (int)(c & 511);
    const int4 L = G.leaf[leaf];
    const int d = L.w;
    const int64_t P[3] = {L.x + (l & 7), L.y + ((l >> 3) & 7), L.z + (l >> 6)};
    const int64_t N = (int64_t)1 << d;    // cells per axis at this depth (>= 8)
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
        const double dx = G.leaf_size[3 * leaf + a] * 0.125;
        double gm = 0, gp = 0, deriv;
        const bool hm = nd_at<R>(G, pot, d, P, a, -1, N, gm);
        const bool hp = nd_at<R>(G, pot, d, P, a, +1, N, gp);
        if (hm && hp) {
            deriv = (gp - gm) / (2.0 * dx);
        } else {                               // isolated edge: one-sided, towards the interior
            const int s = hp ? 1 : -1;
            double g2 = 0;
            nd_at<R>(G, pot, d, P, a, 2 * s, N, g2);
            deriv = (double)s * (-3.0 * (double)pot[c] + 4.0 * (hp ? gp : gm) - g2) / (2.0 * dx);
        }
        acc[3 * c + a] = (R)(-deriv);
    }
}

cudaError_t launch_num_diff(ts_ctx* c, int precision, const void* pot, void* acc) {
    NdGeom G;
    G.blk = c->d_nd_blk;
    G.leaf = c->d_nd_leaf;
    G.leaf_size = c->d_leaf_size;
    for (int a = 0; a < 3; ++a) G.pbc[a] = c->bc[a];
    G.ncell = c->ncell;
    const int grid = (int)((c->ncell + 255) / 256);
    if (precision == TS_PREC_FP64)
        k_num_diff<double><<<grid, 256, 0, c->stream>>>(G, (const double*)pot, (double*)acc);
    else
        k_num_diff<float><<<grid, 256, 0, c->stream>>>(G, (const float*)pot, (float*)acc);
    return cudaGetLastError();
}

// Potential-only walks (one target per lane; BH, and APE with an absolute limit).  Other MAC
// variants return cudaErrorNotSupported and the caller runs the full walk, whose accelerations
// the differentiation then overwrites.
cudaError_t walk_launch_pot(ts_ctx* c, const WalkParams& P, bool fp64, int bck, int mac, bool rel) {
    if (rel || bck == 2 || (mac != TS_MAC_BH && mac != TS_MAC_APE)) return cudaErrorNotSupported;
    const bool bh = mac == TS_MAC_BH;
    if (!fp64) {
        if (bck == 0)
            return bh ? launch_t<float, 0, TS_MAC_BH, false, 1, 2, true>(c, P)
                      : launch_t<float, 0, TS_MAC_APE, false, 1, 2, true>(c, P);
        if (P.ew.taylor)
            return bh ? launch_t<float, 1, TS_MAC_BH, false, 1, 1, true>(c, P)
                      : launch_t<float, 1, TS_MAC_APE, false, 1, 1, true>(c, P);
        return bh ? launch_t<float, 1, TS_MAC_BH, false, 1, 0, true>(c, P)
                  : launch_t<float, 1, TS_MAC_APE, false, 1, 0, true>(c, P);
    }
    if (bck == 0)
        return bh ? launch_t<double, 0, TS_MAC_BH, false, 1, 2, true>(c, P)
                  : launch_t<double, 0, TS_MAC_APE, false, 1, 2, true>(c, P);
    return bh ? launch_t<double, 1, TS_MAC_BH, false, 1, 2, true>(c, P)
              : launch_t<double, 1, TS_MAC_APE, false, 1, 2, true>(c, P);
}
