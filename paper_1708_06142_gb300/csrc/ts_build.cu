// Tree build (Sec. 2.1): cell masses and bottom-up FP64 node moments.
//
// k_blocktree: one CTA of 512 threads per leaf-block.  Each thread reads one density value
// (coalesced, natural cell order), forms m = rho dV and the cell centre in FP64, and stores them
// in shared memory at the cell's Morton slot.  The 64 level-2 nodes, 8 level-1 nodes and the
// leaf-block node are then summed in shared memory, children in octant order.  Products and sums
// use explicitly rounded FP64 operations (no FMA contraction), so masses and centres of mass are
// reproducible bit for bit by any implementation that sums in the same order.
// k_amr_reduce: one CTA walks the amr-tree from the deepest level to the root; each non-leaf
// block sums its 8 contiguous children.
// Both also write the FP32 records of every group of 8 siblings structure-of-arrays (x[8], y[8],
// z[8], m[8]) for the paired FP32 walk: cell group g = cells 8g..8g+7, node group g = nodes
// 1+8g..8+8g (node ids are breadth-first, so every child group starts at 1 mod 8).
// With the FP64 records switched off (ts_tree_fp64_records) the FP64 cell records and the FP64
// records of the nodes inside leaf-blocks are not written; those of the leaf-block and amr-tree
// nodes are (the amr sums read them).
//
// Roofline: bound by GB300's FP64 rate (1/64 of FP32; HBM-bound only once that arithmetic is
// cheap).  Per cell it reads 8 B of density and writes a 16 B FP32 record, its 16 B sibling-group
// copy and a 32 B FP64 record (none with the FP64 records off); per leaf-block 72 + 1 internal
// records of 16 + 16 + 32 B (16 + 16 B for the 72 with the FP64 records off).
#include <algorithm>

#include "ts_internal.cuh"

__device__ __forceinline__ int morton_of(int i, int j, int k) {
    // cell (i,j,k) in [0,8)^3 -> 64 q + 8 o + o2 with octant bits (x, y, z) at each level
    int q = (i >> 2) | ((j >> 2) << 1) | ((k >> 2) << 2);
    int o = ((i >> 1) & 1) | (((j >> 1) & 1) << 1) | (((k >> 1) & 1) << 2);
    int o2 = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return 64 * q + 8 * o + o2;
}

struct Mom {
    double m, sx, sy, sz;
};

__device__ __forceinline__ void mom_add(Mom& a, double m, double x, double y, double z) {
    a.m = __dadd_rn(a.m, m);
    a.sx = __dadd_rn(a.sx, __dmul_rn(m, x));
    a.sy = __dadd_rn(a.sy, __dmul_rn(m, y));
    a.sz = __dadd_rn(a.sz, __dmul_rn(m, z));
}

// node nid >= 1 is sibling (nid - 1) % 8 of node group (nid - 1) / 8; the root belongs to none
__device__ __forceinline__ void store_soa(float* soa, int64_t g, int j, float x, float y, float z, float m) {
    float* q = soa + 32 * g + j;
    q[0] = x; q[8] = y; q[16] = z; q[24] = m;
}

__device__ __forceinline__ dbl4 store_node(float4* n32, dbl4* n64, float* soa, int nid, const Mom& a, const dbl4& cen,
                                           bool w64 = true) {
    double x, y, z;
    if (a.m > 0) {
        x = __ddiv_rn(a.sx, a.m); y = __ddiv_rn(a.sy, a.m); z = __ddiv_rn(a.sz, a.m);
    } else {
        x = cen.x; y = cen.y; z = cen.z;   // empty node: centre of mass := geometric centre
    }
    const dbl4 r{x, y, z, a.m};
    if (w64) n64[nid] = r;
    n32[nid] = make_float4((float)x, (float)y, (float)z, (float)a.m);
    if (nid > 0) store_soa(soa, (nid - 1) >> 3, (nid - 1) & 7, (float)x, (float)y, (float)z, (float)a.m);
    return r;
}

__global__ void __launch_bounds__(512) k_blocktree(const double* __restrict__ rho, const double* __restrict__ leaf_lo,
                                                   const double* __restrict__ leaf_size, const int* __restrict__ leaf_nid,
                                                   const dbl4* __restrict__ ncen64, int nb, float4* __restrict__ cell32,
                                                   dbl4* __restrict__ cell64, float4* __restrict__ ncom32,
                                                   dbl4* __restrict__ ncom64, float* __restrict__ cellsoa,
                                                   float* __restrict__ ncomsoa, int full64) {
    __shared__ double sm[512], sx[512], sy[512], sz[512];
    __shared__ double l2m[64], l2x[64], l2y[64], l2z[64];
    __shared__ double l1m[8], l1x[8], l1y[8], l1z[8];
    __shared__ double s_cc[3][8], s_dv;
    const int n = blockIdx.x, t = threadIdx.x;
    const int i = t & 7, j = (t >> 3) & 7, k = t >> 6;
    // The 8 cell-centre coordinates per axis and the cell volume, computed once per leaf-block (the
    // kernel is bound by GB300's FP64 rate).  x / 8 and x * 0.125 are the same exact scaling by a
    // power of two, so the results are bit-identical to lo + (i + 1/2) e / 8 and (e/8)^3.
    if (t < 24) {
        const int a = t >> 3, c = t & 7;
        s_cc[a][c] = __dadd_rn(leaf_lo[3 * n + a], __dmul_rn(__dmul_rn(c + 0.5, leaf_size[3 * n + a]), 0.125));
    } else if (t == 32) {
        const double ex = leaf_size[3 * n], ey = leaf_size[3 * n + 1], ez = leaf_size[3 * n + 2];
        s_dv = __dmul_rn(__dmul_rn(__dmul_rn(ex, 0.125), __dmul_rn(ey, 0.125)), __dmul_rn(ez, 0.125));
    }
    __syncthreads();
    const double m = __dmul_rn(rho[(size_t)n * TS_NCB + t], s_dv);
    const double x = s_cc[0][i], y = s_cc[1][j], z = s_cc[2][k];
    const int mt = morton_of(i, j, k);
    sm[mt] = m; sx[mt] = x; sy[mt] = y; sz[mt] = z;
    __syncthreads();
    // cell records in Morton order (coalesced)
    {
        const size_t id = (size_t)n * TS_NCB + t;
        if (full64) cell64[id] = dbl4{sx[t], sy[t], sz[t], sm[t]};
        cell32[id] = make_float4((float)sx[t], (float)sy[t], (float)sz[t], (float)sm[t]);
        store_soa(cellsoa, (int64_t)(id >> 3), t & 7, (float)sx[t], (float)sy[t], (float)sz[t], (float)sm[t]);
    }
    const int base = nb + 72 * n;
    if (t < 64) {   // level-2 node g = 8 q + o: cells 8 g .. 8 g + 7
        Mom a{0, 0, 0, 0};
        for (int c = 0; c < 8; ++c) mom_add(a, sm[8 * t + c], sx[8 * t + c], sy[8 * t + c], sz[8 * t + c]);
        const int nid = base + 8 + t;
        const dbl4 r = store_node(ncom32, ncom64, ncomsoa, nid, a, ncen64[nid], full64);
        l2m[t] = a.m;
        l2x[t] = r.x; l2y[t] = r.y; l2z[t] = r.z;
    }
    __syncthreads();
    if (t < 8) {    // level-1 node q: level-2 nodes 8 q .. 8 q + 7
        Mom a{0, 0, 0, 0};
        for (int c = 0; c < 8; ++c) mom_add(a, l2m[8 * t + c], l2x[8 * t + c], l2y[8 * t + c], l2z[8 * t + c]);
        const int nid = base + t;
        const dbl4 r = store_node(ncom32, ncom64, ncomsoa, nid, a, ncen64[nid], full64);
        l1m[t] = a.m;
        l1x[t] = r.x; l1y[t] = r.y; l1z[t] = r.z;
    }
    __syncthreads();
    if (t == 0) {   // the leaf-block node itself
        Mom a{0, 0, 0, 0};
        for (int c = 0; c < 8; ++c) mom_add(a, l1m[c], l1x[c], l1y[c], l1z[c]);
        const int nid = leaf_nid[n];
        store_node(ncom32, ncom64, ncomsoa, nid, a, ncen64[nid]);
    }
}

__global__ void __launch_bounds__(256) k_amr_reduce(const int* __restrict__ order, const int* __restrict__ level_off,
                                                    int nrounds, const dbl4* __restrict__ ncen64,
                                                    float4* __restrict__ ncom32, dbl4* __restrict__ ncom64,
                                                    float* __restrict__ ncomsoa) {
    for (int r = 0; r < nrounds; ++r) {
        for (int idx = level_off[r] + threadIdx.x; idx < level_off[r + 1]; idx += blockDim.x) {
            const int nid = order[idx];
            const dbl4 cen = ncen64[nid];
            uint32_t cw = (uint32_t)cen.w;
            const int first = (int)(cw & TS_CW_INDEX_MASK);
            Mom a{0, 0, 0, 0};
            for (int c = 0; c < 8; ++c) {
                const dbl4 ch = ncom64[first + c];
                mom_add(a, ch.w, ch.x, ch.y, ch.z);
            }
            store_node(ncom32, ncom64, ncomsoa, nid, a, cen);
        }
        __syncthreads();
        __threadfence_block();
    }
}

cudaError_t launch_tree_build(ts_ctx* c, const double* density) {
    k_blocktree<<<c->nleaf, 512, 0, c->stream>>>(density, c->d_leaf_lo, c->d_leaf_size, c->d_leaf_nid, c->d_ncen64,
                                                 c->nb, c->d_cell32, c->d_cell64, c->d_ncom32, c->d_ncom64,
                                                 (float*)c->d_cellsoa, (float*)c->d_ncomsoa, c->rec64 ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the level offsets are stored after the node ids in the same device array
    const int nrounds = (int)c->amr_level_off.size() - 1;
    if (nrounds > 0 && !c->amr_order.empty()) {
        k_amr_reduce<<<1, 256, 0, c->stream>>>(c->d_amr_order, c->d_amr_order + c->amr_order.size(), nrounds,
                                               c->d_ncen64, c->d_ncom32, c->d_ncom64, (float*)c->d_ncomsoa);
        e = cudaGetLastError();
    }
    return e;
}

// ------------------------------------------------------------------------------ MPE moments
// B_p = sum_i m_i |r_i - r_a|^p (p = 2, 3) over the cells of a node (Sec. 2.2.1, eq. mpe).
// One CTA per leaf-block: each thread holds one cell (Morton order) and adds its terms about the
// centre of mass of each of its ancestors: its level-2 node (8 consecutive threads), level-1 node
// (64), the leaf-block node (512, stored) and every amr ancestor (512 per leaf-block, FP64 atomics
// onto zeroed accumulators).  R is the arithmetic of the terms and of the sums within the CTA:
// double for the FP64 walk; float for the FP32 walk, whose MAC compares the moments in FP32 anyway
// (the FP64 pipe runs at 1/64 of the FP32 rate, and these terms need an FP64 square root each).
template <typename R> struct BM;
template <> struct BM<double> { typedef dbl4 V; typedef double2 P; };
template <> struct BM<float> { typedef float4 V; typedef float2 P; };

__device__ __forceinline__ double2 bterm(const dbl4& cell, const dbl4& ra) {
    const double dx = __dsub_rn(cell.x, ra.x), dy = __dsub_rn(cell.y, ra.y), dz = __dsub_rn(cell.z, ra.z);
    const double u = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double b2 = __dmul_rn(cell.w, u);
    return make_double2(b2, __dmul_rn(b2, sqrt(u)));
}

__device__ __forceinline__ float2 bterm(const float4& cell, const float4& ra) {
    const float dx = cell.x - ra.x, dy = cell.y - ra.y, dz = cell.z - ra.z;
    const float u = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float b2 = cell.w * u;
    return make_float2(b2, b2 * sqrtf(u));
}

template <typename P>
__device__ __forceinline__ P warp_sum2(P v, int width) {
    for (int o = width / 2; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// block-wide sum of 512 threads (16 warps), valid in thread 0; every thread must call it
template <typename P>
__device__ P block_sum2(P v, P* sm) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    v = warp_sum2(v, 32);
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < 16 ? sm[l] : P{0, 0};
        v = warp_sum2(v, 16);
    }
    return v;
}

template <typename R>
__global__ void __launch_bounds__(512) k_bmoments(const typename BM<R>::V* __restrict__ cell,
                                                  const typename BM<R>::V* __restrict__ ncom,
                                                  const int* __restrict__ leaf_nid, const int* __restrict__ anc,
                                                  int anc_max, int nb, double2* __restrict__ bm) {
    typedef typename BM<R>::P P;
    __shared__ P sm[16];
    __shared__ P l1[8][2];
    const int n = blockIdx.x, t = threadIdx.x;
    const typename BM<R>::V c = cell[(size_t)n * TS_NCB + t];
    const int base = nb + 72 * n;
    // level-2 node g = t / 8
    P v = warp_sum2(bterm(c, ncom[base + 8 + (t >> 3)]), 8);
    if ((t & 7) == 0) bm[base + 8 + (t >> 3)] = make_double2(v.x, v.y);
    // level-1 node q = t / 64: two warps
    v = warp_sum2(bterm(c, ncom[base + (t >> 6)]), 32);
    if ((t & 31) == 0) l1[t >> 6][(t >> 5) & 1] = v;
    __syncthreads();
    if (t < 8) bm[base + t] = make_double2((double)l1[t][0].x + (double)l1[t][1].x, (double)l1[t][0].y + (double)l1[t][1].y);
    // the leaf-block node
    const int leaf = leaf_nid[n];
    v = block_sum2(bterm(c, ncom[leaf]), sm);
    if (t == 0) bm[leaf] = make_double2(v.x, v.y);
    // amr ancestors
    for (int a = 0; a < anc_max; ++a) {
        const int id = anc[(size_t)n * anc_max + a];
        if (id < 0) break;   // uniform across the CTA
        v = block_sum2(bterm(c, ncom[id]), sm);
        if (t == 0) {
            atomicAdd(&bm[id].x, (double)v.x);
            atomicAdd(&bm[id].y, (double)v.y);
        }
    }
}

__global__ void k_bmoments_f32(const double2* __restrict__ bm, int nint, float2* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x)
        out[i] = make_float2((float)bm[i].x, (float)bm[i].y);
}

cudaError_t launch_bmoments(ts_ctx* c, bool fp64) {
    cudaError_t e = cudaMemsetAsync(c->d_bmom64, 0, sizeof(double2) * c->nb, c->stream);   // amr accumulators
    if (e != cudaSuccess) return e;
    if (fp64)
        k_bmoments<double><<<c->nleaf, 512, 0, c->stream>>>(c->d_cell64, c->d_ncom64, c->d_leaf_nid, c->d_leaf_anc,
                                                            c->anc_max, c->nb, c->d_bmom64);
    else
        k_bmoments<float><<<c->nleaf, 512, 0, c->stream>>>(c->d_cell32, c->d_ncom32, c->d_leaf_nid, c->d_leaf_anc,
                                                           c->anc_max, c->nb, c->d_bmom64);
    k_bmoments_f32<<<std::min((c->nint + 255) / 256, 152 * 8), 256, 0, c->stream>>>(c->d_bmom64, c->nint, c->d_bmom32);
    return cudaGetLastError();
}
