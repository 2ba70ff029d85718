// Calls for a mesh partitioned over several GPUs (one process per GPU).
//
// The walk of a target cell reads only the tree (Sec. 2.1), so the cells of a mesh split into
// independent units.  A rank owns a contiguous range of leaf-blocks in the mesh's block order,
// which for the meshes of Sec. 2 is the Morton order of the blocks; ranges of equal estimated cost
// come from the interactions of each block's previous walk (the paper balances its MPI domains on
// the same per-block work, Sec. 2.2.6).  The only exchanges are around the walk: every rank needs
// the whole tree (here: the densities of all blocks gathered, then a replicated tree build), and
// the zero mean of a periodic potential needs the FP64 sums (sum dV phi, sum dV) of all ranks.
//   ts_gravity_walk_range   the walk of one range's cells (per-block interaction counts recorded)
//   ts_walk_block_counts    those counts, the cost of the next partition
//   ts_potential_sums       the range's FP64 sums for the zero mean (to be summed over ranks)
//   ts_potential_shift      subtract the global mean over the range
#include <math.h>

#include <algorithm>
#include <vector>

#include "ts_walk_dev.cuh"

cudaError_t make_walk_params(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc, WalkParams* out, int* bck_out);
cudaError_t launch_walk_params(ts_ctx* c, const ts_gravity_params* p, const WalkParams& P, int bck, int T);

static ts_status check_range(ts_ctx* c, int32_t b, int32_t e, const char* who) {
    if (!c->have_tree) return ts_fail(TS_ERR_NOT_BUILT, std::string(who) + ": call ts_tree_build first");
    if (b < 0 || e < b || e > c->nleaf)
        return ts_fail(TS_ERR_INVALID_ARG, std::string(who) + ": need 0 <= leaf_begin <= leaf_end <= nleaf");
    return TS_OK;
}

extern "C" ts_status ts_gravity_walk_range(ts_ctx* c, const ts_gravity_params* p, int32_t leaf_begin, int32_t leaf_end,
                                           void* pot, void* acc) {
    FaultSite fault_site("walk");
    if (!c || !p || !pot || !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk_range: NULL argument");
    ts_status s = check_range(c, leaf_begin, leaf_end, "ts_gravity_walk_range");
    if (s != TS_OK) return s;
    s = validate_gravity(c, p);
    if (s != TS_OK) return s;
    if (p->zero_mean)
        return ts_fail(TS_ERR_INVALID_ARG,
                       "ts_gravity_walk_range: the zero mean needs every range (ts_potential_sums, ts_potential_shift)");
    if (p->accel != TS_ACCEL_DIRECT)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk_range: differences across ranges need the neighbours' potential");
    if (p->mac == TS_MAC_SUMSQ)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk_range: ranges run the warp-shared walks");
    DeviceGuard g(c->device);
    if (ew_kind(c->bc) != TS_EW_NONE && p->ewald == TS_EWALD_TAYLOR) {
        s = ensure_taylor(c);
        if (s != TS_OK) return s;
    }
    if (p->mac == TS_MAC_MPE) {
        s = ensure_bmoments(c, p->precision == TS_PREC_FP64);
        if (s != TS_OK) return s;
    }
    cudaError_t e = cudaSuccess;
    if (!c->d_range_counts) e = ts_malloc((void**)&c->d_range_counts, sizeof(unsigned long long) * c->nleaf);
    if (e == cudaSuccess && !c->range_counts_valid) {
        e = cudaMemsetAsync(c->d_range_counts, 0, sizeof(unsigned long long) * c->nleaf, c->stream);
        c->range_counts_valid = true;
    }
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_gravity_walk_range: counters");
    if (leaf_end == leaf_begin) return TS_OK;
    WalkParams P;
    int bck = 0;
    e = make_walk_params(c, p, pot, acc, &P, &bck);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_range_counts + leaf_begin, 0, sizeof(unsigned long long) * (leaf_end - leaf_begin),
                            c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, 4 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_gravity_walk_range: setup");
    P.leaf_begin = leaf_begin;
    P.leaf_end = leaf_end;
    P.blk_counts = c->d_range_counts;
    cudaEventRecord(c->ev0, c->stream);
    e = launch_walk_params(c, p, P, bck, 1);
    cudaEventRecord(c->ev1, c->stream);
    c->timed = true;
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_gravity_walk_range: walk kernel");
    return TS_OK;
}

extern "C" ts_status ts_walk_block_counts(ts_ctx* c, int64_t* counts) {
    if (!c || !counts) return ts_fail(TS_ERR_INVALID_ARG, "ts_walk_block_counts: NULL argument");
    if (!c->have_tree || !c->d_range_counts || !c->range_counts_valid)
        return ts_fail(TS_ERR_NOT_BUILT, "ts_walk_block_counts: no ts_gravity_walk_range since the mesh was ingested");
    DeviceGuard g(c->device);
    std::vector<unsigned long long> h(c->nleaf);
    TS_CUDA(cudaMemcpyAsync(h.data(), c->d_range_counts, sizeof(unsigned long long) * c->nleaf, cudaMemcpyDeviceToHost,
                            c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    for (int n = 0; n < c->nleaf; ++n) counts[n] = (int64_t)h[n];
    return TS_OK;
}

// FP64 sums (sum dV phi, sum dV) over the cells of leaf-blocks [b, e), one CTA per block, summed
// into out[0..1] in a fixed order by a second pass (deterministic for a given partition).
template <typename R>
__global__ void __launch_bounds__(256) k_range_sums(const R* __restrict__ pot, const double* __restrict__ leaf_size,
                                                    int b, double* __restrict__ part) {
    const int n = b + blockIdx.x;
    const double dv = leaf_size[3 * n] * leaf_size[3 * n + 1] * leaf_size[3 * n + 2] / 512.0;
    double s = 0;
    for (int i = threadIdx.x; i < 512; i += blockDim.x) s += (double)pot[(int64_t)n * 512 + i];
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[2 * blockIdx.x] = dv * t;
        part[2 * blockIdx.x + 1] = dv * 512.0;
    }
}

__global__ void __launch_bounds__(32) k_range_total(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    double s = 0, v = 0;
    for (int k = threadIdx.x; k < nblk; k += 32) {
        s += part[2 * k];
        v += part[2 * k + 1];
    }
    for (int off = 16; off; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    if (threadIdx.x == 0) {
        out[0] = s;
        out[1] = v;
    }
}

template <typename R>
__global__ void k_range_shift(R* __restrict__ pot, int64_t i0, int64_t i1, double shift) {
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x)
        pot[i] = (R)((double)pot[i] - shift);
}

extern "C" ts_status ts_potential_sums(ts_ctx* c, int32_t precision, const void* pot, int32_t leaf_begin, int32_t leaf_end,
                                       double* sums) {
    if (!c || !pot || !sums) return ts_fail(TS_ERR_INVALID_ARG, "ts_potential_sums: NULL argument");
    if (precision != TS_PREC_FP64 && precision != TS_PREC_FP32_KAHAN)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_potential_sums: unknown precision");
    ts_status s = check_range(c, leaf_begin, leaf_end, "ts_potential_sums");
    if (s != TS_OK) return s;
    sums[0] = sums[1] = 0;
    const int nblk = leaf_end - leaf_begin;
    if (nblk == 0) return TS_OK;
    DeviceGuard g(c->device);
    FaultSite fault_site("walk");
    if (c->range_part_cap < nblk) {
        if (c->d_range_part) cudaFree(c->d_range_part);
        c->d_range_part = nullptr;
        c->range_part_cap = 0;
        TS_CUDA(ts_malloc((void**)&c->d_range_part, sizeof(double) * (2 * (size_t)nblk + 2)));
        c->range_part_cap = nblk;
    }
    if (precision == TS_PREC_FP64)
        k_range_sums<double><<<nblk, 256, 0, c->stream>>>((const double*)pot, c->d_leaf_size, leaf_begin, c->d_range_part);
    else
        k_range_sums<float><<<nblk, 256, 0, c->stream>>>((const float*)pot, c->d_leaf_size, leaf_begin, c->d_range_part);
    k_range_total<<<1, 32, 0, c->stream>>>(c->d_range_part, nblk, c->d_range_part + 2 * (size_t)nblk);
    TS_CUDA(cudaGetLastError());
    TS_CUDA(cudaMemcpyAsync(sums, c->d_range_part + 2 * (size_t)nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    return TS_OK;
}

extern "C" ts_status ts_potential_shift(ts_ctx* c, int32_t precision, void* pot, int32_t leaf_begin, int32_t leaf_end,
                                        double shift) {
    if (!c || !pot) return ts_fail(TS_ERR_INVALID_ARG, "ts_potential_shift: NULL argument");
    if (precision != TS_PREC_FP64 && precision != TS_PREC_FP32_KAHAN)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_potential_shift: unknown precision");
    if (!isfinite(shift)) return ts_fail(TS_ERR_INVALID_ARG, "ts_potential_shift: shift must be finite");
    ts_status s = check_range(c, leaf_begin, leaf_end, "ts_potential_shift");
    if (s != TS_OK) return s;
    if (leaf_end == leaf_begin) return TS_OK;
    DeviceGuard g(c->device);
    const int64_t i0 = (int64_t)leaf_begin * 512, i1 = (int64_t)leaf_end * 512;
    const int grid = (int)std::min<int64_t>((i1 - i0 + 255) / 256, 152 * 8);
    if (precision == TS_PREC_FP64)
        k_range_shift<double><<<grid, 256, 0, c->stream>>>((double*)pot, i0, i1, shift);
    else
        k_range_shift<float><<<grid, 256, 0, c->stream>>>((float*)pot, i0, i1, shift);
    TS_CUDA(cudaGetLastError());
    return TS_OK;
}
