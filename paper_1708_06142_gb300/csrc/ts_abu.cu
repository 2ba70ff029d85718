// Adaptive Block Update (Sec. 2.2.6) and the block workload weights.
//
// A call walks only the 8 corner cells of every leaf-block (a target list in space-filling-curve
// order of the corners' positions, 32 neighbouring corners per warp),
// compares their new potential and acceleration with the previous values held in the output
// arrays, and walks in full only the leaf-blocks whose corners changed by at least the tolerance
// (a device-built list of their warps; the grid covers every warp and the surplus warps return).
// Blocks that pass keep their previous values in every cell.  No host round trip between the
// phases.  The workload weight of each leaf-block follows the paper's recurrence on the
// interactions of its last full walk.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ts_walk_dev.cuh"

cudaError_t make_walk_params(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc, WalkParams* out, int* bck_out);
cudaError_t launch_walk_params(ts_ctx* c, const ts_gravity_params* p, const WalkParams& P, int bck, int T);

namespace {

// natural in-block index k*64 + j*8 + i and Morton slot of the 8 corners (i, j, k in {0, 7}),
// corner c = (c & 1 ? i = 7) + (c & 2 ? j = 7) + (c & 4 ? k = 7)
__constant__ int c_corner_nat[8];

int morton_slot(int i, int j, int k) {
    const int q = (i >> 2) | ((j >> 2) << 1) | ((k >> 2) << 2);
    const int o = ((i >> 1) & 1) | (((j >> 1) & 1) << 1) | (((k >> 1) & 1) << 2);
    const int o2 = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return 64 * q + 8 * o + o2;
}

template <typename R>
__global__ void k_abu_compare(int nleaf, const int* __restrict__ slot, const R* __restrict__ pc,
                              const R* __restrict__ ac, const R* __restrict__ pot_old, const R* __restrict__ acc_old,
                              double a_tol, double phi_tol, int* __restrict__ warps, int* __restrict__ count) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nleaf) return;
    bool keep = true;
    for (int k = 0; k < 8; ++k) {
        const int64_t li = slot[(int64_t)n * 8 + k], nat = (int64_t)n * TS_NCB + c_corner_nat[k];
        const double dx = (double)ac[3 * li] - (double)acc_old[3 * nat];
        const double dy = (double)ac[3 * li + 1] - (double)acc_old[3 * nat + 1];
        const double dz = (double)ac[3 * li + 2] - (double)acc_old[3 * nat + 2];
        keep = keep && sqrt(dx * dx + dy * dy + dz * dz) < a_tol;
        if (phi_tol > 0) keep = keep && fabs((double)pc[li] - (double)pot_old[nat]) < phi_tol;
    }
    if (!keep) {
        const int s = atomicAdd(&count[0], 16);
        atomicAdd(&count[1], 1);
        for (int w = 0; w < 16; ++w) warps[s + w] = n * 16 + w;
    }
}

// W = W e^(-1/tau) + (1 - e^(-1/tau)) (2 + omega N / N_max); one CTA
__global__ void k_workload(int nleaf, const unsigned long long* __restrict__ nint, double* __restrict__ w, double f,
                           double omega) {
    __shared__ unsigned long long smax[32];
    unsigned long long m = 0;
    for (int n = threadIdx.x; n < nleaf; n += blockDim.x) m = max(m, nint[n]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = max(m, smax[i]);
    const double nmax = m ? (double)m : 1.0;
    for (int n = threadIdx.x; n < nleaf; n += blockDim.x)
        w[n] = w[n] * f + (1.0 - f) * (2.0 + omega * (double)nint[n] / nmax);
}

__global__ void k_fill(double* w, int n, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = v;
}

// 63-bit Morton key of a point of the unit cube (21 bits per axis)
uint64_t morton_key(double x, double y, double z) {
    auto spread = [](uint64_t v) {
        v &= 0x1fffff;
        v = (v | v << 32) & 0x1f00000000ffffull;
        v = (v | v << 16) & 0x1f0000ff0000ffull;
        v = (v | v << 8) & 0x100f00f00f00f00full;
        v = (v | v << 4) & 0x10c30c30c30c30c3ull;
        v = (v | v << 2) & 0x1249249249249249ull;
        return v;
    };
    auto q = [](double t) { return (uint64_t)std::min(std::max(t, 0.0) * 2097152.0, 2097151.0); };
    return spread(q(x)) | spread(q(y)) << 1 | spread(q(z)) << 2;
}

// Copies of each corner target in the list: a warp then walks for 32 / TS_ABU_SPREAD distinct
// corners (copies share their whole walk, so they add no pops), which spreads the few corner
// targets (8 per leaf-block) over more warps.  On the 2M-cell Plummer mesh (4096 leaf-blocks) the
// decision walk takes 1.05 / 0.86 / 0.75 / 0.89 ms with 1 / 2 / 4 / 8 copies.
#ifndef TS_ABU_SPREAD
#define TS_ABU_SPREAD 4
#endif

ts_status ensure_abu(ts_ctx* c) {
    if (c->d_abu_targets) return TS_OK;
    constexpr int S = TS_ABU_SPREAD;
    const int64_t nc = 8 * (int64_t)c->nleaf, ntp = (S * nc + 31) / 32 * 32;
    // the corner cells in space-filling-curve order of their positions, so that the 32 targets of a
    // warp are neighbours (corners of adjacent blocks) and share most of their walk;
    // slot[8 n + k] = position of corner k of leaf-block n in that list
    std::vector<double> lo(3 * (size_t)c->nleaf), sz(3 * (size_t)c->nleaf);
    TS_CUDA(cudaMemcpy(lo.data(), c->d_leaf_lo, sizeof(double) * lo.size(), cudaMemcpyDeviceToHost));
    TS_CUDA(cudaMemcpy(sz.data(), c->d_leaf_size, sizeof(double) * sz.size(), cudaMemcpyDeviceToHost));
    std::vector<std::pair<uint64_t, int64_t>> key(nc);
    int nat[8];
    for (int k = 0; k < 8; ++k) {
        const int i = (k & 1) ? 7 : 0, j = (k & 2) ? 7 : 0, kk = (k & 4) ? 7 : 0;
        nat[k] = kk * 64 + j * 8 + i;
        for (int n = 0; n < c->nleaf; ++n) {
            const double* l = &lo[3 * (size_t)n];
            const double* e = &sz[3 * (size_t)n];
            const double x = (l[0] + (i + 0.5) * e[0] / 8 - c->dlo[0]) / c->L[0];
            const double y = (l[1] + (j + 0.5) * e[1] / 8 - c->dlo[1]) / c->L[1];
            const double z = (l[2] + (kk + 0.5) * e[2] / 8 - c->dlo[2]) / c->L[2];
            key[(int64_t)n * 8 + k] = {morton_key(x, y, z), (int64_t)n * 8 + k};
        }
    }
    std::stable_sort(key.begin(), key.end());
    std::vector<int64_t> tg(ntp);
    std::vector<int> slot(nc);
    for (int64_t t = 0; t < nc; ++t) {
        const int64_t nk = key[t].second;
        const int n = (int)(nk / 8), k = (int)(nk % 8);
        for (int r = 0; r < S; ++r)
            tg[S * t + r] = (int64_t)n * TS_NCB + morton_slot((k & 1) ? 7 : 0, (k & 2) ? 7 : 0, (k & 4) ? 7 : 0);
        slot[nk] = (int)(S * t);
    }
    for (int64_t t = S * nc; t < ntp; ++t) tg[t] = tg[S * nc - 1];   // padding: repeats, results ignored
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(ts_malloc((void**)&c->d_abu_slot, sizeof(int) * nc));
    chk(cudaMemcpyAsync(c->d_abu_slot, slot.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, c->stream));
    chk(ts_malloc((void**)&c->d_abu_targets, sizeof(int64_t) * ntp));
    chk(ts_malloc(&c->d_abu_out, sizeof(double) * 4 * ntp));
    chk(ts_malloc((void**)&c->d_abu_warps, sizeof(int) * 16 * (size_t)c->nleaf));
    chk(ts_malloc((void**)&c->d_abu_count, sizeof(int) * 2));
    chk(ts_malloc((void**)&c->d_blk_counts, sizeof(unsigned long long) * c->nleaf));
    chk(ts_malloc((void**)&c->d_workload, sizeof(double) * c->nleaf));
    chk(cudaMemcpyToSymbolAsync(c_corner_nat, nat, sizeof(nat), 0, cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(c->d_abu_targets, tg.data(), sizeof(int64_t) * ntp, cudaMemcpyHostToDevice, c->stream));
    if (e == cudaSuccess) {
        k_fill<<<std::min((c->nleaf + 255) / 256, 1024), 256, 0, c->stream>>>(c->d_workload, c->nleaf, 2.0);
        e = cudaGetLastError();
    }
    chk(cudaStreamSynchronize(c->stream));   // tg and slot must outlive the copies
    if (e != cudaSuccess) {
        free_abu(c);
        return ts_cuda_fail(e, "ts_gravity_walk_abu: scratch");
    }
    c->abu_ntp = ntp;
    return TS_OK;
}

}  // namespace

void free_abu(ts_ctx* c) {
    auto f = [](auto*& p) { if (p) cudaFree((void*)p); p = nullptr; };
    f(c->d_abu_targets); f(c->d_abu_out); f(c->d_abu_warps); f(c->d_abu_count); f(c->d_blk_counts);
    f(c->d_workload); f(c->d_abu_slot);
    c->abu_ntp = 0;
}

extern "C" ts_status ts_gravity_walk_abu(ts_ctx* c, const ts_gravity_params* p, double a_tol, double phi_tol,
                                         void* pot, void* acc, int32_t* n_updated) {
    FaultSite fault_site("abu");
    if (!c || !p) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk_abu: NULL ctx or params");
    if (!pot || !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk_abu: NULL potential or acceleration");
    if (!(a_tol >= 0) || isnan(phi_tol)) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk_abu: a_tol must be >= 0");
    ts_status vs = validate_gravity(c, p);
    if (vs != TS_OK) return vs;
    if (p->accel != TS_ACCEL_DIRECT)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk_abu: the block update compares directly summed accelerations");
    if (p->mac == TS_MAC_SUMSQ)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk_abu: the block update runs the warp-shared walks");
    DeviceGuard g(c->device);
    const int kind = (c->bc[0] || c->bc[1] || c->bc[2]) ? 1 : 0;
    if (kind && p->ewald == TS_EWALD_TAYLOR && (vs = ensure_taylor(c)) != TS_OK) return vs;
    if (p->mac == TS_MAC_MPE && (vs = ensure_bmoments(c, p->precision == TS_PREC_FP64)) != TS_OK) return vs;
    if ((vs = ensure_abu(c)) != TS_OK) return vs;
    const bool fp64 = p->precision == TS_PREC_FP64;
    const size_t rs = fp64 ? sizeof(double) : sizeof(float);
    char* tmp = (char*)c->d_abu_out;
    cudaError_t e = cudaMemsetAsync(c->d_counters, 0, 4 * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_abu_count, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_blk_counts, 0, sizeof(unsigned long long) * c->nleaf, c->stream);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_gravity_walk_abu: reset");
    cudaEventRecord(c->ev0, c->stream);
    // phase 1: the corner cells of every leaf-block
    WalkParams P;
    int bck = 0;
    e = make_walk_params(c, p, tmp, tmp + rs * c->abu_ntp, &P, &bck);
    P.targets = c->d_abu_targets;
    P.ntargets = c->abu_ntp;
    if (e == cudaSuccess) e = launch_walk_params(c, p, P, bck, 1);
    // compare with the previous values; list the warps of the blocks to update
    if (e == cudaSuccess) {
        const int grid = (c->nleaf + 127) / 128;
        if (fp64)
            k_abu_compare<double><<<grid, 128, 0, c->stream>>>(c->nleaf, c->d_abu_slot, (const double*)tmp,
                                                               (const double*)(tmp + rs * c->abu_ntp), (const double*)pot,
                                                               (const double*)acc, a_tol, phi_tol, c->d_abu_warps,
                                                               c->d_abu_count);
        else
            k_abu_compare<float><<<grid, 128, 0, c->stream>>>(c->nleaf, c->d_abu_slot, (const float*)tmp,
                                                              (const float*)(tmp + rs * c->abu_ntp), (const float*)pot,
                                                              (const float*)acc, a_tol, phi_tol, c->d_abu_warps,
                                                              c->d_abu_count);
        e = cudaGetLastError();
    }
    // phase 2: the full walk of the listed warps, in place
    if (e == cudaSuccess) e = make_walk_params(c, p, pot, acc, &P, &bck);
    P.warp_list = c->d_abu_warps;
    P.nwarp_dev = c->d_abu_count;
    P.blk_counts = c->d_blk_counts;
    if (e == cudaSuccess) e = launch_walk_params(c, p, P, bck, 1);
    cudaEventRecord(c->ev1, c->stream);
    c->timed = true;
    if (e == cudaSuccess) {
        k_workload<<<1, 1024, 0, c->stream>>>(c->nleaf, c->d_blk_counts, c->d_workload, exp(-1.0 / 10.0), 8.0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p->zero_mean) e = launch_zero_mean(c, p->precision, pot);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_gravity_walk_abu: kernels");
    if (n_updated) {
        int h[2] = {0, 0};
        TS_CUDA(cudaMemcpyAsync(h, c->d_abu_count, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        TS_CUDA(cudaStreamSynchronize(c->stream));
        *n_updated = h[1];
    }
    return TS_OK;
}

extern "C" ts_status ts_block_workload(ts_ctx* c, double* w) {
    if (!c || !w) return ts_fail(TS_ERR_INVALID_ARG, "ts_block_workload: NULL argument");
    if (!c->d_workload) return ts_fail(TS_ERR_NOT_BUILT, "ts_block_workload: no adaptive-block-update walk yet");
    DeviceGuard g(c->device);
    TS_CUDA(cudaMemcpyAsync(w, c->d_workload, sizeof(double) * c->nleaf, cudaMemcpyDeviceToHost, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    return TS_OK;
}
