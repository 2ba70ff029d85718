// Accuracy metrics of a walk against a reference solution (Sec. 3, eq. ea: the acceleration error
// of a cell normalised by the largest reference acceleration of the domain; the potential error is
// the same construction applied to the potential).
//
// All passes are grid-stride loops over the n entries in FP64.  The median and the 99th percentile
// need order statistics; they are selected exactly by an MSB-first radix selection on the FP64 bit
// patterns (non-negative doubles order like their bit patterns as unsigned integers): six passes of
// 11-bit digits, each a shared-memory histogram of the entries whose higher digits match the
// selected prefix, followed by a one-warp-per-selection scan that fixes the next digit.
#include <math.h>

#include "ts_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBins = 2048;   // 11-bit digits
constexpr int kSel = 4;       // order statistics selected together: median (2) and p99 (2)

struct ErrAux {
    double sum[2];                  // sum of phi, sum of phi_ref
    unsigned long long maxb[4];     // bit patterns of max |a_ref|, max |phi_ref|, max e_a, max e_phi
    unsigned long long nonfinite;
    unsigned long long prefix[kSel];
    unsigned long long mask[kSel];
    long long k[kSel];              // rank still to find below the selected prefix
    unsigned int hist[kSel][kBins];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// block-wide reductions; every thread of the block must call them
__device__ double block_sum(double v, double* sm) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? sm[threadIdx.x] : 0.0;
    return w == 0 ? warp_sum(v) : 0.0;
}

__device__ unsigned long long block_max(unsigned long long v, unsigned long long* sm) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? sm[threadIdx.x] : 0ull;
    return w == 0 ? warp_max(v) : 0ull;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
// a positive normaliser, or 1 (absolute errors) when the reference is identically zero
__device__ __forceinline__ double norm_of(unsigned long long b) { const double m = bitsd(b); return m > 0 ? m : 1.0; }

// pass 1: sums of both potentials, max |a_ref|
template <typename R>
__global__ void __launch_bounds__(kThreads) k_err_ref(int64_t n, const R* pot, const double* pref, const double* aref,
                                                      ErrAux* x) {
    __shared__ double sd[kThreads / 32];
    __shared__ unsigned long long su[kThreads / 32];
    double s0 = 0, s1 = 0, am = 0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        if (pot) { s0 += (double)pot[i]; s1 += pref[i]; }
        if (aref) {
            const double ax = aref[3 * i], ay = aref[3 * i + 1], az = aref[3 * i + 2];
            am = fmax(am, sqrt(ax * ax + ay * ay + az * az));
        }
    }
    s0 = block_sum(s0, sd);
    s1 = block_sum(s1, sd);
    const unsigned long long m = block_max(dbits(am), su);
    if (threadIdx.x == 0) {
        if (pot) { atomicAdd(&x->sum[0], s0); atomicAdd(&x->sum[1], s1); }
        atomicMax(&x->maxb[0], m);
    }
}

// pass 2: max |phi_ref - mean(phi_ref)| (mean taken only with mod_const)
__global__ void __launch_bounds__(kThreads) k_err_phimax(int64_t n, const double* pref, int mod_const, ErrAux* x) {
    __shared__ unsigned long long su[kThreads / 32];
    const double mr = mod_const ? x->sum[1] / (double)n : 0.0;
    double pm = 0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        pm = fmax(pm, fabs(pref[i] - mr));
    const unsigned long long m = block_max(dbits(pm), su);
    if (threadIdx.x == 0) atomicMax(&x->maxb[1], m);
}

// pass 3: the per-entry errors and their maxima
template <typename R>
__global__ void __launch_bounds__(kThreads) k_err_eval(int64_t n, const R* pot, const R* acc, const double* pref,
                                                       const double* aref, int mod_const, ErrAux* x, double* e) {
    __shared__ unsigned long long su[kThreads / 32];
    const double an = norm_of(x->maxb[0]), pn = norm_of(x->maxb[1]);
    const double mp = mod_const ? x->sum[0] / (double)n : 0.0, mr = mod_const ? x->sum[1] / (double)n : 0.0;
    unsigned long long ma = 0, mphi = 0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double ea = 0, ep = 0;
        if (acc) {
            const double dx = (double)acc[3 * i] - aref[3 * i], dy = (double)acc[3 * i + 1] - aref[3 * i + 1],
                         dz = (double)acc[3 * i + 2] - aref[3 * i + 2];
            ea = sqrt(dx * dx + dy * dy + dz * dz) / an;
        }
        if (pot) ep = fabs(((double)pot[i] - mp) - (pref[i] - mr)) / pn;
        ea = fabs(ea);   // a NaN keeps a clear sign bit and orders above +inf
        ep = fabs(ep);
        e[i] = ea;
        e[n + i] = ep;
        ma = max(ma, dbits(ea));
        mphi = max(mphi, dbits(ep));
    }
    ma = block_max(ma, su);
    mphi = block_max(mphi, su);
    if (threadIdx.x == 0) { atomicMax(&x->maxb[2], ma); atomicMax(&x->maxb[3], mphi); }
}

// pass 4: count of non-finite errors
__global__ void __launch_bounds__(kThreads) k_err_count(int64_t n, const double* e, ErrAux* x) {
    unsigned long long bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * kThreads)
        bad += !isfinite(e[i]);
    for (int o = 16; o; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&x->nonfinite, bad);
}

__global__ void k_sel_init(ErrAux* x, long long k0, long long k1, long long k2, long long k3) {
    const int s = threadIdx.x;
    if (s < kSel) {
        const long long k[kSel] = {k0, k1, k2, k3};
        x->prefix[s] = 0;
        x->mask[s] = 0;
        x->k[s] = k[s];
    }
    for (int i = threadIdx.x; i < kSel * kBins; i += blockDim.x) (&x->hist[0][0])[i] = 0;
}

// histogram of digit (b >> shift) & 2047 over the entries whose already-fixed bits match
__global__ void __launch_bounds__(kThreads) k_sel_hist(int64_t n, const double* v, ErrAux* x, int shift) {
    __shared__ unsigned int h[kSel][kBins];
    __shared__ unsigned long long pre[kSel], msk[kSel];
    for (int i = threadIdx.x; i < kSel * kBins; i += kThreads) (&h[0][0])[i] = 0;
    if (threadIdx.x < kSel) { pre[threadIdx.x] = x->prefix[threadIdx.x]; msk[threadIdx.x] = x->mask[threadIdx.x]; }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const unsigned long long b = dbits(v[i]);
        const unsigned d = (unsigned)(b >> shift) & (kBins - 1);
#pragma unroll
        for (int s = 0; s < kSel; ++s)
            if ((b & msk[s]) == pre[s]) atomicAdd(&h[s][d], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSel * kBins; i += kThreads) {
        const unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&x->hist[0][0])[i], c);
    }
}

// one warp per selection: find the digit whose cumulative count passes k, fix it, clear the histogram
__global__ void k_sel_scan(ErrAux* x, int shift) {
    const int s = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (s >= kSel) return;
    long long k = x->k[s], run = 0;
    int digit = -1;
    long long below = 0;
    for (int c0 = 0; c0 < kBins && digit < 0; c0 += 32) {
        const long long cnt = x->hist[s][c0 + l];
        long long inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (l >= o) inc += t;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, run + inc > k);
        if (hit) {
            const int j = __ffs(hit) - 1;
            digit = c0 + j;
            below = run + __shfl_sync(0xffffffffu, inc - cnt, j);
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    for (int c = l; c < kBins; c += 32) x->hist[s][c] = 0;
    if (l == 0 && digit >= 0) {
        x->prefix[s] |= (unsigned long long)digit << shift;
        x->mask[s] |= (unsigned long long)(kBins - 1) << shift;
        x->k[s] = k - below;
    }
}

int grid_for(int64_t n) {
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (int)(g < 152 * 8 ? (g > 0 ? g : 1) : 152 * 8);
}

// The four order statistics of v[0..n) at ranks r[4], as their values.
cudaError_t select4(cudaStream_t st, int64_t n, const double* v, ErrAux* x, const long long r[4], double out[4]) {
    k_sel_init<<<1, 256, 0, st>>>(x, r[0], r[1], r[2], r[3]);
    const int shifts[6] = {53, 42, 31, 20, 9, 0};
    for (int p = 0; p < 6; ++p) {
        k_sel_hist<<<grid_for(n), kThreads, 0, st>>>(n, v, x, shifts[p]);
        k_sel_scan<<<1, 32 * kSel, 0, st>>>(x, shifts[p]);
    }
    unsigned long long pre[kSel];
    cudaError_t e = cudaMemcpyAsync(pre, x->prefix, sizeof(pre), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < kSel; ++s) memcpy(&out[s], &pre[s], sizeof(double));
    return cudaGetLastError();
}

// median and 99th percentile: linear interpolation at position q (n - 1)
cudaError_t quantiles(cudaStream_t st, int64_t n, const double* v, ErrAux* x, double* med, double* p99) {
    const double q[2] = {0.5, 0.99};
    long long r[4];
    double w[2];
    for (int j = 0; j < 2; ++j) {
        const double pos = q[j] * (double)(n - 1);
        const long long lo = (long long)floor(pos);
        r[2 * j] = lo;
        r[2 * j + 1] = lo + 1 < n ? lo + 1 : n - 1;
        w[j] = pos - (double)lo;
    }
    double s[4];
    cudaError_t e = select4(st, n, v, x, r, s);
    if (e != cudaSuccess) return e;
    *med = s[0] + w[0] * (s[1] - s[0]);
    *p99 = s[2] + w[1] * (s[3] - s[2]);
    return cudaSuccess;
}

template <typename R>
cudaError_t run_metrics(ts_ctx* c, int64_t n, const void* pot, const void* acc, const double* pref,
                        const double* aref, int mod_const, double* e, ts_error_stats* out) {
    cudaStream_t st = c->stream;
    ErrAux* x = (ErrAux*)c->d_err_aux;
    cudaError_t err = cudaMemsetAsync(x, 0, offsetof(ErrAux, prefix), st);
    if (err != cudaSuccess) return err;
    const int g = grid_for(n);
    k_err_ref<R><<<g, kThreads, 0, st>>>(n, (const R*)pot, pref, aref, x);
    if (pot) k_err_phimax<<<g, kThreads, 0, st>>>(n, pref, mod_const, x);
    k_err_eval<R><<<g, kThreads, 0, st>>>(n, (const R*)pot, (const R*)acc, pref, aref, mod_const, x, e);
    k_err_count<<<g, kThreads, 0, st>>>(n, e, x);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (acc && (err = quantiles(st, n, e, x, &out->e_a_median, &out->e_a_p99)) != cudaSuccess) return err;
    if (pot && (err = quantiles(st, n, e + n, x, &out->e_phi_median, &out->e_phi_p99)) != cudaSuccess) return err;
    unsigned long long h[5];
    err = cudaMemcpyAsync(h, x->maxb, sizeof(h), cudaMemcpyDeviceToHost, st);   // maxb[4] then nonfinite
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    double d[4];
    memcpy(d, h, sizeof(d));
    out->n = n;
    out->a_ref_max = acc ? d[0] : 0.0;
    out->phi_ref_max = pot ? d[1] : 0.0;
    out->e_a_max = acc ? d[2] : 0.0;
    out->e_phi_max = pot ? d[3] : 0.0;
    out->n_nonfinite = (int64_t)h[4];
    if (!acc) out->e_a_median = out->e_a_p99 = 0.0;
    if (!pot) out->e_phi_median = out->e_phi_p99 = 0.0;
    return cudaSuccess;
}

}  // namespace

extern "C" ts_status ts_error_metrics(ts_ctx* c, int32_t precision, int64_t n, const void* pot, const void* acc,
                                      const double* pref, const double* aref, int32_t pot_mod_const, double* e_dev,
                                      ts_error_stats* out) {
    FaultSite fault_site("error_metrics");
    if (!c || !out) return ts_fail(TS_ERR_INVALID_ARG, "ts_error_metrics: ctx or out is NULL");
    if (precision != TS_PREC_FP32_KAHAN && precision != TS_PREC_FP64)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_error_metrics: unknown precision");
    if (n < 1 || n >= (1ll << 31)) return ts_fail(TS_ERR_INVALID_ARG, "ts_error_metrics: n must be in [1, 2^31)");
    if ((pot == nullptr) != (pref == nullptr) || (acc == nullptr) != (aref == nullptr))
        return ts_fail(TS_ERR_INVALID_ARG, "ts_error_metrics: a value array needs its reference and vice versa");
    if (!pot && !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_error_metrics: neither potential nor acceleration given");
    DeviceGuard g(c->device);
    memset(out, 0, sizeof(*out));
    if (!c->d_err_aux) TS_CUDA(ts_malloc((void**)&c->d_err_aux, sizeof(ErrAux)));
    double* e = e_dev;
    if (!e) {
        if (c->err_cap < n) {
            if (c->d_err) cudaFree(c->d_err);
            c->d_err = nullptr;
            c->err_cap = 0;
            TS_CUDA(ts_malloc((void**)&c->d_err, sizeof(double) * 2 * (size_t)n));
            c->err_cap = n;
        }
        e = c->d_err;
    }
    const cudaError_t err = precision == TS_PREC_FP64
                                ? run_metrics<double>(c, n, pot, acc, pref, aref, pot_mod_const, e, out)
                                : run_metrics<float>(c, n, pot, acc, pref, aref, pot_mod_const, e, out);
    if (err != cudaSuccess) return ts_cuda_fail(err, "ts_error_metrics");
    return TS_OK;
}
