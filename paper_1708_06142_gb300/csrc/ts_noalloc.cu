// Allocation-free variant of the zero-mean potential pass.
//
// Some callers cannot call cudaMalloc: a host code that owns the whole device-memory budget through
// its own allocator (and forbids side allocations), a plugin that may only touch memory it was
// handed, or a time step that must not pay for the implicit synchronisation of cudaMalloc/cudaFree.
// For them this entry point does the work of the zero-mean pass of ts_gravity_walk (subtract the
// weighted mean of a potential array) without allocating anything and without a context: the
// caller passes the array and the weights, and the scratch space for the partial sums is a
// file-scope __device__ array that every GPU loading this library holds until the process exits.
//
// The reduction is two-pass and deterministic: each CTA sums a fixed slice of NA_SLICE elements
// into its own slot of the scratch array, one CTA then adds the slots in a fixed order, and a third
// kernel subtracts the mean.  Every slot that is read was written earlier in the same call, so
// nothing has to be cleared between calls.  Calls that overlap on the GPU (on different streams, or
// from different host threads) share the scratch array and race.
#include <mutex>

#include "ts_internal.cuh"

#define NA_THREADS 256
#define NA_SLICE 4096                       // elements per CTA in the first pass
#define NA_MAX_SLICES 4096                  // scratch slots
#define NA_MAX_N ((int64_t)NA_SLICE * NA_MAX_SLICES)   // 16,777,216 elements

// partial (weighted sum, weight) per slice, then the mean in the last slot
static __device__ __align__(256) double g_na_scratch[2 * NA_MAX_SLICES + 2];

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0;
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    return v;   // valid in thread 0
}

__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const float* __restrict__ pot, const double* __restrict__ w,
                                                           int64_t n, double* __restrict__ scratch) {
    __shared__ double sh[NA_THREADS / 32];
    const int64_t lo = (int64_t)blockIdx.x * NA_SLICE;
    const int64_t hi = lo + NA_SLICE < n ? lo + NA_SLICE : n;
    double s = 0, ws = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double wi = w ? w[i] : 1.0;
        s += wi * (double)pot[i];
        ws += wi;
    }
    s = na_block_sum(s, sh);
    ws = na_block_sum(ws, sh);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = s;
        scratch[2 * blockIdx.x + 1] = ws;
    }
}

__global__ void __launch_bounds__(NA_THREADS) k_na_mean(int nslices, double* __restrict__ scratch) {
    __shared__ double sh[NA_THREADS / 32];
    double s = 0, ws = 0;
    for (int k = threadIdx.x; k < nslices; k += blockDim.x) {
        s += scratch[2 * k];
        ws += scratch[2 * k + 1];
    }
    s = na_block_sum(s, sh);
    ws = na_block_sum(ws, sh);
    if (threadIdx.x == 0) scratch[2 * NA_MAX_SLICES] = ws != 0.0 ? s / ws : 0.0;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_subtract(float* __restrict__ pot, int64_t n,
                                                            const double* __restrict__ scratch) {
    const double mean = scratch[2 * NA_MAX_SLICES];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pot[i] = (float)((double)pot[i] - mean);
}

// Device address of the scratch array, looked up once per device (with that device current).
static std::mutex g_na_mutex;
static double* g_na_ptr[64] = {nullptr};

extern "C" ts_status ts_zero_mean_noalloc(int32_t device, float* pot_dev, const double* weight_dev, int64_t n,
                                          void* cuda_stream) {
    if (!pot_dev || n < 1) return ts_fail(TS_ERR_INVALID_ARG, "ts_zero_mean_noalloc: NULL potential or n < 1");
    if (n > NA_MAX_N)
        return ts_fail(TS_ERR_INVALID_ARG,
                       "ts_zero_mean_noalloc: n exceeds the fixed scratch capacity of 16,777,216 elements");
    if (device < 0 || device >= 64) return ts_fail(TS_ERR_INVALID_ARG, "ts_zero_mean_noalloc: bad device");
    // both arrays must be memory of `device` (or managed memory): a pointer of another GPU would be
    // dereferenced by the kernels as a peer address
    const void* ptrs[2] = {pot_dev, weight_dev};
    for (int k = 0; k < 2; ++k) {
        if (!ptrs[k]) continue;
        cudaPointerAttributes a;
        TS_CUDA(cudaPointerGetAttributes(&a, ptrs[k]));
        const bool ok = a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
        if (!ok)
            return ts_fail(TS_ERR_INVALID_ARG, k == 0 ? "ts_zero_mean_noalloc: pot_dev is not device memory of `device`"
                                                      : "ts_zero_mean_noalloc: weight_dev is not device memory of `device`");
    }
    int prev = -1;
    TS_CUDA(cudaGetDevice(&prev));
    if (prev != device) TS_CUDA(cudaSetDevice(device));
    ts_status st = TS_OK;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[device]) {
            cudaError_t e = cudaGetSymbolAddress((void**)&g_na_ptr[device], g_na_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[device] = nullptr;
                st = ts_cuda_fail(e, "ts_zero_mean_noalloc: cudaGetSymbolAddress");
            }
        }
        scratch = g_na_ptr[device];
    }
    if (st == TS_OK) {
        cudaStream_t s = (cudaStream_t)cuda_stream;
        const int nslices = (int)((n + NA_SLICE - 1) / NA_SLICE);
        k_na_partial<<<nslices, NA_THREADS, 0, s>>>(pot_dev, weight_dev, n, scratch);
        k_na_mean<<<1, NA_THREADS, 0, s>>>(nslices, scratch);
        const int grid = (int)((n + NA_THREADS - 1) / NA_THREADS < 152 * 8 ? (n + NA_THREADS - 1) / NA_THREADS : 152 * 8);
        k_na_subtract<<<grid, NA_THREADS, 0, s>>>(pot_dev, n, scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = ts_cuda_fail(e, "ts_zero_mean_noalloc: launch");
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
