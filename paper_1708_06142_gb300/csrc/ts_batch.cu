// Batched execution of many independent grids with persistent kernels.
//
// Work items are 32-cell groups (one warp's targets) of every grid; a column item and a gravity
// item of the same cells are separate items.  Items fall in three classes, each run by one
// persistent launch with its own device queue (on its own stream, so the classes overlap): column
// items, gravity items of periodic/mixed grids (correction table), gravity items of isolated grids.  (One kernel holding both walks
// needs the register budget of the larger one, 96 registers, and ran 27 % slower than separate
// launches; one launch per class keeps each specialisation's own budget.)  Within a class, items
// are grouped in segments (one per grid).  Each warp takes `chunk` consecutive items from its
// class's queue (one atomicAdd per chunk), finds the segment by binary search, reloads the depth
// geometry when the grid changes, and runs the same per-warp walk as the single-grid kernels.
// There is no waiting between warps: the only shared state is the queue counter.
//
// A run (tree builds, queue resets, descriptor upload, the persistent launches, zero-mean passes)
// can be captured once as a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ts_column_dev.cuh"
#include "ts_walk_dev.cuh"

#define TS_BATCH_MAX_GRIDS 256
#define TS_BATCH_MAX_SEG (2 * TS_BATCH_MAX_GRIDS)

struct BatchArgs {
    const WalkParams* wp;        // [n] gravity descriptors
    const ColParams* cp;         // [n] column descriptors
    const int64_t* seg_begin;    // [nseg + 1] first item of each segment
    const int* seg_grid;         // [nseg]
    int nseg;                    // segments of this class
    int64_t item0, total;        // the class's items are item0 .. item0 + total - 1
    unsigned long long* queue;   // this class's queue counter
    int chunk;
    int npix;
};

// per-warp dynamic shared memory: staging, stacks, geometry, pixel maps
struct WarpSmem {
    WalkParams wp;                 // descriptor of the grid being walked (read from shared memory,
    ColParams cp;                  // so its fields need no registers)
    float4 com[8];
    float4 cen[8];
    uint32_t cw[TS_WALK_STACK];
    uint32_t mask[TS_WALK_STACK][1];
    uint2 cstack[TS_WALK_STACK];
    float half[TS_MAX_DEPTH + 1][3];
    float h2[TS_MAX_DEPTH + 1];
};

__host__ __device__ inline size_t batch_warp_smem(int npix) {
    return (sizeof(WarpSmem) + sizeof(float) * (size_t)npix * 32 + 15) / 16 * 16;
}

// CLS: 0 gravity on isolated grids, 1 gravity on periodic/mixed grids, 2 columns
template <int MAC, int CLS, int EWM = 2>
__global__ void __launch_bounds__(32 * TS_WALK_WARPS) k_batch_walk(const __grid_constant__ BatchArgs A) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ int64_t s_begin[TS_BATCH_MAX_SEG + 1];
    __shared__ int s_grid[TS_BATCH_MAX_SEG];
    for (int i = threadIdx.x; i <= A.nseg; i += blockDim.x) {
        s_begin[i] = A.seg_begin[i];
        if (i < A.nseg) s_grid[i] = A.seg_grid[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = s_dyn + (size_t)warp * batch_warp_smem(A.npix);
    WarpSmem& W = *(WarpSmem*)wbase;
    float* map = (float*)(wbase + sizeof(WarpSmem));
    int cur_grid = -1;
    for (;;) {
        unsigned long long q0 = 0;
        if (lane == 0) q0 = atomicAdd(A.queue, (unsigned long long)A.chunk);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if ((int64_t)q0 >= A.total) break;
        const int64_t it0 = A.item0 + (int64_t)q0;
        const int64_t it1 = A.item0 + min((int64_t)q0 + A.chunk, A.total);
        for (int64_t it = it0; it < it1; ++it) {
            int lo = 0, hi = A.nseg - 1;   // last segment with begin <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_begin[mid] <= it) lo = mid; else hi = mid - 1;
            }
            const int g = s_grid[lo];
            const int64_t local = it - s_begin[lo];
            if (g != cur_grid) {   // descriptor and depth geometry of this grid (32 depths, one per lane)
                __syncwarp();
                if constexpr (CLS == 2) {
                    for (int i = lane; i < (int)(sizeof(ColParams) / 4); i += 32)
                        ((uint32_t*)&W.cp)[i] = ((const uint32_t*)&A.cp[g])[i];
                } else {
                    for (int i = lane; i < (int)(sizeof(WalkParams) / 4); i += 32)
                        ((uint32_t*)&W.wp)[i] = ((const uint32_t*)&A.wp[g])[i];
                }
                const WalkGeom* geo = A.wp[g].geom;
                W.half[lane][0] = geo->half32[lane][0];
                W.half[lane][1] = geo->half32[lane][1];
                W.half[lane][2] = geo->half32[lane][2];
                W.h2[lane] = geo->hmax2_32[lane];
                cur_grid = g;
                __syncwarp();
            }
            if constexpr (CLS == 2)
                col_walk_warp(W.cp, local, lane, map, W.com, W.cen, W.cstack, W.half, W.h2);
            else
                walk_warp<float, CLS, MAC, false, 1, EWM>(W.wp, local, warp, lane, W.com, W.cen, W.cw, W.mask, W.half, W.h2,
                                                     nullptr);
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------------------ host side
cudaError_t make_walk_params(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc, WalkParams* out, int* bck_out);
cudaError_t make_col_params(ts_ctx* c, const ts_ctx* tab, const ts_column_params* p, float* cols, ColParams* out);
cudaError_t launch_col_params(ts_ctx* c, const ColParams& P);
cudaError_t launch_walk_params(ts_ctx* c, const ts_gravity_params* p, const WalkParams& P, int bck, int T);

#define TS_BATCH_MAX_STREAMS 16
cudaError_t launch_gravity_walk(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc);

struct ts_batch {
    std::vector<ts_ctx*> ctx;
    int device = 0;
    cudaStream_t stream = nullptr;
    WalkParams *h_wp = nullptr, *d_wp = nullptr;
    ColParams *h_cp = nullptr, *d_cp = nullptr;
    int64_t *h_begin = nullptr, *d_begin = nullptr;
    int *h_seg = nullptr, *d_seg = nullptr;          // [2][MAX_SEG]: grid, kind
    unsigned long long* d_queue = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the three classes run on their own streams, forked from and joined back into `stream`
    cudaStream_t cls_stream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
    // mode 1: every grid's own single-grid kernels, the grids spread over `nstreams` streams
    int mode = 0, nstreams = 8;
    cudaStream_t wstream[TS_BATCH_MAX_STREAMS] = {};
    cudaEvent_t wjoin[TS_BATCH_MAX_STREAMS] = {};
    std::vector<int> bck;              // correction kind of each grid's walk (mode 1)
    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gsig;
    int chunk = 4, ctas_per_sm = 0;
    int cls_seg0[3] = {0, 0, 0}, cls_nseg[3] = {0, 0, 0};        // per class: segment range
    int64_t cls_item0[3] = {0, 0, 0}, cls_items[3] = {0, 0, 0};  // and item range
    int64_t nitems = 0, ncells = 0;
    bool timed = false;
};

extern "C" ts_status ts_batch_destroy(ts_batch* b) {
    if (!b) return TS_OK;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->h_wp) cudaFreeHost(b->h_wp);
    if (b->h_cp) cudaFreeHost(b->h_cp);
    if (b->h_begin) cudaFreeHost(b->h_begin);
    if (b->h_seg) cudaFreeHost(b->h_seg);
    if (b->d_wp) cudaFree(b->d_wp);
    if (b->d_cp) cudaFree(b->d_cp);
    if (b->d_begin) cudaFree(b->d_begin);
    if (b->d_seg) cudaFree(b->d_seg);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->fork) cudaEventDestroy(b->fork);
    for (int k = 0; k < 3; ++k) {
        if (b->cls_stream[k]) cudaStreamDestroy(b->cls_stream[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    for (int k = 0; k < TS_BATCH_MAX_STREAMS; ++k) {
        if (b->wstream[k]) cudaStreamDestroy(b->wstream[k]);
        if (b->wjoin[k]) cudaEventDestroy(b->wjoin[k]);
    }
    delete b;
    return TS_OK;
}

extern "C" ts_status ts_batch_create(ts_batch** out, ts_ctx* const* ctxs, int32_t n) {
    FaultSite fault_site("batch_create");
    if (!out || !ctxs || n < 1) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_create: bad arguments");
    *out = nullptr;
    if (n > TS_BATCH_MAX_GRIDS) return ts_fail(TS_ERR_UNSUPPORTED, "ts_batch_create: at most 256 grids per batch");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_create: NULL context");
        if (ctxs[i]->device != ctxs[0]->device)
            return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_create: all contexts must be on one device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_create: context listed twice");
    }
    ts_batch* b = new ts_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->bck.assign(n, 0);
    b->device = ctxs[0]->device;
    b->stream = ctxs[0]->stream;
    DeviceGuard g(b->device);
    cudaError_t e = ts_malloc_host((void**)&b->h_wp, sizeof(WalkParams) * n);
    if (e == cudaSuccess) e = ts_malloc_host((void**)&b->h_cp, sizeof(ColParams) * n);
    if (e == cudaSuccess) e = ts_malloc_host((void**)&b->h_begin, sizeof(int64_t) * (TS_BATCH_MAX_SEG + 1));
    if (e == cudaSuccess) e = ts_malloc_host((void**)&b->h_seg, sizeof(int) * 2 * TS_BATCH_MAX_SEG);
    if (e == cudaSuccess) e = ts_malloc((void**)&b->d_wp, sizeof(WalkParams) * n);
    if (e == cudaSuccess) e = ts_malloc((void**)&b->d_cp, sizeof(ColParams) * n);
    if (e == cudaSuccess) e = ts_malloc((void**)&b->d_begin, sizeof(int64_t) * (TS_BATCH_MAX_SEG + 1));
    if (e == cudaSuccess) e = ts_malloc((void**)&b->d_seg, sizeof(int) * 2 * TS_BATCH_MAX_SEG);
    if (e == cudaSuccess) e = ts_malloc((void**)&b->d_queue, sizeof(unsigned long long) * 16);
    if (e == cudaSuccess) e = cudaEventCreate(&b->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->e1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->cls_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        ts_batch_destroy(b);
        return ts_cuda_fail(e, "ts_batch_create");
    }
    memset(b->h_wp, 0, sizeof(WalkParams) * n);
    memset(b->h_cp, 0, sizeof(ColParams) * n);
    *out = b;
    return TS_OK;
}

extern "C" ts_status ts_batch_set_tuning(ts_batch* b, int32_t chunk, int32_t ctas_per_sm) {
    if (!b || chunk < 1 || chunk > 64 || ctas_per_sm < 0 || ctas_per_sm > 16)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_set_tuning: items_per_dequeue in [1,64], ctas_per_sm in [0,16]");
    if (b->chunk != chunk || b->ctas_per_sm != ctas_per_sm) {
        b->chunk = chunk;
        b->ctas_per_sm = ctas_per_sm;
        b->gsig.clear();   // launch shape changed: capture again
    }
    return TS_OK;
}

extern "C" ts_status ts_batch_set_mode(ts_batch* b, int32_t mode, int32_t nstreams) {
    if (!b || (mode != 0 && mode != 1) || nstreams < 1 || nstreams > TS_BATCH_MAX_STREAMS)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_set_mode: mode 0 or 1, nstreams in [1, 16]");
    DeviceGuard g(b->device);
    for (int k = 0; k < nstreams; ++k) {
        if (!b->wstream[k]) TS_CUDA(cudaStreamCreateWithFlags(&b->wstream[k], cudaStreamNonBlocking));
        if (!b->wjoin[k]) TS_CUDA(cudaEventCreateWithFlags(&b->wjoin[k], cudaEventDisableTiming));
    }
    if (b->mode != mode || b->nstreams != nstreams) {
        b->mode = mode;
        b->nstreams = nstreams;
        b->gsig.clear();   // launch shape changed: capture again
    }
    return TS_OK;
}

static int periodic_kind(const int bc[3]) {
    if (!bc[0] && !bc[1] && !bc[2]) return TS_EW_NONE;
    if (bc[0] && bc[1] && bc[2]) return TS_EW_3P;
    if (bc[0] && bc[1] && !bc[2]) return TS_EW_2P1I;
    if (bc[0] && !bc[1] && !bc[2]) return TS_EW_1P2I;
    return -1;
}

// One persistent launch of class CLS: as many CTAs as fit (or ctas_per_sm) on every SM.
template <int MAC, int CLS, int EWM = 2>
static cudaError_t launch_cls(ts_batch* b, const BatchArgs& A, cudaStream_t st) {
    const size_t smem = TS_WALK_WARPS * batch_warp_smem(A.npix);
    cudaError_t e = cudaFuncSetAttribute(k_batch_walk<MAC, CLS, EWM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 152, per = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_walk<MAC, CLS, EWM>, 32 * TS_WALK_WARPS, smem);
    if (b->ctas_per_sm > 0) per = std::min(per, b->ctas_per_sm);
    const int64_t need = (A.total + TS_WALK_WARPS - 1) / TS_WALK_WARPS;   // no idle CTAs for small classes
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(per, 1), need));
    k_batch_walk<MAC, CLS, EWM><<<grid, 32 * TS_WALK_WARPS, smem, st>>>(A);
    return cudaGetLastError();
}

// The launches of one run on the batch stream (captured as a graph or issued directly).
// Mode 1: the grids, largest first, each to the least loaded of the worker streams; per grid its
// tree build, walk, column walk and zero mean with the single-grid kernels and the descriptors
// prepared by ts_batch_run (kernel arguments, so a captured graph holds them by value).
static cudaError_t batch_issue_streams(ts_batch* b, const ts_gravity_params* gp, void* const* pot,
                                      const ts_column_params* cp, const double* const* density) {
    const int n = (int)b->ctx.size(), ns = b->nstreams;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->ctx[x]->ncell > b->ctx[y]->ncell; });
    std::vector<int64_t> load(ns, 0);
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->wstream[k], b->fork, 0);
    for (int i : order) {
        if (e != cudaSuccess) break;
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += b->ctx[i]->ncell;
        ts_ctx* c = b->ctx[i];
        cudaStream_t keep = c->stream;
        c->stream = b->wstream[k];
        if (density) e = launch_tree_build(c, density[i]);
        if (density && e == cudaSuccess) c->rec64_valid = c->rec64;
        if (e == cudaSuccess && gp) e = launch_walk_params(c, gp, b->h_wp[i], b->bck[i], 1);
        if (e == cudaSuccess && cp) e = launch_col_params(c, b->h_cp[i]);
        if (e == cudaSuccess && gp && gp->zero_mean) e = launch_zero_mean(c, TS_PREC_FP32_KAHAN, pot[i]);
        c->stream = keep;
    }
    for (int k = 0; k < ns; ++k) {   // join every worker stream (also after a failure)
        cudaError_t ej = cudaEventRecord(b->wjoin[k], b->wstream[k]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->stream, b->wjoin[k], 0);
        if (e == cudaSuccess) e = ej;
    }
    return e;
}

static cudaError_t batch_issue(ts_batch* b, const ts_gravity_params* gp, void* const* pot, const ts_column_params* cp,
                               const double* const* density, int nseg, int npix) {
    const int n = (int)b->ctx.size();
    cudaError_t e = cudaSuccess;
    if (b->mode == 1) {
        e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long) * 16, b->stream);   // counters
        return e == cudaSuccess ? batch_issue_streams(b, gp, pot, cp, density) : e;
    }
    if (density) {
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            ts_ctx* c = b->ctx[i];
            cudaStream_t keep = c->stream;
            c->stream = b->stream;
            e = launch_tree_build(c, density[i]);
            if (e == cudaSuccess) c->rec64_valid = c->rec64;
            c->stream = keep;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_wp, b->h_wp, sizeof(WalkParams) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_cp, b->h_cp, sizeof(ColParams) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_begin, b->h_begin, sizeof(int64_t) * (nseg + 1), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_seg, b->h_seg, sizeof(int) * TS_BATCH_MAX_SEG, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long) * 16, b->stream);
    if (e != cudaSuccess) return e;
    const bool ape = gp && gp->mac == TS_MAC_APE;
    const bool taylor = gp && gp->ewald == TS_EWALD_TAYLOR;
    // fork: each class on its own stream, so that one class's tail overlaps the others' work
    e = cudaEventRecord(b->fork, b->stream);
    bool used[3] = {false, false, false};
    for (int cls = 2; cls >= 0 && e == cudaSuccess; --cls) {   // columns, periodic gravity, isolated gravity
        if (!b->cls_items[cls]) continue;
        cudaStream_t st = b->cls_stream[cls];
        e = cudaStreamWaitEvent(st, b->fork, 0);
        if (e != cudaSuccess) break;
        used[cls] = true;
        BatchArgs A;
        A.wp = b->d_wp;
        A.cp = b->d_cp;
        A.seg_begin = b->d_begin + b->cls_seg0[cls];
        A.seg_grid = b->d_seg + b->cls_seg0[cls];
        A.nseg = b->cls_nseg[cls];
        A.item0 = b->cls_item0[cls];
        A.total = b->cls_items[cls];
        A.queue = b->d_queue + cls;
        A.chunk = b->chunk;
        A.npix = cls == 2 ? npix : 0;
        if (cls == 2) e = ape ? launch_cls<TS_MAC_APE, 2>(b, A, st) : launch_cls<TS_MAC_BH, 2>(b, A, st);
        else if (cls == 1)   // the lookup mode is the same for every grid of the run: a specialised kernel
            e = taylor ? (ape ? launch_cls<TS_MAC_APE, 1, 1>(b, A, st) : launch_cls<TS_MAC_BH, 1, 1>(b, A, st))
                       : (ape ? launch_cls<TS_MAC_APE, 1, 0>(b, A, st) : launch_cls<TS_MAC_BH, 1, 0>(b, A, st));
        else e = ape ? launch_cls<TS_MAC_APE, 0>(b, A, st) : launch_cls<TS_MAC_BH, 0>(b, A, st);
    }
    // join (also after a failed launch, so that no branch of a capture is left open)
    for (int cls = 0; cls < 3; ++cls) {
        if (!used[cls]) continue;
        cudaError_t ej = cudaEventRecord(b->join[cls], b->cls_stream[cls]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->stream, b->join[cls], 0);
        if (e == cudaSuccess) e = ej;
    }
    (void)nseg;
    if (e == cudaSuccess && gp && gp->zero_mean) {
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            ts_ctx* c = b->ctx[i];
            cudaStream_t keep = c->stream;
            c->stream = b->stream;
            e = launch_zero_mean(c, TS_PREC_FP32_KAHAN, pot[i]);
            c->stream = keep;
        }
    }
    return e;
}

extern "C" ts_status ts_batch_run(ts_batch* b, const ts_gravity_params* gp, void* const* pot, void* const* acc,
                                  const ts_column_params* cp, float* const* cols, const double* const* density,
                                  int32_t use_graph) {
    FaultSite fault_site("batch_run");
    if (!b || (!gp && !cp)) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: nothing to do");
    const int n = (int)b->ctx.size();
    if (gp) {
        if (!pot || !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: NULL gravity outputs");
        if (gp->precision != TS_PREC_FP32_KAHAN || gp->ewald == TS_EWALD_MLP || gp->a_old_dev)
            return ts_fail(TS_ERR_UNSUPPORTED, "ts_batch_run: batched gravity is FP32 + Kahan with a table correction "
                                               "(trilinear or Taylor) and an absolute APE limit");
        if (gp->ewald != TS_EWALD_TABLE && gp->ewald != TS_EWALD_TAYLOR)
            return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: unknown Ewald mode");
        if (gp->mac == TS_MAC_MPE || gp->mac == TS_MAC_SUMSQ)
            return ts_fail(TS_ERR_UNSUPPORTED, "ts_batch_run: batched gravity runs BH or APE");
        if (gp->accel != TS_ACCEL_DIRECT)
            return ts_fail(TS_ERR_UNSUPPORTED, "ts_batch_run: batched gravity sums the accelerations directly");
        if (gp->mac == TS_MAC_BH ? !(gp->theta > 0) : (gp->mac != TS_MAC_APE || !(gp->a_lim > 0)))
            return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: bad MAC parameters");
    }
    if (cp) {
        if (!cols) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: NULL column outputs");
        if (cp->n_side < 1 || cp->n_side > 4 || !(cp->theta > 0))
            return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: n_side in [1, 4] and theta > 0");
    }
    for (int i = 0; i < n; ++i) {
        ts_ctx* c = b->ctx[i];
        if (!c->have_mesh || (!density && !c->have_tree))
            return ts_fail(TS_ERR_NOT_BUILT, "ts_batch_run: every context needs a mesh (and a tree, without densities)");
        const int kind = periodic_kind(c->bc);
        if (kind < 0) return ts_fail(TS_ERR_UNSUPPORTED, "ts_batch_run: unsupported periodic axes");
        if (gp && kind != TS_EW_NONE && !c->have_ewald)
            return ts_fail(TS_ERR_NOT_BUILT, "ts_batch_run: periodic/mixed grids need ts_ewald_field first");
        if (gp && kind != TS_EW_NONE && gp->ewald == TS_EWALD_TAYLOR) {
            DeviceGuard g(c->device);
            ts_status s = ensure_taylor(c);
            if (s != TS_OK) return s;
        }
        if ((gp && (!pot[i] || !acc[i])) || (cp && !cols[i]) || (density && !density[i]))
            return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_run: NULL per-grid buffer");
    }
    DeviceGuard g(b->device);
    int npix = 0;
    if (cp) {
        int dims[3], nsub;
        double pmin, pmax;
        ts_status s = column_table_params(cp, dims, &pmin, &pmax, &nsub);
        if (s == TS_OK) s = ensure_noderay(b->ctx[0], cp->n_side, dims, pmin, pmax, nsub);
        if (s != TS_OK) return s;
        npix = 12 * cp->n_side * cp->n_side;
    }
    // per-grid descriptors (pinned host copies, uploaded by the run itself)
    unsigned long long* cnt = b->d_queue;
    for (int i = 0; i < n; ++i) {
        ts_ctx* c = b->ctx[i];
        int bck = 0;
        cudaError_t e = cudaSuccess;
        if (gp) {
            e = make_walk_params(c, gp, pot[i], acc[i], &b->h_wp[i], &bck);
            b->h_wp[i].counters = cnt + 4;   // [0..2] queues, [4..7] gravity, [8..9] column counters
            b->bck[i] = bck;
        } else {
            WalkGeom* dg = nullptr;
            memset(&b->h_wp[i], 0, sizeof(WalkParams));
            if (!c->d_geom) e = ts_malloc((void**)&c->d_geom, sizeof(WalkGeom));
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_geom, &c->geom, sizeof(WalkGeom), cudaMemcpyHostToDevice, c->stream);
            dg = c->d_geom;
            b->h_wp[i].geom = dg;
        }
        if (e == cudaSuccess && cp) {
            e = make_col_params(c, b->ctx[0], cp, cols[i], &b->h_cp[i]);
            b->h_cp[i].counters = cnt + 8;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ts_cuda_fail(e, "ts_batch_run: descriptors");
    }
    // segments grouped by class (columns, periodic gravity, isolated gravity), one per grid, the
    // largest grids first so that the work queue hands out the long items before the short ones
    int64_t cells = 0, items = 0;
    int nseg = 0;
    for (int i = 0; i < n; ++i) cells += b->ctx[i]->ncell;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->ctx[x]->ncell > b->ctx[y]->ncell; });
    for (int cls = 2; cls >= 0; --cls) {
        b->cls_seg0[cls] = nseg;
        b->cls_item0[cls] = items;
        for (int i : order) {
            ts_ctx* c = b->ctx[i];
            const bool per = periodic_kind(c->bc) != TS_EW_NONE;
            const bool in = cls == 2 ? cp != nullptr : (gp != nullptr && (cls == 1) == per);
            if (!in) continue;
            b->h_begin[nseg] = items;
            b->h_seg[nseg] = i;
            items += c->ncell / 32;
            ++nseg;
        }
        b->cls_nseg[cls] = nseg - b->cls_seg0[cls];
        b->cls_items[cls] = items - b->cls_item0[cls];
    }
    b->h_begin[nseg] = items;
    const int64_t acc_items = items;
    b->nitems = items;
    b->ncells = cells;
    // graph signature: everything baked into the captured launches
    std::vector<uint64_t> sig = {(uint64_t)(gp != nullptr), (uint64_t)(cp != nullptr), gp ? (uint64_t)gp->mac : 0,
                                 gp ? (uint64_t)gp->ewald : 0,
                                 gp ? (uint64_t)gp->zero_mean : 0, (uint64_t)npix, (uint64_t)b->chunk,
                                 (uint64_t)b->ctas_per_sm, (uint64_t)nseg, (uint64_t)acc_items,
                                 (uint64_t)(density != nullptr)};
    sig.push_back((uint64_t)b->mode);
    sig.push_back((uint64_t)b->nstreams);
    for (int i = 0; i < n; ++i) {
        sig.push_back(density ? (uint64_t)density[i] : 0);
        sig.push_back(gp ? (uint64_t)pot[i] : 0);
        if (b->mode == 1) {   // kernel arguments captured by value: every descriptor byte matters
            uint64_t h = 1469598103934665603ull;
            const unsigned char* q = (const unsigned char*)&b->h_wp[i];
            for (size_t k = 0; k < sizeof(WalkParams); ++k) h = (h ^ q[k]) * 1099511628211ull;
            q = (const unsigned char*)&b->h_cp[i];
            for (size_t k = 0; k < sizeof(ColParams); ++k) h = (h ^ q[k]) * 1099511628211ull;
            sig.push_back(h);
            sig.push_back((uint64_t)b->bck[i]);
        }
    }
    cudaError_t e = cudaEventRecord(b->e0, b->stream);
    if (use_graph) {
        if (!b->gexec || sig != b->gsig) {
            if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t ei = batch_issue(b, gp, pot, cp, density, nseg, npix);
                e = cudaStreamEndCapture(b->stream, &graph);
                if (ei != cudaSuccess) e = ei;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) { b->gexec = nullptr; b->gsig.clear(); return ts_cuda_fail(e, "ts_batch_run: graph capture"); }
            b->gsig = sig;
        }
        e = cudaGraphLaunch(b->gexec, b->stream);
    } else {
        e = batch_issue(b, gp, pot, cp, density, nseg, npix);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->e1, b->stream);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_batch_run");
    b->timed = true;
    return TS_OK;
}

extern "C" ts_status ts_batch_sync(ts_batch* b, int64_t* out5, double* last_ms) {
    if (!b) return ts_fail(TS_ERR_INVALID_ARG, "ts_batch_sync: NULL batch");
    DeviceGuard g(b->device);
    TS_CUDA(cudaStreamSynchronize(b->stream));
    unsigned long long h[16];
    TS_CUDA(cudaMemcpy(h, b->d_queue, sizeof(h), cudaMemcpyDeviceToHost));
    if (out5) {
        out5[0] = (int64_t)h[4]; out5[1] = (int64_t)h[5]; out5[2] = (int64_t)h[8];
        out5[3] = b->nitems; out5[4] = b->ncells;
    }
    if (last_ms) {
        float ms = 0;
        if (b->timed) TS_CUDA(cudaEventElapsedTime(&ms, b->e0, b->e1));
        *last_ms = ms;
    }
    for (ts_ctx* c : b->ctx) {
        ts_status s = ts_sync(c);
        if (s != TS_OK) return s;
    }
    return TS_OK;
}

extern "C" ts_status ts_autotune_walk(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc, int32_t* best,
                                      double* ms_out) {
    if (!c || !p || !pot || !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_autotune_walk: NULL argument");
    if (p->ewald == TS_EWALD_MLP) return ts_fail(TS_ERR_UNSUPPORTED, "ts_autotune_walk: the learned-correction walk has one grouping");
    if (p->accel != TS_ACCEL_DIRECT || p->mac == TS_MAC_SUMSQ)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_autotune_walk: tunes the warp-shared direct-acceleration walks only");
    const int pi = p->precision == TS_PREC_FP64 ? 1 : 0;
    const int choices[3] = {1, 2, 4};
    double t[3] = {0, 0, 0};
    int keep = c->walk_T[pi], bi = 0;
    for (int k = 0; k < 3; ++k) {
        c->walk_T[pi] = choices[k];
        double best_k = 1e30;
        for (int rep = 0; rep < 2; ++rep) {   // the first launch pays for module loading
            ts_status s = ts_gravity_walk(c, p, pot, acc);
            if (s == TS_OK) s = ts_sync(c);
            double ms = 0;
            if (s == TS_OK) s = ts_stats(c, nullptr, nullptr, &ms);
            if (s != TS_OK) { c->walk_T[pi] = keep; return s; }
            if (rep) best_k = ms;
        }
        t[k] = best_k;
        if (t[k] < t[bi]) bi = k;
    }
    c->walk_T[pi] = choices[bi];
    if (best) *best = choices[bi];
    if (ms_out) for (int k = 0; k < 3; ++k) ms_out[k] = t[k];
    return TS_OK;
}
