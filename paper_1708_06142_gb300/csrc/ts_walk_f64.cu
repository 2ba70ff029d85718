// FP64 gravity walk kernels, the comparator of the FP32 walk (see ts_walk.cu).
#include "ts_walk_kernels.cuh"

cudaError_t walk_launch_f64(ts_ctx* c, const WalkParams& P, int bck, int mac, bool rel, int T) {
    if (bck == 0) return dispatch_bck<double, 0>(c, P, mac, rel, T);
    return dispatch_bck<double, 1>(c, P, mac, rel, T);
}
