// FP32 gravity walk kernels for isolated BCs (see ts_walk.cu).
#include "ts_walk_kernels.cuh"

cudaError_t walk_launch_f32_iso(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T) {
    return dispatch_bck<float, 0>(c, P, mac, rel, T);
}
