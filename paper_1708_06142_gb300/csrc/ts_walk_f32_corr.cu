// FP32 gravity walk kernels for periodic and mixed BCs: correction table (trilinear or Taylor) and
// learned correction (see ts_walk.cu).
#include "ts_walk_kernels.cuh"

cudaError_t walk_launch_f32_table(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T) {
    return dispatch_bck<float, 1>(c, P, mac, rel, T);
}

cudaError_t walk_launch_f32_mlp(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T) {
    return dispatch_bck<float, 2>(c, P, mac, rel, T);
}
