// Gravity walk kernels and their launchers, instantiated in several translation units (one per
// precision and correction kind, compiled in parallel); the design is described in ts_walk.cu.
#pragma once
#include "ts_walk_dev.cuh"

// Walk kernel for one grid: one warp per 32 T target cells.  EWM: correction-table lookup
// (0 trilinear, 1 Taylor, 2 run-time choice; see ewald_pair).
// Resident CTAs per SM asked of the compiler: the paired isolated FP32 BH walk is held to 7 CTAs
// (73 registers a thread), which measured 2.5 % faster than the compiler's own choice at the same
// register count; the other instantiations keep the compiler's choice.
template <typename R, int BCK, int MAC, int T>
struct WalkMinBlocks {
    static constexpr int value = (sizeof(R) == 4 && BCK == 0 && MAC == TS_MAC_BH && T == 1) ? 7 : 1;
};

template <typename R, int BCK, int MAC, bool REL, int T, int EWM, bool POT = false>
__global__ void __launch_bounds__(32 * TS_WALK_WARPS, (WalkMinBlocks<R, BCK, MAC, T>::value))
    k_gravity_walk(const __grid_constant__ WalkParams P) {
    typedef typename RT<R>::V4 V4;
    __shared__ __align__(32) V4 s_com[TS_WALK_WARPS][8];
    __shared__ __align__(32) V4 s_cen[TS_WALK_WARPS][8];
    __shared__ __align__(32) V4 s_bm[MAC == TS_MAC_MPE ? TS_WALK_WARPS : 1][8];   // MPE node moments
    __shared__ uint32_t s_cw[TS_WALK_WARPS][TS_WALK_STACK];
    __shared__ __align__(16) uint32_t s_mask[TS_WALK_WARPS][TS_WALK_STACK][T];
    __shared__ R s_half[TS_MAX_DEPTH + 1][3];
    __shared__ R s_h2[TS_MAX_DEPTH + 1];
    extern __shared__ __align__(16) unsigned char s_dyn[];   // learned-correction mode only

    for (int t = threadIdx.x; t <= TS_MAX_DEPTH; t += blockDim.x) {
        if constexpr (sizeof(R) == 4) {
            s_half[t][0] = P.geom->half32[t][0]; s_half[t][1] = P.geom->half32[t][1];
            s_half[t][2] = P.geom->half32[t][2]; s_h2[t] = P.geom->hmax2_32[t];
        } else {
            s_half[t][0] = P.geom->half64[t][0]; s_half[t][1] = P.geom->half64[t][1];
            s_half[t][2] = P.geom->half64[t][2]; s_h2[t] = P.geom->hmax2_64[t];
        }
    }
    if constexpr (BCK == 2) {   // forward weights and biases of the network -> shared memory
        const uint4* wsrc = (const uint4*)P.mlp_img;
        uint4* wdst = (uint4*)s_dyn;
        for (int i = threadIdx.x; i < MLP_FWD_BF16 * 2 / 16; i += blockDim.x) wdst[i] = wsrc[i];
        const float* fsrc = (const float*)((const char*)P.mlp_img + MLP_NBF16 * 2);
        float* fdst = (float*)(s_dyn + MLP_FWD_BF16 * 2);
        for (int i = threadIdx.x; i < MLP_NF32; i += blockDim.x) fdst[i] = fsrc[i];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t gw = (int64_t)blockIdx.x * TS_WALK_WARPS + warp;
    if (P.warp_list) {                           // a subset of warps (Adaptive Block Update)
        if (gw >= *P.nwarp_dev) return;
        gw = P.warp_list[gw];
    } else if (P.targets) {                      // a list of single targets
        if (gw * 32 >= P.ntargets) return;
    } else {                                     // the cells of leaf-blocks [leaf_begin, leaf_end)
        gw += P.leaf_begin * (16 / T);           // 16 / T warps per leaf-block of 512 cells
        if (gw * 32 * T >= P.leaf_end * 512) return;
    }
    walk_warp<R, BCK, MAC, REL, T, EWM, POT>(P, gw, warp, lane, s_com[warp], s_cen[warp], s_cw[warp], s_mask[warp], s_half,
                                        s_h2, s_dyn, s_bm[MAC == TS_MAC_MPE ? warp : 0]);
}

template <typename R, int BCK, int MAC, bool REL, int T, int EWM = 2, bool POT = false>
static cudaError_t launch_t(ts_ctx* c, const WalkParams& P) {
    // warp lists: an upper bound
    const int64_t nwarps = P.targets ? P.ntargets / 32 : (P.leaf_end - P.leaf_begin) * (16 / T);
    if (nwarps <= 0) return cudaSuccess;
    const int grid = (int)((nwarps + TS_WALK_WARPS - 1) / TS_WALK_WARPS);
    size_t smem = 0;
    if constexpr (BCK == 2) {
        smem = MLP_SMEM_WEIGHTS + TS_WALK_WARPS * MLP_SMEM_WARP;
        cudaError_t e = cudaFuncSetAttribute(k_gravity_walk<R, BCK, MAC, REL, T, EWM, POT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_gravity_walk<R, BCK, MAC, REL, T, EWM, POT><<<grid, 32 * TS_WALK_WARPS, smem, c->stream>>>(P);
    return cudaGetLastError();
}

// One target per lane gets kernels specialised to the table lookup; the grouped variants choose it
// at run time.
template <typename R, int BCK, int MAC, bool REL>
static cudaError_t dispatch_t(ts_ctx* c, const WalkParams& P, int T) {
    if (T == 4) return launch_t<R, BCK, MAC, REL, 4>(c, P);
    if (T == 2) return launch_t<R, BCK, MAC, REL, 2>(c, P);
    if constexpr (BCK == 1)
        return P.ew.taylor ? launch_t<R, BCK, MAC, REL, 1, 1>(c, P) : launch_t<R, BCK, MAC, REL, 1, 0>(c, P);
    else
        return launch_t<R, BCK, MAC, REL, 1>(c, P);
}

// Launch for one (precision, correction kind): bck 0 isolated, 1 correction table, 2 learned
// correction (FP32, one target per lane).
template <typename R, int BCK>
static cudaError_t dispatch_bck(ts_ctx* c, const WalkParams& P, int mac, bool rel, int T) {
    if (mac == TS_MAC_MPE) {   // one target per lane
        if constexpr (BCK == 1) {
            if (P.ew.taylor)
                return rel ? launch_t<R, 1, TS_MAC_MPE, true, 1, 1>(c, P) : launch_t<R, 1, TS_MAC_MPE, false, 1, 1>(c, P);
            return rel ? launch_t<R, 1, TS_MAC_MPE, true, 1, 0>(c, P) : launch_t<R, 1, TS_MAC_MPE, false, 1, 0>(c, P);
        } else if constexpr (BCK == 0) {
            return rel ? launch_t<R, 0, TS_MAC_MPE, true, 1>(c, P) : launch_t<R, 0, TS_MAC_MPE, false, 1>(c, P);
        } else {
            return cudaErrorInvalidValue;   // rejected by the API before launch
        }
    }
    if constexpr (BCK == 2) {
        if (mac == TS_MAC_BH) return launch_t<R, 2, TS_MAC_BH, false, 1>(c, P);
        return rel ? launch_t<R, 2, TS_MAC_APE, true, 1>(c, P) : launch_t<R, 2, TS_MAC_APE, false, 1>(c, P);
    } else {
        if (mac == TS_MAC_BH) return dispatch_t<R, BCK, TS_MAC_BH, false>(c, P, T);
        return rel ? dispatch_t<R, BCK, TS_MAC_APE, true>(c, P, T) : dispatch_t<R, BCK, TS_MAC_APE, false>(c, P, T);
    }
}
