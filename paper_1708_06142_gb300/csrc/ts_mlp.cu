// Training and evaluation of the learned Ewald-correction surrogate (2P1I, box aspect b = Ly/Lx in
// [b_min, b_max]): features (|dx|/(Lx/2), |dy|/(Ly/2), |dz|/F_net, beta) mapped to [-1, 1] -> the
// smooth correction (C, A_cx, A_cy, A_cz) in units Lx = 1, normalised per output.
//
// Training data: FP64 Ewald-series samples (k_ewald_samples_2p1i).  One training step =
// k_mlp_train (per CTA 32 samples: forward pass, loss, backward pass; every GEMM, including the
// weight gradients dW = dZ^T A, on BF16 tensor cores with FP32 accumulation, activations kept in
// shared memory; each CTA stores its own partial gradient) + k_mlp_adam_pack (sums the partials in
// CTA order, so training is deterministic; Adam on FP32 master weights; writes the BF16 weight
// image).  A step is a few microseconds of latency-bound work, so the host captures 256 steps in a
// CUDA graph whose kernels read the step number from the device, and replays it; each kernel is a
// programmatic dependent of the one before, so launches and independent prologues overlap.
#include <math.h>
#include <stdio.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ts_internal.cuh"
#include "ts_mlp.cuh"

#define TR_ROWS 32           // samples per CTA (128 CTAs for a batch of 4096: a step is latency bound)
#define TR_WARPS 8           // warp w: m-tile w % 2, n-tiles of part w / 2 (the CTA is latency bound)
#define TR_MTILES (TR_ROWS / 16)
#define TR_NT (8 * TR_MTILES / TR_WARPS)  // 8-column n-tiles of a 64-wide layer per warp
#define MLP_GRAPH_STEPS 256  // training steps per captured graph
#define ACT_LD 72            // row stride (bf16) of the [TR_ROWS][64] activation buffers
#define IN_LD 16             // row stride of the [TR_ROWS][16] input / output-gradient buffers

// packed FP32 parameter offsets: W1[64][4] b1 W2[64][64] b2 W3[64][64] b3 W4[4][64] b4
#define P_W1 0
#define P_B1 256
#define P_W2 320
#define P_B2 4416
#define P_W3 4480
#define P_B3 8576
#define P_W4 8640
#define P_B4 8896

// Training steps replayed from a captured graph read their step number from the device: the graph
// holds steps base + k, k = 0..G-1, and ends with k_mlp_advance (base += G).
struct MlpSched {
    long long base;      // step number of the graph's first step
    long long total;     // steps of the run (cosine schedule length)
    float lr0;           // peak learning rate
};

struct TrainSmem {   // every member a multiple of 16 bytes (fragment loads need 16-byte rows)
    __nv_bfloat16 img[MLP_NBF16];
    float f[MLP_NF32];
    __nv_bfloat16 a0[TR_ROWS * IN_LD];
    __nv_bfloat16 a1[TR_ROWS * ACT_LD], a2[TR_ROWS * ACT_LD], a3[TR_ROWS * ACT_LD];
    __nv_bfloat16 d1[TR_ROWS * ACT_LD], d2[TR_ROWS * ACT_LD], d3[TR_ROWS * ACT_LD];
    __nv_bfloat16 dz4[TR_ROWS * IN_LD];
    __nv_bfloat16 dza[TR_ROWS * ACT_LD], dzb[TR_ROWS * ACT_LD];
};

static_assert(offsetof(TrainSmem, a0) % 16 == 0 && offsetof(TrainSmem, a1) % 16 == 0 &&
                  offsetof(TrainSmem, a2) % 16 == 0 && offsetof(TrainSmem, a3) % 16 == 0 &&
                  offsetof(TrainSmem, dz4) % 16 == 0 && offsetof(TrainSmem, dza) % 16 == 0 &&
                  offsetof(TrainSmem, dzb) % 16 == 0,
              "fragment rows must be 16-byte aligned");

__device__ __forceinline__ float bf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Programmatic dependent launch: wait until the kernels this one depends on have completed and
// their writes are visible (no-op for a launch without the attribute); let the dependent kernel
// be scheduled.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned), grouped by commits;
// wait until at most N groups are pending
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A fragment of a row-major bf16 matrix (consecutive pairs).
__device__ __forceinline__ void afrag(uint32_t a[4], const __nv_bfloat16* X, int ld, int m0, int k0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = *(const uint32_t*)(X + (m0 + g) * ld + k0 + 2 * t);
    a[1] = *(const uint32_t*)(X + (m0 + g + 8) * ld + k0 + 2 * t);
    a[2] = *(const uint32_t*)(X + (m0 + g) * ld + k0 + 2 * t + 8);
    a[3] = *(const uint32_t*)(X + (m0 + g + 8) * ld + k0 + 2 * t + 8);
}

__device__ __forceinline__ void store2(__nv_bfloat16* X, int ld, int row, int col, float v0, float v1) {
    *(uint32_t*)(X + row * ld + col) = pack_bf16(v0, v1);
}

// One dense layer of the forward pass for this warp's m-tile of 16 rows and its TR_NT n-tiles:
// Z = X W^T + b; A = silu(Z), D = silu'(Z).
__device__ void fwd_hidden(TrainSmem& S, const __nv_bfloat16* X, int ldx, int ksteps, const __nv_bfloat16* W, int ldw,
                           const float* bias, __nv_bfloat16* A, __nv_bfloat16* D, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3, mt = warp % TR_MTILES, nt0 = (warp / TR_MTILES) * TR_NT;
    static_assert(TR_NT == 2, "one fragment load covers the warp's two n-tiles");
    float cc[TR_NT][4];
#pragma unroll
    for (int u = 0; u < TR_NT; ++u) {
        const int col = (nt0 + u) * 8 + 2 * t;
        cc[u][0] = bias[col]; cc[u][1] = bias[col + 1]; cc[u][2] = bias[col]; cc[u][3] = bias[col + 1];
    }
    for (int kt = 0; kt < ksteps; ++kt) {
        uint32_t a[4], b[4];
        afrag(a, X, ldx, mt * 16, kt * 16, lane);
        bfrag_ldsm(b, W, ldw, nt0 * 8, kt * 16, 8, 0, lane);   // n-tiles nt0, nt0 + 1
        mma_bf16_16816(cc[0], a, b);
        mma_bf16_16816(cc[1], a, b + 2);
    }
    {
#pragma unroll
        for (int nt = nt0; nt < nt0 + TR_NT; ++nt) {
            const int col = nt * 8 + 2 * t;
            float* c = cc[nt - nt0];
            const int r0 = mt * 16 + g, r1 = r0 + 8;
            // silu(z) = z s and silu'(z) = s (1 + z (1 - s)) from one sigmoid s = (1 + tanh(z/2)) / 2
            float av[4], dv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float sg = 0.5f * (1.0f + tanh_fast(0.5f * c[e]));
                av[e] = c[e] * sg;
                dv[e] = sg * (1.0f + c[e] * (1.0f - sg));
            }
            store2(A, ACT_LD, r0, col, av[0], av[1]);
            store2(A, ACT_LD, r1, col, av[2], av[3]);
            store2(D, ACT_LD, r0, col, dv[0], dv[1]);
            store2(D, ACT_LD, r1, col, dv[2], dv[3]);
        }
    }
    (void)S;
}

// dX = dZ W (dZ: [TR_ROWS][ldz] rows, K = kdim; W^T given as [in][out] row-major) then dZprev = dX * D.
__device__ void bwd_input(const __nv_bfloat16* dZ, int ldz, int ksteps, const __nv_bfloat16* Wt, int ldwt,
                          const __nv_bfloat16* D, __nv_bfloat16* out, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3, mt = warp % TR_MTILES, nt0 = (warp / TR_MTILES) * TR_NT;
    float cc[TR_NT][4] = {};
    for (int kt = 0; kt < ksteps; ++kt) {
        uint32_t a[4], b[4];
        afrag(a, dZ, ldz, mt * 16, kt * 16, lane);
        bfrag_ldsm(b, Wt, ldwt, nt0 * 8, kt * 16, 8, 0, lane);   // n-tiles nt0, nt0 + 1
        mma_bf16_16816(cc[0], a, b);
        mma_bf16_16816(cc[1], a, b + 2);
    }
    {
#pragma unroll
        for (int nt = nt0; nt < nt0 + TR_NT; ++nt) {
            const float* c = cc[nt - nt0];
            const int col = nt * 8 + 2 * t, r0 = mt * 16 + g, r1 = r0 + 8;
            store2(out, ACT_LD, r0, col, c[0] * bf(D + r0 * ACT_LD + col), c[1] * bf(D + r0 * ACT_LD + col + 1));
            store2(out, ACT_LD, r1, col, c[2] * bf(D + r1 * ACT_LD + col), c[3] * bf(D + r1 * ACT_LD + col + 1));
        }
    }
}

// Transposing fragment loads (ldmatrix .trans): thread l gives the address of row l % 8 of matrix
// l / 8 (16 contiguous bytes); it receives, for each matrix, the element pair (2 (l % 4), l / 4) and
// (2 (l % 4) + 1, l / 4) of the stored 8 x 8 matrix, i.e. row l / 4 of its transpose.
__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], const __nv_bfloat16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t r[2], const __nv_bfloat16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// dW[out][in] = sum_s dZ[s][out] X[s][in] over the CTA's TR_ROWS samples, tiles (mt, nt) split over
// warps; stored into this CTA's slice of the FP32 partial gradients (row stride ldg, nout x nin real
// entries; each entry is written by exactly one warp).  Column `ones` of X holds ones, so the n-tile
// holding it also yields the bias gradient sum_s dZ[s][out] (stored to gbias).  Both operands are stored sample-major, so
// their fragments come from transposing loads: A[m][k] = dZ[k][m] as the four 8 x 8 blocks
// (m 0-7 | 8-15) x (k 0-7 | 8-15), B[k][n] = X[k][n] as k 0-7 and k 8-15.  Rows are 16-byte aligned
// (row strides of 32 and 144 bytes, column offsets in multiples of 8 elements).
template <int MTILES, int NTILES>
__device__ __forceinline__ void bwd_weight(const __nv_bfloat16* dZ, int ldz, const __nv_bfloat16* X, int ldx, int nout,
                                           int nin, int ones, float* grad, int ldg, float* gbias, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3, r = lane & 7, sel = lane >> 3;
    // this warp's tiles warp, warp + TR_WARPS, ...: at most PER of them, all in flight together
    constexpr int TOT = MTILES * NTILES, PER = (TOT + TR_WARPS - 1) / TR_WARPS;
    float c[PER][4];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        c[u][0] = c[u][1] = c[u][2] = c[u][3] = 0.f;
        const int tile = warp + u * TR_WARPS;
        if (tile < TOT) {
            const int mt = tile / NTILES, nt = tile % NTILES;
#pragma unroll
            for (int k0 = 0; k0 < TR_ROWS; k0 += 16) {
                uint32_t a[4], b[2];
                ldsm_x4_trans(a, dZ + (k0 + r + 8 * (sel >> 1)) * ldz + mt * 16 + 8 * (sel & 1));
                ldsm_x2_trans(b, X + (k0 + r + 8 * (sel & 1)) * ldx + nt * 8);
                mma_bf16_16816(c[u], a, b);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int tile = warp + u * TR_WARPS;
        if (tile >= TOT) continue;
        const int mt = tile / NTILES, nt = tile % NTILES;
        const int o0 = mt * 16 + g, o1 = o0 + 8, i0 = nt * 8 + 2 * t;
        if (i0 == ones) {   // the ones column: bias gradient sum_s dZ[s][out]
            if (o0 < nout) gbias[o0] = c[u][0];
            if (o1 < nout) gbias[o1] = c[u][2];
            continue;
        }
        if (i0 + 1 < nin) {   // (i0 even, ldg even: 8-byte aligned pairs)
            if (o0 < nout) *(float2*)(grad + o0 * ldg + i0) = make_float2(c[u][0], c[u][1]);
            if (o1 < nout) *(float2*)(grad + o1 * ldg + i0) = make_float2(c[u][2], c[u][3]);
        } else if (i0 < nin) {
            if (o0 < nout) grad[o0 * ldg + i0] = c[u][0];
            if (o1 < nout) grad[o1 * ldg + i0] = c[u][2];
        }
    }
}

// One step over the samples [first, first + batch) (first = step * batch mod nall; 0 without a
// schedule), TR_ROWS per CTA; with grad == nullptr the kernel only evaluates the loss.
// scale = 2 / (4 * total batch size): d(mean sq. error)/dy.
__global__ void __launch_bounds__(32 * TR_WARPS) k_mlp_train(const void* __restrict__ img, const float* __restrict__ feat,
                                                            const float* __restrict__ targ,
                                                            const MlpSched* __restrict__ sched, int k, int64_t nall,
                                                            float scale, float* __restrict__ grad,
                                                            float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *(TrainSmem*)smem_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // prologue that depends on no earlier kernel (the inputs are fixed for the run): this step's
    // feature rows and the ones columns; it overlaps the previous step's update (programmatic
    // dependent launch)
    const int64_t first = sched ? ((sched->base + k) * (int64_t)gridDim.x * TR_ROWS) % nall : 0;
    const int64_t r0 = first + (int64_t)blockIdx.x * TR_ROWS;
    for (int i = threadIdx.x; i < TR_ROWS * IN_LD; i += blockDim.x) {
        const int r = i / IN_LD, c = i % IN_LD;
        const int64_t s = (r0 + r) % nall;
        // columns 0-3: the features in BF16; 4-7: the BF16 remainders (see mlp_feat_pack); 8: ones
        const float f = c < 8 ? feat[4 * s + (c & 3)] : 0.f;
        const float hi = __bfloat162float(__float2bfloat16_rn(f));
        S.a0[i] = __float2bfloat16_rn(c < 4 ? hi : (c < 8 ? f - hi : (c == 8 ? 1.f : 0.f)));
    }
    // activation columns 64-71 (never written by the layers): ones, then zeros (bias gradients)
    for (int i = threadIdx.x; i < TR_ROWS * 8; i += blockDim.x) {
        const int r = i >> 3, c = 64 + (i & 7);
        const __nv_bfloat16 v = __float2bfloat16_rn(c == 64 ? 1.f : 0.f);
        S.a1[r * ACT_LD + c] = v; S.a2[r * ACT_LD + c] = v; S.a3[r * ACT_LD + c] = v;
    }
    // targets of the output warps' rows (lane (g, t < 2): rows 16 w + g and + 8, outputs 2t, 2t + 1)
    float tg[4] = {0.f, 0.f, 0.f, 0.f};
    if (warp < TR_MTILES && (lane & 3) < 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t s = (r0 + warp * 16 + (lane >> 2) + 8 * h) % nall;
            tg[2 * h] = targ[4 * s + 2 * (lane & 3)];
            tg[2 * h + 1] = targ[4 * s + 2 * (lane & 3) + 1];
        }
    }
    // the weight image (and the partial-gradient buffer this step overwrites) belong to the
    // previous update until it completes
    grid_dep_wait();
    {   // weight image -> shared memory, all 16-byte copies in flight at once: first group the
        // forward weights and the FP32 block, second group the backward transposes
        const uint4* src = (const uint4*)img;
        uint4* dst = (uint4*)S.img;
        constexpr int fwd16 = MLP_OFF_W2T * 2 / 16, bwd16 = MLP_NBF16 * 2 / 16, all16 = MLP_BYTES / 16;
        static_assert(MLP_OFF_W2T * 2 % 16 == 0 && MLP_NBF16 * 2 % 16 == 0 && MLP_BYTES % 16 == 0, "16-byte pieces");
        for (int i = threadIdx.x; i < fwd16; i += blockDim.x) cp_async16(dst + i, src + i);
        for (int i = bwd16 + threadIdx.x; i < all16; i += blockDim.x) cp_async16(dst + i, src + i);
        cp_async_commit();
        for (int i = fwd16 + threadIdx.x; i < bwd16; i += blockDim.x) cp_async16(dst + i, src + i);
        cp_async_commit();
        cp_async_wait_group<1>();
    }
    grid_dep_launch_dependents();
    __syncthreads();
    const float* fb = S.f;
    fwd_hidden(S, S.a0, IN_LD, 1, S.img + MLP_OFF_W1, MLP_LD1, fb, S.a1, S.d1, warp, lane);
    __syncthreads();
    fwd_hidden(S, S.a1, ACT_LD, 4, S.img + MLP_OFF_W2, MLP_LD, fb + 64, S.a2, S.d2, warp, lane);
    __syncthreads();
    fwd_hidden(S, S.a2, ACT_LD, 4, S.img + MLP_OFF_W3, MLP_LD, fb + 128, S.a3, S.d3, warp, lane);
    __syncthreads();
    if (warp < TR_MTILES) {   // output layer (one n-tile), loss and dZ4: one warp per m-tile
        const int g = lane >> 2, t = lane & 3;
        float lsum = 0;
        {
            const int mt = warp;
            const int col = 2 * t;
            float c[4] = {fb[192 + col], fb[192 + col + 1], fb[192 + col], fb[192 + col + 1]};
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t a[4], b[2];
                afrag(a, S.a3, ACT_LD, mt * 16, kt * 16, lane);
                bfrag(b, S.img + MLP_OFF_W4, MLP_LD, 0, kt, lane);
                mma_bf16_16816(c, a, b);
            }
            const int rr[2] = {mt * 16 + g, mt * 16 + g + 8};
            for (int h = 0; h < 2; ++h) {
                const int r = rr[h];
                float dz0 = 0, dz1 = 0;
                if (t < 2) {
                    const float e0 = c[2 * h] - tg[2 * h], e1 = c[2 * h + 1] - tg[2 * h + 1];
                    lsum += e0 * e0 + e1 * e1;
                    dz0 = scale * e0;
                    dz1 = scale * e1;
                }
                store2(S.dz4, IN_LD, r, col, dz0, dz1);
                store2(S.dz4, IN_LD, r, col + 8, 0.f, 0.f);
            }
        }
        for (int off = 16; off; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if (lane == 0) atomicAdd(loss, lsum);
    }
    cp_async_wait_group<0>();   // the backward transposes
    if (!grad) return;
    grad += (size_t)blockIdx.x * MLP_NPARAM;   // this CTA's partial gradient: summed in a fixed order later
    __syncthreads();
    // layer 4
    bwd_weight<1, 9>(S.dz4, IN_LD, S.a3, ACT_LD, 4, 64, 64, grad + P_W4, 64, grad + P_B4, warp, lane);
    bwd_input(S.dz4, IN_LD, 1, S.img + MLP_OFF_W4T, MLP_LD1, S.d3, S.dza, warp, lane);
    __syncthreads();
    // layer 3
    bwd_weight<4, 9>(S.dza, ACT_LD, S.a2, ACT_LD, 64, 64, 64, grad + P_W3, 64, grad + P_B3, warp, lane);
    bwd_input(S.dza, ACT_LD, 4, S.img + MLP_OFF_W3T, MLP_LD, S.d2, S.dzb, warp, lane);
    __syncthreads();
    // layer 2
    bwd_weight<4, 9>(S.dzb, ACT_LD, S.a1, ACT_LD, 64, 64, 64, grad + P_W2, 64, grad + P_B2, warp, lane);
    bwd_input(S.dzb, ACT_LD, 4, S.img + MLP_OFF_W2T, MLP_LD, S.d1, S.dza, warp, lane);
    __syncthreads();
    // layer 1 (4 real inputs)
    // (columns 0-3 of a0 are the features' BF16 parts, 8 the ones column)
    bwd_weight<4, 2>(S.dza, ACT_LD, S.a0, IN_LD, 64, 4, 8, grad + P_W1, 4, grad + P_B1, warp, lane);
}

// BF16 weight image (padded, with transposes) from the FP32 master parameters.
__global__ void k_mlp_pack(const float* __restrict__ p, const float* __restrict__ norm, void* __restrict__ img) {
    __nv_bfloat16* w = (__nv_bfloat16*)img;
    float* f = (float*)((char*)img + MLP_NBF16 * 2);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NBF16 + MLP_NF32; i += gridDim.x * blockDim.x) {
        if (i >= MLP_NBF16) {
            const int k = i - MLP_NBF16;
            float v;
            if (k < 64) v = p[P_B1 + k];
            else if (k < 128) v = p[P_B2 + k - 64];
            else if (k < 192) v = p[P_B3 + k - 128];
            else if (k < 200) v = k - 192 < 4 ? p[P_B4 + k - 192] : 0.f;
            else v = norm[k - 200];
            f[k] = v;
            continue;
        }
        float v = 0.f;
        int o, in;
        if (i < MLP_OFF_W2) {                // W1p [64][24]
            o = i / MLP_LD1; in = i % MLP_LD1;
            if (in < 8) v = p[P_W1 + o * 4 + (in & 3)];   // W1 twice: hi and lo feature columns
        } else if (i < MLP_OFF_W3) {         // W2 [64][72]
            const int k = i - MLP_OFF_W2; o = k / MLP_LD; in = k % MLP_LD;
            if (in < 64) v = p[P_W2 + o * 64 + in];
        } else if (i < MLP_OFF_W4) {         // W3
            const int k = i - MLP_OFF_W3; o = k / MLP_LD; in = k % MLP_LD;
            if (in < 64) v = p[P_W3 + o * 64 + in];
        } else if (i < MLP_OFF_W2T) {        // W4p [8][72]
            const int k = i - MLP_OFF_W4; o = k / MLP_LD; in = k % MLP_LD;
            if (o < 4 && in < 64) v = p[P_W4 + o * 64 + in];
        } else if (i < MLP_OFF_W3T) {        // W2t [in][out]
            const int k = i - MLP_OFF_W2T; in = k / MLP_LD; o = k % MLP_LD;
            if (o < 64) v = p[P_W2 + o * 64 + in];
        } else if (i < MLP_OFF_W4T) {        // W3t
            const int k = i - MLP_OFF_W3T; in = k / MLP_LD; o = k % MLP_LD;
            if (o < 64) v = p[P_W3 + o * 64 + in];
        } else {                             // W4t [64][24]
            const int k = i - MLP_OFF_W4T; in = k / MLP_LD1; o = k % MLP_LD1;
            if (o < 4) v = p[P_W4 + o * 64 + in];
        }
        w[i] = __float2bfloat16(v);
    }
}

__device__ __forceinline__ void mlp_put(__nv_bfloat16* w, int i, float v) { w[i] = __float2bfloat16(v); }

// Adam step of parameter i (the gradient is the sum of the CTAs' partial gradients in a fixed order,
// so training is deterministic; launched with 8 threads per parameter), then its exponential moving average (the averaged weights are the ones kept
// after training: they sit below the optimiser's noise), then its BF16 image slots (each
// packed parameter lands in one or two image slots: W1 twice for the features' value and remainder
// columns, W2-W4 in the forward matrices and the backward transposes; biases in the FP32 block), so
// no thread reads what another writes.  Step s: learning rate lr0 (0.01 + 0.99 (1 + cos(pi s/S))/2),
// bias corrections 0.9^(s+1) and 0.999^(s+1), average decay min(0.9995, (1+s)/(10+s)).
__global__ void k_mlp_adam_pack(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int nparts, float* __restrict__ ema,
                                const MlpSched* __restrict__ sched, int k, void* __restrict__ img) {
    const long long s = sched->base + k;
    const float lr = sched->lr0 * (0.01f + 0.99f * 0.5f * (1.f + cosf((float)M_PI * (float)s / (float)sched->total)));
    const float b1t = powf(0.9f, (float)(s + 1)), b2t = powf(0.999f, (float)(s + 1));
    const float decay = fminf(0.9995f, (1.f + (float)s) / (10.f + (float)s));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    __nv_bfloat16* w = (__nv_bfloat16*)img;
    float* f = (float*)((char*)img + MLP_NBF16 * 2);
    grid_dep_wait();   // the partial gradients of this step
    grid_dep_launch_dependents();
    // eight threads per parameter, each summing an eighth of the partials (its loads all in
    // flight), combined in a fixed pairwise order
    const int i = blockIdx.x * (blockDim.x / 8) + (threadIdx.x >> 3), q = threadIdx.x & 7;
    const int per = (nparts + 7) / 8, b0 = q * per, b1e = min(nparts, b0 + per);
    float gq = 0.f;
    if (i < MLP_NPARAM) {
#pragma unroll 8
        for (int b = b0; b < b1e; ++b) gq += g[(size_t)b * MLP_NPARAM + i];
    }
    gq += __shfl_down_sync(0xffffffffu, gq, 1);   // (0+1), (2+3), ...
    gq += __shfl_down_sync(0xffffffffu, gq, 2);   // ((0+1)+(2+3)), ...
    gq += __shfl_down_sync(0xffffffffu, gq, 4);
    if (q == 0 && i < MLP_NPARAM) {
        const float gi = gq;
        m[i] = b1 * m[i] + (1 - b1) * gi;
        v[i] = b2 * v[i] + (1 - b2) * gi * gi;
        const float mh = m[i] / (1 - b1t), vh = v[i] / (1 - b2t);
        const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
        p[i] = pi;
        ema[i] = decay * ema[i] + (1 - decay) * pi;
        if (i < P_B1) {                      // W1[o][in]: columns in and 4 + in of W1p
            const int o = i / 4, in = i % 4;
            mlp_put(w, MLP_OFF_W1 + o * MLP_LD1 + in, pi);
            mlp_put(w, MLP_OFF_W1 + o * MLP_LD1 + 4 + in, pi);
        } else if (i < P_W2) {
            f[i - P_B1] = pi;
        } else if (i < P_B2) {               // W2[o][in] and W2t[in][o]
            const int o = (i - P_W2) / 64, in = (i - P_W2) % 64;
            mlp_put(w, MLP_OFF_W2 + o * MLP_LD + in, pi);
            mlp_put(w, MLP_OFF_W2T + in * MLP_LD + o, pi);
        } else if (i < P_W3) {
            f[64 + i - P_B2] = pi;
        } else if (i < P_B3) {
            const int o = (i - P_W3) / 64, in = (i - P_W3) % 64;
            mlp_put(w, MLP_OFF_W3 + o * MLP_LD + in, pi);
            mlp_put(w, MLP_OFF_W3T + in * MLP_LD + o, pi);
        } else if (i < P_W4) {
            f[128 + i - P_B3] = pi;
        } else if (i < P_B4) {               // W4[o][in] (o < 4) and W4t[in][o]
            const int o = (i - P_W4) / 64, in = (i - P_W4) % 64;
            mlp_put(w, MLP_OFF_W4 + o * MLP_LD + in, pi);
            mlp_put(w, MLP_OFF_W4T + in * MLP_LD1 + o, pi);
        } else {
            f[192 + i - P_B4] = pi;
        }
    }
}

__global__ void k_mlp_advance(MlpSched* sched, int n) { sched->base += n; }

// Sum of the CTAs' partial gradients in CTA order.
__global__ void k_mlp_gsum(const float* __restrict__ part, int nparts, float* __restrict__ g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * MLP_NPARAM + i];
        g[i] = s;
    }
}

// Network outputs (de-normalised) for n feature rows: one warp per 16-row tile.
__global__ void __launch_bounds__(128) k_mlp_eval(const void* __restrict__ img, const float* __restrict__ feat,
                                                  int64_t n, float* __restrict__ out) {
    __shared__ __align__(16) unsigned char s_img[MLP_BYTES];
    __shared__ uint4 s_feat[4][16];
    __shared__ float4 s_out[4][16];
    for (int i = threadIdx.x; i < (int)(MLP_BYTES / 16); i += blockDim.x) ((uint4*)s_img)[i] = ((const uint4*)img)[i];
    __syncthreads();
    const MlpView M = mlp_view(s_img);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t m0 = ((int64_t)blockIdx.x * 4 + warp) * 16; m0 < n; m0 += (int64_t)gridDim.x * 64) {
        if (lane < 16) {
            const int64_t r = m0 + lane < n ? m0 + lane : n - 1;
            s_feat[warp][lane] = mlp_feat_pack(feat[4 * r], feat[4 * r + 1], feat[4 * r + 2], feat[4 * r + 3]);
        }
        __syncwarp();
        const int nrows = n - m0 < 16 ? (int)(n - m0) : 16;
        mlp_eval_tile(M, s_feat[warp], s_out[warp], 0, nrows, lane);
        __syncwarp();
        if (lane < nrows) ((float4*)out)[m0 + lane] = s_out[warp][lane];
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------ host side
static cudaError_t mlp_alloc(ts_ctx* c) {
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess && !*p) e = ts_malloc(p, bytes); };
    A((void**)&c->d_mlp_master, sizeof(float) * MLP_NPARAM);
    A((void**)&c->d_mlp_m, sizeof(float) * MLP_NPARAM);
    A((void**)&c->d_mlp_v, sizeof(float) * MLP_NPARAM);
    A((void**)&c->d_mlp_grad, sizeof(float) * MLP_NPARAM);
    A((void**)&c->d_mlp_loss, sizeof(float) * 8);
    A(&c->d_mlp_img, MLP_BYTES);
    return e;
}

void free_mlp(ts_ctx* c) {
    if (c->d_mlp_master) cudaFree(c->d_mlp_master);
    if (c->d_mlp_m) cudaFree(c->d_mlp_m);
    if (c->d_mlp_v) cudaFree(c->d_mlp_v);
    if (c->d_mlp_grad) cudaFree(c->d_mlp_grad);
    if (c->d_mlp_loss) cudaFree(c->d_mlp_loss);
    if (c->d_mlp_img) cudaFree(c->d_mlp_img);
    c->d_mlp_master = c->d_mlp_m = c->d_mlp_v = c->d_mlp_grad = c->d_mlp_loss = nullptr;
    c->d_mlp_img = nullptr;
    c->have_mlp = false;
}

static cudaError_t mlp_pack(ts_ctx* c) {
    float* d_norm = c->d_mlp_loss + 0;   // reuse: the loss scratch holds 8 floats
    cudaError_t e = cudaMemcpyAsync(d_norm, c->mlp_norm, sizeof(float) * 8, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    k_mlp_pack<<<64, 256, 0, c->stream>>>(c->d_mlp_master, d_norm, c->d_mlp_img);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // d_norm is reused after this
    return e;
}

static size_t train_smem() { return sizeof(TrainSmem); }

// Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) initial parameters from a splitmix64 stream.
static void init_params(std::vector<float>& p, uint64_t seed) {
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t x = s;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    const int fan[8] = {4, 4, 64, 64, 64, 64, 64, 64};
    const int off[9] = {P_W1, P_B1, P_W2, P_B2, P_W3, P_B3, P_W4, P_B4, MLP_NPARAM};
    p.resize(MLP_NPARAM);
    for (int seg = 0; seg < 8; ++seg) {
        const double bound = 1.0 / sqrt((double)fan[seg]);
        for (int i = off[seg]; i < off[seg + 1]; ++i) p[i] = (float)((2 * next() - 1) * bound);
    }
}

extern "C" ts_status ts_surrogate_train(ts_ctx* c, const ts_surrogate_params* sp, double* final_loss) {
    FaultSite fault_site("surrogate");
    if (!c || !sp) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_train: NULL argument");
    if (!(sp->b_min > 0) || !(sp->b_max > sp->b_min) || sp->n_samples < 1024 || sp->steps < 1 ||
        sp->batch < 128 || sp->batch % 128 || !(sp->lr > 0))
        return ts_fail(TS_ERR_INVALID_ARG,
                       "ts_surrogate_train: need 0 < b_min < b_max, n_samples >= 1024, steps >= 1, batch a multiple of 128, lr > 0");
    DeviceGuard g(c->device);
    TS_CUDA(mlp_alloc(c));
    const int64_t n = sp->n_samples;
    float* d_feat = nullptr;
    double* d_targ64 = nullptr;
    float* d_targ = nullptr;
    TS_CUDA(ts_malloc((void**)&d_feat, sizeof(float) * 4 * n));
    cudaError_t e = ts_malloc((void**)&d_targ64, sizeof(double) * 4 * n);
    if (e == cudaSuccess) e = ts_malloc((void**)&d_targ, sizeof(float) * 4 * n);
    if (e == cudaSuccess) e = launch_ewald_samples_2p1i(c->stream, n, sp->b_min, sp->b_max, sp->seed, sp->z_power, d_feat, d_targ64);
    std::vector<double> t64;
    if (e == cudaSuccess) {
        t64.resize(4 * n);
        e = cudaMemcpyAsync(t64.data(), d_targ64, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(d_feat); cudaFree(d_targ64); cudaFree(d_targ);
        return ts_cuda_fail(e, "ts_surrogate_train: training data");
    }
    // per-output normalisation
    double mean[4] = {0, 0, 0, 0}, var[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) for (int k = 0; k < 4; ++k) mean[k] += t64[4 * i + k];
    for (int k = 0; k < 4; ++k) mean[k] /= n;
    for (int64_t i = 0; i < n; ++i) for (int k = 0; k < 4; ++k) var[k] += (t64[4 * i + k] - mean[k]) * (t64[4 * i + k] - mean[k]);
    for (int k = 0; k < 4; ++k) {
        c->mlp_norm[k] = (float)sqrt(std::max(var[k] / n, 1e-30));
        c->mlp_norm[4 + k] = (float)mean[k];
    }
    std::vector<float> t32(4 * n);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k) t32[4 * i + k] = (float)((t64[4 * i + k] - mean[k]) / c->mlp_norm[k]);
    e = cudaMemcpyAsync(d_targ, t32.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, c->stream);
    std::vector<float> p0;
    init_params(p0, sp->seed ^ 0x5A5A5A5Aull);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mlp_master, p0.data(), sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_mlp_m, 0, sizeof(float) * MLP_NPARAM, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_mlp_v, 0, sizeof(float) * MLP_NPARAM, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = mlp_pack(c);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
    const int B = sp->batch;
    const float scale = 2.0f / (4.0f * B);
    float* d_lossacc = nullptr;
    float* d_ema = nullptr;
    float* d_gpart = nullptr;   // [B / TR_ROWS][NPARAM] partial gradients of the CTAs
    MlpSched* d_sched = nullptr;
    if (e == cudaSuccess) e = ts_malloc((void**)&d_gpart, sizeof(float) * MLP_NPARAM * (size_t)(B / TR_ROWS));
    if (e == cudaSuccess) e = ts_malloc((void**)&d_lossacc, sizeof(float));
    if (e == cudaSuccess) e = ts_malloc((void**)&d_ema, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = ts_malloc((void**)&d_sched, sizeof(MlpSched));
    const MlpSched h_sched = {0, (long long)sp->steps, (float)sp->lr};
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sched, &h_sched, sizeof(MlpSched), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ema, c->d_mlp_master, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_lossacc, 0, sizeof(float), c->stream);
    // steps base + k, k = 0 .. count - 1, on stream st
    // (kernels after the first of a sequence are programmatic dependents of the one before: their
    // launch and independent prologue overlap its tail)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    auto enqueue = [&](cudaStream_t st, int count) {
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < count && le == cudaSuccess; ++k) {
            cudaLaunchConfig_t tc = {};
            tc.gridDim = dim3(B / TR_ROWS); tc.blockDim = dim3(32 * TR_WARPS); tc.dynamicSmemBytes = train_smem();
            tc.stream = st; tc.attrs = k ? pdl : nullptr; tc.numAttrs = k ? 1 : 0;
            le = cudaLaunchKernelEx(&tc, k_mlp_train, (const void*)c->d_mlp_img, (const float*)d_feat,
                                    (const float*)d_targ, (const MlpSched*)d_sched, k, (int64_t)n, scale, d_gpart,
                                    d_lossacc);
            cudaLaunchConfig_t ac = {};
            ac.gridDim = dim3((MLP_NPARAM + 31) / 32); ac.blockDim = dim3(256); ac.stream = st;
            ac.attrs = pdl; ac.numAttrs = 1;
            if (le == cudaSuccess)
                le = cudaLaunchKernelEx(&ac, k_mlp_adam_pack, c->d_mlp_master, c->d_mlp_m, c->d_mlp_v,
                                        (const float*)d_gpart, B / TR_ROWS, d_ema, (const MlpSched*)d_sched, k,
                                        (void*)c->d_mlp_img);
        }
        if (le == cudaSuccess) k_mlp_advance<<<1, 1, 0, st>>>(d_sched, count);
        return le;
    };
    // all steps but the last from a captured graph of MLP_GRAPH_STEPS steps; the rest one by one,
    // the loss accumulator cleared before the last step
    const int reps = (sp->steps - 1) / MLP_GRAPH_STEPS;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && reps > 0) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = enqueue(cs, MLP_GRAPH_STEPS);
            e = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, c->stream);
    }
    const int rest = sp->steps - reps * MLP_GRAPH_STEPS;
    if (e == cudaSuccess && rest > 1) e = enqueue(c->stream, rest - 1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(d_lossacc, 0, sizeof(float), c->stream);
    if (e == cudaSuccess) e = enqueue(c->stream, 1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float lsum = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lsum, d_lossacc, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    // keep the averaged parameters
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_mlp_master, d_ema, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = mlp_pack(c);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(d_feat); cudaFree(d_targ64); cudaFree(d_targ); cudaFree(d_lossacc); cudaFree(d_ema); cudaFree(d_gpart);
    cudaFree(d_sched);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_surrogate_train: training loop");
    if (final_loss) *final_loss = lsum / (4.0 * B);   // mean squared error of the last batch (normalised units)
    c->mlp_b[0] = sp->b_min;
    c->mlp_b[1] = sp->b_max;
    c->have_mlp = true;
    return TS_OK;
}

extern "C" ts_status ts_surrogate_get(ts_ctx* c, float* params, float* norm, double* b_range) {
    if (!c || !params) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_get: NULL argument");
    if (!c->have_mlp) return ts_fail(TS_ERR_NOT_BUILT, "ts_surrogate_get: no surrogate");
    DeviceGuard g(c->device);
    TS_CUDA(cudaMemcpyAsync(params, c->d_mlp_master, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    if (norm) memcpy(norm, c->mlp_norm, sizeof(float) * 8);
    if (b_range) { b_range[0] = c->mlp_b[0]; b_range[1] = c->mlp_b[1]; }
    return TS_OK;
}

extern "C" ts_status ts_surrogate_set(ts_ctx* c, const float* params, const float* norm, const double* b_range) {
    FaultSite fault_site("surrogate");
    if (!c || !params || !norm || !b_range) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_set: NULL argument");
    if (!(b_range[0] > 0) || !(b_range[1] > b_range[0])) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_set: bad b range");
    for (int i = 0; i < MLP_NPARAM; ++i)
        if (!isfinite(params[i])) return ts_fail(TS_ERR_NUMERIC, "ts_surrogate_set: non-finite parameter");
    DeviceGuard g(c->device);
    TS_CUDA(mlp_alloc(c));
    memcpy(c->mlp_norm, norm, sizeof(float) * 8);
    TS_CUDA(cudaMemcpyAsync(c->d_mlp_master, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    TS_CUDA(mlp_pack(c));
    c->mlp_b[0] = b_range[0];
    c->mlp_b[1] = b_range[1];
    c->have_mlp = true;
    return TS_OK;
}

// Surrogate file: this header, then the FP32 parameters [8900] in the packing of ts_surrogate_get.
// content_hash is the FNV-1a hash of b_range, norm and the parameters.
struct MlpFileHeader {
    char magic[8];          // "TSMLPNET"
    uint32_t version;       // 1
    uint32_t nparam;        // 8900
    double b_range[2];
    float norm[8];
    uint64_t content_hash;
};

static uint64_t mlp_file_hash(const MlpFileHeader& h, const float* params) {
    uint64_t x = ts_fnv1a(h.b_range, sizeof(h.b_range), TS_FNV_INIT);
    x = ts_fnv1a(h.norm, sizeof(h.norm), x);
    return ts_fnv1a(params, sizeof(float) * MLP_NPARAM, x);
}

extern "C" ts_status ts_surrogate_save(ts_ctx* c, const char* path) {
    if (!c || !path) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_save: NULL argument");
    if (!c->have_mlp) return ts_fail(TS_ERR_NOT_BUILT, "ts_surrogate_save: no surrogate");
    std::vector<float> p(MLP_NPARAM);
    MlpFileHeader h;
    memset(&h, 0, sizeof(h));
    ts_status s = ts_surrogate_get(c, p.data(), h.norm, h.b_range);
    if (s != TS_OK) return s;
    memcpy(h.magic, "TSMLPNET", 8);
    h.version = 1;
    h.nparam = MLP_NPARAM;
    h.content_hash = mlp_file_hash(h, p.data());
    FILE* f = fopen(path, "wb");
    if (!f) return ts_fail(TS_ERR_INVALID_ARG, std::string("ts_surrogate_save: cannot open ") + path);
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(p.data(), sizeof(float), MLP_NPARAM, f) == MLP_NPARAM;
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return ts_fail(TS_ERR_INVALID_ARG, std::string("ts_surrogate_save: write failed: ") + path);
    return TS_OK;
}

extern "C" ts_status ts_surrogate_load(ts_ctx* c, const char* path) {
    if (!c || !path) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_load: NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return ts_fail(TS_ERR_INVALID_ARG, std::string("ts_surrogate_load: cannot open ") + path);
    MlpFileHeader h;
    std::vector<float> p(MLP_NPARAM);
    const bool head = fread(&h, sizeof(h), 1, f) == 1;
    const bool body = head && fread(p.data(), sizeof(float), MLP_NPARAM, f) == MLP_NPARAM;
    char extra;
    const bool tail = body && fread(&extra, 1, 1, f) == 0;
    fclose(f);
    if (!head || memcmp(h.magic, "TSMLPNET", 8) != 0)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_load: not a surrogate file");
    if (h.version != 1 || h.nparam != MLP_NPARAM)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_surrogate_load: unknown file version or network shape");
    if (!body || !tail) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_load: truncated or oversized file");
    if (mlp_file_hash(h, p.data()) != h.content_hash)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_load: content hash mismatch (damaged file)");
    return ts_surrogate_set(c, p.data(), h.norm, h.b_range);
}

extern "C" ts_status ts_surrogate_eval(ts_ctx* c, int64_t n, const float* feat, float* out) {
    if (!c || !feat || !out || n < 1) return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_eval: bad argument");
    if (!c->have_mlp) return ts_fail(TS_ERR_NOT_BUILT, "ts_surrogate_eval: no surrogate");
    DeviceGuard g(c->device);
    const int grid = (int)std::min<int64_t>((n + 63) / 64, 152 * 8);
    k_mlp_eval<<<grid, 128, 0, c->stream>>>(c->d_mlp_img, feat, n, out);
    TS_CUDA(cudaGetLastError());
    return TS_OK;
}

extern "C" ts_status ts_surrogate_grad(ts_ctx* c, int64_t n, const float* feat, const float* targ, float* grad,
                                       double* loss) {
    FaultSite fault_site("surrogate");
    if (!c || !feat || !targ || !grad || n < 128 || n % 128)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_surrogate_grad: n must be a positive multiple of 128");
    if (!c->have_mlp) return ts_fail(TS_ERR_NOT_BUILT, "ts_surrogate_grad: no surrogate");
    DeviceGuard g(c->device);
    TS_CUDA(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem()));
    float* d_l = nullptr;
    float* d_part = nullptr;
    const int nparts = (int)(n / TR_ROWS);
    TS_CUDA(ts_malloc((void**)&d_l, sizeof(float)));
    cudaError_t e = ts_malloc((void**)&d_part, sizeof(float) * MLP_NPARAM * (size_t)nparts);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_l, 0, sizeof(float), c->stream);
    if (e == cudaSuccess) {
        k_mlp_train<<<nparts, 32 * TR_WARPS, train_smem(), c->stream>>>(c->d_mlp_img, feat, targ, nullptr, 0, n,
                                                                       2.0f / (4.0f * n), d_part, d_l);
        k_mlp_gsum<<<(MLP_NPARAM + 255) / 256, 256, 0, c->stream>>>(d_part, nparts, c->d_mlp_grad);
        e = cudaGetLastError();
    }
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, c->d_mlp_grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, d_l, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_l);
    if (d_part) cudaFree(d_part);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_surrogate_grad");
    if (loss) *loss = l / (4.0 * n);
    return TS_OK;
}
