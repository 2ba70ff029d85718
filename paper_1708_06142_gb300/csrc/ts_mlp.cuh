// Learned Ewald-correction surrogate: a 4-64-64-64-4 SiLU network, BF16 operands on the tensor
// cores (mma.sync m16n8k16, FP32 accumulation), shared by the training kernels (ts_mlp.cu) and the
// gravity walk (ts_walk.cu).
//
// Device weight image (one contiguous buffer, copied to shared memory by every CTA that uses it);
// matrices are [out][in] row-major bf16 with padded rows (bank-conflict-free fragment loads):
//   W1p [64][24]  (4 real inputs twice, columns 0-3 and 4-7, for the hi and lo parts of the
//                 features; padded to K = 16)
//   W2  [64][72], W3 [64][72]
//   W4p [8][72]   (4 real outputs, padded to N = 8)
//   W2t [64][72], W3t [64][72], W4t [64][24]  transposes used by the backward pass ([in][out])
//   b1[64], b2[64], b3[64], b4[8] (FP32), then the output de-normalisation: scale[4], offset[4].
// SiLU is evaluated as z/2 (1 + tanh(z/2)) with the hardware tanh approximation, in training and in
// inference alike.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#define MLP_H 64
#define MLP_LD 72
#define MLP_LD1 24
#define MLP_OFF_W1 0
#define MLP_OFF_W2 (MLP_OFF_W1 + 64 * MLP_LD1)
#define MLP_OFF_W3 (MLP_OFF_W2 + 64 * MLP_LD)
#define MLP_OFF_W4 (MLP_OFF_W3 + 64 * MLP_LD)
#define MLP_OFF_W2T (MLP_OFF_W4 + 8 * MLP_LD)
#define MLP_OFF_W3T (MLP_OFF_W2T + 64 * MLP_LD)
#define MLP_OFF_W4T (MLP_OFF_W3T + 64 * MLP_LD)
#define MLP_NBF16 (MLP_OFF_W4T + 64 * MLP_LD1)          // bf16 elements
#define MLP_NF32 (64 + 64 + 64 + 8 + 4 + 4)              // biases + de-normalisation
#define MLP_BYTES (MLP_NBF16 * 2 + MLP_NF32 * 4)
#define MLP_NPARAM 8900

struct MlpView {
    const __nv_bfloat16* w;   // MLP_NBF16 elements
    const float* f;           // b1 b2 b3 b4 scale offset
};

__device__ __forceinline__ MlpView mlp_view(const void* base) {
    MlpView v;
    v.w = (const __nv_bfloat16*)base;
    v.f = (const float*)((const char*)base + MLP_NBF16 * 2);
    return v;
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *(const uint32_t*)&v;
}

__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float silu_f(float z) { return 0.5f * z * (1.0f + tanh_fast(0.5f * z)); }

// d silu / dz = s (1 + z (1 - s)), s = sigmoid(z) = (1 + tanh(z/2)) / 2
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 0.5f * (1.0f + tanh_fast(0.5f * z));
    return s * (1.0f + z * (1.0f - s));
}

// B fragment of an [N][ld] row-major ("col" operand) matrix for n-tile nt and k-tile kt.
__device__ __forceinline__ void bfrag(uint32_t b[2], const __nv_bfloat16* W, int ld, int nt, int kt, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16* row = W + (nt * 8 + g) * ld + kt * 16 + 2 * t;
    b[0] = *(const uint32_t*)row;
    b[1] = *(const uint32_t*)(row + 8);
}

// B fragments from shared memory by ldmatrix (thread l addresses row l % 8 of 8 x 8 matrix l / 8
// and receives row l / 4, columns 2 (l % 4) and + 1 of each): n-tiles nt, nt + 1 at k-tile kt
// (b[0..1], b[2..3]), or n-tile nt at k-tiles kt, kt + 1.  Rows 16-byte aligned.
__device__ __forceinline__ void bfrag_ldsm(uint32_t b[4], const __nv_bfloat16* W, int ld, int row0, int col0,
                                           int dr, int dk, int lane) {
    const int sel = lane >> 3, r = lane & 7;   // matrices (row0 + dr h, col0 + dk h + 8 l), h = sel / 2, l = sel % 2
    const __nv_bfloat16* p = W + (row0 + r + dr * (sel >> 1)) * ld + col0 + 8 * (sel & 1) + dk * (sel >> 1);
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(a));
}

// The four FP32 features of one row as the first layer's 8 BF16 operands: the BF16 values (hi)
// in columns 0-3 and the BF16 roundings of the remainders (lo = f - hi) in columns 4-7, which meet
// a second copy of W1 there; the first layer then sees the features to 16 significant bits in the
// same single MMA (BF16 alone resolves |dz|/F to 2^-9, a visible error in the correction's slope).
__device__ __forceinline__ uint4 mlp_feat_pack(float f0, float f1, float f2, float f3) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
    const __nv_bfloat16 h2 = __float2bfloat16_rn(f2), h3 = __float2bfloat16_rn(f3);
    uint4 r;
    r.x = pack_bf16(__bfloat162float(h0), __bfloat162float(h1));
    r.y = pack_bf16(__bfloat162float(h2), __bfloat162float(h3));
    r.z = pack_bf16(f0 - __bfloat162float(h0), f1 - __bfloat162float(h1));
    r.w = pack_bf16(f2 - __bfloat162float(h2), f3 - __bfloat162float(h3));
    return r;
}

// Network output for 16 rows m0 .. m0+15 whose features are feat[row] (mlp_feat_pack: 8 bf16).
// out[row] receives the de-normalised (C, A_cx, A_cy, A_cz) for rows < nrows.
__device__ __forceinline__ void mlp_eval_tile(const MlpView& M, const uint4* feat, float4* out, int m0, int nrows,
                                              int lane) {
    const int g = lane >> 2, t = lane & 3;
    uint32_t a[4];
    {   // columns 2t, 2t + 1 of rows g and g + 8: word t of the packed row
        const uint4 f0 = feat[m0 + g], f1 = feat[m0 + g + 8];
        a[0] = t == 0 ? f0.x : t == 1 ? f0.y : t == 2 ? f0.z : f0.w;
        a[1] = t == 0 ? f1.x : t == 1 ? f1.y : t == 2 ? f1.z : f1.w;
    }
    a[2] = 0u;
    a[3] = 0u;
    uint32_t h[4][4];
    {   // layer 1: K = 16 (4 real), N = 64
        float z[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
            uint32_t b[4];
            bfrag_ldsm(b, M.w + MLP_OFF_W1, MLP_LD1, nt * 8, 0, 8, 0, lane);   // n-tiles nt, nt + 1
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float b0 = M.f[(nt + u) * 8 + 2 * t], b1 = M.f[(nt + u) * 8 + 2 * t + 1];
                z[nt + u][0] = b0; z[nt + u][1] = b1; z[nt + u][2] = b0; z[nt + u][3] = b1;
                mma_bf16_16816(z[nt + u], a, b + 2 * u);
            }
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            h[kt][0] = pack_bf16(silu_f(z[2 * kt][0]), silu_f(z[2 * kt][1]));
            h[kt][1] = pack_bf16(silu_f(z[2 * kt][2]), silu_f(z[2 * kt][3]));
            h[kt][2] = pack_bf16(silu_f(z[2 * kt + 1][0]), silu_f(z[2 * kt + 1][1]));
            h[kt][3] = pack_bf16(silu_f(z[2 * kt + 1][2]), silu_f(z[2 * kt + 1][3]));
        }
    }
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {   // layers 2 and 3: K = N = 64
        const __nv_bfloat16* W = M.w + (layer == 0 ? MLP_OFF_W2 : MLP_OFF_W3);
        const float* bias = M.f + 64 * (layer + 1);
        float z[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
            z[nt][0] = b0; z[nt][1] = b1; z[nt][2] = b0; z[nt][3] = b1;
        }
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t b[4];
                bfrag_ldsm(b, W, MLP_LD, nt * 8, kt * 16, 8, 0, lane);   // n-tiles nt, nt + 1
                mma_bf16_16816(z[nt], h[kt], b);
                mma_bf16_16816(z[nt + 1], h[kt], b + 2);
            }
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            h[kt][0] = pack_bf16(silu_f(z[2 * kt][0]), silu_f(z[2 * kt][1]));
            h[kt][1] = pack_bf16(silu_f(z[2 * kt][2]), silu_f(z[2 * kt][3]));
            h[kt][2] = pack_bf16(silu_f(z[2 * kt + 1][0]), silu_f(z[2 * kt + 1][1]));
            h[kt][3] = pack_bf16(silu_f(z[2 * kt + 1][2]), silu_f(z[2 * kt + 1][3]));
        }
    }
    // layer 4: N = 8 (4 real outputs), K = 64
    const float* b4 = M.f + 192;
    float z[4] = {b4[2 * t], b4[2 * t + 1], b4[2 * t], b4[2 * t + 1]};
#pragma unroll
    for (int kt = 0; kt < 4; kt += 2) {
        uint32_t b[4];
        bfrag_ldsm(b, M.w + MLP_OFF_W4, MLP_LD, 0, kt * 16, 0, 16, lane);   // k-tiles kt, kt + 1
        mma_bf16_16816(z, h[kt], b);
        mma_bf16_16816(z, h[kt + 1], b + 2);
    }
    if (t < 2) {
        const float* sc = M.f + 200;
        const float* of = M.f + 204;
        const int c0 = 2 * t;
        const int r0 = m0 + g, r1 = m0 + g + 8;
        if (r0 < nrows) {
            float* o = (float*)&out[r0];
            o[c0] = z[0] * sc[c0] + of[c0];
            o[c0 + 1] = z[1] * sc[c0 + 1] + of[c0 + 1];
        }
        if (r1 < nrows) {
            float* o = (float*)&out[r1];
            o[c0] = z[2] * sc[c0] + of[c0];
            o[c0 + 1] = z[3] * sc[c0 + 1] + of[c0 + 1];
        }
    }
}
