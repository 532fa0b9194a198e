// Split-precision operand writers shared by the pack kernels (acse_mixed.cu, acse_ny.cu).
//   BF16x3  x = hi + lo, hi = bf16(x), lo = bf16(x - hi);  A rows [hi|hi|lo], B rows [hi|lo|hi]
//   TF32    x -> tf32 (round to nearest, ties away)        A rows, B rows [x]
//   TF32x3  x = hi + lo, hi = tf32(x), lo = tf32(x - hi);  A rows [hi|hi|lo], B rows [hi|lo|hi]
// Each K segment of a row is Kp elements long; ld is the row length in elements (ns * Kp).
#pragma once
#include <cuda_bf16.h>
#include <string.h>

#include "acse_internal.h"

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// PAT 0: operand A ([hi|hi|lo]); PAT 1: operand B ([hi|lo|hi]).  ld = row length in elements.
template <int PREC, int PAT>
__device__ __forceinline__ void put(void* base, size_t row, size_t ld, int Kp, int k, float x) {
    if (PREC == ACSE_BF16X3) {
        __nv_bfloat16* p = (__nv_bfloat16*)base + row * ld;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        p[k] = hi;
        p[Kp + k] = PAT == 0 ? hi : lo;
        p[2 * Kp + k] = PAT == 0 ? lo : hi;
    } else if (PREC == ACSE_TF32X3) {
        float* p = (float*)base + row * ld;
        const float hi = tf32_rna(x);
        const float lo = tf32_rna(x - hi);
        p[k] = hi;
        p[Kp + k] = PAT == 0 ? hi : lo;
        p[2 * Kp + k] = PAT == 0 ? lo : hi;
    } else {
        float* p = (float*)base + row * ld;
        p[k] = tf32_rna(x);
    }
}

// Four consecutive K positions k..k+3 of one row at once (8-byte stores for BF16, 16-byte for TF32);
// requires k % 4 == 0 and a row length that keeps 8/16-byte alignment (true when r is even).
template <int PREC, int PAT>
__device__ __forceinline__ void put4(void* base, size_t row, size_t ld, int Kp, int k, const float (&x)[4]) {
    if (PREC == ACSE_BF16X3) {
        __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            hi[u] = __float2bfloat16_rn(x[u]);
            lo[u] = __float2bfloat16_rn(x[u] - __bfloat162float(hi[u]));
        }
        __nv_bfloat16* p = (__nv_bfloat16*)base + row * ld + k;
        uint2 H, L;
        memcpy(&H, hi, 8);
        memcpy(&L, lo, 8);
        *reinterpret_cast<uint2*>(p) = H;
        *reinterpret_cast<uint2*>(p + Kp) = PAT == 0 ? H : L;
        *reinterpret_cast<uint2*>(p + 2 * Kp) = PAT == 0 ? L : H;
    } else if (PREC == ACSE_TF32X3) {
        float hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            hi[u] = tf32_rna(x[u]);
            lo[u] = tf32_rna(x[u] - hi[u]);
        }
        float* p = (float*)base + row * ld + k;
        const float4 H = make_float4(hi[0], hi[1], hi[2], hi[3]);
        const float4 L = make_float4(lo[0], lo[1], lo[2], lo[3]);
        *reinterpret_cast<float4*>(p) = H;
        *reinterpret_cast<float4*>(p + Kp) = PAT == 0 ? H : L;
        *reinterpret_cast<float4*>(p + 2 * Kp) = PAT == 0 ? L : H;
    } else {
        float4 v = make_float4(tf32_rna(x[0]), tf32_rna(x[1]), tf32_rna(x[2]), tf32_rna(x[3]));
        *reinterpret_cast<float4*>((float*)base + row * ld + k) = v;
    }
}

