// Shared-memory, register-tiled O(r^5) kernels of a contraction pass, for both arithmetic paths
// (T = double for the FP64 path, T = float for the split-precision path).
//
//   Z^{kp}_{js} = sum_q W^{kp}_{qs} 1D^j_q  ->  for each (k, p): Z_kp = 1D . W_kp   (r x r x r)
//   w^k_s = sum_pq W^{kp}_{qs} 1D^p_q = sum_p Z^{kp}_{ps}: the diagonal j = p of Z, so the Z kernel
//       also writes its rows j = p and a small kernel sums them over p
//   B spin types (one block per pair (i, j)): X1 = X_ij . 1D and X2 = w . M_ij^T as r x r x r
//       products plus gathered terms; the block then forms directly
//         H_b^{ij}_{kl} = 4 Y_b^{ij}_{kl} - 12 (P^{ij}_{kl} - P'^{ij}_{lk}),
//       (P, P') = (B_aaaa, B_aaaa), (B_abab, B_abba), (B_bbbb, B_bbbb) for b = aa, ab, bb, so that the
//       residual / update is G_b = H_b - s H_b^T (a plain pair transpose, acse_elem.cu).
// Thread micro-tiles are 4 x 4 outputs over r padded to a multiple of 4; operands sit in shared
// memory laid out so that each thread reads 4-vectors.
#include <cuda_bf16.h>
#include <type_traits>

#include "acse_internal.h"

#define TL_TPB 256
#define ZP_MAX_THREADS 288

__device__ __forceinline__ float tl_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

__host__ __device__ __forceinline__ int pad4(int r) { return (r + 3) & ~3; }

// 4 consecutive elements of a shared array (16-byte aligned: offsets are multiples of 4 elements).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// Double-float: an FP64 value carried as the unevaluated sum h + l of two floats (about 48 significant
// bits).  The Ozaki path runs its O(r^5) products in it: FP32 arithmetic is many times faster than
// FP64 on this GPU.  The all-zero bit pattern is 0.
struct __align__(8) dfl {
    float h, l;
    __device__ __forceinline__ operator double() const { return (double)h + (double)l; }
};
// h = x rounded to the nearest float (ties to even), l = x - h rounded to the nearest float.  With integer
// operations from the bit pattern where x is a normal double whose h and l are normal floats (the FP64
// conversions run on the slow FP64 pipe); the same values through FP64 otherwise.
__device__ __forceinline__ dfl to_dfl(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e >= 949 && e <= 1149) {   // 2^(e - 1075) and h are normal floats
        const unsigned sign = hi & 0x80000000u;
        const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);    // the 23 fraction bits kept
        const unsigned rem = lo & 0x1FFFFFFFu;                        // the 29 dropped ones
        const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
        const float h = __uint_as_float(sign | (((unsigned)(e - 1023 + 127) << 23) + m23 + up));
        const int rr = up ? (int)rem - 0x20000000 : (int)rem;        // x - h in units of 2^(e - 1075)
        const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);
        const float l = __fmul_rn(__int2float_rn(sign ? -rr : rr), scale);
        return dfl{h, l};
    }
    const float h = (float)x;
    return dfl{h, (float)(x - (double)h)};   // x - h is exact in FP64
}
// acc += a b: the rounding error of the product by FMA (the l.l term is dropped), that of the sum by
// Knuth's TwoSum; both go to acc.l.
__device__ __forceinline__ void df_mac(dfl& acc, const dfl& a, const dfl& b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float s = acc.h + p;
    const float bb = s - acc.h;
    const float t = (acc.h - (s - bb)) + (p - bb);
    acc.h = s;
    acc.l += t + e;
}
__device__ __forceinline__ void ld4(const dfl* p, dfl (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    const float4 y = *reinterpret_cast<const float4*>(p + 2);
    v[0] = dfl{x.x, x.y}; v[1] = dfl{x.z, x.w}; v[2] = dfl{y.x, y.y}; v[3] = dfl{y.z, y.w};
}
// conversions and multiply-add for the element types of the tiled kernels
template <typename T> __device__ __forceinline__ T tconv(double x) { return (T)x; }
template <> __device__ __forceinline__ dfl tconv<dfl>(double x) { return to_dfl(x); }
template <typename T> __device__ __forceinline__ void tmac(T& acc, const T& a, const T& b) { acc += a * b; }
template <> __device__ __forceinline__ void tmac<dfl>(dfl& acc, const dfl& a, const dfl& b) { df_mac(acc, a, b); }

// acc[a][b] += sum_q A[q][i0 + a] * B[q][j0 + b]  (A, B: [rp][rp] shared arrays, rp % 4 == 0)
template <typename T>
__device__ __forceinline__ void mma4x4(T (&acc)[4][4], const T* A, const T* B, int rp, int n, int i0, int j0) {
#pragma unroll 4
    for (int q = 0; q < n; ++q) {
        T a[4], b[4];
        ld4(A + q * rp + i0, a);
        ld4(B + q * rp + j0, b);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) tmac(acc[u][v], a[u], b[v]);
    }
}

// --------------------------------------------------------------------------- outputs of Z
struct ZOut {
    void* Zd;      // (2 r^2) rows
    void* Zf[2];   // r^2 rows
    int mode;      // 0 = FP64, 1 = BF16x3 (A pattern [hi|hi|lo]), 2 = TF32, 3 = TF32x3 ([hi|hi|lo])
    int ldd, ldf;  // row length in elements
    int Kp1, Kp2;  // K segment length (split modes)
    void* diag;    // [4][r][r][r]: rows j = p of Zd(a,a), Zd(b,b), Zf1, Zf2
    int ntypes;    // spin types computed (6, or 3 with the spin-flip specialisation) ...
    int tmap[6];   // ... and which: block type index -> t
};

template <typename T>
__device__ __forceinline__ void z_store(const ZOut& o, int which, size_t row, int col, T v) {
    void* base = which < 0 ? o.Zd : o.Zf[which];
    const size_t ld = which < 0 ? (size_t)o.ldd : (size_t)o.ldf;
    const int Kp = which < 0 ? o.Kp2 : o.Kp1;
    if (o.mode == 0) {
        ((double*)base)[row * ld + col] = (double)v;
    } else if (o.mode == 1) {
        __nv_bfloat16* p = (__nv_bfloat16*)base + row * ld;
        const float x = (float)v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        p[col] = hi;
        p[Kp + col] = hi;
        p[2 * Kp + col] = lo;
    } else if (o.mode == 3) {
        float* p = (float*)base + row * ld;
        const float hi = tl_tf32((float)v);
        const float lo = tl_tf32((float)v - hi);
        p[col] = hi;
        p[Kp + col] = hi;
        p[2 * Kp + col] = lo;
    } else {
        ((float*)base + row * ld)[col] = tl_tf32((float)v);
    }
}

// Four consecutive columns col..col+3 of one output row (requires row * ld + col % 4 == 0); MODE is
// the ZOut mode.
template <int MODE, typename T>
__device__ __forceinline__ void z_store4(const ZOut& o, int which, size_t row, int col, const T (&v)[4]) {
    void* base = which < 0 ? o.Zd : o.Zf[which];
    const size_t ld = which < 0 ? (size_t)o.ldd : (size_t)o.ldf;
    const int Kp = which < 0 ? o.Kp2 : o.Kp1;
    if (MODE == 0 || MODE == 4) {
        double* q = (double*)base + row * ld + col;
        *reinterpret_cast<double2*>(q) = make_double2((double)v[0], (double)v[1]);
        *reinterpret_cast<double2*>(q + 2) = make_double2((double)v[2], (double)v[3]);
    } else if (MODE == 1) {
        __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            hi[u] = __float2bfloat16_rn((float)v[u]);
            lo[u] = __float2bfloat16_rn((float)v[u] - __bfloat162float(hi[u]));
        }
        uint2 H, L;
        memcpy(&H, hi, 8);
        memcpy(&L, lo, 8);
        __nv_bfloat16* q = (__nv_bfloat16*)base + row * ld + col;
        *reinterpret_cast<uint2*>(q) = H;
        *reinterpret_cast<uint2*>(q + Kp) = H;
        *reinterpret_cast<uint2*>(q + 2 * Kp) = L;
    } else if (MODE == 3) {
        float hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            hi[u] = tl_tf32((float)v[u]);
            lo[u] = tl_tf32((float)v[u] - hi[u]);
        }
        float* q = (float*)base + row * ld + col;
        *reinterpret_cast<float4*>(q) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(q + Kp) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(q + 2 * Kp) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    } else {
        float* q = (float*)base + row * ld + col;
        *reinterpret_cast<float4*>(q) =
            make_float4(tl_tf32((float)v[0]), tl_tf32((float)v[1]), tl_tf32((float)v[2]), tl_tf32((float)v[3]));
    }
}

// Asynchronous global -> shared copies (cp.async, completion tracked per thread by commit groups).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The r x r slice W_kp[q][s] of spin type t (t = 0..5, see k_Z_pipe) and whether it is stored [s][q].
template <typename WT>
__device__ __forceinline__ const WT* z_slice(int t, int k, int p, int r, const WT* Waa, const WT* Wab, const WT* Wbb,
                                             bool& transposed) {
    const size_t r3 = (size_t)r * r * r, R2 = (size_t)r * r;
    switch (t) {
        case 0: transposed = false; return Waa + k * r3 + p * R2;
        case 1: transposed = false; return Wab + k * r3 + p * R2;
        case 2: transposed = true; return Wab + p * r3 + k * R2;
        case 3: transposed = false; return Wbb + k * r3 + p * R2;
        case 4: transposed = true; return Wab + k * r3 + p * R2;
        default: transposed = false; return Wab + p * r3 + k * R2;
    }
}

// Z_kp = 1D . W_kp for spin type t and all p of a chunk, one block per (t, k, p-chunk):
//   t=0 Zd(a,a): W_kp[q][s] = Waa[k][p][q][s], ga      t=1 Zd(a,b): Wab[k][p][q][s], ga
//   t=2 Zd(b,a): W_kp[q][s] = Wab[p][k][s][q], gb      t=3 Zd(b,b): Wbb[k][p][q][s], gb
//   t=4 Zf1:     W_kp[q][s] = Wab[k][p][s][q], gb      t=5 Zf2:     Wab[p][k][q][s], ga
// (the spin-flip sectors drop a sign -1 that their M operand drops too).  The W slices of the next ipb
// values of p are copied into shared memory (cp.async) while the current ipb slices are multiplied;
// each thread owns one 4 x 4 output tile of one slice (ipb * (rp/4)^2 threads).  W is FP64 on the FP64
// paths (MODE 0, and MODE 4, the Ozaki path: FP64 output as MODE 0, products in double-float) and the
// FP32 copy of W on the split path (MODE 1-3), so that no FP64 conversion runs here.
template <int MODE>
using ZWT = typename std::conditional<MODE == 0 || MODE == 4, double, float>::type;

template <int MODE, int RP = 0>   // RP > 0: compile-time padded size (product loop fully unrolled)
__global__ void __launch_bounds__(ZP_MAX_THREADS, (MODE == 0 || MODE == 4) ? 2 : 3) k_Z_pipe(int r, int ipb, int pchunk, const ZWT<MODE>* __restrict__ Waa,
                                                         const ZWT<MODE>* __restrict__ Wab,
                                                         const ZWT<MODE>* __restrict__ Wbb,
                                                         const double* __restrict__ gam, const __grid_constant__ ZOut o) {
    using T = typename std::conditional<MODE == 0, double,
                                        typename std::conditional<MODE == 4, dfl, float>::type>::type;
    using WT = ZWT<MODE>;
    constexpr int WV = 16 / sizeof(WT);                  // elements of a 16-byte copy
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int rp = RP ? RP : pad4(r), ldw = rp + 4, R2 = r * r, R2e = (R2 + WV - 1) / WV * WV;
    const int nt = rp / 4, nt2 = nt * nt;
    WT* stage = (WT*)tl_smem;                            // [ipb][R2e] raw W slices
    T* gT = (T*)(stage + (size_t)ipb * R2e);             // [q][j] = 1D[j][q], row pitch ldw
    T* Ws = gT + (size_t)rp * ldw;                       // [ipb][q][s], row pitch ldw
    const int nchunk = (r + pchunk - 1) / pchunk;
    const int tb = blockIdx.x / (r * nchunk);
    const int t = o.tmap[tb];
    const int rem = blockIdx.x - tb * r * nchunk;
    const int k = rem / nchunk;
    const int pb = (rem - k * nchunk) * pchunk;
    const int pe = min(r, pb + pchunk);
    const double* g = gam + ((t == 2 || t == 3 || t == 4) ? R2 : 0);
    // (int)((e + 1/2) / r) = e / r for e < r^2: the fraction stays at least 1/(2r) from an integer
    const float invr = 1.f / (float)r;
    const bool vec_ld = R2 % WV == 0 && ((reinterpret_cast<uintptr_t>(Waa) | reinterpret_cast<uintptr_t>(Wab) |
                                          reinterpret_cast<uintptr_t>(Wbb)) & 15) == 0;
    for (int e = threadIdx.x; e < (1 + ipb) * rp * ldw; e += blockDim.x) gT[e] = tconv<T>(0.0);
    __syncthreads();
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const int u = e / r, v = e - u * r;
        gT[v * ldw + u] = tconv<T>(g[e]);                // g[j][q] -> gT[q][j]
    }
    auto issue = [&](int p0) {
        const int n = min(ipb, pe - p0);
        for (int it = 0; it < n; ++it) {
            bool tr;
            const WT* src = z_slice<WT>(t, k, p0 + it, r, Waa, Wab, Wbb, tr);
            WT* dst = stage + (size_t)it * R2e;
            if (vec_ld)
                for (int e = threadIdx.x; e < R2 / WV; e += blockDim.x) cp_async16(dst + WV * e, src + WV * e);
            else if (sizeof(WT) == 8)
                for (int e = threadIdx.x; e < R2; e += blockDim.x) cp_async8(dst + e, src + e);
            else
                for (int e = threadIdx.x; e < R2; e += blockDim.x) cp_async4(dst + e, src + e);
        }
        cp_async_commit();
    };
    issue(pb);
    int which, sK, sP;
    if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
    else { which = t - 4; sK = 0; sP = 0; }
    const int dslot = t == 0 ? 0 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : -1;
    const int it_me = threadIdx.x / nt2, tile = threadIdx.x - it_me * nt2;
    const int j0 = (tile / nt) * 4, s0 = (tile % nt) * 4;
    const size_t ld = which < 0 ? (size_t)o.ldd : (size_t)o.ldf;
    for (int p0 = pb; p0 < pe; p0 += ipb) {
        const int n = min(ipb, pe - p0);
        cp_async_wait_all();
        __syncthreads();                                 // slices landed; previous products done with Ws
        for (int it = 0; it < n; ++it) {
            bool tr;
            z_slice<WT>(t, k, p0 + it, r, Waa, Wab, Wbb, tr);
            const WT* st = stage + (size_t)it * R2e;
            T* W = Ws + (size_t)it * rp * ldw;
            for (int e = threadIdx.x; e < R2; e += blockDim.x) {
                const int u = (int)(((float)e + 0.5f) * invr), v = e - u * r;   // e / r, see invr
                T x;
                if constexpr (std::is_same<T, WT>::value) x = st[e];   // FP32 W on the split path
                else x = tconv<T>((double)st[e]);
                if (tr) W[v * ldw + u] = x;                // src[s][q] -> W[q][s]
                else W[u * ldw + v] = x;
            }
        }
        __syncthreads();                                 // Ws ready, stage free
        if (p0 + ipb < pe) issue(p0 + ipb);              // the next slices load during the products
        if (it_me >= n) continue;
        const int p = p0 + it_me;
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = tconv<T>(0.0);
        const T* W = Ws + (size_t)it_me * rp * ldw;
        // with RP the loop runs over the zero-padded rows too (q < RP), at a constant trip count
        if constexpr (std::is_same<T, float>::value) {
            // packed FP32x2 FMA, pairs along s (the same FMA sequence per element as scalar code)
            float2 c2[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) c2[u][0] = c2[u][1] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int q = 0; q < (RP ? RP : r); ++q) {
                float a[4], b[4];
                ld4(gT + q * ldw + j0, a);
                ld4(W + q * ldw + s0, b);
                const float2 b0 = make_float2(b[0], b[1]), b1 = make_float2(b[2], b[3]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 x = make_float2(a[u], a[u]);
                    c2[u][0] = __ffma2_rn(x, b0, c2[u][0]);
                    c2[u][1] = __ffma2_rn(x, b1, c2[u][1]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[u][0] = c2[u][0].x; acc[u][1] = c2[u][0].y; acc[u][2] = c2[u][1].x; acc[u][3] = c2[u][1].y;
            }
        } else {
#pragma unroll 4
            for (int q = 0; q < (RP ? RP : r); ++q) {
                T a[4], b[4];
                ld4(gT + q * ldw + j0, a);
                ld4(W + q * ldw + s0, b);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) tmac(acc[u][v], a[u], b[v]);
            }
        }
        const int col0 = sP * R2 + p * r + s0;
        const bool vec_st = s0 + 3 < r && ((size_t)col0 & 3) == 0 && (ld & 3) == 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            if (j >= r) continue;
            const size_t row = (size_t)sK * R2 + (size_t)k * r + j;
            if (vec_st) z_store4<MODE, T>(o, which, row, col0, acc[u]);
            else
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (s0 + v < r) z_store<T>(o, which, row, col0 + v, acc[u][v]);
            if (dslot >= 0 && j == p)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (s0 + v < r) {
                        const size_t di = ((size_t)dslot * R2 + (size_t)k * r + p) * r + s0 + v;
                        if (MODE == 4) ((double*)o.diag)[di] = (double)acc[u][v];
                        else ((T*)o.diag)[di] = acc[u][v];
                    }
        }
    }
    cp_async_wait_all();
}

// w_a[k][s] = sum_p (Zd(a,a)[(k,p)][(p,s)] - Zf1[(k,p)][(p,s)]),  w_b likewise with Zd(b,b), Zf2
// (= sum_pq Waa[k][p][q][s] ga[p][q] - sum_pq Wab[k][p][s][q] gb[p][q], and the b analogue).
// One block per (spin, k): warp w sums p = w, w + 8, ...; lanes over s; the 8 partials are added
// in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_w_from_diag(int r, const T* __restrict__ diag, T* __restrict__ wout,
                                                     int flip) {
    __shared__ T part[8][ACSE_MAX_R];
    const int R2 = r * r;
    const int sp = blockIdx.x / r, k = blockIdx.x % r;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // flip: w_b = w_a (spin-flip specialisation; slots 1 and 3 are not formed)
    const T* d0 = diag + (size_t)(sp == 0 || flip ? 0 : 1) * R2 * r;
    const T* d1 = diag + (size_t)(sp == 0 || flip ? 2 : 3) * R2 * r;
    for (int s = lane; s < r; s += 32) {
        T acc = 0;
        for (int p = w; p < r; p += 8) acc += d0[((size_t)k * r + p) * r + s] - d1[((size_t)k * r + p) * r + s];
        part[w][s] = acc;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < r; s += blockDim.x) {
        T acc = 0;
#pragma unroll
        for (int g = 0; g < 8; ++g) acc += part[g][s];
        wout[(size_t)sp * R2 + (size_t)k * r + s] = acc;
    }
}

// ------------------------------------------------------------------------- B -> H
template <typename T>
struct BTiledArgs {
    int r;
    const T* X[3];      // pair GEMM outputs X^{ij}_{kp}, row stride r^2
    const T* Y[3];      // pair GEMM outputs Y^{ij}_{kl}
    const T* X5d;       // (2r^2) x (2r^2), rows (sK,k,j), columns (sI,i,l)
    const T* X5f1;      // r^2 x r^2
    const T* X5f2;
    const T* M[3];
    const T* gam;
    const T* w;
    const T* Q;
    T* H[3];
    const T* ny[4];     // NY three-body term per spin type (acse_ny.cu), added to B; null for V
    int flip;           // spin-flip specialisation: no bb items; the b-led particle-hole blocks and the
                        // second flip sector are read as their alpha-led flips
    const T* bx[8];     // precomputed products (k_B_pipe<.., true>): per type t, x1 rows at bx[2t] and
                        // x2^T rows at bx[2t + 1], r^2 per item (the type's item number, see acse_btc.cu)
};

// Block (i, j).  Spin types t = 0 (aaaa), 1 (bbbb), 2 (abab), 3 (abba):
//   x1 = sgn1 sum_p X[k][p] g1[p][l],  x2 = sgn2 sum_p w[k][p] Mt[p][l]   (r x r x r, register tiled)
//   B_t = (x1 - 2 x2 - x4 + 2 x5 + x7 - 2 x8) / 9 with the gathered x4, x5, x7, x8 of acse_elem.cu.
// B rows are kept in shared memory (Bs[t][k][l]) and combined into
//   H_aa = 4 Y_aa - 12 (B0 - B0_{k<->l}),  H_bb = 4 Y_bb - 12 (B1 - B1_{k<->l}),
//   H_ab = 4 Y_ab - 12 (B2 - B3_{k<->l}).
// STAGE: the particle-hole rows (x5, x8) and the Q / 1D vectors of (x4, x7) are staged in shared
// memory with coalesced loads before the products (off when shared memory would not fit).
// DF (T = double, the Ozaki path): the two products in double-float (C = dfl, the same 8 bytes as
// double in shared memory), everything else in FP64.
// PREX (Ozaki path): x1 and x2^T come precomputed for every pair (a.bx, k_Bx_oz of acse_zoz.cu): no operand
// staging, each thread reads its 4 x 4 tile of both.
template <typename T, bool STAGE, bool DF = false, bool PREX = false>
__global__ void __launch_bounds__(TL_TPB) k_B_tiled(const __grid_constant__ BTiledArgs<T> a) {
    using C = typename std::conditional<DF, dfl, T>::type;
    static_assert(sizeof(C) == sizeof(T), "product operands share the layout of T");
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int r = a.r;
    const int rp = pad4(r);
    const int R2 = r * r;
    C* XT = (C*)tl_smem;      // [p][k]
    C* G1 = XT + rp * rp;     // [p][l]
    C* WT = G1 + rp * rp;     // [p][k]
    C* MT = WT + rp * rp;     // [p][l]
    T* Bs = (T*)(MT + rp * rp);   // [2][r][r]: current pair of B types
    T* X5s = Bs + 2 * R2;     // [k][l] (STAGE)
    T* X8s = X5s + R2;
    T* vq = X8s + R2;         // 4 vectors of r: Q column, 1D row, Q column, 1D row (x4, x7)
    const int i = blockIdx.x / r, j = blockIdx.x % r;
    const size_t ij = (size_t)blockIdx.x;
    const T* ga = a.gam;
    const T* gb = a.gam + R2;
    const T* Qa = a.Q;
    const T* Qb = a.Q + R2;
    const int nt = rp / 4;
    const size_t R22 = 2 * (size_t)R2;
    for (int e = threadIdx.x; e < 4 * rp * rp; e += blockDim.x) XT[e] = tconv<C>(0.0);   // zero padding once
    for (int round = 0; round < 3; ++round) {
        const int ntypes = round < 2 ? 1 : 2;
        for (int tt = 0; tt < ntypes; ++tt) {
            const int t = round < 2 ? round : 2 + tt;
            const T* Xrow;
            const T* g1;
            const T* wv;
            const T* Mrow;
            bool xT = false, mT = true;
            T sgn1 = 1, sgn2 = 1;
            if (t == 0) { Xrow = a.X[0] + ij * R2; g1 = ga; wv = a.w; Mrow = a.M[0] + ij * R2; }
            else if (t == 1) { Xrow = a.X[2] + ij * R2; g1 = gb; wv = a.w + R2; Mrow = a.M[2] + ij * R2; }
            else if (t == 2) { Xrow = a.X[1] + ij * R2; g1 = gb; wv = a.w; Mrow = a.M[1] + ij * R2; mT = false; sgn2 = -1; }
            else { Xrow = a.X[1] + ij * R2; g1 = ga; wv = a.w + R2; Mrow = a.M[1] + ij * R2; xT = true; sgn1 = -1; }
            // particle-hole sources: x5 at row (k, j), column (i, l); x8 at row (k, i), column (j, l):
            //   T0: X5d(a,a) both   T1: X5d(b,b) both   T2: X5f1, X5d(a,b)   T3: X5d(b,a), X5f2
            const T* X5b;
            const T* X8b;
            size_t ld5, ld8;
            if (t == 0) { X5b = a.X5d; X8b = a.X5d; ld5 = ld8 = R22; }
            else if (t == 1) { X5b = X8b = a.X5d + R2 * R22 + R2; ld5 = ld8 = R22; }
            else if (t == 2) { X5b = a.X5f1; ld5 = R2; X8b = a.X5d + R2; ld8 = R22; }
            else { X5b = a.X5d + R2 * R22; ld5 = R22; X8b = a.X5f2; ld8 = R2; }
            // x4 = Q4[k] g4[l], x7 = Q7[k] g7[l] (zero vectors where a type has no such term)
            const T* Q4 = t == 0 ? Qa : t == 1 ? Qb : t == 2 ? Qa : nullptr;
            const T* g4 = t == 0 ? ga : t == 1 ? gb : t == 2 ? gb : nullptr;
            const T* Q7 = t == 0 ? Qa : t == 1 ? Qb : t == 3 ? Qb : nullptr;
            const T* g7 = t == 0 ? ga : t == 1 ? gb : t == 3 ? ga : nullptr;
            __syncthreads();
            for (int e = threadIdx.x; e < R2; e += blockDim.x) {
                const int u = e / r, v = e - u * r;
                if (!PREX) {
                    XT[xT ? u * rp + v : v * rp + u] = tconv<C>(Xrow[e]);   // T3 uses Xab[ij][p][k]
                    G1[u * rp + v] = tconv<C>(g1[e]);
                    WT[v * rp + u] = tconv<C>(wv[e]);                      // w[k][p] -> WT[p][k]
                    MT[mT ? v * rp + u : u * rp + v] = tconv<C>(Mrow[e]);  // M[(l,p)] -> MT[p][l]  or  M[(p,l)]
                }
                if (STAGE) {
                    X5s[e] = X5b[((size_t)u * r + j) * ld5 + (size_t)i * r + v];   // (k, l) = (u, v)
                    X8s[e] = X8b[((size_t)u * r + i) * ld8 + (size_t)j * r + v];
                }
            }
            if (STAGE)
                for (int e = threadIdx.x; e < r; e += blockDim.x) {
                    vq[e] = Q4 ? Q4[e * r + i] : (T)0;            // Q[k][i]
                    vq[r + e] = g4 ? g4[j * r + e] : (T)0;        // g[j][l]
                    vq[2 * r + e] = Q7 ? Q7[e * r + j] : (T)0;    // Q[k][j]
                    vq[3 * r + e] = g7 ? g7[i * r + e] : (T)0;    // g[i][l]
                }
            __syncthreads();
            T* Bt = Bs + (size_t)tt * R2;
            for (int tile = threadIdx.x; tile < nt * nt; tile += blockDim.x) {
                const int k0 = (tile / nt) * 4, l0 = (tile % nt) * 4;
                C x1[4][4], x2[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) x1[u][v] = x2[u][v] = tconv<C>(0.0);
                T p1[4][4], p2[4][4];   // PREX: x1[k][l] = bx[2t] row (ij, k), x2[k][l] = bx[2t + 1] row (ij, l)
                if constexpr (PREX) {
                    const T* b1 = a.bx[2 * t] + ij * R2;
                    const T* b2 = a.bx[2 * t + 1] + ij * R2;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int k = min(k0 + u, r - 1), l = min(l0 + v, r - 1);
                            p1[u][v] = b1[(size_t)k * r + l];
                            p2[u][v] = b2[(size_t)l * r + k];
                        }
                } else {
                    mma4x4<C>(x1, XT, G1, rp, r, k0, l0);
                    mma4x4<C>(x2, WT, MT, rp, r, k0, l0);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            p1[u][v] = (T)x1[u][v];
                            p2[u][v] = (T)x2[u][v];
                        }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + u;
                    if (k >= r) continue;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int l = l0 + v;
                        if (l >= r) continue;
                        T x4, x5, x7, x8;
                        if (STAGE) {
                            x4 = vq[k] * vq[r + l];
                            x7 = vq[2 * r + k] * vq[3 * r + l];
                            x5 = X5s[k * r + l];
                            x8 = X8s[k * r + l];
                        } else {
                            x4 = Q4 ? Q4[k * r + i] * g4[j * r + l] : (T)0;
                            x7 = Q7 ? Q7[k * r + j] * g7[i * r + l] : (T)0;
                            x5 = X5b[((size_t)k * r + j) * ld5 + (size_t)i * r + l];
                            x8 = X8b[((size_t)k * r + i) * ld8 + (size_t)j * r + l];
                        }
                        Bt[k * r + l] = (sgn1 * p1[u][v] - (T)2 * sgn2 * p2[u][v] - x4 + (T)2 * x5 + x7 - (T)2 * x8) *
                                            (T)(1.0 / 9.0) +
                                        (a.ny[t] ? a.ny[t][ij * R2 + (size_t)k * r + l] : (T)0);
                    }
                }
            }
        }
        __syncthreads();
        const int b = round == 0 ? 0 : round == 1 ? 2 : 1;   // output block aa, bb, ab
        const T* P = Bs;
        const T* Px = round < 2 ? Bs : Bs + R2;
        const T* Yrow = a.Y[b] + ij * R2;
        T* Hrow = a.H[b] + ij * R2;
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int k = e / r, l = e - k * r;
            Hrow[e] = (T)4 * Yrow[e] - (T)12 * (P[e] - Px[l * r + k]);
        }
    }
}

// ------------------------------------------------------------- B -> H, split-precision path
// Persistent variant for FP32: each block walks pairs (i, j) with a stride of the grid and, per pair,
// three rounds (aa: type 0, bb: type 1, ab: types 2 and 3).  A round's X and M rows are copied into
// shared memory (cp.async) while the previous round is computed.  1D (as [p][l]) and w (as w^T[p][k])
// of both spins are loaded once per block.  Within a type, the warps of group 1 (threads [0, S),
// S = nt^2 rounded up to a warp) own 4 x 4 tiles of x1 and the warps of group 2 (threads
// [S, S + nt^2)) own tiles of x2, so no warp runs both products; each product uses the tile
// ownership that makes all of its shared loads 16-byte vectors without bank conflicts:
//   RR (A as [k][q], B as [q][l]): rows k = kb + nt a, columns l = 4 lb + b, four q per step
//   CR (A as [q][k], B as [q][l]): k = 4 kb + a, l = 4 lb + b, one q per step
//   CC (A as [q][k], B as [l][q]): k = 4 kb + a, l = lb + nt b, four q per step
// x2 threads also gather x5, x8 (loads issued before their product) and store
// (-2 sgn2 x2 + 2 x5 - 2 x8) / 9 into Bs; x1 threads form x7 - x4 before their product and, after a
// barrier, add (sgn1 x1 - x4 + x7) / 9.
// Each thread's share of the Y row of the round is loaded into registers at the start of the round
// and used when H is formed at its end.
#define BP_MAX_THREADS 512   // r = 64: S = 256, 256 + 256 threads

// RP > 0: the padded size is a compile-time constant (loops fully unrolled, addresses folded); the
// padding rows and columns of the shared tiles are zero, so the loops may run to RP.
template <int KIND, int RP>
__device__ __forceinline__ void bp_product(float (&acc)[4][4], const float* A, const float* B, int ld_, int r_, int rp_,
                                           int nt_, int kb, int lb) {
    const int rp = RP ? RP : rp_, ld = RP ? RP + 4 : ld_, nt = RP ? RP / 4 : nt_, r = RP ? RP : r_;
    // paired accumulators for the packed FP32x2 FMA (two independent round-to-nearest FMAs, the same
    // sequence per element as scalar FMAs): c[a][h] = (acc[a][2h], acc[a][2h+1]) for RR and CR,
    // c[a][h] = (acc[2h][a], acc[2h+1][a]) for CC
    float2 c[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a) c[a][0] = c[a][1] = make_float2(0.f, 0.f);
    if (KIND == 0) {   // RR
        for (int q = 0; q < rp; q += 4) {
            float av[4][4], bv[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a) ld4(A + (kb + nt * a) * ld + q, av[a]);
#pragma unroll
            for (int u = 0; u < 4; ++u) ld4(B + (q + u) * ld + 4 * lb, bv[u]);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 x = make_float2(av[a][u], av[a][u]);
                    c[a][0] = __ffma2_rn(x, make_float2(bv[u][0], bv[u][1]), c[a][0]);
                    c[a][1] = __ffma2_rn(x, make_float2(bv[u][2], bv[u][3]), c[a][1]);
                }
        }
    } else if (KIND == 1) {   // CR
#pragma unroll 4
        for (int q = 0; q < r; ++q) {
            float av[4], bv[4];
            ld4(A + q * ld + 4 * kb, av);
            ld4(B + q * ld + 4 * lb, bv);
            const float2 b0 = make_float2(bv[0], bv[1]), b1 = make_float2(bv[2], bv[3]);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float2 x = make_float2(av[a], av[a]);
                c[a][0] = __ffma2_rn(x, b0, c[a][0]);
                c[a][1] = __ffma2_rn(x, b1, c[a][1]);
            }
        }
    } else {   // CC
        for (int q = 0; q < rp; q += 4) {
            float av[4][4], bv[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) ld4(A + (q + u) * ld + 4 * kb, av[u]);
#pragma unroll
            for (int b = 0; b < 4; ++b) ld4(B + (lb + nt * b) * ld + q, bv[b]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 a0 = make_float2(av[u][0], av[u][1]), a1 = make_float2(av[u][2], av[u][3]);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float2 y = make_float2(bv[b][u], bv[b][u]);
                    c[b][0] = __ffma2_rn(a0, y, c[b][0]);
                    c[b][1] = __ffma2_rn(a1, y, c[b][1]);
                }
            }
        }
    }
    if (KIND == 2) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[0][b] = c[b][0].x; acc[1][b] = c[b][0].y; acc[2][b] = c[b][1].x; acc[3][b] = c[b][1].y;
        }
    } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            acc[a][0] = c[a][0].x; acc[a][1] = c[a][0].y; acc[a][2] = c[a][1].x; acc[a][3] = c[a][1].y;
        }
    }
}

// Output coordinates of element (a, b) of a thread's tile for ownership KIND.
__device__ __forceinline__ int bp_k(int kind, int kb, int nt, int a) { return kind == 0 ? kb + nt * a : 4 * kb + a; }
__device__ __forceinline__ int bp_l(int kind, int lb, int nt, int b) { return kind == 2 ? lb + nt * b : 4 * lb + b; }

// PRE: the products x1 and x2 come precomputed (the tensor-core kernel of acse_btc.cu, r a multiple of
// 16): no operand staging, each thread reads its 4 x 4 tile of x1 and of x2^T with 16-byte loads; the
// shared memory holds only the B rows.
template <int MAXT, int MINB, int RP, bool PRE = false>
__global__ void __launch_bounds__(MAXT, MINB) k_B_pipe(const __grid_constant__ BTiledArgs<float> a) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int r = a.r, rp = RP ? RP : pad4(r), ld = rp + 4, R2 = r * r, bpitch = r + 1;
    const int nt = rp / 4, nt2 = nt * nt, S = (nt2 + 31) & ~31;
    const size_t tile = PRE ? 0 : (size_t)rp * ld;
    float* gA = (float*)tl_smem;          // 1D_a [p][l]
    float* gB = gA + tile;                // 1D_b
    float* wAT = gB + tile;               // w_a^T [p][k]
    float* wBT = wAT + tile;              // w_b^T
    float* buf = wBT + tile;              // [2][X, M] operand tiles, element (u, v) of a row at u * ld + v
    float* Bs = buf + 4 * tile;           // [2][r][r + 1]
    const size_t R22 = 2 * (size_t)R2;
    if (!PRE) {
        for (int e = threadIdx.x; e < 8 * (int)tile; e += blockDim.x) gA[e] = 0.f;
        __syncthreads();
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int u = e / r, v = e - u * r;
            gA[u * ld + v] = a.gam[e];
            gB[u * ld + v] = a.gam[R2 + e];
            wAT[v * ld + u] = a.w[e];          // w[k][p] -> w^T[p][k]
            wBT[v * ld + u] = a.w[R2 + e];
        }
    }
    const bool vec = (r & 3) == 0;
    const bool yvec = (r & 1) == 0;
    // row index of a flat index e < r^2 as (int)((e + 1/2) / r): the fraction stays at least 1/(2r)
    // away from an integer, far above the float rounding of the product for r <= 64
    const float invr = 1.f / (float)r;
    // Work items: [0, P) the aa pairs i < j, [P, 2P) the bb pairs i < j, [2P, 2P + r^2) every ab
    // pair (P = r(r-1)/2).  B and H of a same-spin sector are antisymmetric in (i, j), so the item
    // (i, j) also writes row (j, i) = -row (i, j); the rows (i, i) are zero.
    const int P = r * (r - 1) / 2, NB = a.flip ? 0 : P, NI = P + NB + R2;   // NB: bb items
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * (size_t)r * R2;
         e += (size_t)gridDim.x * blockDim.x) {
        const int sec = e < (size_t)r * R2 ? 0 : 2;
        const size_t f = e - (sec ? (size_t)r * R2 : 0);
        const int d = (int)(f / R2);
        a.H[sec][(size_t)(d * r + d) * R2 + (f - (size_t)d * R2)] = 0.f;
    }
    auto item = [&](int L, int& round, int& i, int& j) {
        if (L < P + NB) {
            round = L < P ? 0 : 1;
            const int q = L - round * P;
            int ii = 0;
            while (q >= ii * r - ii * (ii + 1) / 2 + (r - ii - 1)) ++ii;
            i = ii;
            j = q - (ii * r - ii * (ii + 1) / 2) + ii + 1;
        } else {
            round = 2;
            i = (L - P - NB) / r;
            j = (L - P - NB) - i * r;
        }
    };
    const int nsteps = (int)blockIdx.x < NI ? (NI - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // operands of step s (item blockIdx.x + s gridDim.x): X and M rows of its sector
    // (round 0 -> aa (0), round 1 -> bb (2), round 2 -> ab (1))
    auto issue = [&](int step, int slot) {
        if (PRE) return;
        int round, ii, jj;
        item((int)blockIdx.x + step * (int)gridDim.x, round, ii, jj);
        const size_t ij = (size_t)ii * r + jj;
        const int sec = round == 0 ? 0 : round == 1 ? 2 : 1;
        const float* src[2] = {a.X[sec] + ij * R2, a.M[sec] + ij * R2};
        for (int h = 0; h < 2; ++h) {
            float* dst = buf + (size_t)(2 * slot + h) * tile;
            if (vec) {
                const int c4 = r / 4;
                const float inv_c4 = 4.f / (float)r;
                for (int e = threadIdx.x; e < r * c4; e += blockDim.x) {
                    const int u = (int)(((float)e + 0.5f) * inv_c4), v = (e - u * c4) * 4;
                    cp_async16(dst + u * ld + v, src[h] + u * r + v);
                }
            } else {
                for (int e = threadIdx.x; e < R2; e += blockDim.x) {
                    const int u = e / r, v = e - u * r;
                    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + u * ld + v);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src[h] + e) : "memory");
                }
            }
        }
        cp_async_commit();
    };
    if (nsteps > 0) issue(0, 0);
    const int grp = threadIdx.x < S ? 0 : (threadIdx.x < S + nt2 ? 1 : 2);   // x1, x2, idle
    const int idx = grp == 0 ? threadIdx.x : threadIdx.x - S;
    const bool active = grp == 0 ? idx < nt2 : grp == 1;
    const int kb = idx / nt, lb = idx - (idx / nt) * nt;
    constexpr int YPT = 2;                         // float4 groups of the Y row held per thread
    for (int step = 0; step < nsteps; ++step) {
        int round, i, j;
        item((int)blockIdx.x + step * (int)gridDim.x, round, i, j);
        const int ij = i * r + j;
        const int cur = step & 1;
        const int b = round == 0 ? 0 : round == 1 ? 2 : 1;
        cp_async_wait_all();
        __syncthreads();                                    // operands landed; Bs and the other buffer free
        if (step + 1 < nsteps) issue(step + 1, cur ^ 1);
        // this thread's part of the Y row (used when H is formed at the end of the round)
        const float* Yrow = a.Y[b] + (size_t)ij * R2;
        float4 yv[YPT];
        if (yvec) {
#pragma unroll
            for (int u = 0; u < YPT; ++u) {
                const int g = threadIdx.x + u * blockDim.x;
                yv[u] = g < R2 / 4 ? reinterpret_cast<const float4*>(Yrow)[g] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        const float* Xs = buf + (size_t)(2 * cur) * tile;
        const float* Ms = Xs + tile;
        const int ntypes = round < 2 ? 1 : 2;
        for (int tt = 0; tt < ntypes; ++tt) {
            const int t = round < 2 ? round : 2 + tt;
            float* Bt = Bs + (size_t)tt * r * bpitch;
            float x1[4][4];
            // the particle-hole sources: x5 at row (k, j), column (i, l); x8 at row (k, i), column (j, l)
            const float* X5b;
            const float* X8b;
            size_t ld5, ld8;
            if (t == 0) { X5b = X8b = a.X5d; ld5 = ld8 = R22; }
            else if (t == 1) { X5b = X8b = a.X5d + R2 * R22 + R2; ld5 = ld8 = R22; }
            else if (t == 2) { X5b = a.X5f1; ld5 = R2; X8b = a.X5d + R2; ld8 = R22; }
            else if (!a.flip) { X5b = a.X5d + R2 * R22; ld5 = R22; X8b = a.X5f2; ld8 = R2; }
            else { X5b = a.X5d + R2; ld5 = R22; X8b = a.X5f1; ld8 = R2; }   // flips of X5d(b,a), X5f2
            float part1[4][4];   // x1 group: (s1 x1 + x7 - x4 - 2 x8) / 9, added after the barrier
            // this item's number among the type's items (rows of the precomputed products)
            const int it = round == 0 ? (int)blockIdx.x + step * (int)gridDim.x
                         : round == 1 ? (int)blockIdx.x + step * (int)gridDim.x - P : ij;
            if (grp == 1) {
                // x2 = sum_p w[k][p] M(l, p) (types 0, 1, 3: M row holds M[l][p]; type 2: M[p][l]) and the
                // gathered x5 (loaded before the product)
                // PRE: no product, so every type takes the 4 x 4 ownership k = 4 kb + u, l = 4 lb + v, under
                // which x2^T (four consecutive k) and x5 (four consecutive l) are 16-byte loads (r % 4 == 0)
                const int kind = (PRE || t == 2) ? 1 : 2;
                float g5[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = bp_k(kind, kb, nt, u);
                    const int kc = k < r ? k : r - 1;
                    const float* x5r = X5b + ((size_t)kc * r + j) * ld5 + (size_t)i * r;
                    if (PRE) {
                        const float4 q = *reinterpret_cast<const float4*>(x5r + 4 * lb);
                        g5[u][0] = q.x; g5[u][1] = q.y; g5[u][2] = q.z; g5[u][3] = q.w;
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int l = bp_l(kind, lb, nt, v);
                            g5[u][v] = x5r[l < r ? l : r - 1];
                        }
                    }
                }
                float acc[4][4];
                if (PRE) {   // x2[k][l] = x2^T row l, column k: four consecutive k per load
                    const float* x2t = a.bx[2 * t + 1] + (size_t)it * R2;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int l = bp_l(kind, lb, nt, v);
                        const float4 q = *reinterpret_cast<const float4*>(x2t + (size_t)l * r + 4 * kb);
                        acc[0][v] = q.x; acc[1][v] = q.y; acc[2][v] = q.z; acc[3][v] = q.w;
                    }
                } else {
                    const float* wT = (t == 0 || t == 2) ? wAT : wBT;
                    if (kind == 1) bp_product<1, RP>(acc, wT, Ms, ld, r, rp, nt, kb, lb);
                    else bp_product<2, RP>(acc, wT, Ms, ld, r, rp, nt, kb, lb);
                }
                const float c2 = t == 2 ? 2.f : -2.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = bp_k(kind, kb, nt, u);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int l = bp_l(kind, lb, nt, v);
                        if (k < r && l < r)
                            Bt[k * bpitch + l] = (c2 * acc[u][v] + 2.f * g5[u][v]) * (1.f / 9.f) +
                                                 (a.ny[t] ? a.ny[t][(size_t)ij * R2 + (size_t)k * r + l] : 0.f);
                    }
                }
            } else if (grp == 0 && active) {
                const int kind1 = t == 3 ? 1 : 0;
                // x7 - x4 - 2 x8, x7 - x4 = Q7[k][j] g7[i][l] - Q4[k][i] g4[j][l] (zero where a type has no
                // such term), loaded before the product
                const float* ga = a.gam;
                const float* gb = a.gam + R2;
                const float* Q4 = t == 0 ? a.Q : t == 1 ? a.Q + R2 : t == 2 ? a.Q : nullptr;
                const float* g4 = t == 0 ? ga : t == 1 ? gb : t == 2 ? gb : nullptr;
                const float* Q7 = t == 0 ? a.Q : t == 1 ? a.Q + R2 : t == 3 ? a.Q + R2 : nullptr;
                const float* g7 = t == 0 ? ga : t == 1 ? gb : t == 3 ? ga : nullptr;
                if (PRE) {   // r % 4 == 0: the 1D rows and the x8 row as 16-byte loads
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 g7v = g7 ? *reinterpret_cast<const float4*>(g7 + i * r + 4 * lb) : z4;
                    const float4 g4v = g4 ? *reinterpret_cast<const float4*>(g4 + j * r + 4 * lb) : z4;
                    const float g7a[4] = {g7v.x, g7v.y, g7v.z, g7v.w}, g4a[4] = {g4v.x, g4v.y, g4v.z, g4v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = bp_k(kind1, kb, nt, u);
                        const float q4 = Q4 ? Q4[k * r + i] : 0.f;
                        const float q7 = Q7 ? Q7[k * r + j] : 0.f;
                        const float4 x8 = *reinterpret_cast<const float4*>(X8b + ((size_t)k * r + i) * ld8 + (size_t)j * r + 4 * lb);
                        const float x8a[4] = {x8.x, x8.y, x8.z, x8.w};
#pragma unroll
                        for (int v = 0; v < 4; ++v) part1[u][v] = (q7 * g7a[v] - q4 * g4a[v]) - 2.f * x8a[v];
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = bp_k(kind1, kb, nt, u);
                        const int kc = k < r ? k : r - 1;
                        const float q4 = Q4 ? Q4[kc * r + i] : 0.f;
                        const float q7 = Q7 ? Q7[kc * r + j] : 0.f;
                        const float* x8r = X8b + ((size_t)kc * r + i) * ld8 + (size_t)j * r;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int l = 4 * lb + v;
                            const int lc = l < r ? l : r - 1;
                            const float x47 = (Q7 ? q7 * g7[i * r + lc] : 0.f) - (Q4 ? q4 * g4[j * r + lc] : 0.f);
                            part1[u][v] = x47 - 2.f * x8r[lc];
                        }
                    }
                }
                if (PRE) {   // x1 row k, four consecutive l per load
                    const float* x1r = a.bx[2 * t] + (size_t)it * R2;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = bp_k(kind1, kb, nt, u);
                        const float4 q = *reinterpret_cast<const float4*>(x1r + (size_t)k * r + 4 * lb);
                        x1[u][0] = q.x; x1[u][1] = q.y; x1[u][2] = q.z; x1[u][3] = q.w;
                    }
                } else {
                    const float* g1 = (t == 0 || t == 3) ? gA : gB;
                    if (t == 3) bp_product<1, RP>(x1, Xs, g1, ld, r, rp, nt, kb, lb);
                    else bp_product<0, RP>(x1, Xs, g1, ld, r, rp, nt, kb, lb);
                }
                const float s1 = t == 3 ? -1.f : 1.f;
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) part1[u][v] = (s1 * x1[u][v] + part1[u][v]) * (1.f / 9.f);
            }
            __syncthreads();                                // x2, x5 and ny in Bt
            if (grp == 0 && active) {
                const int kind1 = t == 3 ? 1 : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = bp_k(kind1, kb, nt, u);
                    if (k >= r) continue;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int l = 4 * lb + v;
                        if (l < r) Bt[k * bpitch + l] += part1[u][v];
                    }
                }
            }
        }
        __syncthreads();                                    // B types of this round complete
        const float* Pb = Bs;
        const float* Px = round < 2 ? Bs : Bs + (size_t)r * bpitch;
        float* Hrow = a.H[b] + (size_t)ij * R2;
        float* Hmir = round < 2 ? a.H[b] + (size_t)(j * r + i) * R2 : nullptr;   // row (j, i) = -row (i, j)
        if (yvec) {
#pragma unroll
            for (int u = 0; u < YPT; ++u) {
                const int g = threadIdx.x + u * blockDim.x;
                if (g < R2 / 4) {
                    const float yy[4] = {yv[u].x, yv[u].y, yv[u].z, yv[u].w};
                    float hh[4];
                    int k = (int)(((float)(4 * g) + 0.5f) * invr), l = 4 * g - k * r;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        hh[c] = 4.f * yy[c] - 12.f * (Pb[k * bpitch + l] - Px[l * bpitch + k]);
                        if (++l == r) { l = 0; ++k; }
                    }
                    reinterpret_cast<float4*>(Hrow)[g] = make_float4(hh[0], hh[1], hh[2], hh[3]);
                    if (Hmir) reinterpret_cast<float4*>(Hmir)[g] = make_float4(-hh[0], -hh[1], -hh[2], -hh[3]);
                }
            }
            for (int g = threadIdx.x + YPT * blockDim.x; g < R2 / 4; g += blockDim.x) {   // rows beyond the prefetch
                const float4 y4 = reinterpret_cast<const float4*>(Yrow)[g];
                const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
                float hh[4];
                int k = (int)(((float)(4 * g) + 0.5f) * invr), l = 4 * g - k * r;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    hh[c] = 4.f * yy[c] - 12.f * (Pb[k * bpitch + l] - Px[l * bpitch + k]);
                    if (++l == r) { l = 0; ++k; }
                }
                reinterpret_cast<float4*>(Hrow)[g] = make_float4(hh[0], hh[1], hh[2], hh[3]);
                if (Hmir) reinterpret_cast<float4*>(Hmir)[g] = make_float4(-hh[0], -hh[1], -hh[2], -hh[3]);
            }
        } else {
            for (int e = threadIdx.x; e < R2; e += blockDim.x) {
                const int k = e / r, l = e - k * r;
                const float hv = 4.f * Yrow[e] - 12.f * (Pb[k * bpitch + l] - Px[l * bpitch + k]);
                Hrow[e] = hv;
                if (Hmir) Hmir[e] = -hv;
            }
        }
    }
    cp_async_wait_all();
}

static size_t bp_smem(int r) {
    const size_t rp = pad4(r), tile = rp * (rp + 4);
    return (8 * tile + 2 * (size_t)r * (r + 1)) * sizeof(float);
}

// ------------------------------------------------------------------------------- launch
// Launch shape of k_Z_pipe: ipb slices per round (ipb * (rp/4)^2 <= ZP_MAX_THREADS threads, at most 4) and
// the p-chunk per block, chosen to balance the waves over the SMs (a block's first slices are not
// overlapped, hence the +1 round per block).
struct ZPlan {
    int ipb, threads, pchunk, blocks;
    size_t smem;
};
static ZPlan z_plan_compute(int r, size_t es, size_t ws, const void* kern) {   // es: tile, ws: W element bytes
    ZPlan z;
    const int rp = pad4(r), nt = rp / 4, nt2 = nt * nt;
    z.ipb = ZP_MAX_THREADS / nt2;
    if (z.ipb > 4) z.ipb = 4;
    if (z.ipb < 1) z.ipb = 1;
    z.threads = (z.ipb * nt2 + 31) / 32 * 32;
    const int wv = (int)(16 / ws);
    const int R2e = (r * r + wv - 1) / wv * wv;
    z.smem = (size_t)z.ipb * R2e * ws + (size_t)(1 + z.ipb) * rp * (rp + 4) * es;
    int per_sm = 1, nsm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, z.threads, z.smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long slots = (long)nsm * per_sm;
    double best = 1e30;
    z.pchunk = r;
    for (int pc = z.ipb; pc <= r; pc += z.ipb) {
        const long blocks = 6L * r * ((r + pc - 1) / pc);
        const double cost = (double)((blocks + slots - 1) / slots) * ((pc + z.ipb - 1) / z.ipb + 1);
        if (cost < best - 1e-9) { best = cost; z.pchunk = pc; }
    }
    z.blocks = 6 * r * ((r + z.pchunk - 1) / z.pchunk);
    return z;
}

// cached per host thread, output mode and r (the occupancy query is not free)
static ZPlan z_plan(int r, int mode, size_t es, const void* kern) {
    static thread_local int cached_r[5] = {-1, -1, -1, -1, -1};
    static thread_local ZPlan cached[5];
    if (cached_r[mode] != r) {
        cached[mode] = z_plan_compute(r, es, (mode == 0 || mode == 4) ? sizeof(double) : sizeof(float), kern);
        cached_r[mode] = r;
    }
    return cached[mode];
}

// W: the FP64 operand (FP64 and Ozaki paths); W32: its FP32 copy (split path).
int launch_Z_tiled(acse_ctx* c, const double* const W[3], const float* const W32[3]) {
    const int r = c->r;
    ZOut o;
    Work& w = c->w;
    const int R2 = r * r;
    const bool sf = acse_singlet(c);
    // spin-flip specialisation: Zd(b,b), Zd(b,a), Zf2 are the flips of Zd(a,a), Zd(a,b), Zf1 and only
    // the alpha-led rows of the diagonal particle-hole GEMM are formed
    o.ntypes = sf ? 3 : 6;
    const int tm_sf[6] = {0, 1, 4, 0, 0, 0};
    for (int k = 0; k < 6; ++k) o.tmap[k] = sf ? tm_sf[k] : k;
    if (c->opt.prec == ACSE_FP64) {
        o.Zd = w.Zd; o.Zf[0] = w.Zf1; o.Zf[1] = w.Zf2;
        o.mode = 0; o.ldd = 2 * R2; o.ldf = R2; o.Kp1 = o.Kp2 = 0; o.diag = w.zdiag;
        if (c->oz) {   // Ozaki path: the products on the tensor cores (acse_zoz.cu), else in double-float
            const int zs = launch_Z_oz(c, W, o.ntypes, o.tmap);
            if (zs == ACSE_OK) {
                k_w_from_diag<double><<<2 * r, 256, 0, c->stream>>>(r, w.zdiag, w.w, 0);
                ACSE_LAUNCHED(c);
                return ACSE_OK;
            }
            if (zs != ACSE_ERR_UNSUPPORTED) return zs;
            const ZPlan zp = z_plan(r, 4, sizeof(double), (const void*)k_Z_pipe<4>);
            k_Z_pipe<4><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W[0], W[1], W[2], w.gam, o);
        } else {
            const ZPlan zp = z_plan(r, 0, sizeof(double), (const void*)k_Z_pipe<0>);
            k_Z_pipe<0><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W[0], W[1], W[2], w.gam, o);
        }
        ACSE_LAUNCHED(c);
        k_w_from_diag<double><<<2 * r, 256, 0, c->stream>>>(r, w.zdiag, w.w, 0);
    } else {
        o.Zd = w.tc_Zd; o.Zf[0] = w.tc_Zf[0]; o.Zf[1] = w.tc_Zf[1];
        o.mode = c->opt.prec == ACSE_BF16X3 ? 1 : (c->opt.prec == ACSE_TF32X3 ? 3 : 2);
        o.ldd = c->nsplit * w.Kp2; o.ldf = c->nsplit * w.Kp1; o.Kp1 = w.Kp1; o.Kp2 = w.Kp2; o.diag = w.zdiag32;
        // BF16x3 with r a multiple of 16: the products on the tensor cores (acse_ztc.cu)
        const int zs = launch_Z_tc(c, W32, o.ntypes, o.tmap);
        if (zs == ACSE_OK) {
            k_w_from_diag<float><<<2 * r, 256, 0, c->stream>>>(r, w.zdiag32, w.w32, sf ? 1 : 0);
            ACSE_LAUNCHED(c);
            return ACSE_OK;
        }
        if (zs != ACSE_ERR_UNSUPPORTED) return zs;
        const bool r48 = o.mode == 1 && pad4(r) == 48;
        const void* kern = r48 ? (const void*)k_Z_pipe<1, 48>
                               : o.mode == 1 ? (const void*)k_Z_pipe<1> : o.mode == 3 ? (const void*)k_Z_pipe<3>
                                                                                      : (const void*)k_Z_pipe<2>;
        const ZPlan zp = z_plan(r, o.mode, sizeof(float), kern);
        if (r48)
            k_Z_pipe<1, 48><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W32[0], W32[1], W32[2], w.gam, o);
        else if (o.mode == 1)
            k_Z_pipe<1><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W32[0], W32[1], W32[2], w.gam, o);
        else if (o.mode == 3)
            k_Z_pipe<3><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W32[0], W32[1], W32[2], w.gam, o);
        else
            k_Z_pipe<2><<<zp.blocks / 6 * o.ntypes, zp.threads, zp.smem, c->stream>>>(r, zp.ipb, zp.pchunk, W32[0], W32[1], W32[2], w.gam, o);
        ACSE_LAUNCHED(c);
        k_w_from_diag<float><<<2 * r, 256, 0, c->stream>>>(r, w.zdiag32, w.w32, sf ? 1 : 0);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

static size_t b_smem(int r, size_t es, bool stage) {
    return (4 * (size_t)pad4(r) * pad4(r) + (stage ? 4 : 2) * (size_t)r * r + (stage ? 4 * (size_t)r : 0)) * es;
}
static const size_t k_smem_cap = 227 * 1024;

int launch_B_tiled(acse_ctx* c) {
    const int r = c->r;
    const int R2 = r * r;
    Work& w = c->w;
    if (c->opt.prec == ACSE_FP64) {
        BTiledArgs<double> a;
        a.r = r;
        for (int s = 0; s < 3; ++s) { a.X[s] = w.X[s]; a.Y[s] = w.Y[s]; a.M[s] = w.M[s]; a.H[s] = w.H[s]; }
        a.X5d = w.X5d; a.X5f1 = w.X5f1; a.X5f2 = w.X5f2;
        a.flip = 0;
        for (int t = 0; t < 4; ++t) a.ny[t] = (const double*)ny_terms(c, t);
        a.gam = w.gam; a.w = w.w; a.Q = w.Q;
        const bool st = b_smem(r, sizeof(double), true) <= k_smem_cap;
        const size_t sm = b_smem(r, sizeof(double), st);
        if (c->oz) {
            // Ozaki path: the products on the tensor cores (acse_zoz.cu) where it applies, else in
            // double-float; without staging two blocks fit an SM
            const int bs = launch_Bx_oz(c);
            if (bs == ACSE_OK) {
                for (int k = 0; k < 8; ++k) a.bx[k] = w.bx64[k];
                k_B_tiled<double, false, true, true><<<R2, TL_TPB, b_smem(r, sizeof(double), false), c->stream>>>(a);
            } else if (bs == ACSE_ERR_UNSUPPORTED) {
                k_B_tiled<double, false, true><<<R2, TL_TPB, b_smem(r, sizeof(double), false), c->stream>>>(a);
            } else {
                return bs;
            }
        } else {
            if (st) k_B_tiled<double, true><<<R2, TL_TPB, sm, c->stream>>>(a);
            else k_B_tiled<double, false><<<R2, TL_TPB, sm, c->stream>>>(a);
        }
    } else {
        BTiledArgs<float> a;
        a.r = r;
        for (int s = 0; s < 3; ++s) {
            a.X[s] = w.tc_pairC[s];
            a.Y[s] = w.tc_pairC[s] + (size_t)R2 * R2;   // rows r^2.. of [X; Y]
        }
        for (int s = 0; s < 3; ++s) {
            a.M[s] = w.M32[s];
            a.H[s] = w.H32[s];
        }
        a.flip = acse_singlet(c) ? 1 : 0;
        a.X5d = w.tc_X5d; a.X5f1 = w.tc_X5f[0]; a.X5f2 = w.tc_X5f[1];
        for (int t = 0; t < 4; ++t) a.ny[t] = (const float*)ny_terms(c, t);
        a.gam = w.gam32; a.w = w.w32; a.Q = w.Q32;
        for (int k = 0; k < 8; ++k) a.bx[k] = w.bx[k];
        // BF16x3, r a multiple of 16: the products on the tensor cores first, then the B kernel without them
        const int bs = launch_Bx_tc(c);
        if (bs == ACSE_OK) {
            static thread_local int pre_r = -1, pre_flip = -1, pre_grid = 0;
            const int nt = pad4(r) / 4, nt2 = nt * nt;
            const int threads = (((nt2 + 31) & ~31) + nt2 + 31) / 32 * 32;
            const size_t smem = 2 * (size_t)r * (r + 1) * sizeof(float);
            const bool r48 = r == 48;
            const void* kern = r48 ? (const void*)k_B_pipe<320, 2, 48, true> : threads <= 320
                                   ? (const void*)k_B_pipe<320, 2, 0, true> : (const void*)k_B_pipe<BP_MAX_THREADS, 1, 0, true>;
            if (pre_r != r || pre_flip != a.flip) {
                int per_sm = 1, nsm = 152, dev = 0;
                if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
                    per_sm < 1) {
                    cudaGetLastError();
                    per_sm = 1;
                }
                const int items = (a.flip ? 1 : 2) * (r * (r - 1) / 2) + R2;
                pre_grid = nsm * per_sm < items ? nsm * per_sm : items;
                pre_r = r;
                pre_flip = a.flip;
            }
            if (r48) k_B_pipe<320, 2, 48, true><<<pre_grid, threads, smem, c->stream>>>(a);
            else if (threads <= 320) k_B_pipe<320, 2, 0, true><<<pre_grid, threads, smem, c->stream>>>(a);
            else k_B_pipe<BP_MAX_THREADS, 1, 0, true><<<pre_grid, threads, smem, c->stream>>>(a);
            ACSE_LAUNCHED(c);
            return ACSE_OK;
        }
        if (bs != ACSE_ERR_UNSUPPORTED) return bs;
        static thread_local int cached_r = -1, cached_flip = -1, cached_grid = 0;
        const int nt2 = (pad4(r) / 4) * (pad4(r) / 4);
        const int threads = (((nt2 + 31) & ~31) + nt2 + 31) / 32 * 32;
        const bool small = threads <= 320;
        const bool r48 = pad4(r) == 48;
        const void* kern = r48 ? (const void*)k_B_pipe<320, 2, 48>
                               : small ? (const void*)k_B_pipe<320, 2, 0> : (const void*)k_B_pipe<BP_MAX_THREADS, 1, 0>;
        if (cached_r != r || cached_flip != a.flip) {
            int per_sm = 1, nsm = 152, dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, bp_smem(r)) != cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            const int items = (a.flip ? 1 : 2) * (r * (r - 1) / 2) + R2;   // same-spin pairs i < j, mixed pairs
            cached_grid = nsm * per_sm < items ? nsm * per_sm : items;
            cached_r = r;
            cached_flip = a.flip;
        }
        if (r48) k_B_pipe<320, 2, 48><<<cached_grid, threads, bp_smem(r), c->stream>>>(a);
        else if (small) k_B_pipe<320, 2, 0><<<cached_grid, threads, bp_smem(r), c->stream>>>(a);
        else k_B_pipe<BP_MAX_THREADS, 1, 0><<<cached_grid, threads, bp_smem(r), c->stream>>>(a);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int tiled_set_attrs() {
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)b_smem(ACSE_MAX_R, sizeof(double), false)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)b_smem(ACSE_MAX_R, sizeof(double), false)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)b_smem(ACSE_MAX_R, sizeof(double), false)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_pipe<320, 2, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bp_smem(48)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_pipe<320, 2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bp_smem(48)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_pipe<BP_MAX_THREADS, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bp_smem(ACSE_MAX_R)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<1, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_pipe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k_smem_cap));
    return ACSE_OK;
}
