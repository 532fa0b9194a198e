// Shared-memory tiled O(r^5) kernels of a contraction pass, for both arithmetic paths
// (T = double for the FP64 path, T = float for the split-precision path).
//
//   Z^{kp}_{js} = sum_q W^{kp}_{qs} 1D^j_q     -> for each (k, p): Z_kp = 1D . W_kp   (r x r x r)
//   w^k_s       = sum_pq W^{kp}_{qs} 1D^p_q     -> one block per (spin, k)
//   B spin types T0..T3 from X, M, w, Q, 1D and the particle-hole outputs X5
//                                              -> one block per pair (i, j): X1 = X_ij . 1D and
//                                                 X2 = w . M_ij^T are r x r x r products
// The index maps are the ones of the FP64 reference kernels documented in acse_elem.cu.
#include <cuda_bf16.h>

#include "acse_internal.h"

#define TL_TPB 256

__device__ __forceinline__ float tl_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// --------------------------------------------------------------------------- outputs of Z
// FP64 path: plain rows.  Split path: K-concatenated operand rows (pattern A: [hi|hi|lo]).
struct ZOut {
    void* Zd;      // (2 r^2) rows
    void* Zf[2];   // r^2 rows
    int mode;      // 0 = FP64, 1 = BF16x3, 2 = TF32
    int ldd, ldf;  // row length in elements
    int Kp1, Kp2;  // K segment length (split modes)
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
    } else {
        ((float*)base + row * ld)[col] = tl_tf32((float)v);
    }
}

// Block (t, k, p), t = 0..5:
//   t=0 Zd(a,a): W_kp[q][s] = Waa[k][p][q][s], ga      t=1 Zd(a,b): Wab[k][p][q][s], ga
//   t=2 Zd(b,a): W_kp[q][s] = Wab[p][k][s][q], gb      t=3 Zd(b,b): Wbb[k][p][q][s], gb
//   t=4 Zf1:     W_kp[q][s] = Wab[k][p][s][q], gb      t=5 Zf2:     Wab[p][k][q][s], ga
template <typename T>
__global__ void __launch_bounds__(TL_TPB) k_Z_tiled(int r, const double* __restrict__ Waa,
                                                    const double* __restrict__ Wab,
                                                    const double* __restrict__ Wbb,
                                                    const double* __restrict__ gam, const __grid_constant__ ZOut o) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    T* Ws = (T*)tl_smem;          // [q][s]
    T* gs = Ws + r * r;           // [j][q]
    const int R2 = r * r;
    const int t = blockIdx.x / R2;
    const int kp = blockIdx.x % R2;
    const int k = kp / r, p = kp % r;
    const size_t r3 = (size_t)R2 * r;
    const bool beta_g = (t == 2 || t == 3 || t == 4);
    const double* g = gam + (beta_g ? R2 : 0);
    const double* src;
    bool transposed;
    switch (t) {
        case 0: src = Waa + k * r3 + (size_t)p * R2; transposed = false; break;
        case 1: src = Wab + k * r3 + (size_t)p * R2; transposed = false; break;
        case 2: src = Wab + p * r3 + (size_t)k * R2; transposed = true; break;
        case 3: src = Wbb + k * r3 + (size_t)p * R2; transposed = false; break;
        case 4: src = Wab + k * r3 + (size_t)p * R2; transposed = true; break;
        default: src = Wab + p * r3 + (size_t)k * R2; transposed = false; break;
    }
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const T v = (T)src[e];
        if (transposed) Ws[(e % r) * r + e / r] = v;   // src[s][q] -> Ws[q][s]
        else Ws[e] = v;
        gs[e] = (T)g[e];
    }
    __syncthreads();
    int which, sK, sP;
    if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
    else { which = t - 4; sK = 0; sP = 0; }
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const int j = e / r, s = e % r;
        T acc = 0;
        for (int q = 0; q < r; ++q) acc += gs[j * r + q] * Ws[q * r + s];
        const size_t row = (size_t)sK * R2 + (size_t)k * r + j;
        const int col = sP * R2 + p * r + s;
        z_store<T>(o, which, row, col, acc);
    }
}

// --------------------------------------------------------------------------------- w
// Block (sp, k):
//   w_a[k][s] = sum_pq Waa[k][p][q][s] ga[p][q] - sum_pq Wab[k][p][s][q] gb[p][q]
//   w_b[k][s] = sum_pq Wbb[k][p][q][s] gb[p][q] - sum_pq Wab[p][k][q][s] ga[p][q]
// Thread (g, s) accumulates rows g, g+G, ... of an (rows x r) slice read along s (coalesced);
// the a-spin exchange slice Wab[k][p][s][q] is read row by row along q by whole warps.  All
// partials are combined in a fixed order.
template <typename T>
__global__ void __launch_bounds__(TL_TPB) k_w_tiled(int r, const double* __restrict__ Waa,
                                                    const double* __restrict__ Wab,
                                                    const double* __restrict__ Wbb,
                                                    const double* __restrict__ gam, T* __restrict__ wout) {
    __shared__ double part[TL_TPB];
    __shared__ double wpart[TL_TPB / 32][ACSE_MAX_R];
    const int sp = blockIdx.x / r, k = blockIdx.x % r;
    const int R2 = r * r;
    const size_t r3 = (size_t)R2 * r;
    const double* ga = gam;
    const double* gb = gam + R2;
    const int G = TL_TPB / r;            // row groups (r <= 64 -> G >= 4)
    const int g = threadIdx.x / r, s = threadIdx.x % r;
    double acc = 0.0;
    if (g < G) {
        if (sp == 0) {
            const double* W = Waa + k * r3;
            for (int pq = g; pq < R2; pq += G) acc += W[(size_t)pq * r + s] * ga[pq];
        } else {
            const double* W = Wbb + k * r3;
            for (int pq = g; pq < R2; pq += G) acc += W[(size_t)pq * r + s] * gb[pq];
            // - sum_pq Wab[p][k][q][s] ga[p][q]: rows (p, q) of the slices Wab[p][k]
            for (int pq = g; pq < R2; pq += G) {
                const int pp = pq / r, q = pq % r;
                acc -= Wab[pp * r3 + (size_t)k * R2 + (size_t)q * r + s] * ga[pq];
            }
        }
    }
    part[threadIdx.x] = acc;
    // a-spin exchange term: - sum_p sum_q Wab[k][p][s][q] gb[p][q], warp per row (p, s)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s2 = lane; s2 < r; s2 += 32) wpart[warp][s2] = 0.0;
    __syncwarp();
    if (sp == 0) {
        for (int row = warp; row < R2; row += TL_TPB / 32) {
            const int pp = row / r, s2 = row % r;
            const double* Wr = Wab + k * r3 + (size_t)row * r;
            double d = 0.0;
            for (int q = lane; q < r; q += 32) d += Wr[q] * gb[pp * r + q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
            if (lane == 0) wpart[warp][s2] -= d;
        }
    }
    __syncthreads();
    for (int s2 = threadIdx.x; s2 < r; s2 += blockDim.x) {
        double v = 0.0;
        for (int gg = 0; gg < G; ++gg) v += part[gg * r + s2];
        for (int w = 0; w < TL_TPB / 32; ++w) v += wpart[w][s2];
        wout[(size_t)sp * R2 + k * r + s2] = (T)v;
    }
}

// ------------------------------------------------------------------------- B spin types
template <typename T>
struct BTiledArgs {
    int r;
    const T* X[3];      // pair GEMM outputs X^{ij}_{kp}, row stride r^2
    const T* X5d;       // (2r^2) x (2r^2)
    const T* X5f1;
    const T* X5f2;
    const T* M[3];
    const T* gam;
    const T* w;
    const T* Q;
    T* Tout[4];
};

// Block (i, j).  For each spin type: stage the X and M rows of (i, j) and the needed 1D / w in
// shared memory, then every thread forms outputs (k, l) from two length-r dot products and four
// gathered terms.
template <typename T>
__global__ void __launch_bounds__(TL_TPB) k_B_tiled(const __grid_constant__ BTiledArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int r = a.r;
    const int R2 = r * r;
    const size_t R22 = 2 * (size_t)R2;
    T* Xs = (T*)tl_smem;     // [k][p] (x1 operand)
    T* gs = Xs + R2;         // [p][l]
    T* ws = gs + R2;         // [k][p]
    T* Ms = ws + R2;         // [p][l] (x2 operand, M row transposed as needed)
    const int i = blockIdx.x / r, j = blockIdx.x % r;
    const size_t ij = (size_t)blockIdx.x;
    const T* ga = a.gam;
    const T* gb = a.gam + R2;
    const T* Qa = a.Q;
    const T* Qb = a.Q + R2;
    for (int t = 0; t < 4; ++t) {
        // stage: x1 = sgn1 sum_p Xs[k][p] gs[p][l];  x2 = sgn2 sum_p ws[k][p] Ms[p][l]
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
        __syncthreads();
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int u = e / r, v = e % r;
            Xs[xT ? v * r + u : e] = Xrow[e];   // T3 uses Xab[ij][p][k]: Xs[k][p] = X[(p,k)]
            gs[e] = g1[e];
            ws[e] = wv[e];
            Ms[mT ? v * r + u : e] = Mrow[e];   // M row [l][p] -> Ms[p][l] (types 0, 1, 3)
        }
        __syncthreads();
        T* out = a.Tout[t] + ij * R2;
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int k = e / r, l = e % r;
            T x1 = 0, x2 = 0;
            for (int p = 0; p < r; ++p) {
                x1 += Xs[k * r + p] * gs[p * r + l];
                x2 += ws[k * r + p] * Ms[p * r + l];
            }
            x1 *= sgn1;
            x2 *= sgn2;
            T x4 = 0, x5, x7 = 0, x8;
            if (t < 2) {
                const T* gg = t == 0 ? ga : gb;
                const T* QQ = t == 0 ? Qa : Qb;
                x4 = QQ[k * r + i] * gg[j * r + l];
                x7 = QQ[k * r + j] * gg[i * r + l];
                const size_t off = (size_t)t * R2;
                x5 = a.X5d[(off + (size_t)k * r + j) * R22 + off + (size_t)i * r + l];
                x8 = a.X5d[(off + (size_t)k * r + i) * R22 + off + (size_t)j * r + l];
            } else if (t == 2) {
                x4 = Qa[k * r + i] * gb[j * r + l];
                x5 = a.X5f1[((size_t)k * r + j) * R2 + (size_t)i * r + l];
                x8 = a.X5d[((size_t)k * r + i) * R22 + R2 + (size_t)j * r + l];
            } else {
                x5 = a.X5d[(R2 + (size_t)k * r + j) * R22 + (size_t)i * r + l];
                x7 = Qb[k * r + j] * ga[i * r + l];
                x8 = a.X5f2[((size_t)k * r + i) * R2 + (size_t)j * r + l];
            }
            out[e] = (x1 - (T)2 * x2 - x4 + (T)2 * x5 + x7 - (T)2 * x8) * (T)(1.0 / 9.0);
        }
    }
}

// ------------------------------------------------------------------------------- launch
int launch_Z_tiled(acse_ctx* c, const double* const W[3]) {
    const int r = c->r;
    ZOut o;
    Work& w = c->w;
    const int R2 = r * r;
    if (c->opt.prec == ACSE_FP64) {
        o.Zd = w.Zd; o.Zf[0] = w.Zf1; o.Zf[1] = w.Zf2;
        o.mode = 0; o.ldd = 2 * R2; o.ldf = R2; o.Kp1 = o.Kp2 = 0;
        k_Z_tiled<double><<<6 * R2, TL_TPB, 2 * R2 * sizeof(double), c->stream>>>(r, W[0], W[1], W[2], w.gam, o);
    } else {
        o.Zd = w.tc_Zd; o.Zf[0] = w.tc_Zf[0]; o.Zf[1] = w.tc_Zf[1];
        o.mode = c->opt.prec == ACSE_BF16X3 ? 1 : 2;
        o.ldd = c->nsplit * w.Kp2; o.ldf = c->nsplit * w.Kp1; o.Kp1 = w.Kp1; o.Kp2 = w.Kp2;
        k_Z_tiled<float><<<6 * R2, TL_TPB, 2 * R2 * sizeof(float), c->stream>>>(r, W[0], W[1], W[2], w.gam, o);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int launch_w_tiled(acse_ctx* c, const double* const W[3]) {
    const int r = c->r;
    if (c->opt.prec == ACSE_FP64)
        k_w_tiled<double><<<2 * r, TL_TPB, 0, c->stream>>>(r, W[0], W[1], W[2], c->w.gam, c->w.w);
    else
        k_w_tiled<float><<<2 * r, TL_TPB, 0, c->stream>>>(r, W[0], W[1], W[2], c->w.gam, c->w.w32);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int launch_B_tiled(acse_ctx* c) {
    const int r = c->r;
    const int R2 = r * r;
    Work& w = c->w;
    if (c->opt.prec == ACSE_FP64) {
        BTiledArgs<double> a;
        a.r = r;
        for (int s = 0; s < 3; ++s) { a.X[s] = w.X[s]; a.M[s] = w.M[s]; }
        a.X5d = w.X5d; a.X5f1 = w.X5f1; a.X5f2 = w.X5f2;
        a.gam = w.gam; a.w = w.w; a.Q = w.Q;
        for (int t = 0; t < 4; ++t) a.Tout[t] = w.T[t];
        const size_t sm = 4 * (size_t)R2 * sizeof(double);
        k_B_tiled<double><<<R2, TL_TPB, sm, c->stream>>>(a);
    } else {
        BTiledArgs<float> a;
        a.r = r;
        for (int s = 0; s < 3; ++s) { a.X[s] = w.tc_pairC[s]; a.M[s] = w.M32[s]; }
        a.X5d = w.tc_X5d; a.X5f1 = w.tc_X5f[0]; a.X5f2 = w.tc_X5f[1];
        a.gam = w.gam32; a.w = w.w32; a.Q = w.Q32;
        for (int t = 0; t < 4; ++t) a.Tout[t] = w.T32[t];
        const size_t sm = 4 * (size_t)R2 * sizeof(float);
        k_B_tiled<float><<<R2, TL_TPB, sm, c->stream>>>(a);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int tiled_set_attrs() {
    const int max64 = 4 * ACSE_MAX_R * ACSE_MAX_R * (int)sizeof(double);   // 128 KiB at r = 64
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max64));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max64 / 2));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max64 / 2));
    return ACSE_OK;
}
