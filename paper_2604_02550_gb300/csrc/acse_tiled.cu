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

#include "acse_internal.h"

#define TL_TPB 256

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
            for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
}

// --------------------------------------------------------------------------- outputs of Z
struct ZOut {
    void* Zd;      // (2 r^2) rows
    void* Zf[2];   // r^2 rows
    int mode;      // 0 = FP64, 1 = BF16x3 (A pattern [hi|hi|lo]), 2 = TF32
    int ldd, ldf;  // row length in elements
    int Kp1, Kp2;  // K segment length (split modes)
    void* diag;    // [4][r][r][r]: rows j = p of Zd(a,a), Zd(b,b), Zf1, Zf2
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

#define Z_PCH 8          // p values per block
#define Z_PREF 16        // slice elements prefetched per thread (r^2 <= 4096 = 16 x 256)

// Two consecutive columns col, col + 1 of one output row (col even, row length even).
template <typename T>
__device__ __forceinline__ void z_store2(const ZOut& o, int which, size_t row, int col, T v0, T v1) {
    void* base = which < 0 ? o.Zd : o.Zf[which];
    const size_t ld = which < 0 ? (size_t)o.ldd : (size_t)o.ldf;
    const int Kp = which < 0 ? o.Kp2 : o.Kp1;
    if (o.mode == 0) {
        *reinterpret_cast<double2*>((double*)base + row * ld + col) = make_double2((double)v0, (double)v1);
    } else if (o.mode == 1) {
        __nv_bfloat16* p = (__nv_bfloat16*)base + row * ld + col;
        const float x0 = (float)v0, x1 = (float)v1;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(x0, x1);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(x0 - __low2float(hi), x1 - __high2float(hi));
        *reinterpret_cast<__nv_bfloat162*>(p) = hi;
        *reinterpret_cast<__nv_bfloat162*>(p + Kp) = hi;
        *reinterpret_cast<__nv_bfloat162*>(p + 2 * Kp) = lo;
    } else {
        *reinterpret_cast<float2*>((float*)base + row * ld + col) = make_float2(tl_tf32((float)v0), tl_tf32((float)v1));
    }
}

// Block (t, k, p0..p0+Z_PCH-1), t = 0..5:
//   t=0 Zd(a,a): W_kp[q][s] = Waa[k][p][q][s], ga      t=1 Zd(a,b): Wab[k][p][q][s], ga
//   t=2 Zd(b,a): W_kp[q][s] = Wab[p][k][s][q], gb      t=3 Zd(b,b): Wbb[k][p][q][s], gb
//   t=4 Zf1:     W_kp[q][s] = Wab[k][p][s][q], gb      t=5 Zf2:     Wab[p][k][q][s], ga
// (the spin-flip sectors drop a sign -1 that their M operand drops too).  The 1D is staged once per
// block; the W slice of the next p is loaded into registers while the current one is multiplied.
template <typename T>
__device__ __forceinline__ const double* z_slice(int t, int k, int p, int r, const double* Waa, const double* Wab,
                                                const double* Wbb, bool& tr) {
    const size_t R2 = (size_t)r * r, r3 = R2 * r;
    switch (t) {
        case 0: tr = false; return Waa + k * r3 + p * R2;
        case 1: tr = false; return Wab + k * r3 + p * R2;
        case 2: tr = true; return Wab + p * r3 + k * R2;
        case 3: tr = false; return Wbb + k * r3 + p * R2;
        case 4: tr = true; return Wab + k * r3 + p * R2;
        default: tr = false; return Wab + p * r3 + k * R2;
    }
}

template <typename T>
__global__ void __launch_bounds__(TL_TPB) k_Z_tiled(int r, const double* __restrict__ Waa,
                                                    const double* __restrict__ Wab,
                                                    const double* __restrict__ Wbb,
                                                    const double* __restrict__ gam, const __grid_constant__ ZOut o) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int rp = pad4(r);
    T* Ws = (T*)tl_smem;          // [q][s]
    T* gT = Ws + rp * rp;         // [q][j] = 1D[j][q]
    const int R2 = r * r;
    const int nchunk = (r + Z_PCH - 1) / Z_PCH;
    const int t = blockIdx.x / (r * nchunk);
    const int k = (blockIdx.x / nchunk) % r;
    const int p0 = (blockIdx.x % nchunk) * Z_PCH;
    const int p1 = min(p0 + Z_PCH, r);
    const double* g = gam + ((t == 2 || t == 3 || t == 4) ? R2 : 0);
    for (int e = threadIdx.x; e < rp * rp; e += blockDim.x) {
        Ws[e] = (T)0;
        gT[e] = (T)0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const int u = e / r, v = e - u * r;
        gT[v * rp + u] = (T)g[e];                // g[j][q] -> gT[q][j]
    }
    int which, sK, sP, dslot;
    if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
    else { which = t - 4; sK = 0; sP = 0; }
    dslot = t == 0 ? 0 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : -1;
    const int nt = rp / 4;
    bool tr;
    T pre[Z_PREF];
    {
        const double* src = z_slice<T>(t, k, p0, r, Waa, Wab, Wbb, tr);
#pragma unroll
        for (int u = 0; u < Z_PREF; ++u) {
            const int e = threadIdx.x + u * TL_TPB;
            pre[u] = e < R2 ? (T)src[e] : (T)0;
        }
    }
    T* Os = gT + rp * rp;         // [j][s] output block of the current p
    for (int p = p0; p < p1; ++p) {
        __syncthreads();   // previous slice and output block consumed
#pragma unroll
        for (int u = 0; u < Z_PREF; ++u) {
            const int e = threadIdx.x + u * TL_TPB;
            if (e < R2) {
                const int a = e / r, b = e - a * r;
                if (tr) Ws[b * rp + a] = pre[u];   // src[s][q] -> Ws[q][s]
                else Ws[a * rp + b] = pre[u];
            }
        }
        __syncthreads();
        if (p + 1 < p1) {
            const double* src = z_slice<T>(t, k, p + 1, r, Waa, Wab, Wbb, tr);
#pragma unroll
            for (int u = 0; u < Z_PREF; ++u) {
                const int e = threadIdx.x + u * TL_TPB;
                pre[u] = e < R2 ? (T)src[e] : (T)0;
            }
        }
        for (int tile = threadIdx.x; tile < nt * nt; tile += blockDim.x) {
            const int j0 = (tile / nt) * 4, s0 = (tile % nt) * 4;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0;
            mma4x4<T>(acc, gT, Ws, rp, r, j0, s0);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) Os[(j0 + u) * rp + s0 + v] = acc[u][v];
        }
        __syncthreads();
        // rows (sK, k, j), columns (sP, p, s): r contiguous values per row, stored in pairs
        const int colbase = sP * R2 + p * r;
        if ((r & 1) == 0) {
            const int hr = r >> 1;
            for (int e = threadIdx.x; e < r * hr; e += blockDim.x) {
                const int j = e / hr, s2 = (e - j * hr) * 2;
                z_store2<T>(o, which, (size_t)sK * R2 + (size_t)k * r + j, colbase + s2, Os[j * rp + s2],
                            Os[j * rp + s2 + 1]);
            }
        } else {
            for (int e = threadIdx.x; e < R2; e += blockDim.x) {
                const int j = e / r, s2 = e - j * r;
                z_store<T>(o, which, (size_t)sK * R2 + (size_t)k * r + j, colbase + s2, Os[j * rp + s2]);
            }
        }
        if (dslot >= 0)
            for (int s2 = threadIdx.x; s2 < r; s2 += blockDim.x)
                ((T*)o.diag)[((size_t)dslot * R2 + (size_t)k * r + p) * r + s2] = Os[p * rp + s2];
    }
}

// w_a[k][s] = sum_p (Zd(a,a)[(k,p)][(p,s)] - Zf1[(k,p)][(p,s)]),  w_b likewise with Zd(b,b), Zf2
// (= sum_pq Waa[k][p][q][s] ga[p][q] - sum_pq Wab[k][p][s][q] gb[p][q], and the b analogue).
template <typename T>
__global__ void k_w_from_diag(int r, const T* __restrict__ diag, T* __restrict__ wout) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int R2 = r * r;
    if (e >= 2 * R2) return;
    const int sp = e / R2, k = (e / r) % r, s = e % r;
    const T* d0 = diag + (size_t)(sp == 0 ? 0 : 1) * R2 * r;
    const T* d1 = diag + (size_t)(sp == 0 ? 2 : 3) * R2 * r;
    T acc = 0;
    for (int p = 0; p < r; ++p) acc += d0[((size_t)k * r + p) * r + s] - d1[((size_t)k * r + p) * r + s];
    wout[e] = acc;
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
};

// Block (i, j).  Spin types t = 0 (aaaa), 1 (bbbb), 2 (abab), 3 (abba):
//   x1 = sgn1 sum_p X[k][p] g1[p][l],  x2 = sgn2 sum_p w[k][p] Mt[p][l]   (r x r x r, register tiled)
//   B_t = (x1 - 2 x2 - x4 + 2 x5 + x7 - 2 x8) / 9 with the gathered x4, x5, x7, x8 of acse_elem.cu.
// B rows are kept in shared memory (Bs[t][k][l]) and combined into
//   H_aa = 4 Y_aa - 12 (B0 - B0_{k<->l}),  H_bb = 4 Y_bb - 12 (B1 - B1_{k<->l}),
//   H_ab = 4 Y_ab - 12 (B2 - B3_{k<->l}).
// STAGE: the particle-hole rows (x5, x8) and the Q / 1D vectors of (x4, x7) are staged in shared
// memory with coalesced loads before the products (off when shared memory would not fit).
template <typename T, bool STAGE>
__global__ void __launch_bounds__(TL_TPB) k_B_tiled(const __grid_constant__ BTiledArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int r = a.r;
    const int rp = pad4(r);
    const int R2 = r * r;
    T* XT = (T*)tl_smem;      // [p][k]
    T* G1 = XT + rp * rp;     // [p][l]
    T* WT = G1 + rp * rp;     // [p][k]
    T* MT = WT + rp * rp;     // [p][l]
    T* Bs = MT + rp * rp;     // [2][r][r]: current pair of B types
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
    for (int e = threadIdx.x; e < 4 * rp * rp; e += blockDim.x) XT[e] = (T)0;   // zero padding once
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
                XT[xT ? u * rp + v : v * rp + u] = Xrow[e];   // T3 uses Xab[ij][p][k]
                G1[u * rp + v] = g1[e];
                WT[v * rp + u] = wv[e];                      // w[k][p] -> WT[p][k]
                MT[mT ? v * rp + u : u * rp + v] = Mrow[e];  // M[(l,p)] -> MT[p][l]  or  M[(p,l)]
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
                T x1[4][4], x2[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) x1[u][v] = x2[u][v] = 0;
                mma4x4<T>(x1, XT, G1, rp, r, k0, l0);
                mma4x4<T>(x2, WT, MT, rp, r, k0, l0);
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
                        Bt[k * r + l] = (sgn1 * x1[u][v] - (T)2 * sgn2 * x2[u][v] - x4 + (T)2 * x5 + x7 - (T)2 * x8) *
                                        (T)(1.0 / 9.0);
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

// ------------------------------------------------------------------------------- launch
int launch_Z_tiled(acse_ctx* c, const double* const W[3]) {
    const int r = c->r, rp = pad4(r);
    ZOut o;
    Work& w = c->w;
    const int R2 = r * r;
    if (c->opt.prec == ACSE_FP64) {
        o.Zd = w.Zd; o.Zf[0] = w.Zf1; o.Zf[1] = w.Zf2;
        o.mode = 0; o.ldd = 2 * R2; o.ldf = R2; o.Kp1 = o.Kp2 = 0; o.diag = w.zdiag;
        k_Z_tiled<double><<<6 * r * ((r + Z_PCH - 1) / Z_PCH), TL_TPB, 3 * rp * rp * sizeof(double), c->stream>>>(
            r, W[0], W[1], W[2], w.gam, o);
        ACSE_LAUNCHED(c);
        k_w_from_diag<double><<<(2 * R2 + 127) / 128, 128, 0, c->stream>>>(r, w.zdiag, w.w);
    } else {
        o.Zd = w.tc_Zd; o.Zf[0] = w.tc_Zf[0]; o.Zf[1] = w.tc_Zf[1];
        o.mode = c->opt.prec == ACSE_BF16X3 ? 1 : 2;
        o.ldd = c->nsplit * w.Kp2; o.ldf = c->nsplit * w.Kp1; o.Kp1 = w.Kp1; o.Kp2 = w.Kp2; o.diag = w.zdiag32;
        k_Z_tiled<float><<<6 * r * ((r + Z_PCH - 1) / Z_PCH), TL_TPB, 3 * rp * rp * sizeof(float), c->stream>>>(
            r, W[0], W[1], W[2], w.gam, o);
        ACSE_LAUNCHED(c);
        k_w_from_diag<float><<<(2 * R2 + 127) / 128, 128, 0, c->stream>>>(r, w.zdiag32, w.w32);
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
        a.gam = w.gam; a.w = w.w; a.Q = w.Q;
        if (b_smem(r, sizeof(double), true) <= k_smem_cap)
            k_B_tiled<double, true><<<R2, TL_TPB, b_smem(r, sizeof(double), true), c->stream>>>(a);
        else
            k_B_tiled<double, false><<<R2, TL_TPB, b_smem(r, sizeof(double), false), c->stream>>>(a);
    } else {
        BTiledArgs<float> a;
        a.r = r;
        for (int s = 0; s < 3; ++s) {
            a.X[s] = w.tc_pairC[s];
            a.Y[s] = w.tc_pairC[s] + (size_t)R2 * R2;   // rows r^2.. of [X; Y]
            a.M[s] = w.M32[s];
            a.H[s] = w.H32[s];
        }
        a.X5d = w.tc_X5d; a.X5f1 = w.tc_X5f[0]; a.X5f2 = w.tc_X5f[1];
        a.gam = w.gam32; a.w = w.w32; a.Q = w.Q32;
        k_B_tiled<float, true><<<R2, TL_TPB, b_smem(r, sizeof(float), true), c->stream>>>(a);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int tiled_set_attrs() {
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k_smem_cap));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)b_smem(ACSE_MAX_R, sizeof(double), false)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_B_tiled<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)b_smem(ACSE_MAX_R, sizeof(float), true)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       3 * ACSE_MAX_R * ACSE_MAX_R * (int)sizeof(double)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       3 * ACSE_MAX_R * ACSE_MAX_R * (int)sizeof(float)));
    return ACSE_OK;
}
