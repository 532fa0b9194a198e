// Adjoint of the ACSE trajectory (new; the paper has no adjoint): gradients of
//     f = wE E(D_n) + wN ||A(D_n)||^2,   D_{k+1} = D_k + eps U(D_k),   U(D) = 1/2 G(mask(A(D)); D),
//     A(D) = G(K/2; D)
// with respect to h, V (through K, Eq. 2) and D_0, FP64 path.
//
// Two vector-Jacobian products of a contraction pass G(W; D) are needed:
//  * with respect to W: the commutator bilinear form beta(X, Y) = sum_spin-orbital X . G(Y) is
//    antisymmetric, beta(X, Y) = -beta(Y, X), with the Valdemoro 3-RDM as with the exact one
//    (checked by the oracle tests).  For block cotangents Gb this gives
//        dL/dW_aa = -G(Gh)_aa,  dL/dW_bb = -G(Gh)_bb,  dL/dW_ab = -4 G(Gh)_ab,
//    Gh = (P Gb_aa, Gb_ab / 4, P Gb_bb) (P: antisymmetriser within the index pairs), evaluated as
//    two forward passes on the pair-Hermitian (s = +1) and anti-Hermitian (s = -1) parts of Gh;
//  * with respect to D: a reverse pass through the factorisation of acse_elem.cu / acse_tiled.cu
//    (G = H - s H^T, H = 4Y - 12(P - P'_{k<->l}), the B spin types, the pair and particle-hole GEMMs,
//    Z, w, Q, M = 3D - 2(1D^1D), 1D = 2/(N-1) tr D), written out below term by term.
#include <math.h>
#include <string.h>

#include "acse_internal.h"

#define AD_TPB 256

int acse_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int sW, double scale, int mask,
                  double* const out[3], double* norm2_dst, int prep_D);

static inline int ad_grid(size_t n) {
    size_t g = (n + AD_TPB - 1) / AD_TPB;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

__device__ __forceinline__ double ad_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double ad_block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = ad_warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = ad_warp_sum(v);
    __syncthreads();
    return v;
}

#define FOR_N(e, n) for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (n); e += (size_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------------ small helpers
// out_b[ij][kl] = a in_b[ij][kl] + b in_b[kl][ij] for the three blocks (pair transpose).
__global__ void k_pair_combine(int r, const double* __restrict__ i0, const double* __restrict__ i1,
                               const double* __restrict__ i2, double a, double b, double* o0, double* o1, double* o2) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4, ij = g / R2, kl = g % R2;
        const double* in = blk == 0 ? i0 : blk == 1 ? i1 : i2;
        double* out = blk == 0 ? o0 : blk == 1 ? o1 : o2;
        out[g] = a * in[g] + b * in[kl * R2 + ij];
    }
}

// Block cotangent -> Gh (spin-orbital normalised): aa, bb antisymmetrised within pairs, ab / 4;
// scaled by `scale`.
__global__ void k_to_so_cotangent(int r, const double* __restrict__ g0, const double* __restrict__ g1,
                                  const double* __restrict__ g2, double scale, double* o0, double* o1, double* o2) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4;
        const int i = (int)(g / (R2 * r)), j = (int)((g / R2) % r), k = (int)((g / r) % r), l = (int)(g % r);
        if (blk == 1) {
            o1[g] = 0.25 * scale * g1[g];
        } else {
            const double* x = blk == 0 ? g0 : g2;
            const size_t ji = (size_t)j * r + i, ij = (size_t)i * r + j, kl = (size_t)k * r + l, lk = (size_t)l * r + k;
            const double v = 0.25 * (x[ij * R2 + kl] - x[ji * R2 + kl] - x[ij * R2 + lk] + x[ji * R2 + lk]);
            (blk == 0 ? o0 : o2)[g] = scale * v;
        }
    }
}

// acc_b += mul_b * x_b with mul = (m0, m1, m2) per block.
__global__ void k_axpy3(size_t n4, const double* __restrict__ x0, const double* __restrict__ x1,
                        const double* __restrict__ x2, double m0, double m1, double m2, double* a0, double* a1,
                        double* a2) {
    FOR_N(e, 3 * n4) {
        const int b = (int)(e / n4);
        const size_t g = e % n4;
        if (b == 0) a0[g] += m0 * x0[g];
        else if (b == 1) a1[g] += m1 * x1[g];
        else a2[g] += m2 * x2[g];
    }
}

// out = in with the all-active entries zeroed (or a copy when mask is off).
__global__ void k_mask_copy(int r, const double* __restrict__ i0, const double* __restrict__ i1,
                            const double* __restrict__ i2, int mask, int lo, int hi, double* o0, double* o1, double* o2) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4;
        const int i = (int)(g / (R2 * r)), j = (int)((g / R2) % r), k = (int)((g / r) % r), l = (int)(g % r);
        const double* in = blk == 0 ? i0 : blk == 1 ? i1 : i2;
        double v = in[g];
        if (mask && i >= lo && i < hi && j >= lo && j < hi && k >= lo && k < hi && l >= lo && l < hi) v = 0.0;
        (blk == 0 ? o0 : blk == 1 ? o1 : o2)[g] = v;
    }
}

// ------------------------------------------------------------------ reverse of the assembly
// From Hb (cotangent of H): Yb = 4 Hb;  tau = Bbar / 9 with
//   B0bar = -12 Hb_aa + 12 Hb_aa(k<->l), B1bar likewise, B2bar = -12 Hb_ab, B3bar = 12 Hb_ab(k<->l).
__global__ void k_adj_tau(int r, const double* __restrict__ Haa, const double* __restrict__ Hab,
                          const double* __restrict__ Hbb, double* Y0, double* Y1, double* Y2, double* t0, double* t1,
                          double* t2, double* t3) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    const double c = 12.0 / 9.0;
    FOR_N(g, n4) {
        const size_t ij = g / R2;
        const int k = (int)((g / r) % r), l = (int)(g % r);
        const size_t lk = ij * R2 + (size_t)l * r + k;
        Y0[g] = 4.0 * Haa[g];
        Y1[g] = 4.0 * Hab[g];
        Y2[g] = 4.0 * Hbb[g];
        t0[g] = c * (Haa[lk] - Haa[g]);
        t1[g] = c * (Hbb[lk] - Hbb[g]);
        t2[g] = -c * Hab[g];
        t3[g] = c * Hab[lk];
    }
}

struct AdjB {
    int r;
    const double* tau[4];
    const double* X[3];
    const double* M[3];
    const double* gam;
    const double* w;
    const double* Q;
    double* Xb[3];
    double* Mb[3];
    double* X5bd;
    double* X5bf[2];
    double* wb;
    double* Qb;
    double* gb;
};

// Xbar (x1 part):  Xb_aa[ij][kp] = sum_l t0[ij][k][l] ga[p][l];  Xb_bb likewise (t1, gb);
//                  Xb_ab[ij][(a,b)] = sum_l t2[ij][a][l] gb[b][l] - sum_l t3[ij][b][l] ga[a][l].
// Mbar (x2 part):  Mb_aa[ij][l][p] = -2 sum_k t0[ij][k][l] wa[k][p];  Mb_bb likewise (t1, wb);
//                  Mb_ab[ij][u][v] = 2 sum_k t2[ij][k][v] wa[k][u] - 2 sum_k t3[ij][k][u] wb[k][v].
__global__ void k_adj_X_M(const __grid_constant__ AdjB a) {
    const int r = a.r;
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    const double* ga = a.gam;
    const double* gb = a.gam + R2;
    const double* wa = a.w;
    const double* wb = a.w + R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4, ij = g / R2;
        const int u = (int)((g / r) % r), v = (int)(g % r);
        const double* T0 = a.tau[0] + ij * R2;
        const double* T1 = a.tau[1] + ij * R2;
        const double* T2 = a.tau[2] + ij * R2;
        const double* T3 = a.tau[3] + ij * R2;
        double xb = 0.0, mb = 0.0;
        if (blk == 0) {
            for (int l = 0; l < r; ++l) xb += T0[u * r + l] * ga[v * r + l];
            for (int k = 0; k < r; ++k) mb += T0[k * r + u] * wa[k * r + v];
            mb *= -2.0;
        } else if (blk == 2) {
            for (int l = 0; l < r; ++l) xb += T1[u * r + l] * gb[v * r + l];
            for (int k = 0; k < r; ++k) mb += T1[k * r + u] * wb[k * r + v];
            mb *= -2.0;
        } else {
            for (int l = 0; l < r; ++l) xb += T2[u * r + l] * gb[v * r + l] - T3[v * r + l] * ga[u * r + l];
            for (int k = 0; k < r; ++k) mb += 2.0 * T2[k * r + v] * wa[k * r + u] - 2.0 * T3[k * r + u] * wb[k * r + v];
        }
        a.Xb[blk][g] = xb;
        a.Mb[blk][g] = mb;
    }
}

// X5bar, in the forward (row-major) layouts:
//   X5bd(a,a)[(k,j)][(i,l)] = 2 t0[ijkl] - 2 t0[jikl]     X5bd(b,b) likewise with t1
//   X5bd(a,b)[(k,j)][(i,l)] = -2 t2[jikl]                  X5bd(b,a)[(k,j)][(i,l)] = 2 t3[ijkl]
//   X5bf1[(k,j)][(i,l)] = 2 t2[ijkl]                        X5bf2[(k,j)][(i,l)] = -2 t3[jikl]
__global__ void k_adj_X5(const __grid_constant__ AdjB a) {
    const int r = a.r;
    const size_t R2 = (size_t)r * r, n4 = R2 * R2, R22 = 2 * R2;
    FOR_N(e, 6 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4, row = g / R2, col = g % R2;
        const int k = (int)(row / r), j = (int)(row % r), i = (int)(col / r), l = (int)(col % r);
        const size_t ijkl = (((size_t)i * r + j) * r + k) * r + l, jikl = (((size_t)j * r + i) * r + k) * r + l;
        double v;
        switch (blk) {
            case 0: v = 2.0 * (a.tau[0][ijkl] - a.tau[0][jikl]); break;
            case 1: v = -2.0 * a.tau[2][jikl]; break;
            case 2: v = 2.0 * a.tau[3][ijkl]; break;
            case 3: v = 2.0 * (a.tau[1][ijkl] - a.tau[1][jikl]); break;
            case 4: v = 2.0 * a.tau[2][ijkl]; break;
            default: v = -2.0 * a.tau[3][jikl]; break;
        }
        if (blk < 4) {
            const int sK = blk >> 1, sI = blk & 1;
            a.X5bd[(sK * R2 + row) * R22 + sI * R2 + col] = v;
        } else {
            a.X5bf[blk - 4][g] = v;
        }
    }
}

// wbar, Qbar (block per output):
//   wb_a[k][p] = -2 sum_{ij,l} t0[ijkl] Maa[ijlp] + 2 sum t2[ijkl] Mab[ij][p][l]
//   wb_b[k][p] = -2 sum t1[ijkl] Mbb[ijlp] - 2 sum t3[ijkl] Mab[ij][l][p]
//   Qb_a[k][i] = -sum_{jl} t0[ijkl] ga[jl] + sum_{i'l} t0[i' i k l] ga[i'l] - sum_{jl} t2[ijkl] gb[jl]
//   Qb_b[k][i] = -sum t1[ijkl] gb[jl] + sum t1[i' i k l] gb[i'l] + sum t3[i' i k l] ga[i'l]
__global__ void k_adj_wQ(const __grid_constant__ AdjB a) {
    const int r = a.r;
    const size_t R2 = (size_t)r * r;
    const int which = blockIdx.x / (2 * (int)R2);     // 0: w, 1: Q
    const int t = blockIdx.x % (2 * (int)R2);
    const int sp = t / (int)R2, k = (t / r) % r, q = t % r;   // q = p (w) or i (Q)
    const double* ga = a.gam;
    const double* gb = a.gam + R2;
    double acc = 0.0;
    if (which == 0) {
        const size_t n = R2 * r;   // (ij, l)
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            const size_t ij = e / r;
            const int l = (int)(e % r);
            const size_t kl = ij * R2 + (size_t)k * r + l;
            if (sp == 0)
                acc += -2.0 * a.tau[0][kl] * a.M[0][ij * R2 + (size_t)l * r + q] +
                       2.0 * a.tau[2][kl] * a.M[1][ij * R2 + (size_t)q * r + l];
            else
                acc += -2.0 * a.tau[1][kl] * a.M[2][ij * R2 + (size_t)l * r + q] -
                       2.0 * a.tau[3][kl] * a.M[1][ij * R2 + (size_t)l * r + q];
        }
    } else {
        const int i = q;
        for (size_t e = threadIdx.x; e < R2; e += blockDim.x) {
            const int jj = (int)(e / r), l = (int)(e % r);
            const size_t ijkl = (((size_t)i * r + jj) * r + k) * r + l;      // j = jj
            const size_t jikl = (((size_t)jj * r + i) * r + k) * r + l;      // i' = jj
            if (sp == 0)
                acc += -a.tau[0][ijkl] * ga[jj * r + l] + a.tau[0][jikl] * ga[jj * r + l] - a.tau[2][ijkl] * gb[jj * r + l];
            else
                acc += -a.tau[1][ijkl] * gb[jj * r + l] + a.tau[1][jikl] * gb[jj * r + l] + a.tau[3][jikl] * ga[jj * r + l];
        }
    }
    acc = ad_block_sum(acc);
    if (threadIdx.x == 0) (which == 0 ? a.wb : a.Qb)[t] = acc;
}

// gbar from x1, x4, x7 (block per output (sp, a, b)):
//   gb_a[p][l] += sum_{ij,k} t0[ijkl] Xaa[ij][kp] - sum t3[ijkl] Xab[ij][pk]
//               - sum_{ik} t0[i p k l] Qa[k][i] + sum_{jk} t0[p j k l] Qa[k][j] + sum_{jk} t3[p j k l] Qb[k][j]
//   gb_b[p][l] += sum t1[ijkl] Xbb[ij][kp] + sum t2[ijkl] Xab[ij][kp]
//               - sum t1[i p k l] Qb[k][i] + sum t1[p j k l] Qb[k][j] - sum t2[i p k l] Qa[k][i]
__global__ void k_adj_gamma_x(const __grid_constant__ AdjB a) {
    const int r = a.r;
    const size_t R2 = (size_t)r * r;
    const int t = blockIdx.x;
    const int sp = t / (int)R2, pp = (t / r) % r, l = t % r;
    const double* Qa = a.Q;
    const double* Qb = a.Q + R2;
    double acc = 0.0;
    for (size_t e = threadIdx.x; e < R2 * r; e += blockDim.x) {   // (ij, k)
        const size_t ij = e / r;
        const int k = (int)(e % r);
        const size_t kl = ij * R2 + (size_t)k * r + l;
        if (sp == 0)
            acc += a.tau[0][kl] * a.X[0][ij * R2 + (size_t)k * r + pp] - a.tau[3][kl] * a.X[1][ij * R2 + (size_t)pp * r + k];
        else
            acc += a.tau[1][kl] * a.X[2][ij * R2 + (size_t)k * r + pp] + a.tau[2][kl] * a.X[1][ij * R2 + (size_t)k * r + pp];
    }
    for (size_t e = threadIdx.x; e < R2; e += blockDim.x) {   // (x, k): x = i or j
        const int x = (int)(e / r), k = (int)(e % r);
        const size_t xpkl = (((size_t)x * r + pp) * r + k) * r + l;   // t[x p k l]
        const size_t pxkl = (((size_t)pp * r + x) * r + k) * r + l;   // t[p x k l]
        if (sp == 0)
            acc += -a.tau[0][xpkl] * Qa[k * r + x] + a.tau[0][pxkl] * Qa[k * r + x] + a.tau[3][pxkl] * Qb[k * r + x];
        else
            acc += -a.tau[1][xpkl] * Qb[k * r + x] + a.tau[1][pxkl] * Qb[k * r + x] - a.tau[2][xpkl] * Qa[k * r + x];
    }
    acc = ad_block_sum(acc);
    if (threadIdx.x == 0) a.gb[t] = acc;   // first contribution: overwrite
}

// Qbar -> Xbar:  Xb_aa[(i,p)][(k,p)] += Qb_a[k][i];  Xb_ab[(i,p)][(k,p)] += Qb_a[k][i];
//                Xb_bb[(i,p)][(k,p)] += Qb_b[k][i];  Xb_ab[(p,i)][(p,k)] += Qb_b[k][i].
__global__ void k_adj_Q_to_X(int r, const double* __restrict__ Qb, double* Xaa, double* Xab, double* Xbb) {
    const size_t R2 = (size_t)r * r;
    FOR_N(e, R2 * r) {
        const int k = (int)(e / R2), i = (int)((e / r) % r), p = (int)(e % r);
        const double qa = Qb[k * r + i], qb = Qb[R2 + k * r + i];
        Xaa[((size_t)i * r + p) * R2 + (size_t)k * r + p] += qa;
        Xbb[((size_t)i * r + p) * R2 + (size_t)k * r + p] += qb;
        // the two ab updates touch different elements unless (i,p) = (p,i) and (k,p) = (p,k): serialise them
        Xab[((size_t)i * r + p) * R2 + (size_t)k * r + p] += qa;
    }
}

__global__ void k_adj_Q_to_X_ab2(int r, const double* __restrict__ Qb, double* Xab) {
    const size_t R2 = (size_t)r * r;
    FOR_N(e, R2 * r) {
        const int k = (int)(e / R2), i = (int)((e / r) % r), p = (int)(e % r);
        Xab[((size_t)p * r + i) * R2 + (size_t)p * r + k] += Qb[R2 + k * r + i];
    }
}

// wbar -> Zbar diagonals: Zb_d(a,a)[(k,p)][(p,s)] += wb_a[k][s], Zb_f1[(k,p)][(p,s)] -= wb_a[k][s],
//                         Zb_d(b,b)[(k,p)][(p,s)] += wb_b[k][s], Zb_f2[(k,p)][(p,s)] -= wb_b[k][s].
__global__ void k_adj_w_to_Z(int r, const double* __restrict__ wb, double* Zbd, double* Zbf1, double* Zbf2) {
    const size_t R2 = (size_t)r * r, R22 = 2 * R2;
    FOR_N(e, 2 * R2 * r) {
        const int sp = (int)(e / (R2 * r)), k = (int)((e / R2) % r), p = (int)((e / r) % r), s = (int)(e % r);
        const double v = wb[sp * R2 + k * r + s];
        const size_t rowL = (size_t)k * r + p, colL = (size_t)p * r + s;
        Zbd[(sp * R2 + rowL) * R22 + sp * R2 + colL] += v;
        (sp == 0 ? Zbf1 : Zbf2)[rowL * R2 + colL] -= v;
    }
}

// Zbar -> gbar: for each Z type t, gbar[j][q] += sum_{(k,p),s} Zb_t[(k,j)][(p,s)] W_kp^t[q][s] with the
// W maps of the Z kernel (block per (t, j, q); outputs summed into gbar by a fixed-order kernel).
struct AdjZ {
    int r;
    const double* Waa;
    const double* Wab;
    const double* Wbb;
    const double* Zbd;
    const double* Zbf[2];
    double* part;   // [6][r][r]
};

__global__ void k_adj_Z_gamma(const __grid_constant__ AdjZ a) {
    const int r = a.r;
    const size_t R2 = (size_t)r * r, r3 = R2 * r, R22 = 2 * R2;
    const int t = blockIdx.x / (int)R2, jq = blockIdx.x % (int)R2, j = jq / r, q = jq % r;
    double acc = 0.0;
    for (size_t e = threadIdx.x; e < R2 * r; e += blockDim.x) {   // (k, p, s)
        const int k = (int)(e / R2), p = (int)((e / r) % r), s = (int)(e % r);
        double zb, w;
        switch (t) {
            case 0: zb = a.Zbd[((size_t)k * r + j) * R22 + (size_t)p * r + s]; w = a.Waa[k * r3 + p * R2 + (size_t)q * r + s]; break;
            case 1: zb = a.Zbd[((size_t)k * r + j) * R22 + R2 + (size_t)p * r + s]; w = a.Wab[k * r3 + p * R2 + (size_t)q * r + s]; break;
            case 2: zb = a.Zbd[(R2 + (size_t)k * r + j) * R22 + (size_t)p * r + s]; w = a.Wab[p * r3 + k * R2 + (size_t)s * r + q]; break;
            case 3: zb = a.Zbd[(R2 + (size_t)k * r + j) * R22 + R2 + (size_t)p * r + s]; w = a.Wbb[k * r3 + p * R2 + (size_t)q * r + s]; break;
            case 4: zb = a.Zbf[0][((size_t)k * r + j) * R2 + (size_t)p * r + s]; w = a.Wab[k * r3 + p * R2 + (size_t)s * r + q]; break;
            default: zb = a.Zbf[1][((size_t)k * r + j) * R2 + (size_t)p * r + s]; w = a.Wab[p * r3 + k * R2 + (size_t)q * r + s]; break;
        }
        acc += zb * w;
    }
    acc = ad_block_sum(acc);
    if (threadIdx.x == 0) a.part[blockIdx.x] = acc;
}

// gbar_a += part0 + part1 + part5, gbar_b += part2 + part3 + part4 (spin of the 1D in each Z type).
__global__ void k_adj_Z_gamma_sum(int r, const double* __restrict__ part, double* gb) {
    const int R2 = r * r;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R2) return;
    gb[e] += part[0 * R2 + e] + part[1 * R2 + e] + part[5 * R2 + e];
    gb[R2 + e] += part[2 * R2 + e] + part[3 * R2 + e] + part[4 * R2 + e];
}

// particle-hole Mbar (forward layouts) -> Mbar blocks:
//   Mb_aa[i][p][l][s] += Mbd(a,a)[(i,l)][(p,s)]   Mb_ab[i][p][l][s] += Mbd(a,b)[(i,l)][(p,s)]
//   Mb_ab[p][i][s][l] += Mbd(b,a)[(i,l)][(p,s)]   Mb_bb[i][p][l][s] += Mbd(b,b)[(i,l)][(p,s)]
//   Mb_ab[i][p][s][l] += Mbf1[(i,l)][(p,s)]        Mb_ab[p][i][l][s] += Mbf2[(i,l)][(p,s)]
// gathered per Mbar element (no write conflicts).
__global__ void k_adj_Mph_to_M(int r, const double* __restrict__ Mbd, const double* __restrict__ Mbf1,
                               const double* __restrict__ Mbf2, double* Maa, double* Mab, double* Mbb) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2, R22 = 2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4;
        const int a0 = (int)(g / (R2 * r)), a1 = (int)((g / R2) % r), a2 = (int)((g / r) % r), a3 = (int)(g % r);
        if (blk == 0) {   // Maa[i=a0][p=a1][l=a2][s=a3]
            Maa[g] += Mbd[((size_t)a0 * r + a2) * R22 + (size_t)a1 * r + a3];
        } else if (blk == 2) {
            Mbb[g] += Mbd[(R2 + (size_t)a0 * r + a2) * R22 + R2 + (size_t)a1 * r + a3];
        } else {
            // Mab[a0][a1][a2][a3] from: (a,b) i=a0 p=a1 l=a2 s=a3;  (b,a) p=a0 i=a1 s=a2 l=a3;
            //                            f1 i=a0 p=a1 s=a2 l=a3;     f2 p=a0 i=a1 l=a2 s=a3
            double v = Mbd[((size_t)a0 * r + a2) * R22 + R2 + (size_t)a1 * r + a3];
            v += Mbd[(R2 + (size_t)a1 * r + a3) * R22 + (size_t)a0 * r + a2];
            v += Mbf1[((size_t)a0 * r + a3) * R2 + (size_t)a1 * r + a2];
            v += Mbf2[((size_t)a1 * r + a2) * R2 + (size_t)a0 * r + a3];
            Mab[g] += v;
        }
    }
}

// Mbar -> gbar through M = 3D - 2(1D^1D) (block per (sp, a, b)):
//   gb_a[a][b] += -sum_{jl} Mb_aa[a j b l] ga[jl] - sum_{ik} Mb_aa[i a k b] ga[ik] + sum_{il} Mb_aa[i a b l] ga[il]
//                + sum_{jk} Mb_aa[a j k b] ga[jk] - sum_{jl} Mb_ab[a j b l] gb[jl]
//   gb_b[a][b] += (the same with Mb_bb, gb) - sum_{ik} Mb_ab[i a k b] ga[ik]
__global__ void k_adj_M_gamma(int r, const double* __restrict__ Maa, const double* __restrict__ Mab,
                              const double* __restrict__ Mbb, const double* __restrict__ gam, double* gb) {
    const size_t R2 = (size_t)r * r;
    const int t = blockIdx.x;
    const int sp = t / (int)R2, a = (t / r) % r, b = t % r;
    const double* g = gam + (sp == 0 ? 0 : R2);
    const double* go = gam + (sp == 0 ? R2 : 0);
    const double* Ms = sp == 0 ? Maa : Mbb;
    double acc = 0.0;
    for (size_t e = threadIdx.x; e < R2; e += blockDim.x) {
        const int x = (int)(e / r), y = (int)(e % r);
        acc += -Ms[(((size_t)a * r + x) * r + b) * r + y] * g[x * r + y]     // (j,l) = (x,y)
               - Ms[(((size_t)x * r + a) * r + y) * r + b] * g[x * r + y]    // (i,k) = (x,y)
               + Ms[(((size_t)x * r + a) * r + b) * r + y] * g[x * r + y]    // (i,l) = (x,y)
               + Ms[(((size_t)a * r + x) * r + y) * r + b] * g[x * r + y];   // (j,k) = (x,y)
        if (sp == 0) acc -= Mab[(((size_t)a * r + x) * r + b) * r + y] * go[x * r + y];
        else acc -= Mab[(((size_t)x * r + a) * r + y) * r + b] * go[x * r + y];
    }
    acc = ad_block_sum(acc);
    if (threadIdx.x == 0) gb[t] += acc;
}

// D accumulation: Db += 3 Mb, and the 1D adjoint: Db_aa[p][q][r'][q] += c gb_a[p][r'],
// Db_ab[p][q][r'][q] += c gb_a[p][r'], Db_bb[p][q][r'][q] += c gb_b[p][r'], Db_ab[q][p][q][r'] += c gb_b[p][r'].
__global__ void k_adj_to_D(int r, double cN, const double* __restrict__ Maa, const double* __restrict__ Mab,
                           const double* __restrict__ Mbb, const double* __restrict__ gb, double* Daa, double* Dab,
                           double* Dbb) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4;
        const int a0 = (int)(g / (R2 * r)), a1 = (int)((g / R2) % r), a2 = (int)((g / r) % r), a3 = (int)(g % r);
        if (blk == 0) {
            Daa[g] += 3.0 * Maa[g] + (a1 == a3 ? cN * gb[a0 * r + a2] : 0.0);
        } else if (blk == 2) {
            Dbb[g] += 3.0 * Mbb[g] + (a1 == a3 ? cN * gb[R2 + a0 * r + a2] : 0.0);
        } else {
            double v = 3.0 * Mab[g];
            if (a1 == a3) v += cN * gb[a0 * r + a2];          // gamma_a part
            if (a0 == a2) v += cN * gb[R2 + a1 * r + a3];     // gamma_b part: Dab[q][p][q][r']
            Dab[g] += v;
        }
    }
}

// ----------------------------------------------------------------------- K -> (h, V)
// Kb: cotangent of the FULL K blocks.  Vb[abcd] = 1/2 (Kaa+Kbb+Kab)[a c b d] - 1/2 (Kaa+Kbb)[a c d b];
// hb[a][b] = (sum_j (Kaa+Kbb+Kab)[a j b j] + sum_i (Kaa+Kbb+Kab)[i a i b]
//             - sum_j (Kaa+Kbb)[a j j b] - sum_i (Kaa+Kbb)[i a b i]) / (2(N-1)).
// Then symmetrised: h over p<->q, V over the 8-fold permutational symmetry.
__global__ void k_adj_K_to_V(int r, const double* __restrict__ Kaa, const double* __restrict__ Kab,
                             const double* __restrict__ Kbb, double* Vraw) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(g, n4) {
        const int a = (int)(g / (R2 * r)), b = (int)((g / R2) % r), c = (int)((g / r) % r), d = (int)(g % r);
        const size_t acbd = (((size_t)a * r + c) * r + b) * r + d, acdb = (((size_t)a * r + c) * r + d) * r + b;
        Vraw[g] = 0.5 * (Kaa[acbd] + Kbb[acbd] + Kab[acbd]) - 0.5 * (Kaa[acdb] + Kbb[acdb]);
    }
}

__global__ void k_sym_V(int r, const double* __restrict__ Vr, double* dV) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(g, n4) {
        const int p = (int)(g / (R2 * r)), q = (int)((g / R2) % r), s1 = (int)((g / r) % r), s2 = (int)(g % r);
#define VI(a, b, c, d) Vr[(((size_t)(a) * r + (b)) * r + (c)) * r + (d)]
        dV[g] = 0.125 * (VI(p, q, s1, s2) + VI(q, p, s1, s2) + VI(p, q, s2, s1) + VI(q, p, s2, s1) + VI(s1, s2, p, q) +
                         VI(s2, s1, p, q) + VI(s1, s2, q, p) + VI(s2, s1, q, p));
#undef VI
    }
}

__global__ void k_adj_K_to_h(int r, double inv2N1, const double* __restrict__ Kaa, const double* __restrict__ Kab,
                             const double* __restrict__ Kbb, double* hraw) {
    const int t = blockIdx.x;
    const int a = t / r, b = t % r;
    double acc = 0.0;
    for (int x = threadIdx.x; x < r; x += blockDim.x) {
        const size_t axbx = (((size_t)a * r + x) * r + b) * r + x, xaxb = (((size_t)x * r + a) * r + x) * r + b;
        const size_t axxb = (((size_t)a * r + x) * r + x) * r + b, xabx = (((size_t)x * r + a) * r + b) * r + x;
        acc += Kaa[axbx] + Kbb[axbx] + Kab[axbx] + Kaa[xaxb] + Kbb[xaxb] + Kab[xaxb] - Kaa[axxb] - Kbb[axxb] -
               Kaa[xabx] - Kbb[xabx];
    }
    acc = ad_block_sum(acc);
    if (threadIdx.x == 0) hraw[t] = acc * inv2N1;
}

__global__ void k_sym_h(int r, const double* __restrict__ hr, double* dh) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r * r) return;
    const int a = e / r, b = e % r;
    dh[e] = 0.5 * (hr[a * r + b] + hr[b * r + a]);
}

// dD projection onto 2-RDM symmetries: aa, bb antisymmetric within pairs and pair-Hermitian;
// ab pair-Hermitian.
__global__ void k_project_D(int r, const double* __restrict__ i0, const double* __restrict__ i1,
                            const double* __restrict__ i2, double* o0, double* o1, double* o2) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    FOR_N(e, 3 * n4) {
        const int blk = (int)(e / n4);
        const size_t g = e % n4;
        const int i = (int)(g / (R2 * r)), j = (int)((g / R2) % r), k = (int)((g / r) % r), l = (int)(g % r);
        const size_t ij = (size_t)i * r + j, ji = (size_t)j * r + i, kl = (size_t)k * r + l, lk = (size_t)l * r + k;
        if (blk == 1) {
            o1[g] = 0.5 * (i1[ij * R2 + kl] + i1[kl * R2 + ij]);
        } else {
            const double* x = blk == 0 ? i0 : i2;
            const double A = 0.25 * (x[ij * R2 + kl] - x[ji * R2 + kl] - x[ij * R2 + lk] + x[ji * R2 + lk]);
            const double At = 0.25 * (x[kl * R2 + ij] - x[lk * R2 + ij] - x[kl * R2 + ji] + x[lk * R2 + ji]);
            (blk == 0 ? o0 : o2)[g] = 0.5 * (A + At);
        }
    }
}

// ------------------------------------------------------------------------------ workspace
struct AdjWork {
    double* Hb[3];
    double* Yb[3];
    double* tau[4];
    double* Xb[3];
    double* X5bd;
    double* X5bf[2];
    double* Zbd;
    double* Zbf[2];
    double* Mbd;
    double* Mbf[2];
    double* Mb[3];
    double* wb;
    double* Qb;
    double* gb;
    double* zpart;
    double* Gh[3];     // spin-orbital normalised cotangent
    double* Gp[3];     // its pair-Hermitian / anti-Hermitian part
    double* Wb[3];     // dL/dW
    double* Db[3];     // running dL/dD_k
    double* Dn[3];     // next dL/dD
    double* Kb[3];     // dL/dK (full K)
    double* Dk[3];     // D_k (recomputed)
    double* Araw[3];
    double* Am[3];
    double* Ab[3];
    double* hraw;
    double* Vraw;
};

static int adj_alloc(acse_ctx* c) {
    if (c->adj) return ACSE_OK;
    AdjWork* a = (AdjWork*)calloc(1, sizeof(AdjWork));
    if (!a) return ACSE_ERR_NOMEM;
    c->adj = a;
    const size_t r = c->r, R2 = r * r, n4 = R2 * R2, b4 = n4 * sizeof(double);
    double** ptrs[] = {&a->Hb[0], &a->Hb[1], &a->Hb[2], &a->Yb[0], &a->Yb[1], &a->Yb[2], &a->tau[0], &a->tau[1],
                       &a->tau[2], &a->tau[3], &a->Xb[0], &a->Xb[1], &a->Xb[2], &a->X5bf[0], &a->X5bf[1], &a->Zbf[0],
                       &a->Zbf[1], &a->Mbf[0], &a->Mbf[1], &a->Mb[0], &a->Mb[1], &a->Mb[2], &a->Gh[0], &a->Gh[1],
                       &a->Gh[2], &a->Gp[0], &a->Gp[1], &a->Gp[2], &a->Wb[0], &a->Wb[1], &a->Wb[2], &a->Db[0],
                       &a->Db[1], &a->Db[2], &a->Dn[0], &a->Dn[1], &a->Dn[2], &a->Kb[0], &a->Kb[1], &a->Kb[2],
                       &a->Dk[0], &a->Dk[1], &a->Dk[2], &a->Araw[0], &a->Araw[1], &a->Araw[2], &a->Am[0], &a->Am[1],
                       &a->Am[2], &a->Ab[0], &a->Ab[1], &a->Ab[2], &a->Vraw};
    for (double** p : ptrs)
        if (cudaMalloc((void**)p, b4) != cudaSuccess) { cudaGetLastError(); return ACSE_ERR_NOMEM; }
    if (cudaMalloc((void**)&a->X5bd, 4 * b4) != cudaSuccess || cudaMalloc((void**)&a->Zbd, 4 * b4) != cudaSuccess ||
        cudaMalloc((void**)&a->Mbd, 4 * b4) != cudaSuccess || cudaMalloc((void**)&a->wb, 2 * R2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&a->Qb, 2 * R2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&a->gb, 2 * R2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&a->zpart, 6 * R2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&a->hraw, R2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    return ACSE_OK;
}

void adj_free(acse_ctx* c) {
    AdjWork* a = (AdjWork*)c->adj;
    if (!a) return;
    double* ptrs[] = {a->Hb[0], a->Hb[1], a->Hb[2], a->Yb[0], a->Yb[1], a->Yb[2], a->tau[0], a->tau[1], a->tau[2],
                      a->tau[3], a->Xb[0], a->Xb[1], a->Xb[2], a->X5bd, a->X5bf[0], a->X5bf[1], a->Zbd, a->Zbf[0],
                      a->Zbf[1], a->Mbd, a->Mbf[0], a->Mbf[1], a->Mb[0], a->Mb[1], a->Mb[2], a->wb, a->Qb, a->gb,
                      a->zpart, a->Gh[0], a->Gh[1], a->Gh[2], a->Gp[0], a->Gp[1], a->Gp[2], a->Wb[0], a->Wb[1],
                      a->Wb[2], a->Db[0], a->Db[1], a->Db[2], a->Dn[0], a->Dn[1], a->Dn[2], a->Kb[0], a->Kb[1],
                      a->Kb[2], a->Dk[0], a->Dk[1], a->Dk[2], a->Araw[0], a->Araw[1], a->Araw[2], a->Am[0],
                      a->Am[1], a->Am[2], a->Ab[0], a->Ab[1], a->Ab[2], a->hraw, a->Vraw};
    for (double* p : ptrs)
        if (p) cudaFree(p);
    free(a);
    c->adj = nullptr;
}

#define AL(c) ACSE_LAUNCHED(c)

// -------------------------------------------------------------------------- VJP w.r.t. D
// Requires the forward intermediates of G(W; D) (acse_contract just called with this W and D).
// Adds dL/dD to Dacc for L = <Gb, scale (H - s H^T)>.
static int vjp_D(acse_ctx* c, const double* const W[3], int sW, double scale, const double* const Gb[3],
                 double* const Dacc[3]) {
    AdjWork* a = (AdjWork*)c->adj;
    Work& w = c->w;
    const int r = c->r, R2 = r * r, R22 = 2 * R2;
    const size_t n4 = (size_t)R2 * R2;
    // assembly: Hb = scale (Gb - s Gb^T)
    k_pair_combine<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, Gb[0], Gb[1], Gb[2], scale, -scale * sW, a->Hb[0],
                                                            a->Hb[1], a->Hb[2]);
    AL(c);
    k_adj_tau<<<ad_grid(n4), AD_TPB, 0, c->stream>>>(r, a->Hb[0], a->Hb[1], a->Hb[2], a->Yb[0], a->Yb[1], a->Yb[2],
                                                     a->tau[0], a->tau[1], a->tau[2], a->tau[3]);
    AL(c);
    AdjB ab;
    ab.r = r;
    for (int t = 0; t < 4; ++t) ab.tau[t] = a->tau[t];
    for (int s = 0; s < 3; ++s) { ab.X[s] = w.X[s]; ab.M[s] = w.M[s]; ab.Xb[s] = a->Xb[s]; ab.Mb[s] = a->Mb[s]; }
    ab.gam = w.gam; ab.w = w.w; ab.Q = w.Q;
    ab.X5bd = a->X5bd; ab.X5bf[0] = a->X5bf[0]; ab.X5bf[1] = a->X5bf[1];
    ab.wb = a->wb; ab.Qb = a->Qb; ab.gb = a->gb;
    k_adj_X_M<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(ab);
    AL(c);
    k_adj_X5<<<ad_grid(6 * n4), AD_TPB, 0, c->stream>>>(ab);
    AL(c);
    k_adj_wQ<<<4 * R2, AD_TPB, 0, c->stream>>>(ab);
    AL(c);
    k_adj_gamma_x<<<2 * R2, AD_TPB, 0, c->stream>>>(ab);
    AL(c);
    k_adj_Q_to_X<<<ad_grid((size_t)R2 * r), AD_TPB, 0, c->stream>>>(r, a->Qb, a->Xb[0], a->Xb[1], a->Xb[2]);
    AL(c);
    k_adj_Q_to_X_ab2<<<ad_grid((size_t)R2 * r), AD_TPB, 0, c->stream>>>(r, a->Qb, a->Xb[1]);
    AL(c);
    // particle-hole GEMMs reversed: Zb = X5b . Mph (B stored [K][N]); Mphb = X5b^T . Z (both transposed)
    GemmF64 g[6];
    int n = 0;
    g[n++] = GemmF64{a->X5bd, w.Md, a->Zbd, R22, R22, R22, R22, R22, R22, 1.0, 0.0, 0, 0, 1};
    g[n++] = GemmF64{a->X5bf[0], w.Mf1, a->Zbf[0], R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 0, 1};
    g[n++] = GemmF64{a->X5bf[1], w.Mf2, a->Zbf[1], R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 0, 1};
    g[n++] = GemmF64{a->X5bd, w.Zd, a->Mbd, R22, R22, R22, R22, R22, R22, 1.0, 0.0, 0, 1, 1};
    g[n++] = GemmF64{a->X5bf[0], w.Zf1, a->Mbf[0], R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 1, 1};
    g[n++] = GemmF64{a->X5bf[1], w.Zf2, a->Mbf[1], R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 1, 1};
    ACSE_TRY(c->oz ? oz_gemm_list(c, g, n, 0) : gemm_f64_grouped(c, g, n, c->stream));
    // w routes into the diagonals of Z; then Zb -> gbar
    k_adj_w_to_Z<<<ad_grid(2 * (size_t)R2 * r), AD_TPB, 0, c->stream>>>(r, a->wb, a->Zbd, a->Zbf[0], a->Zbf[1]);
    AL(c);
    AdjZ az;
    az.r = r; az.Waa = W[0]; az.Wab = W[1]; az.Wbb = W[2];
    az.Zbd = a->Zbd; az.Zbf[0] = a->Zbf[0]; az.Zbf[1] = a->Zbf[1]; az.part = a->zpart;
    k_adj_Z_gamma<<<6 * R2, AD_TPB, 0, c->stream>>>(az);
    AL(c);
    k_adj_Z_gamma_sum<<<(R2 + 127) / 128, 128, 0, c->stream>>>(r, a->zpart, a->gb);
    AL(c);
    // Mbar: x2 part (already in Mb) + particle-hole relayout + pair GEMM f Xb W; Db += f Yb W
    k_adj_Mph_to_M<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Mbd, a->Mbf[0], a->Mbf[1], a->Mb[0], a->Mb[1],
                                                             a->Mb[2]);
    AL(c);
    n = 0;
    for (int s = 0; s < 3; ++s) {
        const double f = s == 1 ? 2.0 : 1.0;
        g[n++] = GemmF64{a->Xb[s], W[s], a->Mb[s], R2, R2, R2, R2, R2, R2, f, 1.0, 0, 0, 1};
        g[n++] = GemmF64{a->Yb[s], W[s], Dacc[s], R2, R2, R2, R2, R2, R2, f, 1.0, 0, 0, 1};
    }
    ACSE_TRY(c->oz ? oz_gemm_list(c, g, n, 1) : gemm_f64_grouped(c, g, n, c->stream));
    k_adj_M_gamma<<<2 * R2, AD_TPB, 0, c->stream>>>(r, a->Mb[0], a->Mb[1], a->Mb[2], w.gam, a->gb);
    AL(c);
    k_adj_to_D<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, 2.0 / (c->N - 1), a->Mb[0], a->Mb[1], a->Mb[2], a->gb,
                                                         Dacc[0], Dacc[1], Dacc[2]);
    AL(c);
    return ACSE_OK;
}

// -------------------------------------------------------------------------- VJP w.r.t. W
// Wb = dL/dW for L = <Gb, G(W; D)> (scale 1), using beta(X, Y) = -beta(Y, X); the 1D and M of D
// must be current (prep_D done).  Overwrites the pass intermediates.
static int vjp_W(acse_ctx* c, const double* const D[3], const double* const Gb[3], double* const Wb[3]) {
    AdjWork* a = (AdjWork*)c->adj;
    const int r = c->r;
    const size_t n4 = (size_t)r * r * r * r;
    k_to_so_cotangent<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, Gb[0], Gb[1], Gb[2], 1.0, a->Gh[0], a->Gh[1],
                                                                a->Gh[2]);
    AL(c);
    // pair-Hermitian part (s = +1) and anti-Hermitian part (s = -1), G(.) accumulated into Wb with
    // block factors -1, -4, -1
    for (int part = 0; part < 2; ++part) {
        const double sgn = part == 0 ? 1.0 : -1.0;
        k_pair_combine<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Gh[0], a->Gh[1], a->Gh[2], 0.5, 0.5 * sgn,
                                                                a->Gp[0], a->Gp[1], a->Gp[2]);
        AL(c);
        const double* Wp[3] = {a->Gp[0], a->Gp[1], a->Gp[2]};
        double* out[3] = {a->Ab[0], a->Ab[1], a->Ab[2]};
        ACSE_TRY(acse_contract(c, D, Wp, part == 0 ? +1 : -1, 1.0, 0, out, nullptr, 0));
        if (part == 0) {
            ACSE_CUDA_TRY(cudaMemsetAsync(Wb[0], 0, n4 * sizeof(double), c->stream));
            ACSE_CUDA_TRY(cudaMemsetAsync(Wb[1], 0, n4 * sizeof(double), c->stream));
            ACSE_CUDA_TRY(cudaMemsetAsync(Wb[2], 0, n4 * sizeof(double), c->stream));
        }
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Ab[0], a->Ab[1], a->Ab[2], -1.0, -4.0, -1.0, Wb[0],
                                                          Wb[1], Wb[2]);
        AL(c);
    }
    return ACSE_OK;
}

// ---------------------------------------------------------------------------- trajectory
extern "C" int acse_residual_backward_impl(acse_ctx* c, const double* const* D_ckpt, int n_steps, double eps,
                                            double wE, double wN, double* dh, double* dV, double* dDaa,
                                            double* dDab, double* dDbb) {
    if (c->opt.prec != ACSE_FP64) return ACSE_ERR_UNSUPPORTED;
    if (!D_ckpt || n_steps < 0 || !D_ckpt[0] || !D_ckpt[1] || !D_ckpt[2]) return ACSE_ERR_ARG;
    ACSE_TRY(adj_alloc(c));
    AdjWork* a = (AdjWork*)c->adj;
    Work& w = c->w;
    const int r = c->r;
    const size_t n4 = (size_t)r * r * r * r, b4 = n4 * sizeof(double);
    const double* Kh[3] = {w.Kh[0], w.Kh[1], w.Kh[2]};
    const int mask = c->opt.mask_active;
    // D_k for k = 0..n: checkpoint if given, else recomputed from D_{k-1} (stored in a->Dk per use)
    auto load_D = [&](int k) -> int {
        // recompute forward from the latest available checkpoint at or below k
        int k0 = k;
        while (k0 > 0 && !(D_ckpt[3 * k0] && D_ckpt[3 * k0 + 1] && D_ckpt[3 * k0 + 2])) --k0;
        for (int b = 0; b < 3; ++b)
            ACSE_CUDA_TRY(cudaMemcpyAsync(a->Dk[b], D_ckpt[3 * k0 + b], b4, cudaMemcpyDefault, c->stream));
        const double* Dc[3] = {a->Dk[0], a->Dk[1], a->Dk[2]};
        for (int kk = k0; kk < k; ++kk) {
            double* Ar[3] = {a->Araw[0], a->Araw[1], a->Araw[2]};
            ACSE_TRY(acse_contract(c, Dc, Kh, +1, 1.0, 0, Ar, nullptr, 1));
            k_mask_copy<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Araw[0], a->Araw[1], a->Araw[2], mask,
                                                                  c->opt.act_lo, c->opt.act_hi, a->Am[0], a->Am[1],
                                                                  a->Am[2]);
            AL(c);
            const double* Amc[3] = {a->Am[0], a->Am[1], a->Am[2]};
            double* Uo[3] = {a->Ab[0], a->Ab[1], a->Ab[2]};
            ACSE_TRY(acse_contract(c, Dc, Amc, -1, 0.5, 0, Uo, nullptr, 0));
            k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Ab[0], a->Ab[1], a->Ab[2], eps, eps, eps,
                                                              a->Dk[0], a->Dk[1], a->Dk[2]);
            AL(c);
        }
        return ACSE_OK;
    };
    const double* Dc[3] = {a->Dk[0], a->Dk[1], a->Dk[2]};
    for (int b = 0; b < 3; ++b) {
        ACSE_CUDA_TRY(cudaMemsetAsync(a->Db[b], 0, b4, c->stream));
        ACSE_CUDA_TRY(cudaMemsetAsync(a->Kb[b], 0, b4, c->stream));
    }
    // ---- terminal: E = sum_b m_b K_b D_b (m = 1, 4, 1), K = 2 Kh
    ACSE_TRY(load_D(n_steps));
    if (wE != 0.0) {
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, w.Kh[0], w.Kh[1], w.Kh[2], 2.0 * wE, 8.0 * wE,
                                                          2.0 * wE, a->Db[0], a->Db[1], a->Db[2]);
        AL(c);
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Dk[0], a->Dk[1], a->Dk[2], wE, 4.0 * wE, wE,
                                                          a->Kb[0], a->Kb[1], a->Kb[2]);
        AL(c);
    }
    if (wN != 0.0) {
        // ||A||^2 = sum_b m_b ||A_b||^2 (before the mask): Ab = 2 wN m_b A_b
        double* Ar[3] = {a->Araw[0], a->Araw[1], a->Araw[2]};
        ACSE_TRY(acse_contract(c, Dc, Kh, +1, 1.0, 0, Ar, nullptr, 1));
        for (int b = 0; b < 3; ++b) ACSE_CUDA_TRY(cudaMemsetAsync(a->Am[b], 0, b4, c->stream));
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Araw[0], a->Araw[1], a->Araw[2], 2.0 * wN,
                                                          8.0 * wN, 2.0 * wN, a->Am[0], a->Am[1], a->Am[2]);
        AL(c);
        const double* Gb[3] = {a->Am[0], a->Am[1], a->Am[2]};
        ACSE_TRY(vjp_D(c, Kh, +1, 1.0, Gb, a->Db));
        ACSE_TRY(vjp_W(c, Dc, Gb, a->Wb));
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Wb[0], a->Wb[1], a->Wb[2], 0.5, 0.5, 0.5,
                                                          a->Kb[0], a->Kb[1], a->Kb[2]);
        AL(c);
    }
    // ---- reverse sweep over the steps
    for (int k = n_steps - 1; k >= 0; --k) {
        ACSE_TRY(load_D(k));
        // Dn = Db (identity part of D_{k+1} = D_k + eps U)
        for (int b = 0; b < 3; ++b)
            ACSE_CUDA_TRY(cudaMemcpyAsync(a->Dn[b], a->Db[b], b4, cudaMemcpyDeviceToDevice, c->stream));
        // forward at D_k: A_raw, Am = mask(A_raw), then the update pass (populates its intermediates)
        double* Ar[3] = {a->Araw[0], a->Araw[1], a->Araw[2]};
        ACSE_TRY(acse_contract(c, Dc, Kh, +1, 1.0, 0, Ar, nullptr, 1));
        k_mask_copy<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Araw[0], a->Araw[1], a->Araw[2], mask,
                                                              c->opt.act_lo, c->opt.act_hi, a->Am[0], a->Am[1],
                                                              a->Am[2]);
        AL(c);
        const double* Amc[3] = {a->Am[0], a->Am[1], a->Am[2]};
        double* Uo[3] = {a->Ab[0], a->Ab[1], a->Ab[2]};
        ACSE_TRY(acse_contract(c, Dc, Amc, -1, 0.5, 0, Uo, nullptr, 0));
        // U = 1/2 G(Am; D_k); cotangent of U is eps Db
        const double* Ub[3] = {a->Db[0], a->Db[1], a->Db[2]};
        ACSE_TRY(vjp_D(c, Amc, -1, 0.5 * eps, Ub, a->Dn));
        // dL/dAm = 1/2 eps VJP_W(Db); the mask zeroes the same entries of dL/dA
        ACSE_TRY(vjp_W(c, Dc, Ub, a->Wb));
        k_mask_copy<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Wb[0], a->Wb[1], a->Wb[2], mask, c->opt.act_lo,
                                                              c->opt.act_hi, a->Ab[0], a->Ab[1], a->Ab[2]);
        AL(c);
        // Abar = 1/2 eps (masked Wb); through A = G(Kh; D_k): Dn += VJP_D, Kb += 1/2 VJP_W
        for (int b = 0; b < 3; ++b) ACSE_CUDA_TRY(cudaMemsetAsync(a->Am[b], 0, b4, c->stream));
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Ab[0], a->Ab[1], a->Ab[2], 0.5 * eps, 0.5 * eps,
                                                          0.5 * eps, a->Am[0], a->Am[1], a->Am[2]);
        AL(c);
        ACSE_TRY(acse_contract(c, Dc, Kh, +1, 1.0, 0, Ar, nullptr, 0));   // repopulate the W = Kh intermediates
        const double* Abar[3] = {a->Am[0], a->Am[1], a->Am[2]};
        ACSE_TRY(vjp_D(c, Kh, +1, 1.0, Abar, a->Dn));
        ACSE_TRY(vjp_W(c, Dc, Abar, a->Wb));
        k_axpy3<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(n4, a->Wb[0], a->Wb[1], a->Wb[2], 0.5, 0.5, 0.5,
                                                          a->Kb[0], a->Kb[1], a->Kb[2]);
        AL(c);
        for (int b = 0; b < 3; ++b)
            ACSE_CUDA_TRY(cudaMemcpyAsync(a->Db[b], a->Dn[b], b4, cudaMemcpyDeviceToDevice, c->stream));
    }
    // ---- outputs
    double* dD[3] = {dDaa, dDab, dDbb};
    if (dDaa || dDab || dDbb) {
        k_project_D<<<ad_grid(3 * n4), AD_TPB, 0, c->stream>>>(r, a->Db[0], a->Db[1], a->Db[2], a->Dn[0], a->Dn[1],
                                                              a->Dn[2]);
        AL(c);
        for (int b = 0; b < 3; ++b)
            if (dD[b]) ACSE_CUDA_TRY(cudaMemcpyAsync(dD[b], a->Dn[b], b4, cudaMemcpyDefault, c->stream));
    }
    if (dV) {
        k_adj_K_to_V<<<ad_grid(n4), AD_TPB, 0, c->stream>>>(r, a->Kb[0], a->Kb[1], a->Kb[2], a->Vraw);
        AL(c);
        k_sym_V<<<ad_grid(n4), AD_TPB, 0, c->stream>>>(r, a->Vraw, a->Dn[0]);
        AL(c);
        ACSE_CUDA_TRY(cudaMemcpyAsync(dV, a->Dn[0], b4, cudaMemcpyDefault, c->stream));
    }
    if (dh) {
        k_adj_K_to_h<<<r * r, 64, 0, c->stream>>>(r, 1.0 / (2.0 * (c->N - 1)), a->Kb[0], a->Kb[1], a->Kb[2], a->hraw);
        AL(c);
        k_sym_h<<<(r * r + 127) / 128, 128, 0, c->stream>>>(r, a->hraw, a->Dn[1]);
        AL(c);
        ACSE_CUDA_TRY(cudaMemcpyAsync(dh, a->Dn[1], (size_t)r * r * sizeof(double), cudaMemcpyDefault, c->stream));
    }
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ACSE_OK;
}
