// Elementwise, O(r^4) and O(r^5) kernels of the ACSE hot path (FP64).
//
// Notation: spin blocks X_aa, X_ab, X_bb in full-square row-major [i][j][k][l]
// (X_ab = X^{ia jb}_{ka lb}); R2 = r^2.  The O(r^6) work (pair-pair and particle-hole
// GEMMs) is done elsewhere; this file builds their operands and consumes their outputs.
//
// The V-reconstructed three-body sum of Appendix C,
//     B^{ij}_{kl} = sum_{pqr} W^{kp}_{rq} 3D^{ijp}_{rql},
// splits (nine M.1D terms, pairs of which coincide by antisymmetry) into
//     B = (X1 - 2 X2 - X4 + 2 X5 + X7 - 2 X8) / 9,
//     X^{ij}_{kp} = sum_rs M^{ij}_{rs} W^{kp}_{rs}   (pair GEMM)     X1 = X . 1D over p
//     w^k_s  = sum_pr W^{kp}_{rs} 1D^p_r                              X2^{ij}_{kl} = sum_s w^k_s M^{ij}_{ls}
//     Q^k_i  = sum_prs W^{kp}_{rs} M^{ip}_{rs}                        X4 = Q^k_i 1D^j_l,  X7 = Q^k_j 1D^i_l
//     Z^{kp}_{js} = sum_r W^{kp}_{rs} 1D^j_r                          X5^{ij}_{kl} = sum_ps Z^{kp}_{js} M^{ip}_{ls}
//     X8 = X5 with i <-> j                                             (particle-hole GEMM)
// (the E^{ij}_{kl} intermediate of Appendix C is 2 X5 - X4), and the residual of
// Eq. (residual) with the commutator sign convention becomes
//     G(W) = 4 (Y - s Y^T) - 12 (B - B_{k<->l}) + 12 s (B^T - B^T_{i<->j}),   Y = D W^T,
// s = +1 for a pair-Hermitian W (W = K/2: the residual A) and -1 for a pair-anti-Hermitian
// W (W = A: the update, whose commutator sign flips, Appendix B last remark).
#include "acse_internal.h"

#define TPB 256

static inline int grid_for(size_t n, int tpb = TPB) {
    size_t g = (n + tpb - 1) / tpb;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum (deterministic); result valid in thread 0.
__device__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// ---------------------------------------------------------------------------------- K
// Eq. (2) read as K = 1/2(<pq|rs> - <pq|sr>) + (h_pr d_qs + h_qs d_pr - h_ps d_qr - h_qr d_ps)/(2(N-1)),
// <pq|rs> = (pr|qs).  Stored halved: the residual's W is K/2 (H = sum (K/2) a+a+aa).
__global__ void k_build_K(int r, double inv2N1, const double* __restrict__ h, const double* __restrict__ V,
                          double* __restrict__ Kaa, double* __restrict__ Kab, double* __restrict__ Kbb) {
    const size_t n = (size_t)r * r * r * r;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % r), k = (int)((e / r) % r), j = (int)((e / ((size_t)r * r)) % r),
                  i = (int)(e / ((size_t)r * r * r));
        const double vd = V[(((size_t)i * r + k) * r + j) * r + l];   // (ik|jl) = <ij|kl>
        const double vx = V[(((size_t)i * r + l) * r + j) * r + k];   // (il|jk) = <ij|lk>
        const double hik = h[i * r + k] * (j == l), hjl = h[j * r + l] * (i == k);
        const double hil = h[i * r + l] * (j == k), hjk = h[j * r + k] * (i == l);
        const double ks = 0.5 * (vd - vx) + (hik + hjl - hil - hjk) * inv2N1;
        const double kx = 0.5 * vd + (hik + hjl) * inv2N1;
        Kaa[e] = 0.5 * ks;
        Kbb[e] = 0.5 * ks;
        Kab[e] = 0.5 * kx;
    }
}

int launch_build_K(acse_ctx* c) {
    const int r = c->r;
    const size_t n = (size_t)r * r * r * r;
    k_build_K<<<grid_for(n), TPB, 0, c->stream>>>(r, 1.0 / (2.0 * (c->N - 1)), c->w.h, c->w.V, c->w.Kh[0],
                                                  c->w.Kh[1], c->w.Kh[2]);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------------------ 1D and M
// 1D^p_r = 2/(N-1) sum_q 2D^{pq}_{rq} over spin orbitals (App. C):
//   g_a[p][r] = c sum_q (Daa[p][q][r][q] + Dab[p][q][r][q]);  g_b[p][r] = c sum_q (Dbb[p][q][r][q] + Dab[q][p][q][r]).
// One warp per output element (lanes over q, fixed-order warp reduction).
__global__ void __launch_bounds__(256) k_gamma(int r, double cN, const double* __restrict__ Daa,
                                               const double* __restrict__ Dab, const double* __restrict__ Dbb,
                                               double* __restrict__ gam) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= 2 * r * r) return;
    const int sp = t / (r * r), p = (t / r) % r, rr = t % r;
    const size_t r3 = (size_t)r * r * r, r2 = (size_t)r * r;
    double s = 0.0;
    if (sp == 0) {
        for (int q = lane; q < r; q += 32) s += Daa[p * r3 + q * r2 + rr * r + q] + Dab[p * r3 + q * r2 + rr * r + q];
    } else {
        for (int q = lane; q < r; q += 32) s += Dbb[p * r3 + q * r2 + rr * r + q] + Dab[q * r3 + p * r2 + q * r + rr];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) gam[t] = cN * s;
}

// M = 3 2Delta + 1D^1D = 3 2D - 2 (1D^1D), (1D^1D)^{ij}_{kl} = 1/2(g^i_k g^j_l - g^j_k g^i_l) (App. C);
// the exchange piece vanishes in the ab block (1D is spin diagonal).
__global__ void k_build_M(int r, const double* __restrict__ gam, const double* __restrict__ Daa,
                          const double* __restrict__ Dab, const double* __restrict__ Dbb, double* __restrict__ Maa,
                          double* __restrict__ Mab, double* __restrict__ Mbb) {
    const size_t n = (size_t)r * r * r * r;
    const double* ga = gam;
    const double* gb = gam + r * r;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % r), k = (int)((e / r) % r), j = (int)((e / ((size_t)r * r)) % r),
                  i = (int)(e / ((size_t)r * r * r));
        Maa[e] = 3.0 * Daa[e] - (ga[i * r + k] * ga[j * r + l] - ga[j * r + k] * ga[i * r + l]);
        Mbb[e] = 3.0 * Dbb[e] - (gb[i * r + k] * gb[j * r + l] - gb[j * r + k] * gb[i * r + l]);
        Mab[e] = 3.0 * Dab[e] - ga[i * r + k] * gb[j * r + l];
    }
}

int launch_gamma(acse_ctx* c, const double* const D[3]) {
    const int r = c->r;
    k_gamma<<<(2 * r * r + 7) / 8, 256, 0, c->stream>>>(r, 2.0 / (c->N - 1), D[0], D[1], D[2], c->w.gam);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int launch_gamma_M(acse_ctx* c, const double* const D[3]) {
    const int r = c->r;
    ACSE_TRY(launch_gamma(c, D));
    const size_t n = (size_t)r * r * r * r;
    k_build_M<<<grid_for(n), TPB, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], c->w.M[0], c->w.M[1], c->w.M[2]);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------ particle-hole layout of M
// Diagonal ph sector: rows (sI,i,l), cols (sP,p,s) of M^{i sI, p sP}_{l sI, s sP}:
//   (a,a) Maa[i][p][l][s]  (a,b) Mab[i][p][l][s]  (b,a) Mab[p][i][s][l]  (b,b) Mbb[i][p][l][s]
// Spin-flip sectors (both Z and M carry a sign -1 there, which cancels in the product):
//   F1: (I,L) = (ia, lb), (P,S) = (pb, sa):  Mf1[(i,l)][(p,s)] = Mab[i][p][s][l]
//   F2: (I,L) = (ib, la), (P,S) = (pa, sb):  Mf2[(i,l)][(p,s)] = Mab[p][i][l][s]
__global__ void k_pack_Mph(int r, const double* __restrict__ Maa, const double* __restrict__ Mab,
                           const double* __restrict__ Mbb, double* __restrict__ Md, double* __restrict__ Mf1,
                           double* __restrict__ Mf2) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    const size_t nd = 4 * n4;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nd + 2 * n4; e += (size_t)gridDim.x * blockDim.x) {
        if (e < nd) {
            const size_t row = e / (2 * R2), col = e % (2 * R2);
            const int sI = (int)(row / R2), sP = (int)(col / R2);
            const int i = (int)((row % R2) / r), l = (int)(row % r);
            const int p = (int)((col % R2) / r), s = (int)(col % r);
            double v;
            if (sI == 0 && sP == 0) v = Maa[((i * r + p) * (size_t)r + l) * r + s];
            else if (sI == 0) v = Mab[((i * r + p) * (size_t)r + l) * r + s];
            else if (sP == 0) v = Mab[((p * r + i) * (size_t)r + s) * r + l];
            else v = Mbb[((i * r + p) * (size_t)r + l) * r + s];
            Md[e] = v;
        } else {
            const size_t f = e - nd;
            const int which = (int)(f / n4);
            const size_t g = f % n4;
            const int i = (int)(g / (R2 * r)), l = (int)((g / R2) % r), p = (int)((g / r) % r), s = (int)(g % r);
            if (which == 0) Mf1[g] = Mab[((i * r + p) * (size_t)r + s) * r + l];
            else Mf2[g] = Mab[((p * r + i) * (size_t)r + l) * r + s];
        }
    }
}

int launch_pack_Mph(acse_ctx* c) {
    const int r = c->r;
    const size_t n = (size_t)6 * r * r * r * r;
    k_pack_Mph<<<grid_for(n), TPB, 0, c->stream>>>(r, c->w.M[0], c->w.M[1], c->w.M[2], c->w.Md, c->w.Mf1, c->w.Mf2);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------- W-dependent intermediates
// Z, w (acse_tiled.cu) and Q (a partial trace of the pair GEMM output X).

// Q^k_i = sum_prs W^{kp}_{rs} M^{ip}_{rs} is a partial trace of the pair GEMM output
// X^{ij}_{kp} = sum_rs M^{ij}_{rs} W^{kp}_{rs}:  Q^k_i = sum_P X^{iP}_{kP}, i.e.
//   Q_a[k][i] = sum_p Xaa[(i,p)][(k,p)] + sum_p Xab[(i,p)][(k,p)]
//   Q_b[k][i] = sum_p Xbb[(i,p)][(k,p)] + sum_p Xab[(p,i)][(p,k)]
// (O(r^3) instead of O(r^5); Xab already carries the factor 2 of the mixed-spin (rs) sum).  With Xpaa /
// Xpbb set (split path), the same-spin X is read from the packed GEMM output (rows and columns over
// the pairs a < b, row pitch P):  X[(i,p)][(k,p)] = s_ip s_kp Xp[pk(i,p)][pk(k,p)], zero for i = p or
// k = p (s_ab = -1 for a > b), the values the unpacked rows hold.
template <typename T>
__device__ __forceinline__ T q_packed(const T* __restrict__ Xp, int r, int P, int i, int k, int p) {
    if (i == p || k == p) return (T)0;
    const T v = Xp[(size_t)(i < p ? pk_pair(r, i, p) : pk_pair(r, p, i)) * P + (k < p ? pk_pair(r, k, p) : pk_pair(r, p, k))];
    return (i < p) == (k < p) ? v : -v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_Q_from_X(int r, const T* __restrict__ Xaa, const T* __restrict__ Xab,
                                                  const T* __restrict__ Xbb, size_t ldx, const T* __restrict__ Xpaa,
                                                  const T* __restrict__ Xpbb, T* __restrict__ Qv) {
    // one warp per output element, lanes over p, fixed-order warp reduction
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= 2 * r * r) return;
    const int sp = t / (r * r), k = (t / r) % r, i = t % r, P = r * (r - 1) / 2;
    T acc = 0;
    for (int p = lane; p < r; p += 32) {
        const T xs = Xpaa ? q_packed(sp == 0 ? Xpaa : Xpbb, r, P, i, k, p)
                          : (sp == 0 ? Xaa : Xbb)[(size_t)(i * r + p) * ldx + k * r + p];
        const T xab = sp == 0 ? Xab[(size_t)(i * r + p) * ldx + k * r + p] : Xab[(size_t)(p * r + i) * ldx + p * r + k];
        acc += xs + xab;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) Qv[t] = acc;
}

int launch_W_intermediates(acse_ctx* c, const double* const W[3]) { return launch_Z_tiled(c, W, nullptr); }

int launch_Q(acse_ctx* c) {
    const int r = c->r;
    const size_t R2 = (size_t)r * r;
    if (c->opt.prec == ACSE_FP64) {
        k_Q_from_X<double><<<(2 * r * r + 7) / 8, 256, 0, c->stream>>>(r, c->w.X[0], c->w.X[1], c->w.X[2], R2,
                                                                          nullptr, nullptr, c->w.Q);
    } else {
        // same-spin X from the packed GEMM output; spin-flip specialisation: Xbb is the flip of Xaa (same
        // values)
        k_Q_from_X<float><<<(2 * r * r + 7) / 8, 256, 0, c->stream>>>(
            r, nullptr, c->w.tc_pairC[1], nullptr, R2, c->w.tc_pairCp[0], c->w.tc_pairCp[acse_singlet(c) ? 0 : 2],
            c->w.Q32);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------------- B spin types
// T0 = B^{ia ja}_{ka la}, T1 = B^{ib jb}_{kb lb}, T2 = B^{ia jb}_{ka lb}, T3 = B^{ia jb}_{kb la}
// (acse_tiled.cu, one block per pair (i, j)):
//   T0: x1 = sum_p Xaa[ij][kp] ga[p][l], x2 = sum_p wa[k][p] Maa[ij][l][p], x4 = Qa[k][i] ga[j][l],
//       x7 = Qa[k][j] ga[i][l], x5 = X5d[(a,k,j)][(a,i,l)], x8 = X5d[(a,k,i)][(a,j,l)];  T1 the same in b
//   T2: x1 = sum_p Xab[ij][kp] gb[p][l], x2 = -sum_p wa[k][p] Mab[ij][p][l], x4 = Qa[k][i] gb[j][l],
//       x5 = X5f1[(k,j)][(i,l)], x8 = X5d[(a,k,i)][(b,j,l)], x7 = 0
//   T3: x1 = -sum_p Xab[ij][pk] ga[p][l], x2 = sum_p wb[k][p] Mab[ij][l][p], x5 = X5d[(b,k,j)][(a,i,l)],
//       x7 = Qb[k][j] ga[i][l], x8 = X5f2[(k,i)][(j,l)], x4 = 0
//   B = (x1 - 2 x2 - x4 + 2 x5 + x7 - 2 x8) / 9.
int launch_build_B(acse_ctx* c) { return launch_B_tiled(c); }

// --------------------------------------------------------------------------- G assembly
// The B kernel (acse_tiled.cu) leaves H_b = 4 Y_b - 12 (P - P'_{k<->l}) per block b, so that
//   G_b[ij][kl] = H_b[ij][kl] - s H_b[kl][ij]
// (= 4(Y - sY^T) - 12(B - B_{k<->l}) + 12 s (B^T - B^T_{i<->j}) of Appendix B).  out = scale * G,
// transposed reads through 32 x 32 shared-memory tiles; ||.||^2 partials (aa + bb + 4 ab, before
// the mask) per block, in a fixed order.
template <typename T>
struct GArgs {
    int r;
    const T* H[3];
    double* out[3];
    T s, scale;
    int mask, lo, hi;
    int flip;   // spin-flip specialisation: H[2] is not formed; G_bb = G_aa (written from blk 0)
    float* out32[3];   // split path, output into the context's A: the same (FP32-valued) result in FP32
    double* partial;
};

#define G_GRID (152 * 16)
#define G_ASM_GRID (152 * 8)   // k_assemble_G: eight resident blocks of 256 threads per SM, one wave

// Tile pair u of the upper triangle (ti <= tj, row by row) of an n x n tile grid: row ti starts at
// ti n - ti (ti - 1) / 2.  The float estimate is corrected by exact integer steps.
__device__ __forceinline__ void tri_decode(int u, int n, int& ti, int& tj) {
    const float b = 2.0f * (float)n + 1.0f;
    int t = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)u, 0.0f))));
    t = max(0, min(n - 1, t));
    while (t > 0 && t * n - t * (t - 1) / 2 > u) --t;
    while (t + 1 < n && (t + 1) * n - (t + 1) * t / 2 <= u) ++t;
    ti = t;
    tj = t + (u - (t * n - t * (t - 1) / 2));
}

// Per-thread accumulator of the norm: FP64 on the FP64 path; on the FP32 path a double-float pair
// (hi, lo) fed with exact products (v*v and its FMA residual) through Knuth's TwoSum, so that the
// sum keeps about 48 significant bits without FP64 arithmetic (slow on this GPU).
template <typename T>
struct NormAcc;
template <>
struct NormAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v, double m) { s += m * v * v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct NormAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v, float m) {   // m = 1 or 4 (exact scaling)
        const float mv = m * v;
        const float p = __fmul_rn(mv, v);  // never contracted into an FMA
        const float e = fmaf(mv, v, -p);   // p + e = m v^2 exactly
        const float s = hi + p;            // TwoSum(hi, p)
        const float bb = s - hi;
        const float t = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += t + e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
__device__ __forceinline__ void g_put(const GArgs<T>& a, int blk, int r, int R2, int ij, int kl, T v, NormAcc<T>& nrm) {
    nrm.add(v, blk == 1 ? (T)4 : (a.flip ? (T)2 : (T)1));
    T o = v;
    if (a.mask) {
        const int i = ij / r, j = ij - i * r, k = kl / r, l = kl - k * r;
        if (i >= a.lo && i < a.hi && j >= a.lo && j < a.hi && k >= a.lo && k < a.hi && l >= a.lo && l < a.hi) o = (T)0;
    }
    if (a.out[blk]) {
        const double od = (double)o;   // the one conversion of the FP32 path (FP64 conversions are slow here)
        a.out[blk][(size_t)ij * R2 + kl] = od;
        if (a.flip && blk == 0) a.out[2][(size_t)ij * R2 + kl] = od;
    }
    if (a.out32[0]) {   // the split path's FP32 copy: o itself (an FP32 value)
        a.out32[blk][(size_t)ij * R2 + kl] = (float)o;
        if (a.flip && blk == 0) a.out32[2][(size_t)ij * R2 + kl] = (float)o;
    }
}

// G_b = scale (H_b - s H_b^T) (pair transpose), the masked result in FP64 and the unmasked norm
// partials.  Work items are pairs of 32 x 32 tiles (ti <= tj): the tiles P = H[ti rows][tj cols] and
// Q = H[tj rows][ti cols] are read once and give both output tiles, since
//   G[ij][kl] = scale (P[ij][kl] - s Q[kl][ij]),   G[kl][ij] = scale (Q[kl][ij] - s P[ij][kl]).
template <typename T>
__global__ void __launch_bounds__(256) k_assemble_G(const __grid_constant__ GArgs<T> a) {
    __shared__ T P[32][33];
    __shared__ T Q[32][33];
    const int r = a.r;
    const int R2 = r * r;
    const int nT = (R2 + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    NormAcc<T> nrm;
    const int nblk = a.flip ? 2 : 3;
    const int ntri = nT * (nT + 1) / 2;   // tile pairs ti <= tj of one block, dealt out evenly
    for (int w = blockIdx.x; w < nblk * ntri; w += gridDim.x) {
        const int blk = w / ntri;
        int ti, tj;
        tri_decode(w - blk * ntri, nT, ti, tj);
        const T* H = a.H[blk];
        for (int y = ty; y < 32; y += 8) {
            const int pr = ti * 32 + y, pc = tj * 32 + tx;
            P[y][tx] = (pr < R2 && pc < R2) ? H[(size_t)pr * R2 + pc] : (T)0;
            const int qr = tj * 32 + y, qc = ti * 32 + tx;
            Q[y][tx] = (qr < R2 && qc < R2) ? H[(size_t)qr * R2 + qc] : (T)0;
        }
        __syncthreads();
        for (int y = ty; y < 32; y += 8) {
            const int ij = ti * 32 + y, kl = tj * 32 + tx;
            if (ij < R2 && kl < R2) g_put(a, blk, r, R2, ij, kl, a.scale * (P[y][tx] - a.s * Q[tx][y]), nrm);
        }
        if (ti != tj)
            for (int y = ty; y < 32; y += 8) {
                const int kl = tj * 32 + y, ij = ti * 32 + tx;
                if (ij < R2 && kl < R2) g_put(a, blk, r, R2, kl, ij, a.scale * (Q[y][tx] - a.s * P[tx][y]), nrm);
            }
        __syncthreads();
    }
    const double tot = block_sum(nrm.value());
    if (threadIdx.x == 0) a.partial[blockIdx.x] = tot;
}

// Fixed-order final sum of `n` partials into dst (one block).
__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ dst) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
    v = block_sum(v);
    if (threadIdx.x == 0) *dst = v;
}

template <typename T>
static void fill_G(acse_ctx* c, GArgs<T>& a, int sW, double scale, int apply_mask, double* const out[3]) {
    a.r = c->r;
    for (int s = 0; s < 3; ++s) a.out[s] = out[s];
    a.s = (T)sW;
    a.scale = (T)scale;
    a.mask = apply_mask && c->opt.mask_active;
    a.lo = c->opt.act_lo;
    a.hi = c->opt.act_hi;
    a.partial = c->w.partial;
    a.flip = acse_singlet(c) ? 1 : 0;
    for (int s = 0; s < 3; ++s) a.out32[s] = nullptr;
}

int launch_assemble_G(acse_ctx* c, int sW, double scale, int apply_mask, double* const out[3], double* norm2_dst) {
    if (c->opt.prec == ACSE_FP64) {
        GArgs<double> a;
        fill_G(c, a, sW, scale, apply_mask, out);
        for (int s = 0; s < 3; ++s) a.H[s] = c->w.H[s];
        k_assemble_G<double><<<G_ASM_GRID, 256, 0, c->stream>>>(a);
    } else {
        GArgs<float> a;
        fill_G(c, a, sW, scale, apply_mask, out);
        for (int s = 0; s < 3; ++s) a.H[s] = c->w.H32[s];
        // into the context's A: also its FP32 copy, the W of the update pass that follows
        const bool intoA = out[0] == c->w.A[0] && out[1] == c->w.A[1] && out[2] == c->w.A[2];
        if (intoA)
            for (int s = 0; s < 3; ++s) {
                a.out32[s] = c->w.A32[s];
                if (c->a64_skip) a.out[s] = nullptr;   // only the FP32 copy is read after this pass
            }
        c->a32_valid = intoA ? 1 : c->a32_valid;
        k_assemble_G<float><<<G_ASM_GRID, 256, 0, c->stream>>>(a);
    }
    ACSE_LAUNCHED(c);
    if (norm2_dst) {
        k_sum_partials<<<1, TPB, 0, c->stream>>>(c->w.partial, G_ASM_GRID, norm2_dst);
        ACSE_LAUNCHED(c);
    }
    return ACSE_OK;
}

// ----------------------------------------------------------------------------- energy
// E = sum K.2D = 2 [sum Kh_aa D_aa + sum Kh_bb D_bb + 4 sum Kh_ab D_ab]   (Kh = K/2)
__global__ void __launch_bounds__(TPB) k_energy(int r, const double* __restrict__ Kaa, const double* __restrict__ Kab,
                                                const double* __restrict__ Kbb, const double* __restrict__ Daa,
                                                const double* __restrict__ Dab, const double* __restrict__ Dbb,
                                                double* __restrict__ partial) {
    const size_t n4 = (size_t)r * r * r * r;
    double s = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x)
        s += Kaa[e] * Daa[e] + Kbb[e] * Dbb[e] + 4.0 * Kab[e] * Dab[e];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = 2.0 * s;
}

int launch_energy(acse_ctx* c, const double* const D[3], double* E_dst) {
    k_energy<<<G_GRID, TPB, 0, c->stream>>>(c->r, c->w.Kh[0], c->w.Kh[1], c->w.Kh[2], D[0], D[1], D[2],
                                            c->w.partial + G_GRID);
    ACSE_LAUNCHED(c);
    k_sum_partials<<<1, TPB, 0, c->stream>>>(c->w.partial + G_GRID, G_GRID, E_dst);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------------------ axpy
// out = D + (mul * eps) U, eps read from device memory (the line search writes it there); grid y
// selects the block.  double2 accesses when every pointer is 16-byte aligned, with a scalar tail.
__global__ void k_axpy(int n, int vec, const double* __restrict__ D0, const double* __restrict__ D1,
                       const double* __restrict__ D2, const double* __restrict__ U0, const double* __restrict__ U1,
                       const double* __restrict__ U2, const double* __restrict__ eps, double mul, double* O0,
                       double* O1, double* O2) {
    const double e = mul * (*eps);
    const int b = blockIdx.y;
    const double* D = b == 0 ? D0 : b == 1 ? D1 : D2;
    const double* U = b == 0 ? U0 : b == 1 ? U1 : U2;
    double* O = b == 0 ? O0 : b == 1 ? O1 : O2;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const int n2 = n >> 1;
        const double2* D2v = reinterpret_cast<const double2*>(D);
        const double2* U2v = reinterpret_cast<const double2*>(U);
        double2* O2v = reinterpret_cast<double2*>(O);
        for (int i = t0; i < n2; i += stride) {
            const double2 d = D2v[i], u = U2v[i];
            O2v[i] = make_double2(d.x + e * u.x, d.y + e * u.y);
        }
        if ((n & 1) && t0 == 0) O[n - 1] = D[n - 1] + e * U[n - 1];
    } else {
        for (int i = t0; i < n; i += stride) O[i] = D[i] + e * U[i];
    }
}

int launch_axpy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev, double eps_mul,
                double* const out[3]) {
    const int n = c->r * c->r * c->r * c->r;
    uintptr_t bits = 0;
    for (int b = 0; b < 3; ++b) bits |= (uintptr_t)D[b] | (uintptr_t)U[b] | (uintptr_t)out[b];
    const int vec = (bits & 15) == 0;
    k_axpy<<<dim3(grid_for((size_t)n) / 2 + 1, 3), TPB, 0, c->stream>>>(n, vec, D[0], D[1], D[2], U[0], U[1], U[2],
                                                                      eps_dev, eps_mul, out[0], out[1], out[2]);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// D <- D + eps U fused with the energy of the new D: E = 2 [sum Kh_aa D_aa + sum Kh_bb D_bb
// + 4 sum Kh_ab D_ab].  Grid (AXE_X, 3): block row y handles spin block y; block partials
// (partial[y * AXE_X + x]) are summed in a fixed order by k_sum_partials.
#define AXE_X (152 * 4)
__global__ void __launch_bounds__(TPB) k_axpy_energy(int n, int vec, double* D0, double* D1, double* D2,
                                                     const double* __restrict__ U0, const double* __restrict__ U1,
                                                     const double* __restrict__ U2, const double* __restrict__ K0,
                                                     const double* __restrict__ K1, const double* __restrict__ K2,
                                                     const double* __restrict__ eps, double* __restrict__ partial) {
    const double e = *eps;
    const int b = blockIdx.y;
    double* D = b == 0 ? D0 : b == 1 ? D1 : D2;
    const double* U = b == 0 ? U0 : b == 1 ? U1 : U2;
    const double* K = b == 0 ? K0 : b == 1 ? K1 : K2;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (vec) {
        const int n2 = n >> 1;
        double2* Dv = reinterpret_cast<double2*>(D);
        const double2* Uv = reinterpret_cast<const double2*>(U);
        const double2* Kv = reinterpret_cast<const double2*>(K);
        for (int i = t0; i < n2; i += stride) {
            const double2 d = Dv[i], u = Uv[i], k = Kv[i];
            const double2 o = make_double2(d.x + e * u.x, d.y + e * u.y);
            Dv[i] = o;
            acc += k.x * o.x + k.y * o.y;
        }
        if ((n & 1) && t0 == 0) {
            const double o = D[n - 1] + e * U[n - 1];
            D[n - 1] = o;
            acc += K[n - 1] * o;
        }
    } else {
        for (int i = t0; i < n; i += stride) {
            const double o = D[i] + e * U[i];
            D[i] = o;
            acc += K[i] * o;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[b * gridDim.x + blockIdx.x] = (b == 1 ? 8.0 : 2.0) * acc;
}

int launch_axpy_energy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev,
                       double* E_dst) {
    const int n = c->r * c->r * c->r * c->r;
    uintptr_t bits = 0;
    for (int b = 0; b < 3; ++b) bits |= (uintptr_t)D[b] | (uintptr_t)U[b] | (uintptr_t)c->w.Kh[b];
    const int vec = (bits & 15) == 0;
    double* part = c->w.partial + 2 * G_GRID;
    k_axpy_energy<<<dim3(AXE_X, 3), TPB, 0, c->stream>>>(n, vec, D[0], D[1], D[2], U[0], U[1], U[2], c->w.Kh[0],
                                                          c->w.Kh[1], c->w.Kh[2], eps_dev, part);
    ACSE_LAUNCHED(c);
    k_sum_partials<<<1, TPB, 0, c->stream>>>(part, 3 * AXE_X, E_dst);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------------ line search
// scal[2] = e0 (state), scal[4..6] = f(0), f(e0), f(2 e0)  ->  scal[3] = eps, scal[2] = eps.
// Trial values within LS_FLAT f(0) of f(0) are rounding of the merit, not a slope: the step is then e0/4,
// so that implementations whose evaluations differ by rounding take the same steps.
#define LS_FLAT 1e-10

__global__ void k_line_search(double* scal) {
    const double e0 = scal[2], f0 = scal[4], f1 = scal[5], f2 = scal[6];
    const double cc = (f2 - 2.0 * f1 + f0) / (2.0 * e0 * e0);
    double x;
    if (fabs(f1 - f0) <= LS_FLAT * fabs(f0) && fabs(f2 - f0) <= LS_FLAT * fabs(f0)) {
        x = 0.25 * e0;
    } else if (cc > 0.0) {
        const double b = (f1 - f0) / e0 - cc * e0;
        x = -b / (2.0 * cc);
        x = fmin(fmax(x, 0.25 * e0), 2.0 * e0);
    } else {
        x = (f1 <= f2) ? e0 : 2.0 * e0;
    }
    scal[3] = x;
    scal[2] = x;
}

int launch_line_search(acse_ctx* c) {
    k_line_search<<<1, 1, 0, c->stream>>>(c->w.scal);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// --------------------------------------------------------------------------- checks
// scal[7] = spin-orbital trace Tr 2D = Tr aa + Tr bb + 2 Tr ab;  scal[8] = 1 if any entry of D is not finite.
__global__ void k_trace_check(int r, const double* __restrict__ Daa, const double* __restrict__ Dab,
                              const double* __restrict__ Dbb, double* scal) {
    const size_t n4 = (size_t)r * r * r * r, R2 = (size_t)r * r;
    double tr = 0.0, bad = 0.0;
    for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
        const double a = Daa[e], b = Dab[e], c = Dbb[e];
        if (!isfinite(a) || !isfinite(b) || !isfinite(c)) bad = 1.0;
        const size_t row = e / R2, col = e % R2;
        if (row == col) tr += a + c + 2.0 * b;
    }
    tr = block_sum(tr);
    bad = block_sum(bad);
    if (threadIdx.x == 0) {
        scal[7] = tr;
        scal[8] = bad;
    }
}

int launch_trace_check(acse_ctx* c, const double* const D[3]) {
    k_trace_check<<<1, 1024, 0, c->stream>>>(c->r, D[0], D[1], D[2], c->w.scal);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

__global__ void k_copy1(double* dst, const double* src) { *dst = *src; }

int launch_copy_scalar(acse_ctx* c, double* dst, const double* src) {
    k_copy1<<<1, 1, 0, c->stream>>>(dst, src);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}
