// Nakatsuji-Yasuda (NY) 3-cumulant contribution to a contraction pass (Eq. NY and its appendix).
//
// With the NY reconstruction the three-body sum of every pass gains
//     T^{ij}_{kl} = sum_{pqr} W^{kp}_{rq} 3Delta^{ijp}_{rql},
//     3Delta^{ijp}_{rql} = 1/6 sum_a sigma_a A(2Delta^{ia}_{rq} 2Delta^{jp}_{al})  (36 signed terms),
// sigma_a = +1 for HF-occupied spin orbitals (aufbau by orbital index), -1 otherwise.  Using the
// pair antisymmetry of W and 2Delta the 36 terms collapse (nine-term form of the appendix, then
// terms 7-9 equal 4-6) to
//     T = 4/6 [ S1^{ij}_{kl} - S1^{ji}_{kl} - S3 - 2 S4^{ij}_{kl} + 2 S4^{ji}_{kl} + 2 S6 ],
//     X^{ia}_{kp} = sum_{rq} 2Delta^{ia}_{rq} W^{kp}_{rq}          (GEMM, rows (i,a), K (r,q))
//     Y4^{kq}_{ja} = sum_{pr} W^{kp}_{rq} 2Delta^{jp}_{ar}         (GEMM, rows (k,q), K (p,r))
//     Y6^{kr}_{al} = sum_{pq} W^{kp}_{rq} 2Delta^{pa}_{lq}         (GEMM, rows (k,r), K (p,q))
//     S1[k][i][j][l] = sum_{ap} X^{ia}_{kp} sigma_a 2Delta^{jp}_{al} (GEMM, rows (k,i), K (a,p))
//     S4[k][j][i][l] = sum_{aq} Y4^{kq}_{ja} sigma_a 2Delta^{ia}_{lq} (GEMM, rows (k,j), K (a,q))
//     S6[j][i][k][l] = sum_{ar} 2Delta^{ji}_{ar} sigma_a Y6^{kr}_{al} (GEMM, rows (j,i), K (a,r))
//     S3^{ij}_{kl} = sum_a Q[a][k] sigma_a 2Delta^{ji}_{al},  Q[a][k] = sum_p X^{pa}_{kp}.
// This first GPU form works in the dense spin-orbital basis (n = 2r, every GEMM n^2 x n^2 x n^2,
// zero spin blocks included): pack kernels write each operand directly in the GEMM's row layout
// (index permutation, sigma scaling and, in the split precisions, the hi/lo split); the six GEMMs
// run as two grouped launches (FP64 DFMA or tcgen05 split precision, like the V pass); a final
// kernel forms T for the four spin types of the B kernel, which adds it to B.
#include <math.h>

#include "acse_internal.h"
#include "acse_split.cuh"

struct NyWork {
    int n;                 // spin orbitals
    size_t n2, n4;
    int Kp;                // padded K per split term (split precisions)
    double* delta[3];      // 2Delta blocks aa, ab, bb (FP64)
    double* sig;           // [n] sigma_a
    void* opA[3];          // operand rows of the three GEMMs of a stage
    void* opB[3];
    void* out[6];          // X, Y4, Y6, S1, S4, S6 (n^4 each; double or float)
    void* Q;               // [n][n]
    void* tny[4];          // T for the B spin types (r^4 each; double or float)
    TcTable st[2];         // split precisions: the two GEMM stages
};

// Element T^{x1 x2}_{x3 x4} (spin-orbital indices, alpha first) of a pair-antisymmetric tensor stored
// as its aa, ab, bb blocks (the other nonzero blocks follow by antisymmetry within each pair).
__device__ __forceinline__ double so_get(const double* aa, const double* ab, const double* bb, int r, int x1, int x2,
                                         int x3, int x4) {
    const int s1 = x1 >= r, s2 = x2 >= r, s3 = x3 >= r, s4 = x4 >= r;
    const int a = x1 - s1 * r, b = x2 - s2 * r, c = x3 - s3 * r, d = x4 - s4 * r;
    const size_t R = r;
    auto at = [&](const double* t, int i, int j, int k, int l) { return t[((i * R + j) * R + k) * R + l]; };
    if (s1 + s2 != s3 + s4) return 0.0;
    if (s1 == s2) return s1 ? at(bb, a, b, c, d) : at(aa, a, b, c, d);
    if (s1 == 0 && s3 == 0) return at(ab, a, b, c, d);     // (a b | a b)
    if (s1 == 1 && s3 == 1) return at(ab, b, a, d, c);     // (b a | b a)
    if (s1 == 0) return -at(ab, a, b, d, c);               // (a b | b a)
    return -at(ab, b, a, c, d);                            // (b a | a b)
}

// 2Delta = 2D - 1D^1D per block: aa/bb: D - 1/2 (g_ik g_jl - g_jk g_il), ab: D - 1/2 ga_ik gb_jl.
__global__ void k_ny_delta(int r, const double* __restrict__ gam, const double* __restrict__ Daa,
                           const double* __restrict__ Dab, const double* __restrict__ Dbb, double* daa, double* dab,
                           double* dbb) {
    const size_t R2 = (size_t)r * r, n4 = R2 * R2;
    const double* ga = gam;
    const double* gb = gam + R2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % r), k = (int)((e / r) % r), j = (int)((e / R2) % r), i = (int)(e / (R2 * r));
        daa[e] = Daa[e] - 0.5 * (ga[i * r + k] * ga[j * r + l] - ga[j * r + k] * ga[i * r + l]);
        dbb[e] = Dbb[e] - 0.5 * (gb[i * r + k] * gb[j * r + l] - gb[j * r + k] * gb[i * r + l]);
        dab[e] = Dab[e] - 0.5 * ga[i * r + k] * gb[j * r + l];
    }
}

// sigma_a: +1 for the first n_alpha alpha and the first n_beta beta orbitals, -1 otherwise.
__global__ void k_ny_sigma(int r, int na, int nb, double* sig) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * r) return;
    sig[x] = (x < r ? x < na : x - r < nb) ? 1.0 : -1.0;
}

// Operand rows: row (u0, u1) = u0 * n + u1, column (u2, u3) = u2 * n + u3, value
//   [sigma[u2]] * src(u[P0], u[P1], u[P2], u[P3]),
// src = a pair-antisymmetric tensor given by blocks (blk != null) or a dense n^4 tensor (dense).
// PREC = ACSE_FP64: plain double rows of length n^2; otherwise split rows (PAT 0: A, 1: B) of
// ns * Kp elements.  One block per row, threads over groups of four columns.
struct NyPack {
    const double* blk[3];
    const void* dense;     // double (FP64 path) or float (split path)
    int P[4];
    int use_sigma;
    const double* sig;
    void* dst;
    size_t ld;             // row length of dst in elements
    int Kp;
};

template <int PREC, int PAT>
__global__ void __launch_bounds__(256) k_ny_pack(int r, const __grid_constant__ NyPack a) {
    const int n = 2 * r;
    const int n2 = n * n;
    const int row = blockIdx.x;
    const int u0 = row / n, u1 = row - (row / n) * n;
    for (int g = threadIdx.x; g < n2 / 4; g += blockDim.x) {
        float xf[4];
        double xd[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = 4 * g + c;
            const int u2 = col / n, u3 = col - (col / n) * n;
            const int u[4] = {u0, u1, u2, u3};
            const int s0 = u[a.P[0]], s1 = u[a.P[1]], s2 = u[a.P[2]], s3 = u[a.P[3]];
            double v;
            if (a.blk[0]) {
                v = so_get(a.blk[0], a.blk[1], a.blk[2], r, s0, s1, s2, s3);
            } else {
                const size_t e = (((size_t)s0 * n + s1) * n + s2) * n + s3;
                v = PREC == ACSE_FP64 ? ((const double*)a.dense)[e] : (double)((const float*)a.dense)[e];
            }
            if (a.use_sigma) v *= a.sig[u2];
            xd[c] = v;
            xf[c] = (float)v;
        }
        if (PREC == ACSE_FP64) {
            double* d = (double*)a.dst + (size_t)row * a.ld + 4 * g;
            *reinterpret_cast<double2*>(d) = make_double2(xd[0], xd[1]);
            *reinterpret_cast<double2*>(d + 2) = make_double2(xd[2], xd[3]);
        } else {
            put4<PREC, PAT>(a.dst, (size_t)row, a.ld, a.Kp, 4 * g, xf);
        }
    }
}

// Q[a][k] = sum_p X^{pa}_{kp}  (X dense, [p][a][k][p]): one warp per (a, k).
template <typename T>
__global__ void __launch_bounds__(256) k_ny_Q(int n, const T* __restrict__ X, T* __restrict__ Q) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= n * n) return;
    const int a = t / n, k = t - (t / n) * n;
    T s = 0;
    for (int p = lane; p < n; p += 32) s += X[(((size_t)p * n + a) * n + k) * n + p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) Q[t] = s;
}

// T for the spin type tt of block (i', j') (types of the B kernel: 0 aaaa, 1 bbbb, 2 (ia jb | ka lb),
// 3 (ia jb | kb la)); threads over (k', l').  S3 uses 1D-free factors staged in shared memory:
// qs[a][k'] = sigma_a Q[a][k], dv[a][l'] = 2Delta^{ji}_{al}.
template <typename T>
__global__ void __launch_bounds__(256) k_ny_assemble(int r, const T* __restrict__ S1, const T* __restrict__ S4,
                                                     const T* __restrict__ S6, const T* __restrict__ Q,
                                                     const double* __restrict__ daa, const double* __restrict__ dab,
                                                     const double* __restrict__ dbb, const double* __restrict__ sig,
                                                     T* t0, T* t1, T* t2, T* t3) {
    extern __shared__ __align__(16) unsigned char ny_smem[];
    const int n = 2 * r, R2 = r * r;
    T* qs = (T*)ny_smem;           // [n][r]
    T* dv = qs + (size_t)n * r;    // [n][r]
    const int tt = blockIdx.x / R2, ij = blockIdx.x % R2;
    const int ip = ij / r, jp = ij % r;
    const int si = tt == 1, sj = tt == 0 ? 0 : 1, sk = tt == 1 || tt == 3, sl = tt == 1 || tt == 2;
    const int i = si * r + ip, j = sj * r + jp;
    for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
        const int aa_ = e / r, c = e % r;
        qs[e] = (T)(sig[aa_] * (double)Q[(size_t)aa_ * n + sk * r + c]);
        dv[e] = (T)so_get(daa, dab, dbb, r, j, i, aa_, sl * r + c);
    }
    __syncthreads();
    T* out = tt == 0 ? t0 : tt == 1 ? t1 : tt == 2 ? t2 : t3;
    const size_t nn = (size_t)n;
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const int kp = e / r, lp = e % r;
        const int k = sk * r + kp, l = sl * r + lp;
        T s3 = 0;
        for (int a_ = 0; a_ < n; ++a_) s3 += qs[a_ * r + kp] * dv[a_ * r + lp];
        const T s1a = S1[((k * nn + i) * nn + j) * nn + l], s1b = S1[((k * nn + j) * nn + i) * nn + l];
        const T s4a = S4[((k * nn + j) * nn + i) * nn + l], s4b = S4[((k * nn + i) * nn + j) * nn + l];
        const T s6 = S6[((j * nn + i) * nn + k) * nn + l];
        out[(size_t)ij * R2 + e] = (T)(4.0 / 6.0) * (s1a - s1b - s3 - (T)2 * s4a + (T)2 * s4b + (T)2 * s6);
    }
}

// ------------------------------------------------------------------------------ host side
static int ny_malloc(void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ACSE_ERR_NOMEM;
    }
    return ACSE_OK;
}

void ny_free(acse_ctx* c) {
    NyWork* y = (NyWork*)c->ny;
    if (!y) return;
    void* ptrs[] = {y->delta[0], y->delta[1], y->delta[2], y->sig, y->opA[0], y->opA[1], y->opA[2], y->opB[0],
                    y->opB[1], y->opB[2], y->out[0], y->out[1], y->out[2], y->out[3], y->out[4], y->out[5], y->Q,
                    y->tny[0], y->tny[1], y->tny[2], y->tny[3]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int s = 0; s < 2; ++s)
        if (y->st[s].host) tc_table_free(&y->st[s]);
    free(y);
    c->ny = nullptr;
}

static int ny_pack_launch(acse_ctx* c, const NyPack& pk, int pat) {
    const int r = c->r, n2 = 4 * r * r;
    switch (c->opt.prec) {
        case ACSE_FP64: k_ny_pack<ACSE_FP64, 0><<<n2, 256, 0, c->stream>>>(r, pk); break;
        case ACSE_BF16X3:
            if (pat) k_ny_pack<ACSE_BF16X3, 1><<<n2, 256, 0, c->stream>>>(r, pk);
            else k_ny_pack<ACSE_BF16X3, 0><<<n2, 256, 0, c->stream>>>(r, pk);
            break;
        case ACSE_TF32X3:
            if (pat) k_ny_pack<ACSE_TF32X3, 1><<<n2, 256, 0, c->stream>>>(r, pk);
            else k_ny_pack<ACSE_TF32X3, 0><<<n2, 256, 0, c->stream>>>(r, pk);
            break;
        default:
            if (pat) k_ny_pack<ACSE_TF32, 1><<<n2, 256, 0, c->stream>>>(r, pk);
            else k_ny_pack<ACSE_TF32, 0><<<n2, 256, 0, c->stream>>>(r, pk);
            break;
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int ny_alloc(acse_ctx* c) {
    NyWork* y = (NyWork*)calloc(1, sizeof(NyWork));
    if (!y) return ACSE_ERR_NOMEM;
    c->ny = y;
    const int r = c->r, n = 2 * r;
    y->n = n;
    y->n2 = (size_t)n * n;
    y->n4 = y->n2 * y->n2;
    const size_t r4 = (size_t)r * r * r * r;
    const bool f64 = c->opt.prec == ACSE_FP64;
    const size_t es = f64 ? 8 : 4;                                  // GEMM output / T element
    for (int b = 0; b < 3; ++b) ACSE_TRY(ny_malloc((void**)&y->delta[b], r4 * sizeof(double)));
    ACSE_TRY(ny_malloc((void**)&y->sig, n * sizeof(double)));
    size_t op_bytes;
    if (f64) {
        op_bytes = y->n4 * sizeof(double);
    } else {
        const int ops = c->opt.prec == ACSE_BF16X3 ? 2 : 4;         // operand element bytes
        const int kb = 128 / ops;
        y->Kp = (int)((y->n2 + kb - 1) / kb * kb);
        op_bytes = y->n2 * (size_t)c->nsplit * y->Kp * ops;
    }
    for (int s = 0; s < 3; ++s) {
        ACSE_TRY(ny_malloc(&y->opA[s], op_bytes));
        ACSE_TRY(ny_malloc(&y->opB[s], op_bytes));
        if (!f64) {   // K padding is never written afterwards
            ACSE_CUDA_TRY(cudaMemset(y->opA[s], 0, op_bytes));
            ACSE_CUDA_TRY(cudaMemset(y->opB[s], 0, op_bytes));
        }
    }
    for (int o = 0; o < 6; ++o) ACSE_TRY(ny_malloc(&y->out[o], y->n4 * es));
    ACSE_TRY(ny_malloc(&y->Q, y->n2 * es));
    for (int t = 0; t < 4; ++t) ACSE_TRY(ny_malloc(&y->tny[t], r4 * es));
    k_ny_sigma<<<(n + 127) / 128, 128, 0, c->stream>>>(r, c->opt.n_alpha, c->opt.n_beta, y->sig);
    ACSE_LAUNCHED(c);
    if (!f64) {
        const int kind = (c->opt.prec == ACSE_TF32 || c->opt.prec == ACSE_TF32X3) ? 1 : 0;
        const int L = c->nsplit * y->Kp;
        const int N2 = (int)y->n2;
        for (int s = 0; s < 2; ++s) {
            ACSE_TRY(tc_table_init(&y->st[s], kind, 256));
            for (int g = 0; g < 3; ++g)
                ACSE_TRY(tc_table_add(&y->st[s], y->opA[g], y->opB[g], (float*)y->out[3 * s + g], N2, N2, L, N2, 1.0f));
            tc_table_set_err(&y->st[s], c->w.tc_err);
            ACSE_TRY(tc_table_upload(&y->st[s]));
        }
    }
    return ACSE_OK;
}

static NyPack ny_pk(const double* const blk[3], const void* dense, int p0, int p1, int p2, int p3, int sigma,
                    const double* sig, void* dst, size_t ld, int Kp) {
    NyPack k;
    for (int b = 0; b < 3; ++b) k.blk[b] = blk ? blk[b] : nullptr;
    k.dense = dense;
    k.P[0] = p0;
    k.P[1] = p1;
    k.P[2] = p2;
    k.P[3] = p3;
    k.use_sigma = sigma;
    k.sig = sig;
    k.dst = dst;
    k.ld = ld;
    k.Kp = Kp;
    return k;
}

// The NY term T for the pass in flight (D = c->cur_D, W = c->cur_W, 1D in c->w.gam), left in the
// four spin-type buffers the B kernel adds to B.
int ny_pass(acse_ctx* c) {
    NyWork* y = (NyWork*)c->ny;
    if (!y) return ACSE_ERR_UNSUPPORTED;
    const int r = c->r;
    const bool f64 = c->opt.prec == ACSE_FP64;
    const size_t r4 = (size_t)r * r * r * r;
    k_ny_delta<<<152 * 8, 256, 0, c->stream>>>(r, c->w.gam, c->cur_D[0], c->cur_D[1], c->cur_D[2], y->delta[0],
                                               y->delta[1], y->delta[2]);
    ACSE_LAUNCHED(c);
    const double* Dl[3] = {y->delta[0], y->delta[1], y->delta[2]};
    const double* W[3] = {c->cur_W[0], c->cur_W[1], c->cur_W[2]};
    const size_t ld = f64 ? y->n2 : (size_t)c->nsplit * y->Kp;
    // stage 1: X (rows (i,a), K (r,q)), Y4 (rows (k,q), K (p,r)), Y6 (rows (k,r), K (p,q))
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 0, 1, 2, 3, 0, y->sig, y->opA[0], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(W, nullptr, 0, 1, 2, 3, 0, y->sig, y->opB[0], ld, y->Kp), 1));
    ACSE_TRY(ny_pack_launch(c, ny_pk(W, nullptr, 0, 2, 3, 1, 0, y->sig, y->opA[1], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 0, 2, 1, 3, 0, y->sig, y->opB[1], ld, y->Kp), 1));
    ACSE_TRY(ny_pack_launch(c, ny_pk(W, nullptr, 0, 2, 1, 3, 0, y->sig, y->opA[2], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 2, 0, 1, 3, 0, y->sig, y->opB[2], ld, y->Kp), 1));
    const int N2 = (int)y->n2;
    auto gemms = [&](int s) -> int {
        if (f64) {
            GemmF64 g[3];
            for (int k = 0; k < 3; ++k)
                g[k] = GemmF64{(const double*)y->opA[k], (const double*)y->opB[k], (double*)y->out[3 * s + k], N2, N2,
                               N2, N2, N2, N2, 1.0, 0.0, 0, 0, 0};
            return gemm_f64_grouped(c, g, 3, c->stream);
        }
        ACSE_TRY(tc_table_launch(&y->st[s], c->stream));
        c->launches++;
        return ACSE_OK;
    };
    ACSE_TRY(gemms(0));
    // stage 2: S1 (rows (k,i), K (a,p)), S4 (rows (k,j), K (a,q)), S6 (rows (j,i), K (a,r))
    ACSE_TRY(ny_pack_launch(c, ny_pk(nullptr, y->out[0], 1, 2, 0, 3, 1, y->sig, y->opA[0], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 0, 3, 2, 1, 0, y->sig, y->opB[0], ld, y->Kp), 1));
    ACSE_TRY(ny_pack_launch(c, ny_pk(nullptr, y->out[1], 0, 3, 1, 2, 1, y->sig, y->opA[1], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 0, 2, 1, 3, 0, y->sig, y->opB[1], ld, y->Kp), 1));
    ACSE_TRY(ny_pack_launch(c, ny_pk(Dl, nullptr, 0, 1, 2, 3, 1, y->sig, y->opA[2], ld, y->Kp), 0));
    ACSE_TRY(ny_pack_launch(c, ny_pk(nullptr, y->out[2], 0, 3, 2, 1, 0, y->sig, y->opB[2], ld, y->Kp), 1));
    ACSE_TRY(gemms(1));
    const int n = y->n;
    const size_t smem = 2 * (size_t)n * r * (f64 ? sizeof(double) : sizeof(float));
    if (f64) {
        k_ny_Q<double><<<(n * n + 7) / 8, 256, 0, c->stream>>>(n, (const double*)y->out[0], (double*)y->Q);
        ACSE_LAUNCHED(c);
        k_ny_assemble<double><<<4 * r * r, 256, smem, c->stream>>>(
            r, (const double*)y->out[3], (const double*)y->out[4], (const double*)y->out[5], (const double*)y->Q, Dl[0],
            Dl[1], Dl[2], y->sig, (double*)y->tny[0], (double*)y->tny[1], (double*)y->tny[2], (double*)y->tny[3]);
    } else {
        k_ny_Q<float><<<(n * n + 7) / 8, 256, 0, c->stream>>>(n, (const float*)y->out[0], (float*)y->Q);
        ACSE_LAUNCHED(c);
        k_ny_assemble<float><<<4 * r * r, 256, smem, c->stream>>>(
            r, (const float*)y->out[3], (const float*)y->out[4], (const float*)y->out[5], (const float*)y->Q, Dl[0],
            Dl[1], Dl[2], y->sig, (float*)y->tny[0], (float*)y->tny[1], (float*)y->tny[2], (float*)y->tny[3]);
    }
    ACSE_LAUNCHED(c);
    (void)r4;
    return ACSE_OK;
}

// T buffers of the four B spin types (null without NY).
const void* ny_terms(acse_ctx* c, int t) {
    NyWork* y = (NyWork*)c->ny;
    return y ? y->tny[t] : nullptr;
}

int ny_set_attrs() {
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_ny_assemble<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 2 * ACSE_MAX_R * ACSE_MAX_R * (int)sizeof(double)));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_ny_assemble<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 2 * ACSE_MAX_R * ACSE_MAX_R * (int)sizeof(float)));
    return ACSE_OK;
}
