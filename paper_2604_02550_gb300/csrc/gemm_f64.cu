// FP64 grouped "NT" GEMM on the DFMA pipe:  C = alpha * A . B^T (+ beta C), A and B K-major.
//
// One launch runs every tile of up to GEMM_F64_MAXP problems (the sector GEMMs of one
// contraction pass).  GB300's FP64 rate is low (about 2 DFMA per clock per SM), so each
// 64x64 tile with a 4x4 register block per thread is bound by the DFMA pipe, not by shared
// memory or HBM; the kernel keeps the loads simple and guarded (any M, N, K, lda, ldb).
#include "acse_internal.h"

#define GEMM_F64_MAXP 40
#define GF_BM 64
#define GF_BN 64
#define GF_BK 16

struct GemmF64Batch {
    GemmF64 p[GEMM_F64_MAXP];
    int prefix[GEMM_F64_MAXP + 1];
    int tiles_n[GEMM_F64_MAXP];
    int nprob;
};

__global__ void __launch_bounds__(256) k_gemm_f64(const __grid_constant__ GemmF64Batch b) {
    const int t = blockIdx.x;
    int pi = 0;
    while (pi + 1 < b.nprob && b.prefix[pi + 1] <= t) ++pi;
    const GemmF64& P = b.p[pi];
    const int local = t - b.prefix[pi];
    const int m0 = (local / b.tiles_n[pi]) * GF_BM;
    const int n0 = (local % b.tiles_n[pi]) * GF_BN;

    __shared__ double As[GF_BK][GF_BM + 1];
    __shared__ double Bs[GF_BK][GF_BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid & 15;   // n direction
    const int ty = tid >> 4;   // m direction
    const int lrow = tid >> 2;          // 0..63 : row of the operand tile this thread loads
    const int lk = (tid & 3) * 4;       // 0,4,8,12

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    const int M = P.M, N = P.N, K = P.K;
    const double* __restrict__ A = P.A;
    const double* __restrict__ B = P.B;
    const bool arow_ok = (m0 + lrow) < M;
    const bool brow_ok = (n0 + lrow) < N;
    // element (row, k) of each operand: row-major (K-major) or transposed storage
    const size_t a_rs = P.transA ? 1 : (size_t)P.lda, a_ks = P.transA ? (size_t)P.lda : 1;
    const size_t b_rs = P.transB ? 1 : (size_t)P.ldb, b_ks = P.transB ? (size_t)P.ldb : 1;
    const double* Arow = A + (size_t)(m0 + lrow) * a_rs;
    const double* Brow = B + (size_t)(n0 + lrow) * b_rs;

    for (int k0 = 0; k0 < K; k0 += GF_BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + lk + q;
            As[lk + q][lrow] = (arow_ok && k < K) ? Arow[(size_t)k * a_ks] : 0.0;
            Bs[lk + q][lrow] = (brow_ok && k < K) ? Brow[(size_t)k * b_ks] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GF_BK; ++kk) {
            double a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    const double alpha = P.alpha, beta = P.beta;
    const int pr = P.perm_r, pR2 = pr * pr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            size_t dst;
            if (pr) {   // row (sK, k, j), column (sI, i, l) -> Cp[sK * nsb + sI][(i, j)][(k, l)]
                const int nsb = N / pR2;
                const int sK = m / pR2, kk = (m % pR2) / pr, jj = m % pr;
                const int sI = n / pR2, ii = (n % pR2) / pr, ll = n % pr;
                dst = ((size_t)(sK * nsb + sI) * pR2 + (size_t)ii * pr + jj) * pR2 + (size_t)kk * pr + ll;
            } else {
                dst = (size_t)m * P.ldc + n;
            }
            double v = alpha * acc[i][j];
            if (beta != 0.0) v += beta * P.C[dst];
            P.C[dst] = v;
        }
    }
}

int gemm_f64_grouped(acse_ctx* c, const GemmF64* probs, int nprob, cudaStream_t s) {
    int done = 0;
    while (done < nprob) {
        GemmF64Batch b;
        int np = nprob - done;
        if (np > GEMM_F64_MAXP) np = GEMM_F64_MAXP;
        int tiles = 0;
        int used = 0;
        for (int i = 0; i < np; ++i) {
            const GemmF64& q = probs[done + i];
            if (q.M <= 0 || q.N <= 0) continue;
            b.p[used] = q;
            b.prefix[used] = tiles;
            b.tiles_n[used] = (q.N + GF_BN - 1) / GF_BN;
            tiles += ((q.M + GF_BM - 1) / GF_BM) * b.tiles_n[used];
            ++used;
        }
        b.prefix[used] = tiles;
        b.nprob = used;
        if (tiles > 0) {
            ACSE_TRY(prof_begin(c));
            k_gemm_f64<<<tiles, 256, 0, s>>>(b);
            ACSE_LAUNCHED(c);
            ACSE_TRY(prof_end(c));
        }
        done += np;
    }
    return ACSE_OK;
}
