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
// Layout: spin-orbital index pairs are numbered spin-major, pair (x, y) -> (2 s_x + s_y) r^2 + x' r + y'
// (x = s_x r + x'), so every spin block of an n^2 x n^2 matrix (n = 2r) is a contiguous r^2 x r^2
// block.  Pack kernels write each GEMM operand in its row layout (index permutation, sigma scaling
// and, in the split precisions, the hi/lo split, K arranged per spin block); spin conservation of
// the operands leaves about 10 of the 64 (row, column, K) spin-block triples of a GEMM nonzero, and
// the K blocks of each nonzero output block are ordered to be contiguous, so each output block is
// one r^2 x r^2 problem of one grouped launch (FP64 DFMA or tcgen05).  A final kernel forms T for
// the four spin types of the B kernel, which adds it to B.
#include <math.h>

#include "acse_internal.h"
#include "acse_split.cuh"

struct NyWork {
    int n;                 // spin orbitals
    size_t n2, n4;
    int Kb;                // padded r^2: K elements of one spin block per split term
    double* delta[3];      // 2Delta blocks aa, ab, bb (FP64)
    double* sig;           // [n] sigma_a
    void* opA[3];          // operand rows of the three GEMMs of a stage
    void* opB[3];
    void* out[6];          // X, Y4, Y6, S1, S4, S6 (n^4 each; double or float)
    void* Q;               // [n][n]
    void* tny[4];          // T for the B spin types (r^4 each; double or float)
    TcTable st[2];         // split precisions: the two GEMM stages
    int Kbw;               // elements of one K spin block of an operand row (ns * padded r^2)
    int korder[6][4];      // per GEMM: spin pair (2 s + s') of K block position q
    int nprob[6];
    int prob[6][16][4];    // per GEMM: (row block, column block, first K block, K blocks)
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

// Spin-major number of the spin-orbital pair (x, y).
__device__ __forceinline__ size_t ny_pidx(int r, int x, int y) {
    const int sx = x >= r, sy = y >= r;
    return (size_t)(2 * sx + sy) * r * r + (size_t)(x - sx * r) * r + (y - sy * r);
}

// Element (x1 x2 | x3 x4) of a dense intermediate stored as [pair(x1,x2)][pair(x3,x4)].
template <typename T>
__device__ __forceinline__ T ny_dense(const T* t, int r, int x1, int x2, int x3, int x4) {
    return t[ny_pidx(r, x1, x2) * (size_t)(4 * r * r) + ny_pidx(r, x3, x4)];
}

// Operand row `row` (spin-major pair (u0, u1)); K position (q, t): spin block q holds the pair
// korder[q], t = u2' r + u3'.  Value [sigma[u2]] * src(u[P0], u[P1], u[P2], u[P3]), src a
// pair-antisymmetric tensor given by blocks (blk != null) or a dense intermediate.  FP64: rows of
// 4 r^2 doubles (block q at q r^2); split: rows of 4 Kbw elements (block q at q Kbw, its hi/lo
// segments Kb apart).
struct NyPack {
    const double* blk[3];
    const void* dense;     // double (FP64 path) or float (split path)
    int P[4];
    int use_sigma;
    const double* sig;
    void* dst;
    size_t ld;             // row length of dst in elements
    int Kb, Kbw;
    int korder[4];
    int need[4];           // per row block: bit kb set when some problem reads K spin block kb
};

template <int PREC, int PAT>
__global__ void __launch_bounds__(256) k_ny_pack(int r, const __grid_constant__ NyPack a) {
    const int R2 = r * r;
    const int row = blockIdx.x;
    const int rb = row / R2, rr = row - rb * R2;
    const int u0 = (rb >> 1) * r + rr / r, u1 = (rb & 1) * r + rr % r;
    const bool vec = (R2 & 3) == 0;
    const int ngroups = vec ? R2 / 4 : R2;
    const int per = vec ? 4 : 1;
    for (int e = threadIdx.x; e < 4 * ngroups; e += blockDim.x) {
        const int q = e / ngroups, t0 = (e - q * ngroups) * per;
        const int code = a.korder[q];
        if (!(a.need[rb] >> code & 1)) continue;   // no problem reads this block
        float xf[4];
        double xd[4];
        for (int c = 0; c < per; ++c) {
            const int t = t0 + c;
            const int u2 = (code >> 1) * r + t / r, u3 = (code & 1) * r + t % r;
            const int u[4] = {u0, u1, u2, u3};
            const int s0 = u[a.P[0]], s1 = u[a.P[1]], s2 = u[a.P[2]], s3 = u[a.P[3]];
            double v;
            if (a.blk[0]) v = so_get(a.blk[0], a.blk[1], a.blk[2], r, s0, s1, s2, s3);
            else if (PREC == ACSE_FP64) v = ny_dense((const double*)a.dense, r, s0, s1, s2, s3);
            else v = (double)ny_dense((const float*)a.dense, r, s0, s1, s2, s3);
            if (a.use_sigma) v *= a.sig[u2];
            xd[c] = v;
            xf[c] = (float)v;
        }
        if (PREC == ACSE_FP64) {
            double* d = (double*)a.dst + (size_t)row * a.ld + (size_t)q * R2 + t0;
            if (vec) {
                *reinterpret_cast<double2*>(d) = make_double2(xd[0], xd[1]);
                *reinterpret_cast<double2*>(d + 2) = make_double2(xd[2], xd[3]);
            } else {
                d[0] = xd[0];
            }
        } else {
            const size_t off = (size_t)q * a.Kbw;    // elements; the block's segments start here
            void* base = PREC == ACSE_BF16X3 ? (void*)((__nv_bfloat16*)a.dst + off) : (void*)((float*)a.dst + off);
            if (vec) put4<PREC, PAT>(base, (size_t)row, a.ld, a.Kb, t0, xf);
            else put<PREC, PAT>(base, (size_t)row, a.ld, a.Kb, t0, xf[0]);
        }
    }
}

// Q[a][k] = sum_p X^{pa}_{kp}: one warp per (a, k).
template <typename T>
__global__ void __launch_bounds__(256) k_ny_Q(int r, const T* __restrict__ X, T* __restrict__ Q) {
    const int n = 2 * r;
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= n * n) return;
    const int a = t / n, k = t - (t / n) * n;
    T s = 0;
    for (int p = lane; p < n; p += 32) s += ny_dense(X, r, p, a, k, p);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) Q[t] = s;
}

// T for the spin type tt of block (i', j') (types of the B kernel: 0 aaaa, 1 bbbb, 2 (ia jb | ka lb),
// 3 (ia jb | kb la)); threads over (k', l').  S3 from factors staged in shared memory:
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
    for (int e = threadIdx.x; e < R2; e += blockDim.x) {
        const int kp = e / r, lp = e % r;
        const int k = sk * r + kp, l = sl * r + lp;
        T s3 = 0;
        for (int a_ = 0; a_ < n; ++a_) s3 += qs[a_ * r + kp] * dv[a_ * r + lp];
        const T s1a = ny_dense(S1, r, k, i, j, l), s1b = ny_dense(S1, r, k, j, i, l);
        const T s4a = ny_dense(S4, r, k, j, i, l), s4b = ny_dense(S4, r, k, i, j, l);
        const T s6 = ny_dense(S6, r, j, i, k, l);
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

// Operands of the six GEMMs (stage 1: X, Y4, Y6; stage 2: S1, S4, S6).  src: 0 = 2Delta blocks,
// 1 = W blocks, 2 + o = dense intermediate o; cons: 0 when the source conserves s1 + s2 = s3 + s4
// (2Delta, W, X), 1 when it conserves s1 + s4 = s2 + s3 (Y4, Y6).
struct NyOp {
    int src, P[4], sigma, cons;
};
static const NyOp k_ny_ops[6][2] = {
    {{0, {0, 1, 2, 3}, 0, 0}, {1, {0, 1, 2, 3}, 0, 0}},   // X  = 2Delta(i,a|r,q) . W(k,p|r,q)
    {{1, {0, 2, 3, 1}, 0, 0}, {0, {0, 2, 1, 3}, 0, 0}},   // Y4 = W(k,q|p,r) . 2Delta(j,a|p,r)
    {{1, {0, 2, 1, 3}, 0, 0}, {0, {2, 0, 1, 3}, 0, 0}},   // Y6 = W(k,r|p,q) . 2Delta(a,l|p,q)
    {{2, {1, 2, 0, 3}, 1, 0}, {0, {0, 3, 2, 1}, 0, 0}},   // S1 = sigma X(k,i|a,p) . 2Delta(j,l|a,p)
    {{3, {0, 3, 1, 2}, 1, 1}, {0, {0, 2, 1, 3}, 0, 0}},   // S4 = sigma Y4(k,j|a,q) . 2Delta(i,l|a,q)
    {{0, {0, 1, 2, 3}, 1, 0}, {4, {0, 3, 2, 1}, 0, 1}},   // S6 = sigma 2Delta(j,i|a,r) . Y6(k,l|a,r)
};

static bool ny_allowed(const NyOp& op, int rb, int kb) {
    const int su[4] = {rb >> 1, rb & 1, kb >> 1, kb & 1};
    const int v0 = su[op.P[0]], v1 = su[op.P[1]], v2 = su[op.P[2]], v3 = su[op.P[3]];
    return op.cons == 0 ? v0 + v1 == v2 + v3 : v0 + v3 == v1 + v2;
}

// Spin-block problems of GEMM g: for each output block (rb, cb) the K blocks allowed by both
// operands, with a K order that makes every such set contiguous.
static int ny_plan_gemm(NyWork* y, int g) {
    int mask[4][4];
    for (int rb = 0; rb < 4; ++rb)
        for (int cb = 0; cb < 4; ++cb) {
            mask[rb][cb] = 0;
            for (int kb = 0; kb < 4; ++kb)
                if (ny_allowed(k_ny_ops[g][0], rb, kb) && ny_allowed(k_ny_ops[g][1], cb, kb)) mask[rb][cb] |= 1 << kb;
        }
    int order[4] = {0, 1, 2, 3};
    for (int trial = 0; trial < 24; ++trial) {
        // trial-th permutation (Lehmer code)
        int pool[4] = {0, 1, 2, 3}, np_ = 4, code = trial;
        for (int q = 0; q < 4; ++q) {
            const int f = q == 0 ? 6 : q == 1 ? 2 : 1;
            const int pick = q < 3 ? code / f : 0;
            if (q < 3) code %= f;
            order[q] = pool[pick];
            for (int m = pick; m < np_ - 1; ++m) pool[m] = pool[m + 1];
            --np_;
        }
        int pos[4];
        for (int q = 0; q < 4; ++q) pos[order[q]] = q;
        bool ok = true;
        int np = 0;
        for (int rb = 0; rb < 4 && ok; ++rb)
            for (int cb = 0; cb < 4 && ok; ++cb) {
                const int m = mask[rb][cb];
                if (!m) continue;
                int lo = 4, hi = -1, cnt = 0;
                for (int kb = 0; kb < 4; ++kb)
                    if (m >> kb & 1) {
                        lo = pos[kb] < lo ? pos[kb] : lo;
                        hi = pos[kb] > hi ? pos[kb] : hi;
                        ++cnt;
                    }
                if (hi - lo + 1 != cnt) ok = false;
                else {
                    y->prob[g][np][0] = rb;
                    y->prob[g][np][1] = cb;
                    y->prob[g][np][2] = lo;
                    y->prob[g][np][3] = cnt;
                    ++np;
                }
            }
        if (ok) {
            for (int q = 0; q < 4; ++q) y->korder[g][q] = order[q];
            y->nprob[g] = np;
            return ACSE_OK;
        }
    }
    return ACSE_ERR_UNSUPPORTED;
}

int ny_alloc(acse_ctx* c) {
    NyWork* y = (NyWork*)calloc(1, sizeof(NyWork));
    if (!y) return ACSE_ERR_NOMEM;
    c->ny = y;
    const int r = c->r, n = 2 * r, R2 = r * r;
    y->n = n;
    y->n2 = (size_t)n * n;
    y->n4 = y->n2 * y->n2;
    const size_t r4 = (size_t)R2 * R2;
    const bool f64 = c->opt.prec == ACSE_FP64;
    const size_t es = f64 ? 8 : 4;                                  // GEMM output / T element
    for (int g = 0; g < 6; ++g) ACSE_TRY(ny_plan_gemm(y, g));
    for (int b = 0; b < 3; ++b) ACSE_TRY(ny_malloc((void**)&y->delta[b], r4 * sizeof(double)));
    ACSE_TRY(ny_malloc((void**)&y->sig, n * sizeof(double)));
    size_t op_bytes;
    if (f64) {
        y->Kb = R2;
        y->Kbw = R2;
        op_bytes = y->n4 * sizeof(double);
    } else {
        const int ops = c->opt.prec == ACSE_BF16X3 ? 2 : 4;         // operand element bytes
        const int kb = 128 / ops;
        y->Kb = (R2 + kb - 1) / kb * kb;
        y->Kbw = c->nsplit * y->Kb;
        op_bytes = y->n2 * (size_t)4 * y->Kbw * ops;
    }
    for (int s = 0; s < 3; ++s) {
        ACSE_TRY(ny_malloc(&y->opA[s], op_bytes));
        ACSE_TRY(ny_malloc(&y->opB[s], op_bytes));
        if (!f64) {   // K padding is never written afterwards
            ACSE_CUDA_TRY(cudaMemset(y->opA[s], 0, op_bytes));
            ACSE_CUDA_TRY(cudaMemset(y->opB[s], 0, op_bytes));
        }
    }
    for (int o = 0; o < 6; ++o) {   // blocks that no problem writes stay zero
        ACSE_TRY(ny_malloc(&y->out[o], y->n4 * es));
        ACSE_CUDA_TRY(cudaMemset(y->out[o], 0, y->n4 * es));
    }
    ACSE_TRY(ny_malloc(&y->Q, y->n2 * es));
    for (int t = 0; t < 4; ++t) ACSE_TRY(ny_malloc(&y->tny[t], r4 * es));
    k_ny_sigma<<<(n + 127) / 128, 128, 0, c->stream>>>(r, c->opt.n_alpha, c->opt.n_beta, y->sig);
    ACSE_LAUNCHED(c);
    if (!f64) {
        const int kind = (c->opt.prec == ACSE_TF32 || c->opt.prec == ACSE_TF32X3) ? 1 : 0;
        const int ops = kind == 0 ? 2 : 4;
        const size_t ld = (size_t)4 * y->Kbw;
        for (int s = 0; s < 2; ++s) {
            ACSE_TRY(tc_table_init_mode(&y->st[s], kind, tc_default_bn(r), tc_use_pairs(c)));
            for (int g = 3 * s; g < 3 * s + 3; ++g)
                for (int k = 0; k < y->nprob[g]; ++k) {
                    const int rb = y->prob[g][k][0], cb = y->prob[g][k][1], q0 = y->prob[g][k][2], cnt = y->prob[g][k][3];
                    const char* A = (const char*)y->opA[g % 3] + ((size_t)rb * R2 * ld + (size_t)q0 * y->Kbw) * ops;
                    const char* B = (const char*)y->opB[g % 3] + ((size_t)cb * R2 * ld + (size_t)q0 * y->Kbw) * ops;
                    float* C = (float*)y->out[g] + (size_t)rb * R2 * y->n2 + (size_t)cb * R2;
                    ACSE_TRY(tc_table_add_ld(&y->st[s], A, ld, B, ld, C, R2, R2, cnt * y->Kbw, (int)y->n2, 1.0f));
                }
            tc_table_set_err(&y->st[s], c->w.tc_err);
            ACSE_TRY(tc_table_upload(&y->st[s]));
        }
    }
    return ACSE_OK;
}

static NyPack ny_pk(NyWork* y, int g, int side, const double* const Dl[3], const double* const W[3], void* dst,
                    size_t ld) {
    const NyOp& op = k_ny_ops[g][side];
    NyPack k;
    const double* const* blk = op.src == 0 ? Dl : op.src == 1 ? W : nullptr;
    for (int b = 0; b < 3; ++b) k.blk[b] = blk ? blk[b] : nullptr;
    k.dense = op.src >= 2 ? y->out[op.src - 2] : nullptr;
    for (int q = 0; q < 4; ++q) {
        k.P[q] = op.P[q];
        k.korder[q] = y->korder[g][q];
    }
    for (int b = 0; b < 4; ++b) k.need[b] = 0;
    for (int p = 0; p < y->nprob[g]; ++p) {   // row block of this operand -> K blocks its problems read
        const int rowb = y->prob[g][p][side];
        for (int q = y->prob[g][p][2]; q < y->prob[g][p][2] + y->prob[g][p][3]; ++q) k.need[rowb] |= 1 << y->korder[g][q];
    }
    k.use_sigma = op.sigma;
    k.sig = y->sig;
    k.dst = dst;
    k.ld = ld;
    k.Kb = y->Kb;
    k.Kbw = y->Kbw;
    return k;
}

// The NY term T for the pass in flight (D = c->cur_D, W = c->cur_W, 1D in c->w.gam), left in the
// four spin-type buffers the B kernel adds to B.
int ny_pass(acse_ctx* c) {
    NyWork* y = (NyWork*)c->ny;
    if (!y) return ACSE_ERR_UNSUPPORTED;
    const int r = c->r, R2 = r * r;
    const bool f64 = c->opt.prec == ACSE_FP64;
    k_ny_delta<<<152 * 8, 256, 0, c->stream>>>(r, c->w.gam, c->cur_D[0], c->cur_D[1], c->cur_D[2], y->delta[0],
                                               y->delta[1], y->delta[2]);
    ACSE_LAUNCHED(c);
    const double* Dl[3] = {y->delta[0], y->delta[1], y->delta[2]};
    const double* W[3] = {c->cur_W[0], c->cur_W[1], c->cur_W[2]};
    const size_t ld = (size_t)4 * y->Kbw;
    for (int s = 0; s < 2; ++s) {
        for (int g = 3 * s; g < 3 * s + 3; ++g) {
            ACSE_TRY(ny_pack_launch(c, ny_pk(y, g, 0, Dl, W, y->opA[g % 3], ld), 0));
            ACSE_TRY(ny_pack_launch(c, ny_pk(y, g, 1, Dl, W, y->opB[g % 3], ld), 1));
        }
        if (f64) {
            GemmF64 gl[48];
            int ng = 0;
            for (int g = 3 * s; g < 3 * s + 3; ++g)
                for (int k = 0; k < y->nprob[g]; ++k) {
                    const int rb = y->prob[g][k][0], cb = y->prob[g][k][1], q0 = y->prob[g][k][2], cnt = y->prob[g][k][3];
                    const double* A = (const double*)y->opA[g % 3] + (size_t)rb * R2 * ld + (size_t)q0 * R2;
                    const double* B = (const double*)y->opB[g % 3] + (size_t)cb * R2 * ld + (size_t)q0 * R2;
                    double* C = (double*)y->out[g] + (size_t)rb * R2 * y->n2 + (size_t)cb * R2;
                    gl[ng++] = GemmF64{A, B, C, R2, R2, cnt * R2, (int)ld, (int)ld, (int)y->n2, 1.0, 0.0, 0, 0, 0};
                }
            ACSE_TRY(gemm_f64_grouped(c, gl, ng, c->stream));
        } else {
            ACSE_TRY(tc_table_launch(&y->st[s], c->stream));
            c->launches++;
        }
    }
    const int n = y->n;
    const size_t smem = 2 * (size_t)n * r * (f64 ? sizeof(double) : sizeof(float));
    if (f64) {
        k_ny_Q<double><<<(n * n + 7) / 8, 256, 0, c->stream>>>(r, (const double*)y->out[0], (double*)y->Q);
        ACSE_LAUNCHED(c);
        k_ny_assemble<double><<<4 * R2, 256, smem, c->stream>>>(
            r, (const double*)y->out[3], (const double*)y->out[4], (const double*)y->out[5], (const double*)y->Q, Dl[0],
            Dl[1], Dl[2], y->sig, (double*)y->tny[0], (double*)y->tny[1], (double*)y->tny[2], (double*)y->tny[3]);
    } else {
        k_ny_Q<float><<<(n * n + 7) / 8, 256, 0, c->stream>>>(r, (const float*)y->out[0], (float*)y->Q);
        ACSE_LAUNCHED(c);
        k_ny_assemble<float><<<4 * R2, 256, smem, c->stream>>>(
            r, (const float*)y->out[3], (const float*)y->out[4], (const float*)y->out[5], (const float*)y->Q, Dl[0],
            Dl[1], Dl[2], y->sig, (float*)y->tny[0], (float*)y->tny[1], (float*)y->tny[2], (float*)y->tny[3]);
    }
    ACSE_LAUNCHED(c);
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
