// FP64-accurate GEMMs of the contraction pass on the BF16 tensor cores by the Ozaki scheme
// (error-free splitting: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, Numer. Algorithms 59 (2012)).
//
// C = alpha A B^T with A (M x K) and B (N x K) FP64, both K-major.  Each operand row is scaled by a
// power of two 2^e chosen so that |a| 2^-e < 1/2 over the row, and cut into S signed digits of base
// 2^6:  x_1 = a 2^-e,  d_s = rint(2^6 x_s),  x_{s+1} = 2^6 x_s - d_s,  so that
//     a = 2^e (sum_{s=1..S} d_s 2^-6s + x_{S+1} 2^-6S),   |d_s| <= 32,  |x_{S+1}| <= 1/2,
// every step exact in FP64 and every digit exact in bf16.  Then
//     A B^T = 2^(ea + eb) sum_{s,t} 2^-6(s+t) D_s E_t^T,
// of which the levels L = s + t <= S + 1 are kept (the rest is below 2^-6(S+1) relative).  A product
// of digit matrices is an integer matrix with entries of at most K 32^2; g products of one level
// summed in one FP32 accumulator stay exact while g K 2^10 < 2^24, so each level is run as
// ceil((L-1)/g) such groups, and the groups are added in FP64.
//
// Operand layout: slice s of an A row at K segment s-1, slice t of a B row at K segment S-t
// (reversed), each segment Kp = K rounded up to 64 elements (zero padded).  The products (s, L-s),
// s0 <= s <= s1, of level L are then one contiguous K range of A, [(s0-1) Kp, s1 Kp), against one
// of B, [(S-L+s0) Kp, (S-L+s1+1) Kp): a single UMMA accumulation of (s1-s0+1) Kp.
//
// Kernels: the persistent tcgen05 GEMM of gemm_tc.cu with the accumulation unit changed from a tile
// to a (tile, group): the MMA thread runs the groups of a tile one after another into the two TMEM
// buffers, and the epilogue warps store each group's exact integer sum (int32) to a staging array.
// A second, HBM-bound kernel adds the groups of every element exactly in int64 and writes the FP64
// result with one rounding.  (Adding the groups into the FP64 output from the epilogue instead, a
// read-modify-write of the tile per group, measured eight times slower.)  Every wait is bounded as
// in gemm_tc.cu.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include "acse_internal.h"
#include "oz_arith.cuh"
#include "tc_ptx.cuh"

#define OZ_BETA 6            // bits per digit (base 2^6, |digit| <= 32)
#define OZ_MAXP 12           // GEMMs of one launch
#define OZ_MAXJ 16           // operands of one slicing launch
#define OZ_THREADS 192
#define OZ_BN 256
#define OZ_STAGES 4
#define OZ2_STAGES 6         // ring depth of the CTA-pair form (32 KB a stage per CTA)
#define OZ_DRAIN_NS 2000000000ull
#define OZ_WAIT_NS 4000000000ull
#define OZ_SLICE_PPT 8       // element pairs per thread of a sliced row: K <= 2 * 512 * 8 = 2 * 64^2 with
                             // 512 threads; rows with K <= 2048 / 4096 take 128 / 256 threads

struct OzProb {
    double* C;
    int* stage;         // [ngroups][M][N]: the exact integer sum of each group
    const double* sa;   // 2^ea per row of A
    const double* sb;   // 2^eb per row of B
    double alpha;
    int ealpha;         // alpha = 2^ealpha
    int M, N, ldc;
    int kbs;            // 64-element K blocks per slice segment
    int g;              // slice products per exactly accumulated group
    int ngroups;
    int tiles_n, tile_start;
    int accum;          // 1: C += result (one FP64 addition), 0: C = result
};

struct __align__(128) OzBatch {
    CUtensorMap tmA[OZ_MAXP];
    CUtensorMap tmB[OZ_MAXP];
    OzProb p[OZ_MAXP];
    int nprob;
    int total_tiles;
    int S;
    int* err;
    unsigned long long wait_ns;
    int inject_stall;
    const int* order;     // tiles of CTA c: order[cta_start[c] .. cta_start[c+1]) (longest first)
    const int* cta_start;
};

__host__ __device__ inline int oz_ngroups(int S, int g) {
    int n = 0;
    for (int L = 2; L <= S + 1; ++L) n += (L - 2) / g + 1;   // ceil((L - 1) / g)
    return n;
}

// group index -> level L and the A slices [s0, s1] of its products (s, L - s)
__device__ __forceinline__ void oz_group(int S, int g, int idx, int& L, int& s0, int& s1) {
    for (L = 2; L <= S + 1; ++L) {
        const int n = (L - 2) / g + 1;
        if (idx < n) {
            s0 = 1 + idx * g;
            s1 = min(L - 1, s0 + g - 1);
            return;
        }
        idx -= n;
    }
    L = S + 1;
    s0 = s1 = 1;
}

__device__ __forceinline__ int oz_find_problem(const OzBatch& b, int t) {
    int lo = 0, hi = b.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.p[mid].tile_start <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------------ slicing
struct OzSliceJob {
    const double* src;
    size_t lds;             // source row stride (elements)
    const int* rowmap;      // source row of each output row (null: the same row)
    const int* colmap;      // source column of each K index (null: the same column)
    __nv_bfloat16* dst;     // first output row of the job
    size_t ldd;             // S * Kp
    double* scale;          // 2^e per output row (NaN for a row with a non-finite entry)
    int rows, K, Kp, reverse, row0;
};

struct OzSliceBatch {
    OzSliceJob j[OZ_MAXJ];
    int njobs;
    int S;
};

// One block per operand row.  The row's bit patterns are held in registers, its largest magnitude
// fixes e (|a| 2^-e < 1/2), and every element's fixed-point value X is cut into S balanced base-64
// digits from the least significant one up (d = ((X + 32) mod 64) - 32, X <- (X - d) / 64, exact;
// the last quotient is the leading digit, of magnitude at most 32).  Digits go out as bf16 pairs,
// each slice to its K segment of the row.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_oz_slice(const __grid_constant__ OzSliceBatch b) {
    __shared__ unsigned long long red[THREADS / 32];
    __shared__ unsigned short tab[65];   // bf16 bits of the digits -32..32
    if (threadIdx.x < 65) tab[threadIdx.x] = __bfloat16_as_ushort(__float2bfloat16_rn((float)((int)threadIdx.x - 32)));
    int ji = 0;
    while (ji + 1 < b.njobs && b.j[ji + 1].row0 <= (int)blockIdx.x) ++ji;
    const OzSliceJob& J = b.j[ji];
    const int row = (int)blockIdx.x - J.row0;
    const int srow = J.rowmap ? J.rowmap[row] : row;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(J.src + (size_t)srow * J.lds);
    const int K = J.K;
    const int* cm = J.colmap;
    unsigned long long v[2 * OZ_SLICE_PPT];
    unsigned long long mx = 0;
#pragma unroll
    for (int u = 0; u < OZ_SLICE_PPT; ++u) {
        const int k = 2 * ((int)threadIdx.x + u * THREADS);
        v[2 * u] = k < K ? src[cm ? cm[k] : k] : 0ull;
        v[2 * u + 1] = k + 1 < K ? src[cm ? cm[k + 1] : k + 1] : 0ull;
        mx = max(mx, max(v[2 * u] & 0x7FFFFFFFFFFFFFFFull, v[2 * u + 1] & 0x7FFFFFFFFFFFFFFFull));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[w] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int i = 1; i < THREADS / 32; ++i) mx = max(mx, red[i]);
    // non-negative doubles order like their bit patterns; an all-ones exponent is Inf or NaN
    const bool bad = mx >= 0x7FF0000000000000ull;
    int e = 0;
    if (!bad && mx != 0) e = min(1000, max(-1000, (int)(mx >> 52) - 1023 + 2));
    if (threadIdx.x == 0) J.scale[row] = bad ? __longlong_as_double(0x7ff8000000000000ll) : oz_pow2(e);
    __nv_bfloat16* drow = J.dst + (size_t)row * J.ldd;
    const int S = b.S;
#pragma unroll
    for (int u = 0; u < OZ_SLICE_PPT; ++u) {
        const int k = 2 * ((int)threadIdx.x + u * THREADS);
        if (k >= K) continue;
        long long X0 = bad ? 0 : oz_fixed(v[2 * u], S, e);
        long long X1 = bad ? 0 : oz_fixed(v[2 * u + 1], S, e);
        for (int t = 0; t < S; ++t) {   // slice s = S - t
            int d0, d1;
            if (t < S - 1) {
                d0 = (int)(((X0 + 32) & 63) - 32);
                d1 = (int)(((X1 + 32) & 63) - 32);
                X0 = (X0 - d0) >> 6;
                X1 = (X1 - d1) >> 6;
            } else {
                d0 = (int)X0;
                d1 = (int)X1;
            }
            const int sl = S - t;
            const int seg = J.reverse ? S - sl : sl - 1;
            __nv_bfloat16* dst = drow + (size_t)seg * J.Kp + k;
            if (k + 1 < K)
                *reinterpret_cast<unsigned int*>(dst) = (unsigned int)tab[d0 + 32] | ((unsigned int)tab[d1 + 32] << 16);
            else
                *reinterpret_cast<unsigned short*>(dst) = tab[d0 + 32];
        }
    }
}

// ------------------------------------------------------------------------------- GEMM
// PAIR: the CTA-pair form of gemm_tc.cu (launched in clusters of two CTAs; pair MMA of M = 256 on
// 256 x BN tiles, each CTA loading its 128 rows of A and BN / 2 rows of B; the even CTA issues the MMAs
// and commits to the barriers of both; both CTAs' loads complete on the even CTA's full[s]; both
// CTAs' epilogue warps arrive on the even CTA's acce[ab]).
template <int BN, int STAGES, bool PAIR>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_gemm_oz(const OzBatch* __restrict__ bp) {
    const OzBatch& b = *bp;
    constexpr int A_BYTES = TC_BM * 128;
    constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * 128;
    constexpr int BM = PAIR ? 2 * TC_BM : TC_BM;   // rows of an output tile
    constexpr int KELEM = 64;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;   // [2]
    uint64_t* acce = accf + 2;         // [2]
    uint64_t* never = acce + 2;
    uint64_t* drainb = never + 1;
    uint32_t* tmem_slot = (uint32_t*)(drainb + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = b.S;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;   // CTA, or CTA pair
    const int q0 = b.cta_start[unit], q1 = b.cta_start[unit + 1];        // this unit's tiles
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], PAIR ? 8 : 4);
        }
        mbar_init(never, 1);
        mbar_init(drainb, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        if constexpr (PAIR) tmem_alloc_pair(tmem_slot, 2 * BN);
        else tmem_alloc(tmem_slot, 2 * BN);
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all();
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t full0 = PAIR ? mapa_rank(smem_u32(full), 0) : 0u;   // the even CTA's full[0]
            int it = 0;
            bool stop = false;
            for (int qi = q0; qi < q1 && !stop; ++qi) {
                const int t = b.order[qi];
                const int pi = oz_find_problem(b, t);
                const OzProb& P = b.p[pi];
                const int local = t - P.tile_start;
                const int m0 = (local / P.tiles_n) * BM + (int)rank * TC_BM;
                const int n0 = (local % P.tiles_n) * BN + (int)rank * (BN / 2);
                for (int gi = 0; gi < P.ngroups && !stop; ++gi) {
                    int L, s0, s1;
                    oz_group(S, P.g, gi, L, s0, s1);
                    const int ka = (s0 - 1) * P.kbs, kb0 = (S - L + s0) * P.kbs, n = (s1 - s0 + 1) * P.kbs;
                    for (int kb = 0; kb < n; ++kb, ++it) {
                        const int s = it % STAGES;
                        if (it >= STAGES && !bounded_wait(&empty[s], ((it / STAGES) & 1) ^ 1, b.wait_ns, abort_flag)) {
                            raise_abort(b.err, abort_flag);
                            stop = true;
                            break;
                        }
                        if constexpr (PAIR) {
                            if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * (A_BYTES + B_BYTES));
                            tma_load_2d_pair(sA + s * A_BYTES, &b.tmA[pi], (ka + kb) * KELEM, m0, full0 + 8u * s);
                            tma_load_2d_pair(sB + s * B_BYTES, &b.tmB[pi], (kb0 + kb) * KELEM, n0, full0 + 8u * s);
                        } else {
                            mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                            tma_load_2d(sA + s * A_BYTES, &b.tmA[pi], (ka + kb) * KELEM, m0, &full[s]);
                            tma_load_2d(sB + s * B_BYTES, &b.tmB[pi], (kb0 + kb) * KELEM, n0, &full[s]);
                        }
                    }
                }
            }
            // every issued copy must have landed before the CTA may exit (with pairs: the even CTA's
            // full[s] counts both CTAs' bytes; the odd CTA also waits for the MMAs that read its last
            // stages, briefly after an abort)
            for (int k = it > STAGES ? it - STAGES : 0; k < it; ++k) {
                const unsigned long long lim = *abort_flag ? b.wait_ns : OZ_DRAIN_NS;
                const bool ok = rank == 0 ? bounded_wait(&full[k % STAGES], (k / STAGES) & 1, lim, nullptr)
                                          : bounded_wait(&empty[k % STAGES], (k / STAGES) & 1, lim, nullptr);
                if (!ok) {
                    raise_abort(b.err, abort_flag);
                    if (rank != 0) break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            const uint32_t idesc = PAIR ? make_idesc_pair<0, BN>() : make_idesc<0, BN>();
            if (b.inject_stall && !bounded_wait(never, 0, b.wait_ns, abort_flag)) raise_abort(b.err, abort_flag);
            int it = 0, lt = 0;
            for (int qi = q0; qi < q1 && !*abort_flag; ++qi) {
                const OzProb& P = b.p[oz_find_problem(b, b.order[qi])];
                for (int gi = 0; gi < P.ngroups && !*abort_flag; ++gi, ++lt) {
                    int L, s0, s1;
                    oz_group(S, P.g, gi, L, s0, s1);
                    const int n = (s1 - s0 + 1) * P.kbs;
                    const int ab = lt & 1, use = lt >> 1;
                    if (use >= 1) {
                        const bool ok = PAIR ? bounded_wait_cluster(&acce[ab], (use - 1) & 1, b.wait_ns + OZ_DRAIN_NS, abort_flag)
                                             : bounded_wait(&acce[ab], (use - 1) & 1, b.wait_ns + OZ_DRAIN_NS, abort_flag);
                        if (!ok) {
                            raise_abort(b.err, abort_flag);
                            break;
                        }
                    }
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(ab * BN);
                    for (int kb = 0; kb < n; ++kb, ++it) {
                        const int s = it % STAGES;
                        if (!bounded_wait(&full[s], (it / STAGES) & 1, b.wait_ns, abort_flag)) {
                            raise_abort(b.err, abort_flag);
                            break;
                        }
                        tc_fence_after();
                        const uint64_t da = smem_desc(sA + s * A_BYTES);
                        const uint64_t db = smem_desc(sB + s * B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if constexpr (PAIR) umma_pair<0>(acc, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                            else umma<0>(acc, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                        }
                        if constexpr (PAIR) umma_commit_pair(&empty[s]);
                        else umma_commit(&empty[s]);
                    }
                    // the epilogue of this group may start when its MMAs are done
                    if constexpr (PAIR) umma_commit_pair(&accf[ab]);
                    else umma_commit(&accf[ab]);
                }
            }
            if constexpr (PAIR) umma_commit_pair(drainb);
            else umma_commit(drainb);
        }
        // no MMA is in flight past this point (bounded; with pairs in both CTAs)
        if (lane == 0 && (PAIR || rank == 0) && !bounded_wait(drainb, 0, b.wait_ns + 2 * OZ_DRAIN_NS, nullptr))
            raise_abort(b.err, abort_flag);
    } else {
        const int q = warp & 3;   // TMEM lane quadrant this warp may access
        const uint32_t acce0 = PAIR ? mapa_rank(smem_u32(acce), 0) : 0u;
        int lt = 0;
        bool run = true;
        for (int qi = q0; qi < q1 && run; ++qi) {
            const int t = b.order[qi];
            const OzProb& P = b.p[oz_find_problem(b, t)];
            const int local = t - P.tile_start;
            const int m0 = (local / P.tiles_n) * BM + (int)rank * TC_BM, n0 = (local % P.tiles_n) * BN;
            const int row = m0 + q * 32 + lane;
            const bool rok = row < P.M;
            const bool vec = (P.N & 3) == 0 && (reinterpret_cast<uintptr_t>(P.stage) & 15) == 0;
            for (int gi = 0; gi < P.ngroups; ++gi, ++lt) {
                const int ab = lt & 1, use = lt >> 1;
                int go = 0;
                if (lane == 0) {
                    const bool ok = bounded_wait(&accf[ab], use & 1, b.wait_ns + OZ_DRAIN_NS, abort_flag);
                    if (!ok) raise_abort(b.err, abort_flag);
                    go = ok && !*abort_flag;
                }
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) {
                    run = false;
                    break;
                }
                tc_fence_after();
                // the group's sum is an integer below 2^24 in magnitude: exact in FP32 and in int32
                int* srow = P.stage + (size_t)gi * P.M * P.N + (size_t)(rok ? row : 0) * P.N;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t v[32];
                    __syncwarp();
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + c * 32), v);   // warp-collective
                    const int col0 = n0 + c * 32;
                    if (!rok || col0 >= P.N) continue;
                    if (vec && col0 + 32 <= P.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<int4*>(srow + col0 + j) =
                                make_int4(__float2int_rn(__uint_as_float(v[j])), __float2int_rn(__uint_as_float(v[j + 1])),
                                          __float2int_rn(__uint_as_float(v[j + 2])), __float2int_rn(__uint_as_float(v[j + 3])));
                    } else {
                        const int nc = min(32, P.N - col0);
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nc) srow[col0 + j] = __float2int_rn(__uint_as_float(v[j]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {   // this warp's quarter of the buffer is free
                    if constexpr (PAIR) mbar_arrive_cluster(acce0 + 8u * ab);
                    else mbar_arrive(&acce[ab]);
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all();   // neither CTA exits while the other may still signal it
    else __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc_pair(tmem, 2 * BN);
        else tmem_dealloc(tmem, 2 * BN);
    }
}

// C = alpha 2^(ea_i + eb_j) sum_g 2^-6L_g v_g for every element, from the staged group sums v_g.
// With w_L = 36 - 6 (L - 2) the terms v_g 2^w_L (an arithmetic right shift where w_L < 0, which drops
// only bits below 2^-48 of the level-2 unit) are added in int64 (|sum| < 2^61), and the conversion of
// the sum, scaled by the power of two alpha 2^(ea + eb - 48), to FP64 is the single rounding.
// HBM-bound: the groups of an element are read once, coalesced, and C is written once.
__device__ __forceinline__ long long oz_term(int v, int w) {
    return w >= 0 ? (long long)v * (1ll << w) : ((long long)v >> -w);   // arithmetic shift: floor
}

__global__ void __launch_bounds__(256) k_oz_reduce(const OzBatch* __restrict__ bp) {
    __shared__ signed char wtab[64];   // the weight 36 - 6 (L - 2) of every group, in the staging order
    const OzBatch& b = *bp;
    const OzProb& P = b.p[blockIdx.y];
    const int N = P.N, g = P.g, S = b.S, ng = P.ngroups;
    if (threadIdx.x == 0) {
        int gi = 0;
        for (int L = 2; L <= S + 1; ++L)
            for (int q = 0; q < (L - 2) / g + 1 && gi < 64; ++q) wtab[gi++] = (signed char)(36 - OZ_BETA * (L - 2));
    }
    __syncthreads();
    const size_t MN = (size_t)P.M * N;
    const int* __restrict__ st = P.stage;
    // four consecutive elements of one row per thread (int4 loads) when N % 4 == 0, else one; the group
    // sums are loaded eight at a time before they are added
    const int vw = (N & 3) == 0 ? 4 : 1;
    const size_t nunit = MN / vw;
    for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunit; u += (size_t)gridDim.x * blockDim.x) {
        const size_t e = u * vw;
        long long acc[4] = {0, 0, 0, 0};
        for (int g0 = 0; g0 < ng; g0 += 8) {
            if (vw == 4) {
                int4 vv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (g0 + q < ng) vv[q] = *reinterpret_cast<const int4*>(st + e + (size_t)(g0 + q) * MN);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (g0 + q < ng) {
                        const int w = wtab[g0 + q];
                        acc[0] += oz_term(vv[q].x, w);
                        acc[1] += oz_term(vv[q].y, w);
                        acc[2] += oz_term(vv[q].z, w);
                        acc[3] += oz_term(vv[q].w, w);
                    }
            } else {
                int vv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (g0 + q < ng) vv[q] = st[e + (size_t)(g0 + q) * MN];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (g0 + q < ng) acc[0] += oz_term(vv[q], wtab[g0 + q]);
            }
        }
        const int i = (int)(e / N), j0 = (int)(e - (size_t)i * N);
        const int ea = (int)((__double_as_longlong(P.sa[i]) >> 52) & 0x7FF);   // row scales are powers of two
        double* crow = P.C + (size_t)i * P.ldc;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < vw) {
                const int eb = (int)((__double_as_longlong(P.sb[j0 + k]) >> 52) & 0x7FF);
                const double v = (ea == 0x7FF || eb == 0x7FF) ? __longlong_as_double(0x7ff8000000000000ll)
                                                               : oz_ll_scaled(acc[k], ea + eb - 2046 + P.ealpha - 48);
                crow[j0 + k] = P.accum ? crow[j0 + k] + v : v;
            }
        }
    }
}

// Same-spin pair GEMMs on packed pairs (as on the split path): in the aa and bb sectors the rows (ij),
// the columns (kp) and the contraction (rs) of [M; D] W^T are antisymmetric pairs, so those GEMMs run
// on pairs i < j only (P = r(r-1)/2; alpha 2 for the halved (rs) sum) and k_oz_unpack rebuilds the
// full X and Y rows by antisymmetry.  pk(a, b), a < b, numbers the pairs row by row.
__host__ __device__ __forceinline__ int oz_pk(int r, int a, int b) { return a * r - a * (a + 1) / 2 + (b - a - 1); }

// X_s, Y_s (s = aa, bb; r^2 x r^2 FP64) from the packed [X; Y] (2P x P): one block per output row, the
// packed source row staged in shared memory, the full row written two columns at a time.
__global__ void __launch_bounds__(256) k_oz_unpack(int r, const double* __restrict__ Cp0, const double* __restrict__ Cp2,
                                                   double* X0, double* Y0, double* X2, double* Y2) {
    __shared__ double srow[ACSE_MAX_R * (ACSE_MAX_R - 1) / 2];
    const int R2 = r * r, P = r * (r - 1) / 2;
    const int sec = blockIdx.x / (2 * R2);
    const int row = blockIdx.x - sec * 2 * R2;
    const int part = row / R2, ij = row - part * R2, i = ij / r, j = ij - i * r;
    double* dst = (sec == 0 ? (part ? Y0 : X0) : (part ? Y2 : X2)) + (size_t)ij * R2;
    if (i == j) {   // block-uniform
        for (int c = threadIdx.x; c < R2; c += blockDim.x) dst[c] = 0.0;
        return;
    }
    const double si = i < j ? 1.0 : -1.0;
    const double* src = (sec == 0 ? Cp0 : Cp2) + (size_t)(part * P + (i < j ? oz_pk(r, i, j) : oz_pk(r, j, i))) * P;
    for (int e = threadIdx.x; e < P; e += blockDim.x) srow[e] = si * src[e];
    __syncthreads();
    auto val = [&](int k, int q) { return k == q ? 0.0 : (k < q ? srow[oz_pk(r, k, q)] : -srow[oz_pk(r, q, k)]); };
    if ((R2 & 1) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        for (int g = threadIdx.x; g < R2 / 2; g += blockDim.x) {
            int k = (2 * g) / r, q = 2 * g - k * r;
            const double v0 = val(k, q);
            if (++q == r) { q = 0; ++k; }
            reinterpret_cast<double2*>(dst)[g] = make_double2(v0, val(k, q));
        }
    } else {
        for (int c = threadIdx.x; c < R2; c += blockDim.x) dst[c] = val(c / r, c - (c / r) * r);
    }
}

// --------------------------------------------------------------------------- host plan
// Operands of the GEMMs of a pass (the products of acse_gemm_list_f64, the same-spin ones packed):
//   A: [M_aa; D_aa] packed (2P x P), M_ab, D_ab (r^2 x r^2), [M_bb; D_bb] packed, Zd (2r^2 x 2r^2),
//      Zf1, Zf2 (r^2 x r^2);
//   B: W_aa packed (P x P), W_ab (r^2 x r^2), W_bb packed, Md (2r^2 x 2r^2), Mf1, Mf2 (r^2 x r^2).
struct OzOp {
    __nv_bfloat16* sl;
    double* scale;
    int rows, K, Kp;
};

struct OzPlan {
    OzBatch* host;
    OzBatch* dev;
    int S, bn;
    int pair;           // 1: CTA-pair kernel (256 x 256 tiles on clusters of two CTAs)
    int bm;             // rows of a tile: 128, or 256 with pairs
    int nclusters;      // co-resident CTA pairs (the persistent grid of the pair kernel)
    size_t smem;
    int nsm;
    int tiles;
    OzOp A[OZ_MAXP], B[OZ_MAXP];
    int* pmap;          // pair index -> i r + j (i < j), P entries
    double* Cp[2];      // packed [X; Y] of the aa and bb sectors (2P x P)
    int* sched;         // tile lists of the persistent kernel (OzBatch::order, cta_start)
    int* err;
    // GEMM lists of the adjoint (oz_gemm_list): a plan per list slot, and the column maps of the
    // transposed operands (K index k -> source offset k ld)
    struct OzPlan* lists[2];
    int cm_K[4], cm_ld[4];
    int* cm[4];
};

static size_t oz_smem(int bn) { return (size_t)OZ_STAGES * (TC_BM + bn) * 128 + 1024 + 256; }
static size_t oz_smem_pair() { return (size_t)OZ2_STAGES * (TC_BM + OZ_BN / 2) * 128 + 1024 + 256; }

// Launch of the GEMM kernel of plan pl (pl->tiles > 0): one CTA per SM, or one cluster of two per pair.
static int oz_launch_gemm(const OzPlan* pl, cudaStream_t st) {
    if (pl->pair) {
        const int g = pl->tiles < pl->nclusters ? pl->tiles : pl->nclusters;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * g, 1, 1);
        cfg.blockDim = dim3(OZ_THREADS, 1, 1);
        cfg.dynamicSmemBytes = pl->smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ACSE_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gemm_oz<OZ_BN, OZ2_STAGES, true>, (const OzBatch*)pl->dev));
        return ACSE_OK;
    }
    const int g = pl->tiles < pl->nsm ? pl->tiles : pl->nsm;
    if (pl->bn == 256) k_gemm_oz<256, OZ_STAGES, false><<<g, OZ_THREADS, pl->smem, st>>>(pl->dev);
    else k_gemm_oz<128, OZ_STAGES, false><<<g, OZ_THREADS, pl->smem, st>>>(pl->dev);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

static int oz_op_alloc(OzOp& o, int rows, int K, int S) {
    o.rows = rows;
    o.K = K;
    o.Kp = (K + 63) / 64 * 64;
    const size_t bytes = (size_t)rows * S * o.Kp * sizeof(__nv_bfloat16);
    if (cudaMalloc((void**)&o.sl, bytes) != cudaSuccess || cudaMalloc((void**)&o.scale, rows * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    ACSE_CUDA_TRY(cudaMemset(o.sl, 0, bytes));   // the K padding of every segment stays zero
    return ACSE_OK;
}

static int oz_add(OzPlan* pl, const OzOp& a, const OzOp& b, double* C, int ldc, double alpha) {
    OzBatch& B = *pl->host;
    if (B.nprob >= OZ_MAXP || a.K != b.K || a.Kp != b.Kp) return ACSE_ERR_SHAPE;
    const int n = B.nprob;
    const size_t ld = (size_t)pl->S * a.Kp;
    ACSE_TRY(tc_encode_map_bf16(&B.tmA[n], a.sl, a.rows, (int)ld, TC_BM, ld));
    ACSE_TRY(tc_encode_map_bf16(&B.tmB[n], b.sl, b.rows, (int)ld, pl->pair ? pl->bn / 2 : pl->bn, ld));
    OzProb& p = B.p[n];
    p.C = C;
    p.sa = a.scale;
    p.sb = b.scale;
    p.alpha = alpha;
    int ex = 0;
    if (frexp(alpha, &ex) != 0.5) return ACSE_ERR_ARG;   // alpha must be a power of two
    p.ealpha = ex - 1;
    p.M = a.rows;
    p.N = b.rows;
    p.ldc = ldc;
    p.kbs = a.Kp / 64;
    // g K 2^(2 (OZ_BETA - 1)) < 2^24: the FP32 accumulation of a group is exact
    const long long cap = ((1ll << 24) - 1) / ((long long)a.K << (2 * (OZ_BETA - 1)));
    p.g = cap < 1 ? 1 : (int)(cap < pl->S ? cap : pl->S);
    p.ngroups = oz_ngroups(pl->S, p.g);
    if (cudaMalloc((void**)&p.stage, (size_t)p.ngroups * p.M * p.N * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        p.stage = nullptr;
        return ACSE_ERR_NOMEM;
    }
    p.tiles_n = (p.N + pl->bn - 1) / pl->bn;
    p.tile_start = B.total_tiles;
    B.total_tiles += ((p.M + pl->bm - 1) / pl->bm) * p.tiles_n;
    B.nprob = n + 1;
    return cap < 1 ? ACSE_ERR_SHAPE : ACSE_OK;
}

static int oz_plan_finish(OzPlan* pl);

// Kernel attributes, SM count and the zeroed problem table of a plan.
static int oz_plan_init(OzPlan* pl, int S, int bn, int pair) {
    pl->S = S;
    pl->bn = bn;
    pl->pair = pair && bn == OZ_BN;
    pl->bm = pl->pair ? 2 * TC_BM : TC_BM;
    pl->smem = pl->pair ? oz_smem_pair() : oz_smem(pl->bn);
    if (pl->pair)
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_gemm_oz<OZ_BN, OZ2_STAGES, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)pl->smem));
    else if (pl->bn == 256)
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_gemm_oz<256, OZ_STAGES, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)pl->smem));
    else
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_gemm_oz<128, OZ_STAGES, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)pl->smem));
    pl->nsm = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&pl->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        pl->nsm = 152;
    }
    if (pl->pair) {   // co-resident clusters of two (the persistent grid)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (pl->nsm / 2), 1, 1);
        cfg.blockDim = dim3(OZ_THREADS, 1, 1);
        cfg.dynamicSmemBytes = pl->smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (void*)k_gemm_oz<OZ_BN, OZ2_STAGES, true>, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = pl->nsm / 2;
        }
        pl->nclusters = n < pl->nsm / 2 ? n : pl->nsm / 2;
    }
    pl->host = (OzBatch*)calloc(1, sizeof(OzBatch));
    if (!pl->host) return ACSE_ERR_NOMEM;
    pl->host->S = S;
    pl->host->wait_ns = OZ_WAIT_NS;
    return ACSE_OK;
}

int oz_plan_create(acse_ctx* c) {
    OzPlan* pl = (OzPlan*)calloc(1, sizeof(OzPlan));
    if (!pl) return ACSE_ERR_NOMEM;
    c->oz_plan = pl;
    const int r = c->r, R2 = r * r, R22 = 2 * R2, P = r * (r - 1) / 2;
    ACSE_TRY(oz_plan_init(pl, c->opt.oz_slices, R2 >= 256 ? OZ_BN : 128, c->opt.gemm_tile != 1));
    // the B products on the tensor cores (acse_zoz.cu): x1 and x2^T of the four types for every pair
    if (r % 16 == 0 && r <= 64 && c->opt.oz_slices <= 8)
        for (int k = 0; k < 8; ++k)
            if (cudaMalloc((void**)&c->w.bx64[k], (size_t)R2 * R2 * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                c->w.bx64[k] = nullptr;
                return ACSE_ERR_NOMEM;
            }
    ACSE_TRY(oz_op_alloc(pl->A[0], 2 * P, P, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[1], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[2], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[3], 2 * P, P, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[4], R22, R22, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[5], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->A[6], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[0], P, P, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[1], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[2], P, P, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[3], R22, R22, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[4], R2, R2, pl->S));
    ACSE_TRY(oz_op_alloc(pl->B[5], R2, R2, pl->S));
    {
        int* hm = (int*)malloc((size_t)P * sizeof(int));
        if (!hm) return ACSE_ERR_NOMEM;
        for (int a = 0; a < r; ++a)
            for (int b = a + 1; b < r; ++b) hm[oz_pk(r, a, b)] = a * r + b;
        const bool ok = cudaMalloc((void**)&pl->pmap, (size_t)P * sizeof(int)) == cudaSuccess &&
                        cudaMemcpy(pl->pmap, hm, (size_t)P * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        free(hm);
        if (!ok) {
            cudaGetLastError();
            return ACSE_ERR_NOMEM;
        }
    }
    for (int s = 0; s < 2; ++s)
        if (cudaMalloc((void**)&pl->Cp[s], (size_t)2 * P * P * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return ACSE_ERR_NOMEM;
        }
    if (cudaMalloc((void**)&pl->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    ACSE_CUDA_TRY(cudaMemset(pl->err, 0, sizeof(int)));
    if (!c->w.tc_err) c->w.tc_err = pl->err;   // read by acse_sync_status
    pl->host->err = pl->err;
    Work& w = c->w;
    // the largest-K GEMM first, then the mixed-spin pair GEMMs (X_ab = 2 M_ab W_ab^T, Y_ab = 2 D_ab W_ab^T),
    // the spin-flip ones and the packed same-spin ones (alpha 2 for the halved (rs) sum)
    ACSE_TRY(oz_add(pl, pl->A[4], pl->B[3], w.X5d, R22, 1.0));
    ACSE_TRY(oz_add(pl, pl->A[1], pl->B[1], w.X[1], R2, 2.0));
    ACSE_TRY(oz_add(pl, pl->A[2], pl->B[1], w.Y[1], R2, 2.0));
    ACSE_TRY(oz_add(pl, pl->A[5], pl->B[4], w.X5f1, R2, 1.0));
    ACSE_TRY(oz_add(pl, pl->A[6], pl->B[5], w.X5f2, R2, 1.0));
    ACSE_TRY(oz_add(pl, pl->A[0], pl->B[0], pl->Cp[0], P, 2.0));
    ACSE_TRY(oz_add(pl, pl->A[3], pl->B[2], pl->Cp[1], P, 2.0));
    return oz_plan_finish(pl);
}

// Longest-processing-time tile lists of the persistent kernel (tile cost: its K blocks over all groups)
// and the device copy of the problem table.
static int oz_plan_finish(OzPlan* pl) {
    OzBatch& B = *pl->host;
    pl->tiles = B.total_tiles;
    if (pl->tiles > 0) {
        const int units = pl->pair ? pl->nclusters : pl->nsm;   // CTAs, or CTA pairs, of the persistent grid
        const int T = pl->tiles, G = T < units ? T : units;
        const int nprod = pl->S * (pl->S + 1) / 2;
        int* hs = (int*)malloc((size_t)(T + G + 1) * sizeof(int));
        long long* cost = (long long*)malloc((size_t)T * sizeof(long long));
        if (!hs || !cost) {
            free(hs);
            free(cost);
            return ACSE_ERR_NOMEM;
        }
        for (int p = 0; p < B.nprob; ++p) {
            const int n = ((B.p[p].M + pl->bm - 1) / pl->bm) * B.p[p].tiles_n;
            for (int k = 0; k < n; ++k) cost[B.p[p].tile_start + k] = (long long)nprod * B.p[p].kbs + 4 * B.p[p].ngroups;
        }
        tc_lpt_schedule(cost, T, G, hs, hs + T);
        const bool ok = cudaMalloc((void**)&pl->sched, (size_t)(T + G + 1) * sizeof(int)) == cudaSuccess &&
                        cudaMemcpy(pl->sched, hs, (size_t)(T + G + 1) * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        free(hs);
        free(cost);
        if (!ok) {
            cudaGetLastError();
            return ACSE_ERR_NOMEM;
        }
        B.order = pl->sched;
        B.cta_start = pl->sched + T;
    }
    if (cudaMalloc((void**)&pl->dev, sizeof(OzBatch)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    ACSE_CUDA_TRY(cudaMemcpy(pl->dev, pl->host, sizeof(OzBatch), cudaMemcpyHostToDevice));
    return ACSE_OK;
}

static void oz_plan_free(OzPlan* pl) {
    if (!pl) return;
    for (int i = 0; i < OZ_MAXP; ++i) {
        if (pl->A[i].sl) cudaFree(pl->A[i].sl);
        if (pl->A[i].scale) cudaFree(pl->A[i].scale);
        if (pl->B[i].sl) cudaFree(pl->B[i].sl);
        if (pl->B[i].scale) cudaFree(pl->B[i].scale);
    }
    if (pl->pmap) cudaFree(pl->pmap);
    if (pl->sched) cudaFree(pl->sched);
    for (int s = 0; s < 2; ++s) {
        if (pl->Cp[s]) cudaFree(pl->Cp[s]);
        oz_plan_free(pl->lists[s]);
    }
    for (int i = 0; i < 4; ++i)
        if (pl->cm[i]) cudaFree(pl->cm[i]);
    if (pl->err) cudaFree(pl->err);
    if (pl->host)
        for (int i = 0; i < pl->host->nprob; ++i)
            if (pl->host->p[i].stage) cudaFree(pl->host->p[i].stage);
    if (pl->dev) cudaFree(pl->dev);
    free(pl->host);
    free(pl);
}

void oz_plan_destroy(acse_ctx* c) {
    for (int k = 0; k < 8; ++k)
        if (c->w.bx64[k]) {
            cudaFree(c->w.bx64[k]);
            c->w.bx64[k] = nullptr;
        }
    OzPlan* pl = (OzPlan*)c->oz_plan;
    if (!pl) return;
    if (pl->err && c->w.tc_err == pl->err) c->w.tc_err = nullptr;
    oz_plan_free(pl);
    c->oz_plan = nullptr;
}

// One slicing job: `rows` rows of operand o starting at output row `orow`, read from src (row stride
// lds) through the optional row / column maps.
static void oz_job(OzSliceBatch& b, int& rows, const OzOp& o, int orow, int nrows, const double* src, size_t lds,
                   const int* rowmap, const int* colmap, int reverse) {
    OzSliceJob& j = b.j[b.njobs++];
    j.src = src;
    j.lds = lds;
    j.rowmap = rowmap;
    j.colmap = colmap;
    j.ldd = (size_t)b.S * o.Kp;
    j.dst = o.sl + (size_t)orow * j.ldd;
    j.scale = o.scale + orow;
    j.rows = nrows;
    j.K = o.K;
    j.Kp = o.Kp;
    j.reverse = reverse;
    j.row0 = rows;
    rows += nrows;
}

// Launch the slicing of every job of `all`: the jobs go to up to three launches by row length (128 threads
// a row for K <= 2048, 256 for K <= 4096, 512 above), so that short rows keep more blocks resident.
static int oz_slice_launch(acse_ctx* c, const OzSliceBatch& all) {
    for (int cls = 0; cls < 3; ++cls) {
        OzSliceBatch b;
        memset(&b, 0, sizeof(b));
        b.S = all.S;
        int rows = 0;
        for (int i = 0; i < all.njobs; ++i) {
            const int K = all.j[i].K;
            const int jc = K <= 2 * 128 * OZ_SLICE_PPT ? 0 : K <= 2 * 256 * OZ_SLICE_PPT ? 1 : 2;
            if (jc != cls) continue;
            b.j[b.njobs] = all.j[i];
            b.j[b.njobs].row0 = rows;
            rows += all.j[i].rows;
            b.njobs++;
        }
        if (b.njobs == 0) continue;
        if (cls == 0) k_oz_slice<128><<<rows, 128, 0, c->stream>>>(b);
        else if (cls == 1) k_oz_slice<256><<<rows, 256, 0, c->stream>>>(b);
        else k_oz_slice<512><<<rows, 512, 0, c->stream>>>(b);
        ACSE_LAUNCHED(c);
    }
    return ACSE_OK;
}

int oz_slice_operands(acse_ctx* c, int prep_D) {
    OzPlan* pl = (OzPlan*)c->oz_plan;
    if (!pl) return ACSE_ERR_UNSUPPORTED;
    const int r = c->r, P = r * (r - 1) / 2;
    const size_t R2 = (size_t)r * r;
    const int iR2 = (int)R2;
    Work& w = c->w;
    OzSliceBatch b;
    memset(&b, 0, sizeof(b));
    b.S = pl->S;
    int rows = 0;
    const int* pm = pl->pmap;
    // A slices in order (segment s - 1), B slices reversed (segment S - t)
    if (prep_D) {
        oz_job(b, rows, pl->A[0], 0, P, w.M[0], R2, pm, pm, 0);
        oz_job(b, rows, pl->A[0], P, P, c->cur_D[0], R2, pm, pm, 0);
        oz_job(b, rows, pl->A[1], 0, iR2, w.M[1], R2, nullptr, nullptr, 0);
        oz_job(b, rows, pl->A[2], 0, iR2, c->cur_D[1], R2, nullptr, nullptr, 0);
        oz_job(b, rows, pl->A[3], 0, P, w.M[2], R2, pm, pm, 0);
        oz_job(b, rows, pl->A[3], P, P, c->cur_D[2], R2, pm, pm, 0);
        oz_job(b, rows, pl->B[3], 0, 2 * iR2, w.Md, 2 * R2, nullptr, nullptr, 1);
        oz_job(b, rows, pl->B[4], 0, iR2, w.Mf1, R2, nullptr, nullptr, 1);
        oz_job(b, rows, pl->B[5], 0, iR2, w.Mf2, R2, nullptr, nullptr, 1);
    }
    oz_job(b, rows, pl->B[0], 0, P, c->cur_W[0], R2, pm, pm, 1);
    oz_job(b, rows, pl->B[1], 0, iR2, c->cur_W[1], R2, nullptr, nullptr, 1);
    oz_job(b, rows, pl->B[2], 0, P, c->cur_W[2], R2, pm, pm, 1);
    oz_job(b, rows, pl->A[4], 0, 2 * iR2, w.Zd, 2 * R2, nullptr, nullptr, 0);
    oz_job(b, rows, pl->A[5], 0, iR2, w.Zf1, R2, nullptr, nullptr, 0);
    oz_job(b, rows, pl->A[6], 0, iR2, w.Zf2, R2, nullptr, nullptr, 0);
    (void)rows;
    return oz_slice_launch(c, b);
}

int oz_gemm_launch(acse_ctx* c) {
    OzPlan* pl = (OzPlan*)c->oz_plan;
    if (!pl) return ACSE_ERR_UNSUPPORTED;
    if (pl->tiles == 0) return ACSE_OK;
    ACSE_TRY(prof_begin(c));
    ACSE_TRY(oz_launch_gemm(pl, c->stream));
    ACSE_LAUNCHED(c);
    k_oz_reduce<<<dim3(2 * pl->nsm, pl->host->nprob), 256, 0, c->stream>>>(pl->dev);
    ACSE_LAUNCHED(c);
    ACSE_TRY(prof_end(c));
    Work& w = c->w;
    k_oz_unpack<<<2 * 2 * c->r * c->r, 256, 0, c->stream>>>(c->r, pl->Cp[0], pl->Cp[1], w.X[0], w.Y[0], w.X[2], w.Y[2]);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

int oz_set_wait_ns(acse_ctx* c, unsigned long long ns, int inject_stall) {
    OzPlan* pl = (OzPlan*)c->oz_plan;
    if (!pl) return ACSE_ERR_UNSUPPORTED;
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    pl->host->wait_ns = ns ? ns : OZ_WAIT_NS;
    pl->host->inject_stall = inject_stall;
    ACSE_CUDA_TRY(cudaMemcpy(pl->dev, pl->host, sizeof(OzBatch), cudaMemcpyHostToDevice));
    return ACSE_OK;
}

// ------------------------------------------------------------------ GEMM lists of the adjoint
// The reverse sweep's FP64 GEMMs (acse_adjoint.cu) of an Ozaki context run through the same kernels:
// any list of up to OZ_MAXP GEMMs C (+)= alpha A B^T, alpha a power of two, beta 0 or 1, either operand
// stored transposed (GemmF64::transA / transB).  A transposed operand is sliced through a column map
// (K index k at source offset k ld, row n at offset n): its reads are strided, one 8-byte element per
// 32-byte sector, cheap next to the GEMM.  One plan per list slot, built on the first call (its slices
// and group-sum staging stay until the context is destroyed); a later call whose shapes differ from
// the slot's plan is refused (ACSE_ERR_SHAPE).

// Column map k -> k ld for K indices, cached per (K, ld).
static int oz_colmap(OzPlan* root, int K, int ld, const int** out) {
    for (int i = 0; i < 4; ++i)
        if (root->cm[i] && root->cm_K[i] == K && root->cm_ld[i] == ld) {
            *out = root->cm[i];
            return ACSE_OK;
        }
    for (int i = 0; i < 4; ++i) {
        if (root->cm[i]) continue;
        int* h = (int*)malloc((size_t)K * sizeof(int));
        if (!h) return ACSE_ERR_NOMEM;
        for (int k = 0; k < K; ++k) h[k] = k * ld;
        const bool ok = cudaMalloc((void**)&root->cm[i], (size_t)K * sizeof(int)) == cudaSuccess &&
                        cudaMemcpy(root->cm[i], h, (size_t)K * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        free(h);
        if (!ok) {
            cudaGetLastError();
            return ACSE_ERR_NOMEM;
        }
        root->cm_K[i] = K;
        root->cm_ld[i] = ld;
        *out = root->cm[i];
        return ACSE_OK;
    }
    return ACSE_ERR_UNSUPPORTED;
}

static int oz_list_create(OzPlan* root, const GemmF64* g, int n, OzPlan** out) {
    OzPlan* pl = (OzPlan*)calloc(1, sizeof(OzPlan));
    if (!pl) return ACSE_ERR_NOMEM;
    *out = pl;
    int maxN = 0;
    for (int i = 0; i < n; ++i) maxN = g[i].N > maxN ? g[i].N : maxN;
    ACSE_TRY(oz_plan_init(pl, root->S, maxN >= 256 ? OZ_BN : 128, root->pair));
    pl->host->err = root->err;
    for (int i = 0; i < n; ++i) {
        ACSE_TRY(oz_op_alloc(pl->A[i], g[i].M, g[i].K, pl->S));
        ACSE_TRY(oz_op_alloc(pl->B[i], g[i].N, g[i].K, pl->S));
        ACSE_TRY(oz_add(pl, pl->A[i], pl->B[i], g[i].C, g[i].ldc, g[i].alpha));
    }
    return oz_plan_finish(pl);
}

int oz_gemm_list(acse_ctx* c, const GemmF64* g, int n, int slot) {
    OzPlan* root = (OzPlan*)c->oz_plan;
    if (!root || slot < 0 || slot > 1 || n < 1 || n > OZ_MAXP) return ACSE_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) {
        int ex = 0;
        if (frexp(g[i].alpha, &ex) != 0.5 || (g[i].beta != 0.0 && g[i].beta != 1.0) || g[i].perm_r) return ACSE_ERR_ARG;
    }
    if (!root->lists[slot]) {
        const int s = oz_list_create(root, g, n, &root->lists[slot]);
        if (s != ACSE_OK) {
            oz_plan_free(root->lists[slot]);
            root->lists[slot] = nullptr;
            return s;
        }
    }
    OzPlan* pl = root->lists[slot];
    OzBatch& B = *pl->host;
    if (B.nprob != n) return ACSE_ERR_SHAPE;
    for (int i = 0; i < n; ++i)
        if (B.p[i].M != g[i].M || B.p[i].N != g[i].N || pl->A[i].K != g[i].K) return ACSE_ERR_SHAPE;
    // slices of every operand (A in order, B reversed), at most OZ_MAXJ jobs a launch
    OzSliceBatch sb;
    memset(&sb, 0, sizeof(sb));
    sb.S = pl->S;
    int rows = 0;
    for (int i = 0; i < n; ++i) {
        for (int side = 0; side < 2; ++side) {
            const double* src = side ? g[i].B : g[i].A;
            const int tr = side ? g[i].transB : g[i].transA;
            const int ld = side ? g[i].ldb : g[i].lda;
            const OzOp& o = side ? pl->B[i] : pl->A[i];
            const int* cm = nullptr;
            if (tr) ACSE_TRY(oz_colmap(root, o.K, ld, &cm));
            oz_job(sb, rows, o, 0, o.rows, src, tr ? 1 : (size_t)ld, nullptr, cm, side);
            if (sb.njobs == OZ_MAXJ) {
                ACSE_TRY(oz_slice_launch(c, sb));
                memset(&sb, 0, sizeof(sb));
                sb.S = pl->S;
                rows = 0;
            }
        }
    }
    if (sb.njobs) {
        ACSE_TRY(oz_slice_launch(c, sb));
    }
    // this call's outputs, scales and accumulation
    for (int i = 0; i < n; ++i) {
        OzProb& p = B.p[i];
        int ex = 0;
        frexp(g[i].alpha, &ex);
        p.C = g[i].C;
        p.ldc = g[i].ldc;
        p.alpha = g[i].alpha;
        p.ealpha = ex - 1;
        p.accum = g[i].beta != 0.0;
    }
    B.wait_ns = root->host->wait_ns;
    B.inject_stall = root->host->inject_stall;
    ACSE_CUDA_TRY(cudaMemcpyAsync(pl->dev, pl->host, sizeof(OzBatch), cudaMemcpyHostToDevice, c->stream));
    if (pl->tiles == 0) return ACSE_OK;
    ACSE_TRY(oz_launch_gemm(pl, c->stream));
    ACSE_LAUNCHED(c);
    k_oz_reduce<<<dim3(2 * pl->nsm, B.nprob), 256, 0, c->stream>>>(pl->dev);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}
