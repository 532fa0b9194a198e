// Split-precision O(r^6) contractions on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// C[m][n] = alpha * sum_k A'[m][k] B'[n][k] in FP32, where A' and B' are K-major operand copies
// written by the pack kernels of acse_mixed.cu:
//   BF16x3: A' = [hi(A) | hi(A) | lo(A)], B' = [hi(B) | lo(B) | hi(B)] (bf16, kind::f16), so the
//           single K-concatenated product is hi.hi + hi.lo + lo.hi with FP32 accumulation;
//   TF32:   A' = tf32(A), B' = tf32(B) (kind::tf32), one product.
// Each K segment is zero padded to a multiple of the 128-byte K block.
//
// Kernel: one 128 x BN output tile per CTA, 6 warps.  Warp 0 lane 0 issues TMA loads (128B
// swizzle) into a STAGES-deep shared-memory ring; warp 1 owns the TMEM accumulator (128 lanes x BN
// fp32 columns) and its lane 0 issues tcgen05.mma (M=128, N=BN, K=16/8 per instruction, 4 per
// K block) and tcgen05.commit to release stages; warps 2-5 read TMEM with tcgen05.ld and store
// FP32 rows.  Every mbarrier wait is bounded: on expiry the kernel raises the device error flag,
// lets the in-flight copies and MMAs land (again bounded), frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <queue>
#include <utility>
#include <vector>

#include "acse_internal.h"

#define TC_MAXP 160          // problems of one grouped launch (16 instances x 9 GEMMs fit)
#define TC_BM 128
#define TC_THREADS 192
#define TC_DRAIN_NS 2000000000ull      // bound of the clean-up waits (2 s)
#define TC_WAIT_NS 4000000000ull       // default bound of the pipeline waits (4 s)

struct TcProb {
    float* C;
    int M, N, kblocks, ldc;
    float alpha;
    int tiles_n;
    int tile_start;
    int perm_r;   // 0: C row-major.  r: particle-hole output C[(sK,k,j)][(sI,i,l)] stored as
                  // Cp[sK * nsb + sI][(i,j)][(k,l)] (nsb = N / r^2), the row order the B kernel reads
};

struct __align__(128) TcBatch {
    CUtensorMap tmA[TC_MAXP];
    CUtensorMap tmB[TC_MAXP];
    TcProb p[TC_MAXP];
    int nprob;
    int total_tiles;
    int* err;
    unsigned long long wait_ns;
    int inject_stall;     // test knob: the MMA thread first waits on a barrier nothing signals
    const int* order;     // persistent kernel: tiles of CTA c are order[cta_start[c] .. cta_start[c+1])
    const int* cta_start;
};

#include "tc_ptx.cuh"

// ------------------------------------------------------------------------------ kernel
template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc(const TcBatch* __restrict__ bp) {
    const TcBatch& b = *bp;   // problem table in device memory (tensor maps written by the host)
    constexpr int A_BYTES = TC_BM * 128;
    constexpr int B_BYTES = BN * 128;
    constexpr int KELEM = KIND == 0 ? 64 : 32;      // elements per 128-byte K block
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;
    uint64_t* never = accf + 1;                     // signalled by nobody (fault-injection knob)
    uint32_t* tmem_slot = (uint32_t*)(never + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x;
    int lo = 0, hi = b.nprob - 1;   // last problem with tile_start <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.p[mid].tile_start <= t) lo = mid;
        else hi = mid - 1;
    }
    const int pi = lo;
    const TcProb& P = b.p[pi];
    const int local = t - P.tile_start;
    const int m0 = (local / P.tiles_n) * TC_BM;
    const int n0 = (local % P.tiles_n) * BN;
    const int nk = P.kblocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(never, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch(&b.tmA[pi]);
            tma_prefetch(&b.tmB[pi]);
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES &&
                    !bounded_wait(&empty[s], ((kb / STAGES) & 1) ^ 1, b.wait_ns, abort_flag)) {
                    raise_abort(b.err, abort_flag);
                    break;
                }
                mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                tma_load_2d(sA + s * A_BYTES, &b.tmA[pi], kb * KELEM, m0, &full[s]);
                tma_load_2d(sB + s * B_BYTES, &b.tmB[pi], kb * KELEM, n0, &full[s]);
                ++issued;
            }
            // every issued copy must have landed before the CTA may exit
            for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
                if (!bounded_wait(&full[kb % STAGES], (kb / STAGES) & 1, TC_DRAIN_NS, nullptr))
                    raise_abort(b.err, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc<KIND, BN>();
            if (b.inject_stall && !bounded_wait(never, 0, b.wait_ns, abort_flag)) raise_abort(b.err, abort_flag);
            for (int kb = 0; kb < nk && !*abort_flag; ++kb) {
                const int s = kb % STAGES;
                if (!bounded_wait(&full[s], (kb / STAGES) & 1, b.wait_ns, abort_flag)) {
                    raise_abort(b.err, abort_flag);
                    break;
                }
                tc_fence_after();
                const uint64_t da = smem_desc(sA + s * A_BYTES);
                const uint64_t db = smem_desc(sB + s * B_BYTES);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) umma<KIND>(tmem, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                umma_commit(&empty[s]);
            }
            umma_commit(accf);   // arrives when every MMA issued above has completed (also after an abort)
        }
    } else {
        const int q = warp & 3;   // TMEM lane quadrant this warp may access
        const bool ok = bounded_wait(accf, 0, b.wait_ns + TC_DRAIN_NS, nullptr);
        if (!ok) raise_abort(b.err, abort_flag);
        tc_fence_after();
        const bool store = ok && !*abort_flag && nk > 0;
        const int row = m0 + q * 32 + lane;
        float* Crow = P.C + (size_t)row * P.ldc;
        const bool vec = (P.ldc & 3) == 0 && P.perm_r == 0 && (reinterpret_cast<uintptr_t>(P.C) & 15) == 0;
        // permuted particle-hole store: row (sK, kk, jj) fixed per thread, columns (sI, i, l)
        const int pr = P.perm_r, pR2 = pr * pr;
        int sK = 0, kk = 0, jj = 0, nsb = 1;
        if (pr) {
            sK = row / pR2;
            kk = (row % pR2) / pr;
            jj = row % pr;
            nsb = P.N / pR2;
        }
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32), v);   // warp-collective
            const int col0 = n0 + c * 32;
            if (store && row < P.M && col0 < P.N) {
                if (pr) {
                    int sI = col0 / pR2, ii = (col0 % pR2) / pr, ll = col0 % pr;
                    for (int j = 0; j < 32 && col0 + j < P.N; ++j) {
                        const size_t dst = ((size_t)(sK * nsb + sI) * pR2 + (size_t)ii * pr + jj) * pR2 + (size_t)kk * pr + ll;
                        P.C[dst] = P.alpha * __uint_as_float(v[j]);
                        if (++ll == pr) {
                            ll = 0;
                            if (++ii == pr) { ii = 0; ++sI; }
                        }
                    }
                } else if (vec && col0 + 32 <= P.N) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        float4 o = make_float4(P.alpha * __uint_as_float(v[j]), P.alpha * __uint_as_float(v[j + 1]),
                                               P.alpha * __uint_as_float(v[j + 2]),
                                               P.alpha * __uint_as_float(v[j + 3]));
                        *reinterpret_cast<float4*>(Crow + col0 + j) = o;
                    }
                } else {
                    for (int j = 0; j < 32 && col0 + j < P.N; ++j) Crow[col0 + j] = P.alpha * __uint_as_float(v[j]);
                }
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// ------------------------------------------------------------------ persistent variant
// One CTA per SM walks its list of tiles, assigned on the host by longest processing time (tile cost =
// its K blocks plus a per-tile epilogue allowance), costliest first: static round-robin over tiles of
// unequal K left the busiest SM about 8 % above the mean at r = 48.  The shared-memory ring runs on across tiles (a global K-block counter
// gives stage and phase), and the accumulator is double-buffered in TMEM (2 x BN columns): the MMA
// thread fills buffer (tile & 1) while warps 2-5 drain the other one, so a tile's epilogue and the
// next tile's first loads and MMAs overlap.  Barriers: full/empty per stage, accf[2] (MMA -> epilogue,
// one commit per tile), acce[2] (epilogue -> MMA, one arrival per epilogue warp).  All waits are
// bounded as in k_gemm_tc; at the end the MMA thread commits to drainb and waits for it, so no MMA is
// in flight when TMEM is freed.

__device__ __forceinline__ int tc_find_problem(const TcBatch& b, int t) {
    int lo = 0, hi = b.nprob - 1;   // last problem with tile_start <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.p[mid].tile_start <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tile coordinates of local tile `local` of problem P for the persistent kernel: row-major over the
// tile grid (measured faster here than walking groups of 16 tile rows column by column).
template <int BN>
__device__ __forceinline__ void tc_tile_coords(const TcProb& P, int local, int& m0, int& n0) {
    m0 = (local / P.tiles_n) * TC_BM;
    n0 = (local % P.tiles_n) * BN;
}

template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc_pers(const TcBatch* __restrict__ bp) {
    const TcBatch& b = *bp;
    constexpr int A_BYTES = TC_BM * 128;
    constexpr int B_BYTES = BN * 128;
    constexpr int KELEM = KIND == 0 ? 64 : 32;
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
    const int q0 = b.cta_start[blockIdx.x], q1 = b.cta_start[blockIdx.x + 1];   // this CTA's tiles
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], 4);
        }
        mbar_init(never, 1);
        mbar_init(drainb, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool stop = false;
            for (int qi = q0; qi < q1 && !stop; ++qi) {
                const int t = b.order[qi];
                const int pi = tc_find_problem(b, t);
                const TcProb& P = b.p[pi];
                int m0, n0;
                tc_tile_coords<BN>(P, t - P.tile_start, m0, n0);
                for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !bounded_wait(&empty[s], ((it / STAGES) & 1) ^ 1, b.wait_ns, abort_flag)) {
                        raise_abort(b.err, abort_flag);
                        stop = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                    tma_load_2d(sA + s * A_BYTES, &b.tmA[pi], kb * KELEM, m0, &full[s]);
                    tma_load_2d(sB + s * B_BYTES, &b.tmB[pi], kb * KELEM, n0, &full[s]);
                }
            }
            // every issued copy must have landed before the CTA may exit
            for (int k = it > STAGES ? it - STAGES : 0; k < it; ++k)
                if (!bounded_wait(&full[k % STAGES], (k / STAGES) & 1, TC_DRAIN_NS, nullptr))
                    raise_abort(b.err, abort_flag);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc<KIND, BN>();
            if (b.inject_stall && !bounded_wait(never, 0, b.wait_ns, abort_flag)) raise_abort(b.err, abort_flag);
            int it = 0, lt = 0;
            for (int qi = q0; qi < q1 && !*abort_flag; ++qi, ++lt) {
                const int t = b.order[qi];
                const int pi = tc_find_problem(b, t);
                const int nk = b.p[pi].kblocks;
                const int ab = lt & 1, use = lt >> 1;
                if (use >= 1 && !bounded_wait(&acce[ab], (use - 1) & 1, b.wait_ns + TC_DRAIN_NS, abort_flag)) {
                    raise_abort(b.err, abort_flag);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(ab * BN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!bounded_wait(&full[s], (it / STAGES) & 1, b.wait_ns, abort_flag)) {
                        raise_abort(b.err, abort_flag);
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = smem_desc(sA + s * A_BYTES);
                    const uint64_t db = smem_desc(sB + s * B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) umma<KIND>(acc, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                    umma_commit(&empty[s]);
                }
                umma_commit(&accf[ab]);   // the epilogue of this tile may start when these MMAs are done
            }
            umma_commit(drainb);
            if (!bounded_wait(drainb, 0, TC_DRAIN_NS, nullptr)) raise_abort(b.err, abort_flag);
        }
    } else {
        const int q = warp & 3;   // TMEM lane quadrant this warp may access
        int lt = 0;
        for (int qi = q0; qi < q1; ++qi, ++lt) {
            const int t = b.order[qi];
            const int ab = lt & 1, use = lt >> 1;
            // lane 0 waits and the warp follows its verdict (tcgen05.ld below is warp-collective)
            int go = 0;
            if (lane == 0) {
                const bool ok = bounded_wait(&accf[ab], use & 1, b.wait_ns + TC_DRAIN_NS, abort_flag);
                if (!ok) raise_abort(b.err, abort_flag);
                go = ok && !*abort_flag;
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            tc_fence_after();
            const int pi = tc_find_problem(b, t);
            const TcProb& P = b.p[pi];
            int m0, n0;
            tc_tile_coords<BN>(P, t - P.tile_start, m0, n0);
            const int row = m0 + q * 32 + lane;
            float* Crow = P.C + (size_t)row * P.ldc;
            const bool vec = (P.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(P.C) & 15) == 0;
            const bool store = P.kblocks > 0;
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + c * 32), v);   // warp-collective
                const int col0 = n0 + c * 32;
                if (store && row < P.M && col0 < P.N) {
                    if (vec && col0 + 32 <= P.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 o = make_float4(P.alpha * __uint_as_float(v[j]), P.alpha * __uint_as_float(v[j + 1]),
                                                   P.alpha * __uint_as_float(v[j + 2]),
                                                   P.alpha * __uint_as_float(v[j + 3]));
                            *reinterpret_cast<float4*>(Crow + col0 + j) = o;
                        }
                    } else {
                        for (int j = 0; j < 32 && col0 + j < P.N; ++j) Crow[col0 + j] = P.alpha * __uint_as_float(v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[ab]);   // this warp's quarter of the buffer is free
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ------------------------------------------------------------ persistent CTA-pair variant
// A cluster of two CTAs on two SMs computes 256 x 256 output tiles with the pair MMA (cta_group::2,
// M = 256, N = 256): each CTA loads its 128 rows of A and its 128 rows of B (the rows n0 .. n0 + 127
// in the even CTA, n0 + 128 .. n0 + 255 in the odd one) per K block, so per SM a K block moves
// 32 KB through shared memory for 128 x 256 x 64 MACs instead of the 48 KB of a one-SM 128 x 256
// tile; shared-memory bandwidth, which the TMA writes and the MMA reads share, bounds the one-SM
// kernel.  The even CTA's thread issues the MMAs and the commits, which arrive on the barriers of
// both CTAs (empty[s], accf[ab], drainb); both CTAs' TMA loads complete on the even CTA's full[s]
// (it expects the bytes of both); the epilogue warps of both CTAs arrive on the even CTA's acce[ab].
// The clusters walk the tile lists of the host's LPT schedule (one list per cluster); every wait is
// bounded as in k_gemm_tc_pers, and the CTAs meet at a cluster barrier before the TMEM is freed.
template <int KIND, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc2_pers(const TcBatch* __restrict__ bp) {
    const TcBatch& b = *bp;
    constexpr int BN = 256;
    constexpr int A_BYTES = TC_BM * 128;     // this CTA's 128 rows of A per K block
    constexpr int B_BYTES = 128 * 128;       // this CTA's 128 rows of B per K block
    constexpr int KELEM = KIND == 0 ? 64 : 32;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;   // [2]
    uint64_t* acce = accf + 2;         // [2], used in the even CTA
    uint64_t* never = acce + 2;
    uint64_t* drainb = never + 1;
    uint32_t* tmem_slot = (uint32_t*)(drainb + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int cl = blockIdx.x >> 1;
    const int q0 = b.cta_start[cl], q1 = b.cta_start[cl + 1];   // this cluster's tiles
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], 8);
        }
        mbar_init(never, 1);
        mbar_init(drainb, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, 2 * BN);
    tc_fence_before();
    cluster_sync_all();   // both CTAs' barriers are initialised before either signals the other's
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t full0 = mapa_rank(smem_u32(full), 0);   // the even CTA's full[0]
            int it = 0;
            bool stop = false;
            for (int qi = q0; qi < q1 && !stop; ++qi) {
                const int t = b.order[qi];
                const int pi = tc_find_problem(b, t);
                const TcProb& P = b.p[pi];
                const int local = t - P.tile_start;
                const int m0 = (local / P.tiles_n) * 256 + (int)rank * 128;
                const int n0 = (local % P.tiles_n) * BN + (int)rank * 128;
                for (int kb = 0; kb < P.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !bounded_wait(&empty[s], ((it / STAGES) & 1) ^ 1, b.wait_ns, abort_flag)) {
                        raise_abort(b.err, abort_flag);
                        stop = true;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * (A_BYTES + B_BYTES));
                    tma_load_2d_pair(sA + s * A_BYTES, &b.tmA[pi], kb * KELEM, m0, full0 + 8u * s);
                    tma_load_2d_pair(sB + s * B_BYTES, &b.tmB[pi], kb * KELEM, n0, full0 + 8u * s);
                }
            }
            // every issued copy must have landed before the CTA may exit: the even CTA's full[s]
            // counts both CTAs' bytes (and the CTAs leave together, after the cluster barrier below);
            // the odd CTA also waits for the MMAs that read its last stages, briefly after an abort
            for (int k = it > STAGES ? it - STAGES : 0; k < it; ++k) {
                const unsigned long long lim = *abort_flag ? b.wait_ns : TC_DRAIN_NS;
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
            const uint32_t idesc = make_idesc_pair<KIND, BN>();
            if (b.inject_stall && !bounded_wait(never, 0, b.wait_ns, abort_flag)) raise_abort(b.err, abort_flag);
            int it = 0, lt = 0;
            for (int qi = q0; qi < q1 && !*abort_flag; ++qi, ++lt) {
                const int t = b.order[qi];
                const int pi = tc_find_problem(b, t);
                const int nk = b.p[pi].kblocks;
                const int ab = lt & 1, use = lt >> 1;
                if (use >= 1 &&
                    !bounded_wait_cluster(&acce[ab], (use - 1) & 1, b.wait_ns + TC_DRAIN_NS, abort_flag)) {
                    raise_abort(b.err, abort_flag);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(ab * BN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!bounded_wait(&full[s], (it / STAGES) & 1, b.wait_ns, abort_flag)) {
                        raise_abort(b.err, abort_flag);
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = smem_desc(sA + s * A_BYTES);
                    const uint64_t db = smem_desc(sB + s * B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_pair<KIND>(acc, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                    umma_commit_pair(&empty[s]);
                }
                umma_commit_pair(&accf[ab]);
            }
            umma_commit_pair(drainb);
        }
        // both CTAs: no MMA of the pair is in flight past this point (bounded)
        if (lane == 0 && !bounded_wait(drainb, 0, b.wait_ns + 2 * TC_DRAIN_NS, nullptr)) raise_abort(b.err, abort_flag);
    } else {
        const int q = warp & 3;   // TMEM lane quadrant this warp may access
        const uint32_t acce0 = mapa_rank(smem_u32(acce), 0);
        int lt = 0;
        for (int qi = q0; qi < q1; ++qi, ++lt) {
            const int t = b.order[qi];
            const int ab = lt & 1, use = lt >> 1;
            int go = 0;
            if (lane == 0) {
                const bool ok = bounded_wait(&accf[ab], use & 1, b.wait_ns + TC_DRAIN_NS, abort_flag);
                if (!ok) raise_abort(b.err, abort_flag);
                go = ok && !*abort_flag;
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            tc_fence_after();
            const int pi = tc_find_problem(b, t);
            const TcProb& P = b.p[pi];
            const int local = t - P.tile_start;
            const int row = (local / P.tiles_n) * 256 + (int)rank * 128 + q * 32 + lane;
            const int n0 = (local % P.tiles_n) * BN;
            float* Crow = P.C + (size_t)row * P.ldc;
            const bool vec = (P.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(P.C) & 15) == 0;
            const bool store = P.kblocks > 0;
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + c * 32), v);   // warp-collective
                const int col0 = n0 + c * 32;
                if (store && row < P.M && col0 < P.N) {
                    if (vec && col0 + 32 <= P.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 o = make_float4(P.alpha * __uint_as_float(v[j]), P.alpha * __uint_as_float(v[j + 1]),
                                                   P.alpha * __uint_as_float(v[j + 2]),
                                                   P.alpha * __uint_as_float(v[j + 3]));
                            *reinterpret_cast<float4*>(Crow + col0 + j) = o;
                        }
                    } else {
                        for (int j = 0; j < 32 && col0 + j < P.N; ++j) Crow[col0 + j] = P.alpha * __uint_as_float(v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acce0 + 8u * ab);   // this warp's quarter is free
        }
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();   // neither CTA exits while the other may still signal its barriers
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 2 * BN);
    }
}

// --------------------------------------------------------------------------- host plan
// A table (TcTable, acse_internal.h) holds the problems of one grouped launch; its TcBatch lives in
// device memory (the tensor maps are written by the host before any launch reads them).
struct TcPlan {
    PFN_cuTensorMapEncodeTiled_v12000 encode;
    TcTable tab;
};

static int stages_for(int bn) { return bn == 256 ? 4 : 6; }

static size_t smem_for(int bn, int stages) { return (size_t)stages * (TC_BM + bn) * 128 + 1024 + 256; }

#ifndef TC2_STAGES
#define TC2_STAGES 6                         // ring depth of the CTA-pair kernel (32 KB a stage per CTA)
#endif
static size_t smem_pair() { return (size_t)TC2_STAGES * (TC_BM + 128) * 128 + 1024 + 256; }

// Clusters of the CTA-pair kernel that fit on the device at once (its persistent grid).
template <int KIND>
static int pair_attr_and_clusters(int nsm, int* nclusters) {
    auto kern = k_gemm_tc2_pers<KIND, TC2_STAGES>;
    ACSE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pair()));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (nsm / 2), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem_pair();
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = nsm / 2;
    }
    *nclusters = n < nsm / 2 ? n : nsm / 2;
    return ACSE_OK;
}

template <int KIND, int BN>
static int set_attr() {
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<KIND, BN, BN == 256 ? 4 : 6>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_for(BN, stages_for(BN))));
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_pers<KIND, BN, BN == 256 ? 4 : 6>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_for(BN, stages_for(BN))));
    return ACSE_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encode(PFN_cuTensorMapEncodeTiled_v12000* out) {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return ACSE_ERR_CUDA;
        }
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    *out = g_encode;
    return ACSE_OK;
}

// 2-D map over `rows` rows of `inner_elems` elements, consecutive rows `row_stride` elements apart.
static int encode_map(int kind, CUtensorMap* m, const void* base, int rows, int inner_elems, int box_rows,
                      size_t row_stride) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    ACSE_TRY(get_encode(&enc));
    const CUtensorMapDataType dt = kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const int es = kind == 0 ? 2 : 4;
    cuuint64_t gdim[2] = {(cuuint64_t)inner_elems, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)row_stride * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, dt, 2, const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? ACSE_OK : ACSE_ERR_CUDA;
}

int tc_encode_map_bf16(void* map, const void* base, int rows, int inner_elems, int box_rows, size_t row_stride) {
    return encode_map(0, (CUtensorMap*)map, base, rows, inner_elems, box_rows, row_stride);
}

int tc_table_init_mode(TcTable* t, int kind, int bn, int pair) {
    memset(t, 0, sizeof(*t));
    t->kind = kind;
    t->bn = bn;
    t->pair = pair && bn == 256;
    t->bm = t->pair ? 2 * TC_BM : TC_BM;
    t->stages = t->pair ? TC2_STAGES : stages_for(bn);
    t->smem = t->pair ? smem_pair() : smem_for(bn, t->stages);
    if (kind == 0) ACSE_TRY(bn == 256 ? (set_attr<0, 256>()) : (set_attr<0, 128>()));
    else ACSE_TRY(bn == 256 ? (set_attr<1, 256>()) : (set_attr<1, 128>()));
    t->pers = 1;
    t->nsm = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        t->nsm = 152;
    }
    if (t->pair) ACSE_TRY(kind == 0 ? pair_attr_and_clusters<0>(t->nsm, &t->nclusters)
                                    : pair_attr_and_clusters<1>(t->nsm, &t->nclusters));
    t->host = (TcBatch*)calloc(1, sizeof(TcBatch));
    if (!t->host) return ACSE_ERR_NOMEM;
    t->host->wait_ns = TC_WAIT_NS;
    if (cudaMalloc((void**)&t->dev, sizeof(TcBatch)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    return ACSE_OK;
}

int tc_table_init(TcTable* t, int kind, int bn) { return tc_table_init_mode(t, kind, bn, 0); }

void tc_table_free(TcTable* t) {
    if (t->dev) cudaFree(t->dev);
    if (t->sched) cudaFree(t->sched);
    free(t->host);
    memset(t, 0, sizeof(*t));
}

void tc_lpt_schedule(const long long* cost, int T, int G, int* order, int* start) {
    std::vector<int> idx(T);
    for (int i = 0; i < T; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // min-heap of (load, cta)
    std::priority_queue<std::pair<long long, int>, std::vector<std::pair<long long, int>>,
                        std::greater<std::pair<long long, int>>> heap;
    for (int c = 0; c < G; ++c) heap.push({0, c});
    std::vector<std::vector<int>> lists(G);
    for (int i : idx) {
        auto top = heap.top();
        heap.pop();
        lists[top.second].push_back(i);
        heap.push({top.first + cost[i], top.second});
    }
    int q = 0;
    for (int c = 0; c < G; ++c) {
        start[c] = q;
        for (int i : lists[c]) order[q++] = i;
    }
    start[G] = q;
}

// Uploads the table and the persistent kernel's tile schedule (for the grid tc_table_launch uses).
int tc_table_upload(TcTable* t) {
    TcBatch& b = *t->host;
    const int T = b.total_tiles;
    const int slots = t->pair ? t->nclusters : t->nsm;   // CTAs, or CTA pairs, of the persistent grid
    const int G = T < slots ? T : slots;
    if (T > 0) {
        std::vector<long long> cost(T);
        for (int p = 0; p < b.nprob; ++p) {
            const int n = ((b.p[p].M + t->bm - 1) / t->bm) * b.p[p].tiles_n;
            for (int k = 0; k < n; ++k) cost[b.p[p].tile_start + k] = b.p[p].kblocks + 4;
        }
        const int need = T + G + 1;
        if (t->sched_cap < need) {
            if (t->sched) cudaFree(t->sched);
            t->sched = nullptr;
            t->sched_cap = 0;
            if (cudaMalloc((void**)&t->sched, (size_t)need * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return ACSE_ERR_NOMEM;
            }
            t->sched_cap = need;
        }
        std::vector<int> h(need);
        tc_lpt_schedule(cost.data(), T, G, h.data(), h.data() + T);
        ACSE_CUDA_TRY(cudaMemcpy(t->sched, h.data(), (size_t)need * sizeof(int), cudaMemcpyHostToDevice));
        b.order = t->sched;
        b.cta_start = t->sched + T;
    }
    ACSE_CUDA_TRY(cudaMemcpy(t->dev, t->host, sizeof(TcBatch), cudaMemcpyHostToDevice));
    return ACSE_OK;
}

// Append one problem C[M][N] = alpha * A'[M][L] B'[N][L]^T (K-major split operand rows: L elements
// used, a multiple of the 128-byte K block, consecutive rows lda / ldb elements apart) to table t.
int tc_table_add_ld(TcTable* t, const void* A, size_t lda, const void* B, size_t ldb, float* C, int M, int N, int L,
                    int ldc, float alpha) {
    TcBatch& b = *t->host;
    const int kel = t->kind == 0 ? 64 : 32;
    if (b.nprob + 1 > TC_MAXP || L % kel || lda < (size_t)L || ldb < (size_t)L) return ACSE_ERR_SHAPE;
    const int n = b.nprob;
    ACSE_TRY(encode_map(t->kind, &b.tmA[n], A, M, L, TC_BM, lda));
    ACSE_TRY(encode_map(t->kind, &b.tmB[n], B, N, L, t->pair ? t->bn / 2 : t->bn, ldb));
    TcProb& p = b.p[n];
    p.C = C;
    p.M = M;
    p.N = N;
    p.kblocks = L / kel;
    p.ldc = ldc;
    p.alpha = alpha;
    p.tiles_n = (N + t->bn - 1) / t->bn;
    p.tile_start = b.total_tiles;
    p.perm_r = 0;
    b.total_tiles += ((M + t->bm - 1) / t->bm) * p.tiles_n;
    b.nprob = n + 1;
    return ACSE_OK;
}

int tc_table_add(TcTable* t, const void* A, const void* B, float* C, int M, int N, int L, int ldc, float alpha) {
    return tc_table_add_ld(t, A, (size_t)L, B, (size_t)L, C, M, N, L, ldc, alpha);
}

// Device flag raised by a launch of table t when a bounded wait runs out.
void tc_table_set_err(TcTable* t, int* err) { t->host->err = err; }

// Append the nine GEMMs of one contraction pass of context c to table t (tile width t->bn).
int tc_table_append(TcTable* t, acse_ctx* c) {
    TcBatch& b = *t->host;
    Work& w = c->w;
    const int r = c->r, R2 = r * r, R22 = 2 * R2;
    const int ns = c->nsplit;
    const int L1 = ns * w.Kp1, L2 = ns * w.Kp2;      // operand row lengths (elements)
    if (b.nprob + 6 > TC_MAXP) return ACSE_ERR_SHAPE;
    // the diagonal particle-hole GEMM first (largest K), then the pair-pair and spin-flip ones; with the
    // spin-flip specialisation only the alpha-led rows of the diagonal sector, the aa and ab pair
    // sectors and the first flip sector
    const bool sf = acse_singlet(c);
    ACSE_TRY(tc_table_add(t, w.tc_Zd, w.tc_Md, w.tc_X5d, sf ? R2 : R22, R22, L2, R22, 1.0f));
    // same-spin sectors on packed pairs (i < j rows, k < p columns, r < s K; alpha 2 for the (r, s) sum),
    // the mixed sector on full pairs (alpha 2: both orders of the mixed (r, s) pairs)
    const int P = r * (r - 1) / 2, LP = ns * w.KpP;
    for (int s = 0; s < 3; ++s) {
        if (s == 1) ACSE_TRY(tc_table_add(t, w.tc_pairA[s], w.tc_pairB[s], w.tc_pairC[s], R22, R2, L1, R2, 2.0f));
        else if (!(sf && s == 2))
            ACSE_TRY(tc_table_add(t, w.tc_pairA[s], w.tc_pairB[s], w.tc_pairCp[s], 2 * P, P, LP, P, 2.0f));
    }
    for (int f = 0; f < (sf ? 1 : 2); ++f)
        ACSE_TRY(tc_table_add(t, w.tc_Zf[f], w.tc_Mf[f], w.tc_X5f[f], R2, R2, L1, R2, 1.0f));
    b.err = w.tc_err;
    return ACSE_OK;
}

int tc_table_launch(const TcTable* t, cudaStream_t st) {
    const int tiles = t->host->total_tiles;
    if (tiles == 0) return ACSE_OK;
    if (t->pair) {
        const int g = tiles < t->nclusters ? tiles : t->nclusters;
        if (t->kind == 0) k_gemm_tc2_pers<0, TC2_STAGES><<<2 * g, TC_THREADS, t->smem, st>>>(t->dev);
        else k_gemm_tc2_pers<1, TC2_STAGES><<<2 * g, TC_THREADS, t->smem, st>>>(t->dev);
        ACSE_CUDA_TRY(cudaGetLastError());
        return ACSE_OK;
    }
    if (t->pers) {
        const int g = tiles < t->nsm ? tiles : t->nsm;
        if (t->kind == 0) {
            if (t->bn == 256) k_gemm_tc_pers<0, 256, 4><<<g, TC_THREADS, t->smem, st>>>(t->dev);
            else k_gemm_tc_pers<0, 128, 6><<<g, TC_THREADS, t->smem, st>>>(t->dev);
        } else {
            if (t->bn == 256) k_gemm_tc_pers<1, 256, 4><<<g, TC_THREADS, t->smem, st>>>(t->dev);
            else k_gemm_tc_pers<1, 128, 6><<<g, TC_THREADS, t->smem, st>>>(t->dev);
        }
        ACSE_CUDA_TRY(cudaGetLastError());
        return ACSE_OK;
    }
    if (t->kind == 0) {
        if (t->bn == 256) k_gemm_tc<0, 256, 4><<<tiles, TC_THREADS, t->smem, st>>>(t->dev);
        else k_gemm_tc<0, 128, 6><<<tiles, TC_THREADS, t->smem, st>>>(t->dev);
    } else {
        if (t->bn == 256) k_gemm_tc<1, 256, 4><<<tiles, TC_THREADS, t->smem, st>>>(t->dev);
        else k_gemm_tc<1, 128, 6><<<tiles, TC_THREADS, t->smem, st>>>(t->dev);
    }
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

int tc_default_bn(int r) { return r * r >= 256 ? 256 : 128; }

// The CTA-pair form is the default of the 256-wide tiles; acse_opts.gemm_tile = 1 keeps one SM per tile.
int tc_use_pairs(const acse_ctx* c) { return c->opt.gemm_tile != 1 && tc_default_bn(c->r) == 256; }

int tc_mixed_alloc(acse_ctx* c);
void tc_mixed_free(acse_ctx* c);

int tc_plan_create(acse_ctx* c) {
    TcPlan* pl = (TcPlan*)calloc(1, sizeof(TcPlan));
    if (!pl) return ACSE_ERR_NOMEM;
    c->tc_plan = pl;
    ACSE_TRY(get_encode(&pl->encode));
    ACSE_TRY(tc_mixed_alloc(c));
    ACSE_TRY(tc_table_init_mode(&pl->tab, (c->opt.prec == ACSE_TF32 || c->opt.prec == ACSE_TF32X3) ? 1 : 0,
                                tc_default_bn(c->r), tc_use_pairs(c)));
    ACSE_TRY(tc_table_append(&pl->tab, c));
    return tc_table_upload(&pl->tab);
}

void tc_plan_destroy(acse_ctx* c) {
    if (!c->tc_plan) return;
    tc_table_free(&((TcPlan*)c->tc_plan)->tab);
    tc_mixed_free(c);
    free(c->tc_plan);
    c->tc_plan = nullptr;
}

int tc_set_wait_ns(acse_ctx* c, unsigned long long ns, int inject_stall) {
    if (!c->tc_plan) return ACSE_ERR_UNSUPPORTED;
    TcTable& t = ((TcPlan*)c->tc_plan)->tab;
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    t.host->wait_ns = ns ? ns : TC_WAIT_NS;
    t.host->inject_stall = inject_stall;
    return tc_table_upload(&t);
}

int tc_gemm_launch(acse_ctx* c) {
    TcPlan* pl = (TcPlan*)c->tc_plan;
    ACSE_TRY(prof_begin(c));
    ACSE_TRY(tc_table_launch(&pl->tab, c->stream));
    c->launches++;
    ACSE_TRY(prof_end(c));
    return ACSE_OK;
}

int tc_contract_pre(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D) {
    if (prep_D) ACSE_TRY(tc_mixed_prep_D(c, D));
    return tc_mixed_prep_W(c, W);
}

int tc_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D) {
    ACSE_TRY(tc_contract_pre(c, D, W, prep_D));
    return tc_gemm_launch(c);
}
