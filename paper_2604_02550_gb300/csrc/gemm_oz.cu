// FP64-accurate GEMMs of the contraction pass on the BF16 tensor cores by the modular form of the Ozaki
// scheme (K. Ozaki, Y. Uchino, T. Imamura, "Ozaki Scheme II: a GEMM-oriented emulation of floating-point
// matrix multiplication using an integer modular technique", 2025).
//
// C = alpha A B^T with A (M x K) and B (N x K) FP64, both K-major.  Every operand row is scaled by a power
// of two and rounded to an integer row: with |a| 2^-e < 1/2 over the row, X = round(a 2^(nb - e)), so that
// |X| <= 2^(nb-1) and a = 2^(e - nb) X up to half a unit of the last kept bit (nb - 1 = min(6S, 53) bits
// below the row's leading bit for oz_slices = S).  The integer product X_A X_B^T then has entries of at
// most K 2^(2 nb - 2) in magnitude.  It is computed modulo T pairwise coprime moduli p_t <= 127 (the
// first T of a fixed list, T the least with 4 K 2^(2 nb - 2) <= P = prod p_t):
//   * the residue kernel writes near-balanced residues X mod p_t (|.| <= 64, exact in bf16), the B rows
//     premultiplied by y_t = (P / p_t)^-1 mod p_t, each modulus to its K segment of the row;
//   * the tensor cores multiply the residue matrices of each modulus in FP32; a chunk of at most 64 * 64
//     K elements keeps every partial sum an integer of magnitude at most 64 * 64 * 64^2 = 2^24, so the
//     accumulation is exact, and the epilogue stores a residue w (|w| <= 65) of the chunk sum (one byte);
//   * the reconstruction kernel forms s = sum_t w_t (P / p_t) exactly in FP32 sums of 10- or 11-bit
//     limbs, which is congruent to X_A X_B^T modulo every p_t and hence modulo P (Chinese remainder theorem), takes
//     q = round(s / P) (the product lies within P / 4 of zero, so a float estimate of s / P decides q),
//     and x = s - q P is the exact integer product, rounded once to FP64 and scaled by alpha 2^(ea + eb - 2 nb).
// The result is the FP64 product up to the rounding of the operands to nb - 1 bits below each row's
// leading bit and one final rounding: no product level is dropped.  Against the six-bit slice form of
// the scheme (36 slice products at S = 8) this takes 17 residue products at S = 8 and r = 48.
//
// Kernels: the persistent tcgen05 GEMM of gemm_tc.cu with the accumulation unit changed from a tile
// to a (tile, modulus, K chunk) group: the MMA thread runs the groups of a tile one after another into the
// two TMEM buffers, and the epilogue warps store each group's residue (a byte) to a staging array.  A
// second kernel rebuilds every element from its residues and writes the FP64 result once.  Every wait
// is bounded as in gemm_tc.cu.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include "acse_internal.h"
#include "oz_arith.cuh"
#include "tc_ptx.cuh"

#define OZ_NMOD 19           // moduli of the fixed list
#define OZ_CHUNK_KB 64       // 64-element K blocks of one exactly accumulated chunk: 64 * 64 * 64^2 = 2^24
#define OZ_MAXCH 2           // chunks of one residue product (K <= 2 * 64 * 64 = 8192)
#define OZ_MAXP 12           // GEMMs of one launch
#define OZ_MAXJ 16           // operands of one slicing launch
#define OZ_THREADS 192
#define OZ_BN 256
#define OZ_STAGES 4
#define OZ2_STAGES 6         // ring depth of the CTA-pair form (32 KB a stage per CTA)
#define OZ_DRAIN_NS 2000000000ull
#define OZ_WAIT_NS 4000000000ull
// limbs of the reconstruction: 14 of 10 bits for two K chunks, 12 of 11 bits for one (their limb sums stay
// below 2^22 in magnitude either way)
#define OZ_LB2 10
#define OZ_NL2 14
#define OZ_LB1 11
#define OZ_NL1 12
#ifndef OZ_CRT_MINB
#define OZ_CRT_MINB 3        // resident blocks of 256 threads per SM the reconstruction is compiled for
#endif

// Pairwise coprime moduli, largest first: 127, 5^3, 3 * 41, 11^2, 7 * 17 and the primes 113 .. 59.
static const int oz_moduli[OZ_NMOD] = {127, 125, 123, 121, 119, 113, 109, 107, 103, 101, 97, 89, 83, 79, 73, 71, 67, 61, 59};

// The constants of a set of T moduli (host-computed, exact).
struct OzMods {
    int T;
    float p[OZ_NMOD];         // p_t
    float pinv[OZ_NMOD];      // 1 / p_t, rounded
    float cA[OZ_NMOD][4];     // 2^(14 l) mod p_t, l = 0..3 (limb weights of an A row)
    float cB[OZ_NMOD][4];     // 2^(14 l) y_t mod p_t, y_t = (P / p_t)^-1 mod p_t (limb weights of a B row)
    float q10[OZ_NMOD][OZ_NL2];   // P / p_t in base-2^10 limbs, least significant first (exact floats)
    float P10[OZ_NL2];            // P in base-2^10 limbs
    float q11[OZ_NMOD][OZ_NL1];   // the same in base-2^11 limbs
    float P11[OZ_NL1];
    float pinvs;              // 2^120 / P, rounded (between 2^-5 and 2^114)
};

struct OzProb {
    double* C;
    unsigned char* stage;   // [ngroups][M][N]: the residue w + 128 of each (modulus, chunk) group
    const double* sa;   // 2^ea per row of A
    const double* sb;   // 2^eb per row of B
    double alpha;
    int ealpha;         // alpha = 2^ealpha
    int M, N, ldc;
    int kbs;            // 64-element K blocks per modulus segment
    int nch, cb;        // K chunks per modulus and 64-element blocks per chunk (the last may be shorter)
    int nb;             // operand rows rounded to X = round(a 2^(nb - e))
    int ngroups;        // T nch, modulus-major
    int tiles_n, tile_start;
    int accum;          // 1: C += result (one FP64 addition), 0: C = result
};

struct __align__(128) OzBatch {
    CUtensorMap tmA[OZ_MAXP];
    CUtensorMap tmB[OZ_MAXP];
    OzProb p[OZ_MAXP];
    OzMods mods;
    int nprob;
    int total_tiles;
    int* err;
    unsigned long long wait_ns;
    int inject_stall;
    const int* order;     // tiles of CTA c: order[cta_start[c] .. cta_start[c+1]) (longest first)
    const int* cta_start;
};

__device__ __forceinline__ int oz_find_problem(const OzBatch& b, int t) {
    int lo = 0, hi = b.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.p[mid].tile_start <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Near-balanced residue of an integer-valued float |v| <= 2^24 modulo p <= 127: q = round(v pinv) (the
// fused multiply-add rounds v pinv + 1.5 * 2^23 once, to an integer), r = v - q p exactly.  pinv = 1/p
// rounded moves v / p by at most |v / p| 2^-24 <= 0.017 of a unit, so |r| <= p (1/2 + 0.017): at most 64
// for |v| < 2^23 and at most 65 for |v| <= 2^24.  No correction into the balanced range is needed: the
// residue products and the reconstruction are bounded with these limits.
__device__ __forceinline__ float oz_bal_mod(float v, float p, float pinv) {
    const float q = fmaf(v, pinv, 12582912.0f) - 12582912.0f;
    return fmaf(-q, p, v);
}

// ------------------------------------------------------------------------------ slicing
struct OzSliceJob {
    const double* src;
    size_t lds;             // source row stride (elements)
    const int* rowmap;      // source row of each output row (null: the same row)
    const int* colmap;      // source column of each K index (null: the same column)
    __nv_bfloat16* dst;     // first output row of the job
    size_t ldd;             // T * Kp
    double* scale;          // 2^e per output row (NaN for a row with a non-finite entry)
    int rows, K, Kp, nb, mul_y, row0;
};

struct OzSliceBatch {
    OzSliceJob j[OZ_MAXJ];
    int njobs;
    int T;
    float p[OZ_NMOD], pinv[OZ_NMOD];
    float cA[OZ_NMOD][4], cB[OZ_NMOD][4];
};

// Row scales: one warp per operand row takes the largest magnitude over the row (through the maps), which
// fixes e (|a| 2^-e < 1/2); scale = 2^e, NaN for a row with a non-finite entry.
__global__ void __launch_bounds__(256) k_oz_rowscale(const __grid_constant__ OzSliceBatch b, int rows) {
    const int grow = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (grow >= rows) return;
    int ji = 0;
    while (ji + 1 < b.njobs && b.j[ji + 1].row0 <= grow) ++ji;
    const OzSliceJob& J = b.j[ji];
    const int row = grow - J.row0;
    const int srow = J.rowmap ? J.rowmap[row] : row;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(J.src + (size_t)srow * J.lds);
    const int* cm = J.colmap;
    unsigned long long mx = 0;
    for (int k = lane; k < J.K; k += 32) mx = max(mx, src[cm ? cm[k] : k] & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        // non-negative doubles order like their bit patterns; an all-ones exponent is Inf or NaN
        const bool bad = mx >= 0x7FF0000000000000ull;
        const int e = (bad || mx == 0) ? 0 : min(1000, max(-1000, (int)(mx >> 52) - 1023 + 2));
        J.scale[row] = bad ? __longlong_as_double(0x7ff8000000000000ll) : oz_pow2(e);
    }
}

// Residues: block (x, y) covers elements 1024 x .. 1024 x + 1023 of operand row y (rows of all jobs in
// order), four consecutive elements a thread (8-byte stores of their four bf16 residues per modulus).  The integer X = round(a 2^(nb - e)) (|X| <= 2^53) is cut into
// four base-2^14 limbs of |X|, each made an exact float through the bits of 2^23 + limb (no 64-bit
// conversion: those run on the slow FP64 unit) and given the sign of X; modulus by modulus, the residue
// is sum_l limb_l c_l (c_l = 2^(14 l) mod p_t, times y_t for a B operand; an integer below 2^23 in
// magnitude, exact in FP32) reduced by oz_bal_mod (|residue| <= 64, exact in bf16: the upper half of its
// float).  Modulus t goes to K segment t of the row.
__device__ __forceinline__ void oz_limbs(unsigned long long bits, int nb, int e, bool bad, float* L) {
    const long long X = bad ? 0 : oz_fixedb(bits, nb, e);
    const unsigned long long uX = X < 0 ? 0ull - (unsigned long long)X : (unsigned long long)X;
    const float sg = X < 0 ? -1.0f : 1.0f;
    const unsigned int lo = (unsigned int)uX, hi = (unsigned int)(uX >> 32);
    const unsigned int l0 = lo & 0x3FFF, l1 = (lo >> 14) & 0x3FFF, l2 = (lo >> 28) | ((hi & 0x3FF) << 4), l3 = hi >> 10;
    L[0] = sg * (__uint_as_float(0x4B000000u | l0) - 8388608.0f);
    L[1] = sg * (__uint_as_float(0x4B000000u | l1) - 8388608.0f);
    L[2] = sg * (__uint_as_float(0x4B000000u | l2) - 8388608.0f);
    L[3] = sg * (__uint_as_float(0x4B000000u | l3) - 8388608.0f);
}

__global__ void __launch_bounds__(256) k_oz_residue(const __grid_constant__ OzSliceBatch b) {
    const int grow = (int)blockIdx.y;
    int ji = 0;
    while (ji + 1 < b.njobs && b.j[ji + 1].row0 <= grow) ++ji;
    const OzSliceJob& J = b.j[ji];
    const int K = J.K;
    const int qi = (int)blockIdx.x * 256 + (int)threadIdx.x;
    if (qi >= (K + 3) >> 2) return;
    const int row = grow - J.row0, k = 4 * qi;
    const int srow = J.rowmap ? J.rowmap[row] : row;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(J.src + (size_t)srow * J.lds);
    const int* cm = J.colmap;
    unsigned long long v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = k + i < K ? src[cm ? cm[k + i] : k + i] : 0ull;
    const int es = (int)((__double_as_longlong(J.scale[row]) >> 52) & 0x7FF);   // 2^e, or NaN
    const bool bad = es == 0x7FF;
    float L[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) oz_limbs(v[i], J.nb, es - 1023, bad, L[i]);
    __nv_bfloat16* dst = J.dst + (size_t)row * J.ldd + k;
    const int nk = min(4, K - k);
    const float(*c)[4] = J.mul_y ? b.cB : b.cA;
    const int T = b.T;
#pragma unroll 2
    for (int t = 0; t < T; ++t, dst += J.Kp) {
        const float p = b.p[t], pinv = b.pinv[t];
        const float c0 = c[t][0], c1 = c[t][1], c2 = c[t][2], c3 = c[t][3];
        unsigned int h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)   // |r| <= 64: the bf16 of r is the upper half of its float (exact)
            h[i] = __float_as_uint(oz_bal_mod(fmaf(L[i][3], c3, fmaf(L[i][2], c2, fmaf(L[i][1], c1, L[i][0] * c0))), p, pinv));
        if (nk == 4) {
            *reinterpret_cast<uint2*>(dst) = make_uint2(__byte_perm(h[0], h[1], 0x7632), __byte_perm(h[2], h[3], 0x7632));
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < nk) reinterpret_cast<unsigned short*>(dst)[i] = (unsigned short)(h[i] >> 16);
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
                    // group gi = (modulus t, chunk c): the same K range of A and B
                    const int tm = gi / P.nch, c = gi - tm * P.nch;
                    const int ka = tm * P.kbs + c * P.cb, n = min(P.cb, P.kbs - c * P.cb);
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
                            tma_load_2d_pair(sB + s * B_BYTES, &b.tmB[pi], (ka + kb) * KELEM, n0, full0 + 8u * s);
                        } else {
                            mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                            tma_load_2d(sA + s * A_BYTES, &b.tmA[pi], (ka + kb) * KELEM, m0, &full[s]);
                            tma_load_2d(sB + s * B_BYTES, &b.tmB[pi], (ka + kb) * KELEM, n0, &full[s]);
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
                    const int c = gi % P.nch;
                    const int n = min(P.cb, P.kbs - c * P.cb);
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
            // 16- or 8-byte stores of a row's 32 residues when the row starts on such a boundary
            const int vec = (reinterpret_cast<uintptr_t>(P.stage) & 15) ? 0 : (P.N & 15) == 0 ? 16 : (P.N & 7) == 0 ? 8 : 0;
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
                const int tm = gi / P.nch;
                const float pm = b.mods.p[tm], pinv = b.mods.pinv[tm];
                // the chunk sum is an integer of magnitude at most 2^24 (exact in FP32); its residue w modulo
                // p_t (|w| <= 65) goes out as the byte w + 128 (the low byte of the float w + 128 + 1.5 * 2^23)
                unsigned char* srow = P.stage + (size_t)gi * P.M * P.N + (size_t)(rok ? row : 0) * P.N;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t v[32];
                    __syncwarp();
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + c * 32), v);   // warp-collective
                    const int col0 = n0 + c * 32;
                    if (!rok || col0 >= P.N) continue;
                    uint32_t wd[8];
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        uint32_t x[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            x[i] = __float_as_uint(oz_bal_mod(__uint_as_float(v[j + i]), pm, pinv) + 12583040.0f);
                        wd[j / 4] = __byte_perm(__byte_perm(x[0], x[1], 0x0040), __byte_perm(x[2], x[3], 0x0040), 0x5410);
                    }
                    if (col0 + 32 <= P.N && vec == 16) {
                        *reinterpret_cast<uint4*>(srow + col0) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                        *reinterpret_cast<uint4*>(srow + col0 + 16) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
                    } else if (col0 + 32 <= P.N && vec == 8) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) *reinterpret_cast<uint2*>(srow + col0 + 8 * j) = make_uint2(wd[2 * j], wd[2 * j + 1]);
                    } else {
                        const int nc = min(32, P.N - col0);
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nc) srow[col0 + j] = (unsigned char)((wd[j / 4] >> (8 * (j & 3))) & 0xFF);
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

// --------------------------------------------------------------------------- reconstruction
// s = sum_t w_t (P / p_t) is accumulated in NL float limb sums of weight 2^(LB l): each is a sum of w_t
// times a limb of P / p_t below 2^LB, so with T <= 19 it stays an integer below 2^22 in magnitude
// (|w_t| <= 130 with two chunks and 10-bit limbs: 2^21.3; |w_t| <= 65 with one chunk and 11-bit limbs:
// 2^21.3) -- exact, and within the range of the float-to-int step below.

// x = s - round(s / P) P from the limb sums, rounded once to FP64 and scaled by 2^ex.  The product lies
// within P / 4 of zero, so q needs s / P to within 1/4: the estimate is summed from the limb sums as they
// are (each a sum of w_t times non-negative limbs of P / p_t, so the float rounding errors stay near
// 2^-20 sum_t |w_t| / p_t of s / P).  x's limbs (integers below 2^22) become int32 through the float
// 1.5 * 2^23 + x, carries normalise them to [0, 2^LB) under a signed top limb, the value is assembled
// modulo 2^128 (|x| < 2^123), and a negative x is negated as a 128-bit two's complement.
template <int LB, int NL>
__device__ __forceinline__ double oz_crt_value(const float* a, const float* Pl, float pinvs, int ex) {
    float sf = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) sf = fmaf(a[l], __int_as_float((127 + LB * l - 120) << 23), sf);   // s 2^-120
    const float q = fmaf(sf, pinvs, 12582912.0f) - 12582912.0f;
    int x[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) x[l] = __float_as_int(fmaf(-q, Pl[l], a[l]) + 12582912.0f) - 0x4B400000;
    int c = x[0];
#pragma unroll
    for (int l = 0; l < NL - 1; ++l) {
        const int cl = c;
        x[l] = cl & ((1 << LB) - 1);
        c = (cl >> LB) + x[l + 1];   // arithmetic shift: floor
    }
    typedef unsigned long long u64;
    u64 lo = 0, hi = 0;
#pragma unroll
    for (int l = 0; l < NL - 1; ++l) {   // limbs in [0, 2^LB) at bit LB l
        const int pos = LB * l;
        const u64 v = (u64)(unsigned int)x[l];
        if (pos < 64) {
            lo |= v << pos;
            if (pos + LB > 64) hi |= v >> (64 - pos);
        } else if (pos < 128) {
            hi |= v << (pos - 64);
        }
    }
    constexpr int TOP = LB * (NL - 1);   // the signed top limb c: sign-extended, modulo 2^128
    if constexpr (TOP < 128) hi |= (u64)(long long)c << (TOP - 64);
    if (c < 0) {   // |x| = -(the assembled value) modulo 2^128, since |x| < 2^128
        const u64 nlo = 0ull - lo;
        hi = ~hi + (lo == 0 ? 1ull : 0ull);
        return oz_u128_scaled(hi, nlo, true, ex);
    }
    return oz_u128_scaled(hi, lo, false, ex);
}

// The constants of the reconstruction, passed as a kernel parameter: with the modulus and limb loops
// unrolled, every limb of P / p_t is an immediate constant-bank operand of its FMA (no load).
struct OzCrtParams {
    float q10[OZ_NMOD][OZ_NL2];
    float P10[OZ_NL2];
    float q11[OZ_NMOD][OZ_NL1];
    float P11[OZ_NL1];
    float pinvs;
    int T;
};

// Two consecutive elements of one row per thread (16-bit loads of their residue bytes when N is even):
// every residue word of the element pair (all moduli and chunks) is loaded before any is used, so that
// about 2 KB per warp is in flight.  A byte b = w + 128 becomes the float 2^23 + b by a byte permute
// (exact), so w = that - (2^23 + 128).
template <int NCH, int VW>
__device__ __forceinline__ void oz_crt_rows(const OzProb& P, const OzCrtParams& cp) {
    constexpr int LB = NCH == 1 ? OZ_LB1 : OZ_LB2, NL = NCH == 1 ? OZ_NL1 : OZ_NL2;
    const float(*qt)[NL] = NCH == 1 ? (const float(*)[NL])cp.q11 : (const float(*)[NL])cp.q10;
    const float* Pl = NCH == 1 ? cp.P11 : cp.P10;
    const int T = cp.T, N = P.N;
    const size_t MN = (size_t)P.M * N;
    const size_t nunit = MN / VW;
    for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunit; u += (size_t)gridDim.x * blockDim.x) {
        const size_t e = u * VW;
        const unsigned char* __restrict__ sp = P.stage + e;
        unsigned int xw[OZ_NMOD][NCH];
#pragma unroll
        for (int t = 0; t < OZ_NMOD; ++t)
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                xw[t][c] = 0x8080u;   // w = 0 past the last modulus
                if (t < T) {
                    xw[t][c] = VW == 2 ? (unsigned int)__ldg(reinterpret_cast<const unsigned short*>(sp)) : (unsigned int)__ldg(sp);
                    sp += MN;
                }
            }
        float acc[VW][NL];
#pragma unroll
        for (int k = 0; k < VW; ++k)
#pragma unroll
            for (int l = 0; l < NL; ++l) acc[k][l] = 0.0f;
#pragma unroll
        for (int t = 0; t < OZ_NMOD; ++t) {
            if (t >= T) break;
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                float w = 0.0f;
#pragma unroll
                for (int c = 0; c < NCH; ++c) w += __uint_as_float(__byte_perm(xw[t][c], 0x4B000000u, 0x7540u | k)) - 8388736.0f;
#pragma unroll
                for (int l = 0; l < NL; ++l) acc[k][l] = fmaf(w, qt[t][l], acc[k][l]);
            }
        }
        const int i = (int)(e / N), j0 = (int)(e - (size_t)i * N);
        const int ea = (int)((__double_as_longlong(P.sa[i]) >> 52) & 0x7FF);   // row scales are powers of two
        double* crow = P.C + (size_t)i * P.ldc;
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const int eb = (int)((__double_as_longlong(P.sb[j0 + k]) >> 52) & 0x7FF);
            const double v = (ea == 0x7FF || eb == 0x7FF)
                                 ? __longlong_as_double(0x7ff8000000000000ll)
                                 : oz_crt_value<LB, NL>(acc[k], Pl, cp.pinvs, ea + eb - 2046 + P.ealpha - 2 * P.nb);
            crow[j0 + k] = P.accum ? crow[j0 + k] + v : v;
        }
    }
}

// C = alpha 2^(e_i + e_j - 2 nb) x for every element, x rebuilt from the staged residues.  The residues of
// an element are read once, coalesced, and C is written once.
__global__ void __launch_bounds__(256, OZ_CRT_MINB) k_oz_crt(const OzBatch* __restrict__ bp, const __grid_constant__ OzCrtParams cp) {
    const OzProb& P = bp->p[blockIdx.y];
    const bool v2 = (P.N & 1) == 0;
    if (P.nch == 1) v2 ? oz_crt_rows<1, 2>(P, cp) : oz_crt_rows<1, 1>(P, cp);
    else v2 ? oz_crt_rows<2, 2>(P, cp) : oz_crt_rows<2, 1>(P, cp);
}

// The reconstruction launch of a plan.
static int oz_launch_crt(const OzBatch* host, const OzBatch* dev, int nsm, cudaStream_t st) {
    OzCrtParams cp;
    memset(&cp, 0, sizeof(cp));
    const OzMods& m = host->mods;
    cp.T = m.T;
    memcpy(cp.q10, m.q10, sizeof(cp.q10));
    memcpy(cp.P10, m.P10, sizeof(cp.P10));
    memcpy(cp.q11, m.q11, sizeof(cp.q11));
    memcpy(cp.P11, m.P11, sizeof(cp.P11));
    cp.pinvs = m.pinvs;
    k_oz_crt<<<dim3(2 * nsm, host->nprob), 256, 0, st>>>(dev, cp);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
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
    int nb;             // rows rounded to X = round(a 2^(nb - e)), |X| <= 2^(nb-1)
};

struct OzPlan {
    OzBatch* host;
    OzBatch* dev;
    int S, bn;
    int bits;           // bits kept below a row's leading bit: min(6S, 53)
    unsigned __int128 P;   // product of the plan's moduli
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

// The moduli of a plan: the least T whose product P covers 4 Kmax 2^(2 bits) (every product of the plan
// then lies within P / 4 of zero), at most the whole list, and the exact constants of the set.
static int oz_mods_init(OzPlan* pl, int S, long long Kmax) {
    const int bt = 6 * S < 53 ? 6 * S : 53;
    if (Kmax < 1) Kmax = 1;
    if (Kmax > (1ll << 18)) return ACSE_ERR_SHAPE;
    pl->bits = bt;
    const unsigned __int128 need = (unsigned __int128)Kmax << (2 * bt + 2);   // below 2^126
    unsigned __int128 P = 1;
    int T = 0;
    while (T < OZ_NMOD && P < need) P *= (unsigned __int128)oz_moduli[T++];
    pl->P = P;
    OzMods& m = pl->host->mods;
    memset(&m, 0, sizeof(m));
    m.T = T;
    const unsigned __int128 m10 = ((unsigned __int128)1 << OZ_LB2) - 1, m11 = ((unsigned __int128)1 << OZ_LB1) - 1;
    for (int t = 0; t < T; ++t) {
        const int pt = oz_moduli[t];
        const unsigned __int128 Q = P / (unsigned __int128)pt;
        const int qm = (int)(Q % (unsigned __int128)pt);
        int y = 1;
        while (y < pt && (qm * y) % pt != 1) ++y;   // pairwise coprime: the inverse exists
        m.p[t] = (float)pt;
        m.pinv[t] = 1.0f / (float)pt;
        for (int l = 0; l < 4; ++l) {
            const long long cl = (1ll << (14 * l)) % pt;
            m.cA[t][l] = (float)cl;
            m.cB[t][l] = (float)((cl * y) % pt);
        }
        for (int l = 0; l < OZ_NL2; ++l) m.q10[t][l] = (float)(int)((Q >> (OZ_LB2 * l)) & m10);
        for (int l = 0; l < OZ_NL1; ++l) m.q11[t][l] = (float)(int)((Q >> (OZ_LB1 * l)) & m11);
    }
    for (int l = 0; l < OZ_NL2; ++l) m.P10[l] = (float)(int)((P >> (OZ_LB2 * l)) & m10);
    for (int l = 0; l < OZ_NL1; ++l) m.P11[l] = (float)(int)((P >> (OZ_LB1 * l)) & m11);
    m.pinvs = (float)(ldexp(1.0, 120) / (double)P);
    return ACSE_OK;
}

// nb of an operand of contraction length K: the largest b <= bits with 4 K 2^(2b) <= P, plus one.
static int oz_op_nb(const OzPlan* pl, int K) {
    int b = pl->bits;
    while (b > 0 && ((unsigned __int128)K << (2 * b + 2)) > pl->P) --b;
    return b + 1;
}

static int oz_op_alloc(OzPlan* pl, OzOp& o, int rows, int K) {
    o.rows = rows;
    o.K = K;
    o.Kp = (K + 63) / 64 * 64;
    o.nb = oz_op_nb(pl, K);
    if (o.nb < 2) return ACSE_ERR_SHAPE;
    const size_t bytes = (size_t)rows * pl->host->mods.T * o.Kp * sizeof(__nv_bfloat16);
    if (cudaMalloc((void**)&o.sl, bytes) != cudaSuccess || cudaMalloc((void**)&o.scale, rows * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_NOMEM;
    }
    ACSE_CUDA_TRY(cudaMemset(o.sl, 0, bytes));   // the K padding of every segment stays zero
    return ACSE_OK;
}

static int oz_add(OzPlan* pl, const OzOp& a, const OzOp& b, double* C, int ldc, double alpha) {
    OzBatch& B = *pl->host;
    if (B.nprob >= OZ_MAXP || a.K != b.K || a.Kp != b.Kp || a.nb != b.nb) return ACSE_ERR_SHAPE;
    const int n = B.nprob;
    const size_t ld = (size_t)B.mods.T * a.Kp;
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
    p.nb = a.nb;
    // chunks of at most OZ_CHUNK_KB blocks: every partial sum of residue products stays below 2^24
    p.nch = (p.kbs + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;
    if (p.nch > OZ_MAXCH) return ACSE_ERR_SHAPE;
    p.cb = (p.kbs + p.nch - 1) / p.nch;
    p.ngroups = B.mods.T * p.nch;
    if (cudaMalloc((void**)&p.stage, (size_t)p.ngroups * p.M * p.N) != cudaSuccess) {
        cudaGetLastError();
        p.stage = nullptr;
        return ACSE_ERR_NOMEM;
    }
    p.tiles_n = (p.N + pl->bn - 1) / pl->bn;
    p.tile_start = B.total_tiles;
    B.total_tiles += ((p.M + pl->bm - 1) / pl->bm) * p.tiles_n;
    B.nprob = n + 1;
    return ACSE_OK;
}

static int oz_plan_finish(OzPlan* pl);

// Kernel attributes, SM count, the moduli for the plan's longest contraction Kmax and the zeroed problem
// table of a plan.
static int oz_plan_init(OzPlan* pl, int S, int bn, int pair, long long Kmax) {
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
    pl->host->wait_ns = OZ_WAIT_NS;
    return oz_mods_init(pl, S, Kmax);
}

// The plan figures of one GEMM, on the host only (acse_ozaki_plan_info in include/acse.h).
extern "C" int acse_ozaki_plan_info(int oz_slices, int kmax, int k, int* moduli_count, int* bits, int* chunks,
                                    int* moduli) {
    if (oz_slices < 4 || oz_slices > 10 || kmax < 1 || kmax > 8192 || k < 1 || k > kmax) return ACSE_ERR_ARG;
    OzPlan pl;
    memset(&pl, 0, sizeof(pl));
    pl.host = (OzBatch*)calloc(1, sizeof(OzBatch));
    if (!pl.host) return ACSE_ERR_NOMEM;
    const int st = oz_mods_init(&pl, oz_slices, kmax);
    if (st == ACSE_OK) {
        const int T = pl.host->mods.T, kbs = (k + 63) / 64;
        if (moduli_count) *moduli_count = T;
        if (bits) *bits = oz_op_nb(&pl, k) - 1;
        if (chunks) *chunks = (kbs + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;
        if (moduli)
            for (int t = 0; t < T; ++t) moduli[t] = oz_moduli[t];
    }
    free(pl.host);
    return st;
}

int oz_plan_create(acse_ctx* c) {
    OzPlan* pl = (OzPlan*)calloc(1, sizeof(OzPlan));
    if (!pl) return ACSE_ERR_NOMEM;
    c->oz_plan = pl;
    const int r = c->r, R2 = r * r, R22 = 2 * R2, P = r * (r - 1) / 2;
    ACSE_TRY(oz_plan_init(pl, c->opt.oz_slices, R2 >= 256 ? OZ_BN : 128, c->opt.gemm_tile != 1, R22));
    // the B products on the tensor cores (acse_zoz.cu): x1 and x2^T of the four types for every pair
    if (r % 16 == 0 && r <= 64 && c->opt.oz_slices <= 8)
        for (int k = 0; k < 8; ++k)
            if (cudaMalloc((void**)&c->w.bx64[k], (size_t)R2 * R2 * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                c->w.bx64[k] = nullptr;
                return ACSE_ERR_NOMEM;
            }
    ACSE_TRY(oz_op_alloc(pl, pl->A[0], 2 * P, P));
    ACSE_TRY(oz_op_alloc(pl, pl->A[1], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->A[2], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->A[3], 2 * P, P));
    ACSE_TRY(oz_op_alloc(pl, pl->A[4], R22, R22));
    ACSE_TRY(oz_op_alloc(pl, pl->A[5], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->A[6], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->B[0], P, P));
    ACSE_TRY(oz_op_alloc(pl, pl->B[1], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->B[2], P, P));
    ACSE_TRY(oz_op_alloc(pl, pl->B[3], R22, R22));
    ACSE_TRY(oz_op_alloc(pl, pl->B[4], R2, R2));
    ACSE_TRY(oz_op_alloc(pl, pl->B[5], R2, R2));
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
        const int nmod = B.mods.T;
        int* hs = (int*)malloc((size_t)(T + G + 1) * sizeof(int));
        long long* cost = (long long*)malloc((size_t)T * sizeof(long long));
        if (!hs || !cost) {
            free(hs);
            free(cost);
            return ACSE_ERR_NOMEM;
        }
        for (int p = 0; p < B.nprob; ++p) {
            const int n = ((B.p[p].M + pl->bm - 1) / pl->bm) * B.p[p].tiles_n;
            for (int k = 0; k < n; ++k) cost[B.p[p].tile_start + k] = (long long)nmod * B.p[p].kbs + 4 * B.p[p].ngroups;
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

// The moduli constants of a slicing launch.
static void oz_slice_batch_init(OzSliceBatch& b, const OzMods& m) {
    memset(&b, 0, sizeof(b));
    b.T = m.T;
    for (int t = 0; t < m.T; ++t) {
        b.p[t] = m.p[t];
        b.pinv[t] = m.pinv[t];
        for (int l = 0; l < 4; ++l) {
            b.cA[t][l] = m.cA[t][l];
            b.cB[t][l] = m.cB[t][l];
        }
    }
}

// One slicing job: `rows` rows of operand o starting at output row `orow`, read from src (row stride
// lds) through the optional row / column maps; mul_y for a B operand (residues times y_t).
static void oz_job(OzSliceBatch& b, int& rows, const OzOp& o, int orow, int nrows, const double* src, size_t lds,
                   const int* rowmap, const int* colmap, int mul_y) {
    OzSliceJob& j = b.j[b.njobs++];
    j.src = src;
    j.lds = lds;
    j.rowmap = rowmap;
    j.colmap = colmap;
    j.ldd = (size_t)b.T * o.Kp;
    j.dst = o.sl + (size_t)orow * j.ldd;
    j.scale = o.scale + orow;
    j.rows = nrows;
    j.K = o.K;
    j.Kp = o.Kp;
    j.nb = o.nb;
    j.mul_y = mul_y;
    j.row0 = rows;
    rows += nrows;
}

// Launch the slicing of every job of `all`: the row scales (a warp per row), then the residues (a
// block row per operand row, 1024 elements a block).
static int oz_slice_launch(acse_ctx* c, const OzSliceBatch& all, int rows) {
    if (all.njobs == 0 || rows == 0) return ACSE_OK;
    if (rows > 65535) return ACSE_ERR_SHAPE;
    k_oz_rowscale<<<(rows + 7) / 8, 256, 0, c->stream>>>(all, rows);
    ACSE_LAUNCHED(c);
    int maxq = 1;
    for (int i = 0; i < all.njobs; ++i) maxq = (all.j[i].K + 3) / 4 > maxq ? (all.j[i].K + 3) / 4 : maxq;
    k_oz_residue<<<dim3((maxq + 255) / 256, rows), 256, 0, c->stream>>>(all);
    ACSE_LAUNCHED(c);
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
    oz_slice_batch_init(b, pl->host->mods);
    int rows = 0;
    const int* pm = pl->pmap;
    // A residues as they are, B residues times y_t
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
    return oz_slice_launch(c, b, rows);
}

int oz_gemm_launch(acse_ctx* c) {
    OzPlan* pl = (OzPlan*)c->oz_plan;
    if (!pl) return ACSE_ERR_UNSUPPORTED;
    if (pl->tiles == 0) return ACSE_OK;
    ACSE_TRY(prof_begin(c));
    ACSE_TRY(oz_launch_gemm(pl, c->stream));
    ACSE_LAUNCHED(c);
    ACSE_TRY(oz_launch_crt(pl->host, pl->dev, pl->nsm, c->stream));
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
// and residue staging stay until the context is destroyed); a later call whose shapes differ from
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
    long long maxK = 1;
    for (int i = 0; i < n; ++i) maxK = g[i].K > maxK ? g[i].K : maxK;
    ACSE_TRY(oz_plan_init(pl, root->S, maxN >= 256 ? OZ_BN : 128, root->pair, maxK));
    pl->host->err = root->err;
    for (int i = 0; i < n; ++i) {
        ACSE_TRY(oz_op_alloc(pl, pl->A[i], g[i].M, g[i].K));
        ACSE_TRY(oz_op_alloc(pl, pl->B[i], g[i].N, g[i].K));
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
    // residues of every operand (B times y_t), at most OZ_MAXJ jobs a launch
    OzSliceBatch sb;
    oz_slice_batch_init(sb, B.mods);
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
                ACSE_TRY(oz_slice_launch(c, sb, rows));
                oz_slice_batch_init(sb, B.mods);
                rows = 0;
            }
        }
    }
    ACSE_TRY(oz_slice_launch(c, sb, rows));
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
    ACSE_TRY(oz_launch_crt(&B, pl->dev, pl->nsm, c->stream));
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}
