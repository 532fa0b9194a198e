// Z = 1D . W_kp on the tensor cores in an FP64-accurate (Ozaki) context: the O(r^5) particle-hole operand
// of a contraction pass, Z^{kp}_{js} = sum_q W^{kp}_{qs} 1D^j_q, by the error-free splitting of the Ozaki
// scheme (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012) that gemm_oz.cu applies to the O(r^6)
// GEMMs, instead of double-float FMAs on the CUDA cores.
//
// Tile: 128 consecutive (p, s) of one (spin type, k), rows m = p r + s, as in acse_ztc.cu:
//     Z[m][j] = sum_q A[m][q] B[j][q],   A[m][q] = W_kp[q][s] (FP64),  B[j][q] = 1D[j][q] (FP64).
// Every row of A and of B gets a power-of-two scale 2^e (|x| 2^-e < 1/2 over the row) and each element the
// fixed-point value X = round(x 2^(6S - e)), cut into S balanced base-64 digits (most significant first,
// each exact in bf16).  The digit tiles A_s, B_t sit in shared memory in the 128-byte-swizzled K-major
// layout (K = q, one 64-element block); the products of one level L = s + t <= S + 1 are accumulated in
// FP32 in their own TMEM accumulator (columns (L - 2) r .. (L - 1) r): a level holds at most S products
// of K <= 64 terms of magnitude <= 2^10, below 2^24, so every level sum is an exact integer.  The epilogue
// adds the levels exactly in int64 (sum_L v_L 2^(6 (S + 1 - L)), below 2^61 for S <= 8) and rounds once
// to FP64, scaled by 2^(e_m + e_j - 6 (S + 1)).  The levels dropped (s + t > S + 1) and the fixed-point
// rounding leave an error of order 2^-6S of |A_m| |B_j| r, that of the Ozaki GEMMs.
//
// One block per SM (the S digit tiles of A and B take up to 192 KB of shared memory) walks a contiguous
// range of tiles; the B tiles are rebuilt only when the spin of the tile's 1D changes.  Producer: four
// threads per A row (partners in one warp share the row maximum); one thread issues the MMAs; epilogue:
// each warp reads its TMEM lane quarter (one row m per thread) for a quarter of the columns j and writes the
// FP64 rows of Zd / Zf (row (sK, k, j), column (sP, p, s)) and the diagonal rows j = p of w.  The wait for
// the MMAs is bounded; on expiry the kernel raises the device flag and stops.  Used for r a multiple of
// 16 (r <= 64) and S <= 8; other cases take the double-float kernel of acse_tiled.cu.
#include <cuda_bf16.h>

#include "acse_internal.h"
#include "oz_arith.cuh"
#include "tc_ptx.cuh"

#define ZOZ_THREADS 512                  // four threads per A row; four warps per TMEM lane quarter
#define ZOZ_TPR (ZOZ_THREADS / TC_BM)
#define ZOZ_SMAX 8                       // digit slices this kernel holds
#define ZOZ_A_SLICE (TC_BM * 128)        // one digit tile of A: 128 rows x 128 bytes
#define ZOZ_WAIT_NS 4000000000ull

struct ZozArgs {
    const double* W[3];     // FP64 W blocks aa, ab, bb (r^4 each)
    const double* gam;      // 1D per spin [2][r][r]
    double* Zd;             // (2 r^2) rows of ldd doubles
    double* Zf[2];          // r^2 rows of ldf doubles
    double* diag;           // [4][r][r][r]: rows j = p of Zd(a,a), Zd(b,b), Zf1, Zf2
    int ldd, ldf;
    int tmap[6];            // block type index -> spin type t
    int S;                  // slices (<= ZOZ_SMAX)
    int* err;
};

static __device__ __forceinline__ uint32_t zoz_sw128(int n, int c) {
    return (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) << 4);
}

// Row scale from the largest magnitude's bit pattern (non-negative doubles order like their bits): e with
// |x| 2^-e < 1/2, 0 for an all-zero row, ZOZ_BAD for a row holding Inf or NaN.
#define ZOZ_BAD 0x7FFF
static __device__ __forceinline__ int zoz_row_exp(unsigned long long mx) {
    if (mx >= 0x7FF0000000000000ull) return ZOZ_BAD;
    if (mx == 0) return 0;
    return min(1000, max(-1000, (int)(mx >> 52) - 1023 + 2));
}

// The S digits of the eight elements x[0..7] (scale e) as bf16, written to the 16-byte chunk `off` of the
// S digit tiles at base, base + stride, ...: digit tile s - 1 holds digit s (most significant first).
// Balanced base-64 digits from the least significant one up: d = ((X + 32) mod 64) - 32, X <- (X - d) / 64;
// the last quotient is the leading digit (|d| <= 32).
static __device__ __forceinline__ void zoz_digits8(const unsigned long long (&x)[8], int e, int S, uint8_t* base,
                                                   uint32_t stride, uint32_t off, const unsigned short* tab) {
    long long X[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) X[u] = (e == ZOZ_BAD) ? 0 : oz_fixed(x[u], S, e);
    for (int t = 0; t < S; ++t) {   // digit s = S - t
        unsigned short h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            int d;
            if (t < S - 1) {
                d = (int)(((X[u] + 32) & 63) - 32);
                X[u] = (X[u] - d) >> 6;
            } else {
                d = (int)X[u];
            }
            h[u] = tab[d + 32];
        }
        uint4 v;
        v.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
        v.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
        v.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
        v.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
        *reinterpret_cast<uint4*>(base + (size_t)(S - t - 1) * stride + off) = v;
    }
}

static __device__ __forceinline__ void zoz_tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr));
}

template <int R>
__global__ void __launch_bounds__(ZOZ_THREADS, 1) k_Z_oz(const __grid_constant__ ZozArgs a, int ntiles) {
    static_assert(R % 16 == 0 && R <= 64, "N = r a multiple of 16, K = r within one 64-element block");
    constexpr int R2 = R * R, NT = R2 / TC_BM, NCH = R / 8;   // 16-byte chunks of a digit row
    static_assert(R2 % TC_BM == 0, "whole tiles");
    constexpr int B_SLICE = R * 128;                            // one digit tile of B: R rows x 128 B
    const int S = a.S;
    extern __shared__ uint8_t zo_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)zo_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                         // [S][128 x 128 B]
    uint8_t* sB = sA + ZOZ_SMAX * ZOZ_A_SLICE;                  // [S][R x 128 B]
    int* eA = reinterpret_cast<int*>(sB + ZOZ_SMAX * B_SLICE);  // row scales of the A tile [128]
    int* eB = eA + TC_BM;                                       // row scales of B [64]
    unsigned short* tab = reinterpret_cast<unsigned short*>(eB + 64);   // bf16 of the digits -32 .. 32
    uint64_t* bar = reinterpret_cast<uint64_t*>(tab + 72);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t r3 = (size_t)R * R2;
    if (threadIdx.x < 65) tab[threadIdx.x] = __bfloat16_as_ushort(__float2bfloat16_rn((float)((int)threadIdx.x - 32)));
    // the K padding q >= R of every digit tile stays zero
    for (int e = threadIdx.x; e < (ZOZ_SMAX * ZOZ_A_SLICE + ZOZ_SMAX * B_SLICE) / 16; e += ZOZ_THREADS)
        reinterpret_cast<uint4*>(sA)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    uint32_t phase = 0;
    int cur_sp = -1;
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_end = min(ntiles, ((int)blockIdx.x + 1) * per);
    for (int tile = (int)blockIdx.x * per; tile < t_end && ok; ++tile, phase ^= 1) {
        const int tb = tile / (R * NT);
        const int t = a.tmap[tb];
        const int rem = tile - tb * R * NT;
        const int k = rem / NT;
        const int m0 = (rem - k * NT) * TC_BM;
        const int sp = (t == 2 || t == 3 || t == 4) ? 1 : 0;
        if (sp != cur_sp) {   // B: the digits of 1D of this tile's spin, rows j, K = q (the last MMAs are done)
            const unsigned long long* g = reinterpret_cast<const unsigned long long*>(a.gam + (size_t)sp * R2);
            for (int j = threadIdx.x; j < R; j += ZOZ_THREADS) {
                unsigned long long mx = 0;
                for (int q = 0; q < R; ++q) mx = max(mx, g[j * R + q] & 0x7FFFFFFFFFFFFFFFull);
                eB[j] = zoz_row_exp(mx);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < R * NCH; e += ZOZ_THREADS) {
                const int j = e / NCH, c = e - j * NCH;
                unsigned long long x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = g[j * R + 8 * c + u];
                zoz_digits8(x, eB[j], S, sB, B_SLICE, zoz_sw128(j, c), tab);
            }
            cur_sp = sp;
        }
        // A: row m = p r + s of W_k^T, K = q: W_kp[q][s] of type t (see k_Z_pipe); ZOZ_TPR threads per row
        {
            const int ml = threadIdx.x / ZOZ_TPR, half = threadIdx.x % ZOZ_TPR, m = m0 + ml;
            const int p = m / R, s = m - p * R;
            const double* base;
            bool tr;
            switch (t) {
                case 0: tr = false; base = a.W[0] + k * r3 + (size_t)p * R2; break;
                case 1: tr = false; base = a.W[1] + k * r3 + (size_t)p * R2; break;
                case 2: tr = true; base = a.W[1] + (size_t)p * r3 + (size_t)k * R2; break;
                case 3: tr = false; base = a.W[2] + k * r3 + (size_t)p * R2; break;
                case 4: tr = true; base = a.W[1] + k * r3 + (size_t)p * R2; break;
                default: tr = false; base = a.W[1] + (size_t)p * r3 + (size_t)k * R2; break;
            }
            const unsigned long long* b64 = reinterpret_cast<const unsigned long long*>(base);
            constexpr int MYCH = (NCH + ZOZ_TPR - 1) / ZOZ_TPR;   // chunks c = half, half + TPR, ... of this thread
            unsigned long long x[MYCH][8];
            unsigned long long mx = 0;
#pragma unroll
            for (int i = 0; i < MYCH; ++i) {
                const int c = ZOZ_TPR * i + half;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = 8 * c + u;
                    x[i][u] = c < NCH ? (tr ? b64[(size_t)s * R + q] : b64[(size_t)q * R + s]) : 0ull;
                    mx = max(mx, x[i][u] & 0x7FFFFFFFFFFFFFFFull);
                }
            }
#pragma unroll
            for (int o = 1; o < ZOZ_TPR; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int e = zoz_row_exp(mx);
            if (half == 0) eA[ml] = e;
#pragma unroll
            for (int i = 0; i < MYCH; ++i) {
                const int c = ZOZ_TPR * i + half;
                if (c < NCH) zoz_digits8(x[i], e, S, sA, ZOZ_A_SLICE, zoz_sw128(ml, c), tab);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc<0, R>();
            for (int L = 2; L <= S + 1; ++L) {
                const uint32_t acc = tmem + (uint32_t)((L - 2) * R);
                bool first = true;
                for (int sa = max(1, L - S); sa <= min(S, L - 1); ++sa) {
                    const uint64_t da = smem_desc(sA + (size_t)(sa - 1) * ZOZ_A_SLICE);
                    const uint64_t db = smem_desc(sB + (size_t)(L - sa - 1) * B_SLICE);
#pragma unroll
                    for (int kk = 0; kk < R / 16; ++kk) {
                        umma<0>(acc, da + 2 * kk, db + 2 * kk, idesc, first ? 0u : 1u);
                        first = false;
                    }
                }
            }
            umma_commit(bar);
        }
        ok = __syncthreads_and(bounded_wait(bar, phase, ZOZ_WAIT_NS, nullptr)) != 0;
        if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        tc_fence_after();
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows m) for its share of the columns j
        {
            constexpr int NJG = ZOZ_THREADS / 128, JW = R / NJG;   // warps per lane quarter, columns each
            static_assert(JW % 4 == 0, "whole groups of four columns");
            const int q4 = warp & 3, jh = warp >> 2;
            const int ml = q4 * 32 + lane, m = m0 + ml;
            const int p = m / R, s = m - p * R;
            const int em = eA[ml];
            int which, sK, sP;
            if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
            else { which = t - 4; sK = 0; sP = 0; }
            const int dslot = t == 0 ? 0 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : -1;
            double* zb = which < 0 ? a.Zd : a.Zf[which];
            const size_t ld = which < 0 ? (size_t)a.ldd : (size_t)a.ldf;
            const size_t col = (size_t)sP * R2 + m;
            for (int j0 = jh * JW; j0 < (jh + 1) * JW; j0 += 4) {
                long long acc[4] = {0, 0, 0, 0};
                for (int L = 2; L <= S + 1; ++L) {
                    uint32_t v[4];
                    __syncwarp();
                    zoz_tmem_ld4(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((L - 2) * R + j0), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int sh = 6 * (S + 1 - L);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[jj] += (long long)__float2int_rn(__uint_as_float(v[jj])) * (1ll << sh);
                }
                if (!ok) continue;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = j0 + jj;
                    const int ej = eB[j];
                    const double z = (em == ZOZ_BAD || ej == ZOZ_BAD) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                      : oz_ll_scaled(acc[jj], em + ej - 6 * (S + 1));
                    zb[((size_t)sK * R2 + (size_t)k * R + j) * ld + col] = z;
                    if (dslot >= 0 && j == p) a.diag[(((size_t)dslot * R2 + (size_t)k * R + p) * R) + s] = z;
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM read and the A tiles free before the next tile's digits and MMAs
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int R>
static int zoz_launch(const ZozArgs& a, int ntypes, cudaStream_t st) {
    constexpr int R2 = R * R, NT = R2 / TC_BM;
    const size_t smem = 1024 + (size_t)ZOZ_SMAX * ZOZ_A_SLICE + (size_t)ZOZ_SMAX * R * 128 + 4 * (TC_BM + 64) + 2 * 72 + 64;
    static int nsm = 0;
    if (!nsm) {
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_oz<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0;
        ACSE_CUDA_TRY(cudaGetDevice(&dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const int ntiles = ntypes * R * NT;
    const int grid = ntiles < nsm ? ntiles : nsm;
    k_Z_oz<R><<<grid, ZOZ_THREADS, smem, st>>>(a, ntiles);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

// Z (FP64 rows of Zd, Zf) and the diagonal rows of w on the tensor cores for an Ozaki context with r a
// multiple of 16 (r <= 64) and at most 8 slices; ACSE_ERR_UNSUPPORTED otherwise (the caller then runs
// the double-float kernel).
int launch_Z_oz(acse_ctx* c, const double* const W[3], int ntypes, const int* tmap) {
    const int r = c->r;
    if (!c->oz || r % 16 != 0 || r > 64 || c->opt.oz_slices > ZOZ_SMAX) return ACSE_ERR_UNSUPPORTED;
    Work& w = c->w;
    ZozArgs a;
    for (int s = 0; s < 3; ++s) a.W[s] = W[s];
    a.gam = w.gam;
    a.Zd = w.Zd;
    a.Zf[0] = w.Zf1;
    a.Zf[1] = w.Zf2;
    a.diag = w.zdiag;
    a.ldd = 2 * r * r;
    a.ldf = r * r;
    for (int i = 0; i < 6; ++i) a.tmap[i] = tmap[i];
    a.S = c->opt.oz_slices;
    a.err = c->w.tc_err;
    int s;
    switch (r) {
        case 16: s = zoz_launch<16>(a, ntypes, c->stream); break;
        case 32: s = zoz_launch<32>(a, ntypes, c->stream); break;
        case 48: s = zoz_launch<48>(a, ntypes, c->stream); break;
        default: s = zoz_launch<64>(a, ntypes, c->stream); break;
    }
    if (s == ACSE_OK) c->launches++;
    return s;
}

// ---------------------------------------------------------------------------------- B products
// The two r x r x r products of every B spin type in an Ozaki context, for every pair (i, j) (the B kernel
// of the FP64 paths, k_B_tiled, walks all r^2 pairs):
//     x1[k][l] = sum_q X_ij[k][q] 1D[q][l]      (types 0, 1, 2; type 3 reads X_ij transposed)
//     x2[k][l] = sum_p w[k][p] M_ij[l][p]       (types 0, 1, 3; type 2 reads M_ij transposed)
// as tall GEMMs over the rows (ij, k) of x1 against 1D^T and (ij, l) of x2^T against w (the class
// structure of acse_btc.cu), each by the Ozaki splitting of k_Z_oz: digit tiles in shared memory, one
// exact FP32 accumulator per level, the levels added in int64 and rounded once to FP64.  Outputs: class
// c = 2 t + (0: x1, 1: x2^T), rows (ij, .) of r doubles, read by k_B_tiled in its precomputed mode.
struct BxozArgs {
    const double* X[3];     // pair GEMM outputs (rows ij of r^2: X^{ij}_{kq} at [k][q])
    const double* M[3];     // M blocks (rows ij: M^{ij}_{lp} at [l][p])
    const double* gam;      // 1D per spin [2][r][r]
    const double* w;        // w per spin [2][r][r], w[k][p]
    double* out[8];
    int S;
    int* err;
};

template <int R>
__global__ void __launch_bounds__(ZOZ_THREADS, 1) k_Bx_oz(const __grid_constant__ BxozArgs a, int ntiles) {
    constexpr int R2 = R * R, NCH = R / 8, TPC = R * R2 / TC_BM;   // tiles per class
    static_assert((R * R2) % TC_BM == 0, "whole tiles");
    constexpr int B_SLICE = R * 128;
    const int S = a.S;
    extern __shared__ uint8_t zo_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)zo_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = sA + ZOZ_SMAX * ZOZ_A_SLICE;
    int* eA = reinterpret_cast<int*>(sB + ZOZ_SMAX * B_SLICE);
    int* eB = eA + TC_BM;
    unsigned short* tab = reinterpret_cast<unsigned short*>(eB + 64);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tab + 72);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 65) tab[threadIdx.x] = __bfloat16_as_ushort(__float2bfloat16_rn((float)((int)threadIdx.x - 32)));
    for (int e = threadIdx.x; e < (ZOZ_SMAX * ZOZ_A_SLICE + ZOZ_SMAX * B_SLICE) / 16; e += ZOZ_THREADS)
        reinterpret_cast<uint4*>(sA)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    uint32_t phase = 0;
    int cur_sel = -1;
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_end = min(ntiles, ((int)blockIdx.x + 1) * per);
    for (int tile = (int)blockIdx.x * per; tile < t_end && ok; ++tile, phase ^= 1) {
        const int c = tile / TPC;
        const int t = c >> 1, x2 = c & 1;
        const int m0 = (tile - c * TPC) * TC_BM;
        // x1: 1D^T of spin a for types 0, 3, b for 1, 2;  x2: w of spin a for types 0, 2, b for 1, 3
        const int sel = x2 ? ((t == 0 || t == 2) ? 2 : 3) : ((t == 0 || t == 3) ? 0 : 1);
        if (sel != cur_sel) {   // B rows n, K = q: 1D^T[n][q] = 1D[q][n], or w[n][q]
            const unsigned long long* g =
                reinterpret_cast<const unsigned long long*>((sel < 2 ? a.gam : a.w) + (size_t)(sel & 1) * R2);
            for (int n = threadIdx.x; n < R; n += ZOZ_THREADS) {
                unsigned long long mx = 0;
                for (int q = 0; q < R; ++q) mx = max(mx, (sel < 2 ? g[q * R + n] : g[n * R + q]) & 0x7FFFFFFFFFFFFFFFull);
                eB[n] = zoz_row_exp(mx);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < R * NCH; e += ZOZ_THREADS) {
                const int n = e / NCH, cc = e - n * NCH;
                unsigned long long x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = 8 * cc + u;
                    x[u] = sel < 2 ? g[q * R + n] : g[n * R + q];
                }
                zoz_digits8(x, eB[n], S, sB, B_SLICE, zoz_sw128(n, cc), tab);
            }
            cur_sel = sel;
        }
        // A: row m = (ij, row) of X_ij (x1) or M_ij (x2), K = q; types 3 (x1) and 2 (x2) transposed
        {
            const int ml = threadIdx.x / ZOZ_TPR, part = threadIdx.x % ZOZ_TPR, m = m0 + ml;
            const int ij = m / R, row = m - ij * R;
            const int sec = t == 0 ? 0 : t == 1 ? 2 : 1;
            const unsigned long long* base =
                reinterpret_cast<const unsigned long long*>((x2 ? a.M[sec] : a.X[sec]) + (size_t)ij * R2);
            const bool tr = x2 ? (t == 2) : (t == 3);
            constexpr int MYCH = (NCH + ZOZ_TPR - 1) / ZOZ_TPR;
            unsigned long long x[MYCH][8];
            unsigned long long mx = 0;
#pragma unroll
            for (int i = 0; i < MYCH; ++i) {
                const int cc = ZOZ_TPR * i + part;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = 8 * cc + u;
                    x[i][u] = cc < NCH ? (tr ? base[(size_t)q * R + row] : base[(size_t)row * R + q]) : 0ull;
                    mx = max(mx, x[i][u] & 0x7FFFFFFFFFFFFFFFull);
                }
            }
#pragma unroll
            for (int o = 1; o < ZOZ_TPR; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int e = zoz_row_exp(mx);
            if (part == 0) eA[ml] = e;
#pragma unroll
            for (int i = 0; i < MYCH; ++i) {
                const int cc = ZOZ_TPR * i + part;
                if (cc < NCH) zoz_digits8(x[i], e, S, sA, ZOZ_A_SLICE, zoz_sw128(ml, cc), tab);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc<0, R>();
            for (int L = 2; L <= S + 1; ++L) {
                const uint32_t acc = tmem + (uint32_t)((L - 2) * R);
                bool first = true;
                for (int sa = max(1, L - S); sa <= min(S, L - 1); ++sa) {
                    const uint64_t da = smem_desc(sA + (size_t)(sa - 1) * ZOZ_A_SLICE);
                    const uint64_t db = smem_desc(sB + (size_t)(L - sa - 1) * B_SLICE);
#pragma unroll
                    for (int kk = 0; kk < R / 16; ++kk) {
                        umma<0>(acc, da + 2 * kk, db + 2 * kk, idesc, first ? 0u : 1u);
                        first = false;
                    }
                }
            }
            umma_commit(bar);
        }
        ok = __syncthreads_and(bounded_wait(bar, phase, ZOZ_WAIT_NS, nullptr)) != 0;
        if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        tc_fence_after();
        {
            constexpr int NJG = ZOZ_THREADS / 128, JW = R / NJG;
            static_assert(JW % 4 == 0, "whole groups of four columns");
            const int q4 = warp & 3, jh = warp >> 2;
            const int ml = q4 * 32 + lane;
            const int em = eA[ml];
            double* orow = a.out[c] + (size_t)(m0 + ml) * R;
            for (int n0 = jh * JW; n0 < (jh + 1) * JW; n0 += 4) {
                long long acc[4] = {0, 0, 0, 0};
                for (int L = 2; L <= S + 1; ++L) {
                    uint32_t v[4];
                    __syncwarp();
                    zoz_tmem_ld4(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((L - 2) * R + n0), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int sh = 6 * (S + 1 - L);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[jj] += (long long)__float2int_rn(__uint_as_float(v[jj])) * (1ll << sh);
                }
                if (!ok) continue;
                double z[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int en = eB[n0 + jj];
                    z[jj] = (em == ZOZ_BAD || en == ZOZ_BAD) ? __longlong_as_double(0x7ff8000000000000ll)
                                                             : oz_ll_scaled(acc[jj], em + en - 6 * (S + 1));
                }
                *reinterpret_cast<double2*>(orow + n0) = make_double2(z[0], z[1]);
                *reinterpret_cast<double2*>(orow + n0 + 2) = make_double2(z[2], z[3]);
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int R>
static int bxoz_launch(const BxozArgs& a, cudaStream_t st) {
    const size_t smem = 1024 + (size_t)ZOZ_SMAX * ZOZ_A_SLICE + (size_t)ZOZ_SMAX * R * 128 + 4 * (TC_BM + 64) + 2 * 72 + 64;
    static int nsm = 0;
    if (!nsm) {
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Bx_oz<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0;
        ACSE_CUDA_TRY(cudaGetDevice(&dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const int ntiles = 8 * (R * R * R / TC_BM);
    const int grid = ntiles < nsm ? ntiles : nsm;
    k_Bx_oz<R><<<grid, ZOZ_THREADS, smem, st>>>(a, ntiles);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

// x1 and x2^T of every B spin type and every pair into w.bx64 (Ozaki contexts with the scratch allocated:
// r a multiple of 16, r <= 64, at most 8 slices); ACSE_ERR_UNSUPPORTED otherwise (the B kernel then forms
// the products itself in double-float).
int launch_Bx_oz(acse_ctx* c) {
    const int r = c->r;
    Work& w = c->w;
    if (!c->oz || !w.bx64[0] || r % 16 != 0 || r > 64 || c->opt.oz_slices > ZOZ_SMAX) return ACSE_ERR_UNSUPPORTED;
    BxozArgs a;
    for (int s = 0; s < 3; ++s) {
        a.X[s] = w.X[s];
        a.M[s] = w.M[s];
    }
    a.gam = w.gam;
    a.w = w.w;
    for (int k = 0; k < 8; ++k) a.out[k] = w.bx64[k];
    a.S = c->opt.oz_slices;
    a.err = w.tc_err;
    int s;
    switch (r) {
        case 16: s = bxoz_launch<16>(a, c->stream); break;
        case 32: s = bxoz_launch<32>(a, c->stream); break;
        case 48: s = bxoz_launch<48>(a, c->stream); break;
        default: s = bxoz_launch<64>(a, c->stream); break;
    }
    if (s == ACSE_OK) c->launches++;
    return s;
}
