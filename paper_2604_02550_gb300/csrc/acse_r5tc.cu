// The O(r^5) products of a BF16x3 contraction pass on the tensor cores (r a multiple of 16, r <= 64):
//
//   Z (the particle-hole operand): Z^{kp}_{js} = sum_q W^{kp}_{qs} 1D^j_q for the six spin types of
//     k_Z_pipe (acse_tiled.cu), i.e. per (type, k) the rows m = (p, s) of
//         D[(p, s)][j] = sum_q W_kp[q][s] 1D[j][q],
//     written as the split rows of the particle-hole GEMM operand ([hi | hi | lo] at row (sK, k, j),
//     column (sP, p, s)) plus the diagonal rows j = p that give w;
//   the B products: x1[k][l] = sum_q X_ij[k][q] 1D[q][l] (type 3 with X_ij transposed) and
//     x2[k][l] = sum_p w[k][p] M_ij[l][p] (type 2 with M_ij transposed) for every item (pair ij) of
//     the four B spin types (aa pairs i < j, bb pairs, every ab pair twice), as the rows
//         x1: D[(item, k)][l] = sum_q X_ij[k][q] 1D^T[l][q],   x2^T: D[(item, l)][k] = sum_p M_ij[l][p] w[k][p]
//     into per-type scratch that the B kernel (k_B_pipe in its precomputed mode) reads.
//
// Both are tall GEMMs whose A rows come from r x r FP32 blocks (W_kp, X_ij or M_ij, each contiguous) and
// whose B operand is one r x r matrix (1D or w of one spin).  A tile holds NB = 128 / r such blocks
// (96 rows at r = 48; the rest of the 128 UMMA rows stay zero), UMMA M = 128, N = r, K = r in one
// 64-element block, both operands as hi and lo bf16 blocks and the accumulations hi.hi + lo.hi + hi.lo in
// FP32 (TMEM, 64 columns).  Blocks stay resident and walk the tiles; per tile the source blocks are
// copied with cp.async into a raw FP32 stage (rows padded to r + 4 floats: conflict-free row and column
// reads) one tile ahead, so the copies overlap the previous tile's conversion, MMAs and stores; the
// 128 threads convert the stage into the 128-byte-swizzled K-major layout (one row per thread, 16-byte
// stores, chunk c of row n at c XOR (n mod 8)); one thread issues the MMAs; each warp stores its TMEM
// lane quarter.  The MMA wait is bounded and its outcome agreed on by the block.
#include <cuda_bf16.h>

#include "acse_internal.h"
#include "tc_ptx.cuh"

#define R5_THREADS 128
#define R5_A_SEG (TC_BM * 128)
#define R5_WAIT_NS 4000000000ull

struct R5Args {
    int mode;               // 0: Z, 1: B products
    // Z
    const float* W[3];      // FP32 W blocks aa, ab, bb
    __nv_bfloat16* Zd;      // (2 r^2) rows of ldd elements, K segments of Kp2
    __nv_bfloat16* Zf[2];   // r^2 rows of ldf elements, K segments of Kp1
    float* diag;            // [4][r][r][r]
    int ldd, ldf, Kp1, Kp2;
    int tmap[6];            // Z: block type index -> spin type t
    int ntypes;
    // B products
    const float* X[3];
    const float* M[3];
    const int* pair_ij;
    float* out[8];          // class c = 2 t + (0: x1, 1: x2^T)
    int items[4];
    // both
    const double* gam64;    // 1D per spin [2][r][r] (FP64; Z)
    const float* gam;       // 1D per spin (FP32; B products)
    const float* w;         // w per spin [2][r][r] (B products)
    int tile_start[9];      // first tile of each group (Z: type index; B products: class), [8] = total
    int* err;
};

static __device__ __forceinline__ void r5_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
static __device__ __forceinline__ uint32_t r5_sw128(int n, int c) {
    return (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) << 4);
}
static __device__ __forceinline__ uint4 r5_pack8(const __nv_bfloat16 (&x)[8]) {
    uint4 u;
    memcpy(&u, x, 16);
    return u;
}
static __device__ __forceinline__ void r5_cp16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// Tile t of the launch: its group g, the first source block b0 and the number of blocks nb; the spin
// type (Z: t of k_Z_pipe; B: the B type), k (Z) and which product (B: 0 x1, 1 x2).
struct R5Tile {
    int g, typ, k, x2, b0, nb;
};

template <int R>
__device__ __forceinline__ R5Tile r5_tile(const R5Args& a, int tile) {
    constexpr int NB = TC_BM / R;
    R5Tile T;
    int g = 0;
    while (g < 7 && a.tile_start[g + 1] <= tile) ++g;
    T.g = g;
    const int local = tile - a.tile_start[g];
    if (a.mode == 0) {   // Z: group = type index; within it R values of k, each with ceil(R / NB) tiles of p
        constexpr int PT = (R + NB - 1) / NB;
        T.typ = a.tmap[g];
        T.k = local / PT;
        T.x2 = 0;
        T.b0 = (local - T.k * PT) * NB;
        T.nb = min(NB, R - T.b0);
    } else {             // B products: group = class 2 t + x2; items in order
        T.typ = g >> 1;
        T.x2 = g & 1;
        T.k = 0;
        T.b0 = local * NB;
        T.nb = min(NB, a.items[T.typ] - T.b0);
    }
    return T;
}

// Source block b of a tile (r x r contiguous FP32) and whether the A row `row` of it is a column
// (A[row][q] = blk[q r + row]) or a row (A[row][q] = blk[row r + q]) of the block.
template <int R>
__device__ __forceinline__ const float* r5_src(const R5Args& a, const R5Tile& T, int b, bool& colread) {
    constexpr int R2 = R * R;
    constexpr size_t r3 = (size_t)R * R2;
    if (a.mode == 0) {
        const int p = T.b0 + b, k = T.k;
        switch (T.typ) {   // W_kp[q][s] of type t; A[(p, s)][q] = W_kp[q][s]
            case 0: colread = true; return a.W[0] + k * r3 + (size_t)p * R2;
            case 1: colread = true; return a.W[1] + k * r3 + (size_t)p * R2;
            case 2: colread = false; return a.W[1] + (size_t)p * r3 + (size_t)k * R2;   // stored [s][q]
            case 3: colread = true; return a.W[2] + k * r3 + (size_t)p * R2;
            case 4: colread = false; return a.W[1] + k * r3 + (size_t)p * R2;           // stored [s][q]
            default: colread = true; return a.W[1] + (size_t)p * r3 + (size_t)k * R2;
        }
    }
    const int t = T.typ, item = T.b0 + b;
    const int sec = t == 0 ? 0 : t == 1 ? 2 : 1;
    const size_t ij = t < 2 ? (size_t)a.pair_ij[item] : (size_t)item;
    colread = T.x2 ? (t == 2) : (t == 3);
    return (T.x2 ? a.M[sec] : a.X[sec]) + ij * R2;
}

template <int R>
__global__ void __launch_bounds__(R5_THREADS) k_r5_tc(const __grid_constant__ R5Args a) {
    static_assert(R % 16 == 0 && R <= 64, "N = r must be a multiple of 16 and K = r fit one 64-element block");
    constexpr int R2 = R * R, NB = TC_BM / R, LDS = R + 4;        // raw stage rows padded to r + 4 floats
    constexpr int B_SEG = R * 128;
    constexpr int STAGE = NB * R * LDS;                           // floats of one raw stage
    extern __shared__ uint8_t r5_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)r5_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                           // [hi | lo] K blocks of 128 x 128 B
    uint8_t* sB = smem + 2 * R5_A_SEG;                            // [hi | lo] K blocks of R x 128 B
    float* raw = (float*)(sB + 2 * B_SEG);                        // [2] stages of NB blocks x R rows x LDS
    uint64_t* bar = (uint64_t*)(raw + 2 * STAGE);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = a.tile_start[8];

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, 64);
    // the A rows beyond NB R stay zero for the whole kernel (so do the K columns beyond R of every row)
    for (int e = threadIdx.x; e < 2 * R5_A_SEG / 16; e += R5_THREADS) reinterpret_cast<uint4*>(sA)[e] = make_uint4(0, 0, 0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // copies of a tile's source blocks into raw stage s (cp.async, one commit group)
    auto issue = [&](int tile, int s) {
        if (tile < ntiles) {
            const R5Tile T = r5_tile<R>(a, tile);
            float* dst = raw + (size_t)s * STAGE;
            constexpr int CPR = R / 4;                                 // 16-byte chunks of a row
            for (int e = threadIdx.x; e < T.nb * R * CPR; e += R5_THREADS) {
                const int b = e / (R * CPR), rem = e - b * R * CPR, row = rem / CPR, ch = rem - row * CPR;
                bool cr;
                const float* src = r5_src<R>(a, T, b, cr);
                r5_cp16(dst + (b * R + row) * LDS + 4 * ch, src + row * R + 4 * ch);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    bool ok = true;
    uint32_t phase = 0;
    int cur_sel = -1;   // the matrix in sB: 0/1 1D^T spin a/b, 2/3 w spin a/b, 4/5 1D spin a/b
    issue(blockIdx.x, 0);
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it, phase ^= 1) {
        const int s = it & 1;
        issue(tile + gridDim.x, s ^ 1);                                // the next tile's copies fly meanwhile
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");          // this tile's stage has landed
        __syncthreads();
        const R5Tile T = r5_tile<R>(a, tile);
        // B: row n, K = q.  Z: 1D[n][q] of the type's spin.  x1: 1D^T[n][q] = 1D[q][n].  x2: w[n][q].
        int sel;
        if (a.mode == 0) sel = 4 + ((T.typ == 2 || T.typ == 3 || T.typ == 4) ? 1 : 0);
        else sel = T.x2 ? ((T.typ == 0 || T.typ == 2) ? 2 : 3) : ((T.typ == 0 || T.typ == 3) ? 0 : 1);
        if (sel != cur_sel) {   // (the previous tile's MMAs are complete)
            for (int e = threadIdx.x; e < R * 8; e += R5_THREADS) {
                const int n = e >> 3, cc = e & 7;
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = 8 * cc + u;
                    float x = 0.f;
                    if (q < R) {
                        if (sel >= 4) x = (float)a.gam64[(size_t)(sel - 4) * R2 + n * R + q];
                        else if (sel < 2) x = a.gam[(size_t)sel * R2 + q * R + n];
                        else x = a.w[(size_t)(sel - 2) * R2 + n * R + q];
                    }
                    hi[u] = __float2bfloat16_rn(x);
                    lo[u] = __float2bfloat16_rn(x - __bfloat162float(hi[u]));
                }
                const uint32_t off = r5_sw128(n, cc);
                *reinterpret_cast<uint4*>(sB + off) = r5_pack8(hi);
                *reinterpret_cast<uint4*>(sB + B_SEG + off) = r5_pack8(lo);
            }
            cur_sel = sel;
        }
        // A: row m = (block b, row), K = q, from the raw stage
        if (threadIdx.x < T.nb * R) {
            const int b = threadIdx.x / R, row = threadIdx.x - b * R;
            bool cr;
            r5_src<R>(a, T, b, cr);
            const float* blk = raw + (size_t)s * STAGE + (size_t)b * R * LDS;
#pragma unroll
            for (int cc = 0; cc < R / 8; ++cc) {
                float x[8];
                if (cr) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = blk[(8 * cc + u) * LDS + row];
                } else {
                    const float4 v0 = *reinterpret_cast<const float4*>(blk + row * LDS + 8 * cc);
                    const float4 v1 = *reinterpret_cast<const float4*>(blk + row * LDS + 8 * cc + 4);
                    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
                    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
                }
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    hi[u] = __float2bfloat16_rn(x[u]);
                    lo[u] = __float2bfloat16_rn(x[u] - __bfloat162float(hi[u]));
                }
                const uint32_t off = r5_sw128(threadIdx.x, cc);
                *reinterpret_cast<uint4*>(sA + off) = r5_pack8(hi);
                *reinterpret_cast<uint4*>(sA + R5_A_SEG + off) = r5_pack8(lo);
            }
        } else if (threadIdx.x < NB * R) {   // a short last tile: its unused rows back to zero
#pragma unroll
            for (int cc = 0; cc < R / 8; ++cc) {
                const uint32_t off = r5_sw128(threadIdx.x, cc);
                *reinterpret_cast<uint4*>(sA + off) = make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4*>(sA + R5_A_SEG + off) = make_uint4(0, 0, 0, 0);
            }
        }
        r5_fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc<0, R>();
            const uint64_t ah = smem_desc(sA), al = smem_desc(sA + R5_A_SEG);
            const uint64_t bh = smem_desc(sB), bl = smem_desc(sB + B_SEG);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bh + 2 * kk, idesc, kk != 0);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, al + 2 * kk, bh + 2 * kk, idesc, 1);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1);
            umma_commit(bar);
        }
        ok = __syncthreads_and(bounded_wait(bar, phase, R5_WAIT_NS, nullptr)) != 0;
        if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        tc_fence_after();
        {   // epilogue: warp w holds TMEM lanes 32 w .. 32 w + 31 (rows m), columns 0 .. R - 1
            const int m = warp * 32 + lane;
            uint32_t v[2][32];
            __syncwarp();
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v[0]);
            if (R > 32) tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, v[1]);
            if (ok && m < T.nb * R) {
                const int b = m / R, row = m - b * R;
                if (a.mode == 0) {
                    const int t = T.typ, k = T.k, p = T.b0 + b, sv = row;
                    int which, sK, sP;
                    if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
                    else { which = t - 4; sK = 0; sP = 0; }
                    const int dslot = t == 0 ? 0 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : -1;
                    __nv_bfloat16* base = which < 0 ? a.Zd : a.Zf[which];
                    const size_t ld = which < 0 ? (size_t)a.ldd : (size_t)a.ldf;
                    const int Kp = which < 0 ? a.Kp2 : a.Kp1;
                    const size_t col = (size_t)sP * R2 + (size_t)p * R + sv;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const float x = __uint_as_float(v[j >> 5][j & 31]);
                        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                        __nv_bfloat16* rowp = base + ((size_t)sK * R2 + (size_t)k * R + j) * ld + col;
                        rowp[0] = hi;
                        rowp[Kp] = hi;
                        rowp[2 * Kp] = lo;
                        if (dslot >= 0 && j == p) a.diag[(((size_t)dslot * R2 + (size_t)k * R + p) * R) + sv] = x;
                    }
                } else {
                    float* dst = a.out[T.g] + ((size_t)(T.b0 + b) * R + row) * R;
#pragma unroll
                    for (int n = 0; n < R; n += 4)
                        *reinterpret_cast<float4*>(dst + n) =
                            make_float4(__uint_as_float(v[n >> 5][n & 31]), __uint_as_float(v[(n + 1) >> 5][(n + 1) & 31]),
                                        __uint_as_float(v[(n + 2) >> 5][(n + 2) & 31]),
                                        __uint_as_float(v[(n + 3) >> 5][(n + 3) & 31]));
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM read, A and this raw stage free before they are reused
        tc_fence_after();
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
}

template <int R>
static int r5_launch(const R5Args& a, cudaStream_t st) {
    constexpr int NB = TC_BM / R;
    const size_t smem = 1024 + 2 * (size_t)R5_A_SEG + 2 * (size_t)R * 128 + 2 * (size_t)NB * R * (R + 4) * 4 + 64;
    static int blocks_per_sm = 0, nsm = 0;
    if (!blocks_per_sm) {
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_r5_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, smem_sm = 0;
        ACSE_CUDA_TRY(cudaGetDevice(&dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        blocks_per_sm = (int)((size_t)smem_sm / (smem + 1024));   // 1 KiB of shared memory reserved per block
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        if (blocks_per_sm > 8) blocks_per_sm = 8;                   // 8 x 64 TMEM columns
    }
    const int ntiles = a.tile_start[8];
    if (ntiles == 0) return ACSE_OK;
    const int grid = ntiles < nsm * blocks_per_sm ? ntiles : nsm * blocks_per_sm;
    k_r5_tc<R><<<grid, R5_THREADS, smem, st>>>(a);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

static int r5_dispatch(acse_ctx* c, const R5Args& a) {
    int s;
    switch (c->r) {
        case 16: s = r5_launch<16>(a, c->stream); break;
        case 32: s = r5_launch<32>(a, c->stream); break;
        case 48: s = r5_launch<48>(a, c->stream); break;
        default: s = r5_launch<64>(a, c->stream); break;
    }
    if (s == ACSE_OK) c->launches++;
    return s;
}

static bool r5_supported(const acse_ctx* c) { return c->opt.prec == ACSE_BF16X3 && c->r % 16 == 0 && c->r <= 64; }

// Z, its split rows and the diagonal rows of w; ACSE_ERR_UNSUPPORTED outside BF16x3 with r a multiple of
// 16 (the caller then uses the FP32 kernel).
int launch_Z_tc(acse_ctx* c, const float* const W32[3], int ntypes, const int* tmap) {
    if (!r5_supported(c)) return ACSE_ERR_UNSUPPORTED;
    Work& w = c->w;
    const int r = c->r, NB = TC_BM / r, PT = (r + NB - 1) / NB;
    R5Args a;
    memset(&a, 0, sizeof(a));
    a.mode = 0;
    for (int s = 0; s < 3; ++s) a.W[s] = W32[s];
    a.gam64 = w.gam;
    a.Zd = (__nv_bfloat16*)w.tc_Zd;
    a.Zf[0] = (__nv_bfloat16*)w.tc_Zf[0];
    a.Zf[1] = (__nv_bfloat16*)w.tc_Zf[1];
    a.diag = w.zdiag32;
    a.Kp1 = w.Kp1;
    a.Kp2 = w.Kp2;
    a.ldd = c->nsplit * w.Kp2;
    a.ldf = c->nsplit * w.Kp1;
    for (int i = 0; i < 6; ++i) a.tmap[i] = tmap[i];
    a.ntypes = ntypes;
    for (int g = 0; g < 8; ++g) a.tile_start[g + 1] = a.tile_start[g] + (g < ntypes ? r * PT : 0);
    a.err = w.tc_err;
    return r5_dispatch(c, a);
}

// The x1 and x2^T rows of every B spin type into w.bx (allocated for BF16x3 contexts with r a multiple of
// 16); ACSE_ERR_UNSUPPORTED otherwise (the B kernel then forms the products itself).
int launch_Bx_tc(acse_ctx* c) {
    Work& w = c->w;
    if (!w.bx[0] || !r5_supported(c)) return ACSE_ERR_UNSUPPORTED;
    const int r = c->r, NB = TC_BM / r;
    R5Args a;
    memset(&a, 0, sizeof(a));
    a.mode = 1;
    for (int s = 0; s < 3; ++s) {
        a.X[s] = w.tc_pairC[s];
        a.M[s] = w.M32[s];
    }
    a.gam = w.gam32;
    a.w = w.w32;
    a.pair_ij = w.pair_ij;
    for (int k = 0; k < 8; ++k) a.out[k] = w.bx[k];
    const int P = r * (r - 1) / 2, R2 = r * r;
    a.items[0] = P;
    a.items[1] = acse_singlet(c) ? 0 : P;
    a.items[2] = R2;
    a.items[3] = R2;
    for (int g = 0; g < 8; ++g) a.tile_start[g + 1] = a.tile_start[g] + (a.items[g >> 1] + NB - 1) / NB;
    a.err = w.tc_err;
    return r5_dispatch(c, a);
}
