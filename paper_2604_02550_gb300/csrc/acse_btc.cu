// The two r x r x r products of every B spin type on the tensor cores (BF16x3 path):
//     x1[k][l] = sum_q X_ij[k][q] 1D[q][l]      (types 0, 1, 2; type 3 reads X_ij transposed)
//     x2[k][l] = sum_p w[k][p] M_ij[l][p]       (types 0, 1, 3; type 2 reads M_ij transposed)
// for every pair (i, j) of a type's sector (aa pairs i < j for type 0, bb pairs for type 1, every ab pair
// for types 2 and 3), as tall GEMMs over the rows of X and M:
//     x1 rows (item, k):  D[(item, k)][l] = sum_q A[(item, k)][q] G[l][q],  G = 1D^T of the type's spin
//     x2^T rows (item, l): D[(item, l)][k] = sum_p A[(item, l)][p] w[k][p]
// (UMMA M = 128 rows, N = r, K = r in one 64-element block; both operands as hi and lo bf16 blocks and the
// accumulations hi.hi + lo.hi + hi.lo in FP32).  The results go to per-type scratch rows (x1 and x2^T,
// r^2 floats per item) that the B kernel (k_B_pipe in its precomputed mode) reads instead of forming the
// products on the CUDA cores.  Structure as the tensor-core Z kernel (acse_ztc.cu): resident blocks walk
// contiguous ranges of 128-row tiles (the resident B operand rebuilt only when the tile's class
// changes); the threads convert the tile's FP32 rows into the 128-byte-swizzled K-major layout, one
// thread per row; one thread issues the MMAs; each warp stores its TMEM lane quarter (one output row per
// thread, 16-byte stores).  Used for r a multiple of 16 (r <= 64).
#include <cuda_bf16.h>

#include "acse_internal.h"
#include "tc_ptx.cuh"

#define BXT_THREADS 256   // two threads per tile row (producer), two warps per TMEM lane quarter (epilogue)
#define BXT_A_SEG (TC_BM * 128)
#define BXT_WAIT_NS 4000000000ull

struct BxtArgs {
    const float* X[3];       // pair GEMM outputs (rows ij of r^2 floats: X^{ij}_{kq} at [k][q])
    const float* M[3];       // M blocks (rows ij: M^{ij}_{lp} at [l][p])
    const float* gam;        // 1D per spin [2][r][r]
    const float* w;          // w per spin [2][r][r], w[k][p]
    const int* pair_ij;      // same-spin item -> i r + j (pairs i < j in packed order)
    float* out[8];           // class c = 2 t + (0: x1, 1: x2^T): rows (item, .) of r floats
    int items[4];            // items of type t (0 for the types not computed)
    int tile_start[9];       // first tile of class c (classes in order, 8 = total)
    int* err;
};

static __device__ __forceinline__ void bxt_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
static __device__ __forceinline__ uint32_t bxt_sw128(int n, int c) {
    return (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) << 4);
}
static __device__ __forceinline__ uint4 bxt_pack8(const __nv_bfloat16 (&x)[8]) {
    uint4 u;
    memcpy(&u, x, 16);
    return u;
}

template <int R>
__global__ void __launch_bounds__(BXT_THREADS, 4) k_Bx_tc(const __grid_constant__ BxtArgs a) {
    static_assert(R % 16 == 0 && R <= 64, "N = r must be a multiple of 16 and K = r fit one 64-element block");
    constexpr int R2 = R * R;
    constexpr int B_SEG = R * 128;
    extern __shared__ uint8_t bx_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)bx_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                       // [hi | lo] K blocks of 128 x 128 B
    uint8_t* sB = smem + 2 * BXT_A_SEG;       // [hi | lo] K blocks of R x 128 B
    uint64_t* bar = (uint64_t*)(sB + 2 * B_SEG);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = a.tile_start[8];

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    uint32_t phase = 0;
    int cur_sel = -1;   // which resident matrix sB holds: 0 / 1 = 1D^T of spin a / b, 2 / 3 = w of spin a / b
    // a contiguous range of tiles per block: consecutive tiles share the type (and the B operand in
    // shared memory, rebuilt only when it changes) and read neighbouring source rows
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_end = min(ntiles, ((int)blockIdx.x + 1) * per);
    for (int tile = (int)blockIdx.x * per; tile < t_end && ok; ++tile, phase ^= 1) {
        int c = 0;
        while (c < 7 && a.tile_start[c + 1] <= tile) ++c;
        const int t = c >> 1, x2 = c & 1;
        const int m0 = (tile - a.tile_start[c]) * TC_BM;
        const int nrows = a.items[t] * R;
        // x1: 1D^T of spin a for types 0, 3, b for 1, 2;  x2: w of spin a for types 0, 2, b for 1, 3
        const int sel = x2 ? ((t == 0 || t == 2) ? 2 : 3) : ((t == 0 || t == 3) ? 0 : 1);
        if (sel != cur_sel) {   // row n, K = q: 1D^T[n][q] = 1D[q][n];  w[n][q]
            const float* src = (sel < 2 ? a.gam : a.w) + (size_t)(sel & 1) * R2;
            for (int e = threadIdx.x; e < R * 8; e += BXT_THREADS) {
                const int n = e >> 3, cc = e & 7;
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = 8 * cc + u;
                    const float x = q < R ? (sel < 2 ? src[q * R + n] : src[n * R + q]) : 0.f;
                    hi[u] = __float2bfloat16_rn(x);
                    lo[u] = __float2bfloat16_rn(x - __bfloat162float(hi[u]));
                }
                const uint32_t off = bxt_sw128(n, cc);
                *reinterpret_cast<uint4*>(sB + off) = bxt_pack8(hi);
                *reinterpret_cast<uint4*>(sB + B_SEG + off) = bxt_pack8(lo);
            }
            cur_sel = sel;
        }
        // A: row m = (item, row) of X_ij (x1) or M_ij (x2), K = q; types 3 (x1) and 2 (x2) transposed
        {
            const int ml = threadIdx.x & 127, half = threadIdx.x >> 7, m = m0 + ml;
            const bool valid = m < nrows;
            const int item = valid ? m / R : 0, row = valid ? m - item * R : 0;
            const int sec = t == 0 ? 0 : t == 1 ? 2 : 1;
            const size_t ij = t < 2 ? (size_t)a.pair_ij[item] : (size_t)item;
            const float* base = (x2 ? a.M[sec] : a.X[sec]) + ij * R2;
            const bool tr = x2 ? (t == 2) : (t == 3);
#pragma unroll
            for (int i = 0; i < 4; ++i) {   // this thread's half of the row: chunks cc = half, half + 2, ...
                const int cc = 2 * i + half;
                __nv_bfloat16 hi[8], lo[8];
                if (valid && 8 * cc < R) {
                    float xv[8];
                    if (!tr) {   // A[row][q] = base[row R + q]: 32 contiguous bytes per thread
                        const float4 v0 = *reinterpret_cast<const float4*>(base + (size_t)row * R + 8 * cc);
                        const float4 v1 = *reinterpret_cast<const float4*>(base + (size_t)row * R + 8 * cc + 4);
                        xv[0] = v0.x; xv[1] = v0.y; xv[2] = v0.z; xv[3] = v0.w;
                        xv[4] = v1.x; xv[5] = v1.y; xv[6] = v1.z; xv[7] = v1.w;
                    } else {     // A[row][q] = base[q R + row]: coalesced across the warp's consecutive rows
#pragma unroll
                        for (int u = 0; u < 8; ++u) xv[u] = base[(size_t)(8 * cc + u) * R + row];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        hi[u] = __float2bfloat16_rn(xv[u]);
                        lo[u] = __float2bfloat16_rn(xv[u] - __bfloat162float(hi[u]));
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 8; ++u) hi[u] = lo[u] = __float2bfloat16_rn(0.f);
                }
                const uint32_t off = bxt_sw128(ml, cc);
                *reinterpret_cast<uint4*>(sA + off) = bxt_pack8(hi);
                *reinterpret_cast<uint4*>(sA + BXT_A_SEG + off) = bxt_pack8(lo);
            }
        }
        bxt_fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc<0, R>();
            const uint64_t ah = smem_desc(sA), al = smem_desc(sA + BXT_A_SEG);
            const uint64_t bh = smem_desc(sB), bl = smem_desc(sB + B_SEG);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bh + 2 * kk, idesc, kk != 0);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, al + 2 * kk, bh + 2 * kk, idesc, 1);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1);
            umma_commit(bar);
        }
        ok = __syncthreads_and(bounded_wait(bar, phase, BXT_WAIT_NS, nullptr)) != 0;
        if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        tc_fence_after();
        // epilogue: warp w holds TMEM lanes 32 (w mod 4) .. + 31 (rows m), columns 32 (w / 4) .. + 31; the rows
        // go through shared memory (the A tile is free once the MMAs are done; row stride SP floats, 16-byte
        // chunks XOR-permuted by the row when r is a multiple of 32) and out as the contiguous block of the
        // tile's 128 output rows, coalesced 16-byte stores
        constexpr int SP = (R % 32 == 0) ? R : R + 4;
        static_assert(TC_BM * SP * 4 <= 2 * BXT_A_SEG, "staging fits the A tile");
        float* stg = reinterpret_cast<float*>(sA);
        const int q4 = warp & 3, ch = warp >> 2;
        if (32 * ch < R) {
            const int ml = q4 * 32 + lane;
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(32 * ch), v);
#pragma unroll
            for (int n = 0; n < 32; n += 4)
                if (32 * ch + n < R) {
                    const int cq = (32 * ch + n) >> 2;
                    const int pc = (R % 32 == 0) ? (cq ^ (ml & 7)) : cq;
                    *reinterpret_cast<float4*>(stg + ml * SP + 4 * pc) =
                        make_float4(__uint_as_float(v[n]), __uint_as_float(v[n + 1]), __uint_as_float(v[n + 2]),
                                    __uint_as_float(v[n + 3]));
                }
        }
        __syncthreads();
        if (ok) {
            float* dst = a.out[c] + (size_t)m0 * R;
            for (int e = threadIdx.x; e < TC_BM * (R / 4); e += BXT_THREADS) {
                const int row = e / (R / 4), cq = e - row * (R / 4);
                if (m0 + row >= nrows) break;
                const int pc = (R % 32 == 0) ? (cq ^ (row & 7)) : cq;
                *reinterpret_cast<float4*>(dst + (size_t)e * 4) = *reinterpret_cast<const float4*>(stg + row * SP + 4 * pc);
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
        tmem_dealloc(tmem, 64);
    }
}

template <int R>
static int bxt_launch(const BxtArgs& a, cudaStream_t st) {
    const size_t smem = 1024 + 2 * (size_t)BXT_A_SEG + 2 * (size_t)R * 128 + 64;
    static int blocks_per_sm = 0, nsm = 0;
    if (!blocks_per_sm) {
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Bx_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
    k_Bx_tc<R><<<grid, BXT_THREADS, smem, st>>>(a);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

// The x1 and x2^T rows of every B spin type into w.bx (BF16x3 contexts with r a multiple of 16 and the
// scratch allocated); ACSE_ERR_UNSUPPORTED otherwise (the B kernel then forms the products itself).
int launch_Bx_tc(acse_ctx* c) {
    Work& w = c->w;
    const int r = c->r;
    if (!w.bx[0] || c->opt.prec != ACSE_BF16X3 || r % 16 != 0 || r > 64) return ACSE_ERR_UNSUPPORTED;
    BxtArgs a;
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
    a.tile_start[0] = 0;
    for (int k = 0; k < 8; ++k) a.tile_start[k + 1] = a.tile_start[k] + (a.items[k >> 1] * r + TC_BM - 1) / TC_BM;
    a.err = w.tc_err;
    int s;
    switch (r) {
        case 16: s = bxt_launch<16>(a, c->stream); break;
        case 32: s = bxt_launch<32>(a, c->stream); break;
        case 48: s = bxt_launch<48>(a, c->stream); break;
        default: s = bxt_launch<64>(a, c->stream); break;
    }
    if (s == ACSE_OK) c->launches++;
    return s;
}
