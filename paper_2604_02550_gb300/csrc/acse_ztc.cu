// Z = 1D . W_kp on the tensor cores (BF16x3 path): the O(r^5) particle-hole operand of a contraction
// pass, Z^{kp}_{js} = sum_q W^{kp}_{qs} 1D^j_q for the six spin types of k_Z_pipe (acse_tiled.cu), as
// one tcgen05 GEMM per tile instead of FP32 FMAs on the CUDA cores.
//
// Tile: 128 consecutive (p, s) of one (type, k), i.e. rows m = p r + s of W_k^T; per tile
//     D[m][j] = sum_q W_kp[q][s] 1D[j][q]          (UMMA M = 128, N = r, K = q padded to 64)
// in BF16x3: A = W^T rows and B = 1D rows each held as a hi and a lo K block (x = hi + lo, two bf16),
// and the three accumulations hi.hi + lo.hi + hi.lo run into one FP32 TMEM accumulator.
// Blocks stay resident and walk a contiguous range of tiles (TMEM allocated once, the 1D block of the
// tile's spin rebuilt only when the spin changes).  Per tile the 128 threads convert the tile's W values (FP32,
// read coalesced, the transposed spin types with 32-byte vector loads) into the 128-byte-swizzled
// K-major layout the UMMA descriptors expect, one thread per row; one thread issues the MMAs; each warp
// then reads its TMEM lane quarter (one row m per thread, r columns j) and writes the split Z rows of the
// particle-hole GEMM operand ([hi | hi | lo] at row (sK, k, j), column (sP, p, s)) and, for j = p, the
// diagonal rows of w.  Several blocks share an SM, so one block's copies overlap another's MMAs and
// stores.  The wait for the MMAs is bounded; on expiry the kernel raises the device flag and stops.
// Used for r a multiple of 16 (r <= 64); other r take the FP32 kernel.
#include <cuda_bf16.h>

#include "acse_internal.h"
#include "tc_ptx.cuh"

#define ZTC_THREADS 256   // two threads per tile row (producer), two warps per TMEM lane quarter (epilogue)
#define ZTC_A_SEG (TC_BM * 128)     // one K block of the A tile: 128 rows x 128 bytes
#define ZTC_WAIT_NS 4000000000ull

struct ZtcArgs {
    const float* W[3];      // FP32 W blocks aa, ab, bb (r^4 each)
    const double* gam;      // 1D per spin [2][r][r]
    __nv_bfloat16* Zd;      // (2 r^2) rows of ldd elements, K segments of Kp2
    __nv_bfloat16* Zf[2];   // r^2 rows of ldf elements, K segments of Kp1
    float* diag;            // [4][r][r][r]: rows j = p of Zd(a,a), Zd(b,b), Zf1, Zf2
    int ldd, ldf, Kp1, Kp2;
    int tmap[6];            // block type index -> spin type t
    int* err;
};

static __device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Byte offset of the 16-byte chunk c of row n in a 128-byte-swizzled K-major tile (8-row atoms).
static __device__ __forceinline__ uint32_t sw128(int n, int c) { return (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) << 4); }

static __device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&x)[8]) {
    uint4 u;
    memcpy(&u, x, 16);
    return u;
}

template <int R>
__global__ void __launch_bounds__(ZTC_THREADS, 4) k_Z_tc(const __grid_constant__ ZtcArgs a, int ntiles) {
    static_assert(R % 16 == 0 && R <= 64, "N = r must be a multiple of 16 and K = r fit one 64-element block");
    constexpr int R2 = R * R, NT = (R2 + TC_BM - 1) / TC_BM;
    constexpr int B_SEG = R * 128;                       // one K block of a 1D tile: R rows x 128 B
    extern __shared__ uint8_t zs_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)zs_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                  // [hi | lo] K blocks of 128 x 128 B
    uint8_t* sB = smem + 2 * ZTC_A_SEG;                  // [hi | lo] K blocks of R x 128 B (1D of one spin)
    uint64_t* bar = (uint64_t*)(sB + 2 * B_SEG);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t r3 = (size_t)R * R2;

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
    int cur_sp = -1;                                     // spin of the 1D tile in sB
    // a contiguous range of tiles per block: consecutive tiles share the type (and the B operand in
    // shared memory, rebuilt only when it changes) and read neighbouring source rows
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_end = min(ntiles, ((int)blockIdx.x + 1) * per);
    for (int tile = (int)blockIdx.x * per; tile < t_end && ok; ++tile, phase ^= 1) {
        const int tb = tile / (R * NT);
        const int t = a.tmap[tb];
        const int rem = tile - tb * R * NT;
        const int k = rem / NT;
        const int m0 = (rem - k * NT) * TC_BM;
        const int sp = (t == 2 || t == 3 || t == 4) ? 1 : 0;
        if (sp != cur_sp) {   // B: 1D of this tile's spin, row j, K = q, as [hi | lo] (the last MMAs are done)
            const double* g = a.gam + (size_t)sp * R2;
            for (int e = threadIdx.x; e < R * 8; e += ZTC_THREADS) {
                const int j = e >> 3, c = e & 7;
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float x = 8 * c + u < R ? (float)g[j * R + 8 * c + u] : 0.f;
                    hi[u] = __float2bfloat16_rn(x);
                    lo[u] = __float2bfloat16_rn(x - __bfloat162float(hi[u]));
                }
                const uint32_t off = sw128(j, c);
                *reinterpret_cast<uint4*>(sB + off) = pack8(hi);
                *reinterpret_cast<uint4*>(sB + B_SEG + off) = pack8(lo);
            }
            cur_sp = sp;
        }
        // A: row m = p r + s of W_k^T, K = q; the slice W_kp[q][s] of type t (see k_Z_pipe)
        {
            const int ml = threadIdx.x & 127, half = threadIdx.x >> 7, m = m0 + ml;
            const bool valid = m < R2;
            const int p = valid ? m / R : 0, s = valid ? m - p * R : 0;
            const float* base;
            bool tr;
            switch (t) {
                case 0: tr = false; base = a.W[0] + k * r3 + (size_t)p * R2; break;
                case 1: tr = false; base = a.W[1] + k * r3 + (size_t)p * R2; break;
                case 2: tr = true; base = a.W[1] + (size_t)p * r3 + (size_t)k * R2; break;
                case 3: tr = false; base = a.W[2] + k * r3 + (size_t)p * R2; break;
                case 4: tr = true; base = a.W[1] + k * r3 + (size_t)p * R2; break;
                default: tr = false; base = a.W[1] + (size_t)p * r3 + (size_t)k * R2; break;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {   // this thread's half of the row: chunks c = half, half + 2, ...
                const int c = 2 * i + half;
                __nv_bfloat16 hi[8], lo[8];
                if (valid && 8 * c < R) {
                    float x[8];
                    if (tr) {   // W_kp[q][s] = base[s R + q]: 32 contiguous bytes per thread
                        const float4 v0 = *reinterpret_cast<const float4*>(base + (size_t)s * R + 8 * c);
                        const float4 v1 = *reinterpret_cast<const float4*>(base + (size_t)s * R + 8 * c + 4);
                        x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
                        x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
                    } else {    // W_kp[q][s] = base[q R + s]: coalesced across the warp's consecutive s
#pragma unroll
                        for (int u = 0; u < 8; ++u) x[u] = base[(size_t)(8 * c + u) * R + s];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        hi[u] = __float2bfloat16_rn(x[u]);
                        lo[u] = __float2bfloat16_rn(x[u] - __bfloat162float(hi[u]));
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 8; ++u) hi[u] = lo[u] = __float2bfloat16_rn(0.f);
                }
                const uint32_t off = sw128(ml, c);
                *reinterpret_cast<uint4*>(sA + off) = pack8(hi);
                *reinterpret_cast<uint4*>(sA + ZTC_A_SEG + off) = pack8(lo);
            }
        }
        fence_proxy_async_smem();   // the generic-proxy writes above, visible to the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc<0, R>();
            const uint64_t ah = smem_desc(sA), al = smem_desc(sA + ZTC_A_SEG);
            const uint64_t bh = smem_desc(sB), bl = smem_desc(sB + B_SEG);
            // hi.hi + lo.hi + hi.lo, FP32 accumulation
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bh + 2 * kk, idesc, kk != 0);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, al + 2 * kk, bh + 2 * kk, idesc, 1);
#pragma unroll
            for (int kk = 0; kk < R / 16; ++kk) umma<0>(tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1);
            umma_commit(bar);
        }
        // every thread polls the barrier; the block agrees on the outcome (so the loop exit is uniform)
        ok = __syncthreads_and(bounded_wait(bar, phase, ZTC_WAIT_NS, nullptr)) != 0;
        if (!ok && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        tc_fence_after();
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows m), columns 32 (w / 4) .. + 31 (j)
        const int q4 = warp & 3, ch = warp >> 2;
        if (32 * ch < R) {
            const int ml = q4 * 32 + lane, m = m0 + ml;
            const bool valid = ok && m < R2;
            const int p = m / R, s = m - p * R;
            int which, sK, sP;
            if (t < 4) { which = -1; sK = t >> 1; sP = t & 1; }
            else { which = t - 4; sK = 0; sP = 0; }
            const int dslot = t == 0 ? 0 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : -1;
            __nv_bfloat16* base = which < 0 ? a.Zd : a.Zf[which];
            const size_t ld = which < 0 ? (size_t)a.ldd : (size_t)a.ldf;
            const int Kp = which < 0 ? a.Kp2 : a.Kp1;
            const size_t col = (size_t)sP * R2 + m;
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(32 * ch), v);
            if (valid) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = 32 * ch + jj;
                    if (j >= R) break;
                    const float x = __uint_as_float(v[jj]);
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                    __nv_bfloat16* row = base + ((size_t)sK * R2 + (size_t)k * R + j) * ld + col;
                    row[0] = hi;
                    row[Kp] = hi;
                    row[2 * Kp] = lo;
                    if (dslot >= 0 && j == p) a.diag[(((size_t)dslot * R2 + (size_t)k * R + p) * R) + s] = x;
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM read and A tile free before the next tile's MMAs and copies
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
static int ztc_launch(const ZtcArgs& a, int ntypes, cudaStream_t st) {
    constexpr int R2 = R * R, NT = (R2 + TC_BM - 1) / TC_BM;
    const size_t smem = 1024 + 2 * (size_t)ZTC_A_SEG + 2 * (size_t)R * 128 + 64;
    static int blocks_per_sm = 0, nsm = 0;
    if (!blocks_per_sm) {
        ACSE_CUDA_TRY(cudaFuncSetAttribute(k_Z_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, smem_sm = 0;
        ACSE_CUDA_TRY(cudaGetDevice(&dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        ACSE_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        // resident blocks: shared memory (1 KiB of it reserved per block), at most 8 (8 x 64 TMEM columns)
        blocks_per_sm = (int)((size_t)smem_sm / (smem + 1024));
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        if (blocks_per_sm > 8) blocks_per_sm = 8;
    }
    const int ntiles = ntypes * R * NT;
    const int grid = ntiles < nsm * blocks_per_sm ? ntiles : nsm * blocks_per_sm;
    k_Z_tc<R><<<grid, ZTC_THREADS, smem, st>>>(a, ntiles);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

// Z, its split rows and the diagonal rows of w on the tensor cores (BF16x3 contexts with r a multiple
// of 16); ACSE_ERR_UNSUPPORTED when the context is outside that range (the caller then uses the FP32
// kernel).
int launch_Z_tc(acse_ctx* c, const float* const W32[3], int ntypes, const int* tmap) {
    const int r = c->r;
    if (c->opt.prec != ACSE_BF16X3 || r % 16 != 0 || r > 64) return ACSE_ERR_UNSUPPORTED;
    Work& w = c->w;
    ZtcArgs a;
    for (int s = 0; s < 3; ++s) a.W[s] = W32[s];
    a.gam = w.gam;
    a.Zd = (__nv_bfloat16*)w.tc_Zd;
    a.Zf[0] = (__nv_bfloat16*)w.tc_Zf[0];
    a.Zf[1] = (__nv_bfloat16*)w.tc_Zf[1];
    a.diag = w.zdiag32;
    a.Kp1 = w.Kp1;
    a.Kp2 = w.Kp2;
    a.ldd = c->nsplit * w.Kp2;
    a.ldf = c->nsplit * w.Kp1;
    for (int i = 0; i < 6; ++i) a.tmap[i] = tmap[i];
    a.err = w.tc_err;
    int s;
    switch (r) {
        case 16: s = ztc_launch<16>(a, ntypes, c->stream); break;
        case 32: s = ztc_launch<32>(a, ntypes, c->stream); break;
        case 48: s = ztc_launch<48>(a, ntypes, c->stream); break;
        default: s = ztc_launch<64>(a, ntypes, c->stream); break;
    }
    if (s == ACSE_OK) c->launches++;
    return s;
}
