// Allocation-free energy trace: acse_energy_noalloc.
//
// Some callers cannot allocate device memory at the moment they need an energy: code that runs
// under a framework or memory manager that owns the whole device heap (a second allocator would
// fragment it or exceed its budget), code on a latency-critical path that must not risk the
// implicit device synchronisation of cudaMalloc/cudaFree, and callers that hold only the integrals
// and the 2-RDM and no ACSE context (the context's workspace is sized for the full residual).
// This entry point serves them: it takes device pointers to h, V and the three 2-RDM blocks,
// forms the reduced Hamiltonian element by element inside the kernel (no K buffer), and keeps
// its only scratch -- one FP64 partial sum per (i, j) row of the pair index -- in a file-scope
// static device array.  It calls no allocating routine.
#include <cuda.h>

#include <mutex>

#include "acse_internal.h"

// Largest r the static scratch supports: one partial per (i, j), r^2 slots.
#define ACSE_NOALLOC_MAX_R 64
#define ACSE_NOALLOC_SLOTS (ACSE_NOALLOC_MAX_R * ACSE_NOALLOC_MAX_R)
#define ACSE_NOALLOC_MAX_DEVICES 64

// 32 KiB of device memory, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_energy_scratch[ACSE_NOALLOC_SLOTS];

// Device address of the array per device, and the identity of the CUDA context it belongs to: a
// device reset (or any other end of the primary context) unloads the module, and the array of the
// next context lives at another address, so a cached address is reused only within its context.
static void* g_scratch_addr[ACSE_NOALLOC_MAX_DEVICES];
static unsigned long long g_scratch_ctx[ACSE_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

typedef CUresult (*pfn_ctx_current)(CUcontext*);
typedef CUresult (*pfn_ctx_id)(CUcontext, unsigned long long*);
static pfn_ctx_current g_ctx_current;
static pfn_ctx_id g_ctx_id;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double na_block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = na_warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = na_warp_sum(v);
    __syncthreads();
    return v;
}

// Block (i, j): sum over (k, l) of K_aa (D_aa + D_bb) + 4 K_ab D_ab, with
//   K_aa^{ij}_{kl} = 1/2((ik|jl) - (il|jk)) + (h_ik d_jl + h_jl d_ik - h_il d_jk - h_jk d_il)/(2(N-1))
//   K_ab^{ij}_{kl} = 1/2 (ik|jl) + (h_ik d_jl + h_jl d_ik)/(2(N-1))      (Eq. 2; K_bb = K_aa)
__global__ void k_energy_noalloc_rows(int r, double inv2N1, const double* __restrict__ h,
                                      const double* __restrict__ V, const double* __restrict__ Daa,
                                      const double* __restrict__ Dab, const double* __restrict__ Dbb,
                                      double* __restrict__ scratch) {
    const int i = blockIdx.x / r, j = blockIdx.x % r;
    const size_t R2 = (size_t)r * r;
    const size_t row = (size_t)blockIdx.x * R2;
    double s = 0.0;
    for (int kl = threadIdx.x; kl < (int)R2; kl += blockDim.x) {
        const int k = kl / r, l = kl % r;
        const double vd = V[(((size_t)i * r + k) * r + j) * r + l];
        const double vx = V[(((size_t)i * r + l) * r + j) * r + k];
        const double hik = h[i * r + k] * (j == l), hjl = h[j * r + l] * (i == k);
        const double hil = h[i * r + l] * (j == k), hjk = h[j * r + k] * (i == l);
        const double ks = 0.5 * (vd - vx) + (hik + hjl - hil - hjk) * inv2N1;
        const double kx = 0.5 * vd + (hik + hjl) * inv2N1;
        s += ks * (Daa[row + kl] + Dbb[row + kl]) + 4.0 * kx * Dab[row + kl];
    }
    s = na_block_sum(s);
    if (threadIdx.x == 0) scratch[blockIdx.x] = s;
}

// Fixed-order sum of the first n slots (each written earlier in the same call).
__global__ void k_energy_noalloc_final(int n, const double* __restrict__ scratch, double* __restrict__ E) {
    double v = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) v += scratch[t];
    v = na_block_sum(v);
    if (threadIdx.x == 0) *E = v;
}

// 1 if p is memory the current device `dev` reads as its own: device memory of that device, or
// managed memory; 0 for host memory and for another GPU's device memory (which the kernels would
// reach only through peer access, if at all).
static int is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeManaged) return 1;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Unique id of the current CUDA context (0 when it cannot be had: the address is then looked up on
// every call, which is correct, only slower).
static unsigned long long current_ctx_id() {
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return 0;
        }
        g_ctx_current = (pfn_ctx_current)f1;
        g_ctx_id = (pfn_ctx_id)f2;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device `dev`, looked up once per device and
// context (the caller has made a runtime call on `dev` before, so its primary context is current).
static int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= ACSE_NOALLOC_MAX_DEVICES) return ACSE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_scratch_addr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            g_scratch_addr[dev] = nullptr;
            return ACSE_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = id;
    }
    *out = (double*)g_scratch_addr[dev];
    return ACSE_OK;
}

extern "C" int acse_energy_noalloc(int r, int n_alpha, int n_beta, const double* h, const double* V,
                                   const double* Daa, const double* Dab, const double* Dbb, double* E,
                                   void* cuda_stream) {
    if (!h || !V || !Daa || !Dab || !Dbb || !E) return ACSE_ERR_ARG;
    const int N = n_alpha + n_beta;
    // the shape rules of acse_create, then the static scratch's own limit
    if (r < 2 || n_alpha < 0 || n_beta < 0 || N < 2 || n_alpha > r || n_beta > r) return ACSE_ERR_SHAPE;
    if (r > ACSE_NOALLOC_MAX_R) return ACSE_ERR_TOO_LARGE;
    int dev = 0;
    ACSE_CUDA_TRY(cudaGetDevice(&dev));
    const void* ptrs[] = {h, V, Daa, Dab, Dbb, E};
    for (const void* p : ptrs)
        if (!is_device_ptr(p, dev)) return ACSE_ERR_ARG;
    double* scratch = nullptr;
    ACSE_TRY(scratch_address(dev, &scratch));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_energy_noalloc_rows<<<r * r, 256, 0, st>>>(r, 1.0 / (2.0 * (N - 1)), h, V, Daa, Dab, Dbb, scratch);
    ACSE_CUDA_TRY(cudaGetLastError());
    k_energy_noalloc_final<<<1, 256, 0, st>>>(r * r, scratch, E);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}
