// C ABI of libacse: context management, argument staging and the order of the hot-path passes.
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include "acse_internal.h"

int tc_plan_create(acse_ctx* c);
void tc_plan_destroy(acse_ctx* c);
int tc_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D);
int tc_contract_pre(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D);
int tc_gemm_launch(acse_ctx* c);
int tc_set_wait_ns(acse_ctx* c, unsigned long long ns, int inject_stall);
void adj_free(acse_ctx* c);
extern "C" int acse_residual_backward_impl(acse_ctx* c, const double* const* D_ckpt, int n_steps, double eps,
                                            double wE, double wN, double* dh, double* dV, double* dDaa,
                                            double* dDab, double* dDbb);

static const char* k_version = "libacse 0.1 (sm_103a; FP64 DFMA + tcgen05 split-precision GEMMs)";

extern "C" const char* acse_version(void) { return k_version; }

extern "C" const char* acse_strerror(int s) {
    switch (s) {
        case ACSE_OK: return "ok";
        case ACSE_ERR_ARG: return "invalid argument";
        case ACSE_ERR_SHAPE: return "unsupported shape (r, N or active range)";
        case ACSE_ERR_NONFINITE: return "non-finite value in input or result";
        case ACSE_ERR_TRACE: return "2-RDM trace differs from N(N-1)/2";
        case ACSE_ERR_CUDA: return "CUDA runtime error";
        case ACSE_ERR_TIMEOUT: return "device-side wait timed out";
        case ACSE_ERR_NOMEM: return "device allocation failed";
        case ACSE_ERR_UNSUPPORTED: return "option not supported by this build";
        case ACSE_ERR_TOO_LARGE: return "r exceeds the static scratch of acse_energy_noalloc (r <= 64)";
        default: return "unknown status";
    }
}

extern "C" int acse_last_error(const acse_ctx* c) { return c ? c->last_error : ACSE_ERR_ARG; }

static int latch(acse_ctx* c, int s) {
    if (c && s != ACSE_OK) c->last_error = s;
    return s;
}

// Set while a step is captured into a graph, whose pointers were all found to be device memory first.
static thread_local int tl_capturing = 0;

// 1 if p is host memory (pageable or pinned), 0 if device or managed, -1 on error.
static int is_host_ptr(const void* p) {
    if (!p || tl_capturing) return 0;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 0 : 1;
}

static size_t n4_of(const acse_ctx* c) { return (size_t)c->r * c->r * c->r * c->r; }

// Device-side address of pinned (page-locked) host memory, or null for pageable memory.
static const void* pinned_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Copy of n doubles by the SMs (16-byte accesses when both ends are 16-byte aligned); used for
// pinned host memory, which the GPU reads and writes directly over the host link.
__global__ void __launch_bounds__(256) k_copy_doubles(double* __restrict__ dst, const double* __restrict__ src,
                                                      size_t n) {
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
        const size_t n2 = n / 2;
        for (size_t i = t0; i < n2; i += stride)
            reinterpret_cast<double2*>(dst)[i] = reinterpret_cast<const double2*>(src)[i];
        if ((n & 1) && t0 == 0) dst[n - 1] = src[n - 1];
    } else {
        for (size_t i = t0; i < n; i += stride) dst[i] = src[i];
    }
}

// ------------------------------------------------------------------------------- create
static int alloc_d(void** p, size_t bytes, size_t* total) {
    *total += bytes;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ACSE_ERR_NOMEM;
    }
    return ACSE_OK;
}

static void free_work(acse_ctx* c) {
    Work& w = c->w;
    void* ptrs[] = {w.Kh[0], w.Kh[1], w.Kh[2], w.gam, w.M[0], w.M[1], w.M[2], w.Md, w.Mf1, w.Mf2, w.Zd, w.Zf1,
                    w.Zf2, w.w, w.Q, w.X[0], w.X[1], w.X[2], w.Y[0], w.Y[1], w.Y[2], w.X5d, w.X5f1, w.X5f2,
                    w.H[0], w.H[1], w.H[2], w.zdiag, w.A[0], w.A[1], w.A[2], w.U[0], w.U[1], w.U[2], w.Dt[0],
                    w.Dt[1], w.Dt[2], w.stage_in[0], w.stage_in[1], w.stage_in[2], w.stage_out[0],
                    w.stage_out[1], w.stage_out[2], w.h, w.V, w.scal, w.partial};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    memset(&c->w, 0, sizeof(Work));
}

static int alloc_work(acse_ctx* c) {
    Work& w = c->w;
    memset(&w, 0, sizeof(Work));
    const size_t n4 = n4_of(c), R2 = (size_t)c->r * c->r;
    const size_t b4 = n4 * sizeof(double);
    size_t tot = 0;
#define A_(p, bytes) ACSE_TRY(alloc_d((void**)&(p), (bytes), &tot))
    for (int s = 0; s < 3; ++s) {
        A_(w.Kh[s], b4);
        A_(w.A[s], b4); A_(w.U[s], b4); A_(w.Dt[s], b4);
        A_(w.stage_in[s], b4); A_(w.stage_out[s], b4);
    }
    A_(w.gam, 2 * R2 * sizeof(double));
    if (c->opt.prec == ACSE_FP64) {   // FP64 intermediates (the split path has FP32 ones)
        for (int s = 0; s < 3; ++s) { A_(w.M[s], b4); A_(w.X[s], b4); A_(w.Y[s], b4); }
        for (int t = 0; t < 3; ++t) A_(w.H[t], b4);
        A_(w.zdiag, 4 * R2 * (size_t)c->r * sizeof(double));
        A_(w.w, 2 * R2 * sizeof(double));
        A_(w.Q, 2 * R2 * sizeof(double));
        A_(w.Md, 4 * b4); A_(w.Mf1, b4); A_(w.Mf2, b4);
        A_(w.Zd, 4 * b4); A_(w.Zf1, b4); A_(w.Zf2, b4);
        A_(w.X5d, 4 * b4); A_(w.X5f1, b4); A_(w.X5f2, b4);
    }
    A_(w.h, R2 * sizeof(double));
    A_(w.V, b4);
    A_(w.scal, 16 * sizeof(double));
    w.npartial = 8192;
    A_(w.partial, (size_t)w.npartial * sizeof(double));
#undef A_
    ACSE_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 16 * sizeof(double), c->stream));
    return ACSE_OK;
}

__global__ void k_set1(double* dst, double v) { *dst = v; }

extern "C" int acse_create(acse_ctx** out, const acse_opts* o, const double* h, const double* V, void* stream) {
    if (out) *out = nullptr;   // every failure leaves *out = NULL
    if (!out || !o || !h || !V) return ACSE_ERR_ARG;
    const int N = o->n_alpha + o->n_beta;
    if (o->r < 2 || o->r > ACSE_MAX_R || o->n_alpha < 0 || o->n_beta < 0 || N < 2 || o->n_alpha > o->r ||
        o->n_beta > o->r)
        return ACSE_ERR_SHAPE;
    if (o->prec < ACSE_FP64 || o->prec > ACSE_OZAKI) return ACSE_ERR_ARG;
    const int oz_slices = o->prec == ACSE_OZAKI ? (o->oz_slices ? o->oz_slices : 8) : 0;
    if (o->prec == ACSE_OZAKI && (oz_slices < 4 || oz_slices > 10)) return ACSE_ERR_ARG;
    if (o->recon != ACSE_RECON_V && o->recon != ACSE_RECON_NY) return ACSE_ERR_UNSUPPORTED;
    if (o->singlet && o->n_alpha != o->n_beta) return ACSE_ERR_ARG;
    if (o->mask_active && (o->act_lo < 0 || o->act_hi > o->r || o->act_lo >= o->act_hi)) return ACSE_ERR_SHAPE;
    if (o->refine != 0 && o->refine != 1) return ACSE_ERR_ARG;
    if (o->gemm_tile < 0 || o->gemm_tile > 2) return ACSE_ERR_ARG;
    if (o->refine && (o->singlet || o->refine_tol < 0.0 || !(o->refine_tol == o->refine_tol) ||
                      (o->refine_slices != 0 && (o->refine_slices < 4 || o->refine_slices > 10))))
        return ACSE_ERR_ARG;
    acse_ctx* c = (acse_ctx*)calloc(1, sizeof(acse_ctx));
    if (!c) return ACSE_ERR_NOMEM;
    c->opt = *o;
    if (o->prec == ACSE_OZAKI) {   // an FP64 context whose pass GEMMs run by the Ozaki scheme
        c->opt.prec = ACSE_FP64;
        c->opt.oz_slices = oz_slices;
        c->oz = 1;
    }
    c->r = o->r;
    c->N = N;
    c->stream = (cudaStream_t)stream;
    c->nsplit = (o->prec == ACSE_BF16X3 || o->prec == ACSE_TF32X3) ? 3 : 1;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        free(c);
        return ACSE_ERR_CUDA;
    }
    int s = tiled_set_attrs();
    if (s == ACSE_OK) s = ny_set_attrs();
    if (s == ACSE_OK) s = alloc_work(c);
    if (s == ACSE_OK && c->opt.prec != ACSE_FP64) s = tc_plan_create(c);
    if (s == ACSE_OK && c->oz) s = oz_plan_create(c);
    if (s == ACSE_OK && o->recon == ACSE_RECON_NY) s = ny_alloc(c);
    if (s != ACSE_OK) {
        ny_free(c);
        oz_plan_destroy(c);
        tc_plan_destroy(c);
        free_work(c);
        free(c);
        return s;
    }
    const size_t R2 = (size_t)c->r * c->r;
    const cudaMemcpyKind kh = is_host_ptr(h) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kv = is_host_ptr(V) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(c->w.h, h, R2 * sizeof(double), kh, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->w.V, V, R2 * R2 * sizeof(double), kv, c->stream) != cudaSuccess)
        s = ACSE_ERR_CUDA;
    if (s == ACSE_OK) s = launch_build_K(c);
    if (s == ACSE_OK && c->opt.prec != ACSE_FP64) s = tc_make_Kh32(c);   // the FP32 K/2 of the split path
    if (s == ACSE_OK) {
        k_set1<<<1, 1, 0, c->stream>>>(c->w.scal + 2, o->eps0 > 0.0 ? o->eps0 : 1e-3);
        if (cudaGetLastError() != cudaSuccess) s = ACSE_ERR_CUDA;
    }
    // host sources must stay valid until the copies are done
    if (s == ACSE_OK && (kh == cudaMemcpyHostToDevice || kv == cudaMemcpyHostToDevice) &&
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        s = ACSE_ERR_CUDA;
    if (s == ACSE_OK && o->refine) {   // the FP64-accurate context the schedule switches to
        acse_opts f = *o;
        f.prec = ACSE_OZAKI;
        f.oz_slices = o->refine_slices ? o->refine_slices : 8;
        f.refine = 0;
        s = acse_create(&c->fine, &f, c->w.h, c->w.V, stream);
        c->sched_n2 = -1.0;
    }
    if (s != ACSE_OK) {
        ny_free(c);
        oz_plan_destroy(c);
        tc_plan_destroy(c);
        free_work(c);
        free(c);
        return s;
    }
    *out = c;
    return ACSE_OK;
}

extern "C" int acse_destroy(acse_ctx* c) {
    if (!c) return ACSE_ERR_ARG;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 2 * ACSE_PROF_MAX; ++i)
        if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
    if (c->shadow) acse_destroy(c->shadow);
    if (c->fine) acse_destroy(c->fine);
    for (int b = 0; b < 3; ++b) {
        if (c->aux[b]) cudaStreamDestroy(c->aux[b]);
        if (c->ev_join[b]) cudaEventDestroy(c->ev_join[b]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (int g = 0; g < 2; ++g)
        if (c->sg[g].exec) cudaGraphExecDestroy(c->sg[g].exec);
    ny_free(c);
    adj_free(c);
    oz_plan_destroy(c);
    tc_plan_destroy(c);
    free_work(c);
    free(c);
    return ACSE_OK;
}

// ------------------------------------------------------------------------ contraction pass
// G(W) for the current D: builds the operands, runs every O(r^6) GEMM of the pass in one
// grouped launch, assembles B and G.  prep_D = 1 recomputes 1D, M and the ph layout of M.
int acse_contract_pre(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D) {
    for (int s = 0; s < 3; ++s) {
        c->cur_D[s] = D[s];
        c->cur_W[s] = W[s];
    }
    if (c->opt.prec == ACSE_FP64) {
        if (prep_D) {
            ACSE_TRY(launch_gamma_M(c, D));
            ACSE_TRY(launch_pack_Mph(c));
        }
        ACSE_TRY(launch_W_intermediates(c, W));
        return c->oz ? oz_slice_operands(c, prep_D) : ACSE_OK;
    }
    if (prep_D) ACSE_TRY(launch_gamma(c, D));
    return tc_contract_pre(c, D, W, prep_D);
}

// The nine FP64 GEMMs of the pass whose operands acse_contract_pre prepared.
int acse_gemm_list_f64(acse_ctx* c, GemmF64* g, int* n) {
    Work& w = c->w;
    const int r = c->r, R2 = r * r, R22 = 2 * R2;
    int k = 0;
    for (int s = 0; s < 3; ++s) {
        const double f = (s == 1) ? 2.0 : 1.0;   // mixed-spin (rs) sums count both orders
        g[k++] = GemmF64{w.M[s], c->cur_W[s], w.X[s], R2, R2, R2, R2, R2, R2, f, 0.0, 0, 0, 0};
        g[k++] = GemmF64{c->cur_D[s], c->cur_W[s], w.Y[s], R2, R2, R2, R2, R2, R2, f, 0.0, 0, 0, 0};
    }
    g[k++] = GemmF64{w.Zd, w.Md, w.X5d, R22, R22, R22, R22, R22, R22, 1.0, 0.0, 0, 0, 0};
    g[k++] = GemmF64{w.Zf1, w.Mf1, w.X5f1, R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 0, 0};
    g[k++] = GemmF64{w.Zf2, w.Mf2, w.X5f2, R2, R2, R2, R2, R2, R2, 1.0, 0.0, 0, 0, 0};
    *n = k;
    return ACSE_OK;
}

int acse_contract_gemm(acse_ctx* c) {
    if (c->oz) return oz_gemm_launch(c);
    if (c->opt.prec == ACSE_FP64) {
        GemmF64 g[9];
        int n = 0;
        ACSE_TRY(acse_gemm_list_f64(c, g, &n));
        return gemm_f64_grouped(c, g, n, c->stream);
    }
    return tc_gemm_launch(c);
}

int acse_contract_post(acse_ctx* c, int sW, double scale, int mask, double* const out[3], double* norm2_dst) {
    if (c->opt.prec != ACSE_FP64) ACSE_TRY(tc_unpack_pairs(c));   // rows i < j of the same-spin [X; Y]
    if (c->ny) ACSE_TRY(ny_pass(c));   // NY: the 3-cumulant term, added to B by the B kernel
    ACSE_TRY(launch_Q(c));
    ACSE_TRY(launch_build_B(c));
    return launch_assemble_G(c, sW, scale, mask, out, norm2_dst);
}

// The auxiliary streams and their events, created on first use; ev_fork is created last, so a
// non-null ev_fork means that every stream and event exists.
static int ensure_aux(acse_ctx* c) {
    if (c->ev_fork) return ACSE_OK;
    for (int b = 0; b < 3; ++b) {
        if (!c->aux[b]) ACSE_CUDA_TRY(cudaStreamCreateWithFlags(&c->aux[b], cudaStreamNonBlocking));
        if (!c->ev_join[b]) ACSE_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join[b], cudaEventDisableTiming));
    }
    ACSE_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    return ACSE_OK;
}

// G(W) for the current D: operands, every O(r^6) GEMM of the pass in one grouped launch, assembly.
// prep_D = 1 recomputes 1D, M and the particle-hole layout of M.  On the split path the operands of
// D (M, [M; D], the particle-hole M) and those of W (the W rows, Z, w) are independent once 1D is
// known, so the W side runs on an auxiliary stream forked from and joined back into the context's.
int acse_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int sW, double scale, int mask,
                  double* const out[3], double* norm2_dst, int prep_D) {
    if (prep_D && c->opt.prec != ACSE_FP64 && !c->ny) {
        for (int s = 0; s < 3; ++s) {
            c->cur_D[s] = D[s];
            c->cur_W[s] = W[s];
        }
        ACSE_TRY(ensure_aux(c));
        ACSE_TRY(launch_gamma(c, D));
        ACSE_CUDA_TRY(cudaEventRecord(c->ev_fork, c->stream));
        ACSE_CUDA_TRY(cudaStreamWaitEvent(c->aux[0], c->ev_fork, 0));
        cudaStream_t main = c->stream;
        c->stream = c->aux[0];
        const int sw = tc_mixed_prep_W(c, W);
        c->stream = main;
        ACSE_TRY(sw);
        ACSE_CUDA_TRY(cudaEventRecord(c->ev_join[0], c->aux[0]));
        ACSE_TRY(tc_mixed_prep_D(c, D));
        ACSE_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_join[0], 0));
    } else {
        ACSE_TRY(acse_contract_pre(c, D, W, prep_D));
    }
    ACSE_TRY(acse_contract_gemm(c));
    return acse_contract_post(c, sW, scale, mask, out, norm2_dst);
}

static int residual_dev(acse_ctx* c, const double* const D[3], double* const A[3], double* norm2_dst) {
    const double* W[3] = {c->w.Kh[0], c->w.Kh[1], c->w.Kh[2]};
    return acse_contract(c, D, W, +1, 1.0, 1, A, norm2_dst, 1);
}

// Update for the D whose 1D / M are current: U = 1/2 G(A), A pair-anti-Hermitian (s = -1).
static int update_dev(acse_ctx* c, const double* const D[3], const double* const A[3], double* const U[3]) {
    return acse_contract(c, D, A, -1, 0.5, 0, U, nullptr, 0);
}

// ------------------------------------------------------------------------- staging
struct Staged {
    const double* in[3];
    double* out[3];
    int host_in, host_out;
};

// Copies of up to three r^4 blocks between host and device (null entries skipped), issued on three
// auxiliary streams forked from and joined back into the context's stream, so that the copy engines
// move the blocks concurrently.
static int copy_blocks(acse_ctx* c, void* const dst[3], const void* const src[3], cudaMemcpyKind kind) {
    ACSE_TRY(ensure_aux(c));
    const size_t n4 = n4_of(c), b4 = n4 * sizeof(double);
    ACSE_CUDA_TRY(cudaEventRecord(c->ev_fork, c->stream));
    for (int b = 0; b < 3; ++b) {
        if (!dst[b]) continue;
        ACSE_CUDA_TRY(cudaStreamWaitEvent(c->aux[b], c->ev_fork, 0));
        // pinned host memory: copied by the SMs over the host link; pageable memory: copy engine
        const void* hp = kind == cudaMemcpyHostToDevice ? src[b] : dst[b];
        const void* dp = pinned_device_ptr(hp);
        if (dp) {
            double* d = kind == cudaMemcpyHostToDevice ? (double*)dst[b] : (double*)dp;
            const double* sp = kind == cudaMemcpyHostToDevice ? (const double*)dp : (const double*)src[b];
            k_copy_doubles<<<152 * 4, 256, 0, c->aux[b]>>>(d, sp, n4);
            ACSE_LAUNCHED(c);
        } else {
            ACSE_CUDA_TRY(cudaMemcpyAsync(dst[b], src[b], b4, kind, c->aux[b]));
        }
        ACSE_CUDA_TRY(cudaEventRecord(c->ev_join[b], c->aux[b]));
        ACSE_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_join[b], 0));
    }
    return ACSE_OK;
}

static int stage_inputs(acse_ctx* c, const double* D0, const double* D1, const double* D2, const double* src[3],
                        int* host) {
    const double* Ds[3] = {D0, D1, D2};
    *host = 0;
    void* dst[3] = {nullptr, nullptr, nullptr};
    const void* from[3] = {nullptr, nullptr, nullptr};
    for (int s = 0; s < 3; ++s) {
        if (!Ds[s]) return ACSE_ERR_ARG;
        if (is_host_ptr(Ds[s])) {
            dst[s] = c->w.stage_in[s];
            from[s] = Ds[s];
            src[s] = c->w.stage_in[s];
            *host = 1;
        } else {
            src[s] = Ds[s];
        }
    }
    if (*host) ACSE_TRY(copy_blocks(c, dst, from, cudaMemcpyHostToDevice));
    return ACSE_OK;
}

static int check_D(acse_ctx* c, const double* const D[3]) {
    if (!c->opt.check_inputs) return ACSE_OK;
    ACSE_TRY(launch_trace_check(c, D));
    double hv[2];
    ACSE_CUDA_TRY(cudaMemcpyAsync(hv, c->w.scal + 7, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hv[1] != 0.0) return ACSE_ERR_NONFINITE;
    const double want = 0.5 * c->N * (c->N - 1);
    if (!(fabs(hv[0] - want) <= 1e-8 * want)) return ACSE_ERR_TRACE;
    return ACSE_OK;
}

// After a stream synchronisation: ACSE_ERR_TIMEOUT if a bounded device wait ran out.
static int device_status(acse_ctx* c) {
    if (!c->w.tc_err) return ACSE_OK;
    int flag = 0;
    ACSE_CUDA_TRY(cudaMemcpy(&flag, c->w.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    return flag ? ACSE_ERR_TIMEOUT : ACSE_OK;
}

static int sync_and_status(acse_ctx* c) {
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return device_status(c);
}

static int put_scalar(acse_ctx* c, double* dst, const double* src_dev, int* need_sync) {
    if (!dst) return ACSE_OK;
    if (is_host_ptr(dst)) {
        ACSE_CUDA_TRY(cudaMemcpyAsync(dst, src_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        *need_sync = 1;
    } else {
        ACSE_TRY(launch_copy_scalar(c, dst, src_dev));
    }
    return ACSE_OK;
}

// ------------------------------------------------------------------------------ energy
extern "C" int acse_energy(acse_ctx* c, const double* Daa, const double* Dab, const double* Dbb, double* E) {
    if (!c) return ACSE_ERR_ARG;
    if (c->refined) return latch(c, acse_energy(c->fine, Daa, Dab, Dbb, E));
    if (!E) return latch(c, ACSE_ERR_ARG);
    const double* D[3];
    int host_in = 0, sync = 0;
    int s = stage_inputs(c, Daa, Dab, Dbb, D, &host_in);
    if (s == ACSE_OK) s = launch_energy(c, D, c->w.scal + 1);
    if (s == ACSE_OK) s = put_scalar(c, E, c->w.scal + 1, &sync);
    if (s == ACSE_OK && (sync || host_in)) s = sync_and_status(c);
    return latch(c, s);
}

// ---------------------------------------------------------------------------- residual
extern "C" int acse_residual(acse_ctx* c, const double* Daa, const double* Dab, const double* Dbb, double* Aaa,
                             double* Aab, double* Abb, double* norm2) {
    if (!c) return ACSE_ERR_ARG;
    if (c->refined) return latch(c, acse_residual(c->fine, Daa, Dab, Dbb, Aaa, Aab, Abb, norm2));
    const double* D[3];
    int host_in = 0, sync = 0;
    int s = stage_inputs(c, Daa, Dab, Dbb, D, &host_in);
    if (s == ACSE_OK) s = check_D(c, D);
    double* Aout[3] = {Aaa, Aab, Abb};
    double* A[3];
    int host_out[3] = {0, 0, 0};
    for (int b = 0; b < 3 && s == ACSE_OK; ++b) {
        if (!Aout[b]) {
            A[b] = c->w.A[b];
        } else if (is_host_ptr(Aout[b])) {
            A[b] = c->w.stage_out[b];
            host_out[b] = 1;
        } else {
            A[b] = Aout[b];
        }
    }
    if (s == ACSE_OK) s = residual_dev(c, D, A, c->w.scal + 0);
    if (s == ACSE_OK && (host_out[0] || host_out[1] || host_out[2])) {
        void* dst[3];
        const void* from[3];
        for (int b = 0; b < 3; ++b) {
            dst[b] = host_out[b] ? (void*)Aout[b] : nullptr;
            from[b] = A[b];
        }
        s = copy_blocks(c, dst, from, cudaMemcpyDeviceToHost);
        sync = 1;
    }
    if (s == ACSE_OK) s = put_scalar(c, norm2, c->w.scal + 0, &sync);
    if (s == ACSE_OK && (sync || host_in)) s = sync_and_status(c);
    return latch(c, s);
}

// -------------------------------------------------------------------------------- step
static int step_impl(acse_ctx* c, double* Daa, double* Dab, double* Dbb, double eps, double* E_out,
                     double* norm2_out, double* eps_used);

// Precision schedule: after a step in the starting precision, read ||A||^2 at the D before the step and
// switch once it has fallen by less than refine_tol (relative) since the previous step, or risen; the
// line-search state (the next trial step) moves to the FP64-accurate context with the switch.
static int sched_after_step(acse_ctx* c) {
    double n2 = 0.0;
    ACSE_CUDA_TRY(cudaMemcpyAsync(&n2, c->w.scal + 0, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double tol = c->opt.refine_tol > 0.0 ? c->opt.refine_tol : 1e-2;
    c->sched_steps++;
    if (c->sched_n2 > 0.0 && !(c->sched_n2 - n2 >= tol * c->sched_n2)) {
        ACSE_CUDA_TRY(cudaMemcpyAsync(c->fine->w.scal + 2, c->w.scal + 2, sizeof(double), cudaMemcpyDeviceToDevice,
                                      c->stream));
        c->refined = 1;
    }
    c->sched_n2 = n2;
    return ACSE_OK;
}

// A step runs as a CUDA graph when nothing in it needs the host: device blocks and outputs (or none),
// no input checks, no precision schedule, no profiling, and a stream of the caller's that is neither
// the legacy default stream nor being captured already.  The graph of a set of arguments is captured
// the second time in a row they are passed (so that a caller who changes them every call pays no
// capture) and replayed from then on; the replay launches the same kernels with the same arguments in
// the same order as a direct call, so results are identical.  A capture that fails (an API call the
// capture refuses) switches the context to direct calls.
static int step_graph_eligible(acse_ctx* c, double* const ptrs[6]) {
    if (c->sg_refused || c->fine || c->prof_on || c->opt.check_inputs || c->stream == nullptr) return 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cs != cudaStreamCaptureStatusNone) return 0;
    for (int i = 0; i < 6; ++i)
        if (ptrs[i] && is_host_ptr(ptrs[i])) return 0;
    return 1;
}

static int step_graph_launch(acse_ctx* c, int g) {
    ACSE_CUDA_TRY(cudaGraphLaunch(c->sg[g].exec, c->stream));
    c->launches += c->sg[g].launches;
    c->sg[g].used = ++c->sg_tick;
    return ACSE_OK;
}

// Capture the step with these arguments into slot g (the least recently used) and run it.  Returns
// ACSE_ERR_UNSUPPORTED, having run nothing, when the capture failed.
static int step_graph_capture(acse_ctx* c, double* const ptrs[6], double eps) {
    const int g = c->sg[0].used <= c->sg[1].used ? 0 : 1;
    if (c->sg[g].exec) {
        cudaGraphExecDestroy(c->sg[g].exec);
        c->sg[g].exec = nullptr;
    }
    const long long l0 = c->launches;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return ACSE_ERR_UNSUPPORTED;
    }
    tl_capturing = 1;
    const int s = step_impl(c, ptrs[0], ptrs[1], ptrs[2], eps, ptrs[3], ptrs[4], ptrs[5]);
    tl_capturing = 0;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = s == ACSE_OK && e == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        c->launches = l0;
        return ACSE_ERR_UNSUPPORTED;
    }
    c->sg[g].exec = exec;
    for (int i = 0; i < 6; ++i) c->sg[g].key[i] = ptrs[i];
    c->sg[g].eps = eps;
    c->sg[g].launches = c->launches - l0;
    c->launches = l0;
    return step_graph_launch(c, g);
}

extern "C" int acse_step(acse_ctx* c, double* Daa, double* Dab, double* Dbb, double eps, double* E_out,
                         double* norm2_out, double* eps_used) {
    if (!c) return ACSE_ERR_ARG;
    if (c->refined) return latch(c, acse_step(c->fine, Daa, Dab, Dbb, eps, E_out, norm2_out, eps_used));
    double* const ptrs[6] = {Daa, Dab, Dbb, E_out, norm2_out, eps_used};
    if (Daa && Dab && Dbb && step_graph_eligible(c, ptrs)) {
        auto same = [&](const void* const* key, double keps) {
            for (int i = 0; i < 6; ++i)
                if (key[i] != ptrs[i]) return false;
            return memcmp(&keps, &eps, sizeof(double)) == 0;
        };
        for (int g = 0; g < 2; ++g)
            if (c->sg[g].exec && same(c->sg[g].key, c->sg[g].eps)) return latch(c, step_graph_launch(c, g));
        if (c->sg_seen_valid && same(c->sg_seen, c->sg_seen_eps)) {
            const int s = step_graph_capture(c, ptrs, eps);
            if (s != ACSE_ERR_UNSUPPORTED) return latch(c, s);
            c->sg_refused = 1;
        }
        for (int i = 0; i < 6; ++i) c->sg_seen[i] = ptrs[i];
        c->sg_seen_eps = eps;
        c->sg_seen_valid = 1;
    }
    int s = step_impl(c, Daa, Dab, Dbb, eps, E_out, norm2_out, eps_used);
    if (s == ACSE_OK && c->fine) s = sched_after_step(c);
    return latch(c, s);
}

static int step_impl(acse_ctx* c, double* Daa, double* Dab, double* Dbb, double eps, double* E_out,
                     double* norm2_out, double* eps_used) {
    Work& w = c->w;
    const double* Din[3];
    int host_in = 0, sync = 0;
    int s = stage_inputs(c, Daa, Dab, Dbb, Din, &host_in);
    if (s == ACSE_OK) s = check_D(c, Din);
    double* D[3] = {(double*)Din[0], (double*)Din[1], (double*)Din[2]};
    const double* Dc[3] = {D[0], D[1], D[2]};
    // A at D (masked), ||A||^2 before the mask -> scal[0]; on the split path (V reconstruction) only its FP32
    // copy is written: the update pass reads that, and the FP64 A of a step is not an output
    c->a64_skip = c->opt.prec != ACSE_FP64 && !c->ny;
    if (s == ACSE_OK) s = residual_dev(c, Dc, w.A, w.scal + 0);
    c->a64_skip = 0;
    const double* Ac[3] = {w.A[0], w.A[1], w.A[2]};
    if (s == ACSE_OK) s = update_dev(c, Dc, Ac, w.U);
    const double* Uc[3] = {w.U[0], w.U[1], w.U[2]};
    if (s == ACSE_OK) {
        if (c->opt.line_search) {
            // f(0) = ||A(D)||^2; f(e0), f(2 e0) from trial residuals at D + t e0 U
            s = launch_copy_scalar(c, w.scal + 4, w.scal + 0);
            const double* Dt[3] = {w.Dt[0], w.Dt[1], w.Dt[2]};
            for (int t = 1; t <= 2 && s == ACSE_OK; ++t) {
                s = launch_axpy(c, D, Uc, w.scal + 2, (double)t, w.Dt);
                // the trial residual reuses the X/Y/T buffers; its A goes to the stage_out scratch
                double* At[3] = {w.stage_out[0], w.stage_out[1], w.stage_out[2]};
                if (s == ACSE_OK) s = residual_dev(c, Dt, At, w.scal + 4 + t);
            }
            if (s == ACSE_OK) s = launch_line_search(c);
        } else {
            k_set1<<<1, 1, 0, c->stream>>>(w.scal + 3, eps);
            c->launches++;
            if (cudaGetLastError() != cudaSuccess) s = ACSE_ERR_CUDA;
        }
    }
    if (s == ACSE_OK) s = launch_axpy_energy(c, D, Uc, w.scal + 3, w.scal + 1);
    if (s == ACSE_OK && host_in) {
        double* Dh[3] = {Daa, Dab, Dbb};
        void* dst[3];
        const void* from[3];
        for (int b = 0; b < 3; ++b) {
            dst[b] = D[b] == w.stage_in[b] ? (void*)Dh[b] : nullptr;
            from[b] = D[b];
        }
        s = copy_blocks(c, dst, from, cudaMemcpyDeviceToHost);
        sync = 1;
    }
    if (s == ACSE_OK) s = put_scalar(c, E_out, w.scal + 1, &sync);
    if (s == ACSE_OK) s = put_scalar(c, norm2_out, w.scal + 0, &sync);
    if (s == ACSE_OK) s = put_scalar(c, eps_used, w.scal + 3, &sync);
    if (s == ACSE_OK && sync) s = sync_and_status(c);
    return s;
}

extern "C" int acse_schedule_state(const acse_ctx* c, int* refined, int* steps) {
    if (!c) return ACSE_ERR_ARG;
    if (refined) *refined = c->refined;
    if (steps) *steps = c->sched_steps;
    return ACSE_OK;
}

extern "C" int acse_residual_backward(acse_ctx* c, const double* const* D_ckpt, int n_steps, double eps, double wE,
                                      double wN, double* dh, double* dV, double* dDaa, double* dDab, double* dDbb) {
    if (!c) return ACSE_ERR_ARG;
    if (c->opt.recon != ACSE_RECON_V) return latch(c, ACSE_ERR_UNSUPPORTED);
    if (c->opt.prec == ACSE_FP64)
        return latch(c, acse_residual_backward_impl(c, D_ckpt, n_steps, eps, wE, wN, dh, dV, dDaa, dDab, dDbb));
    // split precision: the reverse sweep runs in an FP64-accurate companion context (same h, V, options;
    // the Ozaki precision, so that its GEMMs run on the tensor cores too)
    if (!c->shadow) {
        acse_opts o = c->opt;
        o.prec = ACSE_OZAKI;
        o.oz_slices = 8;
        o.singlet = 0;
        o.line_search = 0;
        o.refine = 0;
        const int s = acse_create(&c->shadow, &o, c->w.h, c->w.V, (void*)c->stream);
        if (s != ACSE_OK) {
            c->shadow = nullptr;
            return latch(c, s);
        }
    }
    return latch(c, acse_residual_backward_impl(c->shadow, D_ckpt, n_steps, eps, wE, wN, dh, dV, dDaa, dDab, dDbb));
}

// ------------------------------------------------------------------------------ profiling
// Event pairs around every O(r^6) GEMM launch while profiling is on; read back (and summed in
// a fixed order) by acse_profile_read, which synchronises the stream.
int prof_begin(acse_ctx* c) {
    if (!c->prof_on) return ACSE_OK;
    if (c->prof_n >= ACSE_PROF_MAX) return ACSE_OK;   // ring full: later launches not timed
    cudaEvent_t* e = &c->prof_ev[2 * c->prof_n];
    if (!e[0]) {
        ACSE_CUDA_TRY(cudaEventCreate(&e[0]));
        ACSE_CUDA_TRY(cudaEventCreate(&e[1]));
    }
    ACSE_CUDA_TRY(cudaEventRecord(e[0], c->stream));
    return ACSE_OK;
}

int prof_end(acse_ctx* c) {
    if (!c->prof_on || c->prof_n >= ACSE_PROF_MAX) return ACSE_OK;
    ACSE_CUDA_TRY(cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->stream));
    c->prof_n++;
    return ACSE_OK;
}

static int prof_drain(acse_ctx* c) {
    if (c->prof_n == 0) return ACSE_OK;
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->prof_n; ++i) {
        float ms = 0.f;
        ACSE_CUDA_TRY(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
        c->prof_ms += ms;
        c->prof_count++;
    }
    c->prof_n = 0;
    return ACSE_OK;
}

extern "C" int acse_profile(acse_ctx* c, int enable) {
    if (!c) return ACSE_ERR_ARG;
    if (c->fine) ACSE_TRY(acse_profile(c->fine, enable));
    int s = prof_drain(c);
    c->prof_on = enable;
    c->prof_ms = 0.0;
    c->prof_count = 0;
    c->launches = 0;
    return latch(c, s);
}

extern "C" int acse_profile_read(acse_ctx* c, double* gemm_ms, long long* gemm_launches, long long* launches) {
    if (!c) return ACSE_ERR_ARG;
    int s = prof_drain(c);
    double fm = 0.0;
    long long fg = 0, fl = 0;
    if (s == ACSE_OK && c->fine) s = acse_profile_read(c->fine, &fm, &fg, &fl);
    if (gemm_ms) *gemm_ms = c->prof_ms + fm;
    if (gemm_launches) *gemm_launches = c->prof_count + fg;
    if (launches) *launches = c->launches + fl;
    return latch(c, s);
}

// ------------------------------------------------------------------------------ status
extern "C" int acse_sync_status(acse_ctx* c) {
    if (!c) return ACSE_ERR_ARG;
    if (c->fine) {
        const int sf = acse_sync_status(c->fine);
        if (sf != ACSE_OK) return latch(c, sf);
    }
    return latch(c, sync_and_status(c));
}

extern "C" int acse_clear_status(acse_ctx* c) {
    if (!c) return ACSE_ERR_ARG;
    c->last_error = ACSE_OK;
    if (c->w.tc_err && cudaMemsetAsync(c->w.tc_err, 0, sizeof(int), c->stream) != cudaSuccess) return ACSE_ERR_CUDA;
    return ACSE_OK;
}

extern "C" int acse_set_wait_bound_ns(acse_ctx* c, unsigned long long ns, int inject_stall) {
    if (!c) return ACSE_ERR_ARG;
    if (c->oz) return latch(c, oz_set_wait_ns(c, ns, inject_stall));
    if (c->opt.prec == ACSE_FP64) return inject_stall ? latch(c, ACSE_ERR_UNSUPPORTED) : ACSE_OK;
    return latch(c, tc_set_wait_ns(c, ns, inject_stall));
}
