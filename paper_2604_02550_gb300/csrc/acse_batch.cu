// Batched ACSE: several independent instances (electronic states, or molecules of different r)
// advanced together, one Euler step at a time, with
//   * one grouped GEMM launch per contraction pass covering every instance, spin sector and tile
//     (tensor-core precisions: a device-resident problem table; FP64: the grouped DFMA kernel),
//   * the per-instance elementwise chains on forked streams,
//   * the stopping rule of the Methods section evaluated on the device (per-instance frozen flags:
//     stop when E or ||A|| increases -- then the previous D is restored -- or when |dE| < 1e-6),
//   * the whole step captured once as a CUDA graph and replayed, so a run of n steps costs n graph
//     launches and no host synchronisation,
//   * tile widths chosen by a small autotuner (timed on the real operands at creation, cached per
//     process by the multiset of r).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "acse_internal.h"

int launch_axpy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev, double eps_mul,
                double* const out[3]);
int launch_energy(acse_ctx* c, const double* const D[3], double* E_dst);
int launch_axpy_energy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev,
                       double* E_dst);

// scalar slots of each instance's device scalar block (acse_ctx::w.scal, 16 doubles)
enum { S_N2 = 0, S_E = 1, S_EPS_USED = 3, S_EPREV = 9, S_N2PREV = 10, S_FROZEN = 11, S_STEPS = 12, S_EPS = 13,
       S_HAVEPREV = 14, S_RESTORE = 15 };

struct acse_batch {
    int n;
    int prec;
    acse_ctx** ctx;
    cudaStream_t stream;       // the batch's own capture stream (non-blocking)
    cudaStream_t user;         // the caller's stream: a run starts after its pending work
    cudaStream_t* sub;
    cudaEvent_t fork;
    cudaEvent_t* join;
    TcTable tab[2];
    int ntab;
    int tune_choice;       // 0: all BN=256, 1: all BN=128, 2: split by r^2 < split_r2
    int split_r2;
    double* D[3 * 64];     // owned D blocks per instance
    double* Dprev[3 * 64];
    int stop_rule;
    cudaGraphExec_t graph;
    int graph_ready;
    // trajectory record per instance (device): lambda and E of every accepted step, D_0 first;
    // instance i at hist + 2 i ACSE_HIST_CAP (lambda) and + ACSE_HIST_CAP (E), hcount[i] points
    double* hist;
    int* hcount;
    double* fitout;    // 6 doubles per instance: the last acse_batch_extrapolate results (device)
    // kernel count of the graph: per replay (counted while it was captured) and over all replays so far
    long long per_replay;
    long long replayed;
    long long tab_launches;   // grouped tensor-core GEMM launches issued (counted during the capture)
};
#define ACSE_HIST_CAP 4096

int fit_launch(const double* lam, const double* E, const int* count, int n_fixed, size_t stride, int ntraj,
               int n_skip, double* out, cudaStream_t st);

// ---------------------------------------------------------------------------- kernels
// Stopping rule for one instance at the start of a step (E = energy of the current D, N2 = ||A||^2 at
// the current D).  Sets the step's eps (0 when frozen) and, on an increase, requests a restore of
// the previous D.
__global__ void k_batch_stop(double* s, int stop_rule) {
    s[S_RESTORE] = 0.0;
    if (s[S_FROZEN] == 0.0 && stop_rule && s[S_HAVEPREV] != 0.0) {
        const bool up = s[S_E] > s[S_EPREV] || s[S_N2] > s[S_N2PREV];
        const bool conv = fabs(s[S_E] - s[S_EPREV]) < 1e-6;
        if (up || conv) {
            s[S_FROZEN] = up ? 1.0 : 2.0;
            if (up) {   // the step that led here is undone
                s[S_RESTORE] = 1.0;
                s[S_E] = s[S_EPREV];
                s[S_N2] = s[S_N2PREV];
                s[S_STEPS] -= 1.0;
            }
        }
    }
    s[S_EPS_USED] = s[S_FROZEN] == 0.0 ? s[S_EPS] : 0.0;
}

// After the update pass: remember the current state as "previous" (unless frozen).
__global__ void k_batch_prev(double* s) {
    if (s[S_FROZEN] == 0.0) {
        s[S_EPREV] = s[S_E];
        s[S_N2PREV] = s[S_N2];
        s[S_HAVEPREV] = 1.0;
        s[S_STEPS] += 1.0;
    }
}

// dst = src for the three blocks when the flag slot equals `when` (restore: flag S_RESTORE == 1;
// remember previous: flag S_FROZEN == 0).
__global__ void k_cond_copy3(size_t n4, const double* __restrict__ s, int slot, double when, const double* a0,
                             const double* a1, const double* a2, double* b0, double* b1, double* b2) {
    if (s[slot] != when) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 3 * n4; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / n4);
        const size_t g = e % n4;
        if (b == 0) b0[g] = a0[g];
        else if (b == 1) b1[g] = a1[g];
        else b2[g] = a2[g];
    }
}

// Trajectory record, at the end of a step: an undone step (restore) drops its point; a step taken
// (eps used > 0) appends lambda + eps and the new E, until the record is full.
__global__ void k_batch_hist(const double* __restrict__ s, double* __restrict__ hist, int* __restrict__ count) {
    int n = *count;
    if (s[S_RESTORE] == 1.0 && n > 1) --n;
    if (s[S_EPS_USED] != 0.0 && n < ACSE_HIST_CAP) {
        hist[n] = hist[n - 1] + s[S_EPS_USED];
        hist[ACSE_HIST_CAP + n] = s[S_E];
        ++n;
    }
    *count = n;
}

// A fresh record: lambda = 0 at the E of D_0.
__global__ void k_batch_hist_reset(const double* __restrict__ s, double* __restrict__ hist, int* __restrict__ count) {
    hist[0] = 0.0;
    hist[ACSE_HIST_CAP] = s[S_E];
    *count = 1;
}

static int cgrid(size_t n) {
    size_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}

// --------------------------------------------------------------------------- one step
static int gemm_pass(acse_batch* B) {
    if (B->prec == ACSE_FP64) {
        // FP64: every instance's nine GEMMs in one grouped DFMA launch (split in chunks of 40 inside)
        std::vector<GemmF64> all;
        for (int i = 0; i < B->n; ++i) {
            acse_ctx* c = B->ctx[i];
            GemmF64 g[9];
            int ng = 0;
            ACSE_TRY(acse_gemm_list_f64(c, g, &ng));
            all.insert(all.end(), g, g + ng);
        }
        return gemm_f64_grouped(B->ctx[0], all.data(), (int)all.size(), B->stream);
    }
    for (int t = 0; t < B->ntab; ++t) {
        ACSE_TRY(tc_table_launch(&B->tab[t], B->stream));
        B->tab_launches++;
    }
    return ACSE_OK;
}

static int fork_all(acse_batch* B) {
    ACSE_CUDA_TRY(cudaEventRecord(B->fork, B->stream));
    for (int i = 0; i < B->n; ++i) ACSE_CUDA_TRY(cudaStreamWaitEvent(B->sub[i], B->fork, 0));
    return ACSE_OK;
}

static int join_all(acse_batch* B) {
    for (int i = 0; i < B->n; ++i) {
        ACSE_CUDA_TRY(cudaEventRecord(B->join[i], B->sub[i]));
        ACSE_CUDA_TRY(cudaStreamWaitEvent(B->stream, B->join[i], 0));
    }
    return ACSE_OK;
}

static int batch_step(acse_batch* B) {
    const int n = B->n;
    ACSE_TRY(fork_all(B));
    for (int i = 0; i < n; ++i) {
        acse_ctx* c = B->ctx[i];
        const double* D[3] = {B->D[3 * i], B->D[3 * i + 1], B->D[3 * i + 2]};
        const double* Kh[3] = {c->w.Kh[0], c->w.Kh[1], c->w.Kh[2]};
        ACSE_TRY(acse_contract_pre(c, D, Kh, 1));
    }
    ACSE_TRY(join_all(B));
    ACSE_TRY(gemm_pass(B));
    ACSE_TRY(fork_all(B));
    for (int i = 0; i < n; ++i) {
        acse_ctx* c = B->ctx[i];
        Work& w = c->w;
        const size_t n4 = (size_t)c->r * c->r * c->r * c->r;
        ACSE_TRY(acse_contract_post(c, +1, 1.0, 1, w.A, w.scal + S_N2));
        k_batch_stop<<<1, 1, 0, c->stream>>>(w.scal, B->stop_rule);
        ACSE_LAUNCHED(c);
        // on an increase: back to the previous D (the residual of this step is then not used)
        k_cond_copy3<<<cgrid(3 * n4), 256, 0, c->stream>>>(n4, w.scal, S_RESTORE, 1.0, B->Dprev[3 * i],
                                                           B->Dprev[3 * i + 1], B->Dprev[3 * i + 2], B->D[3 * i],
                                                           B->D[3 * i + 1], B->D[3 * i + 2]);
        ACSE_LAUNCHED(c);
        const double* D[3] = {B->D[3 * i], B->D[3 * i + 1], B->D[3 * i + 2]};
        const double* Ac[3] = {w.A[0], w.A[1], w.A[2]};
        ACSE_TRY(acse_contract_pre(c, D, Ac, 0));
    }
    ACSE_TRY(join_all(B));
    ACSE_TRY(gemm_pass(B));
    ACSE_TRY(fork_all(B));
    for (int i = 0; i < n; ++i) {
        acse_ctx* c = B->ctx[i];
        Work& w = c->w;
        const size_t n4 = (size_t)c->r * c->r * c->r * c->r;
        ACSE_TRY(acse_contract_post(c, -1, 0.5, 0, w.U, nullptr));
        k_cond_copy3<<<cgrid(3 * n4), 256, 0, c->stream>>>(n4, w.scal, S_FROZEN, 0.0, B->D[3 * i], B->D[3 * i + 1],
                                                           B->D[3 * i + 2], B->Dprev[3 * i], B->Dprev[3 * i + 1],
                                                           B->Dprev[3 * i + 2]);
        ACSE_LAUNCHED(c);
        k_batch_prev<<<1, 1, 0, c->stream>>>(w.scal);
        ACSE_LAUNCHED(c);
        double* Dm[3] = {B->D[3 * i], B->D[3 * i + 1], B->D[3 * i + 2]};
        const double* Uc[3] = {w.U[0], w.U[1], w.U[2]};
        ACSE_TRY(launch_axpy_energy(c, Dm, Uc, w.scal + S_EPS_USED, w.scal + S_E));
        k_batch_hist<<<1, 1, 0, c->stream>>>(w.scal, B->hist + 2 * (size_t)ACSE_HIST_CAP * i, B->hcount + i);
        ACSE_LAUNCHED(c);
    }
    return join_all(B);
}

// ------------------------------------------------------------------------ autotuner
static std::mutex g_tune_mu;
static std::map<std::vector<int>, std::pair<int, int>> g_tune_cache;   // key: prec + sorted r's

static int build_tables(acse_batch* B, int choice, int split_r2) {
    for (int t = 0; t < B->ntab; ++t) tc_table_free(&B->tab[t]);
    B->ntab = 0;
    const int kind = (B->prec == ACSE_TF32 || B->prec == ACSE_TF32X3) ? 1 : 0;
    int bns[2];
    if (choice == 0) { bns[0] = 256; B->ntab = 1; }
    else if (choice == 1) { bns[0] = 128; B->ntab = 1; }
    else { bns[0] = 128; bns[1] = 256; B->ntab = 2; }
    // 256-wide tables run on CTA pairs unless the instances ask for one SM per tile (acse_opts.gemm_tile)
    const int pairs = B->ctx[0]->opt.gemm_tile != 1;
    for (int t = 0; t < B->ntab; ++t) ACSE_TRY(tc_table_init_mode(&B->tab[t], kind, bns[t], pairs));
    for (int i = 0; i < B->n; ++i) {
        acse_ctx* c = B->ctx[i];
        int t = 0;
        if (choice == 2) t = (c->r * c->r < split_r2) ? 0 : 1;
        ACSE_TRY(tc_table_append(&B->tab[t], c));
    }
    for (int t = 0; t < B->ntab; ++t) ACSE_TRY(tc_table_upload(&B->tab[t]));
    return ACSE_OK;
}

static int autotune(acse_batch* B) {
    std::vector<int> key;
    key.push_back(B->prec);
    for (int i = 0; i < B->n; ++i) key.push_back(B->ctx[i]->r);
    std::sort(key.begin() + 1, key.end());
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            B->tune_choice = it->second.first;
            B->split_r2 = it->second.second;
            return build_tables(B, B->tune_choice, B->split_r2);
        }
    }
    // operands: prepare every instance once (residual pass at its D)
    for (int i = 0; i < B->n; ++i) {
        acse_ctx* c = B->ctx[i];
        const double* D[3] = {B->D[3 * i], B->D[3 * i + 1], B->D[3 * i + 2]};
        const double* Kh[3] = {c->w.Kh[0], c->w.Kh[1], c->w.Kh[2]};
        ACSE_TRY(acse_contract_pre(c, D, Kh, 1));
        ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    struct Cand { int choice, split; };
    const Cand cands[] = {{0, 0}, {1, 0}, {2, 256}, {2, 576}, {2, 1024}};
    float best = 1e30f;
    Cand bc = {0, 0};
    cudaEvent_t e0, e1;
    ACSE_CUDA_TRY(cudaEventCreate(&e0));
    ACSE_CUDA_TRY(cudaEventCreate(&e1));
    for (const Cand& cd : cands) {
        ACSE_TRY(build_tables(B, cd.choice, cd.split));
        ACSE_TRY(gemm_pass(B));   // warm-up
        ACSE_CUDA_TRY(cudaEventRecord(e0, B->stream));
        for (int rep = 0; rep < 3; ++rep) ACSE_TRY(gemm_pass(B));
        ACSE_CUDA_TRY(cudaEventRecord(e1, B->stream));
        ACSE_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        ACSE_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            bc = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->tune_choice = bc.choice;
    B->split_r2 = bc.split;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_pair(bc.choice, bc.split);
    }
    return build_tables(B, bc.choice, bc.split);
}

// ------------------------------------------------------------------------------ ABI
extern "C" int acse_batch_destroy(acse_batch* B) {
    if (!B) return ACSE_ERR_ARG;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->graph_ready) cudaGraphExecDestroy(B->graph);
    for (int t = 0; t < B->ntab; ++t) tc_table_free(&B->tab[t]);
    for (int i = 0; i < B->n; ++i) {
        if (B->ctx && B->ctx[i]) acse_destroy(B->ctx[i]);
        if (B->sub && B->sub[i]) cudaStreamDestroy(B->sub[i]);
        if (B->join && B->join[i]) cudaEventDestroy(B->join[i]);
        for (int b = 0; b < 3; ++b) {
            if (B->D[3 * i + b]) cudaFree(B->D[3 * i + b]);
            if (B->Dprev[3 * i + b]) cudaFree(B->Dprev[3 * i + b]);
        }
    }
    if (B->hist) cudaFree(B->hist);
    if (B->hcount) cudaFree(B->hcount);
    if (B->fitout) cudaFree(B->fitout);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->stream) cudaStreamDestroy(B->stream);
    free(B->ctx);
    free(B->sub);
    free(B->join);
    free(B);
    return ACSE_OK;
}

extern "C" int acse_batch_create(acse_batch** out, int n, const acse_opts* opts, const double* const* h,
                                 const double* const* V, void* stream) {
    if (out) *out = nullptr;   // every failure leaves *out = NULL
    if (!out || !opts || !h || !V || n < 1 || n > 64) return ACSE_ERR_ARG;
    for (int i = 1; i < n; ++i)
        if (opts[i].prec != opts[0].prec) return ACSE_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (opts[i].recon != ACSE_RECON_V) return ACSE_ERR_UNSUPPORTED;   // the batch runs the V reconstruction
    if (opts[0].prec == ACSE_OZAKI) return ACSE_ERR_UNSUPPORTED;           // single contexts only
    acse_batch* B = (acse_batch*)calloc(1, sizeof(acse_batch));
    if (!B) return ACSE_ERR_NOMEM;
    B->n = n;
    B->prec = opts[0].prec;
    B->user = (cudaStream_t)stream;
    B->stop_rule = 1;
    B->ctx = (acse_ctx**)calloc(n, sizeof(acse_ctx*));
    B->sub = (cudaStream_t*)calloc(n, sizeof(cudaStream_t));
    B->join = (cudaEvent_t*)calloc(n, sizeof(cudaEvent_t));
    int s = (B->ctx && B->sub && B->join) ? ACSE_OK : ACSE_ERR_NOMEM;
    if (s == ACSE_OK && (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess))
        s = ACSE_ERR_CUDA;
    if (s == ACSE_OK && (cudaMalloc((void**)&B->hist, 2 * (size_t)ACSE_HIST_CAP * n * sizeof(double)) != cudaSuccess ||
                         cudaMalloc((void**)&B->hcount, n * sizeof(int)) != cudaSuccess ||
                         cudaMalloc((void**)&B->fitout, 6 * (size_t)n * sizeof(double)) != cudaSuccess ||
                         cudaMemset(B->hcount, 0, n * sizeof(int)) != cudaSuccess))
        s = ACSE_ERR_NOMEM;
    for (int i = 0; i < n && s == ACSE_OK; ++i) {
        if (cudaStreamCreateWithFlags(&B->sub[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming) != cudaSuccess) {
            s = ACSE_ERR_CUDA;
            break;
        }
        acse_opts o = opts[i];
        o.line_search = 0;
        o.check_inputs = 0;
        o.refine = 0;      // the batch steps in one precision
        s = acse_create(&B->ctx[i], &o, h[i], V[i], B->sub[i]);
        const size_t b4 = (size_t)o.r * o.r * o.r * o.r * sizeof(double);
        for (int b = 0; b < 3 && s == ACSE_OK; ++b)
            if (cudaMalloc((void**)&B->D[3 * i + b], b4) != cudaSuccess ||
                cudaMalloc((void**)&B->Dprev[3 * i + b], b4) != cudaSuccess ||
                cudaMemset(B->D[3 * i + b], 0, b4) != cudaSuccess)
                s = ACSE_ERR_NOMEM;
    }
    if (s != ACSE_OK) {
        acse_batch_destroy(B);
        return s;
    }
    *out = B;
    return ACSE_OK;
}

extern "C" int acse_batch_set_D(acse_batch* B, int i, const double* Daa, const double* Dab, const double* Dbb,
                                double eps) {
    if (!B || i < 0 || i >= B->n || !Daa || !Dab || !Dbb) return ACSE_ERR_ARG;
    acse_ctx* c = B->ctx[i];
    const size_t b4 = (size_t)c->r * c->r * c->r * c->r * sizeof(double);
    const double* src[3] = {Daa, Dab, Dbb};
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    for (int b = 0; b < 3; ++b) {
        ACSE_CUDA_TRY(cudaMemcpy(B->D[3 * i + b], src[b], b4, cudaMemcpyDefault));
        ACSE_CUDA_TRY(cudaMemcpy(B->Dprev[3 * i + b], src[b], b4, cudaMemcpyDefault));
    }
    // fresh trajectory: E of D, nothing previous, not frozen
    double sc[16];
    memset(sc, 0, sizeof(sc));
    sc[S_EPS] = eps;
    ACSE_CUDA_TRY(cudaMemcpy(c->w.scal, sc, sizeof(sc), cudaMemcpyHostToDevice));
    const double* Dc[3] = {B->D[3 * i], B->D[3 * i + 1], B->D[3 * i + 2]};
    ACSE_TRY(launch_energy(c, Dc, c->w.scal + S_E));
    k_batch_hist_reset<<<1, 1, 0, c->stream>>>(c->w.scal, B->hist + 2 * (size_t)ACSE_HIST_CAP * i, B->hcount + i);
    ACSE_LAUNCHED(c);
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ACSE_OK;
}

extern "C" int acse_batch_get_D(acse_batch* B, int i, double* Daa, double* Dab, double* Dbb) {
    if (!B || i < 0 || i >= B->n) return ACSE_ERR_ARG;
    acse_ctx* c = B->ctx[i];
    const size_t b4 = (size_t)c->r * c->r * c->r * c->r * sizeof(double);
    double* dst[3] = {Daa, Dab, Dbb};
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    for (int b = 0; b < 3; ++b)
        if (dst[b]) ACSE_CUDA_TRY(cudaMemcpy(dst[b], B->D[3 * i + b], b4, cudaMemcpyDefault));
    return ACSE_OK;
}

// Run nsteps steps (graph replays).  Per-instance results (host arrays of n): E after the run, ||A||^2
// at the last evaluated D, the number of steps taken (fewer than nsteps when the stopping rule
// froze the instance) and the stop reason (0 running, 1 E or ||A|| increased, 2 |dE| < 1e-6).
extern "C" int acse_batch_run(acse_batch* B, int nsteps, int stop_rule, double* E_out, double* norm2_out,
                              int* steps_out, int* reason_out) {
    if (!B || nsteps < 0) return ACSE_ERR_ARG;
    // order after the caller's pending work
    ACSE_CUDA_TRY(cudaEventRecord(B->fork, B->user));
    ACSE_CUDA_TRY(cudaStreamWaitEvent(B->stream, B->fork, 0));
    if (B->ntab == 0 && B->prec != ACSE_FP64) ACSE_TRY(autotune(B));
    if (B->stop_rule != stop_rule && B->graph_ready) {
        cudaGraphExecDestroy(B->graph);
        B->graph_ready = 0;
    }
    B->stop_rule = stop_rule;
    if (!B->graph_ready) {
        cudaGraph_t g;
        // the kernels the capture records are counted once per replay, not at the capture
        long long before[64];
        for (int i = 0; i < B->n; ++i) before[i] = B->ctx[i]->launches;
        B->tab_launches = 0;
        ACSE_CUDA_TRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
        int s = batch_step(B);
        cudaError_t e = cudaStreamEndCapture(B->stream, &g);
        B->per_replay = B->tab_launches;
        for (int i = 0; i < B->n; ++i) {
            B->per_replay += B->ctx[i]->launches - before[i];
            B->ctx[i]->launches = before[i];
        }
        if (s != ACSE_OK) return s;
        if (e != cudaSuccess) return ACSE_ERR_CUDA;
        e = cudaGraphInstantiate(&B->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return ACSE_ERR_CUDA;
        B->graph_ready = 1;
    }
    for (int k = 0; k < nsteps; ++k) {
        ACSE_CUDA_TRY(cudaGraphLaunch(B->graph, B->stream));
        B->replayed += B->per_replay;
    }
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    for (int i = 0; i < B->n; ++i) {
        double sc[16];
        ACSE_CUDA_TRY(cudaMemcpy(sc, B->ctx[i]->w.scal, sizeof(sc), cudaMemcpyDeviceToHost));
        if (E_out) E_out[i] = sc[S_E];
        if (norm2_out) norm2_out[i] = sc[S_N2];
        if (steps_out) steps_out[i] = (int)sc[S_STEPS];
        if (reason_out) reason_out[i] = (int)sc[S_FROZEN];
    }
    return ACSE_OK;
}

extern "C" int acse_batch_history(acse_batch* B, int i, double* lam, double* E, int cap, int* count) {
    if (!B || i < 0 || i >= B->n || cap < 0 || (cap > 0 && (!lam || !E))) return ACSE_ERR_ARG;
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    int n = 0;
    ACSE_CUDA_TRY(cudaMemcpy(&n, B->hcount + i, sizeof(int), cudaMemcpyDeviceToHost));
    const double* h = B->hist + 2 * (size_t)ACSE_HIST_CAP * i;
    const int k = n < cap ? n : cap;
    if (k > 0) {
        ACSE_CUDA_TRY(cudaMemcpy(lam, h, k * sizeof(double), cudaMemcpyDefault));
        ACSE_CUDA_TRY(cudaMemcpy(E, h + ACSE_HIST_CAP, k * sizeof(double), cudaMemcpyDefault));
    }
    if (count) *count = n;
    return ACSE_OK;
}

extern "C" int acse_batch_extrapolate(acse_batch* B, int n_skip, double* out) {
    if (!B || !out || n_skip < 0) return ACSE_ERR_ARG;
    ACSE_TRY(fit_launch(B->hist, B->hist + ACSE_HIST_CAP, B->hcount, 0, 2 * (size_t)ACSE_HIST_CAP, B->n, n_skip,
                        B->fitout, B->stream));
    ACSE_CUDA_TRY(cudaMemcpyAsync(out, B->fitout, 6 * (size_t)B->n * sizeof(double), cudaMemcpyDefault, B->stream));
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    return ACSE_OK;
}

extern "C" int acse_batch_info(const acse_batch* B, int* tune_choice, int* split_r2, long long* launches) {
    if (!B) return ACSE_ERR_ARG;
    if (tune_choice) *tune_choice = B->tune_choice;
    if (split_r2) *split_r2 = B->split_r2;
    if (launches) {
        long long s = B->replayed;
        for (int i = 0; i < B->n; ++i) s += B->ctx[i]->launches;
        *launches = s;
    }
    return ACSE_OK;
}

// The adjoint of one instance: acse_residual_backward in the instance's context, ordered after the
// batch's replays (its intermediate buffers are the replays' scratch; the trajectory state of the
// batch, D, the previous D and the per-instance scalars, is not touched).
extern "C" int acse_batch_residual_backward(acse_batch* B, int i, const double* const* D_ckpt, int n_steps,
                                            double eps, double wE, double wN, double* dh, double* dV, double* dDaa,
                                            double* dDab, double* dDbb) {
    if (!B || i < 0 || i >= B->n) return ACSE_ERR_ARG;
    ACSE_CUDA_TRY(cudaStreamSynchronize(B->stream));
    acse_ctx* c = B->ctx[i];
    ACSE_TRY(acse_residual_backward(c, D_ckpt, n_steps, eps, wE, wN, dh, dV, dDaa, dDab, dDbb));
    ACSE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ACSE_OK;
}
