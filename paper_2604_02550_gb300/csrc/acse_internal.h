// Internal declarations shared by the translation units of libacse.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/acse.h"

#define ACSE_MAX_R 64

// Packed number of the pair (a, b), a < b, among the r(r-1)/2 same-spin pairs (row-major over a):
// the row and column order of the packed same-spin GEMM operands and outputs of the split path.
__host__ __device__ __forceinline__ int pk_pair(int r, int a, int b) { return a * r - a * (a + 1) / 2 + (b - a - 1); }

// ------------------------------------------------------------------------------------------
// Dense GEMM problem: C[m*ldc + n] = alpha * sum_k A(m,k) B(n,k) (+ beta*C), with
//   A(m,k) = A[m*lda + k] (transA = 0, K-major) or A[k*lda + m] (transA = 1),
//   B(n,k) = B[n*ldb + k] (transB = 0, K-major) or B[k*ldb + n] (transB = 1).
// ------------------------------------------------------------------------------------------
struct GemmF64 {
    const double* A;
    const double* B;
    double* C;
    int M, N, K;
    int lda, ldb, ldc;
    double alpha, beta;
    int perm_r;   // 0: C row-major; r: particle-hole output stored permuted (see gemm_tc.cu)
    int transA, transB;
};

// Split-precision operand problem for the tensor-core path.  A and B are 16-bit (BF16) or
// 32-bit (TF32) element arrays with K' = nsplit * K columns (zero padded to a multiple of the
// K tile).  C is FP32.
struct GemmTC {
    const void* A;
    const void* B;
    float* C;
    int M, N, Kp;          // Kp = padded split-K length in elements
    int lda, ldb, ldc;     // elements
    float alpha;
};

// Problem table of one grouped tensor-core GEMM launch (gemm_tc.cu); TcBatch lives in device memory.
struct TcBatch;
struct TcTable {
    TcBatch* dev;
    TcBatch* host;
    int kind;        // 0 = bf16 (kind::f16), 1 = tf32
    int bn;          // tile width
    int bm;          // tile height: 128, or 256 for CTA pairs
    int pair;        // 1: CTA-pair kernel (cta_group::2, 256 x 256 tiles, one cluster of two CTAs per tile)
    int nclusters;   // CTA pairs of the persistent grid (co-resident clusters)
    int stages;
    size_t smem;
    int pers;        // 1: persistent kernel (one CTA per SM, double-buffered TMEM accumulators)
    int nsm;         // multiprocessors of the device (grid of the persistent kernel)
    int* sched;      // device: tile order of the persistent kernel, then the CTAs' start offsets
    int sched_cap;   // ints allocated at sched
};
// Longest-processing-time assignment of T tiles of the given costs to G CTAs: order[] lists the tile
// indices CTA by CTA (costliest first within a CTA), CTA c owning order[start[c] .. start[c+1]).
void tc_lpt_schedule(const long long* cost, int T, int G, int* order, int* start);
int tc_table_init(TcTable* t, int kind, int bn);
int tc_table_init_mode(TcTable* t, int kind, int bn, int pair);
int tc_use_pairs(const struct acse_ctx* c);   // CTA-pair GEMM tiles for this context (acse_opts.gemm_tile)
void tc_table_free(TcTable* t);
int tc_table_upload(TcTable* t);
int tc_table_append(TcTable* t, struct acse_ctx* c);
void tc_table_set_err(TcTable* t, int* err);
int tc_default_bn(int r);
int tc_unpack_pairs(struct acse_ctx* c);
int tc_mixed_prep_D(struct acse_ctx* c, const double* const D[3]);   // split operands of D (needs 1D)
int tc_mixed_prep_W(struct acse_ctx* c, const double* const W[3]);   // split operands of W, Z and w
int tc_make_Kh32(struct acse_ctx* c);                                  // FP32 copy of K/2 (once)
int tc_table_add_ld(TcTable* t, const void* A, size_t lda, const void* B, size_t ldb, float* C, int M, int N, int L,
                    int ldc, float alpha);
int tc_table_add(TcTable* t, const void* A, const void* B, float* C, int M, int N, int L, int ldc, float alpha);
int tc_table_launch(const TcTable* t, cudaStream_t st);

// Scratch layout of one context (all device memory, owned by the context).
struct Work {
    // K/2 blocks (the W of the residual), r^4 each
    double* Kh[3];
    // 1-RDM per spin (r^2 each) and the M blocks (r^4 each)
    double* gam;          // [2][r][r]
    double* M[3];
    // particle-hole layouts of M: diag (2r^2 x 2r^2), flips (r^2 x r^2)
    double* Md;
    double* Mf1;
    double* Mf2;
    // per-W intermediates
    double* Zd;
    double* Zf1;
    double* Zf2;
    double* w;            // [2][r][r]
    double* Q;            // [2][r][r]
    double* X[3];         // pair GEMM outputs M W^T (r^4 each)
    double* Y[3];         // pair GEMM outputs D W^T
    double* X5d;          // 4 r^4
    double* X5f1;
    double* X5f2;
    double* H[3];         // H_b = 4 Y_b - 12 (P - P'_{k<->l}) per block (r^4 each); G_b = H_b - s H_b^T
    double* zdiag;        // [4][r][r][r]: diagonal rows j = p of Z (for w)
    // residual, update, trial D for the line search
    double* A[3];
    double* U[3];
    double* Dt[3];
    // host-argument staging
    double* stage_in[3];
    double* stage_out[3];
    double* h;            // r^2 copy of h
    double* V;            // r^4 copy of V
    // scalars: [0] norm2, [1] E, [2] eps0 (line-search state), [3] eps used, [4..6] f0,f1,f2,
    //          [7] trace, [8] nonfinite flag
    double* scal;
    double* partial;      // reduction partials
    int npartial;
    // mixed-precision operand copies (bf16 or tf32 bit patterns), allocated when prec != FP64
    void* tc_pairA[3];    // [M; D] split, (2 r^2) x Kp
    void* tc_pairB[3];    // W split, r^2 x Kp
    void* tc_Md;          // (2r^2) x Kp2
    void* tc_Zd;
    void* tc_Mf[2];
    void* tc_Zf[2];
    float* tc_pairC[3];   // [X; Y] FP32 (2r^2 x r^2); same-spin sectors: only the rows i < j are formed
    float* tc_pairCp[3];  // same-spin sectors (aa, bb): the GEMM's packed [X; Y] (2P x P, P = r(r-1)/2
                          // pairs i < j on rows and columns), expanded into tc_pairC by antisymmetry
    int KpP;              // padded K (per split term) of the packed same-spin pair operands
    float* tc_X5d;
    float* tc_X5f[2];
    int Kp1, Kp2;         // padded K (per split term) for r^2 and 2 r^2 contractions
    // FP32 intermediates of the split-precision path
    float* M32[3];
    float* gam32;         // [2][r][r]
    float* w32;
    float* Q32;
    float* H32[3];
    float* zdiag32;
    int* tc_err;          // device flag: a bounded wait inside the tensor-core GEMM ran out
    // FP32 copies of the W operand of a pass (split path; Z and the W packs read these): K/2 (made
    // once), the residual A (written by the G assembly beside w.A) and a scratch copy for any other W
    float* Kh32[3];
    float* A32[3];
    float* W32s[3];
    // BF16x3 with r a multiple of 16: the B products x1 and x2^T of the four spin types, precomputed on
    // the tensor cores (acse_btc.cu; class 2 t + {0, 1}, r^2 floats per item), and the same-spin item ->
    // i r + j table (pairs i < j in packed order); null otherwise
    float* bx[8];
    int* pair_ij;
    double* bx64[8];   // Ozaki contexts: x1 and x2^T of the four B spin types for every pair (acse_zoz.cu)
};

struct acse_ctx {
    acse_opts opt;
    int r, N;
    cudaStream_t stream;
    int last_error;
    int device;
    int nsplit;           // split terms for the tensor-core path (3 for BF16x3, 1 for TF32)
    Work w;
    void* tc_plan;        // tensor-core GEMM plan (tensor maps etc.)
    void* adj;            // adjoint workspace (allocated by the first acse_residual_backward call)
    struct acse_ctx* shadow;   // ACSE_OZAKI companion of a split-precision context (its adjoint), or null
    void* ny;             // NY reconstruction workspace (acse_ny.cu), or null for V
    cudaStream_t aux[3];  // host <-> device copies of the three blocks run concurrently on these
    cudaEvent_t ev_fork, ev_join[3];
    int a32_valid;        // split path: w.A32 holds the FP32 values of the last A written to w.A
    int a64_skip;         // set by acse_step around its residual pass on the split path: the G assembly
                          // into w.A writes only the FP32 copy (all the update pass reads)
    int oz;               // ACSE_OZAKI: an FP64 context (opt.prec = ACSE_FP64) whose pass GEMMs run by
                          // the Ozaki scheme on the BF16 tensor cores (gemm_oz.cu)
    void* oz_plan;
    const double* cur_D[3];   // operands of the contraction pass in flight (FP64 GEMM list)
    const double* cur_W[3];
    // profiling: kernel launch count and CUDA-event timing of the O(r^6) GEMM launches
    long long launches;
    int prof_on;
    int prof_n;           // recorded event pairs (ring of ACSE_PROF_MAX)
    cudaEvent_t prof_ev[2 * 256];
    double prof_ms;       // summed GEMM time of pairs already read back
    long long prof_count;
    // precision schedule (opts.refine): the FP64-accurate context the steps continue in, whether the
    // switch has happened, and ||A||^2 of the last step taken before it (host copy; < 0: none yet)
    struct acse_ctx* fine;
    int refined;
    double sched_n2;
    int sched_steps;      // steps taken in the starting precision
    // CUDA graphs of acse_step: a call whose arguments (block and output pointers, eps) repeat those of
    // the previous call is captured once and replayed from then on (two executables kept, least
    // recently used replaced)
    struct StepGraph {
        cudaGraphExec_t exec;
        const void* key[6];
        double eps;
        long long launches;   // kernels one replay runs
        unsigned long long used;
    } sg[2];
    const void* sg_seen[6];   // arguments of the previous direct call
    double sg_seen_eps;
    int sg_seen_valid;
    int sg_refused;           // a capture failed once: direct calls only
    unsigned long long sg_tick;
};
#define ACSE_PROF_MAX 256

// Spin-flip specialisation in force (opts.singlet on a split-precision context): only the alpha-led
// half of the spin sectors is computed and the beta-beta results are taken from alpha-alpha.
static inline bool acse_singlet(const acse_ctx* c) { return c->opt.singlet && c->opt.prec != ACSE_FP64; }

// count a kernel launch of context c and check the launch error
#define ACSE_LAUNCHED(c)                                                      \
    do {                                                                      \
        (c)->launches++;                                                      \
        if (cudaGetLastError() != cudaSuccess) return ACSE_ERR_CUDA;          \
    } while (0)

int prof_begin(acse_ctx* c);

// NY reconstruction (acse_ny.cu)
int ny_alloc(acse_ctx* c);
void ny_free(acse_ctx* c);
int ny_pass(acse_ctx* c);
const void* ny_terms(acse_ctx* c, int t);
int ny_set_attrs();
int prof_end(acse_ctx* c);

// error helpers ---------------------------------------------------------------------------
#define ACSE_CUDA_TRY(expr)                                                   \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) return ACSE_ERR_CUDA;                          \
    } while (0)

#define ACSE_TRY(expr)                                                        \
    do {                                                                      \
        int _s = (expr);                                                      \
        if (_s != ACSE_OK) return _s;                                         \
    } while (0)

// kernels (acse_elem.cu) -------------------------------------------------------------------
int launch_build_K(acse_ctx* c);
int launch_gamma(acse_ctx* c, const double* const D[3]);
int launch_gamma_M(acse_ctx* c, const double* const D[3]);
int launch_pack_Mph(acse_ctx* c);
int launch_W_intermediates(acse_ctx* c, const double* const W[3]);
int launch_build_B(acse_ctx* c);
int launch_Z_tiled(acse_ctx* c, const double* const W[3], const float* const W32[3]);
int launch_B_tiled(acse_ctx* c);
int launch_Z_tc(acse_ctx* c, const float* const W32[3], int ntypes, const int* tmap);   // acse_ztc.cu
int launch_Z_oz(struct acse_ctx* c, const double* const W[3], int ntypes, const int* tmap);   // acse_zoz.cu
int launch_Bx_oz(struct acse_ctx* c);                                                           // acse_zoz.cu
int launch_Bx_tc(acse_ctx* c);                                                           // acse_btc.cu
int tiled_set_attrs();
int launch_Q(acse_ctx* c);
int launch_assemble_G(acse_ctx* c, int sW, double scale, int apply_mask, double* const out[3],
                      double* norm2_dst);
int launch_energy(acse_ctx* c, const double* const D[3], double* E_dst);
int launch_axpy_energy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev,
                       double* E_dst);
int launch_axpy(acse_ctx* c, double* const D[3], const double* const U[3], const double* eps_dev,
                double eps_mul, double* const out[3]);
int launch_line_search(acse_ctx* c);
int launch_trace_check(acse_ctx* c, const double* const D[3]);
int launch_copy_scalar(acse_ctx* c, double* dst, const double* src);

// GEMM back ends ------------------------------------------------------------------------------
int gemm_f64_grouped(acse_ctx* c, const GemmF64* probs, int nprob, cudaStream_t s);
// 2-D bf16 tensor map (128-byte swizzle, box 64 x box_rows) over `rows` rows of `inner_elems`
// elements, consecutive rows `row_stride` elements apart; `map` points to a CUtensorMap.
int tc_encode_map_bf16(void* map, const void* base, int rows, int inner_elems, int box_rows, size_t row_stride);
// Ozaki-scheme FP64 GEMMs of the contraction pass (gemm_oz.cu)
int oz_plan_create(acse_ctx* c);
void oz_plan_destroy(acse_ctx* c);
int oz_slice_operands(acse_ctx* c, int prep_D);   // the pass's FP64 operands -> scaled bf16 slices
int oz_gemm_launch(acse_ctx* c);                   // every GEMM of the pass, one persistent launch
int oz_set_wait_ns(acse_ctx* c, unsigned long long ns, int inject_stall);
// Any list of up to 12 FP64 GEMMs (alpha a power of two, beta 0 or 1, operands possibly transposed) by
// the Ozaki scheme; `slot` (0 or 1) names the list's plan, built on its first use (the adjoint's lists)
int oz_gemm_list(acse_ctx* c, const GemmF64* g, int n, int slot);

// contraction pass in three phases (acse_api.cu): operands, the O(r^6) GEMMs, assembly
int acse_contract_pre(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D);
int acse_contract_gemm(acse_ctx* c);
int acse_contract_post(acse_ctx* c, int sW, double scale, int mask, double* const out[3], double* norm2_dst);
int acse_gemm_list_f64(acse_ctx* c, GemmF64* g, int* n);
int acse_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int sW, double scale, int mask,
                  double* const out[3], double* norm2_dst, int prep_D);
