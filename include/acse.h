/*
 * acse.h -- C ABI of libacse: the ACSE residual / propagation hot path on one GB300 GPU.
 *
 * Method (arXiv 2604.02550): the anti-Hermitian contracted Schroedinger equation residual
 *     A^{ij}_{kl} = <psi| [a+_i a+_j a_l a_k, H] |psi>                         (Eq. residual_2quant)
 * written in the 2-RDM 2D and the 3-RDM 3D (Eq. residual, Appendix B), with 3D replaced by
 * the Valdemoro reconstruction from the 1-RDM and the 2-cumulant (Eq. 3rdm_recon,
 * Appendix C) and contracted without ever being stored, and the Euler propagation step
 *     2U^{ij}_{kl} = <psi| [a+_i a+_j a_l a_k, A^] |psi>,  2D <- 2D + eps 2U     (Eq. update).
 *
 * Conventions (fixed by brute-force Fock-space checks where the printed equations are garbled):
 *   * 2D^{pq}_{rs} = 1/2 <a+_p a+_q a_s a_r>;  Tr 2D = N(N-1)/2.
 *   * Spin blocks, spatial indices 0..r-1, full-square row-major [i][j][k][l]:
 *       X_aa = X^{ia ja}_{ka la},  X_ab = X^{ia jb}_{ka lb},  X_bb = X^{ib jb}_{kb lb}.
 *     Each block is r^4 doubles.  The aa and bb blocks are antisymmetric in (i,j) and in (k,l).
 *   * h: r x r one-electron integrals; V: r^4 two-electron integrals in chemist's notation
 *     (pq|rs) stored [p][q][r][s].
 *   * Reduced Hamiltonian (Eq. 2):  K = 1/2(<pq|rs> - <pq|sr>)
 *         + (h_pr d_qs + h_qs d_pr - h_ps d_qr - h_qr d_ps) / (2(N-1)),  <pq|rs> = (pr|qs),
 *     so that E = sum K.2D = sum_aa + sum_bb + 4 sum_ab.
 *   * A is the commutator itself; the printed Eq. (residual) equals -A.
 *   * 2U = 1/2 <[a+a+aa, A^]> with A^ = sum A^{pq}_{rs} a+_p a+_q a_s a_r (so dE/deps = -||A||^2).
 *   * ||A||^2 = ||A_aa||^2 + ||A_bb||^2 + 4 ||A_ab||^2 (spin-orbital Frobenius norm), taken
 *     before the optional all-active mask (Results: norms before zeroing).
 *
 * Pointers: every array argument may be a device pointer or a host pointer (pageable or
 * pinned); the library checks each with cudaPointerGetAttributes.  Device pointers are used
 * in place and the call is asynchronous on the context's stream.  Host arguments are staged
 * through context-owned device buffers; a call with any host output returns only after the
 * stream has finished it.  The caller owns every buffer it passes; the library never frees
 * them.  Scalar outputs (E, norm2, eps) follow the same rule.
 *
 * Errors: every function returns ACSE_OK (0) or a negative acse_status.  No exception or
 * abort crosses the ABI.  The last error is also latched in the context (acse_last_error).
 */
#ifndef ACSE_H
#define ACSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acse_ctx acse_ctx;

typedef enum {
    ACSE_OK = 0,
    ACSE_ERR_ARG = -1,        /* null or inconsistent argument                         */
    ACSE_ERR_SHAPE = -2,      /* r, N or active range out of the supported range        */
    ACSE_ERR_NONFINITE = -3,  /* NaN or Inf detected in an input or a result           */
    ACSE_ERR_TRACE = -4,      /* Tr 2D differs from N(N-1)/2 beyond 1e-8 relative        */
    ACSE_ERR_CUDA = -5,       /* a CUDA runtime / driver call failed                   */
    ACSE_ERR_TIMEOUT = -6,    /* a bounded device-side wait ran out                    */
    ACSE_ERR_NOMEM = -7,      /* device allocation failed at context creation          */
    ACSE_ERR_UNSUPPORTED = -8, /* option not built (e.g. a reconstruction not available) */
    ACSE_ERR_TOO_LARGE = -9    /* r above the static scratch of acse_energy_noalloc (64)  */
} acse_status;

/* Arithmetic of the O(r^6) contractions (everything else, the 1-RDM, norms, energy, axpy and line search,
 * stays FP64; the r^5 and r^4 intermediates run in FP32 in the split modes):
 *   ACSE_FP64    FP64 FMA throughout;
 *   ACSE_BF16X3  x = hi + lo (two bf16), products hi.hi + hi.lo + lo.hi, FP32 accumulation (about 2^-16
 *                relative per product);
 *   ACSE_TF32    one tf32 product, FP32 accumulation (about 2^-11);
 *   ACSE_TF32X3  x = hi + lo (two tf32), products hi.hi + hi.lo + lo.hi, FP32 accumulation (about 2^-21;
 *                limited by the FP32 intermediates);
 *   ACSE_OZAKI   FP64-accurate: every intermediate is FP64 as in ACSE_FP64, and each O(r^6) GEMM runs by
 *                the modular form of the Ozaki scheme (Ozaki, Uchino and Imamura, "Ozaki Scheme II",
 *                2025) on the BF16 tensor cores: each row of an operand is scaled by a power of two and
 *                rounded to an integer of min(6 oz_slices, 53) bits below its leading bit; the integer
 *                product is computed modulo T pairwise coprime moduli <= 127 (residues exact in bf16,
 *                sums exact in FP32, T the least count that covers the product: 17 at r = 48 with 8
 *                slices) and rebuilt exactly by the Chinese remainder theorem, with one rounding to FP64.
 *                With the default 8 (48 bits) the GEMM error is of the order of 2^-48 |A||B| K, below
 *                that of FP64 FMA.  The O(r^5) products of the pass (Z and the B products, r a multiple
 *                of 16) run by the six-bit slice form of the scheme (error-free splitting, Ozaki, Ogita,
 *                Oishi and Rump, Numer. Algorithms 59, 2012) with `oz_slices` slices.  The adjoint's
 *                O(r^6) GEMMs run by the modular form. */
typedef enum { ACSE_FP64 = 0, ACSE_BF16X3 = 1, ACSE_TF32 = 2, ACSE_TF32X3 = 3, ACSE_OZAKI = 4 } acse_prec;
/* 3-RDM reconstruction (Eq. 3rdm_recon / Eq. NY):
 *   ACSE_RECON_V   Valdemoro: the 3-cumulant is neglected;
 *   ACSE_RECON_NY  Nakatsuji-Yasuda: the 3-cumulant 1/6 sum_a sigma_a A(2Delta^{ia}_{rq} 2Delta^{jp}_{al})
 *                  is added, sigma_a = +1 for the first n_alpha alpha and the first n_beta beta spatial
 *                  orbitals (the Hartree-Fock occupation by orbital index), -1 otherwise.  Its
 *                  contractions run as dense spin-orbital GEMMs (n = 2r; memory about 12 n^4 elements);
 *                  not available for acse_residual_backward or the batch (ACSE_ERR_UNSUPPORTED). */
typedef enum { ACSE_RECON_V = 0, ACSE_RECON_NY = 1 } acse_recon;

typedef struct {
    int r;             /* spatial orbitals, 2 <= r <= 64                                    */
    int n_alpha;       /* alpha electrons                                                   */
    int n_beta;        /* beta electrons; N = n_alpha + n_beta >= 2                         */
    int prec;          /* acse_prec: arithmetic of the O(r^6) contractions                  */
    int recon;         /* acse_recon                                                        */
    int mask_active;   /* 1: zero A where i,j,k,l all lie in [act_lo, act_hi) (Methods)     */
    int act_lo, act_hi;
    int line_search;   /* 1: acse_step picks eps from ||A(D + e U)||^2 at {0, e0, 2 e0}     */
    double eps0;       /* initial trial step of the line search (e0); 0 -> 1e-3             */
    int check_inputs;  /* 1: acse_residual / acse_step verify Tr 2D and finiteness (syncs)  */
    int singlet;       /* 1: the caller asserts spin-flip symmetry (n_alpha = n_beta, D_aa = D_bb,
                        * D_ab^{ij}_{kl} = D_ab^{ji}_{lk}: singlets and any Ms = 0 state with that
                        * symmetry); the split precisions then compute only the alpha-led half of
                        * the spin sectors and copy the beta-beta block of A, U from alpha-alpha
                        * (Theory: for a singlet the aa and bb residual blocks coincide).  Ignored
                        * by ACSE_FP64 and ACSE_OZAKI; rejected (ACSE_ERR_ARG) when n_alpha !=
                        * n_beta.  The library does not symmetrise D: on an asymmetric D the
                        * beta-beta results are those of the alpha-alpha block.             */
    int oz_slices;     /* ACSE_OZAKI: accuracy in 6-bit units, 4..10; 0 -> 8: the O(r^6) GEMM
                        * operands keep min(6 oz_slices, 53) bits, the O(r^5) products use
                        * oz_slices six-bit slices                                          */
    int refine;        /* precision schedule of acse_step: 0 off; 1 the steps run in `prec` (any precision,
                        * ACSE_OZAKI with oz_slices included) until the switch rule fires, every later step
                        * in ACSE_OZAKI with refine_slices slices (FP64-accurate), from the same D and
                        * line-search state.  Rule, checked after every step: switch once ||A||^2 has
                        * fallen by less than refine_tol (relative) over the step, or risen.  The
                        * FP64-accurate context is created here with this one (its workspace besides);
                        * while the schedule has not switched, acse_step reads ||A||^2 back to the host
                        * after every step (one stream synchronisation per step).  acse_residual and
                        * acse_energy run in the precision in force.  Not with opts.singlet.            */
    int refine_slices; /* slices of the refined precision, 4..10; 0 -> 8                                */
    double refine_tol; /* relative fall of ||A||^2 per step below which the schedule switches; 0 -> 1e-2 */
    int gemm_tile;     /* tiling of the tensor-core O(r^6) GEMMs (every precision but ACSE_FP64; r >= 16):
                        * 0 default (the CTA-pair form), 1 one SM per 128 x 256 output tile, 2 CTA pairs:
                        * clusters of two CTAs on two SMs share each 256 x 256 tile through the pair MMA
                        * (tcgen05 cta_group::2), each CTA loading half of both operand tiles.  The results
                        * are the same in both forms (same products, same FP32 accumulation order).  For
                        * r < 16 the tiles are 128 x 128 on one SM whatever the value.  The NY GEMMs and the
                        * adjoint's Ozaki GEMMs follow it; a batch follows its first instance's value.   */
} acse_opts;

/* Create a context for one problem.  h (r*r) and V (r^4, chemist's (pq|rs)) are read once to
 * build the spin-blocked reduced Hamiltonian K of Eq. (2); they may be freed afterwards.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream) on which every call of this
 * context is ordered.  All device workspace of the forward calls is allocated here (about 40 r^4
 * doubles plus the split-precision operand copies, and the FP64-accurate context of a precision
 * schedule), so acse_energy, acse_residual and acse_step allocate nothing.  The one exception is
 * acse_residual_backward: its first call on a context allocates the adjoint workspace (about 65 r^4
 * doubles, 2.8 GB at r = 48) and, for a split precision, the ACSE_OZAKI companion context; both stay
 * until acse_destroy.  On any failure *ctx is set to NULL (when ctx itself is not NULL) and nothing stays
 * allocated. */
int acse_create(acse_ctx** ctx, const acse_opts* opts, const double* h, const double* V,
                void* cuda_stream);

/* Free the context and its workspace (synchronises its stream first). */
int acse_destroy(acse_ctx* ctx);

/* Energy E = sum K.2D (Eq. 2 with the convention above), FP64 with a fixed reduction order.
 * D blocks: 3 x r^4 doubles; E: one double. */
int acse_energy(acse_ctx* ctx, const double* Daa, const double* Dab, const double* Dbb, double* E);

/* Residual A = <[a+_i a+_j a_l a_k, H]> (Eq. residual with the Valdemoro 3-RDM of App. C,
 * contracted without storing it) for the 2-RDM D.  Writes the three A blocks (3 x r^4 doubles)
 * and ||A||^2 (one double, before the mask).  The mask, if enabled, is applied to A. */
int acse_residual(acse_ctx* ctx, const double* Daa, const double* Dab, const double* Dbb,
                  double* Aaa, double* Aab, double* Abb, double* norm2);

/* One Euler step of Eq. (update) in place: A = residual(D) (masked if enabled),
 * U = 1/2 <[a+a+aa, A^]> with the same reconstructed 3-RDM, D <- D + eps U.
 * eps: the fixed step, or ignored when opts.line_search = 1 (then eps is chosen on the
 * device from ||A(D + e U)||^2 at e in {0, e0, 2 e0}: the minimiser of the parabola through
 * them when it is convex, clamped to [e0/4, 2 e0], otherwise the better of e0 and 2 e0; the
 * next step's e0 is the accepted eps).
 * Outputs (each may be NULL): E_out = E after the step, norm2_out = ||A||^2 at the D before the
 * step, eps_used = the step taken.
 * When the blocks and outputs are device memory (or NULL), input checks, the precision schedule and
 * profiling are off and cuda_stream is a stream of the caller's (not the legacy default stream, not being
 * captured), a call whose arguments (pointers and eps) repeat those of the previous call is captured
 * into a CUDA graph, and later calls with those arguments replay it (two graphs are kept per context);
 * the replay runs the same kernels with the same arguments in the same order, so the results are those
 * of a direct call.  If a capture fails, the context runs every later step directly. */
int acse_step(acse_ctx* ctx, double* Daa, double* Dab, double* Dbb, double eps,
              double* E_out, double* norm2_out, double* eps_used);

/* Adjoint (not in the paper).  For f = wE * E(D_n) + wN * ||A(D_n)||^2 after n fixed Euler steps
 * D_{k+1} = D_k + eps U(D_k) from D_0 (mask as in opts, no line search), returns the gradient of
 * f with respect to h (r*r), V (r^4, chemist's order) and the three blocks of D_0.
 * D_ckpt: n_steps+1 checkpoints, D_ckpt[3k+0..2] = (Daa, Dab, Dbb) of D_k (any of them may be
 * NULL except D_0; missing ones are recomputed from the previous one).  dh and dV are
 * symmetrised (h: p<->q; V: the 8-fold permutational symmetry); dD is projected onto tensors
 * with the symmetries of a 2-RDM (antisymmetric within pairs, pair-Hermitian).  Each output
 * may be NULL.  The reverse sweep is FP64-accurate: FP64 FMA GEMMs in an ACSE_FP64 context, GEMMs by
 * the Ozaki scheme on the tensor cores in an ACSE_OZAKI context; a context in a split precision runs it
 * in an ACSE_OZAKI companion context the library creates on first use (same integrals and options,
 * 8 slices), so the gradient is the FP64-accurate adjoint along the trajectory the checkpoints
 * describe: pass every checkpoint of the split-precision forward run (checkpoints left NULL are
 * recomputed in the companion's precision). */
int acse_residual_backward(acse_ctx* ctx, const double* const* D_ckpt, int n_steps, double eps,
                           double wE, double wN, double* dh, double* dV,
                           double* dDaa, double* dDab, double* dDbb);

/* State of the precision schedule (opts.refine): *refined = 1 once acse_step has switched to the
 * FP64-accurate precision, *steps = the steps taken in the starting precision (host pointers, each may be
 * NULL; both 0 without a schedule). */
int acse_schedule_state(const acse_ctx* ctx, int* refined, int* steps);

/* Batched propagation: n independent instances (electronic states, or molecules with different r)
 * advanced together.  Each Euler step runs one grouped GEMM launch per contraction pass over all
 * instances, spin sectors and tiles, with the per-instance elementwise work on forked streams; the
 * step is captured once as a CUDA graph and replayed.  The Methods-section stopping rule runs on the
 * device per instance: when E or ||A|| increases the previous D is restored and the instance is
 * frozen; when |dE| < 1e-6 Eh it is frozen at the new D.  Tile widths of the grouped tensor-core
 * launch are chosen on the first run by timing candidate partitions on the real operands (cached per
 * process by the multiset of r and the precision).
 *   opts, h, V: arrays of n (all instances share opts[0].prec; line search and input checks are off).
 *   acse_batch_set_D: instance i's 2-RDM (device or host pointers, copied) and its step eps; resets
 *     its trajectory state.  acse_batch_get_D copies the current blocks out.
 *   acse_batch_run: nsteps graph replays; per instance (host arrays of n, each may be NULL): E and
 *     ||A||^2 at the current D, accepted steps, stop reason (0 running, 1 E or ||A|| rose, 2 converged).
 *   acse_batch_info: the tile choice (0 all 256 wide, 1 all 128 wide, 2 split at r^2 = split_r2) and
 *     the kernels launched so far (a graph replay counts the kernels it runs).  1 <= n <= 64 (ACSE_ERR_ARG otherwise, and for mixed precisions);
 *     ACSE_ERR_UNSUPPORTED for the NY reconstruction or ACSE_OZAKI; a failed create leaves *batch NULL.
 *   acse_batch_residual_backward: acse_residual_backward for instance i (its integrals and options; the
 *     checkpoints D_ckpt as there, for example read with acse_batch_get_D after one-step runs), run in
 *     the instance's own context once the batch's pending replays are done; synchronous (returns when
 *     the outputs are written).  Its first call on an instance allocates that instance's adjoint
 *     workspace as acse_create describes. */
typedef struct acse_batch acse_batch;
int acse_batch_create(acse_batch** batch, int n, const acse_opts* opts, const double* const* h,
                      const double* const* V, void* cuda_stream);
int acse_batch_destroy(acse_batch* batch);
int acse_batch_set_D(acse_batch* batch, int i, const double* Daa, const double* Dab, const double* Dbb,
                     double eps);
int acse_batch_get_D(acse_batch* batch, int i, double* Daa, double* Dab, double* Dbb);
int acse_batch_run(acse_batch* batch, int nsteps, int stop_rule, double* E_out, double* norm2_out,
                   int* steps_out, int* reason_out);
int acse_batch_info(const acse_batch* batch, int* tune_choice, int* split_r2, long long* launches);
int acse_batch_residual_backward(acse_batch* batch, int i, const double* const* D_ckpt, int n_steps, double eps,
                                 double wE, double wN, double* dh, double* dV, double* dDaa, double* dDab,
                                 double* dDbb);

/* Fit of the asymptotic regime of an energy trajectory.  The Results section describes the energy along
 * lambda = eps n (eps the Euler step, n the iteration; with varying steps lambda_n is the sum of the steps
 * before n) as an exponentially damped region followed by an asymptotic regime in which E changes about
 * linearly in lambda, and the Conclusions propose extrapolation and fitting to estimate the solution once a
 * trajectory stably enters that regime; the paper gives no fit.  The library fits
 *     E(lambda) ~ a + b lambda + c exp(-k lambda),  k > 0,
 * by least squares over the points n >= n_skip: in t = (lambda - lambda_first)/span, kappa = k span is
 * scanned on 256 points evenly spaced in log kappa over [0.25, 4 (m - 1)] (m fitted points), the best
 * point refined to dF/dkappa = 0 by bisection between its neighbours; a is the extrapolated energy (the
 * asymptote's value at lambda = 0), b its slope.
 *   acse_extrapolate: lam, E (n doubles each) and out (6 doubles: a, b, c, k, rss, flag) are device memory
 *     of the current device (or managed); 4 <= n - n_skip <= 4096 (ACSE_ERR_SHAPE otherwise); asynchronous
 *     on cuda_stream.  flag: 0 refined minimum, 1 minimum on the edge of the kappa grid or not bracketed
 *     (no refinement), 3 lambda not increasing (then a..rss are NaN).
 *   acse_batch_history: the batch records, per instance, lambda and E of D_0 and of every accepted step
 *     (an undone step's point is dropped; at most 4096 points).  Copies up to cap points of instance i
 *     into lam and E (host or device) and sets *count to the number recorded.
 *   acse_batch_extrapolate: the fit of every instance's record in one launch (one block per instance);
 *     out: host array of 6 n doubles (flag 2 and NaNs for an instance with fewer than n_skip + 4 points). */
int acse_extrapolate(int n, const double* lam, const double* E, int n_skip, double* out, void* cuda_stream);
int acse_batch_history(acse_batch* batch, int i, double* lam, double* E, int cap, int* count);
int acse_batch_extrapolate(acse_batch* batch, int n_skip, double* out);

/* Profiling (not part of the method).  acse_profile(ctx, 1) resets the counters and starts
 * recording a CUDA-event pair around every O(r^6) GEMM launch of this context (up to 256
 * launches between reads; while it is on, acse_step runs directly, without its CUDA graph);
 * acse_profile(ctx, 0) stops and resets the counters too.  acse_profile_read synchronises the
 * context's stream and returns the summed GEMM time in ms, the number of timed GEMM launches,
 * and the number of kernels this context launched since the last reset (a graph replay counts the
 * kernels it runs).  Host pointers. */
int acse_profile(acse_ctx* ctx, int enable);
int acse_profile_read(acse_ctx* ctx, double* gemm_ms, long long* gemm_launches, long long* launches);

/* Device status.  The tensor-core GEMM bounds every device-side wait; when one runs out the
 * kernel raises a device flag, drains its copies, frees its tensor memory and returns.
 * acse_sync_status synchronises the context's stream and returns ACSE_ERR_TIMEOUT if the flag is
 * set (calls that synchronise anyway report it too); acse_clear_status clears the flag and the
 * latched error.  acse_set_wait_bound_ns sets the bound of those waits (0 = default, 4 s);
 * with inject_stall = 1 the GEMM's MMA-issuing thread first waits on a barrier that nothing
 * signals, so every tile runs into the bound and the call ends with ACSE_ERR_TIMEOUT (a
 * host-side fault-injection knob for testing the timeout path; no fault, no hang).  Tensor-core
 * precisions only (ACSE_ERR_UNSUPPORTED for inject_stall on FP64). */
int acse_sync_status(acse_ctx* ctx);
int acse_clear_status(acse_ctx* ctx);
int acse_set_wait_bound_ns(acse_ctx* ctx, unsigned long long ns, int inject_stall);

/* Allocation-free energy trace.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they need an energy -- code running under a
 * framework or memory manager that owns the whole device heap, code on a latency-critical path
 * that must not risk the implicit device synchronisation of cudaMalloc/cudaFree, or callers that
 * hold only integrals and a 2-RDM and no context.  It computes the same E = sum K.2D as
 * acse_energy (K formed element by element inside the kernel from h and V, so no K buffer) and
 * allocates nothing: its only scratch is a file-scope static device array of 64 x 64 doubles
 * (32 KiB, held by every GPU that loads the library until the process exits), one FP64 partial
 * sum per (i, j).
 *   r, n_alpha, n_beta: as in acse_opts and checked as acse_create checks them (2 <= r,
 *     n_alpha <= r, n_beta <= r, N = n_alpha + n_beta >= 2; ACSE_ERR_SHAPE otherwise); r <= 64,
 *     larger r returns ACSE_ERR_TOO_LARGE.
 *   h (r*r), V (r^4, chemist's (pq|rs)), Daa, Dab, Dbb (r^4 each), E (one double): device memory
 *     of the CURRENT device, or managed memory (a host pointer or another GPU's memory returns
 *     ACSE_ERR_ARG); the caller owns all of them.
 *   cuda_stream: the cudaStream_t the two kernels are launched on; the call is asynchronous.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and caches it with the identity of the device's CUDA context (after a device
 * reset the next call looks it up again); make that first call before any stream capture.  Every
 * call shares the one array and it keeps the last call's contents; nothing in it needs to start
 * at zero (each call writes every slot it reads before reading it), but calls whose kernels
 * overlap on the GPU (other streams, other threads) race on it and must be ordered by the
 * caller. */
int acse_energy_noalloc(int r, int n_alpha, int n_beta, const double* h, const double* V,
                        const double* Daa, const double* Dab, const double* Dbb, double* E,
                        void* cuda_stream);

/* Plan of the modular Ozaki GEMM (ACSE_OZAKI), on the host only (no device access; not part of the
 * method): for a context with oz_slices = S (4..10) whose longest O(r^6) contraction has length kmax
 * (2 r^2 for the pass; 1 <= kmax <= 8192), and one of its GEMMs of contraction length k (1 <= k <= kmax),
 * the number T of moduli (the least whose product P covers 4 kmax 2^(2 min(6S, 53))), the bits kept below
 * a row's leading bit (min(6S, 53), fewer only if P cannot cover the product at that k), the K chunks of
 * one residue product (64 * 64 elements at most each), and the moduli themselves (moduli: room for 19
 * ints, or NULL; any other output may be NULL too).  ACSE_ERR_ARG outside those ranges. */
int acse_ozaki_plan_info(int oz_slices, int kmax, int k, int* moduli_count, int* bits, int* chunks,
                         int* moduli);

/* Text of a status code. */
const char* acse_strerror(int status);

/* Last error latched in the context (ACSE_OK if none since creation). */
int acse_last_error(const acse_ctx* ctx);

/* Version string of the library build. */
const char* acse_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ACSE_H */
