// Fit of the asymptotic regime of an ACSE energy trajectory (Results: with lambda = eps n the energy
// runs through an exponentially damped region into an asymptotic regime where it changes about
// linearly in lambda; Conclusions: extrapolation and fitting to estimate the solution once a
// trajectory stably enters that regime).  The paper gives no fit; the library's reading:
//     E(lambda) ~ a + b lambda + c exp(-k lambda),  k > 0,
// least squares over the points n >= n_skip, in the scaled coordinate t = (lambda - lambda_first) / span
// (span = lambda_last - lambda_first, kappa = k span).  For a fixed kappa the best (a, b, c) is a linear
// least-squares problem; its residual sum of squares F(kappa) is scanned on FIT_NGRID points evenly
// spaced in log kappa over [FIT_KAPPA_MIN, FIT_KAPPA_STEPS (m - 1)], the best grid point j (the first
// on ties) is taken, and for 0 < j < FIT_NGRID - 1 the stationarity condition
//     dF/dkappa = 2 c_t sum_n r_n t_n exp(-kappa t_n) = 0
// (variable projection: at the optimal linear coefficients only the exponential column depends on
// kappa; r the residual vector, c_t the exponential coefficient) is solved by bisection in
// [kappa_{j-1}, kappa_{j+1}].  Out: a, b, c, k, rss, flag (0 refined; 1 minimum on the grid's edge
// or no sign change of dF/dkappa in the bracket; 2 fewer than four points; 3 lambda not increasing).
//
// Numerics: the columns 1 and t are orthonormalised once (q1 = 1/sqrt(m), q2 = (t - mean t) / s), E
// and every exponential column are projected off them (the exponential twice, classical Gram-Schmidt
// with one re-orthogonalisation), and F and dF/dkappa are formed from the explicit residual vector,
// never as a difference of sums of squares.  Every sum runs in a fixed order (one thread per grid
// point over n in order; fixed-shape block reductions), so a fit is reproducible bit for bit.
#include <math.h>

#include "acse_internal.h"

#define FIT_THREADS 256
#define FIT_NGRID 256              // one grid point per thread of the scan
#define FIT_MAX_POINTS 4096        // points held in shared memory (4 arrays of doubles: 128 KiB)
#define FIT_KAPPA_MIN 0.25
#define FIT_KAPPA_STEPS 4.0
static_assert(FIT_NGRID == FIT_THREADS, "the scan gives each thread one grid point");

struct FitArgs {
    const double* lam;     // trajectory i: lam + i * stride, E + i * stride
    const double* E;
    const int* count;      // points of trajectory i (device), or null: every trajectory has n_fixed
    int n_fixed;
    size_t stride;
    int n_skip;
    double* out;           // 6 doubles per trajectory
};

// Fixed-order block sum (FIT_THREADS threads): each thread's value, then a tree in shared memory.
__device__ double fit_block_sum(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = FIT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// F(kappa), the exponential coefficient and dF/dkappa, by one thread over all m points in order.
struct FitEval {
    double F, c, g;
};

__device__ FitEval fit_eval_serial(double kappa, int m, const double* t, const double* q2, const double* ep) {
    const double im = 1.0 / m;
    double s1 = 0.0, s2 = 0.0;
    for (int n = 0; n < m; ++n) {
        const double u = exp(-kappa * t[n]);
        s1 += u;
        s2 += u * q2[n];
    }
    double s1b = 0.0, s2b = 0.0;
    for (int n = 0; n < m; ++n) {
        const double u1 = exp(-kappa * t[n]) - s1 * im - s2 * q2[n];
        s1b += u1;
        s2b += u1 * q2[n];
    }
    double nu = 0.0, pe = 0.0;
    for (int n = 0; n < m; ++n) {
        const double up = exp(-kappa * t[n]) - (s1 + s1b) * im - (s2 + s2b) * q2[n];
        nu += up * up;
        pe += ep[n] * up;
    }
    FitEval r;
    r.c = pe / nu;
    double F = 0.0, G = 0.0;
    for (int n = 0; n < m; ++n) {
        const double u = exp(-kappa * t[n]);
        const double up = u - (s1 + s1b) * im - (s2 + s2b) * q2[n];
        const double res = ep[n] - r.c * up;
        F += res * res;
        G += res * t[n] * u;
    }
    r.F = F;
    r.g = 2.0 * r.c * G;
    return r;
}

// The same quantities computed by the whole block (strided partial sums, fixed-order reductions).
__device__ FitEval fit_eval_block(double kappa, int m, const double* t, const double* q2, const double* ep,
                                  double* red) {
    const double im = 1.0 / m;
    double a = 0.0, b = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double u = exp(-kappa * t[n]);
        a += u;
        b += u * q2[n];
    }
    const double s1 = fit_block_sum(a, red), s2 = fit_block_sum(b, red);
    a = b = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double u1 = exp(-kappa * t[n]) - s1 * im - s2 * q2[n];
        a += u1;
        b += u1 * q2[n];
    }
    const double s1b = fit_block_sum(a, red), s2b = fit_block_sum(b, red);
    a = b = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double up = exp(-kappa * t[n]) - (s1 + s1b) * im - (s2 + s2b) * q2[n];
        a += up * up;
        b += ep[n] * up;
    }
    const double nu = fit_block_sum(a, red), pe = fit_block_sum(b, red);
    FitEval r;
    r.c = pe / nu;
    a = b = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double u = exp(-kappa * t[n]);
        const double up = u - (s1 + s1b) * im - (s2 + s2b) * q2[n];
        const double res = ep[n] - r.c * up;
        a += res * res;
        b += res * t[n] * u;
    }
    r.F = fit_block_sum(a, red);
    r.g = 2.0 * r.c * fit_block_sum(b, red);
    return r;
}

__device__ double fit_kappa_grid(int j, int m) {
    const double l0 = log(FIT_KAPPA_MIN), l1 = log(FIT_KAPPA_STEPS * (m - 1));
    const double step = (l1 - l0) / (FIT_NGRID - 1);
    return exp(j == FIT_NGRID - 1 ? l1 : l0 + j * step);
}

__global__ void __launch_bounds__(FIT_THREADS) k_fit_trajectory(FitArgs a) {
    extern __shared__ double sm[];
    __shared__ double red[FIT_THREADS];
    __shared__ double gridF[FIT_NGRID];
    const int tr = blockIdx.x;
    const double* lam = a.lam + tr * a.stride;
    const double* Eg = a.E + tr * a.stride;
    const int cnt = a.count ? a.count[tr] : a.n_fixed;
    double* out = a.out + 6 * (size_t)tr;
    const int m = min(cnt, FIT_MAX_POINTS + a.n_skip) - a.n_skip;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (m < 4) {
        if (threadIdx.x < 5) out[threadIdx.x] = nan;
        if (threadIdx.x == 5) out[5] = 2.0;
        return;
    }
    double* t = sm;
    double* q2 = sm + m;
    double* ep = sm + 2 * m;
    double* Es = sm + 3 * m;
    const double l0 = lam[a.n_skip], span = lam[a.n_skip + m - 1] - l0;
    if (!(span > 0.0)) {
        if (threadIdx.x < 5) out[threadIdx.x] = nan;
        if (threadIdx.x == 5) out[5] = 3.0;
        return;
    }
    const double im = 1.0 / m;
    double p = 0.0, q = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        t[n] = (lam[a.n_skip + n] - l0) / span;
        Es[n] = Eg[a.n_skip + n];
        p += t[n];
        q += Es[n];
    }
    const double tbar = fit_block_sum(p, red) * im, Ebar = fit_block_sum(q, red) * im;
    p = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) p += (t[n] - tbar) * (t[n] - tbar);
    const double s = sqrt(fit_block_sum(p, red));
    p = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        q2[n] = (t[n] - tbar) / s;
        p += (Es[n] - Ebar) * q2[n];
    }
    const double beta = fit_block_sum(p, red);
    p = q = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        ep[n] = (Es[n] - Ebar) - beta * q2[n];
        p += ep[n];
        q += ep[n] * q2[n];
    }
    const double e1 = fit_block_sum(p, red), e2 = fit_block_sum(q, red);
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) ep[n] -= e1 * im + e2 * q2[n];
    __syncthreads();

    // scan: one grid point per thread
    {
        const FitEval r = fit_eval_serial(fit_kappa_grid(threadIdx.x, m), m, t, q2, ep);
        gridF[threadIdx.x] = (r.F == r.F) ? r.F : INFINITY;
    }
    __syncthreads();
    __shared__ int jbest;
    if (threadIdx.x == 0) {
        int j = 0;
        for (int i = 1; i < FIT_NGRID; ++i)
            if (gridF[i] < gridF[j]) j = i;
        jbest = j;
    }
    __syncthreads();
    const int j = jbest;
    double kappa = fit_kappa_grid(j, m);
    int flag = 1;
    if (j > 0 && j < FIT_NGRID - 1) {
        double lo = fit_kappa_grid(j - 1, m), hi = fit_kappa_grid(j + 1, m);
        const FitEval rl = fit_eval_block(lo, m, t, q2, ep, red);
        const FitEval rh = fit_eval_block(hi, m, t, q2, ep, red);
        if (rl.g < 0.0 && rh.g > 0.0) {
            flag = 0;
            for (int it = 0; it < 200 && hi - lo > 4.0 * 2.220446049250313e-16 * hi; ++it) {
                const double mid = 0.5 * (lo + hi);
                const FitEval rm = fit_eval_block(mid, m, t, q2, ep, red);
                if (rm.g == 0.0) {
                    lo = hi = mid;
                    break;
                }
                if (rm.g < 0.0) lo = mid;
                else hi = mid;
            }
            kappa = 0.5 * (lo + hi);
        }
    }
    // coefficients at kappa: c_t from the projected problem, then a_t, b_t from E - c_t exp(-kappa t)
    const FitEval rf = fit_eval_block(kappa, m, t, q2, ep, red);
    const double ct = rf.c;
    p = q = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double y = Es[n] - ct * exp(-kappa * t[n]);
        p += y;
        q += y * q2[n];
    }
    const double al1 = fit_block_sum(p, red) * im, al2 = fit_block_sum(q, red);
    const double bt = al2 / s, at = al1 - al2 * tbar / s;
    p = 0.0;
    for (int n = threadIdx.x; n < m; n += FIT_THREADS) {
        const double res = Es[n] - at - bt * t[n] - ct * exp(-kappa * t[n]);
        p += res * res;
    }
    const double rss = fit_block_sum(p, red);
    if (threadIdx.x == 0) {
        out[0] = at - bt * l0 / span;
        out[1] = bt / span;
        out[2] = ct * exp(kappa * l0 / span);
        out[3] = kappa / span;
        out[4] = rss;
        out[5] = (double)flag;
    }
}

static int fit_set_attrs() {
    static int done = 0;
    if (done) return ACSE_OK;
    ACSE_CUDA_TRY(cudaFuncSetAttribute(k_fit_trajectory, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       4 * FIT_MAX_POINTS * (int)sizeof(double)));
    done = 1;
    return ACSE_OK;
}

// Fits `ntraj` trajectories stored `stride` doubles apart (counts per trajectory on the device, or
// n_fixed points each) in one launch, one block per trajectory.
int fit_launch(const double* lam, const double* E, const int* count, int n_fixed, size_t stride, int ntraj,
               int n_skip, double* out, cudaStream_t st) {
    ACSE_TRY(fit_set_attrs());
    FitArgs a{lam, E, count, n_fixed, stride, n_skip, out};
    const size_t smem = 4 * (size_t)FIT_MAX_POINTS * sizeof(double);
    k_fit_trajectory<<<ntraj, FIT_THREADS, smem, st>>>(a);
    ACSE_CUDA_TRY(cudaGetLastError());
    return ACSE_OK;
}

static int fit_device_ptr(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeManaged) return 1;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

extern "C" int acse_extrapolate(int n, const double* lam, const double* E, int n_skip, double* out,
                                void* cuda_stream) {
    if (!lam || !E || !out || n_skip < 0) return ACSE_ERR_ARG;
    if (n - n_skip < 4 || n - n_skip > FIT_MAX_POINTS) return ACSE_ERR_SHAPE;
    int dev = 0;
    ACSE_CUDA_TRY(cudaGetDevice(&dev));
    if (!fit_device_ptr(lam, dev) || !fit_device_ptr(E, dev) || !fit_device_ptr(out, dev)) return ACSE_ERR_ARG;
    return fit_launch(lam, E, nullptr, n, 0, 1, n_skip, out, (cudaStream_t)cuda_stream);
}
