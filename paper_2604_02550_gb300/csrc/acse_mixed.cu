// Operand packing and FP32 intermediates of the split-precision (BF16x3 / TF32) path.
//
// Every O(r^6) GEMM operand is written once per contraction pass, directly in the K-major
// layout the tensor-core GEMM reads (one row per output row / column, K segments zero padded to
// a multiple of the 128-byte K block):
//   BF16x3  x = hi + lo, hi = bf16(x), lo = bf16(x - hi);  A rows [hi|hi|lo], B rows [hi|lo|hi]
//   TF32    x -> tf32 (round to nearest, ties away)        A rows, B rows [x]
//   TF32x3  x = hi + lo, hi = tf32(x), lo = tf32(x - hi);  A rows [hi|hi|lo], B rows [hi|lo|hi]
// The logical operands are those of the FP64 path (acse_elem.cu): the pair-pair [M; D] and W
// blocks, and the particle-hole layouts of M and Z.  The 1-RDM is accumulated in FP64 (exactly
// as in the FP64 path) and rounded to FP32 here; M, Z and w are formed in FP32.
#include <cuda_bf16.h>
#include <string.h>

#include "acse_internal.h"
#include "acse_split.cuh"

struct MxPtrs {
    void* pairA[3];
    void* pairB[3];
    void* Md;
    void* Zd;
    void* Mf[2];
    void* Zf[2];
    float* M32[3];
    float* gam32;
    int Kp1, Kp2, ns, KpP;
};

static MxPtrs mx_ptrs(acse_ctx* c) {
    MxPtrs p;
    Work& w = c->w;
    for (int s = 0; s < 3; ++s) {
        p.pairA[s] = w.tc_pairA[s];
        p.pairB[s] = w.tc_pairB[s];
        p.M32[s] = w.M32[s];
    }
    p.Md = w.tc_Md;
    p.Zd = w.tc_Zd;
    for (int f = 0; f < 2; ++f) {
        p.Mf[f] = w.tc_Mf[f];
        p.Zf[f] = w.tc_Zf[f];
    }
    p.gam32 = w.gam32;
    p.Kp1 = w.Kp1;
    p.Kp2 = w.Kp2;
    p.KpP = w.KpP;
    p.ns = c->nsplit;
    return p;
}

// --------------------------------------------------------------------------- per D
// M = 3 2D - 2 (1D^1D) in FP32 (App. C), stored plain (M32) and as rows 0..r^2-1 of the pair
// operand [M; D]; rows r^2..2r^2-1 hold D.  Also rounds the FP64 1-RDM to FP32.  One block per
// (sector, pair ij): the D row ij is read and rounded to FP32 once and gives both the M row ij and the
// D row r^2 + ij (the FP64 -> FP32 conversions run on the slow FP64 pipe); each thread handles groups
// of four consecutive columns (16-byte loads and vector stores when r is even); the two 1-RDM rows the
// M row needs are staged in shared memory.  RC: r as a compile-time constant (0: runtime r).
template <int PREC, int RC>
__global__ void __launch_bounds__(192) k_mx_prepD(int r_, const double* __restrict__ gam, const double* __restrict__ Daa,
                                                  const double* __restrict__ Dab, const double* __restrict__ Dbb,
                                                  const __grid_constant__ MxPtrs p) {
    __shared__ float g1[ACSE_MAX_R], g2[ACSE_MAX_R];
    const int r = RC ? RC : r_;
    const int R2 = r * r;
    const int c4 = (R2 + 3) >> 2;
    const int s = blockIdx.x / R2;
    const int row = blockIdx.x - s * R2;   // pair ij: M row ij and D row r^2 + ij
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < 2 * R2; e += blockDim.x) p.gam32[e] = (float)gam[e];
    const int i = row / r, j = row - (row / r) * r;
    {
        // s = 0: rows i, j of 1D_a; s = 2: of 1D_b; s = 1: row i of 1D_a and row j of 1D_b
        const double* G1 = gam + (s == 2 ? R2 : 0) + (size_t)i * r;
        const double* G2 = gam + (s == 0 ? 0 : R2) + (size_t)j * r;
        for (int e = threadIdx.x; e < r; e += blockDim.x) {
            g1[e] = (float)G1[e];
            g2[e] = (float)G2[e];
        }
    }
    __syncthreads();
    const size_t ld = (size_t)p.ns * p.Kp1;
    const size_t ldP = (size_t)p.ns * p.KpP;
    // packed rows of a same-spin sector (pairs i < j only): M at pk(i, j), D at P + pk(i, j)
    const int P = r * (r - 1) / 2;
    const int prow = i < j ? pk_pair(r, i, j) : -1;
    const double* D = (s == 0 ? Daa : (s == 1 ? Dab : Dbb)) + (size_t)row * R2;
    float* Mrow = p.M32[s] + (size_t)row * R2;
    const bool vec = (r & 1) == 0 && ((reinterpret_cast<uintptr_t>(s == 0 ? Daa : (s == 1 ? Dab : Dbb)) & 15) == 0);
    for (int q4 = threadIdx.x; q4 < c4; q4 += blockDim.x) {
        const int k0 = q4 * 4;
        const int nk = R2 - k0 < 4 ? R2 - k0 : 4;
        float x[4] = {0.f, 0.f, 0.f, 0.f}, m[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec && nk == 4) {
            const double2 d01 = *reinterpret_cast<const double2*>(D + k0);
            const double2 d23 = *reinterpret_cast<const double2*>(D + k0 + 2);
            x[0] = (float)d01.x; x[1] = (float)d01.y; x[2] = (float)d23.x; x[3] = (float)d23.y;
        } else {
            for (int u = 0; u < nk; ++u) x[u] = (float)D[k0 + u];
        }
        {
            int kk = k0 / r, l = k0 - kk * r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u < nk) m[u] = s == 1 ? 3.0f * x[u] - g1[kk] * g2[l] : 3.0f * x[u] - (g1[kk] * g2[l] - g2[kk] * g1[l]);
                if (++l == r) { l = 0; ++kk; }
            }
        }
        if (vec && nk == 4) *reinterpret_cast<float4*>(Mrow + k0) = make_float4(m[0], m[1], m[2], m[3]);
        else
            for (int u = 0; u < nk; ++u) Mrow[k0 + u] = m[u];
        if (s == 1) {
            if (vec && nk == 4) {
                put4<PREC, 0>(p.pairA[s], row, ld, p.Kp1, k0, m);
                put4<PREC, 0>(p.pairA[s], (size_t)R2 + row, ld, p.Kp1, k0, x);
            } else {
                for (int u = 0; u < nk; ++u) {
                    put<PREC, 0>(p.pairA[s], row, ld, p.Kp1, k0 + u, m[u]);
                    put<PREC, 0>(p.pairA[s], (size_t)R2 + row, ld, p.Kp1, k0 + u, x[u]);
                }
            }
        } else if (prow >= 0) {
            // same-spin sector: rows and K restricted to pairs a < b (antisymmetry; the GEMM's alpha
            // carries the factor 2 of the (r, s) sum)
            int kk = k0 / r, l = k0 - kk * r;
            for (int u = 0; u < nk; ++u) {
                if (kk < l) {
                    const int kq = pk_pair(r, kk, l);
                    put<PREC, 0>(p.pairA[s], (size_t)prow, ldP, p.KpP, kq, m[u]);
                    put<PREC, 0>(p.pairA[s], (size_t)(P + prow), ldP, p.KpP, kq, x[u]);
                }
                if (++l == r) { l = 0; ++kk; }
            }
        }
    }
}

template <int PREC>
static void launch_prepD(acse_ctx* c, int nsec, const double* const D[3], const MxPtrs& p) {
    const int r = c->r, g = nsec * r * r;
    switch (r) {
        case 16: k_mx_prepD<PREC, 16><<<g, 192, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], p); break;
        case 32: k_mx_prepD<PREC, 32><<<g, 192, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], p); break;
        case 48: k_mx_prepD<PREC, 48><<<g, 192, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], p); break;
        case 64: k_mx_prepD<PREC, 64><<<g, 192, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], p); break;
        default: k_mx_prepD<PREC, 0><<<g, 192, 0, c->stream>>>(r, c->w.gam, D[0], D[1], D[2], p); break;
    }
}

// Particle-hole layouts of M (the B operands of the ph GEMMs), copied as r x r blocks per (t, i, p):
//   t=0 Md(a,a) rows (a,i,l) cols (a,p,s) <- Maa[i][p][l][s]      t=1 Md(a,b) <- Mab[i][p][l][s]
//   t=2 Md(b,a) rows (b,i,l) cols (a,p,s) <- Mab[p][i][s][l]      t=3 Md(b,b) <- Mbb[i][p][l][s]
//   t=4 Mf1[(i,l)][(p,s)] <- Mab[i][p][s][l]                        t=5 Mf2[(i,l)][(p,s)] <- Mab[p][i][l][s]
// (transposed source blocks go through shared memory so that reads and writes stay coalesced).
template <int PREC, int RC>
__global__ void __launch_bounds__(256) k_mx_pack_Mph(int r_, const __grid_constant__ MxPtrs p) {
    __shared__ float tile[ACSE_MAX_R][ACSE_MAX_R + 1];
    const int r = RC ? RC : r_;   // compile-time r where it is one of the tensor-core sizes
    const int R2 = r * r;
    const int t = blockIdx.x / R2, ip = blockIdx.x % R2;
    const int i = ip / r, pp = ip % r;
    const size_t r3 = (size_t)R2 * r;
    const float* src;
    bool tr;
    switch (t) {
        case 0: src = p.M32[0] + i * r3 + (size_t)pp * R2; tr = false; break;
        case 1: src = p.M32[1] + i * r3 + (size_t)pp * R2; tr = false; break;
        case 2: src = p.M32[1] + pp * r3 + (size_t)i * R2; tr = true; break;
        case 3: src = p.M32[2] + i * r3 + (size_t)pp * R2; tr = false; break;
        case 4: src = p.M32[1] + i * r3 + (size_t)pp * R2; tr = true; break;
        default: src = p.M32[1] + pp * r3 + (size_t)i * R2; tr = false; break;
    }
    if ((r & 1) == 0) {   // r^2 % 4 == 0 and every source block starts on a 16-byte boundary
        for (int e4 = threadIdx.x; e4 < R2 / 4; e4 += blockDim.x) {
            const float4 q = reinterpret_cast<const float4*>(src)[e4];
            const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = 4 * e4 + c, u = e / r, v = e - u * r;
                if (tr) tile[v][u] = qv[c];
                else tile[u][v] = qv[c];
            }
        }
    } else {
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int u = e / r, v = e % r;
            if (tr) tile[v][u] = src[e];
            else tile[u][v] = src[e];
        }
    }
    __syncthreads();
    void* dst;
    size_t ld;
    int Kp, rowbase, colbase;
    if (t < 4) {
        dst = p.Md; ld = (size_t)p.ns * p.Kp2; Kp = p.Kp2;
        rowbase = (t >> 1) * R2 + i * r; colbase = (t & 1) * R2 + pp * r;
    } else {
        dst = p.Mf[t - 4]; ld = (size_t)p.ns * p.Kp1; Kp = p.Kp1;
        rowbase = i * r; colbase = pp * r;
    }
    if ((r & 3) == 0) {   // four consecutive columns of one row per thread, vector stores
        for (int g = threadIdx.x; g < R2 / 4; g += blockDim.x) {
            const int l = (4 * g) / r, s0 = 4 * g - l * r;
            const float x[4] = {tile[l][s0], tile[l][s0 + 1], tile[l][s0 + 2], tile[l][s0 + 3]};
            put4<PREC, 1>(dst, (size_t)rowbase + l, ld, Kp, colbase + s0, x);
        }
    } else {
        for (int e = threadIdx.x; e < R2; e += blockDim.x) {
            const int l = e / r, s2 = e % r;
            put<PREC, 1>(dst, (size_t)rowbase + l, ld, Kp, colbase + s2, tile[l][s2]);
        }
    }
}

template <int PREC>
static void launch_pack_Mph(acse_ctx* c, int nph, const MxPtrs& q) {
    const int r = c->r, g = nph * r * r;
    switch (r) {
        case 16: k_mx_pack_Mph<PREC, 16><<<g, 256, 0, c->stream>>>(r, q); break;
        case 32: k_mx_pack_Mph<PREC, 32><<<g, 256, 0, c->stream>>>(r, q); break;
        case 48: k_mx_pack_Mph<PREC, 48><<<g, 256, 0, c->stream>>>(r, q); break;
        case 64: k_mx_pack_Mph<PREC, 64><<<g, 256, 0, c->stream>>>(r, q); break;
        default: k_mx_pack_Mph<PREC, 0><<<g, 256, 0, c->stream>>>(r, q); break;
    }
}

int tc_mixed_prep_D(acse_ctx* c, const double* const D[3]) {
    MxPtrs p = mx_ptrs(c);
    // spin-flip specialisation: M_bb = M_aa (the bb sector of [M; D] is not formed) and Mf2 feeds only
    // the second spin-flip GEMM, which is not run
    const bool sf = acse_singlet(c);
    const int nph = sf ? 5 : 6, nsec = sf ? 2 : 3;
    MxPtrs q = p;
    if (sf) q.M32[2] = q.M32[0];
    if (c->opt.prec == ACSE_BF16X3) {
        launch_prepD<ACSE_BF16X3>(c, nsec, D, p);
        ACSE_LAUNCHED(c);
        launch_pack_Mph<ACSE_BF16X3>(c, nph, q);
    } else if (c->opt.prec == ACSE_TF32X3) {
        launch_prepD<ACSE_TF32X3>(c, nsec, D, p);
        ACSE_LAUNCHED(c);
        launch_pack_Mph<ACSE_TF32X3>(c, nph, q);
    } else {
        launch_prepD<ACSE_TF32>(c, nsec, D, p);
        ACSE_LAUNCHED(c);
        launch_pack_Mph<ACSE_TF32>(c, nph, q);
    }
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// --------------------------------------------------------------------------- per W
// Pair operand B: W blocks as (kp) x (rs) rows.
template <int PREC, int RC>
__global__ void k_mx_pack_W(int r_, const float* __restrict__ Waa, const float* __restrict__ Wab,
                            const float* __restrict__ Wbb, const __grid_constant__ MxPtrs p) {
    // grid: x over groups of four columns, y over (sector, row); RC: compile-time r (0: runtime)
    const int r = RC ? RC : r_;
    const int R2 = r * r;
    const int c4 = (R2 + 3) >> 2;
    const int q4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (q4 >= c4) return;
    const int s = blockIdx.y / R2;
    const int row = blockIdx.y - s * R2;
    const size_t ld = (size_t)p.ns * p.Kp1;
    const float* W = (s == 0 ? Waa : (s == 1 ? Wab : Wbb)) + (size_t)row * R2;   // FP32 copy of W
    const int k0 = q4 * 4;
    const int nk = R2 - k0 < 4 ? R2 - k0 : 4;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if ((r & 1) == 0 && nk == 4) {   // r^2 % 4 == 0: every row starts on a 16-byte boundary
        const float4 v = *reinterpret_cast<const float4*>(W + k0);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
        for (int u = 0; u < nk; ++u) x[u] = W[k0 + u];
    }
    if (s == 1) {
        if ((r & 1) == 0 && nk == 4) put4<PREC, 1>(p.pairB[s], row, ld, p.Kp1, k0, x);
        else
            for (int u = 0; u < nk; ++u) put<PREC, 1>(p.pairB[s], row, ld, p.Kp1, k0 + u, x[u]);
        return;
    }
    // same-spin sector: rows (k, p) and K (r, s) restricted to pairs a < b
    const int kr = row / r, pr = row - (row / r) * r;
    if (kr >= pr) return;
    const size_t ldP = (size_t)p.ns * p.KpP;
    const int prow = pk_pair(r, kr, pr);
    int a = k0 / r, b = k0 - a * r;
    for (int u = 0; u < nk; ++u) {
        if (a < b) put<PREC, 1>(p.pairB[s], (size_t)prow, ldP, p.KpP, pk_pair(r, a, b), x[u]);
        if (++b == r) { b = 0; ++a; }
    }
}

// Rows (i, j), i < j, of [X; Y] of a same-spin sector from the packed GEMM output:
// X^{ij}_{kp} = s_kp Xp[pk(ij)][pk(kp)] (s_kp = -1 for k > p, 0 for k = p), rows r^2 + (i, j) for Y
// likewise.  These are the only rows read: the B kernel's same-spin items are the pairs i < j, and Q
// reads the packed output itself; rows i >= j are not formed.  Each block writes nrow consecutive
// packed rows (a contiguous range of the packed output): the range is copied into shared memory
// (cp.async, every copy in flight at once) while a column map (packed index and sign of every column)
// is built there, then the full rows are written four columns at a time.
#define UP_ROWS 8
__device__ __forceinline__ void up_cp_async16(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void up_cp_async4(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}

// rows per block of k_mx_unpack_pairs: its staged rows and column map within 48 KB of shared memory
static int up_rows(int r) {
    const int R2 = r * r, P = r * (r - 1) / 2;
    int n = (48 * 1024 - 4 * R2) / (4 * P);
    return n > UP_ROWS ? UP_ROWS : (n < 1 ? 1 : n);
}

__global__ void __launch_bounds__(256) k_mx_unpack_pairs(int r, int nrow, const float* __restrict__ Cp0,
                                                         const float* __restrict__ Cp2, float* C0, float* C2) {
    extern __shared__ __align__(16) int up_smem[];
    const int R2 = r * r, P = r * (r - 1) / 2;
    int* cmap = up_smem;                                    // [R2]: -1 diagonal; bit 30: negated
    float* srow = reinterpret_cast<float*>(up_smem + R2);   // [nrow][P]: the packed rows of the block
    const int nblk_sec = (2 * P + nrow - 1) / nrow;
    const int sec = blockIdx.x / nblk_sec;
    const int q0 = (blockIdx.x - sec * nblk_sec) * nrow;   // packed row: part * P + pk(i, j)
    const int nr = min(nrow, 2 * P - q0);
    const float* src = (sec == 0 ? Cp0 : Cp2) + (size_t)q0 * P;
    float* Cs = sec == 0 ? C0 : C2;
    // 16-byte copies when the range and every staged row start on a 16-byte boundary
    if ((P & 3) == 0 && (R2 & 3) == 0)
        for (int e = threadIdx.x; e < nr * P / 4; e += blockDim.x) up_cp_async16(srow + 4 * e, src + 4 * e);
    else
        for (int e = threadIdx.x; e < nr * P; e += blockDim.x) up_cp_async4(srow + e, src + e);
    for (int c = threadIdx.x; c < R2; c += blockDim.x) {
        const int k = c / r, q = c - (c / r) * r;
        cmap[c] = k == q ? -1 : (k < q ? pk_pair(r, k, q) : (pk_pair(r, q, k) | 0x40000000));
    }
    // (part, i, j) of the first packed row; the following rows advance over the pairs i < j
    int part = q0 / P, i = 0, j;
    {
        int base = 0;
        const int pr = q0 - part * P;
        while (pr >= base + (r - 1 - i)) {
            base += r - 1 - i;
            ++i;
        }
        j = i + 1 + (pr - base);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    const bool vec = (R2 & 3) == 0 && (reinterpret_cast<uintptr_t>(Cs) & 15) == 0;
    for (int u = 0; u < nr; ++u) {
        float* C = Cs + ((size_t)part * R2 + (size_t)i * r + j) * R2;
        const float* sr = srow + (size_t)u * P;
        auto val = [&](int m) { return m < 0 ? 0.f : ((m & 0x40000000) ? -sr[m & 0x3FFFFFFF] : sr[m]); };
        if (vec) {
            for (int g = threadIdx.x; g < R2 / 4; g += blockDim.x) {
                const int4 m = reinterpret_cast<const int4*>(cmap)[g];
                reinterpret_cast<float4*>(C)[g] = make_float4(val(m.x), val(m.y), val(m.z), val(m.w));
            }
        } else {
            for (int c = threadIdx.x; c < R2; c += blockDim.x) C[c] = val(cmap[c]);
        }
        if (++j == r) {   // next pair; after (r-2, r-1) the first pair of the next part
            ++i;
            j = i + 1;
            if (i == r - 1) {
                ++part;
                i = 0;
                j = 1;
            }
        }
    }
}

int tc_unpack_pairs(acse_ctx* c) {
    const int r = c->r, R2 = r * r, P = r * (r - 1) / 2;
    const int nsec = acse_singlet(c) ? 1 : 2;   // the bb sector is not formed under the spin flip
    const int nrow = up_rows(r);
    const int nblk_sec = (2 * P + nrow - 1) / nrow;
    const size_t smem = (size_t)4 * R2 + (size_t)4 * nrow * P;
    k_mx_unpack_pairs<<<nsec * nblk_sec, 256, smem, c->stream>>>(r, nrow, c->w.tc_pairCp[0], c->w.tc_pairCp[2],
                                                                 c->w.tc_pairC[0], c->w.tc_pairC[2]);
    ACSE_LAUNCHED(c);
    return ACSE_OK;
}

// FP32 copy of n doubles (the W operands: their FP32 values are all the split path reads).
__global__ void __launch_bounds__(256) k_mx_to_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        for (size_t i = t0; i < n / 2; i += stride) {
            const double2 v = reinterpret_cast<const double2*>(src)[i];
            reinterpret_cast<float2*>(dst)[i] = make_float2((float)v.x, (float)v.y);
        }
        if ((n & 1) && t0 == 0) dst[n - 1] = (float)src[n - 1];
    } else {
        for (size_t i = t0; i < n; i += stride) dst[i] = (float)src[i];
    }
}

static int to_f32(acse_ctx* c, const double* const W[3], float* const out[3]) {
    const size_t r = c->r, n4 = r * r * r * r;
    for (int s = 0; s < 3; ++s) {
        k_mx_to_f32<<<152 * 8, 256, 0, c->stream>>>(W[s], out[s], n4);
        ACSE_LAUNCHED(c);
    }
    return ACSE_OK;
}

int tc_make_Kh32(acse_ctx* c) {
    const double* W[3] = {c->w.Kh[0], c->w.Kh[1], c->w.Kh[2]};
    return to_f32(c, W, c->w.Kh32);
}

template <int PREC>
static void launch_pack_W(acse_ctx* c, dim3 grid, const float* const W32[3], const MxPtrs& p) {
    const int r = c->r;
    switch (r) {
        case 16: k_mx_pack_W<PREC, 16><<<grid, 128, 0, c->stream>>>(r, W32[0], W32[1], W32[2], p); break;
        case 32: k_mx_pack_W<PREC, 32><<<grid, 128, 0, c->stream>>>(r, W32[0], W32[1], W32[2], p); break;
        case 48: k_mx_pack_W<PREC, 48><<<grid, 128, 0, c->stream>>>(r, W32[0], W32[1], W32[2], p); break;
        case 64: k_mx_pack_W<PREC, 64><<<grid, 128, 0, c->stream>>>(r, W32[0], W32[1], W32[2], p); break;
        default: k_mx_pack_W<PREC, 0><<<grid, 128, 0, c->stream>>>(r, W32[0], W32[1], W32[2], p); break;
    }
}

int tc_mixed_prep_W(acse_ctx* c, const double* const W[3]) {
    const int r = c->r;
    Work& w = c->w;
    MxPtrs p = mx_ptrs(c);
    // the FP32 copy of W: K/2 (made at creation), the residual just assembled into w.A (its FP32 values
    // written beside it), else converted here
    const float* W32[3];
    if (W[0] == w.Kh[0] && W[1] == w.Kh[1] && W[2] == w.Kh[2]) {
        for (int s = 0; s < 3; ++s) W32[s] = w.Kh32[s];
    } else if (c->a32_valid && W[0] == w.A[0] && W[1] == w.A[1] && W[2] == w.A[2]) {
        for (int s = 0; s < 3; ++s) W32[s] = w.A32[s];
    } else {
        ACSE_TRY(to_f32(c, W, w.W32s));
        for (int s = 0; s < 3; ++s) W32[s] = w.W32s[s];
    }
    const dim3 grid((r * r / 4 + 128) / 128, (acse_singlet(c) ? 2 : 3) * r * r);   // no bb pair GEMM under the spin flip
    if (c->opt.prec == ACSE_BF16X3)
        launch_pack_W<ACSE_BF16X3>(c, grid, W32, p);
    else if (c->opt.prec == ACSE_TF32X3)
        launch_pack_W<ACSE_TF32X3>(c, grid, W32, p);
    else
        launch_pack_W<ACSE_TF32>(c, grid, W32, p);
    ACSE_LAUNCHED(c);
    return launch_Z_tiled(c, W, W32);   // Z packs and w (the diagonal of Z)
}

// ------------------------------------------------------------------------ workspace
static int mx_alloc(void** p, size_t bytes, bool zero) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ACSE_ERR_NOMEM;
    }
    if (zero && cudaMemset(*p, 0, bytes) != cudaSuccess) return ACSE_ERR_CUDA;
    return ACSE_OK;
}

int tc_mixed_alloc(acse_ctx* c) {
    Work& w = c->w;
    const size_t r = c->r, R2 = r * r, n4 = R2 * R2;
    const int es = c->opt.prec == ACSE_BF16X3 ? 2 : 4;
    const int kb = 128 / es;
    w.Kp1 = (int)((R2 + kb - 1) / kb * kb);
    w.Kp2 = (int)((2 * R2 + kb - 1) / kb * kb);
    const size_t ns = c->nsplit;
    const size_t L1 = ns * w.Kp1 * es, L2 = ns * w.Kp2 * es;   // row bytes
    // operand buffers are zeroed once: the K padding is never written afterwards
    const size_t P = r * (r - 1) / 2;
    w.KpP = (int)((P + kb - 1) / kb * kb);
    const size_t LP = ns * w.KpP * es;                            // packed same-spin row bytes
    for (int s = 0; s < 3; ++s) {
        if (s == 1) {
            ACSE_TRY(mx_alloc(&w.tc_pairA[s], 2 * R2 * L1, true));
            ACSE_TRY(mx_alloc(&w.tc_pairB[s], R2 * L1, true));
        } else {
            ACSE_TRY(mx_alloc(&w.tc_pairA[s], 2 * P * LP, true));
            ACSE_TRY(mx_alloc(&w.tc_pairB[s], P * LP, true));
            ACSE_TRY(mx_alloc((void**)&w.tc_pairCp[s], 2 * P * P * sizeof(float), false));
        }
        ACSE_TRY(mx_alloc((void**)&w.tc_pairC[s], 2 * R2 * R2 * sizeof(float), false));
        ACSE_TRY(mx_alloc((void**)&w.M32[s], n4 * sizeof(float), false));
        ACSE_TRY(mx_alloc((void**)&w.Kh32[s], n4 * sizeof(float), false));
        ACSE_TRY(mx_alloc((void**)&w.A32[s], n4 * sizeof(float), false));
        ACSE_TRY(mx_alloc((void**)&w.W32s[s], n4 * sizeof(float), false));
    }
    ACSE_TRY(mx_alloc(&w.tc_Md, 2 * R2 * L2, true));
    ACSE_TRY(mx_alloc(&w.tc_Zd, 2 * R2 * L2, true));
    for (int f = 0; f < 2; ++f) {
        ACSE_TRY(mx_alloc(&w.tc_Mf[f], R2 * L1, true));
        ACSE_TRY(mx_alloc(&w.tc_Zf[f], R2 * L1, true));
        ACSE_TRY(mx_alloc((void**)&w.tc_X5f[f], n4 * sizeof(float), false));
    }
    ACSE_TRY(mx_alloc((void**)&w.tc_X5d, 4 * n4 * sizeof(float), false));
    for (int t = 0; t < 3; ++t) ACSE_TRY(mx_alloc((void**)&w.H32[t], n4 * sizeof(float), false));
    ACSE_TRY(mx_alloc((void**)&w.zdiag32, 4 * R2 * r * sizeof(float), false));
    ACSE_TRY(mx_alloc((void**)&w.gam32, 2 * R2 * sizeof(float), false));
    ACSE_TRY(mx_alloc((void**)&w.w32, 2 * R2 * sizeof(float), false));
    ACSE_TRY(mx_alloc((void**)&w.Q32, 2 * R2 * sizeof(float), false));
    ACSE_TRY(mx_alloc((void**)&w.tc_err, sizeof(int), true));
    if (c->opt.prec == ACSE_BF16X3 && r % 16 == 0 && r <= 64) {   // the B products on the tensor cores
        for (int k = 0; k < 8; ++k) {
            const size_t items = (k >> 1) < 2 ? P : R2;
            ACSE_TRY(mx_alloc((void**)&w.bx[k], items * R2 * sizeof(float), false));
        }
        int* h = (int*)malloc(P * sizeof(int));
        if (!h) return ACSE_ERR_NOMEM;
        for (int i = 0; i < (int)r; ++i)
            for (int j = i + 1; j < (int)r; ++j) h[pk_pair((int)r, i, j)] = i * (int)r + j;
        int s = mx_alloc((void**)&w.pair_ij, P * sizeof(int), false);
        if (s == ACSE_OK && cudaMemcpy(w.pair_ij, h, P * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            s = ACSE_ERR_CUDA;
        free(h);
        ACSE_TRY(s);
    }
    return ACSE_OK;
}

void tc_mixed_free(acse_ctx* c) {
    Work& w = c->w;
    void* ptrs[] = {w.tc_pairCp[0], w.tc_pairCp[2], w.tc_pairA[0], w.tc_pairA[1], w.tc_pairA[2], w.tc_pairB[0], w.tc_pairB[1], w.tc_pairB[2],
                    w.tc_pairC[0], w.tc_pairC[1], w.tc_pairC[2], w.M32[0], w.M32[1], w.M32[2], w.tc_Md, w.tc_Zd,
                    w.tc_Mf[0], w.tc_Mf[1], w.tc_Zf[0], w.tc_Zf[1], w.tc_X5f[0], w.tc_X5f[1], w.tc_X5d,
                    w.H32[0], w.H32[1], w.H32[2], w.zdiag32, w.gam32, w.w32, w.Q32, w.tc_err,
                    w.Kh32[0], w.Kh32[1], w.Kh32[2], w.A32[0], w.A32[1], w.A32[2], w.W32s[0], w.W32s[1], w.W32s[2],
                    w.bx[0], w.bx[1], w.bx[2], w.bx[3], w.bx[4], w.bx[5], w.bx[6], w.bx[7], w.pair_ij};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}
