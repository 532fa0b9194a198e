"""Torch-facing convenience layer over the C ABI (marshalling only).

Spin blocks are passed as a tuple (Daa, Dab, Dbb) of contiguous float64 tensors of shape
(r, r, r, r) on the context's device; scalar results are returned as 1-element float64 device
tensors so that nothing synchronises unless the caller reads them.
"""
from __future__ import annotations

import torch

from . import _lib


def _dev(x, device):
    t = torch.as_tensor(x, dtype=torch.float64)
    return t.to(device).contiguous()


class ACSE:
    """One ACSE problem (integrals and options) bound to a CUDA stream."""

    def __init__(self, r, n_alpha, n_beta, h, V, prec="fp64", mask=None, line_search=False, eps0=1e-3,
                 check_inputs=False, device="cuda", stream=None, recon="V", singlet=False, oz_slices=0,
                 refine=False, refine_slices=0, refine_tol=0.0, gemm_tile=0):
        self.r, self.n_alpha, self.n_beta = r, n_alpha, n_beta
        self.device = torch.device(device)
        self.prec = prec
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.stream(self.stream):
            h_t = _dev(h, self.device)
            V_t = _dev(V, self.device)
            self.ctx = _lib.acse_create(r, n_alpha, n_beta, h_t, V_t, prec, mask, line_search, eps0, check_inputs,
                                        stream=self.stream.cuda_stream, recon=recon, singlet=singlet,
                                        oz_slices=oz_slices, refine=refine, refine_slices=refine_slices,
                                        refine_tol=refine_tol, gemm_tile=gemm_tile)
        self._scal = torch.zeros(3, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            _lib.acse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros_blocks(self):
        return tuple(torch.zeros((self.r,) * 4, dtype=torch.float64, device=self.device) for _ in range(3))

    def to_blocks(self, blocks):
        return tuple(_dev(b, self.device) for b in blocks)

    def energy(self, D):
        E = torch.empty(1, dtype=torch.float64, device=self.device)
        _lib.acse_energy(self.ctx, *D, E)
        return E

    def residual(self, D, out=None):
        A = out if out is not None else self.zeros_blocks()
        n2 = torch.empty(1, dtype=torch.float64, device=self.device)
        _lib.acse_residual(self.ctx, *D, *A, n2)
        return A, n2

    def step(self, D, eps=0.0):
        """In-place Euler step on D; returns (E_after, norm2_before, eps_used) device tensors."""
        s = torch.empty(3, dtype=torch.float64, device=self.device)
        _lib.acse_step(self.ctx, *D, eps, s[0:1], s[1:2], s[2:3])
        return s[0:1], s[1:2], s[2:3]

    def run_until_stop(self, D, cap, eps=0.0, rise_tol=1e-10):
        """Euler steps on D (in place) until the stopping rule of the Methods section fires, at most `cap`:
        stop when E or ||A|| rises (D goes back to the state before that step) or when |dE| < 1e-6 Eh.
        A rise counts when it exceeds the rounding level of the two values compared: ||A||^2 by more than
        rise_tol of itself, E by more than 1e-12 of |E| (near the floor of ||A||^2 two FP64-accurate
        evaluations differ by about 1e-13 relative, so a literal comparison decides on rounding).  Reads E
        and ||A||^2 back after every step.  Returns dict(E = energies of D_0 .. D_last, norm2 = ||A||^2
        before each step, eps = steps taken, reason, accepted = index of the returned D in E)."""
        with torch.cuda.stream(self.stream):   # every read-back below waits for this context's stream
            return self._run_until_stop(D, cap, eps, rise_tol)

    def _run_until_stop(self, D, cap, eps, rise_tol):
        Es = [float(self.energy(D))]
        n2s, epss = [], []
        # D_(k-1) and D_k kept while step k runs: ||A(D_k)||^2 is known only once step k has run
        keep = [tuple(x.clone() for x in D), tuple(x.clone() for x in D)]
        reason, acc = "cap", None
        for k in range(cap):
            for dst, src in zip(keep[k % 2], D):
                dst.copy_(src)                      # keep[k % 2] = D_k
            E, n2, e = self.step(D, eps)
            Es.append(float(E))
            n2s.append(float(n2))
            epss.append(float(e))
            if k >= 1 and n2s[k] > n2s[k - 1] * (1.0 + rise_tol):
                reason, acc = "norm rose", k - 1    # ||A(D_k)|| rose: back to D_(k-1)
                for dst, src in zip(D, keep[(k - 1) % 2]):
                    dst.copy_(src)
                break
            if Es[k + 1] > Es[k] + 1e-12 * abs(Es[k]):
                reason, acc = "energy rose", k      # E(D_(k+1)) rose: back to D_k
                for dst, src in zip(D, keep[k % 2]):
                    dst.copy_(src)
                break
            if abs(Es[k + 1] - Es[k]) < 1e-6:
                reason, acc = "converged", k + 1
                break
        if acc is None:
            acc = len(Es) - 1
        return dict(E=Es, norm2=n2s, eps=epss, reason=reason, accepted=acc, E_stop=Es[acc])

    def backward(self, D_ckpt, n_steps, eps, wE=1.0, wN=0.0):
        """Gradient of wE E(D_n) + wN ||A(D_n)||^2 w.r.t. (h, V, D0 blocks)."""
        r = self.r
        dh = torch.empty((r, r), dtype=torch.float64, device=self.device)
        dV = torch.empty((r,) * 4, dtype=torch.float64, device=self.device)
        dD = self.zeros_blocks()
        flat = []
        for k in range(n_steps + 1):
            blk = D_ckpt[k] if k < len(D_ckpt) else None
            flat.extend(blk if blk is not None else (None, None, None))
        _lib.acse_residual_backward(self.ctx, flat, n_steps, eps, wE, wN, dh, dV, *dD)
        return dh, dV, dD


class ACSEObjective(torch.autograd.Function):
    """f = wE E(D_n) + wN ||A(D_n)||^2 after n fixed Euler steps from D_0, differentiable with respect
    to h, V and the three blocks of D_0 through the library's adjoint (acse_residual_backward).

    forward(h, V, Daa, Dab, Dbb, n_alpha, n_beta, prec, nsteps, eps, wE, wN): h (r, r) and V
    (r, r, r, r) float64 device tensors, D_0 blocks (r, r, r, r); returns a 0-d float64 tensor.
    Every step's D is kept as a checkpoint (n + 1 triples of r^4 doubles), so the reverse sweep
    recomputes nothing.  Gradients are those of the library: dh and dV on the symmetric integrals
    (projected onto the p<->q and 8-fold symmetries), dD_0 on 2-RDM-symmetric tensors.  For a split
    precision the forward steps run in that precision and the reverse sweep in FP64 along them."""

    @staticmethod
    def forward(fctx, h, V, Daa, Dab, Dbb, n_alpha, n_beta, prec="fp64", nsteps=1, eps=1e-3, wE=1.0, wN=0.0):
        r = h.shape[0]
        ctx = ACSE(r, n_alpha, n_beta, h.detach(), V.detach(), prec, device=h.device)
        D = tuple(x.detach().clone().contiguous() for x in (Daa, Dab, Dbb))
        ckpt = [tuple(x.clone() for x in D)]
        for _ in range(nsteps):
            ctx.step(D, eps)
            ckpt.append(tuple(x.clone() for x in D))
        f = torch.zeros((), dtype=torch.float64, device=h.device)
        if wE != 0.0:
            f = f + wE * ctx.energy(D)[0]
        if wN != 0.0:
            _, n2 = ctx.residual(D)
            f = f + wN * n2[0]
        fctx.acse = ctx
        fctx.ckpt = ckpt
        fctx.args = (nsteps, eps, wE, wN)
        return f

    @staticmethod
    def backward(fctx, gf):
        nsteps, eps, wE, wN = fctx.args
        dh, dV, dD = fctx.acse.backward(fctx.ckpt, nsteps, eps, wE, wN)
        fctx.acse.close()
        fctx.ckpt = None
        return (gf * dh, gf * dV, gf * dD[0], gf * dD[1], gf * dD[2]) + (None,) * 7


def acse_objective(h, V, D0, n_alpha, n_beta, prec="fp64", nsteps=1, eps=1e-3, wE=1.0, wN=0.0):
    """Differentiable f = wE E(D_n) + wN ||A(D_n)||^2 (see ACSEObjective); D0 = (Daa, Dab, Dbb)."""
    return ACSEObjective.apply(h, V, *D0, n_alpha, n_beta, prec, nsteps, eps, wE, wN)
