"""ctypes binding of libacse (include/acse.h).  Argument marshalling only: every step of the
hot path runs in the library's CUDA kernels.  There is no fallback: if the shared library is
missing or fails to load, every call raises."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libacse.so")

ACSE_FP64, ACSE_BF16X3, ACSE_TF32, ACSE_TF32X3, ACSE_OZAKI = 0, 1, 2, 3, 4
PREC = {"fp64": ACSE_FP64, "bf16x3": ACSE_BF16X3, "tf32": ACSE_TF32, "tf32x3": ACSE_TF32X3, "ozaki": ACSE_OZAKI}

# symbols declared in include/acse.h
EXPORTS = ("acse_create", "acse_destroy", "acse_energy", "acse_residual", "acse_step",
           "acse_residual_backward", "acse_profile", "acse_profile_read", "acse_sync_status",
           "acse_clear_status", "acse_set_wait_bound_ns", "acse_energy_noalloc", "acse_batch_create",
           "acse_batch_destroy", "acse_batch_set_D", "acse_batch_get_D", "acse_batch_run", "acse_batch_info",
           "acse_extrapolate", "acse_batch_history", "acse_batch_extrapolate", "acse_schedule_state",
           "acse_batch_residual_backward", "acse_ozaki_plan_info",
           "acse_strerror", "acse_last_error", "acse_version")


class AcseOpts(ctypes.Structure):
    _fields_ = [("r", c_int), ("n_alpha", c_int), ("n_beta", c_int), ("prec", c_int), ("recon", c_int),
                ("mask_active", c_int), ("act_lo", c_int), ("act_hi", c_int), ("line_search", c_int),
                ("eps0", c_double), ("check_inputs", c_int), ("singlet", c_int), ("oz_slices", c_int),
                ("refine", c_int), ("refine_slices", c_int), ("refine_tol", c_double), ("gemm_tile", c_int)]


class AcseError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: status {status} ({strerror(status)})")
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libacse.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.acse_create.argtypes = [POINTER(c_void_p), POINTER(AcseOpts), c_void_p, c_void_p, c_void_p]
        L.acse_destroy.argtypes = [c_void_p]
        L.acse_energy.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.acse_residual.argtypes = [c_void_p] + [c_void_p] * 7
        L.acse_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p]
        L.acse_residual_backward.argtypes = [c_void_p, POINTER(c_void_p), c_int, c_double, c_double, c_double,
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.acse_strerror.argtypes = [c_int]
        L.acse_strerror.restype = ctypes.c_char_p
        L.acse_last_error.argtypes = [c_void_p]
        L.acse_version.restype = ctypes.c_char_p
        L.acse_profile.argtypes = [c_void_p, c_int]
        L.acse_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(ctypes.c_longlong),
                                        POINTER(ctypes.c_longlong)]
        L.acse_energy_noalloc.argtypes = [c_int, c_int, c_int] + [c_void_p] * 7
        L.acse_energy_noalloc.restype = c_int
        L.acse_batch_create.argtypes = [POINTER(c_void_p), c_int, POINTER(AcseOpts), POINTER(c_void_p),
                                        POINTER(c_void_p), c_void_p]
        L.acse_batch_destroy.argtypes = [c_void_p]
        L.acse_batch_set_D.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_double]
        L.acse_batch_get_D.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p]
        L.acse_batch_run.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
        L.acse_batch_info.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(ctypes.c_longlong)]
        L.acse_extrapolate.argtypes = [c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p]
        L.acse_batch_history.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, POINTER(c_int)]
        L.acse_batch_extrapolate.argtypes = [c_void_p, c_int, c_void_p]
        L.acse_batch_residual_backward.argtypes = [c_void_p, c_int, POINTER(c_void_p), c_int, c_double, c_double,
                                                   c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.acse_schedule_state.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int)]
        L.acse_schedule_state.restype = c_int
        L.acse_ozaki_plan_info.argtypes = [c_int, c_int, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                           POINTER(c_int)]
        L.acse_ozaki_plan_info.restype = c_int
        for name in ("acse_batch_create", "acse_batch_destroy", "acse_batch_set_D", "acse_batch_get_D",
                     "acse_batch_run", "acse_batch_info", "acse_extrapolate", "acse_batch_history",
                     "acse_batch_extrapolate", "acse_batch_residual_backward"):
            getattr(L, name).restype = c_int
        L.acse_sync_status.argtypes = [c_void_p]
        L.acse_clear_status.argtypes = [c_void_p]
        L.acse_set_wait_bound_ns.argtypes = [c_void_p, ctypes.c_ulonglong, c_int]
        for name in ("acse_create", "acse_destroy", "acse_energy", "acse_residual", "acse_step",
                     "acse_residual_backward", "acse_last_error", "acse_profile", "acse_profile_read",
                     "acse_sync_status", "acse_clear_status", "acse_set_wait_bound_ns"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().acse_strerror(int(status)).decode()


def version() -> str:
    return lib().acse_version().decode()


def ptr(x):
    """Raw address of a torch tensor (device or host) or a numpy array (host); None -> NULL."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported argument type {type(x)}")


def _check(status, what):
    if status != 0:
        raise AcseError(status, what)


def current_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


RECON = {"V": 0, "NY": 1}


def acse_create(r, n_alpha, n_beta, h, V, prec="fp64", mask=None, line_search=False, eps0=1e-3,
                check_inputs=False, stream=None, recon="V", singlet=False, oz_slices=0, refine=False,
                refine_slices=0, refine_tol=0.0, gemm_tile=0):
    o = AcseOpts()
    o.r, o.n_alpha, o.n_beta = r, n_alpha, n_beta
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.recon = RECON[recon] if isinstance(recon, str) else int(recon)
    if mask is not None:
        o.mask_active, o.act_lo, o.act_hi = 1, int(mask[0]), int(mask[1])
    o.line_search = int(bool(line_search))
    o.eps0 = float(eps0)
    o.check_inputs = int(bool(check_inputs))
    o.singlet = int(bool(singlet))
    o.oz_slices = int(oz_slices)
    o.refine = int(bool(refine))
    o.refine_slices = int(refine_slices)
    o.refine_tol = float(refine_tol)
    o.gemm_tile = int(gemm_tile)
    h_ = c_void_p()
    st = current_stream_handle() if stream is None else stream
    _check(lib().acse_create(byref(h_), byref(o), ptr(h), ptr(V), st), "acse_create")
    return h_


def acse_destroy(ctx):
    _check(lib().acse_destroy(ctx), "acse_destroy")


def acse_energy(ctx, Daa, Dab, Dbb, E):
    _check(lib().acse_energy(ctx, ptr(Daa), ptr(Dab), ptr(Dbb), ptr(E)), "acse_energy")


def acse_residual(ctx, Daa, Dab, Dbb, Aaa, Aab, Abb, norm2):
    _check(lib().acse_residual(ctx, ptr(Daa), ptr(Dab), ptr(Dbb), ptr(Aaa), ptr(Aab), ptr(Abb), ptr(norm2)),
           "acse_residual")


def acse_step(ctx, Daa, Dab, Dbb, eps, E_out=None, norm2_out=None, eps_used=None):
    _check(lib().acse_step(ctx, ptr(Daa), ptr(Dab), ptr(Dbb), float(eps), ptr(E_out), ptr(norm2_out),
                           ptr(eps_used)), "acse_step")


def acse_residual_backward(ctx, D_ckpt, n_steps, eps, wE, wN, dh, dV, dDaa, dDab, dDbb):
    arr = (c_void_p * len(D_ckpt))(*[ptr(x) for x in D_ckpt])
    _check(lib().acse_residual_backward(ctx, arr, int(n_steps), float(eps), float(wE), float(wN), ptr(dh),
                                        ptr(dV), ptr(dDaa), ptr(dDab), ptr(dDbb)), "acse_residual_backward")


def acse_batch_residual_backward(b, i, D_ckpt, n_steps, eps, wE, wN, dh, dV, dDaa, dDab, dDbb):
    arr = (c_void_p * len(D_ckpt))(*[ptr(x) for x in D_ckpt])
    _check(lib().acse_batch_residual_backward(b, int(i), arr, int(n_steps), float(eps), float(wE), float(wN),
                                              ptr(dh), ptr(dV), ptr(dDaa), ptr(dDab), ptr(dDbb)),
           "acse_batch_residual_backward")


def acse_profile(ctx, enable):
    _check(lib().acse_profile(ctx, int(enable)), "acse_profile")


def acse_profile_read(ctx):
    """(GEMM milliseconds, timed GEMM launches, kernels launched) since the last reset."""
    ms = c_double()
    ng = ctypes.c_longlong()
    nl = ctypes.c_longlong()
    _check(lib().acse_profile_read(ctx, byref(ms), byref(ng), byref(nl)), "acse_profile_read")
    return ms.value, ng.value, nl.value


def acse_sync_status(ctx):
    _check(lib().acse_sync_status(ctx), "acse_sync_status")


def acse_clear_status(ctx):
    _check(lib().acse_clear_status(ctx), "acse_clear_status")


def acse_ozaki_plan_info(oz_slices, kmax, k):
    """The modular Ozaki GEMM's plan for one GEMM (host only): moduli count, kept bits, K chunks, moduli."""
    T, bits, ch = c_int(), c_int(), c_int()
    mods = (c_int * 19)()
    _check(lib().acse_ozaki_plan_info(int(oz_slices), int(kmax), int(k), ctypes.byref(T), ctypes.byref(bits),
                                      ctypes.byref(ch), mods), "acse_ozaki_plan_info")
    return {"moduli_count": T.value, "bits": bits.value, "chunks": ch.value, "moduli": list(mods[:T.value])}


def acse_set_wait_bound_ns(ctx, ns, inject_stall=False):
    _check(lib().acse_set_wait_bound_ns(ctx, int(ns), int(bool(inject_stall))), "acse_set_wait_bound_ns")


def acse_energy_noalloc(r, n_alpha, n_beta, h, V, Daa, Dab, Dbb, E, stream=None):
    """Energy through the allocation-free entry point (device tensors only)."""
    st = current_stream_handle() if stream is None else stream
    _check(lib().acse_energy_noalloc(int(r), int(n_alpha), int(n_beta), ptr(h), ptr(V), ptr(Daa), ptr(Dab),
                                     ptr(Dbb), ptr(E), st), "acse_energy_noalloc")


def _opts(r, n_alpha, n_beta, prec="fp64", mask=None):
    o = AcseOpts()
    o.r, o.n_alpha, o.n_beta = r, n_alpha, n_beta
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    if mask is not None:
        o.mask_active, o.act_lo, o.act_hi = 1, int(mask[0]), int(mask[1])
    o.eps0 = 1e-3
    return o


def acse_batch_create(problems, prec="bf16x3", masks=None, stream=None):
    """problems: sequence of objects with r, n_alpha, n_beta, h, V (numpy or tensors)."""
    n = len(problems)
    arr = (AcseOpts * n)()
    for i, p in enumerate(problems):
        arr[i] = _opts(p.r, p.n_alpha, p.n_beta, prec, None if masks is None else masks[i])
    hs = (c_void_p * n)(*[ptr(p.h) for p in problems])
    Vs = (c_void_p * n)(*[ptr(p.V) for p in problems])
    h_ = c_void_p()
    st = current_stream_handle() if stream is None else stream
    _check(lib().acse_batch_create(byref(h_), n, arr, hs, Vs, st), "acse_batch_create")
    return h_


def acse_batch_destroy(b):
    _check(lib().acse_batch_destroy(b), "acse_batch_destroy")


def acse_batch_set_D(b, i, Daa, Dab, Dbb, eps):
    _check(lib().acse_batch_set_D(b, int(i), ptr(Daa), ptr(Dab), ptr(Dbb), float(eps)), "acse_batch_set_D")


def acse_batch_get_D(b, i, Daa, Dab, Dbb):
    _check(lib().acse_batch_get_D(b, int(i), ptr(Daa), ptr(Dab), ptr(Dbb)), "acse_batch_get_D")


def acse_batch_run(b, n, nsteps, stop_rule=True):
    """Returns (E, norm2, steps, reason) as numpy arrays of length n."""
    import numpy as np
    E = np.zeros(n)
    N2 = np.zeros(n)
    S = np.zeros(n, dtype=np.int32)
    R = np.zeros(n, dtype=np.int32)
    _check(lib().acse_batch_run(b, int(nsteps), int(bool(stop_rule)), E.ctypes.data, N2.ctypes.data,
                                S.ctypes.data, R.ctypes.data), "acse_batch_run")
    return E, N2, S, R


def acse_batch_info(b):
    t = c_int()
    sp = c_int()
    nl = ctypes.c_longlong()
    _check(lib().acse_batch_info(b, byref(t), byref(sp), byref(nl)), "acse_batch_info")
    return t.value, sp.value, nl.value


FIT_KEYS = ("a", "b", "c", "k", "rss", "flag")


def acse_extrapolate(lam, E, out, n_skip=0, stream=None):
    """E(lambda) fit of one trajectory: lam, E (n float64 device tensors), out (6 float64, device)."""
    st = current_stream_handle() if stream is None else stream
    _check(lib().acse_extrapolate(int(lam.numel()), ptr(lam), ptr(E), int(n_skip), ptr(out), st),
           "acse_extrapolate")


def acse_batch_history(b, i, cap=4096):
    """(lambda, E) recorded for instance i, as numpy arrays."""
    import numpy as np
    lam = np.zeros(cap)
    E = np.zeros(cap)
    n = c_int()
    _check(lib().acse_batch_history(b, int(i), lam.ctypes.data, E.ctypes.data, int(cap), byref(n)),
           "acse_batch_history")
    k = min(n.value, cap)
    return lam[:k].copy(), E[:k].copy()


def acse_batch_extrapolate(b, n, n_skip=0):
    """The fit of every instance's record: a list of n dicts (a, b, c, k, rss, flag)."""
    import numpy as np
    out = np.zeros(6 * n)
    _check(lib().acse_batch_extrapolate(b, int(n_skip), out.ctypes.data), "acse_batch_extrapolate")
    return [dict(zip(FIT_KEYS, out[6 * i:6 * i + 6])) for i in range(n)]


def acse_schedule_state(ctx):
    """(switched to the FP64-accurate precision, steps taken in the starting precision)."""
    r = c_int()
    n = c_int()
    _check(lib().acse_schedule_state(ctx, byref(r), byref(n)), "acse_schedule_state")
    return bool(r.value), n.value
