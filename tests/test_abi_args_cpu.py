"""Argument checks of the C ABI that run before any CUDA call, exercised without a GPU.

`acse_create` validates the options (include/acse.h: 2 <= r <= 64, N >= 2, electrons per spin <= r,
a known precision, 4..10 Ozaki slices, a known reconstruction, n_alpha = n_beta for the spin-flip
option, a non-empty active range inside [0, r), a precision schedule that is off or on, without the
spin-flip option, with 4..10 slices and a finite threshold >= 0) before it allocates anything or touches the device;
`acse_energy_noalloc` rejects null pointers, empty shapes and r above its static scratch first;
`acse_batch_create` rejects 0 or more than 64 instances, mixed precisions, the NY reconstruction and
the Ozaki precision; the entry points taking a context or a batch reject a null one.  Each case must
return its documented status, and a failed create must leave its output handle NULL.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_2604_02550_gb300 import _lib

OK, ARG, SHAPE, UNSUPPORTED, TOO_LARGE = 0, -1, -2, -8, -9


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.lib()


def _opts(**kw):
    o = dict(r=6, n_alpha=2, n_beta=2, prec=_lib.ACSE_BF16X3, recon=0, mask_active=0, act_lo=0, act_hi=0,
             line_search=0, eps0=0.0, check_inputs=0, singlet=0, oz_slices=0)
    o.update(kw)
    return _lib.AcseOpts(**o)


def _create(L, opts, with_h=True, with_V=True, with_out=True):
    h = np.zeros((6, 6))
    V = np.zeros((6,) * 4)
    out = ctypes.c_void_p(123)   # must be reset to NULL on every failure
    st = L.acse_create(ctypes.byref(out) if with_out else None, ctypes.byref(opts),
                       h.ctypes.data if with_h else None, V.ctypes.data if with_V else None, None)
    if with_out:
        assert out.value is None, "a failed create leaves *ctx = NULL"
    return st


@pytest.mark.parametrize("kw,want", [
    (dict(r=1), SHAPE), (dict(r=65), SHAPE), (dict(r=0), SHAPE),
    (dict(n_alpha=1, n_beta=0), SHAPE), (dict(n_alpha=-1), SHAPE), (dict(n_alpha=7), SHAPE), (dict(n_beta=7), SHAPE),
    (dict(prec=-1), ARG), (dict(prec=5), ARG),
    (dict(prec=_lib.ACSE_OZAKI, oz_slices=3), ARG), (dict(prec=_lib.ACSE_OZAKI, oz_slices=11), ARG),
    (dict(recon=2), UNSUPPORTED), (dict(recon=-1), UNSUPPORTED),
    (dict(singlet=1, n_alpha=3, n_beta=2), ARG),
    (dict(mask_active=1, act_lo=2, act_hi=2), SHAPE), (dict(mask_active=1, act_lo=-1, act_hi=3), SHAPE),
    (dict(mask_active=1, act_lo=0, act_hi=7), SHAPE),
    (dict(refine=2), ARG), (dict(refine=1, singlet=1), ARG), (dict(refine=1, refine_slices=3), ARG),
    (dict(refine=1, refine_slices=11), ARG), (dict(refine=1, refine_tol=-1e-3), ARG),
    (dict(refine=1, refine_tol=float("nan")), ARG),
    (dict(gemm_tile=-1), ARG), (dict(gemm_tile=3), ARG),
])
def test_create_rejects_invalid_options(L, kw, want):
    assert _create(L, _opts(**kw)) == want


def test_create_rejects_null_arguments(L):
    assert _create(L, _opts(), with_h=False) == ARG
    assert _create(L, _opts(), with_V=False) == ARG
    assert _create(L, _opts(), with_out=False) == ARG


def test_entry_points_reject_a_null_context(L):
    assert L.acse_destroy(None) == ARG
    assert L.acse_energy(None, None, None, None, None) == ARG
    assert L.acse_residual(None, None, None, None, None, None, None, None) == ARG
    assert L.acse_step(None, None, None, None, 0.0, None, None, None) == ARG
    assert L.acse_residual_backward(None, None, 0, 0.0, 1.0, 0.0, None, None, None, None, None) == ARG
    assert L.acse_last_error(None) == ARG
    assert L.acse_sync_status(None) == ARG
    assert L.acse_clear_status(None) == ARG
    assert L.acse_set_wait_bound_ns(None, 0, 0) == ARG
    assert L.acse_profile(None, 1) == ARG


def test_energy_noalloc_host_checks(L):
    buf = np.zeros(8)
    p = [buf.ctypes.data] * 6
    assert L.acse_energy_noalloc(6, 2, 2, None, *p[1:], None) == ARG
    assert L.acse_energy_noalloc(0, 2, 2, *p, None) == SHAPE
    assert L.acse_energy_noalloc(6, 1, 0, *p, None) == SHAPE
    assert L.acse_energy_noalloc(1, 1, 1, *p, None) == SHAPE       # r = 1: acse_create rejects it too
    assert L.acse_energy_noalloc(3, 4, 0, *p, None) == SHAPE       # more alpha electrons than orbitals
    assert L.acse_energy_noalloc(3, 1, 4, *p, None) == SHAPE
    assert L.acse_energy_noalloc(65, 2, 2, *p, None) == TOO_LARGE


def test_every_status_has_its_own_text(L):
    texts = {s: _lib.strerror(s) for s in range(-9, 1)}
    assert texts[0] == "ok"
    assert len(set(texts.values())) == len(texts)
    assert _lib.strerror(-42) == "unknown status"


def _batch_create(L, n, opts_list, with_out=True):
    h = np.zeros((6, 6))
    V = np.zeros((6,) * 4)
    k = max(n, 1)
    arr = (_lib.AcseOpts * k)(*(opts_list + [_opts()] * (k - len(opts_list))))
    hp = (ctypes.c_void_p * k)(*([h.ctypes.data] * k))
    Vp = (ctypes.c_void_p * k)(*([V.ctypes.data] * k))
    out = ctypes.c_void_p(123)
    st = L.acse_batch_create(ctypes.byref(out) if with_out else None, n, arr, hp, Vp, None)
    if with_out:
        assert out.value is None, "a failed batch create leaves *batch = NULL"
    return st


def test_batch_create_rejects_invalid_arguments(L):
    assert _batch_create(L, 0, []) == ARG
    assert _batch_create(L, 65, []) == ARG
    assert _batch_create(L, 2, [], with_out=False) == ARG
    # one precision for the whole batch
    assert _batch_create(L, 2, [_opts(prec=_lib.ACSE_BF16X3), _opts(prec=_lib.ACSE_TF32)]) == ARG
    # the batch runs the V reconstruction, and not the Ozaki precision
    assert _batch_create(L, 2, [_opts(), _opts(recon=1)]) == UNSUPPORTED
    assert _batch_create(L, 1, [_opts(prec=_lib.ACSE_OZAKI)]) == UNSUPPORTED


def test_batch_entry_points_reject_a_null_batch(L):
    assert L.acse_batch_destroy(None) == ARG
    assert L.acse_batch_set_D(None, 0, None, None, None, 0.0) == ARG
    assert L.acse_batch_get_D(None, 0, None, None, None) == ARG
    assert L.acse_batch_run(None, 1, 0, None, None, None, None) == ARG
    assert L.acse_batch_info(None, None, None, None) == ARG
    assert L.acse_batch_residual_backward(None, 0, None, 1, 1e-3, 1.0, 0.0, None, None, None, None, None) == ARG
