"""Shared helpers of the GPU tests (marshalling between numpy inputs and device tensors)."""
import numpy as np

from oracle import acse_oracle as O


def to_np(blocks):
    return tuple(b.detach().cpu().numpy() for b in blocks)


def oracle_residual_blocks(p, D_blocks, mask=None):
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    D = O.so_from_blocks(*D_blocks)
    A = O.residual(K, D, p.N)
    n2 = O.norm2(A)
    if mask is not None:
        A = O.active_mask(A, p.r, *mask)
    return O.blocks_from_so(A), n2


def oracle_step_blocks(p, D_blocks, eps, mask=None):
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    D = O.so_from_blocks(*D_blocks)
    Dn, A, U = O.step(K, D, p.N, eps, None if mask is None else (p.r, *mask))
    return O.blocks_from_so(Dn), O.energy(K, Dn), O.norm2(A)


def maxrel(got, want):
    """max |got - want| / max |want| over the three blocks."""
    num = max(np.abs(g - w).max() for g, w in zip(got, want))
    den = max(np.abs(w).max() for w in want)
    return num / den
