"""Differentiable band bidiagonalization: ``band_bidiag(A, ...)`` returns B in band storage and carries
its adjoint (``bidiag_band_backward``, the reverse sweep of the library) into torch's autograd.

Reflector store policy (``memory_budget`` bytes):

* the forward result - V tiles, their R copy and the T factors, about the size of A - is kept for the
  backward pass when it fits the budget ("checkpointed");
* otherwise it is freed right after the forward and the backward pass runs the reduction again from
  A before sweeping back ("recomputed"), so that between the two passes only A is held.

Argument marshalling only; both passes run in the library's kernels.
"""
from __future__ import annotations

import torch

from . import Handle

_handles = {}


def _handle(device):
    idx = torch.device(device).index
    idx = torch.cuda.current_device() if idx is None else idx
    h = _handles.get(idx)
    if h is None:
        h = _handles[idx] = Handle(device=idx)
    return h


def reflector_bytes(m, n, nb, ib, variant, esize):
    """Device bytes of a result's reflector store (tiles, R copy, T factors), as the library sizes it."""
    p, q = -(-m // nb), -(-n // nb)
    tiles = p * q + (0 if variant in ("bidiag", 0) else q * q)
    panels = 2 * p * q        # upper bound on the panel tasks of either variant
    return esize * (tiles * nb * nb + panels * ib * nb)


class BandBidiag(torch.autograd.Function):
    """ab = band of B = Q^T A P (Sec. 3.4 / 3.5); backward = the library's reverse sweep."""

    @staticmethod
    def forward(ctx, A, nb, ib, tree, variant, memory_budget, handle):
        h = handle if handle is not None else _handle(A.device)
        res = h.band(A.detach(), nb, ib, tree, variant)
        ab = res.band()
        ctx.cfg = (nb, ib, tree, variant, h)
        keep = memory_budget is None or reflector_bytes(A.shape[0], A.shape[1], nb, ib, variant,
                                                        A.element_size()) <= memory_budget
        if keep:
            ctx.res = res
            ctx.save_for_backward()
        else:
            res.free()
            ctx.res = None
            ctx.save_for_backward(A.detach())
        ctx.recomputed = not keep
        return ab

    @staticmethod
    def backward(ctx, ab_bar):
        nb, ib, tree, variant, h = ctx.cfg
        res = ctx.res
        if res is None:
            (A,) = ctx.saved_tensors
            res = h.band(A, nb, ib, tree, variant)
        A_bar = res.backward(ab_bar.detach())
        h.sync()
        res.free()
        ctx.res = None
        return A_bar, None, None, None, None, None, None


def band_bidiag(A, nb, ib, tree="greedy", variant="bidiag", memory_budget=None, handle=None):
    """Band (nb + 1) x n of B = Q^T A P for a float64 / float32 CUDA matrix A (m >= n), differentiable.

    memory_budget: bytes the reflector store may occupy between the forward and the backward pass
    (None: always keep it); above it the backward pass recomputes the reduction.
    """
    return BandBidiag.apply(A, nb, ib, tree, variant, memory_budget, handle)


def dense_from_band(ab, n=None):
    """Dense n x n B from its band storage (differentiable torch ops)."""
    nbp1, ncols = ab.shape
    nb = nbp1 - 1
    n = ncols if n is None else n
    B = ab.new_zeros((n, n))
    j = torch.arange(n, device=ab.device)
    for d in range(nb + 1):
        i = j + d - nb
        ok = i >= 0
        B = B.index_put((i[ok], j[ok]), ab[d, ok], accumulate=True)
    return B
