"""The allocation-free entry point bidiag_band_noalloc against the regular bidiag_band.

bidiag_band_noalloc serves callers that may not allocate device memory (an application whose GPU
memory is wholly owned by another allocator, or a service that forbids device allocation after
start-up): its scratch is a fixed 8 MiB array that the library declares statically.  Three calls in a
row, with different shapes, variants and trees (the last one smaller than the one before it), must
each give the band of the regular entry point within the parity tolerance (1e-12 * ||A||_F), so that
nothing an earlier call leaves in the shared array leaks into a later one; a problem larger than the
array must be refused before any work.

This file is collected last on purpose (its name sorts after the other test files).
"""
import ctypes

import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu


def _regular_band(torch, h, A, nb, ib, tree, variant):
    res = h.band(A, nb, ib, tree, variant)
    h.sync()
    ab = res.band()
    res.free()
    return ab


def _noalloc_band(torch, A, nb, ib, tree, variant, stream):
    m, n = A.shape
    ab = torch.full((n, nb + 1), float("nan"), dtype=torch.float64, device="cuda").t()   # (nb+1) x n, ld nb+1
    rc = G.bidiag_band_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), nb, ib, G.TREES[tree],
                               G.VARIANTS[variant], ctypes.c_void_p(ab.data_ptr()), nb + 1,
                               ctypes.c_void_p(stream.cuda_stream))
    assert rc == G.OK, rc
    return ab


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    G.load_library()
    h = G.Handle()
    stream = h.stream
    cases = [
        (300, 200, 32, 8, "greedy", "rbidiag", 7),    # ragged 10 x 7 tiles, R-BiDiag
        (512, 512, 64, 16, "auto", "bidiag", 8),      # the small square workload's shape
        # smaller again after the larger call: its tiles, R copy, T factors and flags are a prefix of
        # what the 512 x 512 call left behind, so stale contents would show here
        (256, 160, 32, 8, "flatts", "rbidiag", 9),
    ]
    try:
        for (m, n, nb, ib, tree, variant, seed) in cases:
            A = torch.from_numpy(inputs.gaussian(m, n, seed=seed)).cuda()
            ref = _regular_band(torch, h, A, nb, ib, tree, variant)
            got = _noalloc_band(torch, A, nb, ib, tree, variant, stream)
            torch.cuda.synchronize()
            tol = 1e-12 * torch.linalg.norm(A).item()
            err = (got - ref).abs().max().item()
            assert err <= tol, f"{m}x{n} {tree} {variant}: {err:.3e} > {tol:.3e}"
    finally:
        h.close()


def test_noalloc_refuses_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    G.load_library()
    m = n = 2048                     # the tile copy alone is 32 MiB > 8 MiB
    A = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    ab = torch.zeros((n, 65), dtype=torch.float64, device="cuda").t()
    rc = G.bidiag_band_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), m, 64, 16, G.GREEDY, G.BIDIAG,
                               ctypes.c_void_p(ab.data_ptr()), 65, None)
    assert rc == G.ERR_SCRATCH
    assert not ab.any().item()       # refused before any work was enqueued
    assert G.bidiag_band_noalloc(8, 10, ctypes.c_void_p(A.data_ptr()), 8, 4, 2, 0, 0,
                                 ctypes.c_void_p(ab.data_ptr()), 5, None) == G.ERR_UNSUPPORTED
    assert G.bidiag_band_noalloc(8, 8, None, 8, 4, 2, 0, 0, ctypes.c_void_p(ab.data_ptr()), 5, None) == -3
