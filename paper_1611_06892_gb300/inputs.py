"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

Holds none of the reduction's arithmetic: only random matrices with the structure of the paper's
workloads.  The paper generates its matrices with LAPACK's LATMS with prescribed singular values
(Sec. 6.1); here the stand-ins are

* ``gaussian``: i.i.d. N(0, 1) entries (numpy PCG64 stream of ``seed``), column-major;
* ``prescribed_singular_values``: A = U diag(s) V^T with Haar-distributed U (m x n, orthonormal columns)
  and V (n x n), each the Q factor of a seeded Gaussian matrix with the signs of R's diagonal folded in
  (Mezzadri 2007), so that A's singular values are exactly s up to roundoff;
* ``geometric_sv``: s_i = 10^(-8 i / (n - 1)), i = 0..n-1 (1 down to 1e-8).

Large matrices can be generated on a CUDA device through torch (same recipe, torch's Philox stream);
a given (shape, seed, device kind) always yields the same matrix.
"""
from __future__ import annotations

import numpy as np


def gaussian(m, n, seed):
    """m x n N(0, 1) matrix, column-major (Fortran order) float64."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m)).T)


def haar(m, n, seed):
    """m x n matrix with orthonormal columns, Haar distributed (m >= n)."""
    G = gaussian(m, n, seed)
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d)


def geometric_sv(n, lo=1e-8):
    if n == 1:
        return np.ones(1)
    return 10.0 ** (np.log10(lo) * np.arange(n) / (n - 1))


def prescribed_singular_values(m, n, s, seed_u, seed_v):
    """A = U diag(s) V^T (float64, column-major) with Haar U (m x n) and V (n x n)."""
    U = haar(m, n, seed_u)
    V = haar(n, n, seed_v)
    return np.asfortranarray((U * np.asarray(s)[None, :]) @ V.T)


def torch_gaussian(m, n, seed, device="cuda"):
    """m x n N(0, 1) float64 column-major torch tensor generated on ``device``."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(n, m, dtype=torch.float64, device=device, generator=g).t()


def torch_prescribed_singular_values(m, n, s, seed_u, seed_v, device="cuda"):
    """Same recipe as ``prescribed_singular_values`` on a CUDA device (for the 8192^2 workload)."""
    import torch

    def haar_t(rows, cols, seed):
        G = torch_gaussian(rows, cols, seed, device)
        Q, R = torch.linalg.qr(G)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d[None, :]

    U = haar_t(m, n, seed_u)
    V = haar_t(n, n, seed_v)
    sv = torch.as_tensor(np.asarray(s), dtype=torch.float64, device=device)
    A = (U * sv[None, :]) @ V.t()
    return A.t().contiguous().t()
