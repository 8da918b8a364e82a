"""Batched form: many uneven matrices reduced in one persistent launch.

Each batched result must be bitwise identical to the single-matrix reduction with the same tile size,
inner blocking, tree and variant (the sub-tasks and their dependencies are the same; only the queue
order interleaves matrices), and match the oracle; autotuned and FP32 batches are checked against the
oracle with the configuration the autotuner chose.
"""
import numpy as np
import pytest

import paper_1611_06892_gb300 as G
from oracle import bidiag as OB
from oracle import trees as T
from paper_1611_06892_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


@pytest.fixture(scope="module")
def handle(torch_mod):
    h = G.Handle()
    h.set_option(G.OPT_AUTO_RESOURCES, 3)
    yield h
    h.close()


def shapes(seed, count, mmax):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(8, mmax + 1))
        n = int(rng.integers(1, m + 1))
        out.append((m, n))
    return out


def test_batched_equals_single_and_oracle(handle, torch_mod):
    torch = torch_mod
    sh = shapes(1, 12, 200)
    cfg = [(16, 4, "greedy", "bidiag"), (32, 8, "auto", "rbidiag"), (16, 16, "flatts", "auto"),
           (8, 2, "flattt", "bidiag")]
    As = [inputs.gaussian(m, n, seed=b + 100) for b, (m, n) in enumerate(sh)]
    nb = [cfg[b % 4][0] for b in range(len(As))]
    ib = [cfg[b % 4][1] for b in range(len(As))]
    tree = [cfg[b % 4][2] for b in range(len(As))]
    var = [cfg[b % 4][3] for b in range(len(As))]
    dev = [torch.from_numpy(A).cuda() for A in As]
    res = handle.band_batched(dev, nb, ib, tree, var)
    handle.sync()
    for b, r in enumerate(res):
        single = handle.band(dev[b], nb[b], ib[b], tree[b], var[b])
        handle.sync()
        assert torch.equal(r.band(), single.band()), b
        assert r.desc.variant == single.desc.variant
        ref = OB.bidiag_band(As[b], nb[b], ib[b], G.TREES[tree[b]], r.desc.variant, resources=3)
        assert np.abs(r.band().cpu().numpy() - ref["ab"]).max() <= 1e-12 * np.linalg.norm(As[b])
        assert np.array_equal(r.tasks(), np.array(ref["tasks"], dtype=np.int32).reshape(-1, 6))
        single.free()
    # apply_q of a batched result
    b = 1
    C = inputs.gaussian(sh[b][0], 5, seed=7)
    ref = OB.bidiag_band(As[b], nb[b], ib[b], G.TREES[tree[b]], res[b].desc.variant, resources=3)
    got = res[b].apply_q(torch.from_numpy(C).cuda(), 1)
    handle.sync()
    assert np.abs(got.cpu().numpy() - OB.apply_q(ref, C, 1)).max() <= 1e-11 * np.abs(C).max()
    for r in res:
        r.free()


def test_batched_autotuned(handle, torch_mod):
    torch = torch_mod
    sh = shapes(2, 10, 300)
    As = [inputs.gaussian(m, n, seed=b + 200) for b, (m, n) in enumerate(sh)]
    res = handle.band_batched([torch.from_numpy(A).cuda() for A in As])
    handle.sync()
    for b, r in enumerate(res):
        d = r.desc
        assert d.nb in (32, 64, 128) and d.ib in (8, 16, 32) and d.ib <= d.nb   # the tuner's candidates
        ref = OB.bidiag_band(As[b], d.nb, d.ib, d.tree, d.variant, resources=3)
        assert np.abs(r.band().cpu().numpy() - ref["ab"]).max() <= 1e-12 * np.linalg.norm(As[b])
        r.free()


def test_batched_fp32(handle, torch_mod):
    torch = torch_mod
    sh = shapes(3, 8, 260)
    As = [inputs.gaussian(m, n, seed=b + 300).astype(np.float32) for b, (m, n) in enumerate(sh)]
    res = handle.band_batched([torch.from_numpy(np.asfortranarray(A)).cuda() for A in As])
    handle.sync()
    for b, r in enumerate(res):
        d = r.desc
        assert r.esize == 4
        A64 = As[b].astype(np.float64)
        ref = OB.bidiag_band(A64, d.nb, d.ib, d.tree, d.variant, resources=3)
        assert np.abs(r.band().cpu().numpy() - ref["ab"]).max() <= 5e-6 * np.linalg.norm(A64)
        r.free()


def test_batched_program_cache(handle, torch_mod):
    """A second call with the same shapes reuses the cached batch program: same bands bit for bit, and
    the first call's results stay valid while the second call's exist (and after they are freed)."""
    torch = torch_mod
    shp = shapes(5, 12, 96)
    As = [torch.from_numpy(np.asfortranarray(inputs.gaussian(m, n, seed=m + 3 * n))).cuda() for m, n in shp]
    r1 = handle.band_batched(As)
    handle.sync()
    b1 = [r.band() for r in r1]
    r2 = handle.band_batched(As)
    handle.sync()
    for x, r in zip(b1, r2):
        assert torch.equal(x, r.band())
    for r in r2:
        r.free()
    # other shapes in between, then the first results are still readable
    r3 = handle.band_batched(As[:5])
    handle.sync()
    for x, r in zip(b1, r1):
        assert torch.equal(x, r.band())
    for r in r1 + r3:
        r.free()
