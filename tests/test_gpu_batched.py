"""Batched lock-step CG (one persistent cooperative kernel over all samples):
every sample's residual is recomputed by the oracle, and the batch agrees with
one-sample-per-call dg_cg_solve."""
import os

import numpy as np
import pytest

from oracle import SIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


# uneven levels: sizes and degrees differ inside one batch
LEVELS = [(4, 1), (4, 2), (3, 3), (3, 4), (5, 2), (2, 4)]


def make_batch(dg, levels, seed0=1000):
    import torch
    meshes, bs, xs, Ks = [], [], [], []
    for s, (N, k) in enumerate(levels):
        K = inputs.lognormal_coefficient(N, k, seed=seed0 + s, corr_len=0.1 * 64 / N)
        m = dg.Mesh(N, k)
        m.set_coefficient(torch.from_numpy(K).cuda())
        meshes.append(m)
        Ks.append(K)
        bs.append(torch.from_numpy(inputs.uniform_vector(N, k, 2000 + s)).cuda())
        xs.append(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
    return meshes, bs, xs, Ks


def test_batched_matches_sequential_and_oracle(dg):
    import torch
    meshes, bs, xs, Ks = make_batch(dg, LEVELS)
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10)
    for s, ((N, k), m, b, x, K, st) in enumerate(zip(LEVELS, meshes, bs, xs, Ks, stats)):
        assert st["status"] == 0, (s, st)
        D = SIPG(N, k)
        bn = b.cpu().numpy()
        xn = x.cpu().numpy()
        r = np.linalg.norm(bn - D.apply(K, xn)) / np.linalg.norm(bn)
        assert r <= 1.05e-10, (s, r)
        xseq, sst = m.cg_solve(b, rtol=1e-10)
        # same algorithm per sample, different reduction order
        assert abs(st["iterations"] - sst["iterations"]) <= max(3, sst["iterations"] // 20)
        assert float((x - xseq).norm() / xseq.norm()) <= 1e-6


def test_batched_jacobi_matches_sequential_and_oracle(dg):
    """The same uneven batch with M = diag(A_s): every sample's residual is
    recomputed by the oracle, each agrees with a one-sample Jacobi solve, and
    the batch needs fewer iterations in total than without M."""
    meshes, bs, xs, Ks = make_batch(dg, LEVELS, seed0=1100)
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, precond="jacobi")
    plain = dg.cg_solve_batched(meshes, bs, [x.clone().zero_() for x in xs], rtol=1e-10)
    assert sum(s["iterations"] for s in stats) < sum(s["iterations"] for s in plain)
    for s, ((N, k), m, b, x, K, st) in enumerate(zip(LEVELS, meshes, bs, xs, Ks, stats)):
        assert st["status"] == 0, (s, st)
        bn = b.cpu().numpy()
        r = np.linalg.norm(bn - SIPG(N, k).apply(K, x.cpu().numpy())) / np.linalg.norm(bn)
        assert r <= 1.05e-10, (s, r)
        xseq, sst = m.cg_solve(b, rtol=1e-10, precond="jacobi")
        assert abs(st["iterations"] - sst["iterations"]) <= max(3, sst["iterations"] // 20)
        assert float((x - xseq).norm() / xseq.norm()) <= 1e-6


@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_batched_single_sample_and_zero_rhs(dg, precond):
    import torch
    meshes, bs, xs, Ks = make_batch(dg, [(3, 2), (2, 3)], seed0=77)
    bs[1].zero_()
    xs[1].fill_(1.0)
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, precond=precond)
    assert all(s["status"] == 0 for s in stats)
    assert torch.count_nonzero(xs[1]).item() == 0
    one = dg.cg_solve_batched(meshes[:1], bs[:1], [torch.zeros_like(xs[0])], rtol=1e-10,
                              precond=precond)
    assert one[0]["status"] == 0


@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_batched_high_degrees_in_the_wide_block_kernel(dg, precond):
    """Degrees 5..8 (with a low degree in the same batch) run in the 256-thread
    instantiation of the persistent kernel: every sample's residual is
    recomputed by the oracle."""
    levels = [(2, 5), (2, 6), (1, 7), (2, 8), (3, 2)]
    meshes, bs, xs, Ks = make_batch(dg, levels, seed0=1300)
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, precond=precond)
    for s, ((N, k), b, x, K, st) in enumerate(zip(levels, bs, xs, Ks, stats)):
        assert st["status"] == 0, (s, st)
        bn = b.cpu().numpy()
        r = np.linalg.norm(bn - SIPG(N, k).apply(K, x.cpu().numpy())) / np.linalg.norm(bn)
        assert r <= 1.05e-10, (s, r)


def test_batched_launch_shapes_agree(dg, monkeypatch):
    """The tuner's launch shapes (blocks per SM, cells per work unit) change
    only the reduction order: the batch solved under each forced shape reaches
    the same iterates to rounding."""
    levels = [(4, 2), (3, 3), (3, 4)]
    meshes, bs, xs, Ks = make_batch(dg, levels, seed0=1400)
    results = []
    for shape in ("1,0", "2,1", "3,2", "1,2"):
        monkeypatch.setenv("DG_BATCHED_SHAPE", shape)
        for x in xs:
            x.zero_()
        st = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10, maxit=12, raise_on_error=False)
        assert all(s["iterations"] == 12 for s in st), shape
        results.append([x.clone() for x in xs])
    for t in range(1, len(results)):
        for a, b in zip(results[0], results[t]):
            assert float((a - b).norm() / a.norm()) <= 1e-10


def test_barrier_timeout_is_reported_and_gpu_stays_usable(dg, monkeypatch):
    """A test hook holds one block of the persistent kernel back so that the
    other blocks' bounded barrier waits expire: the call must return
    DG_ERR_TIMEOUT (no trap, no hang) and the context must stay usable."""
    import torch
    meshes, bs, xs, Ks = make_batch(dg, LEVELS[:3], seed0=500)
    monkeypatch.setenv("DG_TEST_BARRIER_STALL", "1")
    with pytest.raises(dg.DGError, match="TIMEOUT"):
        dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10)
    monkeypatch.delenv("DG_TEST_BARRIER_STALL")
    torch.cuda.synchronize()
    for x in xs:
        x.zero_()
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-10)
    assert all(s["status"] == 0 for s in stats)


def test_batched_rejects_bad_arguments(dg):
    import torch
    meshes, bs, xs, Ks = make_batch(dg, [(2, 2), (2, 2)], seed0=5)
    with pytest.raises(dg.DGError, match="share a mesh"):
        dg.cg_solve_batched([meshes[0], meshes[0]], bs, xs)
    # mixed modes are not batched: INVALID_ARG from the C entry point
    import ctypes
    lib = dg.library()
    H = (ctypes.c_void_p * 1)(meshes[0].handle)
    B = (ctypes.c_void_p * 1)(bs[0].data_ptr())
    X = (ctypes.c_void_p * 1)(xs[0].data_ptr())
    rc = lib.dg_cg_solve_batched_mode(H, 1, B, X, 1e-8, 100, dg.DG_CG_MIXED_IR, None, None)
    assert rc == dg.DG_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        dg.cg_solve_batched(meshes[:1], bs[:1], xs[:1], precond="ssor")


@pytest.mark.slow
def test_full_size_batch_first_iterations_match_single_sample_solver(dg):
    """The 256-sample workload at full size (128 x 16^3 Q2, 96 x 24^3 Q3,
    32 x 32^3 Q4, lognormal K, f = 1) in the benchmark's launch
    configuration, stopped after 20 lock-step iterations: every sample's x
    equals 20 iterations of dg_cg_solve on that sample (whose results the
    oracle checks in test_gpu_cg.py) up to reduction order."""
    import torch
    levels = [(128, 16, 2), (96, 24, 3), (32, 32, 4)]
    meshes, bs, xs = [], [], []
    s = 0
    for count, N, k in levels:
        for _ in range(count):
            m = dg.Mesh(N, k)
            m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=1000 + s)).cuda())
            meshes.append(m)
            bs.append(torch.from_numpy(inputs.constant_load_vector(N, k)).cuda())
            xs.append(torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda"))
            s += 1
    stats = dg.cg_solve_batched(meshes, bs, xs, rtol=1e-8, maxit=20, raise_on_error=False)
    assert all(st["iterations"] == 20 for st in stats)
    rng = np.random.default_rng(3)
    picked = [0, 127, 128, 223, 224, 255] + list(rng.choice(256, 6, replace=False))
    for i in picked:
        x1, st = meshes[i].cg_solve(bs[i], rtol=1e-8, maxit=20, raise_on_error=False)
        assert st["iterations"] == 20
        assert float((xs[i] - x1).norm() / x1.norm()) <= 1e-9, i
    for m in meshes:
        m.close()
