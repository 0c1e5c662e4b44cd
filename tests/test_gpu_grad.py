"""Differentiation through the operator and the solve (autograd layer over the
C ABI), checked against the oracle's gradient and central finite differences."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import SIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg(cuda_device):
    import paper_1911_01492_gb300 as dg
    dg.library()
    return dg


def test_apply_gradients_match_oracle(dg):
    import torch
    from paper_1911_01492_gb300 import autograd as dga
    N, k = 3, 2
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=3)
    x = torch.from_numpy(inputs.uniform_vector(N, k, 4)).cuda().requires_grad_()
    w = torch.from_numpy(inputs.uniform_vector(N, k, 5)).cuda()
    logK = torch.from_numpy(np.log(K)).cuda().requires_grad_()
    m = dg.Mesh(N, k)
    y = dga.apply(x, logK, m)
    (w * y).sum().backward()
    A = D.assemble(K)
    gx_ref = A.T @ w.cpu().numpy()
    gk_ref = D.coeff_grad(K, x.detach().cpu().numpy(), w.cpu().numpy()).reshape(-1)
    gx = x.grad.cpu().numpy()
    gk = logK.grad.cpu().numpy()
    assert np.abs(gx - gx_ref).max() <= 1e-12 * np.abs(gx_ref).max()
    assert np.abs(gk - gk_ref).max() <= 1e-12 * np.abs(gk_ref).max()


def test_apply_gradcheck_tiny(dg):
    import torch
    from paper_1911_01492_gb300 import autograd as dga
    N, k = 2, 1
    m = dg.Mesh(N, k)
    x = torch.from_numpy(inputs.uniform_vector(N, k, 6)).cuda().requires_grad_()
    logK = torch.from_numpy(0.3 * inputs.uniform_vector(N, k, 7)).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: dga.apply(a, b, m), (x, logK), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)


def test_coefficient_setup_runs_only_when_log_k_changes(dg, monkeypatch):
    import torch
    from paper_1911_01492_gb300 import autograd as dga
    N, k = 3, 2
    D = SIPG(N, k)
    m = dg.Mesh(N, k)
    calls = []
    orig = m.set_coefficient
    monkeypatch.setattr(m, "set_coefficient", lambda K, stream=None: (calls.append(1), orig(K, stream)))
    K0 = inputs.lognormal_coefficient(N, k, seed=3)
    x = torch.from_numpy(inputs.uniform_vector(N, k, 4)).cuda()
    logK = torch.from_numpy(np.log(K0)).cuda().requires_grad_()
    for _ in range(3):                       # unchanged log K: one setup in all
        y = dga.apply(x, logK, m)
    y.sum().backward()
    assert len(calls) == 1
    # a write that the version counter does not see still re-derives K
    logK.data.add_(0.25)
    y = dga.apply(x, logK, m)
    assert len(calls) == 2
    yref = D.apply(K0 * math.exp(0.25), x.cpu().numpy())
    assert np.abs(y.detach().cpu().numpy() - yref).max() <= 1e-12 * np.abs(yref).max()
    # a coefficient set directly by the caller is not mistaken for log K's
    orig(torch.from_numpy(K0).cuda())
    y = dga.apply(x, logK, m)
    assert len(calls) == 3
    assert np.abs(y.detach().cpu().numpy() - yref).max() <= 1e-12 * np.abs(yref).max()


def observed_solution(D, K_ref_np, b, seed):
    A = D.assemble(K_ref_np).tocsc()
    u = spla.spsolve(A, b)
    rng = np.random.default_rng(seed)
    return u + 0.01 * np.sqrt(np.mean(u ** 2)) * rng.standard_normal(u.shape)


@pytest.mark.parametrize("k,mode,precond,rtol,tol", [
    (2, 0, None, 1e-13, 1e-8), (3, 0, None, 1e-13, 1e-8),
    (3, 0, "jacobi", 1e-13, 1e-8), (3, 1, "jacobi", 1e-11, 1e-6)])
def test_solve_gradient_matches_oracle_on_4cubed(dg, k, mode, precond, rtol, tol):
    """dL/dlogK for L = 0.5 ||u(K) - u_obs||^2 against the oracle's assembled
    adjoint gradient -g(u, A^{-1}(u - u_obs)); forward and adjoint solves by
    FP64 CG, FP64 Jacobi PCG or mixed-precision Jacobi PCG (tolerance from the
    solves' accuracy)."""
    import torch
    from paper_1911_01492_gb300 import autograd as dga
    N = 4
    D = SIPG(N, k)
    K = inputs.lognormal_coefficient(N, k, seed=5)
    b = inputs.constant_load_vector(N, k)
    u_obs = observed_solution(D, inputs.lognormal_coefficient(N, k, seed=40), b, 41)
    A = D.assemble(K).tocsc()
    u = spla.spsolve(A, b)
    lam = spla.spsolve(A, u - u_obs)
    g_ref = -D.coeff_grad(K, u, lam).reshape(-1)

    m = dg.Mesh(N, k)
    logK = torch.from_numpy(np.log(K)).cuda().requires_grad_()
    bd = torch.from_numpy(b).cuda()
    ud = dga.solve(bd, logK, m, rtol=rtol, mode=mode, precond=precond)
    L = 0.5 * ((ud - torch.from_numpy(u_obs).cuda()) ** 2).sum()
    L.backward()
    g = logK.grad.cpu().numpy()
    assert np.abs(g - g_ref).max() <= tol * np.abs(g_ref).max()


@pytest.mark.slow
def test_solve_gradient_central_differences_32cubed_q3(dg):
    """32^3 Q3 lognormal K: gradient by adjoint CG (FP64, Jacobi) against
    finite differences of the loss (mixed-precision Jacobi solves) along 20
    seeded directions.  Solves go to a relative residual of 1e-10
    recomputed in FP64: 1e-12 is below what FP64 CG can attain on this
    operator (its true residual floors near 5e-11, about u_64 times the
    condition number).  The solve error then enters a difference quotient
    divided by eps, so the quotient is the fourth-order central one,
    (-L(2e) + 8 L(e) - 8 L(-e) + L(-2e)) / (12 e), at eps = 1e-2: truncation
    O(eps^4) ~ 1e-8 and the solve error ~10x smaller than in a second-order
    quotient at eps = 1e-3 (whose worst direction sat at ~1e-4)."""
    import torch
    from paper_1911_01492_gb300 import autograd as dga
    N, k = 32, 3
    m = dg.Mesh(N, k)
    b = torch.from_numpy(inputs.constant_load_vector(N, k)).cuda()

    def solve_accurately():
        x, _ = m.cg_solve(b, rtol=1e-10, mode=dg.DG_CG_MIXED_IR, precond="jacobi")
        return x

    m.set_coefficient(torch.from_numpy(inputs.lognormal_coefficient(N, k, seed=40)).cuda())
    uref = solve_accurately()
    rng = np.random.default_rng(41)
    rms = float(torch.sqrt(torch.mean(uref ** 2)))
    u_obs = uref + 0.01 * rms * torch.from_numpy(rng.standard_normal(m.n_dofs)).cuda()
    logK = torch.from_numpy(np.log(inputs.lognormal_coefficient(N, k, seed=5))).cuda()

    def loss(lk):
        m.set_coefficient(torch.exp(lk))
        return 0.5 * float(((solve_accurately() - u_obs) ** 2).sum())

    lk = logK.clone().requires_grad_()
    u = dga.solve(b, lk, m, rtol=1e-10, mode=dg.DG_CG_FP64, precond="jacobi")
    (0.5 * ((u - u_obs) ** 2).sum()).backward()
    g = lk.grad.clone()
    drng = np.random.default_rng(42)
    eps = 1e-2
    worst = 0.0
    for _ in range(20):
        d = torch.from_numpy(drng.standard_normal(m.n_dofs)).cuda()
        fd = (-loss(logK + 2 * eps * d) + 8 * loss(logK + eps * d) - 8 * loss(logK - eps * d)
              + loss(logK - 2 * eps * d)) / (12 * eps)
        an = float(torch.dot(g, d))
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst <= 1e-4, worst
