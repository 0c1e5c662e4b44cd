"""MLMC estimate of the mean inlet flux (Section 5) on the GPU: every sample's
level difference Y = Q_l - Q_{l-1} is recomputed by the FP64 oracle (flow
problem assembled with full quadrature, direct solve, flux by face quadrature)
on the same coupled coefficient, and the estimate is the sum of the level
means."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import SIPG
from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu


def oracle_q(N, k, K):
    D = SIPG(N, k, bc="flow_x")
    g = (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    u = spla.spsolve(D.assemble(K).tocsc(), D.dirichlet_rhs(K, g))
    return D.boundary_flux(K, u, 0, 1.0)


def test_mlmc_samples_match_oracle(cuda_device):
    from paper_1911_01492_gb300 import mlmc
    levels = [(2, 1), (3, 2), (4, 2)]
    r = mlmc.estimate(levels, eps=1e-3, n_init=[6, 4, 3], max_cycles=1, seed0=700,
                      corr_len=0.3, rtol=1e-12)
    assert r["samples"] == [6, 4, 3]
    for l, Y in enumerate(r["Y"]):
        for i, y in enumerate(Y):
            seed = 700 + 100000 * l + i
            lv = [levels[l]] if l == 0 else [levels[l], levels[l - 1]]
            Ks = inputs.lognormal_on_levels(lv, seed, 0.3, 1.0)
            q = [oracle_q(N, k, K) for (N, k), K in zip(lv, Ks)]
            yref = q[0] - (q[1] if l > 0 else 0.0)
            assert abs(y - yref) <= 1e-8 * max(1.0, abs(q[0])), (l, i, y, yref)
    assert abs(r["estimate"] - sum(np.mean(Y) for Y in r["Y"])) <= 1e-12
    assert r["cycles"][0]["next_samples"] == \
        __import__("paper_1911_01492_gb300.mlmc", fromlist=["allocation"]).allocation(
            r["cycles"][0]["variance"], r["cycles"][0]["cost_dof_iterations"], 1e-3)


def test_mlmc_mixed_kron_solver_matches_oracle(cuda_device):
    """The same samples solved one per call by the mixed-precision CG with the
    Kronecker cell blocks: every Y against the oracle's direct solve."""
    from paper_1911_01492_gb300 import mlmc
    levels = [(2, 1), (3, 2), (4, 3)]
    r = mlmc.estimate(levels, eps=1e-3, n_init=[4, 3, 2], max_cycles=1, seed0=900,
                      corr_len=0.3, rtol=1e-11, solver="mixed")
    for l, Y in enumerate(r["Y"]):
        for i, y in enumerate(Y):
            seed = 900 + 100000 * l + i
            lv = [levels[l]] if l == 0 else [levels[l], levels[l - 1]]
            Ks = inputs.lognormal_on_levels(lv, seed, 0.3, 1.0)
            q = [oracle_q(N, k, K) for (N, k), K in zip(lv, Ks)]
            yref = q[0] - (q[1] if l > 0 else 0.0)
            assert abs(y - yref) <= 1e-8 * max(1.0, abs(q[0])), (l, i, y, yref)
