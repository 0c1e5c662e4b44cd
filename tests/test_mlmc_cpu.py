"""Host logic of the multilevel Monte-Carlo driver: the sample allocation is
the minimiser of the total cost under the variance budget (checked against
the constraint and against perturbed allocations), and the process split of
Section 5 distributes all processes in proportion to work."""
import numpy as np

from paper_1911_01492_gb300 import inputs
from paper_1911_01492_gb300.mlmc import allocation, process_split


def test_allocation_meets_the_variance_budget_at_minimal_cost():
    rng = np.random.default_rng(0)
    for _ in range(50):
        L = int(rng.integers(2, 5))
        V = np.exp(rng.normal(-4, 2, L))
        C = np.exp(np.sort(rng.normal(0, 2, L)))
        eps = float(np.exp(rng.normal(-4, 0.5)))
        N = np.array(allocation(V, C, eps), float)
        assert np.sum(V / N) <= eps ** 2 / 2 * (1 + 1e-12)
        # continuous optimum of min sum N C s.t. sum V / N = eps^2 / 2 (Lagrange):
        # N* = 2 eps^-2 sqrt(V / C) sum sqrt(V C); rounding up adds < 1 sample per level
        Ns = 2 / eps ** 2 * np.sqrt(V / C) * np.sum(np.sqrt(V * C))
        assert np.all(N >= Ns - 1e-9) and np.all(N <= Ns + 1)
        # any feasible perturbation of the continuous optimum costs more
        for _ in range(20):
            d = rng.normal(0, 0.2, L)
            Np = Ns * np.exp(d)
            Np *= np.sum(V / Np) / (eps ** 2 / 2)      # rescale onto the constraint
            assert np.sum(Np * C) >= np.sum(Ns * C) * (1 - 1e-12)


def test_process_split_is_proportional_to_work():
    ideal, fl = process_split([64, 16, 4], [0.01, 0.1, 1.0], 152)
    assert abs(sum(ideal) - 152) <= 1e-9
    w = np.array([0.64, 1.6, 4.0])
    assert np.allclose(ideal, 152 * w / w.sum())
    assert fl == [int(v) for v in np.floor(ideal)]


def test_coupled_fields_share_one_realization():
    """The coarse level's coefficient is the fine level's field at the slots
    containing its Gauss points.  At degree 1 every slot of the finest grid
    (M = 4 cells x 2 points) contains exactly one fine Gauss point, so the
    coarse values appear among the fine values; a different seed changes them."""
    Kc, Kf = inputs.lognormal_on_levels([(2, 1), (4, 1)], seed=3)
    assert set(np.round(np.log(Kc), 12)) <= set(np.round(np.log(Kf), 12))
    Kc2, _ = inputs.lognormal_on_levels([(2, 1), (4, 1)], seed=4)
    assert np.abs(Kc - Kc2).max() > 0


def test_flow_levels_rejects_unknown_solver():
    import pytest
    from paper_1911_01492_gb300 import mlmc
    with pytest.raises(ValueError, match="solver"):
        mlmc.FlowLevels([(2, 1)], solver="direct")
