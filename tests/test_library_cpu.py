"""Host-side checks that need no GPU: the library builds, loads and exports every
symbol include/dg.h declares; the binding's argument checks; the input module."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_01492_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_c_abi():
    syms = declared_symbols()
    for s in ("dg_create_mesh", "dg_set_coefficient", "dg_apply", "dg_apply_adjoint",
              "dg_coeff_grad", "dg_cg_solve", "dg_cg_solve_batched", "dg_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_signatures_cover_the_header():
    import paper_1911_01492_gb300 as dg
    assert set(dg._SIGS) == set(declared_symbols())


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    import paper_1911_01492_gb300 as dg
    L = dg.library()
    h = ctypes.c_void_p()
    assert L.dg_create_mesh(0, 2, ctypes.byref(h)) == dg.DG_ERR_INVALID_ARG
    assert b"n_cells" in L.dg_last_error()
    assert L.dg_create_mesh(4, 9, ctypes.byref(h)) == dg.DG_ERR_INVALID_ARG
    assert L.dg_create_mesh(4, 2, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_apply(None, None, None, 0, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_cg_solve(None, None, None, 1e-10, 10, 0, None, None) == dg.DG_ERR_INVALID_ARG
    for fn in (L.dg_to_nodal, L.dg_to_modal, L.dg_apply_nodal):
        assert fn(None, None, None, None) == dg.DG_ERR_INVALID_ARG
        assert b"mesh is NULL" in L.dg_last_error()
    assert L.dg_cg_solve_batched_mode(None, 1, None, None, 1e-10, 10,
                                      dg.DG_CG_FP64 | dg.DG_CG_NODAL | dg.DG_CG_PRECOND_JACOBI,
                                      None, None) == dg.DG_ERR_INVALID_ARG
    assert L.dg_destroy_mesh(None) == dg.DG_OK


def test_missing_library_fails_loudly(tmp_path):
    import paper_1911_01492_gb300 as dg
    saved = dg._lib
    dg._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            dg.library(str(tmp_path / "nope.so"))
    finally:
        dg._lib = saved


def test_lognormal_field_layout_and_statistics():
    from paper_1911_01492_gb300 import inputs
    N, k = 4, 2
    n = k + 1
    K = inputs.lognormal_coefficient(N, k, seed=5)
    g, clipped = inputs.gaussian_random_field(N * n, 5)
    assert clipped == 0.0
    Kr = K.reshape(N, N, N, n, n, n)              # (cz, cy, cx, e, b, a)
    for (cx, cy, cz, a, b, e) in [(0, 0, 0, 0, 0, 0), (1, 2, 3, 2, 0, 1), (3, 3, 3, 2, 2, 2)]:
        assert Kr[cz, cy, cx, e, b, a] == np.exp(g[cx * n + a, cy * n + b, cz * n + e])
    # exact covariance of the embedding reproduces exp(-r/lambda) on the grid
    M = 16
    lam, _ = inputs._embedding_eigenvalues(M, 0.1, 1.0)
    c = np.fft.ifftn(lam).real
    d = 1.0 / M
    for (i, j, l) in [(0, 0, 0), (1, 0, 0), (3, 2, 1), (5, 5, 5)]:
        r = d * np.sqrt(i * i + j * j + l * l)
        assert abs(c[i, j, l] - np.exp(-r / 0.1)) < 1e-12
    # sample variance over many grid points of one large field
    g2, _ = inputs.gaussian_random_field(48, 17)
    assert abs(g2.var() - 1.0) < 0.25
    assert abs(g2.mean()) < 0.25


def test_uniform_vector_is_seeded():
    from paper_1911_01492_gb300 import inputs
    a = inputs.uniform_vector(3, 2, 1)
    b = inputs.uniform_vector(3, 2, 1)
    assert np.array_equal(a, b) and a.min() >= -1 and a.max() <= 1 and len(a) == 27 * 27
