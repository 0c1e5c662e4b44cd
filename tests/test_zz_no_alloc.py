"""dg_apply_static: the operator application for callers that may not allocate
device memory (allocator-free embedded or real-time runtimes that reserve all
device memory when they start, and frameworks that own every device
allocation).  Its temporaries live in a fixed file-scope device array instead
of cudaMalloc'd workspaces.

These tests call it through the C ABI and through the Python wrapper, compare
it with dg_apply and with the FP64 oracle on two calls in a row (the second on
a different mesh after the first has filled the shared array, so a stale
temporary would show), and check that sizes beyond the array are rejected.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1911_01492_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
CASES = [(6, 3, 7, 8), (5, 4, 9, 10)]   # (n_cells, degree, K seed, x seed)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_apply_matches_dg_apply_and_oracle_on_two_calls_in_a_row(cuda_device):
    import torch
    import paper_1911_01492_gb300 as dg
    from oracle import SIPG
    lib = dg.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (N, k, kseed, xseed) in CASES:
        Kh = inputs.lognormal_coefficient(N, k, seed=kseed)
        xh = inputs.uniform_vector(N, k, xseed)
        K = torch.from_numpy(Kh).cuda()
        x = torch.from_numpy(xh).cuda()
        m = dg.Mesh(N, k)
        m.set_coefficient(K)
        y_ref = m.apply(x)
        y = torch.full_like(x, float("nan"))
        rc = lib.dg_apply_static(N, k, _vp(K), _vp(x), _vp(y), stream)
        assert rc == dg.DG_OK, lib.dg_last_error().decode()
        torch.cuda.synchronize()
        err = float((y - y_ref).abs().max() / y_ref.abs().max())
        assert err <= TOL64, (N, k, err)
        yo = SIPG(N, k).apply(Kh, xh)
        err_o = np.abs(y.cpu().numpy() - yo).max() / np.abs(yo).max()
        assert err_o <= TOL64, (N, k, err_o)
        m.close()


def test_static_apply_python_wrapper_writes_the_callers_output(cuda_device):
    import torch
    import paper_1911_01492_gb300 as dg
    from oracle import SIPG
    for (N, k, kseed, xseed) in reversed(CASES):
        Kh = inputs.lognormal_coefficient(N, k, seed=kseed)
        xh = inputs.uniform_vector(N, k, xseed)
        K = torch.from_numpy(Kh).cuda()
        x = torch.from_numpy(xh).cuda()
        y = torch.full_like(x, float("nan"))
        out = dg.apply_static(N, k, K, x, y)
        assert out.data_ptr() == y.data_ptr()
        yo = SIPG(N, k).apply(Kh, xh)
        err = np.abs(y.cpu().numpy() - yo).max() / np.abs(yo).max()
        assert err <= TOL64, (N, k, err)


def test_static_apply_rejects_sizes_beyond_its_array(cuda_device):
    import torch
    import paper_1911_01492_gb300 as dg
    lib = dg.library()
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.dg_apply_static(40, 3, _vp(z), _vp(z), _vp(torch.zeros_like(z)), None)
    assert rc == dg.DG_ERR_INVALID_ARG
    assert b"static scratch" in lib.dg_last_error()
