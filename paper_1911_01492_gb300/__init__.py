"""GB300-native matrix-free SIPG-DG operator and CG solvers.

Thin ctypes binding over the C ABI declared in include/dg.h (libdg_gb300.so,
built in-tree by `paper_1911_01492_gb300.build`).  The binding only marshals
arguments: every step of the operator and the solvers runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream.  If the
library is missing or fails to load, every call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdg_gb300.so")

DG_OK = 0
DG_ERR_INVALID_ARG = 1
DG_ERR_CUDA = 2
DG_ERR_NOT_CONVERGED = 3
DG_ERR_BREAKDOWN = 4
DG_ERR_TIMEOUT = 5
DG_ERR_OOM = 6
DG_FP64 = 0
DG_FP32 = 1
DG_CG_FP64 = 0
DG_CG_MIXED_IR = 1
DG_CG_MIXED_IR_RESTART = 2
DG_CG_PRECOND_JACOBI = 256
DG_CG_PRECOND_BLOCK = 512
DG_CG_PRECOND_KRON = 1024
DG_CG_NODAL = 2048
DG_BC_DIRICHLET = 0x3F
DG_BC_FLOW_X = 0x03
DG_BACKUP_NONE = 0
DG_BACKUP_FULL = 1
DG_BACKUP_X64 = 2
DG_BACKUP_X32 = 3
DG_RECOVER_GLOBAL = 0
DG_RECOVER_LOCAL = 1
DG_RECOVER_LOCAL_AUX = 2

ERROR_NAMES = {
    DG_ERR_INVALID_ARG: "DG_ERR_INVALID_ARG",
    DG_ERR_CUDA: "DG_ERR_CUDA",
    DG_ERR_NOT_CONVERGED: "DG_ERR_NOT_CONVERGED",
    DG_ERR_BREAKDOWN: "DG_ERR_BREAKDOWN",
    DG_ERR_TIMEOUT: "DG_ERR_TIMEOUT",
    DG_ERR_OOM: "DG_ERR_OOM",
}

# every symbol include/dg.h declares, with its ctypes signature
_VP = ctypes.c_void_p
_SIGS = {
    "dg_last_error": (ctypes.c_char_p, []),
    "dg_create_mesh": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
    "dg_destroy_mesh": (ctypes.c_int, [_VP]),
    "dg_mesh_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double)]),
    "dg_set_coefficient": (ctypes.c_int, [_VP, _VP, _VP]),
    "dg_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "dg_apply_adjoint": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "dg_apply_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "dg_coeff_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "dg_cg_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   _VP, _VP]),
    "dg_cg_solve_resilient": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, _VP, _VP, _VP]),
    "dg_cg_solve_batched": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int,
                                           ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                           ctypes.c_double, ctypes.c_int, _VP, _VP]),
    "dg_cg_solve_batched_mode": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int,
                                                ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                _VP, _VP]),
    "dg_apply_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "dg_to_nodal": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "dg_to_modal": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "dg_apply_nodal": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "dg_diagonal": (ctypes.c_int, [_VP, _VP, _VP]),
    "dg_load_vector": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "dg_set_boundary": (ctypes.c_int, [_VP, ctypes.c_int]),
    "dg_set_geometry": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "dg_set_vertices": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "dg_dirichlet_rhs": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), _VP, _VP]),
    "dg_boundary_flux": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_double, _VP, _VP]),
    "dg_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]),
    "dg_timing_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "dg_timing_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
}


class DGError(RuntimeError):
    """A library call returned a DG_ERR_* code."""

    def __init__(self, code: int, func: str, msg: str):
        self.code = code
        super().__init__(f"{func}: {ERROR_NAMES.get(code, code)}: {msg}")


class CGStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int),
                ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double),
                ("rel_residual_rec", ctypes.c_double),
                ("seconds", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Resilience(ctypes.Structure):
    """dg_resilience: backup, injected loss and recovery of the resilient CG."""
    _fields_ = [("backup_interval", ctypes.c_int),
                ("backup", ctypes.c_int),
                ("recovery", ctypes.c_int),
                ("fault_iteration", ctypes.c_int),
                ("fault_cell_begin", ctypes.c_longlong),
                ("fault_cell_end", ctypes.c_longlong),
                ("aux_rtol", ctypes.c_double),
                ("aux_maxit", ctypes.c_int),
                ("fault_injected_at", ctypes.c_int),
                ("backup_iteration", ctypes.c_int),
                ("backups_taken", ctypes.c_int),
                ("aux_iterations", ctypes.c_int),
                ("backup_bytes", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdg_gb300.so (once) and declare its signatures.  Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_1911_01492_gb300.build` "
                "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, func: str):
    if rc != DG_OK:
        raise DGError(rc, func, library().dg_last_error().decode())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, numel: int, name: str, device: bool = True):
    import torch
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if device and not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if not device and t.is_cuda:
        raise TypeError(f"{name}: expected a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """n_cells^3 cubes of the unit cube with Q_degree elements on the current GPU."""

    def __init__(self, n_cells: int, degree: int):
        import torch
        torch.cuda.init()
        lib = library()
        h = ctypes.c_void_p()
        _check(lib.dg_create_mesh(int(n_cells), int(degree), ctypes.byref(h)), "dg_create_mesh")
        self._h = h
        self.n_cells = int(n_cells)
        self.degree = int(degree)
        nd, nc, n1, sg = (ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int(),
                          ctypes.c_double())
        _check(lib.dg_mesh_info(h, ctypes.byref(nd), ctypes.byref(nc), ctypes.byref(n1),
                                ctypes.byref(sg)), "dg_mesh_info")
        self.n_dofs = nd.value
        self.n_cells_total = nc.value
        self.n = n1.value
        self.sigma = sg.value
        self._autograd_logK = None   # log K of the last coefficient set by autograd

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(library().dg_destroy_mesh(self._h), "dg_destroy_mesh")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- boundary conditions and coefficient -----------------------------------
    def set_boundary(self, bc):
        """bc: "dirichlet" (every side, the default), "flow_x" (Dirichlet on
        x = 0 and x = 1, zero flux elsewhere) or a Dirichlet-side bit mask.
        Drops the coefficient: call set_coefficient afterwards."""
        mask = {"dirichlet": DG_BC_DIRICHLET, "flow_x": DG_BC_FLOW_X}.get(bc, bc)
        _check(library().dg_set_boundary(self._h, int(mask)), "dg_set_boundary")
        self._autograd_logK = None

    def set_geometry(self, A):
        """Affine geometry x = A xi (3x3, det A > 0; identity = the unit cube).
        Drops the coefficient: call set_coefficient afterwards."""
        vals = [float(v) for row in A for v in row]
        if len(vals) != 9:
            raise ValueError("A must be 3 x 3")
        _check(library().dg_set_geometry(self._h, (ctypes.c_double * 9)(*vals)),
               "dg_set_geometry")
        self._autograd_logK = None

    def set_vertices(self, X):
        """Multilinear geometry: vertex positions X, an array (N+1, N+1, N+1, 3)
        indexed [i, j, k] along x, y, z.  Drops the coefficient."""
        import numpy as np
        Xa = np.asarray(X, dtype=np.float64)
        n1 = self.n_cells + 1
        if Xa.shape != (n1, n1, n1, 3):
            raise ValueError(f"X must have shape {(n1, n1, n1, 3)}")
        flat = np.ascontiguousarray(Xa.transpose(2, 1, 0, 3)).reshape(-1)
        _check(library().dg_set_vertices(self._h, flat.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double))), "dg_set_vertices")
        self._autograd_logK = None

    def set_coefficient(self, K, stream=None):
        """K: CUDA float64 tensor of n_dofs values at the volume Gauss points."""
        self._autograd_logK = None
        _check(library().dg_set_coefficient(self._h, _ptr(K, _f64(), self.n_dofs, "K"),
                                            _stream(stream)), "dg_set_coefficient")

    # -- operator --------------------------------------------------------------
    def apply(self, x, y=None, stream=None, adjoint: bool = False):
        """y = A x (or A^T x) in the precision of x (float64 or float32)."""
        import torch
        prec = _prec(x.dtype)
        if y is None:
            y = torch.empty_like(x)
        xp = _ptr(x, x.dtype, self.n_dofs, "x")
        yp = _ptr(y, x.dtype, self.n_dofs, "y")
        fn = library().dg_apply_adjoint if adjoint else library().dg_apply
        _check(fn(self._h, xp, yp, prec, _stream(stream)),
               "dg_apply_adjoint" if adjoint else "dg_apply")
        return y

    # -- scaled Gauss-point (collocation) basis ------------------------------------
    def to_nodal(self, x, xhat=None, stream=None):
        """x_hat = Q x: per cell the values at the Gauss points scaled by
        sqrt(w_a w_b w_e) (an orthogonal change of basis; float64)."""
        import torch
        if xhat is None:
            xhat = torch.empty_like(x)
        _check(library().dg_to_nodal(self._h, _ptr(x, _f64(), self.n_dofs, "x"),
                                     _ptr(xhat, _f64(), self.n_dofs, "xhat"), _stream(stream)),
               "dg_to_nodal")
        return xhat

    def to_modal(self, xhat, x=None, stream=None):
        """x = Q^T x_hat, the inverse of to_nodal (float64)."""
        import torch
        if x is None:
            x = torch.empty_like(xhat)
        _check(library().dg_to_modal(self._h, _ptr(xhat, _f64(), self.n_dofs, "xhat"),
                                     _ptr(x, _f64(), self.n_dofs, "x"), _stream(stream)),
               "dg_to_modal")
        return x

    def apply_nodal(self, xhat, yhat=None, stream=None):
        """y_hat = (Q A Q^T) x_hat, the operator in the scaled Gauss-point basis (float64)."""
        import torch
        if yhat is None:
            yhat = torch.empty_like(xhat)
        _check(library().dg_apply_nodal(self._h, _ptr(xhat, _f64(), self.n_dofs, "xhat"),
                                        _ptr(yhat, _f64(), self.n_dofs, "yhat"),
                                        _stream(stream)), "dg_apply_nodal")
        return yhat

    def apply_adjoint(self, ybar, xbar=None, stream=None):
        return self.apply(ybar, xbar, stream, adjoint=True)

    def apply_host(self, x, y=None, stream=None):
        """y = A x for host tensors (pinned or pageable); blocks until y is written."""
        import torch
        prec = _prec(x.dtype)
        if y is None:
            y = torch.empty_like(x)
        _check(library().dg_apply_host(self._h, _ptr(x, x.dtype, self.n_dofs, "x", device=False),
                                       _ptr(y, x.dtype, self.n_dofs, "y", device=False), prec,
                                       _stream(stream)), "dg_apply_host")
        return y

    def coeff_grad(self, u, v, g=None, stream=None):
        """g = d(v^T A(K) u) / d log K at the volume Gauss points (float64)."""
        import torch
        if g is None:
            g = torch.empty_like(u)
        _check(library().dg_coeff_grad(self._h, _ptr(u, _f64(), self.n_dofs, "u"),
                                       _ptr(v, _f64(), self.n_dofs, "v"),
                                       _ptr(g, _f64(), self.n_dofs, "g"), _stream(stream)),
               "dg_coeff_grad")
        return g

    def diagonal(self, d=None, stream=None):
        """diag(A(K)) as a CUDA float64 tensor (the Jacobi preconditioner's diagonal)."""
        import torch
        if d is None:
            d = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        _check(library().dg_diagonal(self._h, _ptr(d, _f64(), self.n_dofs, "d"),
                                     _stream(stream)), "dg_diagonal")
        return d

    def load_vector(self, f, b=None, stream=None):
        """b = integral of f phi_m per DOF, f (CUDA float64) at the volume Gauss
        points in the layout of K."""
        import torch
        if b is None:
            b = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        _check(library().dg_load_vector(self._h, _ptr(f, _f64(), self.n_dofs, "f"),
                                        _ptr(b, _f64(), self.n_dofs, "b"), _stream(stream)),
               "dg_load_vector")
        return b

    def dirichlet_rhs(self, g, b=None, stream=None):
        """b = weak Dirichlet right-hand side of constant data g (six values,
        sides x-, x+, y-, y+, z-, z+; zero-flux sides ignored)."""
        import torch
        if b is None:
            b = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        gv = (ctypes.c_double * 6)(*[float(v) for v in g])
        _check(library().dg_dirichlet_rhs(self._h, gv, _ptr(b, _f64(), self.n_dofs, "b"),
                                          _stream(stream)), "dg_dirichlet_rhs")
        return b

    def boundary_flux(self, u, side: int, g: float, q=None, stream=None):
        """Total flux of u through Dirichlet side `side` with data g (a one-element
        CUDA float64 tensor, written asynchronously)."""
        import torch
        if q is None:
            q = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(library().dg_boundary_flux(self._h, _ptr(u, _f64(), self.n_dofs, "u"), int(side),
                                          float(g), _ptr(q, _f64(), 1, "q"), _stream(stream)),
               "dg_boundary_flux")
        return q

    # -- measurement -------------------------------------------------------------
    def timing_enable(self, max_applies: int):
        """Record CUDA events around both passes of the next max_applies applies."""
        _check(library().dg_timing_enable(self._h, int(max_applies)), "dg_timing_enable")

    def timing_read(self):
        """(applications recorded, summed pass-1 ms, summed pass-2 ms); disables timing."""
        n, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(library().dg_timing_read(self._h, ctypes.byref(n), ctypes.byref(a),
                                        ctypes.byref(b)), "dg_timing_read")
        return n.value, a.value, b.value

    # -- solvers ---------------------------------------------------------------
    def cg_solve(self, b, x=None, rtol: float = 1e-10, maxit: int = 100000,
                 mode: int = DG_CG_FP64, stream=None, raise_on_error: bool = True,
                 precond: str | None = None, nodal: bool = False):
        """Solve A x = b (blocking).  precond: None, "jacobi" (PCG with
        M = diag(A); same as OR-ing DG_CG_PRECOND_JACOBI into mode), "block"
        (M = the inverted cell blocks of A; FP64 mode, degree <= 4) or "kron"
        (M = the Kronecker cell blocks, fast diagonalisation; FP64 or mixed).
        nodal: iterate in the scaled Gauss-point basis (same as OR-ing
        DG_CG_NODAL into mode; FP64 or mixed mode, M = I or Jacobi).
        Returns (x, stats dict)."""
        import torch
        if precond not in (None, "jacobi", "block", "kron"):
            raise ValueError(f"unknown preconditioner {precond!r}")
        if precond == "jacobi":
            mode |= DG_CG_PRECOND_JACOBI
        elif precond == "block":
            mode |= DG_CG_PRECOND_BLOCK
        elif precond == "kron":
            mode |= DG_CG_PRECOND_KRON
        if nodal:
            mode |= DG_CG_NODAL
        if x is None:
            x = torch.zeros_like(b)
        st = CGStats()
        rc = library().dg_cg_solve(self._h, _ptr(b, _f64(), self.n_dofs, "b"),
                                   _ptr(x, _f64(), self.n_dofs, "x"), float(rtol), int(maxit),
                                   int(mode), ctypes.byref(st), _stream(stream))
        if raise_on_error:
            _check(rc, "dg_cg_solve")
        return x, st.as_dict()

    def cg_solve_resilient(self, b, x=None, rtol: float = 1e-10, maxit: int = 100000,
                           backup: str = "full", interval: int = 32, recovery: str = "global",
                           fault_iteration: int = -1, fault_cells=(0, 0),
                           aux_rtol: float = 1e-2, aux_maxit: int = 1000,
                           precond: str | None = None, stream=None,
                           raise_on_error: bool = True):
        """FP64 CG with in-memory backups every `interval` iterations
        (backup "full", "x64", "x32" or "none"), a data loss of the cells
        fault_cells = (begin, end) injected at the first check at or after
        fault_iteration (-1: none) and recovery "global", "local" or
        "local_aux" (local plus the auxiliary problem on the lost cells, to
        aux_rtol or aux_maxit iterations).  Returns (x, stats dict with the
        resilience fields added)."""
        import torch
        kinds = {"none": DG_BACKUP_NONE, "full": DG_BACKUP_FULL, "x64": DG_BACKUP_X64,
                 "x32": DG_BACKUP_X32}
        recs = {"global": DG_RECOVER_GLOBAL, "local": DG_RECOVER_LOCAL,
                "local_aux": DG_RECOVER_LOCAL_AUX}
        if precond not in (None, "jacobi"):
            raise ValueError(f"unknown preconditioner {precond!r}")
        mode = DG_CG_FP64 | (DG_CG_PRECOND_JACOBI if precond == "jacobi" else 0)
        if x is None:
            x = torch.zeros_like(b)
        res = Resilience(int(interval), kinds[backup], recs[recovery], int(fault_iteration),
                         int(fault_cells[0]), int(fault_cells[1]), float(aux_rtol),
                         int(aux_maxit), -1, -1, 0, 0, 0)
        st = CGStats()
        rc = library().dg_cg_solve_resilient(self._h, _ptr(b, _f64(), self.n_dofs, "b"),
                                             _ptr(x, _f64(), self.n_dofs, "x"), float(rtol),
                                             int(maxit), mode, ctypes.byref(res),
                                             ctypes.byref(st), _stream(stream))
        if raise_on_error:
            _check(rc, "dg_cg_solve_resilient")
        out = st.as_dict()
        out.update(res.as_dict())
        return x, out


def cg_solve_batched(meshes, bs, xs, rtol: float = 1e-8, maxit: int = 100000, stream=None,
                     raise_on_error: bool = True, precond: str | None = None,
                     nodal: bool = False):
    """Solve meshes[s] x[s] = b[s] for all s in one lock-step batched solve
    (FP64).  precond: None or "jacobi" (PCG with M = diag(A_s)).  nodal:
    iterate in the scaled Gauss-point basis (M = I only)."""
    if precond not in (None, "jacobi"):
        raise ValueError(f"unknown preconditioner {precond!r}")
    mode = DG_CG_FP64 | (DG_CG_PRECOND_JACOBI if precond == "jacobi" else 0)
    if nodal:
        mode |= DG_CG_NODAL
    count = len(meshes)
    if not (len(bs) == len(xs) == count):
        raise ValueError("meshes, bs and xs must have the same length")
    H = (ctypes.c_void_p * count)(*[m.handle for m in meshes])
    B = (ctypes.c_void_p * count)(*[_ptr(b, _f64(), m.n_dofs, "b") for b, m in zip(bs, meshes)])
    X = (ctypes.c_void_p * count)(*[_ptr(x, _f64(), m.n_dofs, "x") for x, m in zip(xs, meshes)])
    st = (CGStats * count)()
    rc = library().dg_cg_solve_batched_mode(H, count, B, X, float(rtol), int(maxit), mode,
                                            ctypes.cast(st, ctypes.c_void_p), _stream(stream))
    if raise_on_error:
        _check(rc, "dg_cg_solve_batched")
    return [s.as_dict() for s in st]


def apply_static(n_cells: int, degree: int, K, x, y=None, stream=None):
    """y = A(K) x in FP64 with no device allocation by the library: its
    temporaries live in a fixed 64 MiB device array (see dg_apply_static).
    For callers that may not allocate device memory; everyone else should use
    Mesh.  An allocation-free caller must pass y: with y=None this wrapper
    allocates the output itself with torch.empty_like."""
    import torch
    nd = n_cells ** 3 * (degree + 1) ** 3
    if y is None:
        y = torch.empty_like(x)
    _check(library().dg_apply_static(int(n_cells), int(degree), _ptr(K, _f64(), nd, "K"),
                                      _ptr(x, _f64(), nd, "x"), _ptr(y, _f64(), nd, "y"),
                                      _stream(stream)), "dg_apply_static")
    return y


def peak_probe(kind: str = "fp64", stream=None) -> float:
    """Measured fused multiply-add throughput of the current GPU in TFLOP/s:
    kind "fp64", "fp32" or "fp32x2" (packed FP32 pairs)."""
    k = {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind]
    out = ctypes.c_double()
    _check(library().dg_peak_probe(k, ctypes.byref(out), _stream(stream)), "dg_peak_probe")
    return out.value


def _f64():
    import torch
    return torch.float64


def _prec(dtype):
    import torch
    if dtype == torch.float64:
        return DG_FP64
    if dtype == torch.float32:
        return DG_FP32
    raise TypeError(f"unsupported dtype {dtype}: use float64 or float32")
