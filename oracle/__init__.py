"""FP64 CPU oracle (test infrastructure only; see dg_oracle)."""
from .dg_oracle import SIPG, cg, gauss_points, legendre, legendre_deriv  # noqa: F401
