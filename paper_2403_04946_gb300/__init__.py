"""GB300 (sm_103a) tensor-train solver for the Burgers-Hopf characteristic-
function PDE (Rodgers & Venturi, arXiv 2403.04946).

The solver lives in the CUDA library libhopf.so behind the C ABI of
include/hopf.h; ``binding`` is its thin ctypes binding.  Build the library with
``paper_2403_04946_gb300.build.build()``.
"""
from . import binding  # noqa: F401

__all__ = ["binding"]
