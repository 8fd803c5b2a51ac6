"""GB300-native polynomial multigrid for nodal SIPG DG Poisson problems on
periodic 3D Cartesian grids (Stiller, arXiv 1612.04796).

The solver is the C-ABI CUDA library built from csrc/ (see include/mgdg.h);
this package only builds and loads it and marshals arguments.  There is no
CPU fallback: load_library() raises if the library is missing.
"""
from ._lib import LIB_PATH, header_symbols, load_library  # noqa: F401


def build(force=False, verbose=False):
    from .libbuild import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("MGSolver", "MGError", "solve_batch"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
