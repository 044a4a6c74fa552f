"""GB300-native stochastic-Galerkin domain-decomposition solver for the 2-D acoustic wave
equation in random media (arXiv 2512.23027).

The computation lives in the CUDA library ``libsg`` (C ABI in include/sg.h); this package
only marshals arguments to it.  Importing the package does not load the library; the first
use of :class:`Solver` does, and raises if the library has not been built.
"""
from .binding import Solver, solve_batch, library_path, load_library, SGError  # noqa: F401

__all__ = ["Solver", "solve_batch", "library_path", "load_library", "SGError"]
