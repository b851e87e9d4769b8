"""GB300-native semiclassical lattice Boltzmann library (arXiv 1710.09472).

The compute path is the CUDA library liblbm.so (C ABI in include/lbm.h);
this package holds its in-tree build step, a ctypes binding with the same
entry-point names, and the seeded synthetic workloads.  Importing the
package does not load the library; the first call into it does, and fails
loudly when the library is missing.
"""

__all__ = ["LBM", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _build

    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name == "LBM":
        from .lbm import LBM

        return LBM
    raise AttributeError(name)
