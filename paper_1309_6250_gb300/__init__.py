"""GB300-native evaluation of planewave-derived orbitals through tricubic splines.

Method: Parker, Umrigar, Alfe, Hennig, Wilkins, arXiv:1309.6250 (smoothing and
interpolating B-splines with an optional separate Laplacian table, Lagrange and pp
variants).  The arithmetic runs in libqmcspl.so (hand-written CUDA for sm_103a, C ABI
in include/qmcspl.h); this package only marshals arguments and owns no fallback.
"""

__all__ = ["OrbitalSplines", "eval_batched", "SplineOrbitalFunction", "evaluate"]


def __getattr__(name):
    if name in ("OrbitalSplines", "eval_batched"):
        from . import api
        return getattr(api, name)
    if name in ("SplineOrbitalFunction", "evaluate"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
