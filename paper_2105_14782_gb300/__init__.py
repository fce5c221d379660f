"""GB300-native (sm_103a) line-by-line opacity, optical depth and emission
library for the auto-differentiable spectrum model of Kawahara et al.
(arXiv:2105.14782).  The compute lives in libxs.so (csrc/, C ABI in
include/xs.h); paper_2105_14782_gb300.xs is its ctypes binding."""
from . import _build  # noqa: F401

__all__ = ["xs", "build"]


def build(force: bool = False) -> str:
    return _build.build(force=force)
