"""GB300-native (sm_103a) stepper for the FitzHugh-Nagumo RD-CNN of arXiv 2102.10340.

The hot path -- Eq. 1-3 of Sec. II.A on a torus -- runs in hand-written CUDA
kernels behind the C ABI of ``include/rdcnn.h`` (``librdcnn.so``).  This
package is the thin Python binding: torch supplies device memory and
streams.  Importing it does not load the library; the first API call does,
and raises if ``librdcnn.so`` has not been built (there is no CPU fallback).
"""


def build_library(force: bool = False) -> str:
    """Compile librdcnn.so with nvcc for sm_103a (in-tree); returns its path."""
    from .build import build

    return build(force=force)


def load():
    """Load librdcnn.so (raises RuntimeError if it is missing)."""
    from . import _lib

    return _lib.load()


def __getattr__(name):
    if name in ("Grid", "Batch", "RDCNNFunction", "run", "run_static", "launch_count", "grid_summary", "SUMMARY_FIELDS", "DEFAULT_PARAMS", "GRAD_NAMES"):
        from . import rdcnn

        return getattr(rdcnn, name)
    if name in ("RDCNNError",):
        from . import _lib

        return getattr(_lib, name)
    raise AttributeError(name)
