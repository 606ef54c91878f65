"""B300 (sm_103a) implementation of one accelerated majorization-minimization iteration of
DABA (Decentralized and Accelerated Bundle Adjustment, arXiv 2305.07026) behind a C ABI.

``paper_2305_07026_b300.scenes`` builds seeded synthetic scenes; ``paper_2305_07026_b300._lib``
is the ctypes binding of ``include/daba.h`` (imported lazily so that the scene generator and
the build script work without the compiled library).
"""


def load():
    """Import the binding of the compiled CUDA library (raises if it is not built)."""
    from . import _lib
    return _lib
