"""The C-ABI library builds, loads and exports every entry point include/daba.h declares
(no GPU needed: nothing here calls into CUDA)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    """Every function declared by a header under include/."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(daba_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("daba_create", "daba_set_observations", "daba_set_state", "daba_run", "daba_get_state",
                 "daba_export_checkpoint", "daba_import_checkpoint", "daba_last_error", "daba_destroy",
                 "daba_objective", "daba_set_wait_limit", "daba_probe_fma_rate"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2305_07026_b300 import build
    build.build()
    from paper_2305_07026_b300 import _lib
    for name in _declared():
        assert hasattr(_lib.lib, name), name
        assert name in _lib.EXPORTED, name


def test_default_options():
    from paper_2305_07026_b300 import _lib
    o = _lib.options()
    assert o.loss == 1 and o.loss_scale_px == 1.0 and o.xi == 1e-10 and o.eta == 0.5
    assert o.accelerated == 1 and o.cam_alternations == 2 and o.prec == 1


def test_pointer_marshalling():
    from paper_2305_07026_b300 import _lib
    a = np.arange(6, dtype=np.float64)
    assert _lib.ptr(a) == a.ctypes.data
    assert _lib.ptr(None) is None
    import pytest
    with pytest.raises(ValueError):
        _lib.ptr(np.zeros((4, 4))[:, 1])
