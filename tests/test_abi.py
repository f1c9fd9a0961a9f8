"""The C-ABI library without a GPU: it loads, exports every entry point that
include/fsl.h declares, validates configurations, and its lattice tables hold
the published D3Q19/D3Q27 weights.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fsl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fsl_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_14496_gb300 import build
    build.build()
    from paper_2207_14496_gb300 import fsl
    return fsl


def test_library_exports_every_declared_symbol(lib):
    raw = lib.raw_library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(raw, n), f"{n} declared in include/fsl.h but not exported"
    assert set(names) == set(lib.EXPORTED)


def test_config_validation(lib):
    from paper_2207_14496_gb300 import inputs
    w = inputs.standing_wave(64)
    n = lib.workspace_bytes(w["params"])
    assert n > 64 * 64 * 19 * 8 * 2
    assert lib.workspace_bytes(w["params"], "fp16") < n
    bad = dict(w["params"], q=15)
    with pytest.raises(lib.FslError):
        lib.workspace_bytes(bad)
    with pytest.raises(lib.FslError):
        lib.workspace_bytes(dict(w["params"], nu=-1.0))
    with pytest.raises(lib.FslError):
        lib.workspace_bytes(dict(w["params"], shape=(0, 4, 4)))
    with pytest.raises(lib.FslError):
        lib.workspace_bytes(dict(w["params"], refill="eq", options=0, q=19, collision="trt", magic=0.0))


def test_create_rejects_bad_workspace(lib):
    from paper_2207_14496_gb300 import inputs
    w = inputs.standing_wave(16)
    cfg = lib.make_config(w["params"])
    h = ctypes.c_void_p()
    raw = lib.raw_library()
    assert raw.fsl_create(ctypes.byref(cfg), None, 1 << 20, None, ctypes.byref(h)) == -3
    assert raw.fsl_create(ctypes.byref(cfg), ctypes.c_void_p(256), 16, None, ctypes.byref(h)) == -3
    assert raw.fsl_create(ctypes.byref(cfg), ctypes.c_void_p(257), 1 << 30, None, ctypes.byref(h)) == -3
    assert raw.fsl_step(None, 1) == -1
    assert raw.fsl_status_string(-4) == b"unstable: |u| >= c_s or NaN"


@pytest.mark.parametrize("q", [19, 27])
def test_lattice_table(lib, q):
    c, w = lib.lattice_table(q)
    l2 = (c * c).sum(1)
    pub = {19: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}, 27: {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}}[q]
    for i in range(q):
        assert w[i] == pub[int(l2[i])]
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3)


def test_batch_create_rejects_bad_arguments():
    """Argument checks of fsl_batch_create run before any CUDA call."""
    import ctypes
    from paper_2207_14496_gb300 import fsl
    lib = fsl.raw_library()
    out = ctypes.c_void_p()
    assert lib.fsl_batch_create(None, 1, ctypes.c_void_p(1), 8, ctypes.byref(out)) == -1
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.fsl_batch_create(ctypes.cast(arr, ctypes.c_void_p), 1, ctypes.c_void_p(1), 8,
                                ctypes.byref(out)) == -1
    assert lib.fsl_batch_create(ctypes.cast(arr, ctypes.c_void_p), 0, ctypes.c_void_p(1), 8,
                                ctypes.byref(out)) == -1
    assert lib.fsl_batch_step(None, 1) == -1
    assert lib.fsl_batch_destroy(None) == -1
