"""Host-side checks of the C ABI: the in-tree library builds for sm_103a, loads, exports
every function include/*.h declares, and reports errors without a GPU call."""
import os
import re
import subprocess

import pytest

import paper_1707_02245_gb300 as P
from paper_1707_02245_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(pat_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_library_is_in_tree(lib):
    assert os.path.exists(P.library_path())
    assert os.path.commonpath([P.library_path(), ROOT]) == ROOT


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(P.EXPORTED)
    nm = subprocess.run(["nm", "-D", "--defined-only", P.library_path()], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", nm), f"{n} not exported"


def test_error_strings_and_defaults(lib):
    assert P.pat_error_string(0) == "ok"
    assert "invalid" in P.pat_error_string(P.PAT_ERR_INVALID_ARG)
    assert "non-finite" in P.pat_error_string(P.PAT_ERR_NONFINITE)
    p = P.pat_params_default()
    assert (p.reg, p.iters, p.gap_every, p.precond) == (P.PAT_TV, 100, 10, P.PAT_PRECOND_DIAG)
    assert (p.alpha, p.beta, p.theta, p.box_u, p.box_v) == (0.05, 1.0, 1.0, 2.0, 4.0)


def test_invalid_geometry_rejected_before_any_device_call(lib):
    with pytest.raises(P.PatError) as ei:
        P.pat_create_geometry(1, [[0.0, 0.0]], 4, 0.0, 0.1, 16)
    assert ei.value.code == P.PAT_ERR_INVALID_ARG
    with pytest.raises(P.PatError):
        P.pat_create_geometry(8, [[0.0, 0.0]], 4, 0.0, -0.1, 16)
    with pytest.raises(P.PatError):
        P.pat_create_geometry(8, [[0.0, 0.0]], 4, 0.0, 0.1, 100000)
    with pytest.raises(P.PatError):
        P.pat_create_geometry(8, [[float("nan"), 0.0]], 4, 0.0, 0.1, 16)


def test_missing_library_fails_loudly(tmp_path):
    import importlib
    mod = importlib.import_module("paper_1707_02245_gb300")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            mod.load(str(tmp_path / "nope.so"))
    finally:
        mod._lib = saved


def test_nvcc_targets_sm103a_only():
    flags = B.common_flags()
    assert "arch=compute_103a,code=sm_103a" in flags
    assert not any("sm_90" in f or "sm_100" in f for f in flags)


def test_unet_arguments_rejected_before_any_device_call(lib):
    for bad in [dict(in_ch=3), dict(out_ch=0), dict(base_ch=12), dict(levels=0), dict(levels=9)]:
        kw = dict(in_ch=8, out_ch=8, base_ch=8, levels=2)
        kw.update(bad)
        with pytest.raises(P.PatError) as ei:
            P.pat_unet_create(**kw)
        assert ei.value.code == P.PAT_ERR_INVALID_ARG
    with pytest.raises(P.PatError) as ei:
        P.pat_conv3x3_forward(16, 1, 4, 4, 3, 16, None, 8, False, 16)
    assert ei.value.code == P.PAT_ERR_INVALID_ARG
    with pytest.raises(P.PatError) as ei:
        P.pat_conv3x3_backward_weight(16, 16, 1, 4, 4, 8, 12, 16)
    assert ei.value.code == P.PAT_ERR_INVALID_ARG
    # the tensor-memory kernels read x and w, and write y, in 16-byte vectors and TMA boxes:
    # pointers off a 16-byte boundary are refused before any device call
    for x, w, y in [(24, 32, 48), (32, 40, 48), (32, 48, 56)]:
        with pytest.raises(P.PatError) as ei:
            P.pat_conv3x3_forward(x, 1, 4, 4, 8, w, None, 8, False, y)
        assert ei.value.code == P.PAT_ERR_INVALID_ARG
        with pytest.raises(P.PatError) as ei:
            P.pat_conv3x3_backward_data(x, 1, 4, 4, 8, w, 8, y)
        assert ei.value.code == P.PAT_ERR_INVALID_ARG


def test_header_shape_constants_match_the_binding():
    """The launch-shape constants of include/pat.h and the pat_shapes layout are the ones
    the Python binding passes."""
    import ctypes
    import re
    hdr = open(os.path.join(ROOT, "include", "pat.h")).read()
    consts = dict(re.findall(r"#define\s+(PAT_(?:FWD|UPD|ADJ)_\w+)\s+(-?\d+)", hdr))
    assert len(consts) >= 7
    for name, value in consts.items():
        assert getattr(P, name) == int(value), name
    body = re.search(r"typedef struct \{([^}]*)\} pat_shapes;", hdr).group(1)
    fields = re.findall(r"int\s+(\w+);", body)
    assert fields == [f for f, _ in P.pat_shapes._fields_]
    assert ctypes.sizeof(P.pat_shapes) == 4 * len(fields)
