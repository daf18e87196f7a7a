"""Host-side checks of the C ABI that need no GPU: the library builds/loads,
exports every entry point that include/psd.h declares, and validates
parameters before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "psd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_01475_gb300 import _lib
    return _lib.load_library()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("psd_create", "psd_destroy", "psd_residual", "psd_precond_solve", "psd_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_1607_01475_gb300 import psd_status_string
    assert psd_status_string(0) == "PSD_OK"
    assert psd_status_string(4) == "PSD_ERR_NOCONV"
    assert psd_status_string(99) == "PSD_UNKNOWN_STATUS"


def _params(**kw):
    from paper_1607_01475_gb300._lib import PSDParams
    base = dict(order=4, dim=2, n=(ctypes.c_int * 3)(64, 64, 1), h=0.1, p=4.0, s=0.1, eps=0.1,
                lam=0.0, precision=0, tol=1e-10, max_iter=100, max_outer=10, stream=None)
    base.update(kw)
    return PSDParams(**base)


@pytest.mark.parametrize("bad", [
    dict(order=5), dict(dim=4), dict(n=(ctypes.c_int * 3)(48, 64, 1)),
    dict(n=(ctypes.c_int * 3)(4, 64, 1)), dict(n=(ctypes.c_int * 3)(64, 2048, 1)),
    dict(n=(ctypes.c_int * 3)(64, 64, 2)), dict(h=0.0), dict(h=float("nan")), dict(p=1.5),
    dict(dim=3, n=(ctypes.c_int * 3)(8, 8, 8), p=7.0), dict(s=-1.0), dict(eps=0.0),
    dict(lam=-1.0), dict(precision=3), dict(tol=-1.0), dict(max_iter=-1),
    dict(precision=1, max_outer=0), dict(inner_eta=1.0), dict(inner_eta=-0.5), dict(inner_stall=-1),
    "alloc_without_free",
])
def test_create_rejects_invalid_parameters(lib, bad):
    """Invalid parameters are refused with PSD_ERR_INVALID before any device
    work (so this runs without a GPU)."""
    out = ctypes.c_void_p()
    if bad == "alloc_without_free":
        from paper_1607_01475_gb300._lib import ALLOC_FN
        keep = ALLOC_FN(lambda n, ctx: 0)
        prm = _params(alloc=keep)
    else:
        prm = _params(**bad)
    assert lib.psd_create(ctypes.byref(prm), ctypes.byref(out)) == 1
    assert not out.value
    buf = ctypes.create_string_buffer(256)
    assert lib.psd_last_error(None, buf, len(buf)) == 0
    assert len(buf.value) > 0


def test_null_arguments(lib):
    assert lib.psd_create(None, None) == 1
    assert lib.psd_destroy(None) == 0
    assert lib.psd_solve(None, None, None, None, None, None) == 1
    assert lib.psd_residual(None, None, None, None, None, None, None) == 1
    assert lib.psd_precond_solve(None, None, None) == 1


def test_info_and_params_structs_match_the_header():
    """The ctypes mirrors of psd_info and psd_params: field order as in
    include/psd.h, and the info dict the Python API returns."""
    import re
    from paper_1607_01475_gb300._lib import PSDInfo, PSDParams
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "psd.h")).read()
    for cls, name in ((PSDInfo, "psd_info"), (PSDParams, "psd_params")):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), hdr, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)\s*(?:\[\d+\])?\s*;|\(\*(\w+)\)", body)
        names = [a or b for a, b in fields]
        py = [("lambda" if f == "lam" else f) for f, _ in cls._fields_]
        assert names == py, (name, names, py)
    d = PSDInfo(iters=3, status=0).as_dict()
    assert d["iters"] == 3 and "energy" in d and "wall_ms" in d
