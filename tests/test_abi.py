"""The C-ABI library loads, exports every entry point include/collage.h declares, and rejects
invalid arguments before touching the GPU (runs without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300 import _lib as L
    return L


def _declared():
    src = open(os.path.join(ROOT, "include", "collage.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(collage_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for path in (lib.LIB_PATH, lib.LIB_CHECKED_PATH):  # the regular and the bounds-checked build
        so = C.CDLL(path)
        for n in names:
            assert hasattr(so, n), (path, n)
    assert set(names) == set(lib.SIGNATURES), set(names) ^ set(lib.SIGNATURES)


def test_struct_layouts_match_header(lib):
    # field names of the ctypes mirrors appear in the header's structs in the same order
    src = open(os.path.join(ROOT, "include", "collage.h")).read()
    for struct, name in ((lib.collage_problem, "collage_problem"),
                         (lib.collage_options, "collage_options"),
                         (lib.collage_info, "collage_info"),
                         (lib.collage_tuning, "collage_tuning")):
        body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*" + name + ";", src,
                         re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        decl = re.findall(r"\b([a-z_0-9]+)\s*(?:\[\d+\])?\s*[;,]", body)
        assert decl == [f for f, _ in struct._fields_], (name, decl)


def test_defaults_are_the_papers_constants(lib):
    o = lib.default_options()
    golden = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                golden[k.strip()] = float(v)
    assert (o.alpha, o.beta) == (golden["alpha"], golden["beta"])
    assert abs(o.gamma - golden["gamma"]) <= 1e-7 * golden["gamma"]
    assert (o.w_in, o.w_out) == (golden["w_in"], golden["w_out"])
    assert o.segs_per_cubic == 16 and o.rho_px == 1.0 and o.tau == 0.5


def _problem(**over):
    from paper_2406_04008_gb300 import workloads as W
    p = W.config_problem(1, n_elems=3)
    p.update(over)
    return p


@pytest.mark.parametrize("mutate,needle", [
    (lambda p: p.update(kind=np.array([0, 1, 1], np.int32)), "cubic path needs 3N"),
    (lambda p: p.update(kind=np.array([7, 1, 1], np.int32)), "unknown kind"),
    (lambda p: p["params0"].__setitem__(3, 0.0), "scale s must be > 0"),
    (lambda p: p["params0"].__setitem__(0, np.nan), "params must be finite"),
    (lambda p: p.update(ring_off=np.array([0, 2], np.int32)), "ring needs >= 3 points"),
    (lambda p: p.update(grid=-4), "grid must be >= 0"),
])
def test_invalid_problem_is_rejected_before_any_device_work(lib, mutate, needle):
    p = _problem()
    p["params0"] = p["params0"].copy()
    mutate(p)
    arr = lib.ProblemArrays(p)
    h = C.c_void_p()
    opts = lib.make_options(level_res=[128])
    st = lib.load().collage_create(C.byref(arr.struct), 1, C.byref(opts), C.byref(h))
    assert st == -1 and not h.value
    assert needle in lib.load().collage_last_error(None).decode()


@pytest.mark.parametrize("over,needle", [
    (dict(tile=12), "tile must be"),
    (dict(tile=32), "tile must be"),
    (dict(tau=1.0), "tau must be in"),
    (dict(n_levels=0), "n_levels"),
    (dict(rho_px=0.0), "rho_px"),
    (dict(n_dilations=9), "n_dilations"),
    (dict(level_res=[100, 384], n_levels=2), "divisible"),  # 128 * 100 / 384 is not whole
])
def test_invalid_options_are_rejected(lib, over, needle):
    arr = lib.ProblemArrays(_problem())
    kw = dict(level_res=[128])
    kw.update(over)
    opts = lib.make_options(**kw)
    h = C.c_void_p()
    st = lib.load().collage_create(C.byref(arr.struct), 1, C.byref(opts), C.byref(h))
    assert st == -1
    assert needle in lib.load().collage_last_error(None).decode()


def test_null_arguments(lib):
    L = lib.load()
    h = C.c_void_p()
    assert L.collage_create(None, 1, None, C.byref(h)) == -1
    assert L.collage_step(None, None, 1) == -1
    assert L.collage_set_level(None, 0) == -1
    assert L.collage_set_tuning(None, None, None) == -1
    assert L.collage_get_tuning(None, None) == -1
    L.collage_destroy(None)  # no-op
