"""CPU checks of the C ABI: the library loads, exports every function that
include/nbody.h declares, and rejects bad arguments on the host before it
touches a device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbody.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nbody_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_02655_gb300 import build
    path = build.build()
    import paper_2511_02655_gb300 as nbody
    assert nbody.lib_path() == path
    return nbody.load()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("nbody_init", "nbody_forces", "nbody_step", "nbody_energy", "nbody_adjoint"):
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f
    assert lib.nbody_version() >> 16 == 1


def test_status_codes_and_constants_match_header():
    import paper_2511_02655_gb300 as nbody
    text = open(HEADER).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"NBODY_(E[A-Z]+|OK)\s*=\s*(\d+)", text))
    assert {nbody.STATUS[v]: v for v in nbody.STATUS} == codes
    assert int(re.search(r"NBODY_MIXED\s*=\s*(\d)", text).group(1)) == nbody.MIXED
    assert int(re.search(r"NBODY_FLAG_GRAPH\s+(\d+)u", text).group(1)) == nbody.FLAG_GRAPH
    assert ctypes.sizeof(nbody._Config) == 3 * 8 + 10 * 4 + 3 * 8


def _cfg(**kw):
    import paper_2511_02655_gb300 as nbody
    c = nbody._Config(1.0, 0.01, 1e-3, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1.0, 1.0, 0.0)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(eps=-1.0), dict(precision=7), dict(block=96), dict(i_per_thread=3),
                                 dict(j_tile=100), dict(energy_every=-1), dict(flags=64), dict(G=float("nan")),
                                 dict(variant=4), dict(variant=2, precision=0), dict(variant=3, precision=0),
                                 dict(law=2), dict(reserved=1), dict(box=-1.0), dict(law=1, lj_sigma=0.0),
                                 dict(law=1, variant=1)])
def test_init_rejects_bad_config_before_touching_a_device(lib, bad):
    h = ctypes.c_void_p(123)
    offs = (ctypes.c_int64 * 2)(0, 16)
    cfg = _cfg(**bad)
    st = lib.nbody_init(ctypes.byref(h), ctypes.byref(cfg), 1, offs, None)
    assert st == 1 and h.value is None
    assert "config" in lib.nbody_last_error(None).decode()


@pytest.mark.parametrize("offsets,nsys", [((1, 5), 1), ((0, 5, 3), 2), ((0, 1 << 29), 1)])
def test_init_rejects_bad_layouts(lib, offsets, nsys):
    h = ctypes.c_void_p()
    offs = (ctypes.c_int64 * len(offsets))(*offsets)
    cfg = _cfg()
    assert lib.nbody_init(ctypes.byref(h), ctypes.byref(cfg), nsys, offs, None) == 1
    assert h.value is None


def test_calls_with_null_context_are_rejected(lib):
    assert lib.nbody_forces(None, None, None, None, None) == 1
    assert lib.nbody_step(None, None, None, None, None, 0, 1, None) == 1
    assert lib.nbody_energy(None, None, None, None, None) == 1
    assert lib.nbody_adjoint(None, None, None, None, 1, 1, None, None, None, None, None) == 1
    assert lib.nbody_adjoint_params(None, None, None, None, 1, 1, None, None, None, None, None, None) == 1
    assert lib.nbody_sync(None) == 1
    assert lib.nbody_launch_count(None) == 0
    lib.nbody_destroy(None)
