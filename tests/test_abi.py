"""Host-side checks of the C ABI (no GPU work): the library builds for
sm_103a, loads, exports every function declared in include/*.h, and rejects
bad arguments before touching the device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import paper_1710_08124_gb300 as ep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    ep.build()
    return ep.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(epll_\w+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "epll_restore" in names and "epll_gmm_load" in names
    for n in names:
        assert hasattr(L, n), n


def test_gmm_load_validation(L):
    g = C.c_void_p()
    w = np.ones(2)
    U = np.tile(np.eye(64), (2, 1, 1))
    S = np.tile(np.linspace(1, 0.1, 64), (2, 1))
    assert L.epll_gmm_load(0, 64, w.ctypes.data, U.ctypes.data, S.ctypes.data, 0, 8.0, C.byref(g)) == ep.EINVAL
    assert L.epll_gmm_load(2, 49, w.ctypes.data, U.ctypes.data, S.ctypes.data, 0, 8.0, C.byref(g)) == ep.EINVAL
    assert L.epll_gmm_load(2, 64, w.ctypes.data, U.ctypes.data, S.ctypes.data, 0, 65.0, C.byref(g)) == ep.EINVAL
    assert L.epll_gmm_load(2, 64, w.ctypes.data, U.ctypes.data, S.ctypes.data, 1, 1.5, C.byref(g)) == ep.EINVAL
    bad = S.copy()
    bad[1, 3] = 2.0  # not non-increasing
    assert L.epll_gmm_load(2, 64, w.ctypes.data, U.ctypes.data, bad.ctypes.data, 0, 8.0, C.byref(g)) == ep.EINVAL
    assert "non-increasing" in ep.last_error()
    w2 = np.array([1.0, -1.0])
    assert L.epll_gmm_load(2, 64, w2.ctypes.data, U.ctypes.data, S.ctypes.data, 0, 8.0, C.byref(g)) == ep.EINVAL
    assert L.epll_gmm_load(2, 64, None, U.ctypes.data, S.ctypes.data, 0, 8.0, C.byref(g)) == ep.EINVAL
    assert not g.value


def test_restore_rejects_null_handle(L):
    bm = np.array(ep.PAPER_BETA)
    st = L.epll_restore(None, None, 64, 64, None, C.c_float(0.1), bm.ctypes.data, 5, None, None, None)
    assert st == ep.EINVAL


def test_options_default(L):
    o = ep._Options()
    L.epll_options_default(C.byref(o))
    assert o.precision == ep.FP32 and o.subset == ep.SUBSET_ALL and o.cg_iters == 100 and o.tie_gap < 0
    assert o.select == ep.SELECT_EXHAUSTIVE


def test_proposal_layout_and_validation(L):
    from oracle import mlp
    for K in (2, 20, 200, 256):
        assert L.epll_proposal_size(K) == mlp.n_params(K)
    assert L.epll_proposal_size(0) == 0
    h = C.c_void_p()
    assert L.epll_proposal_create(1, 0, C.byref(h)) == ep.EINVAL and not h.value
    assert L.epll_proposal_create(257, 0, C.byref(h)) == ep.EINVAL and not h.value
    assert L.epll_proposal_create(4, 0, None) == ep.EINVAL
    assert L.epll_gmm_attach_proposal(None, None, 4, C.c_float(0.0)) == ep.EINVAL
    assert L.epll_proposal_topm(None, None, 64, 64, None, 0, 1.0, None, None, None) == ep.EINVAL
    assert L.epll_proposal_grad(None, None, 1, 64, 64, None, None, None, None, None, 10, 10, None, None,
                                None) == ep.EINVAL
    assert L.epll_proposal_train(None, None, 1, 64, 64, None, None, None, None, None, 10, 10, C.c_float(1e-3),
                                 C.c_float(0.0), None, None) == ep.EINVAL
    assert L.epll_proposal_get(None, None) == ep.EINVAL
    L.epll_proposal_free(None)


def test_attach_tree_rejects_null_handle(L):
    assert L.epll_gmm_attach_tree(None, 0, None, None, None, None, None) == ep.EINVAL


def test_tile_setters_reject_null_handle(L):
    assert L.epll_set_tiles(None, 256, 1) == ep.EINVAL
    assert L.epll_set_cta_pairs(None, 1) == ep.EINVAL


def test_header_enums_match_binding():
    """Every EPLL_* enum constant of include/epll.h has the value the Python
    binding passes for it (precision forms including EPLL_AUTO, selection
    variants, rank rules, degradations, samplers, status codes)."""
    src = open(os.path.join(ROOT, "include", "epll.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for name, v in re.findall(r"\bEPLL_(\w+)\s*=\s*(-?\d+)", body):
            vals[name] = int(v)
    assert vals["AUTO"] == 5 and vals["BF16X3"] == 3
    for name, v in vals.items():
        py = getattr(ep, name, None)
        assert py is not None, name
        assert py == v, (name, py, v)
