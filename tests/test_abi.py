"""Host-side checks of the C ABI that need no GPU: the library builds and loads, it exports
every function include/lbcg.h declares, and argument validation fails with the documented
status codes before any CUDA call."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_1707_00198_gb300 import build as B
from paper_1707_00198_gb300 import inputs as I
from paper_1707_00198_gb300 import lbcg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbcg.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbcg.library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbcg_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_functions():
    assert set(declared_functions()) == set(lbcg.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_last_error_is_empty_string_initially(lib):
    assert isinstance(lib.lbcg_last_error(), bytes)


def _create_status(geom, prm, precision=1):
    G, P, keep = lbcg._marshal([geom], [prm])
    import ctypes as C
    h = C.c_void_p()
    st = lbcg.library().lbcg_create_batch(1, G, P, precision, None, C.byref(h))
    return st, lbcg.library().lbcg_last_error().decode()


def test_validation_errors_before_any_cuda_call(lib):
    g = I.flat_wall_droplet(20, 10, R=4.0)
    p = I.Params(theta=math.radians(60))
    # closed y without solid edge rows
    bad = I.Geometry(g.nx, g.ny, np.zeros_like(g.solid), g.rhoN0, bc_x="periodic", bc_y="closed")
    st, msg = _create_status(bad, p)
    assert st == 2 and "closed y" in msg
    # contact angle outside (0, pi)
    st, msg = _create_status(g, I.Params(theta=0.0))
    assert st == 3 and "theta" in msg
    # non-positive viscosity
    st, msg = _create_status(g, I.Params(nu_B=0.0))
    assert st == 3
    # colour field outside [-1, 1]
    r = g.rhoN0.copy()
    r[5, 5] = 1.5
    st, msg = _create_status(I.Geometry(g.nx, g.ny, g.solid, r, bc_x="periodic", bc_y="closed"), p)
    assert st == 1 and "rhoN0" in msg
    # all solid
    st, msg = _create_status(I.Geometry(4, 4, np.ones((4, 4), np.uint8), np.zeros((4, 4)), "closed", "closed"), p)
    assert st == 2 and "no fluid" in msg
    # bad precision
    st, msg = _create_status(g, p, precision=9)
    assert st == 1


def test_null_handle_calls_fail_cleanly(lib):
    import ctypes as C
    assert lib.lbcg_step(None, 1) == 1
    assert lib.lbcg_destroy(None) == 0
    assert lib.lbcg_state_bytes(None) == 0


def test_allocator_needs_both_callbacks(lib):
    from paper_1707_00198_gb300 import lbcg
    a = lbcg.lbcg_allocator(lbcg.ALLOC_FN(lambda n, s, c: None), lbcg.RELEASE_FN(), None)
    assert lib.lbcg_set_allocator(C.byref(a)) == 1            # LBCG_E_ARG: no release callback
    assert "alloc and release" in lib.lbcg_last_error().decode()
    assert lib.lbcg_set_allocator(None) == 0


def test_checked_build_compiles_and_exports_every_symbol():
    """The checked build (range checks compiled into the step kernels) builds without a GPU and
    exports the same C ABI."""
    path = B.build(checked=True)
    lib_c = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib_c, name), name
