"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/grins_racipe.h; topology validation (which runs before any
CUDA call) rejects bad edge lists with GRINS_E_TOPOLOGY."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grins_racipe.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2503_18356_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grins_\w+)\s*\(", text)))


def test_header_declares_the_four_entry_points():
    names = declared_functions()
    for n in ("grins_racipe_create", "grins_racipe_sample_params", "grins_racipe_integrate",
              "grins_racipe_unique_states", "grins_racipe_destroy", "grins_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2503_18356_gb300 import api
    assert sorted(api.EXPORTED) == declared_functions()


def _create(lib, n, src, dst, sign):
    src = np.asarray(src, np.int32); dst = np.asarray(dst, np.int32); sign = np.asarray(sign, np.int8)
    h = C.c_void_p()
    lib.grins_racipe_create.restype = C.c_int32
    st = lib.grins_racipe_create(C.c_int32(n), C.c_int32(src.size), src.ctypes.data_as(C.c_void_p),
                                 dst.ctypes.data_as(C.c_void_p), sign.ctypes.data_as(C.c_void_p),
                                 C.byref(h))
    lib.grins_last_error.restype = C.c_char_p
    return st, lib.grins_last_error().decode()


@pytest.mark.parametrize("case", [
    (0, [], [], []),                    # no nodes
    (65, [], [], []),                   # above the node limit
    (3, [0], [3], [1]),                 # index out of range
    (3, [-1], [0], [1]),
    (3, [0], [1], [0]),                 # sign not +-1
    (3, [0, 0], [1, 1], [1, -1]),       # repeated pair
])
def test_topology_errors_need_no_gpu(lib, case):
    st, msg = _create(lib, *case)
    assert st == 2, msg                  # GRINS_E_TOPOLOGY
    assert msg.startswith("create:")


def test_defaults_follow_table1(lib):
    from paper_2503_18356_gb300 import api
    r = api.default_ranges()
    assert (r.G_min, r.G_max, r.k_min, r.k_max) == (1.0, 100.0, 0.1, 1.0)
    assert (r.lam_act_min, r.lam_act_max, r.lam_inh_min, r.lam_inh_max) == (1.0, 100.0, 0.01, 1.0)
    assert (r.n_min, r.n_max, r.thr_lo, r.thr_hi) == (1, 6, 0.02, 1.98)
    o = api.default_opts()
    assert o.precision == api.GRINS_FP32 and o.polish == 1 and o.t0 == 0.0 and o.t_end == 200.0


def test_binding_structs_match_the_header_sizes(lib):
    # the library asserts sizeof(grins_racipe_ranges) == 168 with no padding
    # (its median cache compares the struct bytewise); the ctypes mirrors
    # must have the same sizes and field order
    from paper_2503_18356_gb300 import api
    assert C.sizeof(api.grins_racipe_ranges) == 168
    assert C.sizeof(api.grins_param_range) == 24 == api.PARAM_RANGE_DTYPE.itemsize
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for cls, name in ((api.grins_racipe_ranges, "grins_racipe_ranges"), (api.grins_param_range, "grins_param_range")):
        body = re.search(r"typedef struct \{([^{}]*?)\} " + name + ";", text, flags=re.S).group(1)
        declared = [n for decl in body.split(";") for n in re.findall(r"(\w+)\s*(?:,|$)", decl.strip())]
        assert [f[0] for f in cls._fields_] == declared, name
