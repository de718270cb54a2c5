"""The C-ABI library (include/ttn_heom.h) loads, exports every declared entry
point, and its host-only entry points (validation, rank caps, substep rule)
agree with the oracle. No GPU work is issued here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import sop as osop
from oracle import ttn as ottn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_17711_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ttn_heom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ttn_status|const char\*|void)\s+(\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2603_17711_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 20
    bound = {n for n, _, _ in _lib.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n
        assert n in bound, f"{n} declared in the header but not bound in the Python layer"


def _create(lib, w, ranks=None, precision=0):
    from paper_2603_17711_gb300 import _lib
    par, ln = _lib.as_i32(w.parent), _lib.as_i32(w.leg_node)
    tree = _lib.ttn_tree(len(par), _lib.ptr(par, C.c_int32), len(ln), _lib.ptr(ln, C.c_int32))
    h = C.c_void_p()
    st = lib.ttn_create(C.byref(tree), _lib.ptr(_lib.as_i32(w.leg_dims), C.c_int32),
                        _lib.ptr(_lib.as_i32(ranks if ranks is not None else w.ranks), C.c_int32), precision, C.byref(h))
    return st, h


def _load(lib, h, a):
    from paper_2603_17711_gb300 import _lib
    return lib.sop_load(h, len(a["op_leg"]), _lib.ptr(a["op_leg"], C.c_int32), _lib.ptr(a["op_offset"], C.c_int64),
                        _lib.ptr(a["op_data"], C.c_double), len(a["term_offsets"]) - 1,
                        _lib.ptr(a["term_offsets"], C.c_int32), _lib.ptr(a["term_ops"], C.c_int32),
                        _lib.ptr(a["coef"], C.c_double), _lib.ptr(a["coef_drive"], C.c_int32))


@pytest.mark.parametrize("make", [lambda: W.spin_boson_tt(), lambda: W.exciton_chain(n_steps=1),
                                  lambda: W.spin_boson_tt(depth=6, n_pade=5, rank=7, tree="btt")])
def test_rank_caps_and_substeps_match_oracle(lib, make):
    from paper_2603_17711_gb300 import _lib, heom
    w = make()
    st, h = _create(lib, w)
    assert st == 0
    assert _load(lib, h, heom.heom_sop(w.H, w.baths, w.depth)) == 0
    r = np.zeros(len(w.parent), np.int32)
    assert lib.ttn_get_ranks(h, _lib.ptr(r, C.c_int32)) == 0
    o = ottn.from_workload(w)
    assert list(r) == o.ranks
    for tau in (w.dt / 2, w.dt, 3.7 * w.dt):
        m = C.c_int32()
        assert lib.ttn_substeps(h, tau, C.byref(m)) == 0
        assert m.value == o.m_sub(tau)
    n = C.c_size_t()
    assert lib.ttn_workspace_size(h, C.byref(n)) == 0 and n.value > 0
    # stepping before a workspace is bound is an ordering error, not a crash
    assert lib.ttn_step(h, w.dt, 1, 1) == 6
    lib.ttn_destroy(h)


def test_params_round_trip_and_range_checks(lib):
    from paper_2603_17711_gb300 import _lib, heom
    w = W.spin_boson_tt()
    st, h = _create(lib, w)
    assert st == 0
    p = _lib.ttn_params()
    assert lib.ttn_get_params(h, C.byref(p)) == 0
    assert (p.qr_tol, p.kappa, p.max_rank, p.max_split, p.tensor_cores) == (1e-9, 2.5, 32, 16, 1)
    for field, bad in (("max_split", 0), ("max_split", 17), ("kappa", 0.0), ("ps2_ratio", 0.5), ("max_rank", 0),
                       ("tensor_cores", 3), ("tensor_cores", -1), ("wait_s", -1.0), ("wait_s", 61.0),
                       ("tile_warps", 3), ("tile_warps", 16), ("tile_warps", -1)):
        q = _lib.ttn_params()
        C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
        setattr(q, field, bad)
        assert lib.ttn_set_params(h, C.byref(q)) == 1, field  # TTN_EINVAL
    p.max_split = 1
    assert lib.ttn_set_params(h, C.byref(p)) == 0
    assert _load(lib, h, heom.heom_sop(w.H, w.baths, w.depth)) == 0
    q = _lib.ttn_params()
    assert lib.ttn_get_params(h, C.byref(q)) == 0 and q.max_split == 1
    lib.ttn_destroy(h)


def _tuning_rows(lib, h):
    from paper_2603_17711_gb300 import _lib
    n = C.c_int32()
    assert lib.ttn_tuning_get(h, None, 0, C.byref(n)) == 0
    rows = np.zeros((n.value, _lib.TTN_TUNING_COLS), np.int32)
    assert lib.ttn_tuning_get(h, rows.ctypes.data_as(C.POINTER(C.c_int32)), n.value, C.byref(n)) == 0
    return rows


def test_tile_shapes_rows_round_trip(lib):
    """Tile-shape rows (the autotuner's cache format): the planned shapes,
    tile_warps forcing the warps of every contraction list, rows applied by
    key, and out-of-range rows refused before anything is set."""
    from paper_2603_17711_gb300 import _lib, heom
    w = W.exciton_chain(n_sites=3, rank=6, depth=4)
    st, h = _create(lib, w)
    assert st == 0
    n = C.c_int32()
    assert lib.ttn_tuning_get(h, None, 0, C.byref(n)) == 6  # TTN_ESTATE before sop_load
    assert _load(lib, h, heom.heom_sop(w.H, w.baths, w.depth)) == 0
    rows = _tuning_rows(lib, h)
    assert len(rows) > 0 and set(rows[:, 0]) == {0, 1}
    assert np.all(rows[:, 9] == 8) and np.all(rows[:, 10] >= 1) and np.all(rows[:, 10] <= 16)
    ap = rows[:, 0] == 0
    assert np.all(rows[ap, 7] > 0) and np.all(rows[~ap, 7] == 0)  # terms of contractions; none for projections
    # tile_warps = 2 gives every contraction list two warps per CTA
    p = _lib.ttn_params()
    assert lib.ttn_get_params(h, C.byref(p)) == 0
    p.tile_warps = 2
    assert lib.ttn_set_params(h, C.byref(p)) == 0
    r2 = _tuning_rows(lib, h)
    assert np.all(r2[ap, 9] == 2) and np.all(r2[~ap, 9] == 8)
    assert np.array_equal(r2[:, :9], rows[:, :9])
    # rows applied by key: every list matches its own row
    want = rows.copy()
    want[ap, 9] = 4
    want[:, 10] = 1
    applied = C.c_int32()
    assert lib.ttn_tuning_set(h, want.ctypes.data_as(C.POINTER(C.c_int32)), len(want), C.byref(applied)) == 0
    assert applied.value == len(want)
    assert np.array_equal(_tuning_rows(lib, h), want)
    # a row with an unknown key sets nothing; a bad shape is refused and nothing changes
    other = want[:1].copy()
    other[0, 8] += 1000
    other[0, 9] = 2
    assert lib.ttn_tuning_set(h, other.ctypes.data_as(C.POINTER(C.c_int32)), 1, C.byref(applied)) == 0
    assert applied.value == 0
    for col, bad in ((9, 3), (9, 16), (10, 0), (10, 17)):
        b = want.copy()
        b[-1, col] = bad
        assert lib.ttn_tuning_set(h, b.ctypes.data_as(C.POINTER(C.c_int32)), len(b), C.byref(applied)) == 1
    b = want.copy()
    b[~ap, 9] = 4  # projections keep 8 warps
    if (~ap).any():
        assert lib.ttn_tuning_set(h, b.ctypes.data_as(C.POINTER(C.c_int32)), len(b), C.byref(applied)) == 1
    assert np.array_equal(_tuning_rows(lib, h), want)
    lib.ttn_destroy(h)


def test_invalid_trees_and_operators_are_rejected(lib):
    from paper_2603_17711_gb300 import heom
    w = W.spin_boson_tt(depth=4, n_pade=2)
    bad = W.spin_boson_tt(depth=4, n_pade=2)
    bad.parent = [-1, 2, 1]  # cycle
    assert _create(lib, bad)[0] == 1
    bad = W.spin_boson_tt(depth=4, n_pade=2)
    bad.leg_node = [1, 0, 1, 2, 2]  # system leg off the root
    assert _create(lib, bad)[0] == 1
    assert _create(lib, w, ranks=[0, 0, 3])[0] == 1  # rank < 1
    st, h = _create(lib, w)
    assert st == 0
    a = heom.heom_sop(w.H, w.baths, w.depth)
    a_bad = dict(a)
    a_bad["op_leg"] = a["op_leg"].copy()
    a_bad["op_leg"][0] = 99
    assert _load(lib, h, a_bad) == 1
    a_bad = dict(a)
    a_bad["op_data"] = a["op_data"].copy()
    a_bad["op_data"][3] = np.nan
    assert _load(lib, h, a_bad) == 1
    a_bad = dict(a)
    a_bad["coef_drive"] = a["coef_drive"].copy()
    a_bad["coef_drive"][-1] = 0  # a driven bath term off the root
    assert _load(lib, h, a_bad) == 7
    assert _load(lib, h, a) == 0
    assert lib.ttn_step(h, 0.01, 3, 1) == 6  # no workspace yet
    lib.ttn_destroy(h)


def test_four_leg_nodes_are_unsupported(lib):
    # root with i, j and two child subtrees has four legs
    parent = [-1, 0, 0]
    leg_node = [0, 0, 1, 1, 2, 2]
    w = W.spin_boson_tt(depth=3, n_pade=3)
    w.parent, w.leg_node = parent, leg_node
    w.ranks = [0, 4, 4]
    assert _create(lib, w)[0] == 7


def test_product_sop_equals_oracle_sop():
    # the product's host model builder and the oracle build the same generator
    from paper_2603_17711_gb300 import heom
    from oracle import dense
    rng = np.random.default_rng(4)
    H = W.random_hermitian(rng, 3)
    baths = [W.Bath(Q=np.diag([1.0, 0, -1]).astype(complex), beta=0.9, dl=(0.3, 1.1), n_ltc=2),
             W.Bath(Q=W.random_hermitian(rng, 3), beta=2.0, bo=[(0.1, 1.2, 0.3)], n_ltc=1)]
    depth = [3, 2, 3, 2, 3, 2]
    drives = [W.Drive(V=W.random_hermitian(rng, 3), amp=0.3, omega=2.0)]
    a = heom.heom_sop(H, baths, depth, drives)
    dims = [3, 3] + depth
    ops = []
    for k in range(len(a["op_leg"])):
        d = dims[a["op_leg"][k]]
        o = a["op_offset"][k]
        v = a["op_data"][2 * o:2 * (o + d * d)]
        ops.append((v[0::2] + 1j * v[1::2]).reshape(d, d))
    terms = []
    for m in range(len(a["term_offsets"]) - 1):
        ids = a["term_ops"][a["term_offsets"][m]:a["term_offsets"][m + 1]]
        c = a["coef"][2 * m] + 1j * a["coef"][2 * m + 1]
        dr = int(a["coef_drive"][m])
        terms.append(osop.Term(c, {int(a["op_leg"][i]): ops[i] for i in ids}, None if dr < 0 else dr))
    ref = osop.heom_terms(H, baths, depth, drives=drives)
    for g in (0.0, 0.37):
        L1 = dense.generator(terms, dims, [g])
        L2 = dense.generator(ref, dims, [g])
        assert abs(L1 - L2).max() < 1e-13
