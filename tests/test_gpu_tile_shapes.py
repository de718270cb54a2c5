"""Tile shapes of the contraction launches (warps per CTA x CTAs per tile):
every shape gives the oracle's result to rounding, the autotuner's JSON cache
reproduces a tuning exactly, and the batch tuner leaves the instances where
they were."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def gpu_from(pkg, w, **kw):
    return pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                          drives=w.drives, **kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_every_warp_count_matches_the_oracle(pkg, precision):
    """tile_warps 2, 4 and 8 (with the planned splits) against the FP64 oracle
    on a 3-site chain: 1e-10 in FP64, 1e-6 in the mixed form."""
    w = W.exciton_chain(n_sites=3, rank=6, depth=4)
    o = ottn.from_workload(w)
    for _ in range(4):
        o.step(w.dt, "ps1")
    ref = o.rdm()
    tol = 1e-10 if precision == 0 else 1e-6
    out = {}
    for tw in (8, 4, 2):
        g = gpu_from(pkg, w, precision=precision)
        g.ttn_set_params(tile_warps=tw)
        rows = g.ttn_tuning_get()
        assert np.all(rows[rows[:, 0] == 0, 9] == tw)
        g.ttn_step(w.dt, 1, 4)
        out[tw] = g.ttn_rdm()
        g.close()
        assert np.max(np.abs(out[tw] - ref)) <= tol, tw


def test_autotune_cache_reproduces_the_tuning(pkg, tmp_path):
    """A tuning written to the JSON cache is read back by a second handle of
    the same model without timing anything: the same rows, and the same
    trajectory bit for bit."""
    w = W.exciton_chain(n_sites=4, rank=8, depth=4)
    path = str(tmp_path / "shapes.json")
    g1 = gpu_from(pkg, w)
    assert g1.ttn_autotune(2, cache=path) == "tuned"
    doc = json.load(open(path))
    assert doc["rows"] and len(doc["columns"]) == 11
    g2 = gpu_from(pkg, w)
    assert g2.ttn_autotune(2, cache=path) == "cache"
    assert np.array_equal(g1.ttn_tuning_get(), g2.ttn_tuning_get())
    g1.ttn_step(w.dt, 1, 3)
    g2.ttn_step(w.dt, 1, 3)
    assert np.array_equal(g1.ttn_rdm(), g2.ttn_rdm())
    # a different model adds its own rows and keeps the first model's
    w3 = W.exciton_chain(n_sites=3, rank=6, depth=4)
    g3 = gpu_from(pkg, w3)
    assert g3.ttn_autotune(2, cache=path) == "tuned"
    keys = {tuple(r[:9]) for r in json.load(open(path))["rows"]}
    assert {tuple(r[:9]) for r in g1.ttn_tuning_get().tolist()} <= keys
    for g in (g1, g2, g3):
        g.close()


def test_batch_autotune_puts_the_states_back(pkg):
    """ttn_batch_autotune times the batch with 8, 4 and 2 warps per CTA and
    restores every member: afterwards the batch continues exactly like
    handles that were never tuned but carry the chosen shape."""
    ws = W.spin_boson_batch(n=6)
    hs = [gpu_from(pkg, bw) for bw in ws]
    for h in hs:
        h.ttn_set_params(max_split=1)
    t0 = [h.ttn_time() for h in hs]
    r0 = [h.ttn_rdm() for h in hs]
    s0 = [[h.ttn_stats(k) for k in range(4)] for h in hs]
    res = pkg.ttn_batch_autotune(hs, 0.01, 1)
    assert res["warps"] in (8, 4, 2) and all(v > 0 for v in res["ms_per_batched_step"].values())
    assert [h.ttn_time() for h in hs] == t0
    assert [[h.ttn_stats(k) for k in range(4)] for h in hs] == s0  # counters put back too
    for a, h in zip(r0, hs):
        assert np.array_equal(h.ttn_rdm(), a)
    fresh = [gpu_from(pkg, bw) for bw in ws]
    for h in fresh:
        h.ttn_set_params(max_split=1, tile_warps=res["warps"])
    pkg.ttn_batch_step(hs, 0.01, 1, 3)
    pkg.ttn_batch_step(fresh, 0.01, 1, 3)
    for a, b in zip(hs, fresh):
        assert np.array_equal(a.ttn_rdm(), b.ttn_rdm())
    for h in hs + fresh:
        h.close()
