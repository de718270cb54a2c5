"""Checkpoint save / load (Sec. 7.1): a run interrupted by a checkpoint and
resumed in a fresh handle continues bit for bit as the uninterrupted run (ps1
with its captured step graph, ps2 with rank changes, the mixed form), and a
blob from another generator, a corrupted or a truncated blob is refused."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _make(pkg, w, precision=0, params=None):
    return pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, drives=w.drives,
                          precision=precision, params=params)


@pytest.mark.parametrize("case", ["ps1", "ps2", "mixed", "driven"])
def test_resume_from_checkpoint_is_bitwise(pkg, case, tmp_path):
    if case == "ps2":
        w, scheme, params, prec = W.driven_structured_tls(n_pade=1, depth=6, cap=12), pkg.TTN_PS2, \
            {"max_rank": 12, "ps2_atol": 1e-6}, 0
    elif case == "driven":
        w, scheme, params, prec = W.driven_structured_tls(n_pade=1, depth=6, cap=12), pkg.TTN_PS1, None, 0
        w.ranks = W.uniform_ranks(w.parent, 6)
    else:
        w, scheme, params, prec = W.exciton_chain(n_sites=3, depth=5, rank=8), pkg.TTN_PS1, None, \
            (pkg.TTN_MIXED_FP32 if case == "mixed" else 0)
    a = _make(pkg, w, prec, params)
    a.ttn_step(w.dt, scheme, 5)
    path = str(tmp_path / "state.ckpt")
    blob = a.ttn_checkpoint_save(path)
    a.ttn_step(w.dt, scheme, 6)
    ra, ranks_a, ta = a.ttn_rdm(), list(a.ttn_get_ranks()), a.ttn_time()
    b = _make(pkg, w, prec, params)
    b.ttn_checkpoint_load(path)
    assert abs(b.ttn_time() - 5 * w.dt) < 1e-12
    b.ttn_step(w.dt, scheme, 6)
    assert np.array_equal(b.ttn_rdm(), ra)
    assert list(b.ttn_get_ranks()) == ranks_a and b.ttn_time() == ta
    if case == "ps2":
        assert max(ranks_a) > max(w.ranks)  # the ranks had changed before the checkpoint
    # corrupted, truncated and foreign blobs are refused
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(pkg.TTNError) as e:
        b.ttn_checkpoint_load(bytes(bad))
    assert e.value.status == 1
    with pytest.raises(pkg.TTNError):
        b.ttn_checkpoint_load(blob[: len(blob) // 2])
    w2 = W.exciton_chain(n_sites=3, depth=5, rank=8)
    w2.baths[0].dl = (w2.baths[0].dl[0] * 1.01, w2.baths[0].dl[1])
    c = _make(pkg, w2 if case in ("ps1", "mixed") else w, prec, params)
    if case in ("ps1", "mixed"):
        with pytest.raises(pkg.TTNError):
            c.ttn_checkpoint_load(blob)
    for g in (a, b, c):
        g.close()
