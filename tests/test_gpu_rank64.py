"""Rank-64 trees (the shape of the precision workload: bonds of dimension 64,
QR matricisations up to 4096 x 64) on the GPU against the FP64 oracle.

* a 3-site chain (depth 4) at requested rank 64: QRs of 1024 x 64 and 576 x 64,
  element-wise RDM parity for a few steps, FP64 (1e-10) and mixed FP32 (1e-6);
* a 4-site chain (depth 4): nodes of 64 x 64 x 64, i.e. the 4096 x 64 QR of the
  7-site rank-64 workload, one step against the oracle;
* the 7-site chain at rank 64 itself (the full precision workload): mixed FP32
  against FP64 on the GPU (the oracle would need minutes per step), plus trace
  and Hermiticity of rho_S to the 1e-6 bar (a truncated TTN conserves neither
  exactly)."""
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


def max_rdm_err(pkg, w, n, precision):
    g = gpu_from(pkg, w, precision=precision)
    o = ottn.from_workload(w)
    assert list(g.ttn_get_ranks()) == o.ranks
    assert max(o.ranks) == 64
    err = 0.0
    for _ in range(n):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    return err


def test_rank64_three_site_chain_fp64(pkg):
    w = W.exciton_chain(n_sites=3, depth=4, rank=64)
    assert max_rdm_err(pkg, w, 3, pkg.TTN_FP64) <= 1e-10


def test_rank64_three_site_chain_mixed(pkg):
    w = W.exciton_chain(n_sites=3, depth=4, rank=64)
    assert max_rdm_err(pkg, w, 3, pkg.TTN_MIXED_FP32) <= 1e-6


def test_rank64_four_site_chain_4096x64_qr(pkg):
    w = W.exciton_chain(n_sites=4, depth=4, rank=64)
    o = ottn.from_workload(w)
    assert any(T.shape == (64, 64, 64) for T in o.tensors)
    assert max_rdm_err(pkg, w, 1, pkg.TTN_FP64) <= 1e-10


def test_rank64_seven_site_chain_mixed_vs_fp64(pkg):
    w = W.exciton_chain(rank=64)
    ga = gpu_from(pkg, w)
    gb = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    assert max(ga.ttn_get_ranks()) == 64
    rho0 = ga.ttn_rdm()
    err = 0.0
    for _ in range(2):
        ga.ttn_step(w.dt, pkg.TTN_PS1, 1)
        gb.ttn_step(w.dt, pkg.TTN_PS1, 1)
        ra, rb = ga.ttn_rdm(), gb.ttn_rdm()
        err = max(err, float(np.max(np.abs(ra - rb))))
        assert np.all(np.isfinite(rb))
        # truncated TTN: trace and Hermiticity are held to the accuracy bar, not to roundoff
        assert abs(np.trace(ra) - np.trace(rho0)) <= 1e-6
        assert np.max(np.abs(ra - ra.conj().T)) <= 1e-6
    ga.close()
    gb.close()
    assert err <= 1e-6


def test_rank64_tensor_cores_match_cuda_cores(pkg):
    """The mixed form with its large mode products on the tcgen05 tensor cores
    (3xTF32) against the same form on the FP32 CUDA cores and the oracle. The
    bulk-copy ring (pre-split tensor operand, tensor_cores = 2) and the
    thread-staged kernel (tensor_cores = 1) feed the MMAs the same operands in
    the same order, so their results are identical bit for bit."""
    w = W.exciton_chain(n_sites=3, depth=4, rank=64)
    ga = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    ga.ttn_set_params(tensor_cores=2)
    gs = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    gb = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    gb.ttn_set_params(tensor_cores=0)
    for g in (ga, gs, gb):  # the environment build at bind ran with the default form
        g.ttn_stats_reset()
    o = ottn.from_workload(w)
    e_tc = e_ref = diff = 0.0
    for _ in range(3):
        ga.ttn_step(w.dt, pkg.TTN_PS1, 1)
        gs.ttn_step(w.dt, pkg.TTN_PS1, 1)
        gb.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        ra, rs, rb, ro = ga.ttn_rdm(), gs.ttn_rdm(), gb.ttn_rdm(), o.rdm()
        assert np.array_equal(ra, rs)
        e_tc = max(e_tc, float(np.max(np.abs(ra - ro))))
        e_ref = max(e_ref, float(np.max(np.abs(rb - ro))))
        diff = max(diff, float(np.max(np.abs(ra - rb))))
    for u in range(len(w.parent)):
        assert np.array_equal(ga.ttn_get_node(u), gs.ttn_get_node(u)), u
    assert ga.ttn_stats(4)[0] > 0 and gs.ttn_stats(4)[0] == 0  # the ring path ran (and only where asked)
    ga.close()
    gs.close()
    gb.close()
    assert e_tc <= 1e-6 and e_ref <= 1e-6
    assert diff <= 1e-6


def test_rank64_generic_state_node_tensors_4096x64_qr(pkg):
    """A generic full-rank tree (random semi-unitary cores, random root) on the
    4-site rank-64 chain: after one ps1 step every node tensor -- i.e. the Q
    factors of the 4096 x 64 blocked QRs (panels over the whole GPU) and of the
    cluster QRs, with their phase convention -- matches the oracle element by
    element, not only the gauge-invariant rho_S."""
    w = W.exciton_chain(n_sites=4, depth=4, rank=64)
    o = ottn.from_workload(w)
    assert any(T.shape == (64, 64, 64) for T in o.tensors)
    rng = np.random.default_rng(64)
    tensors = []
    for u, T in enumerate(o.tensors):
        X = rng.normal(size=T.shape) + 1j * rng.normal(size=T.shape)
        if u == 0:
            X /= np.linalg.norm(X)
        else:  # semi-unitary toward the parent (leg 0)
            M = np.moveaxis(X, 0, -1)
            sh = M.shape
            Q, _ = np.linalg.qr(M.reshape(-1, sh[-1]))
            X = np.moveaxis(Q.reshape(sh), -1, 0)
        tensors.append(X)
    o.tensors = [t.copy() for t in tensors]
    for c in o.tree.postorder():
        if c:
            o.update_env(c, o.tree.parent[c])
    g = gpu_from(pkg, w)
    for u, t in enumerate(tensors):
        g.ttn_set_node(u, t)
    g.ttn_step(w.dt, pkg.TTN_PS1, 1)
    o.step(w.dt, "ps1")
    errs = [float(np.max(np.abs(g.ttn_get_node(u) - o.tensors[u]))) for u in range(len(w.parent))]
    rdm_err = float(np.max(np.abs(g.ttn_rdm() - o.rdm())))
    g.close()
    assert max(errs) < 1e-10, errs
    assert rdm_err < 1e-10
