"""Learned rank proposer (not in the paper): GPU forward / gradient / Adam of
the 24-64-64-13 MLP against the FP64 oracle (oracle/mlp.py), training on the
split records that GPU ps2 runs generate, and what the trained network gains
over ps2 without it (accepted cheap factorisations, unchanged accuracy)."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import mlp
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def test_forward_and_gradient_match_oracle(pkg):
    rng = np.random.default_rng(11)
    theta = pkg.RankProposer.init_params(3).astype(np.float64)
    theta[-13:] = rng.normal(size=13)
    x = rng.normal(size=(37, 24))
    y = rng.integers(0, 13, size=37)
    net = pkg.RankProposer(params=theta.astype(np.float32))
    z_gpu = net.forward(x).cpu().numpy()
    z_ref, _ = mlp.forward(theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(z_gpu - z_ref)) <= 1e-5 * (1 + np.max(np.abs(z_ref)))
    loss, g = net.grad(x, y)
    L_ref, g_ref = mlp.grad(theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64), y)
    assert abs(float(loss.item()) - L_ref) <= 1e-5 * max(1.0, L_ref)
    g = g.cpu().numpy()
    assert np.max(np.abs(g - g_ref)) <= 2e-5 * max(1.0, np.max(np.abs(g_ref)))


def test_adam_step_matches_oracle(pkg):
    rng = np.random.default_rng(12)
    theta = pkg.RankProposer.init_params(4)
    x = rng.normal(size=(16, 24))
    y = rng.integers(0, 13, size=16)
    net = pkg.RankProposer(params=theta)
    t64, m, v = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in range(1, 4):
        _, g_ref = mlp.grad(t64, x.astype(np.float32).astype(np.float64), y)
        t64, m, v = mlp.adam_step(t64, m, v, g_ref, t, 1e-3)
        net.grad(x, y)
        net.adam(1e-3)
    assert np.max(np.abs(net.params.cpu().numpy() - t64)) <= 1e-5


def _ps2(pkg, w, proposer=None, steps=12, cap=16, atol=1e-7):
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                       params={"max_rank": cap, "ps2_atol": atol})
    if proposer is not None:
        g.ttn_set_rank_proposer(proposer)
    g.ttn_stats_reset()
    g.ttn_profile(True)
    t0 = time.perf_counter()
    for _ in range(steps):
        g.ttn_step(w.dt, pkg.TTN_PS2, 1)
    rho = g.ttn_rdm()
    wall = time.perf_counter() - t0
    svd_ms = g.ttn_profile_read(2)
    return g, rho, wall, svd_ms


def test_trained_proposer_gain(pkg):
    """Train on splits logged by GPU ps2 runs of one workload family, then run a
    fresh workload with and without the network: the proposals are accepted for
    most splits (each accepted split replaces the full Jacobi SVD of Theta by a
    sketch of rank r+8), the QR/SVD arithmetic drops (FLOPs counted on the host
    from the launched shapes and the sweeps each Jacobi SVD ran, so the check
    does not depend on timing; the kernel times are printed), and rho_S stays
    within 1e-8 of the run without the network and of the oracle."""
    train_w = [W.spin_boson_tt(depth=6, n_pade=4, rank=2, tree="btt"),
               W.spin_boson_tt(depth=5, n_pade=5, rank=3, tree="btt")]
    feats, labels = [], []
    for w in train_w:
        g, _, _, _ = _ps2(pkg, w, steps=15)
        f, y = g.ttn_split_log()
        feats.append(f)
        labels.append(y)
        g.close()
    feats, labels = np.concatenate(feats), np.concatenate(labels)
    net = pkg.RankProposer(seed=1)
    hist = net.train(feats, labels, steps=400, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    acc = float(np.mean(net.forward(feats).argmax(1).cpu().numpy() == labels))
    assert acc > 0.8

    w = W.spin_boson_tt(depth=6, n_pade=5, rank=2, tree="btt")
    g0, rho0, wall0, svd0 = _ps2(pkg, w, None)
    g1, rho1, wall1, svd1 = _ps2(pkg, w, net)
    proposed, accepted = g1.ttn_proposer_stats()
    o = ottn.from_workload(w, params=ottn.Params(ps2_atol=1e-7, max_rank=16))
    for _ in range(12):
        o.step(w.dt, "ps2")
    _, flops0 = g0.ttn_stats(2)
    _, flops1 = g1.ttn_stats(2)
    print(f"proposed {proposed} accepted {accepted}; QR+SVD GFLOP without {flops0 / 1e9:.3f} with "
          f"{flops1 / 1e9:.3f}; kernel ms without {svd0:.2f} with {svd1:.2f}; "
          f"wall s without {wall0:.3f} with {wall1:.3f}")
    assert accepted >= 0.5 * proposed
    assert flops1 < flops0
    assert np.max(np.abs(rho1 - rho0)) <= 1e-8
    assert np.max(np.abs(rho0 - o.rdm())) <= 1e-10
    assert np.max(np.abs(rho1 - o.rdm())) <= 1e-8
    g0.close()
    g1.close()
