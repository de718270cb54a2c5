"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs. Tolerance: RDM max-abs <= 1e-6 for the FP64 path (the
stated bar); short runs are held to 1e-10 since both sides run the same
algorithm in FP64 and differ only by rounding order."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_SHORT = 1e-10
TOL_FP64 = 1e-6
TOL_MIXED = 1e-6  # the accuracy bar of the mixed form on rho_S (max-abs)


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


def run_both(pkg, w, n, scheme="ps1", oracle_setup=None, gpu_setup=None):
    g = gpu_from(pkg, w)
    o = ottn.from_workload(w)
    if oracle_setup:
        oracle_setup(o)
    if gpu_setup:
        gpu_setup(g)
    assert list(g.ttn_get_ranks()) == o.ranks
    err = float(np.max(np.abs(g.ttn_rdm() - o.rdm())))
    code = pkg.TTN_PS1 if scheme == "ps1" else pkg.TTN_PS2
    for _ in range(n):
        g.ttn_step(w.dt, code, 1)
        o.step(w.dt, scheme)
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    return err, g, o


@pytest.mark.parametrize("tree", ["tt", "btt"])
def test_spin_boson_small(pkg, tree):
    w = W.spin_boson_tt(depth=6, n_pade=3, rank=6, tree=tree)
    err, g, _ = run_both(pkg, w, 15)
    g.close()
    assert err <= TOL_SHORT


def test_untruncated_ranks(pkg):
    w = W.spin_boson_tt(depth=4, n_pade=2, rank=1000)
    err, g, _ = run_both(pkg, w, 20)
    g.close()
    assert err <= TOL_SHORT


def test_multibath_exciton_chain_small(pkg):
    w = W.exciton_chain(n_sites=3, rank=7, depth=4, n_steps=8)
    err, g, _ = run_both(pkg, w, 8)
    g.close()
    assert err <= TOL_SHORT


def test_driven_two_level_system(pkg):
    w = W.spin_boson_tt(depth=5, n_pade=2, rank=5, tree="btt")
    w.drives = [W.Drive(V=W.SIGMA_X, amp=0.5, omega=3.0)]
    err, g, _ = run_both(pkg, w, 12)
    g.close()
    assert err <= TOL_SHORT


def test_structured_bath_brownian_features(pkg):
    w = W.driven_structured_tls(n_pade=2, depth=4)
    w.scheme = "ps1"
    w.ranks = W.uniform_ranks(w.parent, 6)
    err, g, _ = run_both(pkg, w, 6)
    g.close()
    assert err <= TOL_SHORT


@pytest.mark.parametrize("K,tree,rank", [(1, "tt", 3), (2, "tt", 1), (2, "btt", 2), (5, "btt", 1)])
def test_edge_shapes(pkg, K, tree, rank):
    # K = 1: a single root node with no bonds; rank 1 bonds; odd binary splits
    w = W.spin_boson_tt(depth=3, n_pade=K - 1, rank=rank, tree=tree)
    err, g, _ = run_both(pkg, w, 6)
    g.close()
    assert err <= TOL_SHORT


def test_depth_one_legs_and_random_rho0(pkg):
    rng = np.random.default_rng(21)
    w = W.spin_boson_tt(depth=1, n_pade=2, rank=2)
    w.rho0 = W.random_density_matrix(rng, 2)
    err, g, _ = run_both(pkg, w, 5)
    g.close()
    assert err <= TOL_SHORT


def test_generic_state_via_set_node(pkg):
    # start both sides from the same generic TTN (HTD of a random EDO) to
    # exercise every kernel away from the sparse product state
    w = W.spin_boson_tt(depth=4, n_pade=3, rank=5, tree="btt")
    rng = np.random.default_rng(5)
    o = ottn.from_workload(w)
    full = rng.normal(size=w.leg_dims) + 1j * rng.normal(size=w.leg_dims)
    tensors = ottn.htd_tensors(o.tree, o.leg_dims, o.ranks, full)

    def setup_oracle(st):
        st.tensors = [t.copy() for t in tensors]
        for c in st.tree.postorder():
            if c:
                st.update_env(c, st.tree.parent[c])

    def setup_gpu(g):
        for u, t in enumerate(tensors):
            g.ttn_set_node(u, t)

    err, g, o = run_both(pkg, w, 5, oracle_setup=setup_oracle, gpu_setup=setup_gpu)
    for u in range(len(w.parent)):
        assert np.max(np.abs(g.ttn_get_node(u) - o.tensors[u])) < 1e-10
    g.close()
    assert err <= TOL_SHORT * 10


def test_spin_boson_tt_1000_steps_against_stored_oracle(pkg):
    """Full spin-boson tensor-train workload (K=4, depth 10, rank 10, dt 0.01,
    1000 steps) against the oracle trajectory stored by tests/golden/make_golden.py."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "spin_boson_tt_k4_n10_r10.txt"))
    steps = rows[:, 0].astype(int)
    ref = (rows[:, 1::2] + 1j * rows[:, 2::2]).reshape(-1, 2, 2)
    w = W.spin_boson_tt(n_steps=1000)
    g = gpu_from(pkg, w)
    err, n = 0.0, 0
    for k, s in enumerate(steps):
        if s > n:
            g.ttn_step(w.dt, pkg.TTN_PS1, int(s - n))
            n = int(s)
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - ref[k]))))
    g.close()
    assert err <= TOL_FP64
    assert err <= 1e-9  # observed far below the bar; flag drifts early


def test_exciton_chain_full_size_first_steps(pkg):
    """The 7-site chain at full size (21 features, depth 8, rank 20, 21 nodes):
    the oracle is slow there, so two steps are compared element by element."""
    w = W.exciton_chain(n_steps=2)
    err, g, _ = run_both(pkg, w, 2)
    g.close()
    assert err <= TOL_SHORT


def test_concurrent_handles_match_oracle(pkg):
    """Handles on their own streams run concurrently; each must still match the
    oracle (guards against cross-CTA read/write hazards that only show under load)."""
    ws = W.spin_boson_batch(n=6, n_steps=6)
    gs = [gpu_from(pkg, w) for w in ws]
    for g, w in zip(gs, ws):
        g.ttn_step(w.dt, pkg.TTN_PS1, 6)
    for g, w in zip(gs, ws):
        o = ottn.from_workload(w)
        for _ in range(6):
            o.step(w.dt, "ps1")
        assert np.max(np.abs(g.ttn_rdm() - o.rdm())) <= TOL_SHORT
        g.close()


def test_bitwise_deterministic(pkg):
    w = W.spin_boson_tt(depth=6, n_pade=3, rank=6, tree="btt")
    outs = []
    for _ in range(2):
        g = gpu_from(pkg, w)
        g.ttn_step(w.dt, pkg.TTN_PS1, 10)
        outs.append(g.ttn_rdm())
        g.close()
    assert np.array_equal(outs[0], outs[1])


def test_overflow_is_reported_as_numeric_error(pkg):
    w = W.spin_boson_tt(depth=3, n_pade=1, rank=2)
    w.rho0 = np.array([[1e308, 0], [0, 0]], complex)  # finite, but the first RK4 stage overflows
    g = gpu_from(pkg, w)
    g.ttn_step(w.dt, pkg.TTN_PS1, 1)
    with pytest.raises(pkg.TTNError) as e:
        g.ttn_rdm()
    assert e.value.status == 4  # TTN_ENUMERIC
    g.close()


def test_vmf_in_the_mixed_form_is_unsupported(pkg):
    w = W.spin_boson_tt(depth=3, n_pade=1, rank=2)
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                       precision=pkg.TTN_MIXED_FP32)
    with pytest.raises(pkg.TTNError) as e:
        g.ttn_step(w.dt, pkg.TTN_VMF, 1)
    assert e.value.status == 7
    g.close()


# ---------------------------------------------------------------------------
# Mixed-precision form: node/bond/environment contractions in FP32 on FP32
# shadows, state + RK4 accumulation + QR + absorb + RDM in FP64. Bar: RDM
# max-abs <= 1e-6 against the FP64 oracle.
# ---------------------------------------------------------------------------
def gpu_mixed(pkg, w):
    return pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                          drives=w.drives, precision=pkg.TTN_MIXED_FP32)


def test_mixed_spin_boson_tt_1000_steps(pkg):
    rows = np.loadtxt(os.path.join(HERE, "golden", "spin_boson_tt_k4_n10_r10.txt"))
    steps = rows[:, 0].astype(int)
    ref = (rows[:, 1::2] + 1j * rows[:, 2::2]).reshape(-1, 2, 2)
    w = W.spin_boson_tt(n_steps=1000)
    g = gpu_mixed(pkg, w)
    err, n = 0.0, 0
    for k, s in enumerate(steps):
        if s > n:
            g.ttn_step(w.dt, pkg.TTN_PS1, int(s - n))
            n = int(s)
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - ref[k]))))
    g.close()
    assert err <= TOL_FP64


@pytest.mark.parametrize("make", [lambda: W.exciton_chain(n_sites=3, rank=7, depth=4, n_steps=30),
                                  lambda: W.exciton_chain(n_steps=2)])
def test_mixed_exciton_chain(pkg, make):
    w = make()
    g = gpu_mixed(pkg, w)
    o = ottn.from_workload(w)
    err = 0.0
    for _ in range(w.n_steps):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err <= TOL_FP64


def test_mixed_driven_tls(pkg):
    w = W.spin_boson_tt(depth=5, n_pade=2, rank=5, tree="btt")
    w.drives = [W.Drive(V=W.SIGMA_X, amp=0.5, omega=3.0)]
    g = gpu_mixed(pkg, w)
    o = ottn.from_workload(w)
    err = 0.0
    for _ in range(40):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err <= TOL_FP64


def test_batched_instances_equal_individual_runs(pkg):
    """Uneven spin-boson instances (K, depth, rank, parameters all different)
    stepped together by ttn_batch_step give bitwise the results of stepping
    each alone, and agree with the oracle."""
    ws = W.spin_boson_batch(n=6, n_steps=6)
    batch = [gpu_from(pkg, w) for w in ws]
    alone = [gpu_from(pkg, w) for w in ws]
    pkg.ttn_batch_step(batch, 0.01, pkg.TTN_PS1, 6)
    for g, w in zip(alone, ws):
        g.ttn_step(w.dt, pkg.TTN_PS1, 6)
    for gb, ga, w in zip(batch, alone, ws):
        rb, ra = gb.ttn_rdm(), ga.ttn_rdm()
        assert np.array_equal(rb, ra)
        assert abs(gb.ttn_time() - 0.06) < 1e-12
    for gb, w in zip(batch, ws):
        o = ottn.from_workload(w)
        for _ in range(6):
            o.step(0.01, "ps1")
        assert np.max(np.abs(gb.ttn_rdm() - o.rdm())) <= TOL_SHORT
    # a second call reuses the cached parent graph
    pkg.ttn_batch_step(batch, 0.01, pkg.TTN_PS1, 2)
    for g in alone:
        g.ttn_step(0.01, pkg.TTN_PS1, 2)
    for gb, ga in zip(batch, alone):
        assert np.array_equal(gb.ttn_rdm(), ga.ttn_rdm())
    for g in batch + alone:
        g.close()


def test_batched_mixed_instances_equal_individual_runs(pkg):
    """The mixed form (FP32 contractions, the largest nodes on the tensor
    cores) under ttn_batch_step: bitwise the results of stepping each
    instance alone in the same form, and within the mixed-form tolerance of
    the FP64 oracle."""
    ws = W.spin_boson_batch(n=6, n_steps=6)
    batch = [gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32) for w in ws]
    alone = [gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32) for w in ws]
    pkg.ttn_batch_step(batch, 0.01, pkg.TTN_PS1, 6)
    for g in alone:
        g.ttn_step(0.01, pkg.TTN_PS1, 6)
    for gb, ga, w in zip(batch, alone, ws):
        assert np.array_equal(gb.ttn_rdm(), ga.ttn_rdm())
        o = ottn.from_workload(w)
        for _ in range(6):
            o.step(0.01, "ps1")
        assert np.max(np.abs(gb.ttn_rdm() - o.rdm())) <= TOL_MIXED
    for g in batch + alone:
        g.close()


# ---------------------------------------------------------------------------
# ps2 (adaptive rank): two-site flows, FP64 one-sided Jacobi SVD, truncation
# r = min(cap, max(1, ceil(ps2_ratio * #{sigma > ps2_atol}))), deterministic
# completion; ranks must follow the oracle exactly.
# ---------------------------------------------------------------------------
def run_ps2(pkg, w, n, max_rank, atol):
    g = gpu_from(pkg, w, params={"max_rank": max_rank, "ps2_atol": atol})
    o = ottn.from_workload(w, params=ottn.Params(ps2_atol=atol, max_rank=max_rank))
    err = 0.0
    for k in range(n):
        g.ttn_step(w.dt, pkg.TTN_PS2, 1)
        o.step(w.dt, "ps2")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
        assert list(g.ttn_get_ranks()) == o.ranks, (k, list(g.ttn_get_ranks()), o.ranks)
    return err, g, o


@pytest.mark.parametrize("tree,rank", [("tt", 1), ("btt", 3)])
def test_ps2_spin_boson(pkg, tree, rank):
    w = W.spin_boson_tt(depth=4, n_pade=3, rank=rank, tree=tree)
    err, g, o = run_ps2(pkg, w, 10, 8, 1e-7)
    assert max(o.ranks) > rank  # the ranks did adapt
    g.close()
    assert err <= TOL_SHORT


def test_ps2_driven_structured_bath(pkg):
    w = W.driven_structured_tls(n_pade=1, depth=4)
    err, g, o = run_ps2(pkg, w, 6, 6, 1e-6)
    g.close()
    assert err <= TOL_SHORT


def test_ps2_multibath_and_reset(pkg):
    w = W.exciton_chain(n_sites=3, rank=2, depth=3)
    err, g, o = run_ps2(pkg, w, 4, 6, 1e-6)
    assert err <= TOL_SHORT
    # a new initial state restores the initial ranks
    g.ttn_set_rdo0(w.rho0)
    o2 = ottn.from_workload(w)
    assert list(g.ttn_get_ranks()) == o2.ranks
    assert np.max(np.abs(g.ttn_rdm() - w.rho0)) == 0.0
    g.close()


def test_ps2_then_ps1_mixed_strategy(pkg):
    """Adaptive phase then fixed-rank phase on the ranks ps2 chose (the paper's
    mixed strategy with ps1 as the main method)."""
    w = W.spin_boson_tt(depth=4, n_pade=3, rank=2, tree="btt")
    err, g, o = run_ps2(pkg, w, 5, 8, 1e-7)
    for _ in range(5):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err <= TOL_SHORT


def test_ps2_and_ps1_runs_are_bitwise_repeatable(pkg):
    """Three fresh handles on the same input give bit-identical trajectories
    (fixed reduction orders everywhere; a race or an unsynchronised host read
    would show up here first)."""
    for scheme, w in (("ps2", W.spin_boson_tt(depth=4, n_pade=3, rank=3, tree="btt")),
                      ("ps1", W.exciton_chain(n_sites=3, rank=7, depth=4))):
        code = pkg.TTN_PS1 if scheme == "ps1" else pkg.TTN_PS2
        runs = []
        for _ in range(3):
            g = gpu_from(pkg, w, params={"max_rank": 8, "ps2_atol": 1e-7})
            traj = []
            for _ in range(8):
                g.ttn_step(w.dt, code, 1)
                traj.append(g.ttn_rdm())
            runs.append(np.array(traj))
            g.close()
        assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2]), scheme


def test_autotuned_handle_matches_oracle(pkg):
    """ttn_autotune changes only launch shapes: the trajectory stays on the
    oracle's, in FP64 and in the mixed form, and tuning twice is harmless."""
    w = W.exciton_chain(n_sites=3, rank=7, depth=4, n_steps=6)
    for prec, tol in ((pkg.TTN_FP64, TOL_SHORT), (pkg.TTN_MIXED_FP32, 1e-6)):
        g = gpu_from(pkg, w, precision=prec)
        o = ottn.from_workload(w)
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        g.ttn_autotune(2)
        g.ttn_autotune(1)
        err = float(np.max(np.abs(g.ttn_rdm() - o.rdm())))
        for _ in range(5):
            g.ttn_step(w.dt, pkg.TTN_PS1, 1)
            o.step(w.dt, "ps1")
            err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
        g.close()
        assert err <= tol, (prec, err)


# ---------------------------------------------------------------------------
# Bonds wider than 64 (ranks up to 256 are accepted): the QR matricisations
# 81 x 81 and 324 x 81 exceed the cluster and blocked kernels' 64 columns and
# run on the one-CTA Householder kernel.
# ---------------------------------------------------------------------------
def _wide_bond_workload():
    w = W.spin_boson_tt(depth=9, n_pade=3, rank=96, tree="btt")
    o = ottn.from_workload(w)
    assert max(o.ranks) == 81
    return w, o


def test_bonds_wider_than_64_product_state(pkg):
    w, _ = _wide_bond_workload()
    err, g, _ = run_both(pkg, w, 10)
    assert max(g.ttn_get_ranks()) == 81
    g.close()
    assert err <= TOL_SHORT


def test_bonds_wider_than_64_generic_state_node_tensors(pkg):
    """From a generic full-rank tree every node tensor after two steps -- the Q
    factors of the 81-column QRs with their phase convention -- matches the
    oracle, in FP64 (1e-10) and, for rho_S, in the mixed form (1e-6)."""
    w, o = _wide_bond_workload()
    rng = np.random.default_rng(81)
    tensors = []
    for u, T in enumerate(o.tensors):
        X = rng.normal(size=T.shape) + 1j * rng.normal(size=T.shape)
        if u == 0:
            X /= np.linalg.norm(X)
        else:
            M = np.moveaxis(X, 0, -1)
            sh = M.shape
            Q, _ = np.linalg.qr(M.reshape(-1, sh[-1]))
            X = np.moveaxis(Q.reshape(sh), -1, 0)
        tensors.append(X)
    o.tensors = [t.copy() for t in tensors]
    for c in o.tree.postorder():
        if c:
            o.update_env(c, o.tree.parent[c])
    ga = gpu_from(pkg, w)
    gb = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    for g in (ga, gb):
        for u, t in enumerate(tensors):
            g.ttn_set_node(u, t)
        g.ttn_step(w.dt, pkg.TTN_PS1, 2)
    for _ in range(2):
        o.step(w.dt, "ps1")
    errs = [float(np.max(np.abs(ga.ttn_get_node(u) - o.tensors[u]))) for u in range(len(w.parent))]
    e_fp64 = float(np.max(np.abs(ga.ttn_rdm() - o.rdm())))
    e_mixed = float(np.max(np.abs(gb.ttn_rdm() - o.rdm())))
    ga.close()
    gb.close()
    assert max(errs) < 1e-10, errs
    assert e_fp64 <= TOL_SHORT
    assert e_mixed <= TOL_MIXED


# ---------------------------------------------------------------------------
# Long fixed-rank trajectories: with the QR dependence threshold at 1e-9 the
# completion of nearly dependent columns no longer depends on rounding, so
# runs that differ only in the order of their sums, or in the precision of
# the contractions, stay together over the whole trajectory.
# ---------------------------------------------------------------------------
def test_long_trajectory_reproducible_and_mixed_within_bar(pkg):
    w = W.exciton_chain(rank=20)
    ga = gpu_from(pkg, w)
    gb = gpu_from(pkg, w)
    gb.ttn_set_params(max_split=1)  # another summation order of every split contraction
    gc = gpu_from(pkg, w, precision=pkg.TTN_MIXED_FP32)
    e_order = e_mixed = 0.0
    for k in range(1000):
        for g in (ga, gb, gc):
            g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        if (k + 1) % 50 == 0:
            ra = ga.ttn_rdm()
            e_order = max(e_order, float(np.max(np.abs(gb.ttn_rdm() - ra))))
            e_mixed = max(e_mixed, float(np.max(np.abs(gc.ttn_rdm() - ra))))
    for g in (ga, gb, gc):
        g.close()
    assert e_order <= 1e-10, e_order  # 8e-6 with the former 1e-12 threshold
    assert e_mixed <= TOL_MIXED, e_mixed
