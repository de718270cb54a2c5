"""Pins for the oracle's direct integration (vmf, Sec. 2.3 and Sec. 7.5) and
its Dormand-Prince integrator: dopri5 against the matrix exponential; vmf at
untruncated ranks (the variational manifold is the whole space) against the
dense hierarchy; vmf on the pure-dephasing manifold from a generic point of
it (the exact solution stays on the manifold, so the projected equations are
exact); the regularisation; the mixed strategy's switch."""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.sparse.linalg import expm_multiply

import workloads as W
from oracle import dense, sop, ttn


def test_dopri5_matches_expm_and_tightens_with_tolerance():
    rng = np.random.default_rng(1)
    A = 0.7 * (rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6)))
    y0 = rng.normal(size=6) + 1j * rng.normal(size=6)
    exact = expm(2.0 * A) @ y0
    errs = []
    for tol in (1e-4, 1e-7, 1e-10):
        y, _, acc, rej = ttn.dopri5(lambda t, y: [A @ y[0]], [y0], 0.0, 2.0, 0.5, tol, tol)
        errs.append(np.max(np.abs(y[0] - exact)))
        assert acc > 0
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8 * np.max(np.abs(exact))


def test_dopri5_is_fifth_order_at_fixed_step():
    # with tolerances that accept every step the controller still picks the
    # step; the fifth-order solution's error ratio shows on a fixed grid
    rng = np.random.default_rng(2)
    A = 0.5 * (rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5)))
    y0 = rng.normal(size=5) + 0j
    exact = expm(A) @ y0

    def fixed(n):
        y = [y0]
        for k in range(n):  # one accepted step per call (huge tolerance, trial step = the interval)
            y, _, acc, _ = ttn.dopri5(lambda t, y: [A @ y[0]], y, k / n, (k + 1) / n, 1.0 / n, 1e9, 1e9)
        return np.max(np.abs(y[0] - exact))
    e1, e2 = fixed(8), fixed(16)
    assert 24 < e1 / e2 < 40  # 2^5 = 32


def _full_rank_start(w, rng, t0=0.2):
    """A generic point: the exact state at t0 plus a small random full-rank
    admixture, as a tree (HTD) at the ranks of w (untruncated here)."""
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    L = dense.generator(terms, w.leg_dims)
    v = expm_multiply(t0 * L, dense.initial_vector(w.rho0, w.depth))
    v = v + 1e-3 * (rng.normal(size=v.shape) + 1j * rng.normal(size=v.shape))
    return L, v


def test_vmf_at_untruncated_ranks_equals_dense():
    w = W.spin_boson_tt(depth=3, n_pade=2, rank=1000, tree="btt")
    rng = np.random.default_rng(3)
    L, v = _full_rank_start(w, rng)
    st = ttn.from_workload(w, params=ttn.Params(ode_rtol=1e-10, ode_atol=1e-12, vmf_atol=0.0))
    st.tensors = ttn.htd_tensors(st.tree, st.leg_dims, st.ranks, v.reshape(w.leg_dims))
    for c in st.tree.postorder():
        if c:
            st.update_env(c, st.tree.parent[c])
    for k in range(5):
        st.step(0.02, "vmf")
    ref = expm_multiply(0.1 * L, v)
    assert np.max(np.abs(st.full_tensor().reshape(-1) - ref)) < 1e-8
    # the non-root tensors stay semi-unitary (the gauge <U|dU/dt> = 0 is kept)
    for u in range(1, st.tree.n_nodes):
        U = st.tensors[u].reshape(st.tensors[u].shape[0], -1)
        assert np.max(np.abs(U.conj() @ U.T - np.eye(U.shape[0]))) < 1e-8


def test_vmf_exact_on_pure_dephasing_manifold():
    E, q = np.array([0.5, -0.5]), np.array([1.0, -1.0])
    bath = W.Bath(Q=np.diag(q).astype(complex), beta=1.0, dl=(0.3, 1.0), n_ltc=2)
    depth = [6, 6, 6]
    parent, leg_node = W.tensor_train(3)
    # the exact state has bond ranks 4 and 3 (the Pade features 2 and 3 see the
    # sectors q_a = q_b alike), so at these ranks every single-hole density
    # matrix is invertible and no regularisation is needed
    w = W.Workload("pd", np.diag(E).astype(complex), [bath], depth, parent, leg_node, [0, 4, 3],
                   0.5 * np.ones((2, 2), complex), 0.05, 20)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    L = dense.generator(terms, w.leg_dims)
    v1 = expm_multiply(0.2 * L, dense.initial_vector(w.rho0, w.depth))
    v2 = expm_multiply(1.0 * L, v1)
    st = ttn.from_workload(w, params=ttn.Params(ode_rtol=1e-9, ode_atol=1e-11, vmf_atol=0.0))
    st.tensors = ttn.htd_tensors(st.tree, st.leg_dims, st.ranks, v1.reshape(w.leg_dims))
    for c in st.tree.postorder():
        if c:
            st.update_env(c, st.tree.parent[c])
    for _ in range(w.n_steps):
        st.step(w.dt, "vmf")
    assert np.max(np.abs(st.rdm() - dense.rdm(v2, 2, w.depth))) < 1e-7


def test_vmf_regularisation_from_the_product_state():
    """From the rank-padded product state the single-hole density matrices are
    singular: without regularisation the inverse is undefined, with vmf_atol
    the flow is finite and stays close to ps1 at small dt (both approximate
    the same projected dynamics)."""
    w = W.spin_boson_tt(depth=5, n_pade=2, rank=4, tree="btt")
    a = ttn.from_workload(w, params=ttn.Params(vmf_atol=1e-8))
    b = ttn.from_workload(w)
    for _ in range(10):
        a.step(0.01, "vmf")
        b.step(0.01, "ps1")
    ra, rb = a.rdm(), b.rdm()
    assert np.all(np.isfinite(ra))
    assert np.max(np.abs(ra - rb)) < 1e-2


def test_mix_switches_from_ps2_to_vmf_at_the_cap():
    w = W.spin_boson_tt(depth=4, n_pade=2, rank=2, tree="btt")
    st = ttn.from_workload(w, params=ttn.Params(ps2_atol=1e-9, max_rank=4))
    ranks = []
    for _ in range(6):
        st.step(0.01, "mix")
        ranks.append(max(st.ranks[1:]))
    assert getattr(st, "_mixed_to_vmf", False)
    k = ranks.index(4)
    assert all(r == 4 for r in ranks[k:])  # frozen after the switch
    assert getattr(st, "vmf_stats", [0, 0])[0] > 0
