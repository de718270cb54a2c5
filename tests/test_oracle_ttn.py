"""Pins for oracle.ttn (Sec. 2.3 TTN decomposition, Eq. semiunitary, the ps1/ps2
projector-splitting propagation) against things fixed independently of it:
LAPACK QR, the matrix exponential, the dense hierarchy of oracle.dense (itself
pinned to closed forms), the exactness of projector splitting on the manifold,
second-order convergence of the symmetric composition, and the gauge invariants."""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.sparse.linalg import expm_multiply

import workloads as W
from oracle import dense, sop, ttn


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("m,n", [(7, 3), (40, 10), (64, 64), (400, 20)])
def test_householder_qr_matches_lapack(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = _rand(rng, m, n)
    Q, R = ttn.householder_qr(A, 1e-12)
    Ql, Rl = np.linalg.qr(A)
    ph = np.diag(Rl) / np.abs(np.diag(Rl))
    Ql, Rl = Ql * ph[None, :], Rl * np.conj(ph)[:, None]
    assert np.max(np.abs(Q - Ql)) < 1e-12 and np.max(np.abs(R - Rl)) < 1e-11
    assert np.allclose(np.diag(R).imag, 0) and np.all(np.diag(R).real > 0)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(n))) < 1e-13


def test_householder_qr_rank_deficient_is_deterministic():
    rng = np.random.default_rng(5)
    B = _rand(rng, 30, 3)
    A = np.concatenate([B, B[:, :1] + 2 * B[:, 1:2], np.zeros((30, 1)), B[:, 2:] * 1j], axis=1)
    Q1, R1 = ttn.householder_qr(A, 1e-12)
    Q2, R2 = ttn.householder_qr(A + 1e-16 * _rand(rng, 30, 6), 1e-12)
    assert np.max(np.abs(Q1.conj().T @ Q1 - np.eye(6))) < 1e-13
    assert np.max(np.abs(Q1 @ R1 - A)) < 1e-12
    assert abs(R1[3, 3]) == 0 and abs(R1[4, 4]) == 0
    # the completion columns do not follow the rounding noise
    assert np.max(np.abs(Q1 - Q2)) < 1e-9


def test_default_qr_threshold_completes_nearly_dependent_columns_deterministically():
    """A column that is dependent up to a 1e-11 relative remainder (what a
    truncated state's padding directions look like after some steps): with the
    default threshold it has no reflector and its Q column is the completion,
    unchanged by 1e-16 noise; a threshold far below the remainder builds a
    reflector from it instead (so rounding-sized noise in the remainder moves
    that Q column at first order)."""
    rng = np.random.default_rng(11)
    B = _rand(rng, 40, 3)
    near = B[:, :1] - 0.5 * B[:, 2:] + 1e-11 * np.linalg.norm(B) * _rand(rng, 40, 1)
    A = np.concatenate([B, near], axis=1)
    tol = ttn.Params().qr_tol
    assert tol >= 1e-10
    Q1, R1 = ttn.householder_qr(A, tol)
    Q2, R2 = ttn.householder_qr(A + 1e-16 * _rand(rng, 40, 4), tol)
    assert R1[3, 3] == 0.0 and R2[3, 3] == 0.0
    assert np.max(np.abs(Q1 - Q2)) < 1e-12
    assert np.max(np.abs(Q1.conj().T @ Q1 - np.eye(4))) < 1e-13
    Qs, Rs = ttn.householder_qr(A, 1e-14)
    assert abs(Rs[3, 3]) > 0.0  # a reflector built from the 1e-11 remainder


def test_rk4_is_fourth_order():
    rng = np.random.default_rng(2)
    A = 0.5 * _rand(rng, 6, 6)
    y0 = _rand(rng, 6)
    exact = expm(A) @ y0
    errs = [np.linalg.norm(ttn.rk4(lambda y: A @ y, y0, 1.0, m) - exact) for m in (8, 16, 32)]
    for e1, e2 in zip(errs, errs[1:]):
        assert 13 < e1 / e2 < 19


def _run(st, n, dt, scheme="ps1"):
    out = [st.rdm()]
    for _ in range(n):
        st.step(dt, scheme)
        out.append(st.rdm())
    return np.array(out)


@pytest.mark.parametrize("tree", ["tt", "btt"])
@pytest.mark.parametrize("scheme", ["ps1", "ps2"])
def test_untruncated_ranks_equal_dense(tree, scheme):
    w = W.spin_boson_tt(depth=4, n_pade=2, rank=1000, tree=tree)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    ref = dense.propagate(terms, w.rho0, w.depth, 0.01, 40)
    st = ttn.from_workload(w, params=ttn.Params(ps2_atol=0.0, max_rank=1000))
    assert max(st.ranks) == 16
    tr = _run(st, 40, 0.01, scheme)
    assert np.max(np.abs(tr - ref)) < 1e-8


def test_untruncated_multibath_and_metric_independence():
    rng = np.random.default_rng(9)
    H = W.random_hermitian(rng, 3)
    baths = [W.Bath(Q=np.diag([1.0, 0, -1]).astype(complex), beta=1.0, dl=(0.3, 1.0), n_ltc=1),
             W.Bath(Q=W.random_hermitian(rng, 3), beta=2.0, bo=[(0.1, 1.2, 0.3)])]
    depth = [3, 3, 3, 3]
    parent, leg_node = W.balanced_binary(4)
    rho0 = W.random_density_matrix(rng, 3)
    ref = dense.propagate(sop.heom_terms(H, baths, depth), rho0, depth, 0.02, 20)
    for metric in ("abs", "conventional"):
        terms = sop.heom_terms(H, baths, depth, metric=metric)
        st = ttn.TTN(parent, leg_node, [3, 3] + depth, [0] + [1000] * 3, terms, rho0)
        tr = _run(st, 20, 0.02)
        assert np.max(np.abs(tr - ref)) < 1e-6  # RK4 truncation at h = 0.02


def _dephasing_model(dt, n, ranks=(0, 4, 4)):
    E, q = np.array([0.5, -0.5]), np.array([1.0, -1.0])
    bath = W.Bath(Q=np.diag(q).astype(complex), beta=1.0, dl=(0.3, 1.0), n_ltc=2)
    depth = [6, 6, 6]
    parent, leg_node = W.tensor_train(3)
    return W.Workload("pd", np.diag(E).astype(complex), [bath], depth, parent, leg_node,
                      list(ranks), 0.5 * np.ones((2, 2), complex), dt, n)


def test_ps2_exact_on_pure_dephasing_manifold():
    # the exact pure-dephasing EDO is sum_ab |a><b| (x) prod_k phi_k^ab: bond rank <= M^2
    w = _dephasing_model(0.02, 50)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    ref = dense.propagate(terms, w.rho0, w.depth, w.dt, w.n_steps)
    st = ttn.from_workload(w, params=ttn.Params(ps2_atol=1e-10, max_rank=4))
    assert np.max(np.abs(_run(st, w.n_steps, w.dt, "ps2") - ref)) < 1e-7


def test_ps1_exact_on_manifold_from_generic_state():
    # Projector splitting is exact up to the RK4 error when the solution stays on
    # the rank-4 manifold and the start point is a generic point of it (HTD of the
    # exact state at t = 0.2).
    w = _dephasing_model(0.01, 100)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    L = dense.generator(terms, w.leg_dims)
    v1 = expm_multiply(0.2 * L, dense.initial_vector(w.rho0, w.depth))
    v2 = expm_multiply(1.0 * L, v1)
    st = ttn.from_workload(w)
    st.tensors = ttn.htd_tensors(st.tree, st.leg_dims, st.ranks, v1.reshape(w.leg_dims))
    for c in st.tree.postorder():
        if c:
            st.update_env(c, st.tree.parent[c])
    assert np.max(np.abs(st.full_tensor().reshape(-1) - v1)) < 1e-12
    _run(st, w.n_steps, w.dt)
    assert np.max(np.abs(st.rdm() - dense.rdm(v2, 2, w.depth))) < 1e-6


@pytest.mark.parametrize("scheme", ["ps1", "ps2"])
def test_driven_second_order_in_dt(scheme):
    w = W.spin_boson_tt(depth=4, n_pade=2, rank=1000)
    w.drives = [W.Drive(V=W.SIGMA_X, amp=0.5, omega=3.0)]
    terms = sop.heom_terms(w.H, w.baths, w.depth, drives=w.drives)
    errs = []
    for dt in (0.02, 0.01):
        n = int(round(0.4 / dt))
        ref = dense.propagate(terms, w.rho0, w.depth, dt, n, drives=w.drives, rk4_sub=16)
        st = ttn.from_workload(w, params=ttn.Params(ps2_atol=0.0, max_rank=1000))
        errs.append(np.max(np.abs(_run(st, n, dt, scheme)[-1] - ref[-1])))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_gauge_invariants_after_truncated_steps():
    w = W.spin_boson_tt(depth=6, n_pade=3, rank=5, tree="btt")
    st = ttn.from_workload(w)
    _run(st, 5, 0.01)
    for u in range(1, st.tree.n_nodes):
        U = st.tensors[u].reshape(st.tensors[u].shape[0], -1)
        assert np.max(np.abs(U.conj() @ U.T - np.eye(U.shape[0]))) < 1e-12
    r = st.rdm()
    assert abs(np.trace(r) - 1) < 1e-6
    assert np.max(np.abs(r - r.conj().T)) < 1e-6


def test_effective_ranks_and_product_state():
    w = W.spin_boson_tt()
    st = ttn.from_workload(w)
    assert st.ranks == [0, 4, 10, 10]
    assert np.allclose(st.rdm(), w.rho0)
    w2 = W.exciton_chain(n_steps=1)
    st2 = ttn.TTN(w2.parent, w2.leg_node, w2.leg_dims, w2.ranks, [], w2.rho0)
    assert st2.tree.n_nodes == 21 and st2.ranks[1] == 20
    assert sum(int(np.prod(T.shape)) for T in st2.tensors) == 83220
    assert np.allclose(st2.rdm(), w2.rho0)


def test_truncated_ps1_converges_with_rank():
    w = W.spin_boson_tt(depth=6, n_pade=3, rank=2, n_steps=40)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    ref = dense.propagate(terms, w.rho0, w.depth, w.dt, w.n_steps)
    errs = []
    for R in (2, 4, 8):
        w.ranks = W.uniform_ranks(w.parent, R)
        errs.append(np.max(np.abs(_run(ttn.from_workload(w), w.n_steps, w.dt) - ref)))
    assert errs[0] > errs[1] > errs[2]


def test_centred_train_custom_frame_equals_dense_and_other_trees():
    """The custom frame of Sec. 7.2 (root in the middle of the train, arm ends
    with two legs): at untruncated ranks it reproduces the dense hierarchy, as
    the tensor train and the balanced binary tree do (all three span the whole
    space there)."""
    w = W.spin_boson_tt(depth=4, n_pade=3, rank=1000)
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    ref = dense.propagate(terms, w.rho0, w.depth, 0.01, 20)
    out = {}
    for name, (parent, leg_node) in (("centred", W.centred_train(4)), ("tt", W.tensor_train(4)),
                                     ("btt", W.balanced_binary(4))):
        st = ttn.TTN(parent, leg_node, w.leg_dims, [0] + [1000] * (len(parent) - 1), terms, w.rho0)
        out[name] = _run(st, 20, 0.01)
        assert np.max(np.abs(out[name] - ref)) < 1e-8, name
    assert any(len(l) == 2 for l in ttn.Tree(*W.centred_train(4)).legs)
