"""Pins for the oracle's ps2 truncation rule and its SVD completion (Sec. 2.3
last paragraph: the adaptive scheme splits the merged pair by an SVD; Sec. 7.5:
a multiple of the kept count re-admits part of the discarded singular values).

The rule read from those passages: r0 = #{sigma > ps2_atol} (strictly above),
r' = min(cap, len(sigma), max(1, ceil(ps2_ratio * r0))). The expected ranks
below are written out by hand from that statement, and the ps2 run checks the
rule end to end on a model whose bond rank follows from the physics (the
pure-dephasing sector argument), not from the oracle.
"""
import types

import numpy as np
import pytest

import workloads as W
from oracle import dense, sop, ttn


def _rule(s, cap, atol=1e-6, ratio=2.0):
    obj = types.SimpleNamespace(params=ttn.Params(ps2_atol=atol, ps2_ratio=ratio))
    return ttn.TTN.truncation_rank(obj, np.asarray(s, float), cap)


@pytest.mark.parametrize("s,cap,atol,ratio,expect", [
    # a singular value exactly at the threshold is not counted (strict >)
    ([1.0, 1e-6, 1e-7], 32, 1e-6, 2.0, 2),
    ([1.0, 1e-6 * (1 + 1e-15), 1e-7], 32, 1e-6, 2.0, 3),
    # nothing above the threshold still keeps one vector
    ([1e-7, 1e-8], 32, 1e-6, 2.0, 1),
    ([0.0, 0.0, 0.0], 32, 1e-6, 2.0, 1),
    # r0 = 3, ratio 2 -> 6
    ([1.0, 0.5, 0.1, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11, 1e-12], 32, 1e-6, 2.0, 6),
    # the cap binds before the ratio does
    ([1.0, 0.5, 0.1, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11, 1e-12], 4, 1e-6, 2.0, 4),
    # the ratio is applied to r0 before the cap (ratio after cap would give 2 * 2 = 4 here)
    ([1.0, 0.5, 0.1, 1e-7, 1e-8, 1e-9], 5, 1e-6, 2.0, 5),
    # a non-integer ratio rounds up: ceil(1.5 * 3) = 5, ceil(1.25 * 3) = 4
    ([1.0, 0.5, 0.1, 1e-7, 1e-8, 1e-9, 1e-10], 32, 1e-6, 1.5, 5),
    ([1.0, 0.5, 0.1, 1e-7, 1e-8, 1e-9, 1e-10], 32, 1e-6, 1.25, 4),
    # an exact integer product is not pushed up by the ceiling: 2 * 2 = 4
    ([1.0, 0.5, 1e-7, 1e-8, 1e-9, 1e-10], 32, 1e-6, 2.0, 4),
    # never more than the number of singular values
    ([1.0, 0.5, 0.1], 32, 1e-6, 2.0, 3),
])
def test_truncation_rank_by_hand(s, cap, atol, ratio, expect):
    assert _rule(s, cap, atol, ratio) == expect


def _dephasing_model(dt, n):
    # H_S and Q commute (pure dephasing); Drude feature first, then 2 Pade features
    E, q = np.array([0.5, -0.5]), np.array([1.0, -1.0])
    bath = W.Bath(Q=np.diag(q).astype(complex), beta=1.0, dl=(0.3, 1.0), n_ltc=2)
    depth = [6, 6, 6]
    parent, leg_node = W.tensor_train(3)
    return W.Workload("pd", np.diag(E).astype(complex), [bath], depth, parent, leg_node,
                      [0, 4, 4], 0.5 * np.ones((2, 2), complex), dt, n)


@pytest.mark.parametrize("ratio,expect", [(1.0, 3), (1.5, 5), (2.0, 6), (3.0, 9)])
def test_ps2_ratio_sets_rank_below_the_cap(ratio, expect):
    """Pure dephasing, TT (i, j, n1 | n2, n3): in the system sector (a, b) the
    bath features see the coupling (q_a c_k - q_b cbar_k) A+ - (q_a - q_b) A-.
    The Pade features have real c_k = cbar_k, so the sectors (0,0) and (1,1)
    (q_a = q_b) drive features 2 and 3 identically: across the bond n2 n3 the EDO
    has exactly 3 independent components, so r0 = 3 there, and the rule keeps
    min(16, ceil(ratio * 3)) -- the cap 16 and the matricisation bounds (24, 36)
    do not bind. The root bond is capped at M^2 = 4 by the tree."""
    w = _dephasing_model(0.02, 20)
    st = ttn.from_workload(w, params=ttn.Params(ps2_atol=1e-7, ps2_ratio=ratio, max_rank=16))
    ref = dense.propagate(sop.heom_terms(w.H, w.baths, w.depth), w.rho0, w.depth, w.dt, w.n_steps)
    for _ in range(w.n_steps):
        st.step(w.dt, "ps2")
    assert st.ranks == [0, 4, expect]
    sv = st.bond_singular_values()
    assert [int(np.sum(s > 1e-7)) for s in sv] == [4, 3]
    assert np.max(np.abs(st.rdm() - ref[-1])) < 1e-7


def _unitary(rng, m, r):
    A = rng.normal(size=(m, r)) + 1j * rng.normal(size=(m, r))
    return np.linalg.qr(A)[0]


def test_svd_completion_keeps_determined_triplets_and_zeroes_the_rest():
    rng = np.random.default_rng(3)
    m, n, r, g = 12, 9, 5, 3
    Wm, Vm = _unitary(rng, m, r), _unitary(rng, n, r)
    s = np.array([2.0, 1.0, 0.3, 1e-14, 1e-15])
    W2, s2, V2 = ttn.svd_completion(Wm, s, Vm.conj().T, 1e-12)
    # determined triplets unchanged
    assert np.array_equal(W2[:, :g], Wm[:, :g]) and np.array_equal(V2[:g], Vm.conj().T[:g])
    assert np.array_equal(s2[:g], s[:g])
    # completed singular values exactly zero
    assert np.all(s2[g:] == 0.0)
    # completion columns orthonormal and orthogonal to the determined ones
    assert np.max(np.abs(W2.conj().T @ W2 - np.eye(r))) < 1e-13
    assert np.max(np.abs(V2 @ V2.conj().T - np.eye(r))) < 1e-13
    # the product is the rank-g truncation of the input
    ref = (Wm[:, :g] * s[:g]) @ Vm.conj().T[:g]
    assert np.max(np.abs((W2 * s2) @ V2 - ref)) < 1e-15


def test_svd_completion_ignores_the_undetermined_vectors():
    """The completion depends only on the determined columns: replacing the
    undetermined singular vectors (what rounding noise does to them) leaves the
    output unchanged bit for bit."""
    rng = np.random.default_rng(4)
    m, n, r = 10, 8, 4
    Wm, Vm = _unitary(rng, m, r), _unitary(rng, n, r)
    s = np.array([1.0, 0.5, 1e-13, 0.0])
    W1, s1, V1 = ttn.svd_completion(Wm, s, Vm.conj().T, 1e-12)
    W_alt = Wm.copy()
    W_alt[:, 2:] = _unitary(rng, m, 2)  # other (not orthogonal to the first two) vectors
    V_alt = Vm.conj().T.copy()
    V_alt[2:] = 1e-16 * rng.normal(size=(2, n))
    W2, s2, V2 = ttn.svd_completion(W_alt, s, V_alt, 1e-12)
    assert np.array_equal(W1, W2) and np.array_equal(s1, s2) and np.array_equal(V1, V2)


def test_svd_completion_of_one_vector_is_the_householder_reflector():
    """g = 1: the completion of a unit vector q is the reflector H = I - 2 v v^H /
    (v^H v), v = q + phi e_0, phi = q_0/|q_0| (it maps e_0 to -phi q), applied to
    e_1 .. e_{r-1}: columns e_j - 2 v conj(v_j) / (v^H v), written out here."""
    rng = np.random.default_rng(6)
    m, r = 7, 4
    q = rng.normal(size=m) + 1j * rng.normal(size=m)
    q /= np.linalg.norm(q)
    Wm = np.concatenate([q[:, None], _unitary(rng, m, r - 1)], axis=1)
    Vm = _unitary(rng, 5, r)
    s = np.array([1.0, 0.0, 0.0, 0.0])
    W2, _, _ = ttn.svd_completion(Wm, s, Vm.conj().T, 1e-12)
    phi = q[0] / abs(q[0])
    v = q.copy()
    v[0] += phi
    vv = np.vdot(v, v).real
    for j in range(1, r):
        col = -2.0 * v * np.conj(v[j]) / vv
        col[j] += 1.0
        assert np.max(np.abs(W2[:, j] - col)) < 1e-14
    assert np.array_equal(W2[:, 0], q)
