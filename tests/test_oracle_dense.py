"""Pins for oracle.dense (Eq. EDO-eom with rho_S = <0|Omega>, Sec. 2.2) against
closed forms: lambda = 0 gives unitary dynamics, pure dephasing ([H, Q] = 0)
gives rho_ab(t) = rho_ab(0) exp(-i w_ab t - Phi_ab(t)) from the influence
functional of Sec. 2.2 with the decomposed C(t); the trace of rho_S is conserved."""
import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import bcf, dense, sop


def test_zero_coupling_is_unitary():
    rng = np.random.default_rng(11)
    H = W.random_hermitian(rng, 3)
    rho0 = W.random_density_matrix(rng, 3)
    bath = W.Bath(Q=W.random_hermitian(rng, 3), beta=1.0, dl=(0.0, 1.0), n_ltc=1)
    depth = [3, 3]
    tr = dense.propagate(sop.heom_terms(H, [bath], depth), rho0, depth, 0.1, 10)
    for n in range(11):
        U = expm(-1j * H * 0.1 * n)
        assert np.max(np.abs(tr[n] - U @ rho0 @ U.conj().T)) < 1e-12


def _dephasing_closed_form(feats, E, q, rho0, t):
    G = sum(c * (np.exp(g * t) - 1 - g * t) / g ** 2 for c, cb, g in feats)
    Gb = sum(cb * (np.exp(g * t) - 1 - g * t) / g ** 2 for c, cb, g in feats)
    M = len(E)
    out = np.zeros((len(t), M, M), complex)
    for a in range(M):
        for b in range(M):
            phi = q[a] ** 2 * G + q[b] ** 2 * Gb - q[a] * q[b] * (G + Gb)
            out[:, a, b] = rho0[a, b] * np.exp(-1j * (E[a] - E[b]) * t - phi)
    return out


@pytest.mark.parametrize("bath_kind", ["drude", "brownian"])
def test_pure_dephasing_closed_form(bath_kind):
    E = np.array([0.5, -0.5])
    q = np.array([1.0, -1.0])
    H = np.diag(E).astype(complex)
    Q = np.diag(q).astype(complex)
    if bath_kind == "drude":
        bath = W.Bath(Q=Q, beta=1.0, dl=(0.3, 1.0), n_ltc=2)
        depth = [16, 16, 16]
    else:
        bath = W.Bath(Q=Q, beta=2.0, bo=[(0.05, 1.0, 0.3)], n_ltc=1)
        depth = [14, 14, 14]
    rho0 = 0.5 * np.ones((2, 2), complex)
    feats = bcf.bath_features(bath.beta, bath.dl, bath.bo, bath.n_ltc)
    dt, n = 0.02, 100
    tr = dense.propagate(sop.heom_terms(H, [bath], depth), rho0, depth, dt, n)
    ref = _dephasing_closed_form(feats, E, q, rho0, dt * np.arange(n + 1))
    assert np.max(np.abs(tr - ref)) < 1e-9


def test_trace_and_hermiticity_conserved():
    wl = W.spin_boson_tt(depth=4, n_pade=2)
    terms = sop.heom_terms(wl.H, wl.baths, wl.depth)
    tr = dense.propagate(terms, wl.rho0, wl.depth, 0.05, 40)
    for r in tr:
        assert abs(np.trace(r) - 1.0) < 1e-12
        assert np.max(np.abs(r - r.conj().T)) < 1e-12
