"""Pins for the oracle's ML-MCTDH star bath (Sec. 3.2.4): the discretised
thermofield bath reproduces the thermal correlation function (Eq. 2) at times
well inside its recurrence, and the TTN propagation of the wavefunction at
untruncated ranks equals the exact exponential of the Hamiltonian."""
import numpy as np
from scipy.integrate import quad
from scipy.linalg import expm

import workloads as W
from oracle import bcf, mctdh, ttn


def test_thermofield_modes_reproduce_the_thermal_bcf():
    w0 = W.star_boson_mctdh()
    b = w0.bo[0]
    J = lambda x: bcf.J_bo(x, *b)  # noqa: E731
    for n_modes, tol in ((50, 0.05), (200, 0.01)):
        w, g = mctdh.modes(w0.bo, w0.beta, w0.cutoff, n_modes)
        for t in (10.0, 50.0, 100.0):  # fs; the recurrence of 50 modes is ~4000 fs
            re = quad(lambda x: J(x) / np.tanh(w0.beta * x / 2), 1e-12, np.inf, weight="cos", wvar=t, limlst=400)[0]
            im = -quad(J, 0, np.inf, weight="sin", wvar=t, limlst=400)[0]
            C = np.sum(g ** 2 * np.exp(-1j * w * t))
            assert abs(C - (re + 1j * im)) < tol * abs(re + 1j * im) + 1e-4 * abs(C), (n_modes, t)


def _tiny(n_modes=4, dim=3):
    w0 = W.star_boson_mctdh(n_modes=n_modes, dim=dim, rank=1000)
    w0.ranks = [0] + [1000] * (len(w0.parent) - 1)  # untruncated, the root bond included
    w, g = mctdh.modes(w0.bo, w0.beta, w0.cutoff, n_modes)
    terms = mctdh.terms(w0.H, w0.Q, w, g, dim)
    return w0, w, g, terms


def test_wavefunction_ttn_at_full_rank_equals_exact_exponential():
    w0, w, g, terms = _tiny()
    # kappa 0.025: a hundred times the default RK4 substeps, so that the RK4
    # error of the sub-flows (the only error left at untruncated ranks) is
    # negligible; the result converges to the exponential as kappa shrinks
    st = ttn.TTN(w0.parent, w0.leg_node, w0.leg_dims, w0.ranks, terms, mctdh.rho0(w0.psi0),
                 params=ttn.Params(kappa=0.025))
    for _ in range(10):
        st.step(2.0, "ps1")
    # exact: psi(t) = exp(-i H t) psi0 on system (x) modes (the spectator stays at 0)
    M, d, n = 2, w0.dim, w0.n_modes
    a = np.diag(np.sqrt(np.arange(1, d)), 1)
    eye = [np.eye(d)] * n

    def kron_all(ops):
        out = np.eye(1)
        for o in ops:
            out = np.kron(out, o)
        return out
    Hm = np.kron(w0.H, kron_all(eye))
    for k in range(n):
        ops = list(eye)
        ops[k] = np.diag(np.arange(d)).astype(float)
        Hm = Hm + w[k] * np.kron(np.eye(M), kron_all(ops))
        ops[k] = a + a.T
        Hm = Hm + g[k] * np.kron(w0.Q, kron_all(ops))
    psi0 = np.kron(w0.psi0, np.eye(d ** n)[0])
    psi = expm(-1j * 20.0 * Hm) @ psi0
    full = st.full_tensor()[:, 0].reshape(-1)
    assert np.max(np.abs(full - psi)) < 1e-6
    assert np.max(np.abs(mctdh.system_rho(st) - mctdh.system_rho_root(st))) < 1e-12
    assert abs(np.trace(mctdh.system_rho(st)) - 1.0) < 1e-6
