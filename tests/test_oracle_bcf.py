"""Pins for oracle.bcf (Sec. 2.1, Eqs. 2-3, Eq. bcfdecores) against mathematics
that does not go through the oracle: Bernoulli-number Taylor series of f_BE,
the Matsubara limit, and direct quadrature of the defining Fourier integral."""
from math import factorial

import numpy as np
import pytest
from scipy import integrate

from oracle import bcf


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_pade_matches_bernoulli_taylor_series(N):
    # (f_BE(x) - 1/x - 1/2)/x = sum_n B_{2n+2}/(2n+2)! x^{2n}; the [N-1/N] Pade in x^2
    # reproduces the first 2N coefficients exactly.
    sympy = pytest.importorskip("sympy")
    xi, eta = bcf.pade_bose_poles(N)
    B = [float(sympy.bernoulli(k)) for k in range(4 * N + 4)]
    for n in range(2 * N):
        exact = B[2 * n + 2] / factorial(2 * n + 2)
        approx = sum(2 * eta[j] * (-1) ** n / xi[j] ** (2 * n + 2) for j in range(N))
        assert abs(approx - exact) <= 1e-9 * abs(exact)
    if N > 3:
        return
    # and not the next one (it is a genuine [N-1/N] approximant)
    exact = B[4 * N + 2] / factorial(4 * N + 2)
    approx = sum(2 * eta[j] * (-1) ** (2 * N) / xi[j] ** (4 * N + 2) for j in range(N))
    assert abs(approx - exact) > 1e-6 * abs(exact)


def test_pade_low_poles_tend_to_matsubara():
    xi, eta = bcf.pade_bose_poles(12)
    assert abs(xi[0] - 2 * np.pi) < 1e-10
    assert abs(xi[1] - 4 * np.pi) < 1e-8
    assert abs(eta[0] - 1.0) < 1e-10


def _quad_bcf(J, beta, t):
    """C(t) = int_0^inf J(w) [coth(beta w/2) cos(wt) - i sin(wt)] dw by QUADPACK QAWF."""
    re = integrate.quad(lambda w: J(w) / np.tanh(beta * w / 2) if w > 0 else 2 / beta * 0,
                        1e-12, np.inf, weight="cos", wvar=t, limlst=200)[0]
    # the integrand is regular at 0: J(w) coth(beta w/2) -> 2 J'(0)/beta
    im = -integrate.quad(J, 0, np.inf, weight="sin", wvar=t, limlst=200)[0]
    return re + 1j * im


@pytest.mark.parametrize("t", [0.5, 1.0, 2.5])
def test_drude_matsubara_sum_equals_quadrature(t):
    lam, wc, beta = 0.5, 1.0, 1.0
    feats = bcf.bath_features(beta, dl=(lam, wc), n_ltc=400, scheme="matsubara")
    C, Cs = bcf.bcf_from_features(feats, np.array([t]))
    ref = _quad_bcf(lambda w: bcf.J_dl(w, lam, wc), beta, t)
    assert abs(C[0] - ref) < 1e-6
    assert abs(Cs[0] - np.conj(ref)) < 1e-6


@pytest.mark.parametrize("t", [0.5, 2.0, 6.0])
def test_brownian_matsubara_sum_equals_quadrature(t):
    lam, w0p, eta, beta = 0.1, 2.0, 0.3, 1.5
    feats = bcf.bath_features(beta, bo=[(lam, w0p, eta)], n_ltc=400, scheme="matsubara")
    C, Cs = bcf.bcf_from_features(feats, np.array([t]))
    ref = _quad_bcf(lambda w: bcf.J_bo(w, lam, w0p, eta), beta, t)
    assert abs(C[0] - ref) < 1e-7
    assert abs(Cs[0] - np.conj(ref)) < 1e-7


def test_pade_features_within_pade_error():
    # C from the Pade features differs from the exact C(t) only through the Pade
    # error of f_BE; with N = 3 and beta*omega_c = 1 that is below 1e-3 for t >= 0.5.
    lam, wc, beta = 0.5, 1.0, 1.0
    feats = bcf.bath_features(beta, dl=(lam, wc), n_ltc=3, scheme="pade")
    assert len(feats) == 4
    ts = np.array([0.5, 1.0, 2.0, 4.0])
    C, _ = bcf.bcf_from_features(feats, ts)
    for t, c in zip(ts, C):
        ref = _quad_bcf(lambda w: bcf.J_dl(w, lam, wc), beta, t)
        assert abs(c - ref) < 1e-3 * abs(ref) + 1e-4


def test_drude_pole_feature_closed_form():
    # c = lam wc (cot(beta wc / 2) - i), gamma = -wc (residue at w = -i wc)
    lam, wc, beta = 0.7, 1.3, 0.9
    (c, cb, g), = bcf.bath_features(beta, dl=(lam, wc))
    assert abs(c - lam * wc * (1 / np.tan(beta * wc / 2) - 1j)) < 1e-13
    assert abs(cb - np.conj(c)) < 1e-15 and g == -wc
