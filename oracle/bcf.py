"""Bath-correlation-function features -- TEST INFRASTRUCTURE ONLY (oracle).

The BCF is C(t) = int_{-inf}^{inf} J(w) f_BE(beta w) exp(-i w t) dw with J the
odd extension of the spectral density and f_BE(x) = 1/(1 - exp(-x)) (Sec. 2.1,
Eqs. 2-3). Closing the contour in the lower half plane gives the residue sum of
Eq. bcfdecores: one feature per lower-half-plane pole of J and one per pole of
f_BE. Every feature is a triple (c_k, cbar_k, gamma_k) with
C(t) = sum_k c_k exp(gamma_k t) and C*(t) = sum_k cbar_k exp(gamma_k t).

Pinned by tests/test_oracle_bcf.py: Pade Taylor coefficients against the
Bernoulli series of f_BE, Matsubara limit, and the feature sums against direct
quadrature of the defining integral.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

Feature = Tuple[complex, complex, complex]  # (c, cbar, gamma)


def f_be(x):
    """f_BE(x) = 1 / (1 - exp(-x)) for complex x (Sec. 2.1)."""
    return 1.0 / (1.0 - np.exp(-x))


def pade_bose_poles(N: int) -> Tuple[np.ndarray, np.ndarray]:
    """[N-1/N] Pade spectrum decomposition of the Bose function (Hu, Xu, Yan 2010,
    cited as the Pade option of Eq. bcfdecores):

        f_BE(x) ~ 1/x + 1/2 + sum_j 2 eta_j x / (x^2 + xi_j^2).

    The xi_j are 2/lambda for the positive eigenvalues lambda of the 2N x 2N
    symmetric tridiagonal matrix with off-diagonal 1/sqrt((2m+1)(2m+3)); the
    zeros zeta_k of the numerator come the same way from the (2N-1) x (2N-1)
    matrix with off-diagonal 1/sqrt((2m+3)(2m+5)); the residues are
    eta_j = N(2N+3)/2 * prod_k (zeta_k^2 - xi_j^2) / prod_{k != j} (xi_k^2 - xi_j^2).
    """
    if N <= 0:
        return np.zeros(0), np.zeros(0)
    m = np.arange(1, 2 * N)
    A = np.diag(1.0 / np.sqrt((2 * m + 1) * (2 * m + 3)), 1)
    ev = np.linalg.eigvalsh(A + A.T)
    xi = np.sort(2.0 / ev[ev > 0])
    if N > 1:
        m = np.arange(1, 2 * N - 1)
        B = np.diag(1.0 / np.sqrt((2 * m + 3) * (2 * m + 5)), 1)
        ev = np.linalg.eigvalsh(B + B.T)
        zeta = np.sort(2.0 / ev[ev > 1e-12])
    else:
        zeta = np.zeros(0)
    eta = np.empty(N)
    for j in range(N):
        num = np.prod(zeta ** 2 - xi[j] ** 2)
        den = np.prod([xi[k] ** 2 - xi[j] ** 2 for k in range(N) if k != j])
        eta[j] = N * (2 * N + 3) / 2.0 * num / den
    return xi, eta


def matsubara_bose_poles(N: int) -> Tuple[np.ndarray, np.ndarray]:
    """Matsubara expansion of f_BE: xi_j = 2 pi j, eta_j = 1 (Eq. bcfdecores)."""
    j = np.arange(1, N + 1)
    return 2.0 * np.pi * j, np.ones(N)


def bose_poles(N: int, scheme: str):
    if scheme == "pade":
        return pade_bose_poles(N)
    if scheme == "matsubara":
        return matsubara_bose_poles(N)
    raise ValueError(scheme)


def J_dl(w, lam, wc):
    """Drude-Lorentz spectral density, Eq. DL (odd in w)."""
    return (2.0 * lam / np.pi) * wc * w / (w ** 2 + wc ** 2)


def J_bo(w, lam, w0p, eta):
    """Brownian oscillator in the factored form used by TENSO (Eq. BO, second form)."""
    W2 = w0p ** 2 + eta ** 2
    return (4.0 * lam * eta / np.pi) * W2 * w / (((w + w0p) ** 2 + eta ** 2) * ((w - w0p) ** 2 + eta ** 2))


def bath_features(beta: float, dl=None, bo=(), n_ltc: int = 0, scheme: str = "pade") -> List[Feature]:
    """All features of one bath with J = J_DL + sum_b J_BO^(b) (Sec. 2.1).

    J-pole features (residue at each lower-half-plane pole z of J, term
    -2 pi i Res J(z) f_BE(beta z) exp(-i z t)):
      * DL pole z = -i wc: Res = lam wc / pi, so c = -2 i lam wc f_BE(-i beta wc),
        gamma = -wc, and cbar = conj(c) because gamma is real.
      * BO poles z = +-w0' - i eta: Res = +-i lam W2 / (2 pi w0') with
        W2 = w0'^2 + eta^2, giving c+ = (lam W2/w0') f_BE(beta(w0' - i eta)),
        gamma+ = -eta - i w0' and c- = -(lam W2/w0') f_BE(-beta(w0' + i eta)),
        gamma- = -eta + i w0'. C* pairs the conjugate exponents:
        cbar+ = conj(c-), cbar- = conj(c+).
    Bose-pole features (pole of f_BE(beta w) at w = -i nu_j, nu_j = xi_j / beta,
    residue eta_j / beta): c_j = -2 pi i (eta_j / beta) J(-i nu_j), real, so
    cbar_j = c_j, gamma_j = -nu_j; the contributions of all J components share
    one feature per pole.
    """
    feats: List[Feature] = []
    if dl is not None:
        lam, wc = dl
        c = -2j * lam * wc * f_be(-1j * beta * wc)
        feats.append((complex(c), complex(np.conj(c)), complex(-wc)))
    for (lam, w0p, eta) in bo:
        W2 = w0p ** 2 + eta ** 2
        cp = (lam * W2 / w0p) * f_be(beta * (w0p - 1j * eta))
        cm = -(lam * W2 / w0p) * f_be(-beta * (w0p + 1j * eta))
        feats.append((complex(cp), complex(np.conj(cm)), complex(-eta - 1j * w0p)))
        feats.append((complex(cm), complex(np.conj(cp)), complex(-eta + 1j * w0p)))
    xi, eta_res = bose_poles(n_ltc, scheme)
    for j in range(n_ltc):
        nu = xi[j] / beta
        Jv = 0.0
        if dl is not None:
            Jv = Jv + J_dl(-1j * nu, *dl)
        for (lam, w0p, eta) in bo:
            Jv = Jv + J_bo(-1j * nu, lam, w0p, eta)
        c = -2j * np.pi * (eta_res[j] / beta) * Jv
        c = complex(np.real(c))  # exactly real: J(-i nu) is purely imaginary
        feats.append((c, c, complex(-nu)))
    return feats


def bcf_from_features(feats: List[Feature], t):
    """C(t) and C*(t) from the features (Eq. bcfdecores, last line)."""
    t = np.asarray(t, dtype=float)
    C = np.zeros(t.shape, np.complex128)
    Cs = np.zeros(t.shape, np.complex128)
    for c, cb, g in feats:
        C += c * np.exp(g * t)
        Cs += cb * np.exp(g * t)
    return C, Cs
