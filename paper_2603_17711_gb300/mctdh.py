"""ML-MCTDH (wavefunction) generators for the TTN library: the thermofield
star bath of Sec. 3.2.4 (TENSO's extension of its tensor-network machinery to
the time-dependent Schroedinger equation), built as sop_load arrays.

A bath with spectral density J (here Brownian peaks in the factored form of
Eq. BO) at inverse temperature beta is represented at zero temperature by
modes of frequency w in [-cutoff, cutoff] (thermofield doubling): the mode at
w > 0 carries the coupling density J(w)(n(w) + 1), the one at -w the density
J(w) n(w), n the Bose occupation, so that sum_k g_k^2 exp(-i w_k t) is the
thermal correlation function int_0^inf J(w)[coth(beta w/2) cos(wt) - i sin(wt)] dw
up to the discretisation. The frequencies are the midpoints of n equal
intervals; g_k^2 = density(w_k) dw.

The generator of d psi/dt = -i H psi with
    H = H_S (x) 1 + sum_k w_k a_k^+ a_k + Q (x) sum_k g_k (a_k + a_k^+)
acts on leg 0 (the system); leg 1 is a spectator of the same dimension that no
operator touches (the library's root carries two system legs), and the state
is loaded as rho0[i][j] = psi0[i] delta_{j0}. Legs 2.. are the modes.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

from .heom import SOPBuilder


def j_brownian(w, peaks: Sequence[Tuple[float, float, float]]):
    """J(w) = sum (4 lam eta / pi) (w0^2 + eta^2) w / ([(w + w0)^2 + eta^2][(w - w0)^2 + eta^2]) (Eq. BO, factored)."""
    w = np.asarray(w, float)
    out = np.zeros_like(w)
    for lam, w0, eta in peaks:
        out += 4.0 * lam * eta / np.pi * (w0 * w0 + eta * eta) * w / (((w + w0) ** 2 + eta ** 2) * ((w - w0) ** 2 + eta ** 2))
    return out


def thermofield_modes(peaks, beta: float, cutoff: float, n: int) -> Tuple[np.ndarray, np.ndarray]:
    """(frequencies, couplings) of the n thermofield modes on [-cutoff, cutoff];
    n even, so that no midpoint falls on zero frequency."""
    if n < 2 or n % 2:
        raise ValueError("n must be even")
    dw = 2.0 * cutoff / n
    w = -cutoff + dw * (np.arange(n) + 0.5)
    a = np.abs(w)
    occ = 1.0 / np.expm1(beta * a)
    dens = j_brownian(a, peaks) * np.where(w > 0, occ + 1.0, occ)
    return w, np.sqrt(dens * dw)


def mctdh_sop(H, Q, freqs, couplings, dim: int) -> dict:
    """sop_load arrays of -i H for the star bath (modes on legs 2..)."""
    H = np.asarray(H, np.complex128)
    M = H.shape[0]
    b = SOPBuilder([M, M] + [dim] * len(freqs))
    b.term(-1j, [b.op(0, H)])
    q = b.op(0, np.asarray(Q, np.complex128))
    n = np.arange(dim)
    a = np.diag(np.sqrt(n[1:].astype(float)), 1).astype(np.complex128)
    for k, (w, g) in enumerate(zip(freqs, couplings)):
        leg = 2 + k
        b.term(-1j * w, [b.op(leg, np.diag(n.astype(np.complex128)))])
        b.term(-1j * g, [q, b.op(leg, a + a.T)])
    return b.arrays()


def rho_from_root(A: np.ndarray) -> np.ndarray:
    """System density matrix of the wavefunction, from the root tensor (i, j, a)
    with every other node semi-unitary toward its parent: the subtree states are
    orthonormal, so rho[i, i'] = sum_a A[i, 0, a] conj(A[i', 0, a])."""
    v = A[:, 0, :]
    return v @ v.conj().T
