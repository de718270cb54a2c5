"""ML-MCTDH star-bath generator for the oracle -- TEST INFRASTRUCTURE ONLY (oracle).

The thermofield representation of a thermal harmonic bath (the wavefunction
method TENSO runs on the same tensor-network machinery, Sec. 3.2.4): modes at
the midpoints w_k of n equal intervals of [-cutoff, cutoff]; mode k couples
with g_k^2 = J(|w_k|) dw (1 + n(|w_k|)) for w_k > 0 and J(|w_k|) dw n(|w_k|)
for w_k < 0 (n the Bose occupation), J the factored Brownian density of Eq. BO
(oracle.bcf.J_bo). Terms of the generator -i H, H = H_S + sum w_k a^+a +
Q sum g_k (a + a^+), on legs (0 = system, 1 = spectator, 2.. = modes), as
oracle.sop.Term objects for oracle.ttn.TTN.

Pinned by tests/test_oracle_mctdh.py: the discretised correlation function
against the quadrature of Eq. 2, and the TTN at untruncated ranks against the
exact exponential of H on a small case.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import bcf
from .sop import Term


def modes(bo, beta: float, cutoff: float, n: int):
    if n < 2 or n % 2:
        raise ValueError("an even number of modes (no mode at zero frequency)")
    dw = 2.0 * cutoff / n
    w = np.array([-cutoff + (k + 0.5) * dw for k in range(n)])
    g = np.zeros(n)
    for k in range(n):
        a = abs(w[k])
        J = sum(bcf.J_bo(a, lam, w0, eta) for (lam, w0, eta) in bo)
        nb = 1.0 / (np.exp(beta * a) - 1.0)
        g[k] = np.sqrt(J * dw * ((1.0 + nb) if w[k] > 0 else nb))
    return w, g


def terms(H, Q, w, g, dim: int) -> List[Term]:
    n = np.arange(dim)
    num = np.diag(n).astype(np.complex128)
    x = np.zeros((dim, dim), np.complex128)
    for m in range(1, dim):
        x[m - 1, m] = x[m, m - 1] = np.sqrt(m)
    out = [Term(-1j, {0: np.asarray(H, np.complex128)})]
    for k in range(len(w)):
        out.append(Term(-1j * w[k], {2 + k: num}))
        out.append(Term(-1j * g[k], {0: np.asarray(Q, np.complex128), 2 + k: x}))
    return out


def rho0(psi0) -> np.ndarray:
    """Root initial tensor input: rho0[i][j] = psi0[i] delta_{j0}."""
    M = len(psi0)
    r = np.zeros((M, M), np.complex128)
    r[:, 0] = psi0
    return r


def system_rho(st) -> np.ndarray:
    """rho_S of the wavefunction: trace over the modes of |psi><psi| (dense
    contraction of the whole tree, small cases) -- spectator index 0."""
    full = st.full_tensor()[:, 0]
    v = full.reshape(full.shape[0], -1)
    return v @ v.conj().T


def system_rho_root(st) -> np.ndarray:
    """The same from the root tensor alone: with every non-root node
    semi-unitary toward its parent the subtree states are orthonormal, so
    rho[i, i'] = sum_a A[i, 0, a] conj(A[i', 0, a])."""
    A = st.tensors[0]
    v = A[:, 0, :]
    return v @ v.conj().T
