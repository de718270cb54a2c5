"""Brute-force dense hierarchy -- TEST INFRASTRUCTURE ONLY (oracle).

The full EDO Omega[i, j, n_1..n_K] is stored as one vector (row-major over
(i, j, n_1, ..., n_K)) and propagated with dOmega/dt = L(t) Omega (Eq. EDO-eom),
L the sum of the product terms of Eq. master_lvn written as sparse Kronecker
products. rho_S = Omega[:, :, 0, ..., 0] (Sec. 2.2, rho_S = <0|Omega>).

Feasible up to ~1e7 amplitudes. Pinned by tests/test_oracle_dense.py against
the closed forms for lambda = 0 (unitary dynamics) and pure dephasing, and by
trace conservation.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply


def leg_dims(M: int, depth: Sequence[int]):
    return [M, M] + list(depth)


def term_matrix(term, dims) -> sp.csr_matrix:
    """coef-free Kronecker product of the term's factors (identity elsewhere)."""
    out = sp.identity(1, dtype=np.complex128, format="csr")
    for leg, d in enumerate(dims):
        op = term.ops.get(leg)
        f = sp.csr_matrix(op) if op is not None else sp.identity(d, dtype=np.complex128, format="csr")
        out = sp.kron(out, f, format="csr")
    return out


def generator(terms, dims, drive_values: Optional[Sequence[float]] = None) -> sp.csr_matrix:
    """L = sum_m coef_m (g_d(t) for driven terms) * kron(factors)."""
    n = int(np.prod(dims))
    L = sp.csr_matrix((n, n), dtype=np.complex128)
    for t in terms:
        c = t.coef
        if t.drive is not None:
            c = c * drive_values[t.drive]
        L = L + c * term_matrix(t, dims)
    return L.tocsr()


def initial_vector(rho0: np.ndarray, depth: Sequence[int]) -> np.ndarray:
    """Omega(0) = rho0 (x) |0...0> (Sec. 2.2)."""
    M = rho0.shape[0]
    dims = leg_dims(M, depth)
    Om = np.zeros(dims, np.complex128)
    Om[(slice(None), slice(None)) + (0,) * len(depth)] = rho0
    return Om.reshape(-1)


def rdm(vec: np.ndarray, M: int, depth: Sequence[int]) -> np.ndarray:
    Om = vec.reshape(leg_dims(M, depth))
    return Om[(slice(None), slice(None)) + (0,) * len(depth)].copy()


def propagate(terms, rho0, depth, dt: float, n_steps: int,
              drives: Sequence = (), rk4_sub: int = 64):
    """rho_S at t = 0, dt, ..., n_steps*dt. Autonomous generators use
    scipy's expm_multiply; driven ones classical RK4 with ``rk4_sub`` substeps per dt."""
    M = rho0.shape[0]
    dims = leg_dims(M, depth)
    v = initial_vector(rho0, depth)
    out = [rdm(v, M, depth)]
    if not drives:
        L = generator(terms, dims)
        traj = expm_multiply(L, v, start=0.0, stop=dt * n_steps, num=n_steps + 1, endpoint=True)
        return np.array([rdm(x, M, depth) for x in traj])
    h = dt / rk4_sub
    L0 = generator([t for t in terms if t.drive is None], dims)
    Ld = [generator([dataclasses.replace(t, drive=None) for t in terms if t.drive == d], dims)
          for d in range(len(drives))]

    def L_at(t):
        return L0 + sum(dr.g(t) * Ld[d] for d, dr in enumerate(drives))

    t = 0.0
    for _ in range(n_steps):
        for _ in range(rk4_sub):
            L1 = L_at(t + h / 2)
            k1 = L_at(t) @ v
            k2 = L1 @ (v + 0.5 * h * k1)
            k3 = L1 @ (v + 0.5 * h * k2)
            k4 = L_at(t + h) @ (v + h * k3)
            v = v + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
            t += h
        out.append(rdm(v, M, depth))
    return np.array(out)
