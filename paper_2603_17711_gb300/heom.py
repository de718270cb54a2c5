"""Host-side model building for the TTN-HEOM library (not on the GPU hot path).

Turns physical parameters into the arrays that ``sop_load`` takes:

* bath features (c_k, cbar_k, gamma_k) from the residue decomposition of the
  bath correlation function C(t) = int J(w) f_BE(beta w) exp(-i w t) dw
  (Sec. 2.1, Eq. bcfdecores) for Drude-Lorentz (Eq. DL) and factored Brownian
  (Eq. BO) spectral densities, with Pade (Hu-Xu-Yan) or Matsubara Bose poles;
* the 5K+2 product terms of the bexcitonic HEOM generator (Eq. heom-std,
  Eq. dissipator, Eq. master_lvn) with the 'abs' metric z_k = f_k,
  f_k = sqrt((|c_k| + |cbar_k|)/2) (Sec. 7.4), packed for the C ABI.

Each distinct local operator is registered once per leg (Q_b and conj(Q_b) on
the system legs once per bath), which lets the library group the two-leg
terms of one bath behind a shared factor.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def _bose(x):
    return 1.0 / (1.0 - np.exp(-x))


def bose_poles(n: int, scheme: str = "pade") -> Tuple[np.ndarray, np.ndarray]:
    """Poles xi_j and residues eta_j of f_BE(x) ~ 1/x + 1/2 + sum_j 2 eta_j x/(x^2 + xi_j^2)."""
    if n <= 0:
        return np.zeros(0), np.zeros(0)
    if scheme == "matsubara":
        return 2.0 * np.pi * np.arange(1, n + 1), np.ones(n)
    if scheme != "pade":
        raise ValueError(f"unknown decomposition scheme {scheme!r}")

    def tri_eigs(size: int, first: int) -> np.ndarray:
        k = np.arange(size - 1)
        off = 1.0 / np.sqrt((2 * (k + first) + 1.0) * (2 * (k + first) + 3.0))
        T = np.diag(off, 1) + np.diag(off, -1)
        ev = np.linalg.eigvalsh(T)
        return np.sort(2.0 / ev[ev > 1e-12])

    xi = tri_eigs(2 * n, 1)            # off-diagonal 1/sqrt((2m+1)(2m+3)), m = 1..2n-1
    zeta = tri_eigs(2 * n - 1, 2) if n > 1 else np.zeros(0)  # 1/sqrt((2m+3)(2m+5))
    xi2, z2 = xi ** 2, zeta ** 2
    eta = np.empty(n)
    for j in range(n):
        others = np.delete(xi2, j)
        eta[j] = 0.5 * n * (2 * n + 3) * np.prod(z2 - xi2[j]) / np.prod(others - xi2[j])
    return xi, eta


def features(beta: float, dl=None, bo: Sequence = (), n_ltc: int = 0, scheme: str = "pade") -> np.ndarray:
    """(K, 3) complex array of (c, cbar, gamma), ordered: Drude pole, Brownian
    (+, -) pairs, then Bose poles."""
    rows: List[Tuple[complex, complex, complex]] = []
    if dl is not None:
        lam, wc = dl
        # -2 pi i Res_{w=-i wc} J_DL = -2 i lam wc; times f_BE(-i beta wc)
        c = -2j * lam * wc * _bose(-1j * beta * wc)
        rows.append((c, np.conj(c), -wc))
    for lam, w0, eta in bo:
        amp = lam * (w0 * w0 + eta * eta) / w0
        cp = amp * _bose(beta * (w0 - 1j * eta))
        cm = -amp * _bose(-beta * (w0 + 1j * eta))
        rows.append((cp, np.conj(cm), -eta - 1j * w0))
        rows.append((cm, np.conj(cp), -eta + 1j * w0))
    xi, res = bose_poles(n_ltc, scheme)
    for x, r in zip(xi, res):
        nu = x / beta
        z = -1j * nu
        J = 0.0
        if dl is not None:
            lam, wc = dl
            J += 2.0 * lam / np.pi * wc * z / (z * z + wc * wc)
        for lam, w0, eta in bo:
            J += 4.0 * lam * eta / np.pi * (w0 * w0 + eta * eta) * z / (((z + w0) ** 2 + eta ** 2) * ((z - w0) ** 2 + eta ** 2))
        c = (-2j * np.pi * r / beta * J).real
        rows.append((c, c, -nu))
    return np.array(rows, dtype=np.complex128).reshape(-1, 3)


class SOPBuilder:
    """Collects local operators and product terms in the layout of sop_load."""

    def __init__(self, leg_dims: Sequence[int]):
        self.leg_dims = list(leg_dims)
        self.ops: List[np.ndarray] = []
        self.op_leg: List[int] = []
        self._index: Dict[Tuple[int, bytes], int] = {}
        self.terms: List[Tuple[complex, List[int], int]] = []

    def op(self, leg: int, M: np.ndarray) -> int:
        M = np.ascontiguousarray(M, dtype=np.complex128)
        d = self.leg_dims[leg]
        if M.shape != (d, d):
            raise ValueError(f"operator on leg {leg} must be {d}x{d}")
        key = (leg, M.tobytes())
        if key not in self._index:
            self._index[key] = len(self.ops)
            self.ops.append(M)
            self.op_leg.append(leg)
        return self._index[key]

    def term(self, coef: complex, op_ids: Sequence[int], drive: int = -1) -> None:
        self.terms.append((complex(coef), list(op_ids), int(drive)))

    def arrays(self) -> dict:
        offs, acc = [], 0
        for M in self.ops:
            offs.append(acc)
            acc += M.size
        data = np.concatenate([M.reshape(-1) for M in self.ops]) if self.ops else np.zeros(0, np.complex128)
        toff = np.zeros(len(self.terms) + 1, np.int32)
        tops: List[int] = []
        coef = np.zeros(2 * len(self.terms))
        drv = np.zeros(len(self.terms), np.int32)
        for m, (c, ids, d) in enumerate(self.terms):
            tops += ids
            toff[m + 1] = len(tops)
            coef[2 * m], coef[2 * m + 1] = c.real, c.imag
            drv[m] = d
        return dict(op_leg=np.array(self.op_leg, np.int32), op_offset=np.array(offs, np.int64),
                    op_data=np.ascontiguousarray(np.stack([data.real, data.imag], -1).reshape(-1)),
                    term_offsets=toff, term_ops=np.array(tops, np.int32), coef=coef, coef_drive=drv)


def heom_sop(H: np.ndarray, baths: Sequence, depth: Sequence[int], drives: Sequence = ()) -> dict:
    """sop_load arrays of -i H_S^x(t) + sum_k D_k (Eq. heom-std, Eq. dissipator).

    ``baths``: objects with Q, beta, dl, bo, n_ltc, scheme; ``drives``: objects
    with V (g(t) is registered separately with ttn_set_drive, drive id = index).
    """
    H = np.asarray(H, np.complex128)
    M = H.shape[0]
    b = SOPBuilder([M, M] + list(depth))
    b.term(-1j, [b.op(0, H)])
    b.term(1j, [b.op(1, H.conj())])
    for d, dr in enumerate(drives):
        V = np.asarray(dr.V, np.complex128)
        b.term(-1j, [b.op(0, V)], drive=d)
        b.term(1j, [b.op(1, V.conj())], drive=d)
    leg = 2
    for bath in baths:
        Q = np.asarray(bath.Q, np.complex128)
        qi, qj = b.op(0, Q), b.op(1, Q.conj())
        for c, cb, g in features(bath.beta, bath.dl, bath.bo, bath.n_ltc, bath.scheme):
            N = depth[leg - 2]
            n = np.arange(N)
            lower = np.diag(np.sqrt(n[1:].astype(float)), 1).astype(np.complex128)  # a
            f = np.sqrt(0.5 * (abs(c) + abs(cb)))
            f = f if f > 0 else 1.0
            raise_op = b.op(leg, lower.T / f)      # z^-1 a^dagger
            lower_op = b.op(leg, lower * f)        # a z
            b.term(g, [b.op(leg, np.diag(n.astype(np.complex128)))])
            b.term(c, [qi, raise_op])
            b.term(-cb, [qj, raise_op])
            b.term(-1.0, [qi, lower_op])
            b.term(1.0, [qj, lower_op])
            leg += 1
    if leg - 2 != len(depth):
        raise ValueError("depth list does not match the number of features")
    return b.arrays()
