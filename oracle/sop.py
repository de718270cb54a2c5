"""Sum-of-products terms of the bexcitonic HEOM generator -- TEST INFRASTRUCTURE ONLY (oracle).

Eq. heom-std: d|Omega>/dt = (-i H_S^x(t) + sum_k D_k)|Omega>, with the convention
A^x B = A^> B - A^< B = A B - B A^dagger (Sec. 2.2), and Eq. dissipator:

    D_k = gamma_k a_k^+ a_k + (c_k Q^> - cbar_k Q^<) z_k^{-1} a_k^+ - Q^x a_k z_k.

On the element array Omega[i, j, n_1, ..., n_K] (Eq. EDO-elements) a left
product A^> acts on leg i with the matrix A; a right product A^< B = B A^dagger
acts on leg j with the matrix conj(A). The Fock legs carry the truncated number
basis n = 0..N_k-1 with a|n> = sqrt(n)|n-1>. Expanding gives exactly 5K + 2
product terms (Eq. master_lvn):

    leg i : -i H_S                                    (1 term)
    leg j : +i conj(H_S)                              (1 term)
    per feature k of the bath with coupling Q_b:
      leg k          : gamma_k n                      (1)
      legs (i, k)    : c_k   Q       x z^{-1} a^+     (1)
      legs (j, k)    : -cbar_k conj(Q) x z^{-1} a^+   (1)
      legs (i, k)    : -1    Q       x a z            (1)
      legs (j, k)    : +1    conj(Q) x a z            (1)

A time-dependent system term g_d(t) V_d adds -i g_d V_d on leg i and
+i g_d conj(V_d) on leg j.

The metric z_k is diagonal in n (Sec. 7.4): ``'abs'`` uses the constant
z = f_k with f_k = sqrt((|c_k| + |cbar_k|)/2) (Listing custommetric; f_k = 1
when c_k = cbar_k = 0, where the abs rule would give a singular metric);
``'conventional'`` uses z(n) = i n^{-1/2} (z(0) = i), the conventional HEOM
(Sec. 2.2); a number uses that constant.

Pinned by tests/test_oracle_sop.py: the dense generator built from these terms
against an independently written textbook HEOM in ADM-index form, the count of
5K+2 terms, and metric independence of rho_S.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import bcf


@dataclasses.dataclass
class Term:
    """coef * prod_{leg} ops[leg]; ``drive`` = index d if coef is multiplied by g_d(t)."""
    coef: complex
    ops: Dict[int, np.ndarray]
    drive: Optional[int] = None


def ladder(N: int):
    """Truncated annihilation operator a (N x N): a|n> = sqrt(n)|n-1>."""
    a = np.zeros((N, N), np.complex128)
    for n in range(1, N):
        a[n - 1, n] = np.sqrt(n)
    return a


def metric_diag(N: int, c: complex, cb: complex, metric) -> np.ndarray:
    """Diagonal of z_k in the number basis (Sec. 7.4)."""
    if metric == "abs":
        f = np.sqrt((abs(c) + abs(cb)) / 2.0)
        # a feature with c = cbar = 0 never feeds the hierarchy; any invertible
        # metric gives the same rho_S, take z = 1 there
        return np.full(N, f if f > 0 else 1.0, np.complex128)
    if metric == "conventional":
        z = np.empty(N, np.complex128)
        z[0] = 1j
        for n in range(1, N):
            z[n] = 1j / np.sqrt(n)
        return z
    return np.full(N, complex(metric), np.complex128)


def heom_terms(H: np.ndarray, baths: Sequence, depth: Sequence[int], metric="abs",
               drives: Sequence = ()) -> List[Term]:
    """All 5K+2 (+2 per drive) product terms of Eq. master_lvn.

    ``baths`` are objects with attributes Q, beta, dl, bo, n_ltc, scheme;
    features are taken from oracle.bcf in bath order.
    """
    terms: List[Term] = [Term(-1j, {0: np.asarray(H, np.complex128)}),
                         Term(+1j, {1: np.conj(np.asarray(H, np.complex128))})]
    for d, dr in enumerate(drives):
        V = np.asarray(dr.V, np.complex128)
        terms.append(Term(-1j, {0: V}, drive=d))
        terms.append(Term(+1j, {1: np.conj(V)}, drive=d))
    k = 0
    for b in baths:
        Q = np.asarray(b.Q, np.complex128)
        feats = bcf.bath_features(b.beta, b.dl, b.bo, b.n_ltc, b.scheme)
        for (c, cb, g) in feats:
            N = depth[k]
            leg = 2 + k
            a = ladder(N)
            z = np.diag(metric_diag(N, c, cb, metric))
            zinv = np.diag(1.0 / np.diag(z))
            Ap = zinv @ a.conj().T      # z^{-1} a^+
            Am = a @ z                  # a z
            num = np.diag(np.arange(N, dtype=np.complex128))
            terms.append(Term(g, {leg: num}))
            terms.append(Term(c, {0: Q, leg: Ap}))
            terms.append(Term(-cb, {1: np.conj(Q), leg: Ap}))
            terms.append(Term(-1.0, {0: Q, leg: Am}))
            terms.append(Term(+1.0, {1: np.conj(Q), leg: Am}))
            k += 1
    return terms


def lambda_bound(terms: Sequence[Term], drive_bounds: Sequence[float] = ()) -> float:
    """Static bound Lambda = sum_terms |coef| prod_legs ||op||_2 on the norm of
    every projected node or bond operator (environments of isometries do not
    increase operator norms). Time-dependent terms use |coef| * max|g_d|."""
    lam = 0.0
    for t in terms:
        v = abs(t.coef)
        if t.drive is not None:
            v *= drive_bounds[t.drive]
        for op in t.ops.values():
            v *= np.linalg.norm(op, 2)
        lam += v
    return lam


def n_substeps(tau: float, lam: float, kappa: float = 2.5) -> int:
    """m = max(1, ceil(|tau| Lambda / kappa - 1e-9)) classical RK4 substeps for a
    flow of length tau (kappa = 2.5 lies inside RK4's real-axis stability limit
    2.785; the 1e-9 keeps an exact integer ratio from rounding up)."""
    return max(1, int(np.ceil(abs(tau) * lam / kappa - 1e-9)))
