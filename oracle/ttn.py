"""Tree tensor network propagation of the HEOM -- TEST INFRASTRUCTURE ONLY (oracle).

Plain numpy complex128 restatement of the TTN-HEOM hot path (Sec. 2.3):

* State. Omega = Con(A^(0), U^(1), ...) (Eq. omega_tensor and the general-tree
  form after it). Every node tensor is stored with its legs in a canonical
  order: parent bond first (absent at the root), then the children -- child
  nodes and open legs -- sorted by the smallest open-leg index below them. The
  root holds the system legs i, j (Sec. 2.3, after Eq. semiunitary). Non-root
  tensors are semi-unitary toward the parent (Eq. semiunitary) except the node
  that currently carries the weight (the orthogonality centre).
* Environments. For every SOP term m (Eq. master_lvn) and directed bond a->b the
  mean-field matrix E_{a->b}(m)[x', x] = <phi_x'| h_m restricted to the subtree
  behind a |phi_x>, with phi the orthonormal basis that the isometries behind a
  define; ``None`` stands for the identity (the term has no factor there). The
  projected generator on the centre node u is
      H_u U = sum_m coef_m (prod_{legs l of u} E_l(m) x_l) U
  and on a bond matrix R between the from-node and the to-node
      H_e R = sum_m coef_m E_{from->to}(m) R E_{to->from}(m)^T.
  This is the Dirac-Frenkel projection of Eq. EDO-eom onto the tree (Sec. 2.3,
  last two paragraphs); the paper defers the node equations to its Ref. chen2025.
* ps1 (fixed rank projector splitting, Sec. 2.3 last paragraph): the centre
  traverses the tree and every core is propagated while it is the centre.
  Reading taken (the paper defers the exact scheme): the recursive
  Lie-Trotter tree sweep Phi_h (children first, backward bond flows on the way
  up, the node last) and its adjoint Phi*_h, composed symmetrically:
  one step = Phi_{dt/2} then Phi*_{dt/2}; for an autonomous generator the two
  adjacent root flows are merged into one flow of dt. A time-dependent system
  term is frozen at t0 + dt/4 during the first half and t0 + 3dt/4 during the
  second.
* ps2 (adaptive rank, Sec. 2.3 last paragraph and Sec. 7.5): neighbouring cores
  are merged, the pair is propagated, and an SVD splits it back with a
  truncated rank.
* vmf (direct integration, Sec. 2.3 and Sec. 7.5): every node is advanced at
  once by the projected equations of motion in the multilayer-MCTDH form
  (non-root nodes kept semi-unitary, the root carries the weight; the inverse
  of each single-hole density matrix regularised by vmf_atol on its diagonal),
  integrated by dopri5 with the ode_rtol / ode_atol controller. 'mix' runs ps2
  until a bond reaches max_rank, then vmf at the ranks ps2 reached.
* Sub-flows use classical RK4 with m = max(1, ceil(|tau| Lambda / 2.5)) substeps,
  Lambda the static operator-norm bound of oracle.sop.lambda_bound.
* Gauge moves use the Householder QR of ``householder_qr`` (diag(R) real >= 0;
  a column whose remaining norm is at most qr_tol * ||A||_F is taken as exactly
  dependent: no reflector, R_jj = 0, and the Q column is the deterministic
  completion H_0 ... H_{j-1} e_j).

Pinned by tests/test_oracle_ttn.py: untruncated ranks against the dense
hierarchy, pure dephasing at rank >= M^2 against the closed form, TT against
BTT, metric independence, QR against LAPACK, RK4 order; by
tests/test_oracle_vmf.py: dopri5 against expm (fifth order), vmf at untruncated
ranks against the dense hierarchy, vmf exact on the pure-dephasing manifold,
the regularisation, the mixed strategy's switch; by tests/test_oracle_ps2_rule.py:
the ps2 truncation rule and the SVD completion.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import sop as sop_mod


# ----------------------------------------------------------------------------
# Tree structure
# ----------------------------------------------------------------------------

class Tree:
    """Topology: ``parent`` (root 0 has parent -1) and ``leg_node`` (node of each
    open leg). ``legs[u]`` lists the legs of node u in canonical order as tuples
    ('p', parent) | ('n', child node) | ('o', open leg)."""

    def __init__(self, parent: Sequence[int], leg_node: Sequence[int]):
        self.parent = list(parent)
        self.leg_node = list(leg_node)
        n = len(self.parent)
        self.n_nodes = n
        if n < 1 or self.parent[0] != -1:
            raise ValueError("node 0 must be the root with parent -1")
        self.children: List[List[int]] = [[] for _ in range(n)]
        for u in range(1, n):
            p = self.parent[u]
            if not (0 <= p < n) or p == u:
                raise ValueError("bad parent")
            self.children[p].append(u)
        for u in range(n):  # walking up from every node must reach the root
            seen, v = 0, u
            while v != 0:
                v = self.parent[v]
                seen += 1
                if seen > n:
                    raise ValueError("parent array has a cycle")
        self.open_legs: List[List[int]] = [[] for _ in range(n)]
        for l, u in enumerate(self.leg_node):
            if not (0 <= u < n):
                raise ValueError("leg not attached to a node")
            self.open_legs[u].append(l)
        self.below: List[List[int]] = [[] for _ in range(n)]
        for u in self.postorder():
            acc = list(self.open_legs[u])
            for c in self.children[u]:
                acc += self.below[c]
            if not acc:
                raise ValueError("node without open legs below it")
            self.below[u] = sorted(acc)
        self.legs: List[List[Tuple[str, int]]] = []
        for u in range(n):
            items = [(l, ("o", l)) for l in self.open_legs[u]]
            items += [(self.below[c][0], ("n", c)) for c in self.children[u]]
            items.sort(key=lambda x: x[0])
            legs = ([] if u == 0 else [("p", self.parent[u])]) + [it[1] for it in items]
            self.legs.append(legs)
        # child nodes in canonical leg order
        self.children = [[v for (k, v) in self.legs[u] if k == "n"] for u in range(n)]

    def postorder(self) -> List[int]:
        out: List[int] = []

        def rec(u):
            for c in self.children[u]:
                rec(c)
            out.append(u)
        rec(0)
        return out


def effective_ranks(tree: Tree, leg_dims: Sequence[int], requested: Sequence[int]) -> List[int]:
    """Rank cap: each bond (u, parent(u)) keeps min(requested, product of the other
    leg dimensions at either end node), iterated to a fixed point, so that every
    core can be semi-unitary toward any of its legs (Sec. 2.3: a bond rank never
    exceeds the matricisation rank across it)."""
    r = [0] + [int(x) for x in requested[1:tree.n_nodes]]
    for u in range(1, tree.n_nodes):
        if r[u] < 1:
            raise ValueError("rank < 1")

    def dim(u, leg):
        kind, v = leg
        if kind == "p":
            return r[u]
        if kind == "n":
            return r[v]
        return leg_dims[v]

    changed = True
    while changed:
        changed = False
        for c in range(1, tree.n_nodes):
            u = tree.parent[c]
            pc = int(np.prod([dim(c, lg) for lg in tree.legs[c] if lg[0] != "p"]))
            pu = int(np.prod([dim(u, lg) for lg in tree.legs[u] if lg != ("n", c)]))
            new = min(r[c], pc, pu)
            if new != r[c]:
                r[c] = new
                changed = True
    return r


def node_shape(tree: Tree, leg_dims: Sequence[int], ranks: Sequence[int], u: int) -> Tuple[int, ...]:
    return tuple(ranks[u] if kind == "p" else ranks[v] if kind == "n" else leg_dims[v]
                 for kind, v in tree.legs[u])


# ----------------------------------------------------------------------------
# Small linear-algebra steps
# ----------------------------------------------------------------------------

def mode_product(Mx: np.ndarray, U: np.ndarray, axis: int) -> np.ndarray:
    """(M x_axis U)[.., a', ..] = sum_a M[a', a] U[.., a, ..]."""
    return np.moveaxis(np.tensordot(Mx, U, axes=([1], [axis])), 0, axis)


def householder_qr(A: np.ndarray, tol: float) -> Tuple[np.ndarray, np.ndarray]:
    """Householder QR of an m x n complex matrix (m >= n), Golub-Van Loan style.

    For column j with remaining part x (rows j..m-1) of norm alpha:
      * alpha <= tol * ||A||_F: no reflector; the remainder is dropped (R_jj = 0)
        and Q's column j is H_0 ... H_{j-1} e_j.
      * otherwise v = x + phi alpha e_0 with phi = x_0/|x_0| (1 if x_0 = 0),
        H_j = I - 2 v v^H / (v^H v), so H_j x = -phi alpha e_0.
    Finally every row j of R with a reflector is multiplied by conj(s_j) and
    column j of Q by s_j, s_j = R_jj / |R_jj|, so that diag(R) is real >= 0.
    Returns Q (m x n, orthonormal columns) and R (n x n upper triangular),
    Q R = A up to the dropped remainders.
    """
    A = np.array(A, dtype=np.complex128)
    m, n = A.shape
    assert m >= n
    thr = tol * np.linalg.norm(A)
    V = A.copy()
    refl: List[Optional[np.ndarray]] = []
    for j in range(n):
        x = V[j:, j]
        alpha = np.linalg.norm(x)
        if alpha <= thr:
            V[j:, j] = 0.0
            refl.append(None)
            continue
        x0 = x[0]
        phi = x0 / abs(x0) if abs(x0) > 0 else 1.0
        v = x.copy()
        v[0] += phi * alpha
        beta = 2.0 / np.vdot(v, v).real
        V[j:, j:] -= beta * np.outer(v, v.conj() @ V[j:, j:])
        V[j + 1:, j] = 0.0
        refl.append(v)
    R = np.triu(V[:n, :n])
    Q = np.zeros((m, n), np.complex128)
    Q[np.arange(n), np.arange(n)] = 1.0
    for j in reversed(range(n)):
        v = refl[j]
        if v is None:
            continue
        beta = 2.0 / np.vdot(v, v).real
        Q[j:, :] -= beta * np.outer(v, v.conj() @ Q[j:, :])
    for j in range(n):
        if refl[j] is not None and abs(R[j, j]) > 0:
            s = R[j, j] / abs(R[j, j])
            R[j, :] *= np.conj(s)
            Q[:, j] *= s
    return Q, R


def rk4(apply, y: np.ndarray, tau: float, m: int) -> np.ndarray:
    """m classical RK4 substeps (Kutta 1901) of dy/dt = apply(y) over a signed
    interval tau."""
    s = tau / m
    for _ in range(m):
        k1 = apply(y)
        k2 = apply(y + 0.5 * s * k1)
        k3 = apply(y + 0.5 * s * k2)
        k4 = apply(y + s * k3)
        y = y + (s / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return y


# Dormand-Prince 5(4) tableau (Dormand & Prince 1980; the FSAL form of
# Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.5).
DP_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0]
DP_A = [[],
        [1 / 5],
        [3 / 40, 9 / 40],
        [44 / 45, -56 / 15, 32 / 9],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
        [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]]
DP_B5 = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0]
DP_B4 = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]


def dopri5(f, y0: List[np.ndarray], t0: float, t1: float, h_try: float, rtol: float, atol: float,
           max_steps: int = 100000):
    """Integrate dy/dt = f(t, y) from t0 to t1 (y a list of arrays) with the
    Dormand-Prince 5(4) pair and the standard step controller. A step of
    length h = min(h_try, t1 - t) has the scaled RMS error
        err = sqrt(mean(|y5 - y4|^2 / (atol + rtol max(|y_n|, |y_n+1|))^2))
    over all entries; it is accepted when err <= 1, and the trial step becomes
    h * min(5, max(0.2, 0.9 err^(-1/5))) (a shortened step that lands on t1
    does not shrink the trial step). Returns (y(t1), the trial step for the next
    interval, accepted, rejected)."""
    y = [np.array(a, np.complex128) for a in y0]
    t = t0
    acc = rej = 0
    k1 = f(t, y)
    n_steps = 0
    while t1 - t > 1e-13 * max(1.0, abs(t1)):
        n_steps += 1
        if n_steps > max_steps:
            raise RuntimeError("dopri5: too many steps")
        last = h_try >= t1 - t
        h = t1 - t if last else h_try
        ks = [k1]
        for i in range(1, 7):
            yi = [y[j] + h * sum(DP_A[i][l] * ks[l][j] for l in range(i)) for j in range(len(y))]
            ks.append(f(t + DP_C[i] * h, yi))
        y5 = yi  # stage 7 is evaluated at the fifth-order solution (first same as last)
        num, cnt = 0.0, 0
        for j in range(len(y)):
            e = h * sum((DP_B5[l] - DP_B4[l]) * ks[l][j] for l in range(7))
            sc = atol + rtol * np.maximum(np.abs(y[j]), np.abs(y5[j]))
            num += float(np.sum(np.abs(e / sc) ** 2))
            cnt += e.size
        err = float(np.sqrt(num / max(cnt, 1)))
        fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** (-0.2)))
        if err <= 1.0:
            t = t1 if last else t + h
            y = y5
            k1 = ks[6]
            acc += 1
            h_try = max(h_try, h * fac) if last else h * fac
        else:
            rej += 1
            h_try = h * fac
    return y, h_try, acc, rej


def svd_completion(W: np.ndarray, s: np.ndarray, Vh: np.ndarray, tol: float):
    """Kept singular triplets with sigma_i <= tol * sigma_1 are numerically
    undetermined; replace them by a deterministic completion (sigma_i := 0, the
    singular vectors by the Householder completion of the determined ones) so
    that the split does not depend on rounding noise."""
    r = len(s)
    if r == 0:
        return W, s, Vh
    smax = s[0]
    good = s > tol * smax if smax > 0 else np.zeros(r, bool)
    if np.all(good):
        return W, s, Vh
    g = int(np.sum(good))  # singular values are sorted: the determined ones come first
    W2 = _complete_columns(W[:, :g], r)
    V2 = _complete_columns(Vh[:g, :].conj().T, r).conj().T
    s2 = s.copy()
    s2[g:] = 0.0
    return W2, s2, V2


def _complete_columns(Qg: np.ndarray, r: int) -> np.ndarray:
    """The g given orthonormal columns followed by the Householder completion
    H_0..H_{g-1} e_j (j = g..r-1) of their span."""
    m, g = Qg.shape
    A = np.zeros((m, r), np.complex128)
    A[:, :g] = Qg
    Q, _ = householder_qr(A, 0.0)
    out = Q.copy()
    out[:, :g] = Qg
    return out


# ----------------------------------------------------------------------------
# TTN state and sweeps
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    qr_tol: float = 1e-9
    kappa: float = 2.5
    ps2_atol: float = 1e-7
    ps2_ratio: float = 2.0
    max_rank: int = 32
    svd_tol: float = 1e-12
    # vmf (direct integration, Sec. 7.5): dopri5 tolerances (Sec. 4 Table
    # defaults ode_rtol / ode_atol) and the regularisation vmf_atol added to
    # the diagonal of the single-hole density matrix before its inversion
    ode_rtol: float = 1e-5
    ode_atol: float = 1e-7
    vmf_atol: float = 1e-10


class TTN:
    """Tree tensor network carrying the EDO, its per-term environments and the
    SOP terms."""

    def __init__(self, parent, leg_node, leg_dims, ranks, terms, rho0,
                 drives: Sequence = (), params: Optional[Params] = None):
        self.tree = Tree(parent, leg_node)
        self.leg_dims = list(leg_dims)
        if len(self.leg_dims) != len(self.tree.leg_node):
            raise ValueError("leg_dims length")
        if self.tree.leg_node[0] != 0 or self.tree.leg_node[1] != 0:
            raise ValueError("system legs i, j must sit on the root")
        self.params = params or Params()
        self.ranks = effective_ranks(self.tree, self.leg_dims, ranks)
        self.terms = list(terms)
        self.drives = list(drives)
        self.lam = sop_mod.lambda_bound(self.terms, [d.bound for d in self.drives])
        self.t = 0.0
        self.g = [0.0] * len(self.drives)  # frozen drive values of the current half-step
        self.discarded: List[float] = []
        self.tensors = [self._initial_tensor(u, np.asarray(rho0, np.complex128))
                        for u in range(self.tree.n_nodes)]
        self.env: Dict[Tuple[int, int], List[Optional[np.ndarray]]] = {}
        for c in self.tree.postorder():
            if c != 0:
                self.update_env(c, self.tree.parent[c])

    # -- initial product state (Sec. 2.2: Omega(0) = rho0 (x) |0..0>) --------
    def _initial_tensor(self, u: int, rho0: np.ndarray) -> np.ndarray:
        shape = node_shape(self.tree, self.leg_dims, self.ranks, u)
        T = np.zeros(shape, np.complex128)
        if u == 0:
            legs = self.tree.legs[0]
            pi, pj = legs.index(("o", 0)), legs.index(("o", 1))
            M = rho0.shape[0]
            for i in range(M):
                for j in range(M):
                    idx = [0] * len(shape)
                    idx[pi], idx[pj] = i, j
                    T[tuple(idx)] = rho0[i, j]
            return T
        # U[a, flat(children)] = delta(a, flat): the first r columns of the identity
        flat = T.reshape(shape[0], -1)
        for a in range(shape[0]):
            flat[a, a] = 1.0
        return flat.reshape(shape)

    # -- environments ------------------------------------------------------
    def leg_env(self, u: int, li: int, m: int) -> Optional[np.ndarray]:
        kind, v = self.tree.legs[u][li]
        if kind == "o":
            return self.terms[m].ops.get(v)
        return self.env[(v, u)][m]

    def _behind(self, a: int, b: int) -> set:
        """Open legs in the subtree behind node a as seen from its neighbour b."""
        if self.tree.parent[a] == b:
            return set(self.tree.below[a])
        return set(range(len(self.leg_dims))) - set(self.tree.below[b])

    def leg_index(self, u: int, v: int) -> int:
        legs = self.tree.legs[u]
        return legs.index(("p", v)) if self.tree.parent[u] == v else legs.index(("n", v))

    def update_env(self, a: int, b: int) -> None:
        """E_{a->b}(m) for all m; requires U_a semi-unitary toward its leg facing b."""
        lb = self.leg_index(a, b)
        U = self.tensors[a]
        behind = self._behind(a, b)
        other = [i for i in range(U.ndim) if i != lb]
        out: List[Optional[np.ndarray]] = []
        for m, term in enumerate(self.terms):
            if not (set(term.ops) & behind):
                out.append(None)
                continue
            W = U
            for li in other:
                E = self.leg_env(a, li, m)
                if E is not None:
                    W = mode_product(E, W, li)
            out.append(np.tensordot(U.conj(), W, axes=(other, other)))
        self.env[(a, b)] = out

    def coef(self, m: int) -> complex:
        t = self.terms[m]
        return t.coef * (self.g[t.drive] if t.drive is not None else 1.0)

    # -- projected generators ----------------------------------------------
    def apply_node(self, u: int, U: np.ndarray) -> np.ndarray:
        """H_u U = sum_m coef_m (prod_l E_l(m) x_l) U."""
        Y = np.zeros_like(U)
        for m in range(len(self.terms)):
            W = U
            for li in range(U.ndim):
                E = self.leg_env(u, li, m)
                if E is not None:
                    W = mode_product(E, W, li)
            Y += self.coef(m) * W
        return Y

    def apply_bond(self, a: int, b: int, R: np.ndarray) -> np.ndarray:
        """H_e R = sum_m coef_m E_{a->b}(m) R E_{b->a}(m)^T for R[x_a, x_b]."""
        Y = np.zeros_like(R)
        Ea, Eb = self.env[(a, b)], self.env[(b, a)]
        for m in range(len(self.terms)):
            W = R
            if Ea[m] is not None:
                W = Ea[m] @ W
            if Eb[m] is not None:
                W = W @ Eb[m].T
            Y += self.coef(m) * W
        return Y

    def m_sub(self, tau: float) -> int:
        return sop_mod.n_substeps(tau, self.lam, self.params.kappa)

    def node_flow(self, u: int, tau: float) -> None:
        self.tensors[u] = rk4(lambda y: self.apply_node(u, y), self.tensors[u], tau, self.m_sub(tau))

    def bond_flow(self, a: int, b: int, R: np.ndarray, tau: float) -> np.ndarray:
        return rk4(lambda y: self.apply_bond(a, b, y), R, tau, self.m_sub(tau))

    # -- gauge moves ---------------------------------------------------------
    def qr_toward(self, u: int, v: int) -> np.ndarray:
        """Make U_u semi-unitary toward neighbour v; return R (acting on the bond
        index) with U_u(old) = R applied to U_u(new) along that leg."""
        li = self.leg_index(u, v)
        Um = np.moveaxis(self.tensors[u], li, -1)
        sh = Um.shape
        Q, R = householder_qr(Um.reshape(-1, sh[-1]), self.params.qr_tol)
        self.tensors[u] = np.moveaxis(Q.reshape(sh), -1, li)
        return R

    def absorb(self, v: int, u: int, R: np.ndarray) -> None:
        """U_v := R x_(leg of v facing u) U_v."""
        self.tensors[v] = mode_product(R, self.tensors[v], self.leg_index(v, u))

    # -- ps1 -----------------------------------------------------------------
    def phi(self, u: int, h: float, flow_u: bool = True) -> None:
        """Lie-Trotter half sweep Phi_h(u) (centre at u on entry and exit)."""
        for c in self.tree.children[u]:
            self.absorb(c, u, self.qr_toward(u, c))
            self.update_env(u, c)
            self.phi(c, h)
            R = self.qr_toward(c, u)
            self.update_env(c, u)
            R = self.bond_flow(c, u, R, -h)
            self.absorb(u, c, R)
        if flow_u:
            self.node_flow(u, h)

    def phi_adj(self, u: int, h: float, flow_u: bool = True) -> None:
        """Adjoint half sweep Phi*_h(u): the steps of Phi_h(u) in reverse order."""
        if flow_u:
            self.node_flow(u, h)
        for c in reversed(self.tree.children[u]):
            R = self.qr_toward(u, c)
            self.update_env(u, c)
            R = self.bond_flow(u, c, R, -h)
            self.absorb(c, u, R)
            self.phi_adj(c, h)
            R = self.qr_toward(c, u)
            self.update_env(c, u)
            self.absorb(u, c, R)

    def step_ps1(self, dt: float) -> None:
        t0 = self.t
        h = 0.5 * dt
        if not self.drives:
            self.phi(0, h, flow_u=False)
            self.node_flow(0, dt)
            self.phi_adj(0, h, flow_u=False)
        else:
            self.g = [d.g(t0 + 0.25 * dt) for d in self.drives]
            self.phi(0, h)
            self.g = [d.g(t0 + 0.75 * dt) for d in self.drives]
            self.phi_adj(0, h)
        self.t = t0 + dt

    # -- ps2 -----------------------------------------------------------------
    def apply_two(self, u: int, c: int, Th: np.ndarray) -> np.ndarray:
        """Two-site projected generator on Theta, whose axes are the legs of u
        except the shared bond, then the legs of c except the shared bond."""
        lu, lc = self.leg_index(u, c), self.leg_index(c, u)
        u_other = [i for i in range(self.tensors[u].ndim) if i != lu]
        c_other = [i for i in range(self.tensors[c].ndim) if i != lc]
        Y = np.zeros_like(Th)
        for m in range(len(self.terms)):
            W = Th
            for ax, li in enumerate(u_other):
                E = self.leg_env(u, li, m)
                if E is not None:
                    W = mode_product(E, W, ax)
            for ax, li in enumerate(c_other):
                E = self.leg_env(c, li, m)
                if E is not None:
                    W = mode_product(E, W, len(u_other) + ax)
            Y += self.coef(m) * W
        return Y

    def truncation_rank(self, s: np.ndarray, cap: int) -> int:
        """r0 = #{sigma > ps2_atol}; keep min(cap, max(1, ceil(ps2_ratio * r0)))
        (reading of Sec. 7.5: a ps2_ratio multiple of the kept count re-admits a
        part of the discarded singular values)."""
        p = self.params
        r0 = int(np.sum(s > p.ps2_atol))
        return int(min(cap, len(s), max(1, int(np.ceil(p.ps2_ratio * r0 - 1e-9)))))

    def two_site(self, u: int, c: int, h: float, centre_to: int) -> None:
        """Forward-evolve the merged pair (u, c) by h, SVD, truncate and split; the
        node ``centre_to`` keeps S, the other one becomes semi-unitary."""
        lu, lc = self.leg_index(u, c), self.leg_index(c, u)
        Th = np.tensordot(self.tensors[u], self.tensors[c], axes=([lu], [lc]))
        nu = self.tensors[u].ndim - 1
        Th = rk4(lambda y: self.apply_two(u, c, y), Th, h, self.m_sub(h))
        shu, shc = Th.shape[:nu], Th.shape[nu:]
        Mx = Th.reshape(int(np.prod(shu)), int(np.prod(shc)))
        W, s, Vh = np.linalg.svd(Mx, full_matrices=False)
        r = self.truncation_rank(s, min(self.params.max_rank, Mx.shape[0], Mx.shape[1]))
        self.discarded.append(float(np.sqrt(np.sum(s[r:] ** 2))))
        W, s, Vh = svd_completion(W[:, :r], s[:r], Vh[:r, :], self.params.svd_tol)
        if centre_to == u:
            Au = (W * s[None, :]).reshape(shu + (r,))
            Ac = Vh.reshape((r,) + shc)
        else:
            Au = W.reshape(shu + (r,))
            Ac = (s[:, None] * Vh).reshape((r,) + shc)
        self.tensors[u] = np.moveaxis(Au, -1, lu)
        self.tensors[c] = np.moveaxis(Ac, 0, lc)
        if self.tree.parent[c] == u:
            self.ranks[c] = r
        else:
            self.ranks[u] = r

    def psi(self, u: int, h: float, last: bool) -> None:
        """ps2 Lie-Trotter half sweep Psi_h(u): for each child (ascending) move the
        centre down without evolution, sweep the child's subtree, then evolve the
        pair (child, u) and split with the centre at u; every such update except
        the last one of the sweep is followed by a backward single-node flow of u."""
        ch = self.tree.children[u]
        for idx, c in enumerate(ch):
            self.absorb(c, u, self.qr_toward(u, c))
            self.update_env(u, c)
            self.psi(c, h, last=False)
            self.two_site(c, u, h, centre_to=u)
            self.update_env(c, u)
            if not (last and idx == len(ch) - 1):
                self.node_flow(u, -h)

    def psi_adj(self, u: int, h: float, first: bool) -> None:
        """Adjoint of Psi_h(u): the same steps in reverse order."""
        ch = self.tree.children[u]
        for idx, c in enumerate(reversed(ch)):
            if not (first and idx == 0):
                self.node_flow(u, -h)
            self.two_site(u, c, h, centre_to=c)
            self.update_env(u, c)
            self.psi_adj(c, h, first=False)
            R = self.qr_toward(c, u)
            self.update_env(c, u)
            self.absorb(u, c, R)

    def step_ps2(self, dt: float) -> None:
        t0 = self.t
        h = 0.5 * dt
        self.g = [d.g(t0 + 0.25 * dt) for d in self.drives]
        self.psi(0, h, last=True)
        self.g = [d.g(t0 + 0.75 * dt) for d in self.drives]
        self.psi_adj(0, h, first=True)
        self.t = t0 + dt

    # -- vmf: direct integration of the node equations (Sec. 2.3, Sec. 7.5) ----
    def _upper(self, tensors):
        """Weighted quantities of the part of the tree above every non-root
        node u (all nodes but u's subtree, with the root's weight), from the
        isometric environments of the subtrees below:
          rho[u][a', a]   = <Psi_up[a'] | Psi_up[a]>
          mf[u][m][a', a] = <Psi_up[a'] | h_m^up | Psi_up[a]>  (None: h_m has
                            no factor above u, i.e. h_m^up = 1 and mf = rho)
        computed top-down: the overlap and the mean field on an edge p -> u
        contract conj(U_p), U_p over p's legs other than u, with the parent
        edge's weighted quantity on p's parent leg, the children's bottom-up
        environments on the sibling legs and the operators on open legs."""
        rho: Dict[int, np.ndarray] = {}
        mf: Dict[int, List[Optional[np.ndarray]]] = {}
        for p in self.tree_preorder():
            U = tensors[p]
            legs = self.tree.legs[p]
            for c in self.tree.children[p]:
                lc = legs.index(("n", c))
                other = [i for i in range(U.ndim) if i != lc]
                # overlap: weight on the parent leg only
                W = U
                if p != 0:
                    W = mode_product(rho[p], W, 0)
                rho[c] = np.tensordot(U.conj(), W, axes=(other, other))
                above = set(range(len(self.leg_dims))) - set(self.tree.below[c])
                out: List[Optional[np.ndarray]] = []
                for m, term in enumerate(self.terms):
                    if not (set(term.ops) & above):
                        out.append(None)
                        continue
                    W = U
                    for li in other:
                        kind, v = legs[li]
                        if kind == "p":
                            F = mf[p][m] if mf[p][m] is not None else rho[p]
                        elif kind == "n":
                            F = self.env[(v, p)][m]
                        else:
                            F = term.ops.get(v)
                        if F is not None:
                            W = mode_product(F, W, li)
                    out.append(np.tensordot(U.conj(), W, axes=(other, other)))
                mf[c] = out
        return rho, mf

    def tree_preorder(self) -> List[int]:
        out: List[int] = []

        def rec(u):
            out.append(u)
            for c in self.tree.children[u]:
                rec(c)
        rec(0)
        return out

    def vmf_rhs(self, tensors) -> List[np.ndarray]:
        """Time derivative of every node tensor under the Dirac-Frenkel
        projected generator with the gauge <U_u | dU_u/dt> = 0 (the standard
        multilayer MCTDH equations, written for the linear generator L):
          root:  dA/dt = sum_m coef_m (prod_l E_l(m) x_l) A
          u:     dU_u/dt = rho_u,reg^-1 x_parent (1 - P_u) G_u,
                 G_u = sum_m coef_m mf_u(m) x_parent (prod_child E_l(m) x_l) U_u,
        with rho_reg = rho + vmf_atol * 1 (the regularisation of Sec. 7.5),
        P_u the projector onto the span of U_u's rows (parent index fixed) and
        mf_u(m) = rho_u when term m has no factor above u."""
        saved = self.tensors
        self.tensors = tensors
        try:
            for c in self.tree.postorder():  # isometric (bottom-up) environments
                if c != 0:
                    self.update_env(c, self.tree.parent[c])
            rho, mf = self._upper(tensors)
            out = [None] * self.tree.n_nodes
            out[0] = self.apply_node(0, tensors[0])
            for u in range(1, self.tree.n_nodes):
                U = tensors[u]
                G = np.zeros_like(U)
                for m in range(len(self.terms)):
                    W = U
                    for li in range(1, U.ndim):
                        E = self.leg_env(u, li, m)
                        if E is not None:
                            W = mode_product(E, W, li)
                    F = mf[u][m] if mf[u][m] is not None else rho[u]
                    G += self.coef(m) * mode_product(F, W, 0)
                Um = U.reshape(U.shape[0], -1)
                Gm = G.reshape(U.shape[0], -1)
                Gm = Gm - (Gm @ Um.conj().T) @ Um
                r = rho[u].shape[0]
                Rinv = np.linalg.inv(rho[u] + self.params.vmf_atol * np.eye(r))
                out[u] = (Rinv @ Gm).reshape(U.shape)
            return out
        finally:
            self.tensors = saved

    def step_vmf(self, dt: float) -> None:
        """One step of length dt of the direct integration: all node tensors
        advanced together by dopri5 (ode_rtol, ode_atol), the first trial step
        dt and then the controller's trial step carried over from the previous
        interval; drive values taken at the stage times. Environments are
        refreshed at the end."""
        p = self.params
        t0 = self.t
        h0 = getattr(self, "_vmf_h", dt)

        def f(t, y):
            self.g = [d.g(t) for d in self.drives]
            return self.vmf_rhs(y)
        y, h_next, acc, rej = dopri5(f, self.tensors, t0, t0 + dt, h0, p.ode_rtol, p.ode_atol)
        self._vmf_h = h_next
        self.vmf_stats = getattr(self, "vmf_stats", [0, 0])
        self.vmf_stats[0] += acc
        self.vmf_stats[1] += rej
        self.tensors = y
        self.t = t0 + dt
        for c in self.tree.postorder():
            if c != 0:
                self.update_env(c, self.tree.parent[c])

    def step(self, dt: float, scheme: str = "ps1") -> None:
        if scheme == "ps1":
            self.step_ps1(dt)
        elif scheme == "ps2":
            self.step_ps2(dt)
        elif scheme == "vmf":
            self.step_vmf(dt)
        elif scheme == "mix":
            # the paper's default strategy (Sec. 3.2.3, Sec. 7.5): ps2 while the ranks
            # adapt, then direct integration at the ranks ps2 reached; read here as:
            # switch after the first ps2 step at which a bond rank reaches max_rank
            if getattr(self, "_mixed_to_vmf", False):
                self.step_vmf(dt)
            else:
                self.step_ps2(dt)
                self._mixed_to_vmf = max(self.ranks[1:] or [0]) >= self.params.max_rank
        else:
            raise ValueError(scheme)

    # -- outputs -------------------------------------------------------------
    def rdm(self) -> np.ndarray:
        """rho_S = <0|Omega> (Sec. 2.2): contract every feature leg with e_0,
        bottom-up; the root keeps i and j."""
        vec: Dict[int, np.ndarray] = {}
        for u in self.tree.postorder():
            T = self.tensors[u]
            legs = self.tree.legs[u]
            for li in reversed(range(len(legs))):
                kind, v = legs[li]
                if kind == "p" or (kind == "o" and v in (0, 1)):
                    continue
                if kind == "n":
                    w = vec[v]
                else:
                    w = np.zeros(self.leg_dims[v], np.complex128)
                    w[0] = 1.0
                T = np.tensordot(T, w, axes=([li], [0]))
            if u == 0:
                return T  # remaining axes: i, j (leg 0 sorts before leg 1)
            vec[u] = T
        raise RuntimeError("unreachable")

    def full_tensor(self) -> np.ndarray:
        """Dense Omega[i, j, n_1..n_K] (small cases only)."""
        def contract(u):
            T = self.tensors[u]
            labels = [("p",) if k == "p" else (k, v) for k, v in self.tree.legs[u]]
            for kind, v in self.tree.legs[u]:
                if kind != "n":
                    continue
                sub, sub_labels = contract(v)
                ax = labels.index(("n", v))
                T = np.tensordot(T, sub, axes=([ax], [0]))
                labels = labels[:ax] + labels[ax + 1:] + sub_labels[1:]
            return T, labels

        T, labels = contract(0)
        return np.transpose(T, [labels.index(("o", l)) for l in range(len(self.leg_dims))])

    def bond_singular_values(self) -> List[np.ndarray]:
        """Singular values of the matricisation across every bond (gauge invariant)."""
        full = self.full_tensor()
        out = []
        for c in range(1, self.tree.n_nodes):
            below = self.tree.below[c]
            rest = [l for l in range(len(self.leg_dims)) if l not in below]
            Mx = np.transpose(full, rest + below).reshape(
                int(np.prod([self.leg_dims[l] for l in rest])), -1)
            out.append(np.linalg.svd(Mx, compute_uv=False))
        return out


def from_workload(w, metric="abs", params: Optional[Params] = None) -> "TTN":
    """Build the oracle TTN for a workloads.Workload."""
    terms = sop_mod.heom_terms(w.H, w.baths, w.depth, metric=metric, drives=w.drives)
    if params is None:
        params = Params(ps2_atol=w.ps2_atol, ps2_ratio=w.ps2_ratio, max_rank=w.max_rank)
    return TTN(w.parent, w.leg_node, w.leg_dims, w.ranks, terms, w.rho0,
               drives=w.drives, params=params)


def htd_tensors(tree: Tree, leg_dims: Sequence[int], ranks: Sequence[int], Omega: np.ndarray):
    """Leaves-to-root hierarchical Tucker decomposition (Sec. 2.3: the tree is
    assembled by repeated SVDs, keeping the leading singular vectors as the bond
    basis). Returns node tensors in canonical leg order, non-root nodes
    semi-unitary toward the parent, the weight in the root. Exact when every rank
    is at least the matricisation rank across its bond."""
    C = np.asarray(Omega, np.complex128)
    labels = [("o", l) for l in range(len(leg_dims))]
    tensors: List[Optional[np.ndarray]] = [None] * tree.n_nodes
    for u in tree.postorder():
        mine = [("o", v) if k == "o" else ("b", v) for k, v in tree.legs[u] if k != "p"]
        axes = [labels.index(x) for x in mine]
        rest = [i for i in range(C.ndim) if i not in axes]
        Cm = np.transpose(C, axes + rest)
        shm = Cm.shape[:len(axes)]
        if u == 0:
            tensors[0] = Cm.reshape(shm)
            break
        Mx = Cm.reshape(int(np.prod(shm)), -1)
        Wl, s, _ = np.linalg.svd(Mx, full_matrices=False)
        r = ranks[u]
        Wr = np.zeros((Mx.shape[0], r), np.complex128)
        k = min(r, Wl.shape[1])
        Wr[:, :k] = Wl[:, :k]
        if k < r:  # pad with a completion (zero weight)
            Wr = _complete_columns(Wl[:, :k], r)
        tensors[u] = Wr.T.reshape((r,) + shm)
        Cnew = (Wr.conj().T @ Mx).reshape((r,) + Cm.shape[len(axes):])
        labels = [("b", u)] + [labels[i] for i in rest]
        C = Cnew
    return tensors
