"""Seeded synthetic workloads for the TTN-HEOM hot path.

This module is shared by the FP64 CPU oracle and by the CUDA path. It holds
only *inputs*: physical parameters (system Hamiltonian, coupling operators,
spectral-density parameters, temperatures), tree topologies, requested bond
ranks, depths, initial reduced density matrices and time grids. It contains no
arithmetic of the method itself (no bath-correlation decomposition, no SOP
terms, no tensor-network algebra): both sides derive those independently.

Leg numbering used everywhere: leg 0 = ket index i of the system, leg 1 = bra
index j, leg 2 + k = Fock leg of feature k (Sec. 2.3, Eq. EDO-elements).
Node 0 is the root; ``parent[0] == -1``. ``leg_node[l]`` is the node that leg l
hangs on. Both system legs sit on the root (Sec. 2.3, after Eq. semiunitary).

Feature ordering inside a bath follows the decomposition order: Drude-Lorentz
pole feature first (if present), then the two features of each Brownian peak
(``+`` then ``-``), then the ``n_ltc`` Bose-pole features (Eq. bcfdecores).
Baths are concatenated in order (bath-major).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

# 1 cm^-1 expressed as an angular frequency in rad/fs (2*pi*c).
CM1_TO_RAD_PER_FS = 2.0 * np.pi * 2.99792458e10 * 1e-15
# Boltzmann constant in cm^-1 per kelvin.
KB_CM1_PER_K = 0.6950348

SIGMA_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


@dataclasses.dataclass
class Bath:
    """One harmonic bath coupled through ``Q`` (Sec. 2.1, Eq. DL / Eq. BO).

    ``dl`` = (lambda, omega_c) or None; ``bo`` = list of (lambda, omega0', eta)
    Brownian peaks in the factored form; ``beta`` = inverse temperature;
    ``n_ltc`` = number of Bose-pole ("low-temperature correction") features;
    ``scheme`` = 'pade' or 'matsubara'.
    """
    Q: np.ndarray
    beta: float
    dl: Optional[Tuple[float, float]] = None
    bo: List[Tuple[float, float, float]] = dataclasses.field(default_factory=list)
    n_ltc: int = 0
    scheme: str = "pade"

    @property
    def n_features(self) -> int:
        return (1 if self.dl is not None else 0) + 2 * len(self.bo) + self.n_ltc


@dataclasses.dataclass
class Drive:
    """Time-dependent system term g(t) * V with g(t) = amp * cos(omega t + phase)."""
    V: np.ndarray
    amp: float
    omega: float
    phase: float = 0.0

    def g(self, t: float) -> float:
        return self.amp * np.cos(self.omega * t + self.phase)

    @property
    def bound(self) -> float:
        return abs(self.amp)


@dataclasses.dataclass
class Workload:
    name: str
    H: np.ndarray                 # static system Hamiltonian, M x M
    baths: List[Bath]
    depth: List[int]              # Fock depth N_k per feature
    parent: List[int]             # tree, node 0 = root
    leg_node: List[int]           # node of every leg
    ranks: List[int]              # requested rank of bond (u, parent(u)); entry 0 ignored
    rho0: np.ndarray              # M x M
    dt: float
    n_steps: int
    scheme: str = "ps1"           # 'ps1' or 'ps2'
    drives: List[Drive] = dataclasses.field(default_factory=list)
    ps2_atol: float = 1e-7
    ps2_ratio: float = 2.0
    max_rank: int = 32

    @property
    def M(self) -> int:
        return self.H.shape[0]

    @property
    def K(self) -> int:
        return sum(b.n_features for b in self.baths)

    @property
    def leg_dims(self) -> List[int]:
        return [self.M, self.M] + list(self.depth)


# ----------------------------------------------------------------------------
# Tree topologies (inputs of ttn_create)
# ----------------------------------------------------------------------------

def tensor_train(K: int) -> Tuple[List[int], List[int]]:
    """Tensor train of Eq. omega_tensor: root A(i, j, a1), then U(a_s, n_s, a_{s+1}),
    the last core holding the last two feature legs. K >= 1."""
    if K < 1:
        raise ValueError("K >= 1")
    if K == 1:
        return [-1], [0, 0, 0]
    n_nodes = K  # root + (K-1) cores
    parent = [-1] + list(range(0, n_nodes - 1))
    leg_node = [0, 0]
    for k in range(K):
        leg_node.append(min(k + 1, n_nodes - 1))
    return parent, leg_node


def balanced_binary(K: int) -> Tuple[List[int], List[int]]:
    """Balanced binary tree: root A(i, j, a) with one child; below it feature
    legs 0..K-1 split ceil(n/2) | floor(n/2) recursively; a two-feature subtree is
    one node with two open legs, a one-feature subtree is the open leg itself."""
    if K < 1:
        raise ValueError("K >= 1")
    parent = [-1]
    leg_node = [0, 0] + [-1] * K
    if K == 1:
        leg_node[2] = 0
        return parent, leg_node

    def build(lo: int, hi: int, par: int) -> None:
        n = hi - lo
        if n == 1:
            leg_node[2 + lo] = par
            return
        u = len(parent)
        parent.append(par)
        if n == 2:
            leg_node[2 + lo] = u
            leg_node[2 + lo + 1] = u
            return
        mid = lo + (n + 1) // 2
        build(lo, mid, u)
        build(mid, hi, u)

    build(0, K, 0)
    return parent, leg_node


def centred_train(K: int) -> Tuple[List[int], List[int]]:
    """The custom tensor train of Sec. 7.2 (Listing customtn1): a chain of
    feature nodes whose junction node -- carrying no feature -- hangs from the
    root, so the root sits in the middle of the train instead of at an end.
    Features 0 .. ceil(K/2)-1 lie on the left arm (the one nearest the
    junction holding the last of them), the rest on the right arm. The arm
    ends have two legs (their parent bond and one feature). K >= 2."""
    if K < 2:
        raise ValueError("K >= 2")
    parent = [-1, 0]          # root, junction
    leg_node = [0, 0] + [-1] * K
    left = (K + 1) // 2
    prev = 1
    for k in reversed(range(left)):  # the left arm walks away from the junction
        parent.append(prev)
        prev = len(parent) - 1
        leg_node[2 + k] = prev
    prev = 1
    for k in range(left, K):
        parent.append(prev)
        prev = len(parent) - 1
        leg_node[2 + k] = prev
    return parent, leg_node


def uniform_ranks(parent: Sequence[int], r: int) -> List[int]:
    return [0] + [r] * (len(parent) - 1)


# ----------------------------------------------------------------------------
# Workloads shaped like the paper's model families
# ----------------------------------------------------------------------------

def spin_boson_tt(n_steps: int = 1000, rank: int = 10, depth: int = 10,
                  n_pade: int = 3, tree: str = "tt") -> Workload:
    """Spin-boson, H = 0.5 sz + 1.0 sx, Q = sz, Drude-Lorentz lambda=0.5,
    omega_c=1, beta=1, 1 Drude + n_pade Pade features, depth 10, tensor train,
    rank 10, dt = 0.01, rho0 = |0><0|."""
    bath = Bath(Q=SIGMA_Z.copy(), beta=1.0, dl=(0.5, 1.0), n_ltc=n_pade)
    K = bath.n_features
    parent, leg_node = tensor_train(K) if tree == "tt" else balanced_binary(K)
    rho0 = np.zeros((2, 2), np.complex128)
    rho0[0, 0] = 1.0
    return Workload(name=f"spin-boson {tree.upper()} K={K} N={depth} R={rank}",
                    H=0.5 * SIGMA_Z + 1.0 * SIGMA_X, baths=[bath],
                    depth=[depth] * K, parent=parent, leg_node=leg_node,
                    ranks=uniform_ranks(parent, rank), rho0=rho0, dt=0.01,
                    n_steps=n_steps)


def exciton_chain(n_sites: int = 7, rank: int = 20, depth: int = 8,
                  n_steps: int = 5000, seed: int = 20260317,
                  n_pade: int = 2) -> Workload:
    """Frenkel exciton chain with one Drude bath per site (Sec. 3.4 model family).

    Site energies ~ N(0, 100 cm^-1), nearest-neighbour couplings ~ U(50, 100) cm^-1
    (seeded); per-site Drude bath lambda = 35 cm^-1, omega_c = 106 cm^-1, T = 300 K,
    1 Drude + n_pade Pade features; Q_b = |b><b|; balanced binary tree; depth 8;
    dt = 0.05 fs; rho0 = |1><1| (first site). Energies in rad/fs, time in fs."""
    rng = np.random.default_rng(seed)
    eps = rng.normal(0.0, 100.0, size=n_sites)
    V = rng.uniform(50.0, 100.0, size=n_sites - 1)
    Hc = np.diag(eps).astype(np.complex128)
    for i in range(n_sites - 1):
        Hc[i, i + 1] = Hc[i + 1, i] = V[i]
    H = Hc * CM1_TO_RAD_PER_FS
    beta = 1.0 / (KB_CM1_PER_K * 300.0 * CM1_TO_RAD_PER_FS)
    baths = []
    for b in range(n_sites):
        Q = np.zeros((n_sites, n_sites), np.complex128)
        Q[b, b] = 1.0
        baths.append(Bath(Q=Q, beta=beta,
                          dl=(35.0 * CM1_TO_RAD_PER_FS, 106.0 * CM1_TO_RAD_PER_FS),
                          n_ltc=n_pade))
    K = sum(b.n_features for b in baths)
    parent, leg_node = balanced_binary(K)
    rho0 = np.zeros((n_sites, n_sites), np.complex128)
    rho0[0, 0] = 1.0
    return Workload(name=f"{n_sites}-site exciton chain BTT K={K} N={depth} R={rank}",
                    H=H, baths=baths, depth=[depth] * K, parent=parent,
                    leg_node=leg_node, ranks=uniform_ranks(parent, rank), rho0=rho0,
                    dt=0.05, n_steps=n_steps)


def spin_boson_batch(n: int = 256, seed: int = 4242, n_steps: int = 1000) -> List[Workload]:
    """Batch of uneven spin-boson instances: lambda ~ U(0.1, 1), omega_c ~ U(0.5, 5),
    beta ~ U(0.5, 5), eps, Delta ~ U(0, 2), H = eps/2 sz + Delta sx, Q = sz,
    K ~ U{2..8} features (1 Drude + K-1 Pade), depth ~ U{6..12}, rank ~ U{8..32},
    balanced binary tree, dt = 0.01."""
    rng = np.random.default_rng(seed)
    out = []
    for idx in range(n):
        lam = rng.uniform(0.1, 1.0)
        wc = rng.uniform(0.5, 5.0)
        beta = rng.uniform(0.5, 5.0)
        eps = rng.uniform(0.0, 2.0)
        delta = rng.uniform(0.0, 2.0)
        K = int(rng.integers(2, 9))
        depth = int(rng.integers(6, 13))
        rank = int(rng.integers(8, 33))
        bath = Bath(Q=SIGMA_Z.copy(), beta=beta, dl=(lam, wc), n_ltc=K - 1)
        parent, leg_node = balanced_binary(K)
        rho0 = np.zeros((2, 2), np.complex128)
        rho0[0, 0] = 1.0
        out.append(Workload(name=f"spin-boson batch #{idx}", H=0.5 * eps * SIGMA_Z + delta * SIGMA_X,
                            baths=[bath], depth=[depth] * K, parent=parent,
                            leg_node=leg_node, ranks=uniform_ranks(parent, rank),
                            rho0=rho0, dt=0.01, n_steps=n_steps))
    return out


def driven_structured_tls(n_steps: int = 2000, n_pade: int = 25, depth: int = 10,
                          cap: int = 128) -> Workload:
    """Driven two-level system, H(t) = 0.75 sz + 0.2 cos(1.5 t) sx, Q = sz, beta = 1,
    Drude lambda = 0.2, omega_c = 1 plus three Brownian peaks omega0' = 1, 2, 3,
    eta = 0.1, lambda_b = 0.1; 1 + 6 + n_pade features; depth 10; balanced binary
    tree; adaptive rank (ps2) with cap ``cap``, ps2_atol = 1e-6; dt = 0.01."""
    bath = Bath(Q=SIGMA_Z.copy(), beta=1.0, dl=(0.2, 1.0),
                bo=[(0.1, 1.0, 0.1), (0.1, 2.0, 0.1), (0.1, 3.0, 0.1)], n_ltc=n_pade)
    K = bath.n_features
    parent, leg_node = balanced_binary(K)
    rho0 = np.zeros((2, 2), np.complex128)
    rho0[0, 0] = 1.0
    # ps2 starts from the product state padded to rank 4: in a binary tree every
    # two-site block of an all-rank-1 state has a rank-1 side, so ranks could not grow
    return Workload(name=f"driven TLS structured bath K={K} N={depth} cap={cap}",
                    H=0.75 * SIGMA_Z, baths=[bath], depth=[depth] * K, parent=parent,
                    leg_node=leg_node, ranks=uniform_ranks(parent, 4), rho0=rho0,
                    dt=0.01, n_steps=n_steps, scheme="ps2",
                    drives=[Drive(V=SIGMA_X.copy(), amp=0.2, omega=1.5)],
                    ps2_atol=1e-6, ps2_ratio=2.0, max_rank=cap)


def random_hermitian(rng: np.random.Generator, M: int) -> np.ndarray:
    A = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    return 0.5 * (A + A.conj().T)


def random_density_matrix(rng: np.random.Generator, M: int) -> np.ndarray:
    A = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    rho = A @ A.conj().T
    return rho / np.trace(rho).real


# ----------------------------------------------------------------------------
# The paper's own example models (Sec. 3): parameters as printed there
# ----------------------------------------------------------------------------

def _kelvin_beta(T: float) -> float:
    """1 / (k_B T) in fs (energies in rad/fs)."""
    return 1.0 / (KB_CM1_PER_K * T * CM1_TO_RAD_PER_FS)


def structured_spin_boson(depth: int = 25, rank: int = 20, tree: str = "btt", n_steps: int = 1000,
                          dt: float = 1.0, T: float = 300.0, n_ltc: int = 1) -> Workload:
    """Example 1 (Sec. 3.2, Table 1 and the listing beside it): spin-boson
    H_S = (1500/2) sz + 300 sx cm^-1 written as diag(-750, 750) + 300 sx (the
    listing's matrix), coupling sys_op = diag(-1/2, 1/2), one bath with a
    Drude-Lorentz term (lambda 540, omega_c 70 cm^-1) and one Brownian peak
    (lambda 161.6, eta 10, omega_0' 1243 cm^-1) at 300 K, Pade with one
    low-temperature correction (K = 1 + 2 + 1 = 4 features), depth 25,
    dt 1 fs, 1000 fs, rho0 = |1><1| (second state, wfn = (0, 1)). The listing
    leaves the tree, the rank and the propagator at TENSO's defaults; here: a
    balanced binary tree, fixed rank (ps1)."""
    c = CM1_TO_RAD_PER_FS
    H = np.array([[-750.0, 300.0], [300.0, 750.0]], np.complex128) * c
    bath = Bath(Q=np.diag([-0.5, 0.5]).astype(np.complex128), beta=_kelvin_beta(T), dl=(540.0 * c, 70.0 * c),
                bo=[(161.6 * c, 1243.0 * c, 10.0 * c)], n_ltc=n_ltc)
    K = bath.n_features
    parent, leg_node = tensor_train(K) if tree == "tt" else balanced_binary(K)
    rho0 = np.zeros((2, 2), np.complex128)
    rho0[1, 1] = 1.0
    return Workload(name=f"structured spin-boson (Table 1) {tree.upper()} K={K} N={depth} R={rank}", H=H,
                    baths=[bath], depth=[depth] * K, parent=parent, leg_node=leg_node,
                    ranks=uniform_ranks(parent, rank), rho0=rho0, dt=dt, n_steps=n_steps)


FMO3_H_CM1 = np.array([[200.0, -87.7, 5.5], [-87.7, 320.0, 30.8], [5.5, 30.8, 0.0]])
# six Brownian peaks of the structured FMO spectral density: (lambda, omega_0', eta) in cm^-1
FMO_BO6_CM1 = [(26.24, 160.0, 133.0), (13.832, 247.0, 53.0), (101.479, 763.0, 76.0),
               (57.575, 1175.0, 29.0), (25.764, 1356.0, 29.0), (9.126, 1521.0, 15.0)]


def fmo3(T: float = 77.0, spectral: str = "bo6", depth: int = 20, rank: int = 16, n_steps: int = 20000,
         dt: float = 0.05, n_ltc: Optional[int] = None) -> Workload:
    """Example 2 (Sec. 3.4 and its listing): the three-site FMO model
    (site Hamiltonian in cm^-1 as printed), an identical independent bath on
    every site coupled through |i><i|, rho0 = |1><1|, dt 0.05 fs, 1000 fs,
    depth 20, ps1. spectral: 'bo6' (six Brownian peaks), 'bo3' (the three
    below 1000 cm^-1) or 'dl' (Drude-Lorentz 35 / 106.18 cm^-1); Pade with
    n_ltc = 1 at 300 K and 3 at 77 K (the paper's choice). bo6 at 77 K gives
    K = 12 + 3 = 15 features per site, 45 in all. Balanced binary tree; the
    listing leaves the rank at TENSO's default, here `rank`."""
    c = CM1_TO_RAD_PER_FS
    if n_ltc is None:
        n_ltc = 3 if T < 150.0 else 1
    if spectral == "bo6":
        bo, dl = [(l * c, w * c, e * c) for (l, w, e) in FMO_BO6_CM1], None
    elif spectral == "bo3":
        bo, dl = [(l * c, w * c, e * c) for (l, w, e) in FMO_BO6_CM1 if w < 1000.0], None
    elif spectral == "dl":
        bo, dl = [], (35.0 * c, 106.18 * c)
    else:
        raise ValueError(spectral)
    baths = []
    for i in range(3):
        Q = np.zeros((3, 3), np.complex128)
        Q[i, i] = 1.0
        baths.append(Bath(Q=Q, beta=_kelvin_beta(T), dl=dl, bo=list(bo), n_ltc=n_ltc))
    K = sum(b.n_features for b in baths)
    parent, leg_node = balanced_binary(K)
    rho0 = np.zeros((3, 3), np.complex128)
    rho0[0, 0] = 1.0
    return Workload(name=f"FMO 3-site {spectral} {T:g} K BTT K={K} N={depth} R={rank}",
                    H=FMO3_H_CM1.astype(np.complex128) * c, baths=baths, depth=[depth] * K, parent=parent,
                    leg_node=leg_node, ranks=uniform_ranks(parent, rank), rho0=rho0, dt=dt, n_steps=n_steps)


def convergence_spin_boson(panel: str = "b", depth: int = 25, rank: int = 40, tree: str = "btt",
                           n_steps: int = 1000, dt: float = 1.0, T: float = 300.0, n_ltc: int = 1) -> Workload:
    """The spin-boson models of the convergence study (Sec. 3.2.3, Table 2):
    panel 'a' -- symmetric (Delta eps = 0, V = 300 cm^-1), Drude-Lorentz bath
    only (540, 70 cm^-1), coupled through sigma_x (the depth sweep);
    panel 'b' -- Delta eps = 1500, V = 300, Drude-Lorentz (540, 70) plus a
    Brownian peak (lambda 330, eta 4, omega_0' 1663) (the rank sweeps, BTT and
    TT), with the system Hamiltonian and coupling of the Example 1 listing.
    The coupling carries the factor 1/2 of H_SB = (sigma_z / 2) X_B of
    Sec. 3.2 in both panels (the listing's sys_op diag(-1/2, 1/2); sigma_x / 2
    in panel a); the text's later shorthand "sigma ⊗ X_B" is read as the same
    convention. Temperature, Pade correction, dt and the initial state follow
    the Example 1 listing (300 K, n_ltc 1, 1 fs, rho0 = |1><1|)."""
    c = CM1_TO_RAD_PER_FS
    if panel == "a":
        H = 300.0 * SIGMA_X * c
        bath = Bath(Q=0.5 * SIGMA_X, beta=_kelvin_beta(T), dl=(540.0 * c, 70.0 * c), n_ltc=n_ltc)
    elif panel == "b":
        H = (np.array([[-750.0, 0.0], [0.0, 750.0]]) + 300.0 * SIGMA_X.real).astype(np.complex128) * c
        bath = Bath(Q=np.diag([-0.5, 0.5]).astype(np.complex128), beta=_kelvin_beta(T), dl=(540.0 * c, 70.0 * c),
                    bo=[(330.0 * c, 1663.0 * c, 4.0 * c)], n_ltc=n_ltc)
    else:
        raise ValueError(panel)
    K = bath.n_features
    parent, leg_node = tensor_train(K) if tree == "tt" else balanced_binary(K)
    rho0 = np.zeros((2, 2), np.complex128)
    rho0[1, 1] = 1.0
    return Workload(name=f"convergence spin-boson panel {panel} {tree.upper()} K={K} N={depth} R={rank}",
                    H=H, baths=[bath], depth=[depth] * K, parent=parent, leg_node=leg_node,
                    ranks=uniform_ranks(parent, rank), rho0=rho0, dt=dt, n_steps=n_steps)


@dataclasses.dataclass
class StarBoson:
    """Wavefunction (ML-MCTDH) model of Sec. 3.2.4 (Listing mctdh): system H,
    coupling sys_op Q, a bath given by Brownian peaks (lambda, omega_0', eta)
    at temperature 1/beta, discretised into n_modes harmonic modes up to
    `cutoff` (the discretisation itself is done by each side), Fock dimension
    `dim` per mode, initial wavefunction psi0, tree over the modes."""
    name: str
    H: np.ndarray
    Q: np.ndarray
    bo: List[Tuple[float, float, float]]
    beta: float
    cutoff: float
    n_modes: int
    dim: int
    psi0: np.ndarray
    parent: List[int]
    leg_node: List[int]
    ranks: List[int]
    dt: float
    n_steps: int

    @property
    def leg_dims(self) -> List[int]:
        M = self.H.shape[0]
        return [M, M] + [self.dim] * self.n_modes


def star_boson_mctdh(n_modes: int = 50, dim: int = 8, rank: int = 8, n_steps: int = 200, dt: float = 1.0,
                     T: float = 300.0, cutoff_cm1: float = 200.0) -> StarBoson:
    """Listing mctdh: one Brownian peak (lambda 200, eta 10, omega_0' 50 cm^-1)
    at 300 K, cutoff 200 cm^-1, 50 modes of Fock dimension 8, dt 1 fs, 200 fs,
    psi0 = (0, 1), the spin-boson H_S and sys_op of Example 1. The thermofield
    form (modes of positive and negative frequency for the thermal state) is
    the one the paper's MCTDH uses; the listing's TEDOPA chain is replaced by a
    star over the modes (same bath correlation up to the discretisation).
    Legs: 0 = system, 1 = a spectator of the same dimension that no operator
    touches (the library's root holds two system legs), 2.. = the modes;
    balanced binary tree over the modes."""
    c = CM1_TO_RAD_PER_FS
    H = np.array([[-750.0, 300.0], [300.0, 750.0]], np.complex128) * c
    parent, leg_node = balanced_binary(n_modes)
    ranks = uniform_ranks(parent, rank)
    ranks[1] = min(rank, H.shape[0])  # the spectator index stays 0: the root bond needs rank M, not M^2
    return StarBoson(name=f"thermofield star boson, {n_modes} modes, dim {dim}, rank {rank}", H=H,
                     Q=np.diag([-0.5, 0.5]).astype(np.complex128), bo=[(200.0 * c, 50.0 * c, 10.0 * c)],
                     beta=_kelvin_beta(T), cutoff=cutoff_cm1 * c, n_modes=n_modes, dim=dim,
                     psi0=np.array([0.0, 1.0], np.complex128), parent=parent, leg_node=leg_node,
                     ranks=ranks, dt=dt, n_steps=n_steps)
