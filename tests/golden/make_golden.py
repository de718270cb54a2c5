"""Writes the stored oracle trajectories used by the GPU parity tests.

Every value here comes from the FP64 CPU oracle (oracle/), never from the CUDA
path. Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ttn  # noqa: E402


def spin_boson_tt_trajectory(path: str, every: int = 10) -> None:
    """Spin-boson (H = 0.5 sz + sx, Q = sz, Drude lambda = 0.5, omega_c = 1,
    beta = 1, 1 Drude + 3 Pade features, depth 10, tensor train, rank 10,
    dt = 0.01, 1000 ps1 steps, rho0 = |0><0|): rho_S every `every` steps."""
    w = W.spin_boson_tt(n_steps=1000)
    st = ttn.from_workload(w)
    rows = [(0, st.rdm())]
    for n in range(1, w.n_steps + 1):
        st.step(w.dt, "ps1")
        if n % every == 0:
            rows.append((n, st.rdm()))
    with open(path, "w") as f:
        f.write("# oracle (oracle/ttn.py, ps1) rho_S of the spin-boson tensor train:\n")
        f.write("# H = 0.5 sz + 1.0 sx, Q = sz, Drude lambda=0.5 omega_c=1 beta=1, 1 Drude + 3 Pade\n")
        f.write("# features (Eq. bcfdecores), depth 10, rank 10, dt = 0.01, rho0 = |0><0|.\n")
        f.write("# columns: step, then Re/Im of rho_11 rho_12 rho_21 rho_22 (row-major, Sec. 3.2 output order)\n")
        for n, r in rows:
            vals = " ".join(f"{x.real:.17e} {x.imag:.17e}" for x in r.reshape(-1))
            f.write(f"{n} {vals}\n")


def exciton_chain_trajectory(path: str, rank: int, n_steps: int, every: int) -> None:
    """7-site Frenkel exciton chain (seeded energies and couplings, per-site
    Drude bath 35 cm^-1 / 106 cm^-1 at 300 K, 1 Drude + 2 Pade features per site,
    21 features, depth 8, balanced binary tree, dt = 0.05 fs, rho0 = |1><1|) at
    bond rank `rank`: rho_S (7 x 7) every `every` ps1 steps."""
    w = W.exciton_chain(rank=rank, n_steps=n_steps)
    st = ttn.from_workload(w)
    rows = [(0, st.rdm())]
    for n in range(1, n_steps + 1):
        st.step(w.dt, "ps1")
        if n % every == 0:
            rows.append((n, st.rdm()))
    with open(path, "w") as f:
        f.write("# oracle (oracle/ttn.py, ps1) rho_S of the 7-site exciton chain (workloads.exciton_chain):\n")
        f.write(f"# 21 Drude/Pade features, depth 8, balanced binary tree, bond rank {rank}, dt = 0.05 fs,\n")
        f.write(f"# rho0 = |1><1|, {n_steps} steps. columns: step, then Re/Im of the 49 entries of rho_S (row-major)\n")
        for n, r in rows:
            vals = " ".join(f"{x.real:.17e} {x.imag:.17e}" for x in r.reshape(-1))
            f.write(f"{n} {vals}\n")


if __name__ == "__main__":
    which = sys.argv[1:] or ["sb", "chain20", "chain64"]
    if "sb" in which:
        spin_boson_tt_trajectory(os.path.join(HERE, "spin_boson_tt_k4_n10_r10.txt"))
    if "chain20" in which:
        exciton_chain_trajectory(os.path.join(HERE, "exciton7_r20_100steps.txt"), 20, 100, 5)
    if "chain64" in which:
        exciton_chain_trajectory(os.path.join(HERE, "exciton7_r64_2steps.txt"), 64, 2, 1)
