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


if __name__ == "__main__":
    spin_boson_tt_trajectory(os.path.join(HERE, "spin_boson_tt_k4_n10_r10.txt"))
