"""The paper's example models (Sec. 3.2 Table 1, Sec. 3.4 FMO, Sec. 3.2.3
Table 2) on the GPU against the FP64 oracle: ranks and rho_S after every step
(1e-10 in FP64), and the full-size FMO model at 77 K (45 features, depth 20)
in both forms."""
import numpy as np
import pytest

import workloads as W
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _parity(pkg, w, n):
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0)
    o = ottn.from_workload(w)
    assert list(g.ttn_get_ranks()) == o.ranks
    err = 0.0
    for _ in range(n):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    return err


@pytest.mark.parametrize("make,n", [
    (lambda: W.structured_spin_boson(depth=25, rank=20), 20),
    (lambda: W.structured_spin_boson(depth=25, rank=12, tree="tt"), 20),
    (lambda: W.fmo3(T=77.0, depth=5, rank=6), 4),
    (lambda: W.convergence_spin_boson("a", depth=14, rank=10), 20),
    (lambda: W.convergence_spin_boson("b", depth=12, rank=8, tree="tt"), 20),
])
def test_paper_models_against_oracle(pkg, make, n):
    assert _parity(pkg, make(), n) <= 1e-10


def test_fmo_77k_full_size_both_forms(pkg):
    """45 features (six Brownian peaks and three Pade corrections per site),
    depth 20, rank 16, balanced binary tree: FP64 and mixed stay within the
    1e-6 bar of each other over 40 steps (2 fs) and the populations move away
    from site 1. At a truncated rank the trace is not conserved exactly (the
    projected generator need not keep the n = 0 tier's trace); it is only
    checked to stay near 1."""
    w = W.fmo3(T=77.0)
    ga = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0)
    gb = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                        precision=pkg.TTN_MIXED_FP32)
    diff = 0.0
    for _ in range(40):
        ga.ttn_step(w.dt, pkg.TTN_PS1, 1)
        gb.ttn_step(w.dt, pkg.TTN_PS1, 1)
        ra, rb = ga.ttn_rdm(), gb.ttn_rdm()
        diff = max(diff, float(np.max(np.abs(ra - rb))))
    assert abs(np.trace(ra) - 1.0) < 1e-4
    assert ra[0, 0].real < 1.0 - 1e-4
    ga.close()
    gb.close()
    assert diff <= 1e-6, diff
