"""ps2 (adaptive rank, Sec. 2.3 last paragraph; truncation as read from
Sec. 7.5) at sizes where the merged two-site matrices are too wide for one CTA:
the driven two-level system with a structured bath (Drude + three Brownian
peaks, Eq. DL / Eq. BO, drive 0.2 cos(1.5 t) sigma_x), balanced binary tree,
Fock depth 10, ps2_atol 1e-6, cap 32. Ranks must follow the FP64 oracle split
by split and rho_S must agree to 1e-10 (both sides run the same algorithm in
FP64)."""
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


def test_ps2_driven_structured_bath_cap32_against_oracle(pkg):
    w = W.driven_structured_tls(n_pade=1, depth=10, cap=32)
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, drives=w.drives,
                       params={"max_rank": 32, "ps2_atol": 1e-6})
    o = ottn.from_workload(w, params=ottn.Params(ps2_atol=1e-6, max_rank=32))
    err = 0.0
    for k in range(12):
        g.ttn_step(w.dt, pkg.TTN_PS2, 1)
        o.step(w.dt, "ps2")
        assert list(g.ttn_get_ranks()) == o.ranks, (k, list(g.ttn_get_ranks()), o.ranks)
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    # the merged matrices outgrew one CTA's Jacobi (>= 24 columns on the smaller side)
    assert max(o.ranks) >= 8
    g.close()
    assert err <= 1e-10, err
