"""Custom tree frames (Sec. 7.2): the centred tensor train of Listing
customtn1, whose arm-end nodes have two legs, runs on the GPU with those nodes
padded by a dimension-1 open leg (pad_to_three_legs); at truncated ranks it
must follow the oracle, which propagates the unpadded tree, step by step."""
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


@pytest.mark.parametrize("K,rank,scheme", [(4, 4, "ps1"), (5, 6, "ps1"), (4, 2, "ps2")])
def test_centred_train_against_oracle(pkg, K, rank, scheme):
    w = W.spin_boson_tt(depth=5, n_pade=K - 1, rank=rank)
    w.parent, w.leg_node = W.centred_train(K)
    w.ranks = W.uniform_ranks(w.parent, rank)
    params = {"max_rank": 8, "ps2_atol": 1e-7}
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, params=params)
    o = ottn.from_workload(w, params=ottn.Params(max_rank=8, ps2_atol=1e-7))
    err = 0.0
    code = pkg.TTN_PS1 if scheme == "ps1" else pkg.TTN_PS2
    for _ in range(10):
        g.ttn_step(w.dt, code, 1)
        o.step(w.dt, scheme)
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
        assert list(g.ttn_get_ranks()) == o.ranks
    g.close()
    assert err <= 1e-10, err
