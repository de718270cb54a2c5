"""Full-size parity against stored oracle trajectories (written by
tests/golden/make_golden.py, which calls only oracle/): the 7-site exciton
chain (21 Drude/Pade features, depth 8, balanced binary tree, ps1) at bond
rank 20 over 100 steps and at bond rank 64 (nodes 64 x 64 x 64, state 1.97 M
complex) over 2 steps, in the FP64 form (held to 1e-10: the same algorithm in
FP64, differing only in the order of the sums) and in the mixed form (FP32
contractions, held to the 1e-6 bar)."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _stored(name):
    rows = np.loadtxt(os.path.join(HERE, "golden", name))
    return [(int(r[0]), (r[1::2] + 1j * r[2::2]).reshape(7, 7)) for r in rows]


def _run(pkg, w, rows, precision):
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, precision=precision)
    err, done = 0.0, 0
    for n, rho in rows:
        if n > done:
            g.ttn_step(w.dt, pkg.TTN_PS1, n - done)
            done = n
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - rho))))
    g.close()
    return err


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_exciton_chain_rank20_100_steps_against_stored_oracle(pkg, precision, tol):
    rows = _stored("exciton7_r20_100steps.txt")
    assert rows[-1][0] == 100
    err = _run(pkg, W.exciton_chain(rank=20), rows, precision)
    assert err <= tol, err


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_exciton_chain_rank64_against_stored_oracle(pkg, precision, tol):
    rows = _stored("exciton7_r64_2steps.txt")
    assert rows[-1][0] == 2
    err = _run(pkg, W.exciton_chain(rank=64), rows, precision)
    assert err <= tol, err
