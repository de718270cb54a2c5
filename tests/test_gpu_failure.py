"""Failure detection in the admitted form: bounded device waits. With the wait
limit set to zero, the grid barriers of the blocked QR's whole-GPU panels and
of the whole-GPU Jacobi SVD give up at their first unsuccessful poll; the
kernels record it in the device flag and run to their end (they exchange only
through global memory, so no CTA leaves while a peer could still write into
its shared memory), the library reports TTN_ETIMEOUT, and the same process then
propagates a fresh handle correctly. No GPU fault, trap or hang is involved."""
import numpy as np
import pytest

import workloads as W
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu

TTN_ETIMEOUT = 5


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def test_grid_panel_qr_zero_wait_then_fresh_handle(pkg):
    w = W.exciton_chain(n_sites=4, depth=4, rank=64)  # a 64 x 64 x 64 node: 4096 x 64 matricisations
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0)
    assert any(int(np.prod(g.ttn_node_shape(u))) >= 4096 * 64 for u in range(len(w.parent)))
    g.ttn_set_params(wait_s=0.0)
    with pytest.raises(pkg.TTNError) as e:
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        g.ttn_rdm()
    assert e.value.status == TTN_ETIMEOUT
    g.close()
    # the context is intact: a fresh handle follows the oracle
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0)
    o = ottn.from_workload(w)
    g.ttn_step(w.dt, pkg.TTN_PS1, 1)
    o.step(w.dt, "ps1")
    err = float(np.max(np.abs(g.ttn_rdm() - o.rdm())))
    g.close()
    assert err <= 1e-10, err


def test_grid_jacobi_zero_wait_in_ps2_then_fresh_handle(pkg):
    # bonds of rank 23 between internal nodes give two-site matrices of 368 x 207,
    # whose Jacobi SVD runs over the whole GPU with one grid barrier per round; the
    # column count is odd, so one CTA holds the dummy pair of every round and
    # reaches the barrier first, where a zero wait gives up at its first poll
    wc = W.exciton_chain(n_sites=3, rank=23, depth=4)

    def generic(g):
        # a generic state (random isometries below a random root): from the product
        # state ps2 would cut every bond to a few directions before the wide pairs
        rng = np.random.default_rng(23)
        for u in range(len(wc.parent)):
            d0, d1, d2 = g.ttn_node_shape(u)
            if u == 0:
                t = rng.normal(size=(d0, d1, d2)) + 1j * rng.normal(size=(d0, d1, d2))
                t /= np.linalg.norm(t)
            else:
                q = np.linalg.qr(rng.normal(size=(d1 * d2, d0)) + 1j * rng.normal(size=(d1 * d2, d0)))[0]
                t = q.T.reshape(d0, d1, d2)  # t[a, b, c] = q[(b, c), a]: orthonormal toward the parent
            g.ttn_set_node(u, t)

    g = pkg.from_model(wc.H, wc.baths, wc.depth, wc.parent, wc.leg_node, wc.ranks, rho0=wc.rho0,
                       params={"max_rank": 32, "ps2_atol": 1e-6, "wait_s": 0.0})
    generic(g)
    nodes0 = [g.ttn_get_node(u) for u in range(len(wc.parent))]
    ranks0, t0 = g.ttn_get_ranks(), g.ttn_time()
    with pytest.raises(pkg.TTNError) as e:
        g.ttn_step(wc.dt, pkg.TTN_PS2, 1)
    assert e.value.status == TTN_ETIMEOUT
    # the ps2 step that gave up put the handle back to the start of the call
    assert np.array_equal(g.ttn_get_ranks(), ranks0) and g.ttn_time() == t0
    for u in range(len(wc.parent)):
        assert np.array_equal(g.ttn_get_node(u), nodes0[u])
    # and it steps on exactly like a handle that never failed
    g.ttn_set_params(wait_s=2.0)
    g.ttn_step(wc.dt, pkg.TTN_PS2, 1)
    g2 = pkg.from_model(wc.H, wc.baths, wc.depth, wc.parent, wc.leg_node, wc.ranks, rho0=wc.rho0,
                        params={"max_rank": 32, "ps2_atol": 1e-6, "wait_s": 2.0})
    generic(g2)
    g2.ttn_step(wc.dt, pkg.TTN_PS2, 1)
    assert np.array_equal(g.ttn_get_ranks(), g2.ttn_get_ranks())
    assert np.array_equal(g.ttn_rdm(), g2.ttn_rdm())
    g.close()
    g2.close()
    w = W.driven_structured_tls(n_pade=1, depth=10, cap=32)
    params = {"max_rank": 32, "ps2_atol": 1e-6, "wait_s": 2.0}
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, drives=w.drives,
                       params=params)
    o = ottn.from_workload(w, params=ottn.Params(ps2_atol=1e-6, max_rank=32))
    for _ in range(3):
        g.ttn_step(w.dt, pkg.TTN_PS2, 1)
        o.step(w.dt, "ps2")
    err = float(np.max(np.abs(g.ttn_rdm() - o.rdm())))
    g.close()
    assert err <= 1e-10, err
