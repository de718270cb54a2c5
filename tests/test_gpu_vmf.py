"""Direct integration (vmf, Sec. 2.3 and Sec. 7.5) and the ps2-then-vmf mix
strategy on the GPU against the FP64 oracle: the same node equations under the
same Dormand-Prince controller. Where both sides take the same steps the
results agree to rounding; the tolerance below also covers a controller
decision taken differently near err = 1 (an error of the order of ode_atol)."""
import numpy as np
import pytest
from scipy.sparse.linalg import expm_multiply

import workloads as W
from oracle import dense, sop
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _both(pkg, w, params):
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, drives=w.drives,
                       params=params)
    o = ottn.from_workload(w, params=ottn.Params(**{k: v for k, v in params.items()
                                                    if k in ottn.Params.__dataclass_fields__}))
    return g, o


def _generic(pkg, g, o, w, rng):
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    L = dense.generator(terms, w.leg_dims)
    v = expm_multiply(0.2 * L, dense.initial_vector(w.rho0, w.depth))
    v = v + 1e-3 * (rng.normal(size=v.shape) + 1j * rng.normal(size=v.shape))
    o.tensors = ottn.htd_tensors(o.tree, o.leg_dims, o.ranks, v.reshape(w.leg_dims))
    for c in o.tree.postorder():
        if c:
            o.update_env(c, o.tree.parent[c])
    for u, t in enumerate(o.tensors):
        g.ttn_set_node(u, t)
    return L, v


def test_vmf_untruncated_against_oracle_and_dense(pkg):
    w = W.spin_boson_tt(depth=3, n_pade=2, rank=1000, tree="btt")
    g, o = _both(pkg, w, {"ode_rtol": 1e-10, "ode_atol": 1e-12, "vmf_atol": 0.0, "max_rank": 1000})
    L, v = _generic(pkg, g, o, w, np.random.default_rng(3))
    err = 0.0
    for _ in range(5):
        g.ttn_step(0.02, pkg.TTN_VMF, 1)
        o.step(0.02, "vmf")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    ref = expm_multiply(0.1 * L, v)
    assert np.max(np.abs(g.ttn_rdm() - dense.rdm(ref, 2, w.depth))) < 1e-8
    g.close()
    assert err < 1e-10, err


@pytest.mark.parametrize("make,n,dt,generic", [
    # product start: singular single-hole density matrices, the regularisation at work
    (lambda: W.exciton_chain(n_sites=3, depth=4, rank=6), 6, 0.05, False),
    # a generic point of the rank-5 manifold (truncated tree of a perturbed exact state)
    (lambda: W.spin_boson_tt(depth=6, n_pade=3, rank=5, tree="tt"), 10, 0.01, True),
])
def test_vmf_truncated_against_oracle(pkg, make, n, dt, generic):
    w = make()
    g, o = _both(pkg, w, {"vmf_atol": 1e-8})
    if generic:
        _generic(pkg, g, o, w, np.random.default_rng(4))
    err = 0.0
    for _ in range(n):
        g.ttn_step(dt, pkg.TTN_VMF, 1)
        o.step(dt, "vmf")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err < 1e-6, err


def test_vmf_driven(pkg):
    w = W.driven_structured_tls(n_pade=1, depth=5, cap=8)
    w.ranks = W.uniform_ranks(w.parent, 4)
    g, o = _both(pkg, w, {"vmf_atol": 1e-8})
    err = 0.0
    for _ in range(8):
        g.ttn_step(w.dt, pkg.TTN_VMF, 1)
        o.step(w.dt, "vmf")
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err < 1e-6, err


def test_mix_ps2_then_vmf_against_oracle(pkg):
    w = W.spin_boson_tt(depth=5, n_pade=2, rank=2, tree="btt")
    params = {"ps2_atol": 1e-9, "max_rank": 6}
    g, o = _both(pkg, w, params)
    err = 0.0
    for k in range(12):
        g.ttn_step(0.01, pkg.TTN_MIX, 1)
        o.step(0.01, "mix")
        assert list(g.ttn_get_ranks()) == o.ranks, k
        err = max(err, float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    assert getattr(o, "_mixed_to_vmf", False)
    g.close()
    assert err < 1e-6, err
