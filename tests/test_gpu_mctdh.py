"""ML-MCTDH (Sec. 3.2.4) as a second sum-of-products workload of the same GPU
path: the thermofield star bath, wavefunction propagation (ps1 and vmf)
against the oracle, and -- the comparison of the paper's MCTDH-versus-HEOM
figure -- the system populations of the MCTDH wavefunction against the HEOM
of the same Brownian bath over the first 100 fs."""
import numpy as np
import pytest

import workloads as W
from oracle import mctdh as omctdh
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _gpu(pkg, w, params=None):
    from paper_2603_17711_gb300 import mctdh
    freqs, gs = mctdh.thermofield_modes(w.bo, w.beta, w.cutoff, w.n_modes)
    t = pkg.TTN(w.parent, w.leg_node, w.leg_dims, w.ranks)
    if params:
        t.ttn_set_params(**params)
    t.sop_load(mctdh.mctdh_sop(w.H, w.Q, freqs, gs, w.dim))
    t.bind()
    t.ttn_set_rdo0(omctdh.rho0(w.psi0))
    return t


def _oracle(w, params=None):
    freqs, gs = omctdh.modes(w.bo, w.beta, w.cutoff, w.n_modes)
    return ottn.TTN(w.parent, w.leg_node, w.leg_dims, w.ranks, omctdh.terms(w.H, w.Q, freqs, gs, w.dim),
                    omctdh.rho0(w.psi0), params=ottn.Params(**(params or {})))


@pytest.mark.parametrize("scheme", ["ps1", "vmf"])
def test_star_boson_wavefunction_against_oracle(pkg, scheme):
    from paper_2603_17711_gb300 import mctdh
    w = W.star_boson_mctdh(n_modes=8, dim=5, rank=6)
    params = {"vmf_atol": 1e-8}  # the product start leaves singular single-hole density matrices
    g, o = _gpu(pkg, w, params), _oracle(w, params)
    code = pkg.TTN_PS1 if scheme == "ps1" else pkg.TTN_VMF
    err = 0.0
    for _ in range(3):  # direct integration after a few fixed-rank steps, as the paper advises
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        o.step(w.dt, "ps1")
    for _ in range(10):
        g.ttn_step(w.dt, code, 1)
        o.step(w.dt, scheme)
        rg = mctdh.rho_from_root(g.ttn_get_node(0).reshape(o.tensors[0].shape))
        err = max(err, float(np.max(np.abs(rg - omctdh.system_rho_root(o)))),
                  float(np.max(np.abs(g.ttn_rdm() - o.rdm()))))
    g.close()
    assert err <= (1e-10 if scheme == "ps1" else 1e-6), err


def test_mctdh_versus_heom_populations(pkg):
    from paper_2603_17711_gb300 import mctdh
    w = W.star_boson_mctdh(n_modes=50, dim=8, rank=8)
    g = _gpu(pkg, w)
    pops = []
    for _ in range(100):
        g.ttn_step(w.dt, pkg.TTN_PS1, 1)
        rho = mctdh.rho_from_root(g.ttn_get_node(0).reshape(w.leg_dims[0], w.leg_dims[1], -1))
        pops.append(rho[1, 1].real)
    g.close()
    # HEOM of the same bath (the Brownian peak alone, Pade with two corrections, depth 20)
    bath = W.Bath(Q=w.Q, beta=w.beta, bo=list(w.bo), n_ltc=2)
    parent, leg_node = W.balanced_binary(bath.n_features)
    h = pkg.from_model(w.H, [bath], [20] * bath.n_features, parent, leg_node, W.uniform_ranks(parent, 20),
                       rho0=np.outer(w.psi0, w.psi0.conj()))
    ref = []
    for _ in range(100):
        h.ttn_step(w.dt, pkg.TTN_PS1, 1)
        ref.append(h.ttn_rdm()[1, 1].real)
    h.close()
    dev = float(np.max(np.abs(np.array(pops) - np.array(ref))))
    print(f"max |P_1(MCTDH) - P_1(HEOM)| over 100 fs: {dev:.3e}")
    assert dev < 0.02, dev
