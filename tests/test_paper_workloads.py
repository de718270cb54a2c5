"""The paper's example models as workloads (Sec. 3.2 Table 1 and its listing,
Sec. 3.4 FMO listing, Sec. 3.2.3 Table 2): their feature counts as the paper
states them, and the oracle on small-depth versions against the dense
hierarchy (untruncated ranks), so that the unit conversions and parameter
mappings of the generators are exercised through independent arithmetic."""
import numpy as np
import pytest

import workloads as W
from oracle import bcf, dense, sop, ttn


def test_feature_counts_as_printed():
    # Example 2: six Brownian peaks at 77 K with three corrections: 15 per site, 45 in all
    w = W.fmo3(T=77.0)
    assert w.K == 45 and all(b.n_features == 15 for b in w.baths)
    assert W.fmo3(T=300.0).K == 3 * (12 + 1)
    assert W.fmo3(T=300.0, spectral="bo3").K == 3 * (6 + 1)
    assert W.fmo3(T=300.0, spectral="dl").K == 3 * (1 + 1)
    # Example 1: Drude + one Brownian peak (two features) + one Pade correction
    assert W.structured_spin_boson().K == 4
    assert W.convergence_spin_boson("a").K == 2 and W.convergence_spin_boson("b").K == 4


def test_structured_bath_bcf_matches_quadrature():
    """The structured spin-boson bath (Drude 540/70 + Brownian 161.6/10/1243 cm^-1
    at 300 K) decomposed into features against the direct integral of its
    spectral density (Eq. 2 with J = J_DL + J_BO), once the low-temperature
    correction is replaced by enough Matsubara terms to converge."""
    from scipy.integrate import quad
    b = W.structured_spin_boson().baths[0]
    feats = bcf.bath_features(b.beta, dl=b.dl, bo=b.bo, n_ltc=2000, scheme="matsubara")

    def J(w):
        return bcf.J_dl(w, *b.dl) + sum(bcf.J_bo(w, *p) for p in b.bo)

    for t in (2.0, 10.0, 30.0):  # fs
        # QUADPACK QAWF over (0, inf) with the oscillatory weight
        re = quad(lambda w: J(w) / np.tanh(b.beta * w / 2), 1e-12, np.inf, weight="cos", wvar=t, limlst=400)[0]
        im = -quad(J, 0, np.inf, weight="sin", wvar=t, limlst=400)[0]
        C, _ = bcf.bcf_from_features(feats, np.array([t]))
        assert abs(C[0] - (re + 1j * im)) < 1e-3 * (abs(re) + abs(im)), (t, C[0], re + 1j * im)


@pytest.mark.parametrize("make", [
    lambda: W.structured_spin_boson(depth=4, rank=1000, dt=0.5),
    lambda: W.convergence_spin_boson("a", depth=5, rank=1000, dt=0.5),
    lambda: W.fmo3(T=300.0, spectral="dl", depth=3, rank=1000, dt=0.5),
])
def test_small_depth_oracle_equals_dense(make):
    """At untruncated ranks the TTN propagation equals the dense hierarchy up
    to the RK4 error; kappa = 0.5 (five times the default substeps) puts that
    error below 1e-7 for these stiff baths."""
    w = make()
    terms = sop.heom_terms(w.H, w.baths, w.depth)
    ref = dense.propagate(terms, w.rho0, w.depth, w.dt, 8)
    st = ttn.from_workload(w, params=ttn.Params(kappa=0.5))
    err = 0.0
    for k in range(8):
        st.step(w.dt, "ps1")
        err = max(err, float(np.max(np.abs(st.rdm() - ref[k + 1]))))
    assert err < 1e-7, err
