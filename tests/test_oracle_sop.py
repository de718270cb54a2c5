"""Pins for oracle.sop (Eq. heom-std, Eq. dissipator, Eq. master_lvn): the dense
generator assembled from the product terms equals an independently written
textbook HEOM in ADM-index form (conventional metric, Sec. 2.2), the term count
is 5K+2, and the reduced density matrix does not depend on the metric (Sec. 7.4)."""
import itertools

import numpy as np
import scipy.sparse as sp

import workloads as W
from oracle import bcf, dense, sop


def _two_bath_model():
    M = 3
    rng = np.random.default_rng(7)
    H = W.random_hermitian(rng, M)
    Q1 = np.diag([1.0, 0.0, -1.0]).astype(complex)
    Q2 = W.random_hermitian(rng, M)
    baths = [W.Bath(Q=Q1, beta=0.8, dl=(0.4, 1.2), n_ltc=1),
             W.Bath(Q=Q2, beta=1.3, bo=[(0.2, 1.5, 0.4)], n_ltc=0)]
    depth = [3, 2, 3, 2]
    return H, baths, depth


def textbook_heom(H, baths, depth):
    """d rho_n/dt = -i[H, rho_n] + sum_k gamma_k n_k rho_n - i sum_k [Q_k, rho_{n+e_k}]
    - i sum_k n_k (c_k Q_k rho_{n-e_k} - cbar_k rho_{n-e_k} Q_k), C(t) = sum c_k e^{gamma_k t}."""
    M = H.shape[0]
    feats, Qs = [], []
    for b in baths:
        for f in bcf.bath_features(b.beta, b.dl, b.bo, b.n_ltc, b.scheme):
            feats.append(f)
            Qs.append(b.Q)
    K = len(feats)
    shape = [M, M] + list(depth)
    n_tot = int(np.prod(shape))
    idx = lambda i, j, n: np.ravel_multi_index((i, j) + tuple(n), shape)
    L = sp.lil_matrix((n_tot, n_tot), dtype=complex)
    for n in itertools.product(*[range(d) for d in depth]):
        for i in range(M):
            for j in range(M):
                row = idx(i, j, n)
                for l in range(M):
                    L[row, idx(l, j, n)] += -1j * H[i, l]
                    L[row, idx(i, l, n)] += 1j * H[l, j]
                L[row, row] += sum(feats[k][2] * n[k] for k in range(K))
                for k in range(K):
                    c, cb, _ = feats[k]
                    Q = Qs[k]
                    up = list(n)
                    up[k] += 1
                    if up[k] < depth[k]:
                        for l in range(M):
                            L[row, idx(l, j, up)] += -1j * Q[i, l]
                            L[row, idx(i, l, up)] += 1j * Q[l, j]
                    dn = list(n)
                    dn[k] -= 1
                    if dn[k] >= 0:
                        for l in range(M):
                            L[row, idx(l, j, dn)] += -1j * n[k] * c * Q[i, l]
                            L[row, idx(i, l, dn)] += 1j * n[k] * cb * Q[l, j]
    return L.tocsr()


def test_term_count_is_5K_plus_2():
    H, baths, depth = _two_bath_model()
    terms = sop.heom_terms(H, baths, depth)
    K = sum(b.n_features for b in baths)
    assert K == 4 and len(terms) == 5 * K + 2


def test_sop_generator_equals_textbook_heom():
    H, baths, depth = _two_bath_model()
    terms = sop.heom_terms(H, baths, depth, metric="conventional")
    L = dense.generator(terms, dense.leg_dims(H.shape[0], depth))
    Lt = textbook_heom(H, baths, depth)
    assert abs(L - Lt).max() < 1e-12


def test_metric_independence_of_rho_s():
    H, baths, depth = _two_bath_model()
    rho0 = W.random_density_matrix(np.random.default_rng(3), H.shape[0])
    ref = None
    for metric in ("abs", "conventional", 0.37 + 0.2j):
        terms = sop.heom_terms(H, baths, depth, metric=metric)
        tr = dense.propagate(terms, rho0, depth, 0.05, 20)
        if ref is None:
            ref = tr
        assert np.max(np.abs(tr - ref)) < 1e-11


def test_lambda_bound_dominates_generator_norm():
    H, baths, depth = _two_bath_model()
    terms = sop.heom_terms(H, baths, depth)
    L = dense.generator(terms, dense.leg_dims(H.shape[0], depth)).toarray()
    assert np.linalg.norm(L, 2) <= sop.lambda_bound(terms) * (1 + 1e-12)
