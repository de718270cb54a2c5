"""GPU Jacobi SVD (the ps2 split, Sec. 2.3 last paragraph) through the C ABI
ttn_svd, against LAPACK (numpy.linalg.svd) on the CPU: singular values,
reconstruction, orthonormality, the sweep count, both the one-CTA and the
whole-GPU kernels, and the bounded grid wait (a zero wait limit must come back
as TTN_ETIMEOUT with the context still usable)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_17711_gb300 as p
    p.library()
    return p


def _rand(rng, m, n):
    return rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))


def _check(pkg, A, tol=1e-13):
    import torch
    a = torch.as_tensor(A, device="cuda")
    U, s, Vh, sweeps = pkg.svd(a)
    U, Vh = U.cpu().numpy(), Vh.cpu().numpy()
    s_ref = np.linalg.svd(A, compute_uv=False)
    scale = max(s_ref[0], 1e-300)
    assert np.max(np.abs(s - s_ref)) <= tol * scale
    assert np.max(np.abs((U * s) @ Vh - A)) <= tol * scale * np.sqrt(max(A.shape))
    k = int(np.sum(s > 1e-12 * scale))
    assert np.max(np.abs(U[:, :k].conj().T @ U[:, :k] - np.eye(k))) <= 1e-12
    assert np.max(np.abs(Vh[:k] @ Vh[:k].conj().T - np.eye(k))) <= 1e-12
    return sweeps


# one CTA up to 16 columns, one thread-block cluster for 17..32 (also with
# many rows, and a wide matrix taken through its conjugate transpose), the
# whole GPU beyond
@pytest.mark.parametrize("m,n", [(20, 12), (12, 20), (30, 16), (33, 17), (40, 24), (24, 40), (50, 32), (200, 33),
                                 (4000, 20), (31, 1500), (64, 64), (100, 37), (37, 100), (300, 120), (144, 100),
                                 (600, 71)])
def test_svd_matches_lapack(pkg, m, n):
    rng = np.random.default_rng(m * 1000 + n)
    sweeps = _check(pkg, _rand(rng, m, n))
    assert 1 <= sweeps <= 15


def test_svd_sweep_count_64x64(pkg):
    """A generic 64 x 64 complex matrix converges in a handful of sweeps with the
    size-scaled threshold (a threshold below the rounding floor would run all
    60 and report TTN_ENUMERIC)."""
    rng = np.random.default_rng(64)
    sweeps = _check(pkg, _rand(rng, 64, 64))
    assert sweeps <= 12


def test_svd_graded_and_rank_deficient(pkg):
    """Singular values spread over 14 decades and an exactly rank-deficient
    matrix (what a two-site Theta after truncation looks like)."""
    rng = np.random.default_rng(7)
    m, n = 200, 60
    Q1 = np.linalg.qr(_rand(rng, m, n))[0]
    Q2 = np.linalg.qr(_rand(rng, n, n))[0]
    s = 10.0 ** (-np.arange(n) / 4.3)
    _check(pkg, (Q1 * s) @ Q2.conj().T, tol=1e-13)
    B = _rand(rng, m, 9) @ _rand(rng, 9, n)
    _check(pkg, B, tol=1e-13)


def test_svd_zero_wait_limit_times_out_then_context_is_usable(pkg):
    """A grid barrier with a zero wait limit gives up at its first unsuccessful
    poll: the call returns TTN_ETIMEOUT (no fault, no hang; the kernel issues
    plain loads and stores only, so a CTA can leave at any barrier), and the
    next call on the same context is correct."""
    import torch
    rng = np.random.default_rng(9)
    # 36 pairs: a grid barrier per round; the odd column count leaves one CTA
    # idle each round, so it reaches the barrier first and gives up there
    A = _rand(rng, 600, 71)
    a = torch.as_tensor(A, device="cuda")
    with pytest.raises(pkg.TTNError) as e:
        pkg.svd(a, wait_s=0.0)
    assert e.value.status == 5  # TTN_ETIMEOUT
    _check(pkg, A)
