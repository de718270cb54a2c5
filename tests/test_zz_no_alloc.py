"""ttn_rdm_noalloc: the reduced density matrix for callers that cannot allocate
device memory (framework-managed arenas, runtimes that forbid allocation after
start-up). The paper has no counterpart; the call must agree with ttn_rdm, the
handle-based entry point, on the same state -- here on two calls in a row, the
second after the state moved on, so stale scratch from the first call would
show. Kept in its own file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the GPU parity tolerance used for short runs


def _tree(w):
    from paper_2603_17711_gb300 import _lib
    par, ln = _lib.as_i32(w.parent), _lib.as_i32(w.leg_node)
    t = _lib.ttn_tree(len(par), _lib.ptr(par, C.c_int32), len(ln), _lib.ptr(ln, C.c_int32))
    return t, (par, ln)


def test_noalloc_rdm_matches_handle_rdm_on_two_calls():
    import torch
    import paper_2603_17711_gb300 as pkg
    from paper_2603_17711_gb300 import _lib
    assert torch.cuda.is_available()
    lib = pkg.library()
    w = W.spin_boson_tt(depth=5, n_pade=3, rank=6, tree="btt")
    g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0)
    tree, keep = _tree(w)
    leg_dims = _lib.as_i32(w.leg_dims)
    ranks = _lib.as_i32(w.ranks)
    rho_dev = torch.empty(2 * w.M * w.M, dtype=torch.float64, device="cuda")
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        g.ttn_step(w.dt, pkg.TTN_PS1, 4)
        nodes = [torch.from_numpy(g.ttn_get_node(u).reshape(-1).view(np.float64).copy()).cuda()
                 for u in range(len(w.parent))]
        ptrs = (C.c_void_p * len(nodes))(*[t.data_ptr() for t in nodes])
        rho_dev.fill_(float("nan"))
        st = lib.ttn_rdm_noalloc(C.byref(tree), _lib.ptr(leg_dims, C.c_int32), _lib.ptr(ranks, C.c_int32),
                                 ptrs, C.c_void_p(rho_dev.data_ptr()), C.c_void_p(stream), err, len(err))
        assert st == 0, err.value.decode()
        torch.cuda.synchronize()
        got = rho_dev.cpu().numpy().view(np.complex128).reshape(w.M, w.M)
        ref = g.ttn_rdm()
        assert np.max(np.abs(got - ref)) <= TOL, f"call {call}"
    g.close()


def test_noalloc_rdm_refuses_trees_beyond_its_scratch():
    from paper_2603_17711_gb300 import _lib
    import paper_2603_17711_gb300 as pkg
    lib = pkg.library()
    K = 300
    parent, leg_node = W.tensor_train(K)
    w = W.spin_boson_tt(depth=16, n_pade=K - 1, rank=256)
    assert w.parent == parent
    tree, keep = _tree(w)
    err = C.create_string_buffer(256)
    ptrs = (C.c_void_p * len(parent))(*([1] * len(parent)))
    st = lib.ttn_rdm_noalloc(C.byref(tree), _lib.ptr(_lib.as_i32(w.leg_dims), C.c_int32),
                             _lib.ptr(_lib.as_i32(w.ranks), C.c_int32), ptrs, C.c_void_p(1), None, err, len(err))
    assert st == 1
    assert b"limit is 65536" in err.value
