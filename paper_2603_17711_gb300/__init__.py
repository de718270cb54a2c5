"""GB300-native TTN-HEOM propagation (TENSO method, arXiv 2603.17711).

The compute path is the CUDA library ``libttnheom.so`` (C ABI in
include/ttn_heom.h); this package only marshals arguments to it and lends it
PyTorch device memory and streams. There is no CPU fallback: constructing a
``TTN`` without the built library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Callable, Optional, Sequence

import numpy as np

from . import heom
from ._lib import (DRIVE_FN, TTN_FP64, TTN_MIXED_FP32, TTN_MIX, TTN_OK, TTN_PS1, TTN_PS2, TTN_VMF,
                   TTNError, as_f64, as_i32, ptr, ttn_params, ttn_tree)
from . import _lib

__all__ = ["TTN", "TTNError", "heom", "TTN_FP64", "TTN_MIXED_FP32", "TTN_PS1", "TTN_PS2", "TTN_VMF", "TTN_MIX",
           "library", "from_model", "ttn_batch_step", "ttn_batch_autotune", "RankProposer"]

_LIB: Optional[C.CDLL] = None
_TUNING_FORMAT = "ttn-heom tile shapes 1"


def library() -> C.CDLL:
    """The loaded libttnheom.so (raises if it is not built)."""
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


class TTN:
    """One TTN-HEOM state on the GPU; methods mirror the C ABI entry points."""

    def __init__(self, parent: Sequence[int], leg_node: Sequence[int], leg_dims: Sequence[int],
                 ranks: Sequence[int], precision: int = TTN_FP64):
        self.lib = library()
        self._parent = as_i32(parent)
        self._leg_node = as_i32(leg_node)
        self.leg_dims = as_i32(leg_dims)
        self.M = int(self.leg_dims[0])
        tree = ttn_tree(len(self._parent), ptr(self._parent, C.c_int32), len(self._leg_node),
                        ptr(self._leg_node, C.c_int32))
        h = C.c_void_p()
        st = self.lib.ttn_create(C.byref(tree), ptr(self.leg_dims, C.c_int32), ptr(as_i32(ranks), C.c_int32),
                                 precision, C.byref(h))
        if st != TTN_OK:
            raise TTNError(st, "ttn_create")
        self.h = h
        self.n_nodes = len(self._parent)
        self._drive_cbs = []
        self._ws = None
        self.device = 0

    # -- plumbing -----------------------------------------------------------
    def _check(self, st: int, what: str) -> None:
        if st != TTN_OK:
            msg = self.lib.ttn_last_error(self.h)
            raise TTNError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.ttn_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -------------------------------------------------------
    def ttn_set_params(self, **kw) -> None:
        p = ttn_params()
        self._check(self.lib.ttn_get_params(self.h, C.byref(p)), "ttn_get_params")
        for k, v in kw.items():
            setattr(p, k, v)
        self._check(self.lib.ttn_set_params(self.h, C.byref(p)), "ttn_set_params")

    def sop_load(self, arrays: dict) -> None:
        a = {k: np.ascontiguousarray(v) for k, v in arrays.items()}
        self._sop = a
        n_ops = len(a["op_leg"])
        n_terms = len(a["term_offsets"]) - 1
        self._check(self.lib.sop_load(self.h, n_ops, ptr(as_i32(a["op_leg"]), C.c_int32),
                                      ptr(a["op_offset"].astype(np.int64), C.c_int64),
                                      ptr(as_f64(a["op_data"]), C.c_double), n_terms,
                                      ptr(as_i32(a["term_offsets"]), C.c_int32),
                                      ptr(as_i32(a["term_ops"]), C.c_int32),
                                      ptr(as_f64(a["coef"]), C.c_double),
                                      ptr(as_i32(a["coef_drive"]), C.c_int32)), "sop_load")

    def ttn_set_drive(self, drive_id: int, g: Callable[[float], float], bound: float) -> None:
        cb = DRIVE_FN(lambda t, _u: float(g(t)))
        self._drive_cbs.append(cb)  # keep the trampoline alive
        self._check(self.lib.ttn_set_drive(self.h, drive_id, cb, None, float(bound)), "ttn_set_drive")

    def ttn_workspace_size(self) -> int:
        n = C.c_size_t()
        self._check(self.lib.ttn_workspace_size(self.h, C.byref(n)), "ttn_workspace_size")
        return int(n.value)

    def bind(self, device: int = 0, stream=None) -> None:
        """Allocate the workspace with PyTorch on ``device`` and bind it (ttn_set_stream +
        ttn_set_workspace). ``stream``: a torch.cuda.Stream for all device work
        (default: a new stream owned by this object; use ``self.stream``)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("TTN needs a CUDA device: the library has no CPU path")
        dev = torch.device("cuda", device)
        self.device = device
        n = self.ttn_workspace_size()
        self._ws = torch.empty(n + 256, dtype=torch.uint8, device=dev)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        # a dedicated stream by default: the legacy default stream cannot be
        # captured into the per-step CUDA graph
        s = stream if stream is not None else torch.cuda.Stream(dev)
        self._stream = s
        self._check(self.lib.ttn_set_stream(self.h, C.c_void_p(s.cuda_stream)), "ttn_set_stream")
        self._check(self.lib.ttn_set_workspace(self.h, C.c_void_p(aligned), n), "ttn_set_workspace")

    @property
    def stream(self):
        return self._stream

    def ttn_set_rdo0(self, rho0: np.ndarray) -> None:
        r = np.ascontiguousarray(np.asarray(rho0, np.complex128)).view(np.float64)
        self._check(self.lib.ttn_set_rdo0(self.h, ptr(r, C.c_double)), "ttn_set_rdo0")

    def ttn_step(self, dt: float, scheme: int = TTN_PS1, n_steps: int = 1) -> None:
        self._check(self.lib.ttn_step(self.h, float(dt), int(scheme), int(n_steps)), "ttn_step")

    def ttn_rdm(self) -> np.ndarray:
        out = np.zeros((self.M, self.M), np.complex128)
        self._check(self.lib.ttn_rdm(self.h, ptr(out.view(np.float64), C.c_double)), "ttn_rdm")
        return out

    def ttn_rdm_device(self, dev_ptr: int) -> None:
        self._check(self.lib.ttn_rdm_device(self.h, C.c_void_p(dev_ptr)), "ttn_rdm_device")

    def ttn_get_ranks(self) -> np.ndarray:
        r = np.zeros(self.n_nodes, np.int32)
        self._check(self.lib.ttn_get_ranks(self.h, ptr(r, C.c_int32)), "ttn_get_ranks")
        return r

    def ttn_node_shape(self, u: int):
        d = np.zeros(3, np.int32)
        self._check(self.lib.ttn_node_shape(self.h, u, ptr(d, C.c_int32)), "ttn_node_shape")
        return tuple(int(x) for x in d)

    def ttn_get_node(self, u: int) -> np.ndarray:
        out = np.zeros(self.ttn_node_shape(u), np.complex128)
        self._check(self.lib.ttn_get_node(self.h, u, ptr(out.view(np.float64), C.c_double)), "ttn_get_node")
        return out

    def ttn_set_node(self, u: int, T: np.ndarray) -> None:
        a = np.ascontiguousarray(np.asarray(T, np.complex128))
        if a.shape != self.ttn_node_shape(u):
            raise ValueError("node tensor shape mismatch")
        self._check(self.lib.ttn_set_node(self.h, u, ptr(a.view(np.float64), C.c_double)), "ttn_set_node")

    def ttn_checkpoint_save(self, path: Optional[str] = None) -> bytes:
        """The checkpoint blob (C ABI ttn_checkpoint_save), also written to `path` if given."""
        n = C.c_size_t()
        self._check(self.lib.ttn_checkpoint_size(self.h, C.byref(n)), "ttn_checkpoint_size")
        buf = C.create_string_buffer(int(n.value))
        self._check(self.lib.ttn_checkpoint_save(self.h, buf, n.value), "ttn_checkpoint_save")
        blob = buf.raw
        if path is not None:
            with open(path, "wb") as f:
                f.write(blob)
        return blob

    def ttn_checkpoint_load(self, blob_or_path) -> None:
        """Restore a checkpoint blob (bytes) or file (C ABI ttn_checkpoint_load)."""
        if isinstance(blob_or_path, (bytes, bytearray)):
            blob = bytes(blob_or_path)
        else:
            with open(blob_or_path, "rb") as f:
                blob = f.read()
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.lib.ttn_checkpoint_load(self.h, buf, len(blob)), "ttn_checkpoint_load")

    def ttn_time(self) -> float:
        t = C.c_double()
        self._check(self.lib.ttn_time(self.h, C.byref(t)), "ttn_time")
        return t.value

    def ttn_stats(self, kind: int):
        n, f = C.c_int64(), C.c_double()
        self._check(self.lib.ttn_stats(self.h, kind, C.byref(n), C.byref(f)), "ttn_stats")
        return int(n.value), float(f.value)

    def ttn_profile(self, on) -> None:
        """on: False/0 off, True/1 events around every launch (no step graph),
        2 events as nodes inside the replayed step graph."""
        mode = 2 if on == 2 else (1 if on else 0)
        self._check(self.lib.ttn_profile(self.h, mode), "ttn_profile")

    def ttn_profile_read(self, kind: int) -> float:
        ms = C.c_double()
        self._check(self.lib.ttn_profile_read(self.h, kind, C.byref(ms)), "ttn_profile_read")
        return float(ms.value)

    def ttn_stats_reset(self) -> None:
        self._check(self.lib.ttn_stats_reset(self.h), "ttn_stats_reset")

    def ttn_autotune(self, reps: int = 3, cache: Optional[str] = None) -> str:
        """Pick the tile shape (warps per CTA, CTAs per tile) of every job list
        by timing (ttn_autotune). cache: path of a JSON file of tile shapes
        keyed by list shape; when it holds a shape for every list of this
        handle on this device those are used as they are ("cache"), else the
        lists are timed ("tuned") and their shapes merged into the file."""
        dev = self._device_tag()
        old_rows = []
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                doc = json.load(f)
            if doc.get("format") == _TUNING_FORMAT and doc.get("device") == dev:
                old_rows = [list(map(int, r)) for r in doc.get("rows", [])]
                if self.ttn_tuning_set(np.asarray(old_rows, np.int32).reshape(-1, _lib.TTN_TUNING_COLS)) == \
                        len(self.ttn_tuning_get()):
                    return "cache"
        self._check(self.lib.ttn_autotune(self.h, int(reps)), "ttn_autotune")
        if cache is not None:
            mine = self.ttn_tuning_get().tolist()
            have = {tuple(r[:9]) for r in mine}
            rows = mine + [r for r in old_rows if tuple(r[:9]) not in have]
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump({"format": _TUNING_FORMAT, "device": dev,
                           "columns": ["kind", "precision", "d0", "d1", "d2", "d3_or_leg", "outputs", "terms",
                                       "tiles", "warps", "split"], "rows": rows}, f)
            os.replace(tmp, cache)
        return "tuned"

    def _device_tag(self) -> str:
        import torch
        pr = torch.cuda.get_device_properties(self.device)
        return f"{pr.name} / {pr.multi_processor_count} SMs"

    def ttn_tuning_get(self) -> np.ndarray:
        """Tile shapes of every job list: int32 [n_lists, 11] rows (9 key values,
        warps per CTA, CTAs per tile)."""
        n = C.c_int32()
        self._check(self.lib.ttn_tuning_get(self.h, None, 0, C.byref(n)), "ttn_tuning_get")
        rows = np.zeros((n.value, _lib.TTN_TUNING_COLS), np.int32)
        if n.value:
            self._check(self.lib.ttn_tuning_get(self.h, ptr(rows, C.c_int32), n.value, C.byref(n)), "ttn_tuning_get")
        return rows

    def ttn_tuning_set(self, rows: np.ndarray) -> int:
        """Give every list whose key matches a row that row's tile shape;
        returns the number of lists set."""
        r = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, _lib.TTN_TUNING_COLS)
        n = C.c_int32()
        self._check(self.lib.ttn_tuning_set(self.h, ptr(r, C.c_int32), len(r), C.byref(n)), "ttn_tuning_set")
        return n.value

    def ttn_split_log(self):
        """(features [n, 24] float32, classes [n] int32) of the full-SVD ps2 splits so far."""
        n = C.c_int32()
        self._check(self.lib.ttn_split_log(self.h, None, None, 0, C.byref(n)), "ttn_split_log")
        f = np.zeros((n.value, 24), np.float32)
        y = np.zeros(n.value, np.int32)
        if n.value:
            self._check(self.lib.ttn_split_log(self.h, f.ctypes.data_as(C.POINTER(C.c_float)), ptr(y, C.c_int32),
                                               n.value, C.byref(n)), "ttn_split_log")
        return f, y

    def ttn_split_log_clear(self) -> None:
        self._check(self.lib.ttn_split_log_clear(self.h), "ttn_split_log_clear")

    def ttn_set_rank_proposer(self, proposer) -> None:
        """Use a RankProposer's parameters at every ps2 split (None: off)."""
        self._proposer = proposer
        addr = proposer.params.data_ptr() if proposer is not None else None
        self._check(self.lib.ttn_set_rank_proposer(self.h, C.c_void_p(addr)), "ttn_set_rank_proposer")

    def ttn_proposer_stats(self):
        a, b = C.c_int64(), C.c_int64()
        self._check(self.lib.ttn_proposer_stats(self.h, C.byref(a), C.byref(b)), "ttn_proposer_stats")
        return int(a.value), int(b.value)

    def ttn_substeps(self, tau: float) -> int:
        m = C.c_int32()
        self._check(self.lib.ttn_substeps(self.h, float(tau), C.byref(m)), "ttn_substeps")
        return int(m.value)


class RankProposer:
    """The 24-64-64-13 rank-proposer MLP: parameters and Adam state live in
    CUDA tensors; forward, gradient and Adam run in the library's kernels."""

    def __init__(self, seed: int = 0, params: Optional[np.ndarray] = None, device: int = 0):
        import torch
        n = C.c_int32()
        library().ttn_mlp_n_params(C.byref(n))
        self.n_params = int(n.value)
        if params is None:
            params = RankProposer.init_params(seed)
        assert params.shape == (self.n_params,)
        dev = torch.device("cuda", device)
        self.params = torch.tensor(params, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.t = 0
        self.dev = dev

    @staticmethod
    def init_params(seed: int) -> np.ndarray:
        """He-normal weights (std sqrt(2/fan_in)), zero biases, in the packed order."""
        rng = np.random.default_rng(seed)
        parts = []
        for fan_out, fan_in in ((64, 24), (64, 64), (13, 64)):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        return np.concatenate(parts).astype(np.float32)

    def _ws(self, batch: int):
        import torch
        b = C.c_size_t()
        library().ttn_mlp_workspace_size(batch, C.byref(b))
        return torch.empty(int(b.value) // 4 + 1, dtype=torch.float32, device=self.dev)

    def forward(self, x):
        import torch
        x = torch.as_tensor(np.ascontiguousarray(x, np.float32), device=self.dev)
        B = x.shape[0]
        z = torch.empty(B, 13, dtype=torch.float32, device=self.dev)
        ws = self._ws(B)
        st = library().ttn_mlp_forward(C.c_void_p(self.params.data_ptr()), C.c_void_p(x.data_ptr()), B,
                                       C.c_void_p(z.data_ptr()), C.c_void_p(ws.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream))
        if st != TTN_OK:
            raise TTNError(st, "ttn_mlp_forward")
        return z

    def grad(self, x, y):
        import torch
        x = torch.as_tensor(np.ascontiguousarray(x, np.float32), device=self.dev)
        y = torch.as_tensor(np.ascontiguousarray(y, np.int32), device=self.dev)
        B = x.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        ws = self._ws(B)
        st = library().ttn_mlp_grad(C.c_void_p(self.params.data_ptr()), C.c_void_p(x.data_ptr()),
                                    C.c_void_p(y.data_ptr()), B, C.c_void_p(self.grads.data_ptr()),
                                    C.c_void_p(loss.data_ptr()), C.c_void_p(ws.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream))
        if st != TTN_OK:
            raise TTNError(st, "ttn_mlp_grad")
        return loss, self.grads

    def adam(self, lr: float) -> None:
        import torch
        self.t += 1
        st = library().ttn_mlp_adam(C.c_void_p(self.params.data_ptr()), C.c_void_p(self.m.data_ptr()),
                                    C.c_void_p(self.v.data_ptr()), C.c_void_p(self.grads.data_ptr()), self.t,
                                    float(lr), C.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream))
        if st != TTN_OK:
            raise TTNError(st, "ttn_mlp_adam")

    def train(self, feats, labels, steps: int = 300, lr: float = 3e-3):
        """Full-batch Adam on (features, classes); returns the loss history."""
        hist = []
        for _ in range(steps):
            loss, _ = self.grad(feats, labels)
            self.adam(lr)
            hist.append(loss)
        return [float(l.item()) for l in hist]


def ttn_batch_step(handles: Sequence["TTN"], dt: float, scheme: int = TTN_PS1, n_steps: int = 1) -> None:
    """Step several TTN handles together (C ABI ttn_batch_step)."""
    if not handles:
        return
    arr = (C.c_void_p * len(handles))(*[t.h for t in handles])
    st = library().ttn_batch_step(arr, len(handles), float(dt), int(scheme), int(n_steps))
    if st != TTN_OK:
        msg = library().ttn_last_error(handles[0].h)
        raise TTNError(st, f"ttn_batch_step: {msg.decode() if msg else ''}")


def ttn_batch_autotune(handles: Sequence["TTN"], dt: float, reps: int = 2) -> dict:
    """Tile shape of a batch (C ABI ttn_batch_autotune): warps per CTA chosen by
    timing the batched step; the members' states are put back afterwards.
    Returns {"warps": w, "ms_per_batched_step": {8: .., 4: .., 2: ..}}."""
    arr = (C.c_void_p * len(handles))(*[t.h for t in handles])
    w = C.c_int32()
    ms = (C.c_float * 3)()
    st = library().ttn_batch_autotune(arr, len(handles), float(dt), int(reps), C.byref(w), ms)
    if st != TTN_OK:
        msg = library().ttn_last_error(handles[0].h)
        raise TTNError(st, f"ttn_batch_autotune: {msg.decode() if msg else ''}")
    return {"warps": int(w.value), "ms_per_batched_step": {8: float(ms[0]), 4: float(ms[1]), 2: float(ms[2])}}


def pad_to_three_legs(parent: Sequence[int], leg_node: Sequence[int], leg_dims: Sequence[int]):
    """The library's nodes have exactly three legs. A tree with two-leg nodes
    (e.g. the arm ends of a centred train, Sec. 7.2 custom frames) is given one
    extra open leg of dimension 1 on each such node, appended after the other
    legs: no operator acts on it and its only index is the n = 0 state, so the
    EDO, the generator and rho_S are unchanged. Returns (leg_node, leg_dims)."""
    n = len(parent)
    count = [0 if u == 0 else 1 for u in range(n)]
    for u in range(1, n):
        count[parent[u]] += 1
    for u in leg_node:
        count[u] += 1
    leg_node, leg_dims = list(leg_node), list(leg_dims)
    for u in range(n):
        if count[u] == 2:
            leg_node.append(u)
            leg_dims.append(1)
    return leg_node, leg_dims


def from_model(H, baths, depth, parent, leg_node, ranks, rho0=None, drives=(), precision=TTN_FP64,
               params: Optional[dict] = None, device: int = 0, stream=None) -> TTN:
    """Build, load and bind a TTN for the HEOM of system ``H`` with ``baths``
    (objects with Q, beta, dl, bo, n_ltc, scheme) and ``drives`` (objects with
    V, g(t), bound). Two-leg nodes are padded (pad_to_three_legs)."""
    M = np.asarray(H).shape[0]
    leg_node, leg_dims = pad_to_three_legs(parent, leg_node, [M, M] + list(depth))
    t = TTN(parent, leg_node, leg_dims, ranks, precision)
    if params:
        t.ttn_set_params(**params)
    t.sop_load(heom.heom_sop(H, baths, depth, drives))
    for d, dr in enumerate(drives):
        t.ttn_set_drive(d, dr.g, dr.bound)
    t.bind(device, stream)
    if rho0 is not None:
        t.ttn_set_rdo0(rho0)
    return t


def svd(a, wait_s: float = 2.0):
    """FP64 Jacobi SVD of a complex128 CUDA matrix through the C ABI ttn_svd:
    returns (U, sigma, Vh, sweeps) with a = U diag(sigma) Vh, sigma descending
    (numpy), U and Vh CUDA tensors."""
    import torch
    if a.dtype != torch.complex128 or not a.is_cuda or a.dim() != 2:
        raise ValueError("svd expects a 2-D complex128 CUDA tensor")
    a = a.contiguous()
    m, n = a.shape
    k = min(m, n)
    nbytes = C.c_size_t()
    st = library().ttn_svd_workspace_size(m, n, C.byref(nbytes))
    if st != TTN_OK:
        raise TTNError(st, "ttn_svd_workspace_size")
    ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=a.device)
    base = (ws.data_ptr() + 255) // 256 * 256
    U = torch.empty(m, k, dtype=torch.complex128, device=a.device)
    Vh = torch.empty(k, n, dtype=torch.complex128, device=a.device)
    sig = np.zeros(k, np.float64)
    sweeps = C.c_int32()
    st = library().ttn_svd(C.c_void_p(a.data_ptr()), m, n, C.c_void_p(U.data_ptr()), ptr(sig, C.c_double),
                           C.c_void_p(Vh.data_ptr()), C.c_void_p(base), int(nbytes.value), float(wait_s),
                           C.byref(sweeps), C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream))
    if st != TTN_OK:
        raise TTNError(st, "ttn_svd")
    return U, sig, Vh, int(sweeps.value)
