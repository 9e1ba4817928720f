"""Python front end: the C-ABI calls with PyTorch providing device memory and streams.

Every numerical step runs in the CUDA library; this module only converts
arguments (numpy couplings -> host double pointers, torch tensors -> device
pointers, the current torch stream -> cudaStream_t) and caches workspaces.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _lib

PREC = {"fp32": 0, "fp64": 1}
METHOD = {"chebyshev": 0, "cf": 1, "remez": 2}
PATH = {"auto": 0, "plain": 1, "fused": 2, "cluster": 3}

_ws_cache = {}


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def precision_of(psi) -> str:
    import torch

    if psi.dtype == torch.complex64:
        return "fp32"
    if psi.dtype == torch.complex128:
        return "fp64"
    raise TypeError(f"psi must be complex64 or complex128, got {psi.dtype}")


def _check_state(psi, n: int):
    import torch

    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("psi must be a CUDA tensor")
    if not psi.is_contiguous() or psi.numel() != (1 << n):
        raise ValueError(f"psi must be contiguous with 2^{n} elements")


def workspace_bytes(n: int, precision: str) -> int:
    return int(_lib.lib().cheb_workspace_bytes(n, PREC[precision]))


def workspace(n: int, precision: str, device=None):
    """A cached device workspace (torch uint8 tensor) large enough for (n, precision)."""
    import torch

    dev = torch.device(device if device is not None else "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    need = workspace_bytes(n, precision)
    if need == 0:
        raise ValueError(f"unsupported n={n}")
    key = dev.index
    ws = _ws_cache.get(key)
    if ws is None or ws.numel() < need:
        _ws_cache.pop(key, None)
        ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        _ws_cache[key] = ws
    return ws


def _ws_ptr(ws):
    p = ws.data_ptr()
    return (p + 255) // 256 * 256, ws.numel() - ((p + 255) // 256 * 256 - p)


def _stream_ptr(device=None):
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def release_workspaces():
    _ws_cache.clear()


def check_status(n: int, precision: str, device=None):
    """Raise if a bounded wait ran out (or a launch was refused) during an earlier call
    that ran without an info struct on the cached workspace of (n, precision)
    (cheb_workspace_status; synchronises, clears the recorded condition)."""
    ws = workspace(n, precision, device)
    p, nb = _ws_ptr(ws)
    _lib.check(_lib.lib().cheb_workspace_status(ctypes.c_void_p(p), nb, _stream_ptr(ws.device)),
               "cheb_workspace_status")


def coefficients(a: float, tol: float, method: str = "chebyshev", phase: complex = 1.0, max_K: int = 1 << 16):
    """Host coefficient generator; returns (complex array c_0..c_K, err_bound)."""
    buf = np.empty(2 * (max_K + 1))
    K = ctypes.c_int(0)
    err = ctypes.c_double(0.0)
    code = _lib.lib().cheb_coefficients(float(a), float(np.real(phase)), float(np.imag(phase)), float(tol),
                                        METHOD[method], int(max_K), _dp(buf), ctypes.byref(K), ctypes.byref(err))
    _lib.check(code, "cheb_coefficients")
    return buf[: 2 * (K.value + 1)].view(np.complex128).copy(), err.value


def ising_bounds(h, J, device=None):
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    ws = workspace(n, "fp32", device)
    p, nb = _ws_ptr(ws)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    code = _lib.lib().cheb_ising_bounds(n, _dp(h), _dp(J), ctypes.c_void_p(p), nb, _stream_ptr(ws.device),
                                        ctypes.byref(lo), ctypes.byref(hi))
    _lib.check(code, "cheb_ising_bounds")
    return lo.value, hi.value


EVAL_BOUND_FLAG = 0x100  # CHEB_FLAG_EVAL_BOUND


def expmv(h, J, gamma: float, t: float, psi, tol: Optional[float] = None, method: str = "chebyshev",
          time_splits: int = 0, path: str = "auto", info: bool = True, eval_bound: bool = False):
    """psi <- exp(-i t H) psi in place on the GPU; returns the info dict (or None).
    eval_bound=True also fills info["eval_bound"] (CHEB_FLAG_EVAL_BOUND)."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    _check_state(psi, n)
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    inf = _lib.Info()
    code = _lib.lib().cheb_expmv_path(n, _dp(h), _dp(J), float(gamma), float(t), ctypes.c_void_p(psi.data_ptr()),
                                      PREC[prec], float(tol), METHOD[method], int(time_splits),
                                      PATH[path] | (EVAL_BOUND_FLAG if eval_bound else 0),
                                      ctypes.c_void_p(p), nb, _stream_ptr(psi.device),
                                      ctypes.byref(inf) if (info or eval_bound) else None)
    _lib.check(code, "cheb_expmv")
    return inf.as_dict() if (info or eval_bound) else None


def anneal(h, J, gammas, ts, psi, tol: Optional[float] = None, method: str = "chebyshev", boundaries=None,
           info: bool = True):
    """psi <- prod_s exp(-i t_s H(gamma_s)) psi in place (piecewise-constant schedule).

    boundaries: optional CUDA tensor of shape (S, 2^n), same dtype as psi, that
    receives the state at the start of every segment. Returns per-segment infos."""
    h, J = _f64(h), _f64(J)
    gammas, ts = _f64(gammas), _f64(ts)
    n = h.shape[0]
    S = gammas.shape[0]
    assert ts.shape[0] == S
    _check_state(psi, n)
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    bptr = None
    if boundaries is not None:
        if boundaries.dtype != psi.dtype or tuple(boundaries.shape) != (S, 1 << n) or not boundaries.is_contiguous():
            raise ValueError("boundaries must be a contiguous (S, 2^n) tensor of psi's dtype")
        bptr = ctypes.c_void_p(boundaries.data_ptr())
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    infos = (_lib.Info * S)() if info else None
    code = _lib.lib().cheb_anneal(n, _dp(h), _dp(J), S, _dp(gammas), _dp(ts), ctypes.c_void_p(psi.data_ptr()),
                                  PREC[prec], float(tol), METHOD[method], bptr, ctypes.c_void_p(p), nb,
                                  _stream_ptr(psi.device), infos)
    _lib.check(code, "cheb_anneal")
    return [x.as_dict() for x in infos] if info else None


def anneal_general(h, J, a_s, b_s, ts, psi, tol: Optional[float] = None, method: str = "chebyshev",
                   boundaries=None, info: bool = True):
    """psi <- prod_s exp(-i t_s (b_s H_P + a_s sum_j X_j)) psi in place (cheb_anneal_general)."""
    h, J = _f64(h), _f64(J)
    a_s, b_s, ts = _f64(a_s), _f64(b_s), _f64(ts)
    n = h.shape[0]
    S = a_s.shape[0]
    assert b_s.shape[0] == S and ts.shape[0] == S
    _check_state(psi, n)
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    bptr = None
    if boundaries is not None:
        if boundaries.dtype != psi.dtype or tuple(boundaries.shape) != (S, 1 << n) or not boundaries.is_contiguous():
            raise ValueError("boundaries must be a contiguous (S, 2^n) tensor of psi's dtype")
        bptr = ctypes.c_void_p(boundaries.data_ptr())
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    infos = (_lib.Info * S)() if info else None
    code = _lib.lib().cheb_anneal_general(n, _dp(h), _dp(J), S, _dp(a_s), _dp(b_s), _dp(ts),
                                          ctypes.c_void_p(psi.data_ptr()), PREC[prec], float(tol), METHOD[method],
                                          bptr, ctypes.c_void_p(p), nb, _stream_ptr(psi.device), infos)
    _lib.check(code, "cheb_anneal_general")
    return [x.as_dict() for x in infos] if info else None


class AnnealGraph:
    """A schedule captured into a CUDA graph (cheb_anneal_graph_create): the host side
    runs once, launch() replays the device work on psi (and boundaries), bit for bit what
    anneal / anneal_general computes from the same state. psi and boundaries are bound
    into the graph; close() (or garbage collection) releases it."""

    def __init__(self, h, J, gammas, ts, psi, boundaries=None, b_s=None, tol: Optional[float] = None,
                 method: str = "chebyshev"):
        import torch

        h, J = _f64(h), _f64(J)
        a_s, ts = _f64(gammas), _f64(ts)
        n, S = h.shape[0], a_s.shape[0]
        assert ts.shape[0] == S
        _check_state(psi, n)
        prec = precision_of(psi)
        if tol is None:
            tol = 2.0 ** -23 if prec == "fp32" else 1e-12
        bptr = None
        if boundaries is not None:
            if (boundaries.dtype != psi.dtype or tuple(boundaries.shape) != (S, 1 << n)
                    or not boundaries.is_contiguous()):
                raise ValueError("boundaries must be a contiguous (S, 2^n) tensor of psi's dtype")
            bptr = ctypes.c_void_p(boundaries.data_ptr())
        bs = None if b_s is None else _f64(b_s)
        need = int(_lib.lib().cheb_anneal_graph_workspace_bytes(n, PREC[prec], S))
        self.workspace = torch.empty(need + 256, dtype=torch.uint8, device=psi.device)
        self.psi, self.boundaries, self.n, self.prec = psi, boundaries, n, prec
        p, nb = _ws_ptr(self.workspace)
        handle = ctypes.c_void_p()
        code = _lib.lib().cheb_anneal_graph_create(n, _dp(h), _dp(J), S, _dp(a_s),
                                                   _dp(bs) if bs is not None else None, _dp(ts),
                                                   ctypes.c_void_p(psi.data_ptr()), PREC[prec], float(tol),
                                                   METHOD[method], bptr, ctypes.c_void_p(p), nb,
                                                   _stream_ptr(psi.device), ctypes.byref(handle))
        _lib.check(code, "cheb_anneal_graph_create")
        self._handle = handle

    def launch(self):
        """Replay the schedule on the current stream (psi <- the schedule applied to psi)."""
        if self._handle is None:
            raise ValueError("graph released")
        _lib.check(_lib.lib().cheb_anneal_graph_launch(self._handle, _stream_ptr(self.psi.device)),
                   "cheb_anneal_graph_launch")

    def status(self):
        """Raise if a bounded wait ran out during a replay (synchronises)."""
        p, nb = _ws_ptr(self.workspace)
        _lib.check(_lib.lib().cheb_workspace_status(ctypes.c_void_p(p), nb, _stream_ptr(self.psi.device)),
                   "cheb_workspace_status")

    def close(self):
        if getattr(self, "_handle", None) is not None:
            _lib.lib().cheb_anneal_graph_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def magnus4_nodes(A, B, T: float, steps: int):
    """Sample the schedule for cheb_magnus4 (cheb_magnus4_nodes): equal steps of [0, T]
    and, per step, (A(t1), B(t1), A(t2), B(t2)) at the Gauss-Legendre points."""
    dt = np.empty(steps)
    nodes = np.empty(4 * steps)
    cb = _lib.schedule_callback(A, B)
    code = _lib.lib().cheb_magnus4_nodes(float(T), int(steps), ctypes.cast(cb, ctypes.c_void_p), None, _dp(dt),
                                         _dp(nodes))
    _lib.check(code, "cheb_magnus4_nodes")
    return dt, nodes.reshape(steps, 4)


def magnus4(h, J, dt, nodes, psi, tol: Optional[float] = None, method: str = "chebyshev", info: bool = False,
            boundaries=None):
    """psi <- the fourth-order commutator-free Magnus propagator of H(t) = A(t) sum_j X_j +
    B(t) H_P, in place (cheb_magnus4); dt, nodes as from magnus4_nodes. boundaries: optional
    CUDA tensor (2*steps, 2^n) that receives the state before each exponential."""
    h, J = _f64(h), _f64(J)
    dt = _f64(dt)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1))
    n = h.shape[0]
    steps = dt.shape[0]
    assert nodes.shape[0] == 4 * steps
    _check_state(psi, n)
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    bptr = None
    if boundaries is not None:
        if (boundaries.dtype != psi.dtype or tuple(boundaries.shape) != (2 * steps, 1 << n)
                or not boundaries.is_contiguous()):
            raise ValueError("boundaries must be a contiguous (2*steps, 2^n) tensor of psi's dtype")
        bptr = ctypes.c_void_p(boundaries.data_ptr())
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    infos = (_lib.Info * (2 * steps))() if info else None
    code = _lib.lib().cheb_magnus4(n, _dp(h), _dp(J), steps, _dp(dt), _dp(nodes), ctypes.c_void_p(psi.data_ptr()),
                                   PREC[prec], float(tol), METHOD[method], bptr, ctypes.c_void_p(p), nb,
                                   _stream_ptr(psi.device), infos)
    _lib.check(code, "cheb_magnus4")
    return [x.as_dict() for x in infos] if info else None


def magnus4_adjoint(h, J, dt, nodes, boundaries, psi_T, grad, tol: Optional[float] = None,
                    method: str = "chebyshev", store_vectors: Optional[int] = None):
    """Gradients through cheb_magnus4 (cheb_magnus4_adjoint): grad holds dL/dpsi_T on entry
    and dL/dpsi_0 on return. Returns dict: dt (steps), nodes (steps x 4), h (n), J (n x n)."""
    h, J = _f64(h), _f64(J)
    dt = _f64(dt)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1))
    n, steps = h.shape[0], dt.shape[0]
    prec = precision_of(psi_T)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    for x in (boundaries, psi_T, grad):
        if not x.is_cuda or not x.is_contiguous() or x.dtype != psi_T.dtype:
            raise ValueError("boundaries, psi_T and grad must be contiguous CUDA tensors of one complex dtype")
    if store_vectors is None:
        nd = nodes.reshape(steps, 4)
        amax = float(np.abs(nd[:, [0, 2]]).max())
        bmax = float(np.abs(nd[:, [1, 3]]).max())
        store_vectors = _auto_store_vectors(n, prec, psi_T.device,
                                            _degree_upper_bound(bmax * h, bmax * J, np.array([amax]),
                                                                np.array([float(np.abs(dt).max())]), tol, method))
    ws = _adjoint_workspace(n, prec, psi_T.device, store_vectors)
    p, nb = _ws_ptr(ws)
    gdt, gnd, gh, gJ = np.zeros(steps), np.zeros(4 * steps), np.zeros(n), np.zeros((n, n))
    code = _lib.lib().cheb_magnus4_adjoint(n, _dp(h), _dp(J), steps, _dp(dt), _dp(nodes),
                                           ctypes.c_void_p(boundaries.data_ptr()), ctypes.c_void_p(psi_T.data_ptr()),
                                           ctypes.c_void_p(grad.data_ptr()), PREC[prec], float(tol), METHOD[method],
                                           _dp(gdt), _dp(gnd), _dp(gh), _dp(gJ), ctypes.c_void_p(p), nb,
                                           _stream_ptr(psi_T.device))
    _lib.check(code, "cheb_magnus4_adjoint")
    return {"dt": gdt, "nodes": gnd.reshape(steps, 4), "h": gh, "J": gJ}


def magnus4_adaptive(h, J, A, B, T: float, psi, tol: float, steps0: int = 8, method: str = "chebyshev"):
    """psi <- psi(T) with the number of equal Magnus steps chosen a posteriori
    (cheb_magnus4_adaptive: step doubling, fourth-order error estimate). Returns the
    number of steps used."""
    import torch

    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    _check_state(psi, n)
    prec = precision_of(psi)
    need = int(_lib.lib().cheb_magnus4_adaptive_workspace_bytes(n, PREC[prec]))
    ws = torch.empty(need + 256, dtype=torch.uint8, device=psi.device)
    p, nb = _ws_ptr(ws)
    cb = _lib.schedule_callback(A, B)
    used = ctypes.c_int(0)
    est = ctypes.c_double(0.0)
    code = _lib.lib().cheb_magnus4_adaptive(n, _dp(h), _dp(J), float(T), ctypes.cast(cb, ctypes.c_void_p), None,
                                            int(steps0), float(tol), ctypes.c_void_p(psi.data_ptr()), PREC[prec],
                                            METHOD[method], ctypes.c_void_p(p), nb, _stream_ptr(psi.device),
                                            ctypes.byref(used), ctypes.byref(est))
    _lib.check(code, "cheb_magnus4_adaptive")
    return used.value


def set_batch_persistent(mode):
    """FP32 batches as one persistent launch (True or 1: one CTA per SM, the default;
    2: two CTAs per SM) or per-size launches (False or 0)."""
    m = int(mode) if not isinstance(mode, bool) else (1 if mode else 0)
    _lib.check(_lib.lib().cheb_set_batch_persistent(m), "cheb_set_batch_persistent")


def get_batch_persistent() -> int:
    return int(_lib.lib().cheb_get_batch_persistent())


def batch_offsets(ns):
    """Contiguous layout of a batch: element offset of each state (padded to even)."""
    off, cur = [], 0
    for n in ns:
        off.append(cur)
        cur += max(1 << int(n), 2)
    return np.array(off, dtype=np.int64), cur


def expmv_batched(ns, hs, Js, gammas, ts, psi_cat, offsets=None, tol: Optional[float] = None,
                  method: str = "chebyshev", info: bool = True):
    """psi_i <- exp(-i t_i H_i) psi_i for independent instances packed in psi_cat."""
    import torch

    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    B = ns.shape[0]
    h_cat = np.ascontiguousarray(np.concatenate([_f64(h) for h in hs]))
    J_cat = np.ascontiguousarray(np.concatenate([_f64(J).ravel() for J in Js]))
    gammas, ts = _f64(gammas), _f64(ts)
    if offsets is None:
        offsets, _ = batch_offsets(ns)
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if not isinstance(psi_cat, torch.Tensor) or not psi_cat.is_cuda or not psi_cat.is_contiguous():
        raise TypeError("psi_cat must be a contiguous CUDA tensor")
    prec = precision_of(psi_cat)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    ip = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    need = int(_lib.lib().cheb_batched_workspace_bytes(B, ip, PREC[prec]))
    if need == 0:
        raise ValueError("invalid batch sizes")
    ws = torch.empty(need + 256, dtype=torch.uint8, device=psi_cat.device)
    p, nb = _ws_ptr(ws)
    infos = (_lib.Info * B)() if info else None
    code = _lib.lib().cheb_expmv_batched(B, ip, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(h_cat),
                                         _dp(J_cat), _dp(gammas), _dp(ts), ctypes.c_void_p(psi_cat.data_ptr()),
                                         PREC[prec], float(tol), METHOD[method], ctypes.c_void_p(p), nb,
                                         _stream_ptr(psi_cat.device), infos)
    _lib.check(code, "cheb_expmv_batched")
    return [x.as_dict() for x in infos] if info else None


def adjoint_workspace_bytes(n: int, precision: str, store_vectors: int) -> int:
    """Bytes of the adjoint workspace with a pool of store_vectors state vectors."""
    return int(_lib.lib().cheb_adjoint_workspace_bytes(n, PREC[precision], max(0, store_vectors)))


def _adjoint_workspace(n: int, prec: str, device, store_vectors: int):
    import torch

    need = int(_lib.lib().cheb_adjoint_workspace_bytes(n, PREC[prec], max(0, store_vectors)))
    if need == 0:
        raise ValueError(f"unsupported n={n}")
    return torch.empty(need + 256, dtype=torch.uint8, device=device)


def adjoint_workspace(n: int, precision: str, store_vectors: int, device=None):
    """A device buffer for the adjoint entry points with a pool of store_vectors state
    vectors (pass it as workspace= to reuse one allocation across calls)."""
    import torch

    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    return _adjoint_workspace(n, precision, device, store_vectors)


def _check_adjoint_ws(ws, n, prec, store_vectors):
    need = int(_lib.lib().cheb_adjoint_workspace_bytes(n, PREC[prec], max(0, store_vectors)))
    if not ws.is_cuda or ws.dtype.itemsize != 1 or _ws_ptr(ws)[1] < need:
        raise ValueError("workspace must be a CUDA byte buffer of adjoint_workspace(n, precision, store_vectors)")


def _degree_upper_bound(h, J, gammas, ts, tol: float, method: str) -> int:
    """Largest Chebyshev degree over the segments, from the 1-norm bound of the spectral
    radius (the library's r never exceeds it, and K grows with r)."""
    n = h.shape[0]
    half = float(np.sum(np.abs(h)) + np.sum(np.abs(np.triu(J, 1))))
    tol_s = tol / gammas.shape[0]
    kmax = 0
    for g, t in zip(gammas, ts):
        c, _ = coefficients(abs(float(t)) * (half + abs(float(g)) * n), tol_s, method)
        kmax = max(kmax, c.shape[0] - 1)
    return kmax


def _auto_store_vectors(n: int, prec: str, device, kmax: int) -> int:
    """Keep every b_k of a segment when that fits in half of the free device memory,
    else a ring plus about sqrt(K) anchor pairs."""
    import torch

    vb = (1 << n) * (8 if prec == "fp32" else 16)
    free, _ = torch.cuda.mem_get_info(device)
    if (kmax + 1) * vb <= free // 2:
        return kmax + 1
    return 6 + 2 * max(1, int(np.ceil(np.sqrt(max(kmax, 1)))))


class Checkpoint:
    """The adjoint workspace that a checkpointed forward run filled (cheb_anneal_checkpointed);
    pass it to anneal_adjoint / anneal_general_adjoint as checkpoint=."""

    def __init__(self, workspace, store_vectors: int):
        self.workspace = workspace
        self.store_vectors = store_vectors


def _checkpointed(fn, n, S, args, psi, boundaries, prec, tol, method, store_vectors, kmax, workspace):
    _check_state(psi, n)
    if boundaries.dtype != psi.dtype or tuple(boundaries.shape) != (S, 1 << n) or not boundaries.is_contiguous():
        raise ValueError("boundaries must be a contiguous (S, 2^n) tensor of psi's dtype")
    if store_vectors is None:
        store_vectors = _auto_store_vectors(n, prec, psi.device, kmax())
    if workspace is not None:
        _check_adjoint_ws(workspace, n, prec, store_vectors)
    ws = workspace if workspace is not None else _adjoint_workspace(n, prec, psi.device, store_vectors)
    p, nb = _ws_ptr(ws)
    code = fn(n, *args, ctypes.c_void_p(psi.data_ptr()), PREC[prec], float(tol), METHOD[method],
              ctypes.c_void_p(boundaries.data_ptr()), ctypes.c_void_p(p), nb, _stream_ptr(psi.device))
    _lib.check(code, fn.__name__)
    return Checkpoint(ws, store_vectors)


def anneal_checkpointed(h, J, gammas, ts, psi, boundaries, tol: Optional[float] = None, method: str = "chebyshev",
                        store_vectors: Optional[int] = None, workspace=None) -> Checkpoint:
    """psi <- prod_s exp(-i t_s H(gamma_s)) psi in place, writing the segment starts to
    boundaries and leaving the last segment's Clenshaw vectors in an adjoint workspace
    (cheb_anneal_checkpointed; workspace: an adjoint_workspace buffer to use, else a new
    one); returns that Checkpoint for anneal_adjoint."""
    h, J = _f64(h), _f64(J)
    gammas, ts = _f64(gammas), _f64(ts)
    n, S = h.shape[0], gammas.shape[0]
    assert ts.shape[0] == S
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    return _checkpointed(_lib.lib().cheb_anneal_checkpointed, n, S, (_dp(h), _dp(J), S, _dp(gammas), _dp(ts)), psi,
                         boundaries, prec, tol, method, store_vectors,
                         lambda: _degree_upper_bound(h, J, gammas, ts, tol, method), workspace)


def anneal_general_checkpointed(h, J, a_s, b_s, ts, psi, boundaries, tol: Optional[float] = None,
                                method: str = "chebyshev", store_vectors: Optional[int] = None,
                                workspace=None) -> Checkpoint:
    """The checkpointed form of anneal_general (cheb_anneal_general_checkpointed)."""
    h, J = _f64(h), _f64(J)
    a_s, b_s, ts = _f64(a_s), _f64(b_s), _f64(ts)
    n, S = h.shape[0], a_s.shape[0]
    assert b_s.shape[0] == S and ts.shape[0] == S
    prec = precision_of(psi)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    return _checkpointed(_lib.lib().cheb_anneal_general_checkpointed, n, S,
                         (_dp(h), _dp(J), S, _dp(a_s), _dp(b_s), _dp(ts)), psi, boundaries, prec, tol, method,
                         store_vectors,
                         lambda: _degree_upper_bound(np.abs(b_s).max() * h, np.abs(b_s).max() * J, a_s, ts, tol,
                                                     method), workspace)


def _adjoint_ws_for(n, prec, device, store_vectors, checkpoint, kmax, workspace):
    if checkpoint is not None:
        return checkpoint.workspace
    if workspace is not None:
        _check_adjoint_ws(workspace, n, prec, 0 if store_vectors is None else store_vectors)
        return workspace
    if store_vectors is None:
        store_vectors = _auto_store_vectors(n, prec, device, kmax())
    return _adjoint_workspace(n, prec, device, store_vectors)


def anneal_adjoint(h, J, gammas, ts, boundaries, psi_T, grad, tol: Optional[float] = None,
                   method: str = "chebyshev", store_vectors: Optional[int] = None,
                   checkpoint: Optional[Checkpoint] = None, workspace=None):
    """Gradients of a loss on the final state of a schedule (see cheb_anneal_adjoint).

    grad (CUDA tensor like psi_T) holds dL/dpsi_T on entry and dL/dpsi_0 on return.
    store_vectors: state vectors of workspace for the Clenshaw vectors b_k (>= K keeps
    all of them; fewer regenerates them from anchors; None chooses by free memory).
    checkpoint: the result of anneal_checkpointed for this schedule, psi_T and
    boundaries (its workspace is used, and the last segment is not recomputed).
    workspace: an adjoint_workspace buffer to use instead of a new one (its pool size
    decides how the b_k are kept).
    Returns dict of numpy arrays: gamma (S), t (S), h (n), J (n x n, upper triangle)."""
    h, J = _f64(h), _f64(J)
    gammas, ts = _f64(gammas), _f64(ts)
    n, S = h.shape[0], gammas.shape[0]
    prec = precision_of(psi_T)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    for x in (boundaries, psi_T, grad):
        if not x.is_cuda or not x.is_contiguous() or x.dtype != psi_T.dtype:
            raise ValueError("boundaries, psi_T and grad must be contiguous CUDA tensors of one complex dtype")
    ws = _adjoint_ws_for(n, prec, psi_T.device, store_vectors, checkpoint,
                         lambda: _degree_upper_bound(h, J, gammas, ts, tol, method), workspace)
    p, nb = _ws_ptr(ws)
    gg, gt, gh, gJ = np.zeros(S), np.zeros(S), np.zeros(n), np.zeros((n, n))
    code = _lib.lib().cheb_anneal_adjoint(n, _dp(h), _dp(J), S, _dp(gammas), _dp(ts),
                                          ctypes.c_void_p(boundaries.data_ptr()), ctypes.c_void_p(psi_T.data_ptr()),
                                          ctypes.c_void_p(grad.data_ptr()), PREC[prec], float(tol), METHOD[method],
                                          _dp(gg), _dp(gt), _dp(gh), _dp(gJ), ctypes.c_void_p(p), nb,
                                          _stream_ptr(psi_T.device))
    _lib.check(code, "cheb_anneal_adjoint")
    return {"gamma": gg, "t": gt, "h": gh, "J": gJ}


def anneal_general_adjoint(h, J, a_s, b_s, ts, boundaries, psi_T, grad, tol: Optional[float] = None,
                           method: str = "chebyshev", store_vectors: Optional[int] = None,
                           checkpoint: Optional[Checkpoint] = None, workspace=None):
    """Gradients through cheb_anneal_general (see cheb_anneal_general_adjoint); grad holds
    dL/dpsi_T on entry and dL/dpsi_0 on return; checkpoint as in anneal_adjoint.
    Returns dict: a, b, t (S), h (n), J (n x n)."""
    h, J = _f64(h), _f64(J)
    a_s, b_s, ts = _f64(a_s), _f64(b_s), _f64(ts)
    n, S = h.shape[0], a_s.shape[0]
    prec = precision_of(psi_T)
    if tol is None:
        tol = 2.0 ** -23 if prec == "fp32" else 1e-12
    for x in (boundaries, psi_T, grad):
        if not x.is_cuda or not x.is_contiguous() or x.dtype != psi_T.dtype:
            raise ValueError("boundaries, psi_T and grad must be contiguous CUDA tensors of one complex dtype")
    ws = _adjoint_ws_for(n, prec, psi_T.device, store_vectors, checkpoint,
                         lambda: _degree_upper_bound(np.abs(b_s).max() * h, np.abs(b_s).max() * J, a_s, ts, tol,
                                                     method), workspace)
    p, nb = _ws_ptr(ws)
    ga, gb, gt, gh, gJ = np.zeros(S), np.zeros(S), np.zeros(S), np.zeros(n), np.zeros((n, n))
    code = _lib.lib().cheb_anneal_general_adjoint(
        n, _dp(h), _dp(J), S, _dp(a_s), _dp(b_s), _dp(ts), ctypes.c_void_p(boundaries.data_ptr()),
        ctypes.c_void_p(psi_T.data_ptr()), ctypes.c_void_p(grad.data_ptr()), PREC[prec], float(tol), METHOD[method],
        _dp(ga), _dp(gb), _dp(gt), _dp(gh), _dp(gJ), ctypes.c_void_p(p), nb, _stream_ptr(psi_T.device))
    _lib.check(code, "cheb_anneal_general_adjoint")
    return {"a": ga, "b": gb, "t": gt, "h": gh, "J": gJ}


def energy_grad(h, J, psi):
    """(energy, dL/dpsi = 2 H_P psi as a new tensor, dL/dh, dL/dJ) for L = <psi|H_P|psi>."""
    import torch

    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    _check_state(psi, n)
    prec = precision_of(psi)
    ws = _adjoint_workspace(n, prec, psi.device, 0)
    p, nb = _ws_ptr(ws)
    g = torch.empty_like(psi)
    e = ctypes.c_double()
    gh, gJ = np.zeros(n), np.zeros((n, n))
    code = _lib.lib().cheb_energy_grad(n, _dp(h), _dp(J), ctypes.c_void_p(psi.data_ptr()),
                                       ctypes.c_void_p(g.data_ptr()), PREC[prec], ctypes.byref(e), _dp(gh), _dp(gJ),
                                       ctypes.c_void_p(p), nb, _stream_ptr(psi.device))
    _lib.check(code, "cheb_energy_grad")
    return e.value, g, gh, gJ


def monomial_to_chebyshev(a):
    """Chebyshev coefficients c of p(x) = sum_m a_m x^m (cheb_monomial_to_chebyshev)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    out = np.empty_like(a)
    K = a.shape[0] - 1
    _lib.check(_lib.lib().cheb_monomial_to_chebyshev(K, _dp(a.view(np.float64)), _dp(out.view(np.float64))),
               "cheb_monomial_to_chebyshev")
    return out


def poly_apply_monomial(h, J, gamma: float, center: float, radius: float, a, psi, path: str = "auto"):
    """psi <- sum_m a_m ((H - center)/radius)^m psi in place: the monomial coefficients are
    converted to the Chebyshev basis on the host and evaluated by the Clenshaw recurrence."""
    poly_apply(h, J, gamma, center, radius, monomial_to_chebyshev(a), psi, path=path)


def poly_apply(h, J, gamma: float, center: float, radius: float, coeffs, psi, path: str = "auto"):
    """psi <- sum_m c_m T_m((H - center)/radius) psi in place on the GPU."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    _check_state(psi, n)
    prec = precision_of(psi)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.complex128)).view(np.float64)
    K = c.shape[0] // 2 - 1
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    code = _lib.lib().cheb_poly_apply(n, _dp(h), _dp(J), float(gamma), float(center), float(radius), K, _dp(c),
                                      ctypes.c_void_p(psi.data_ptr()), PREC[prec], PATH[path], ctypes.c_void_p(p),
                                      nb, _stream_ptr(psi.device))
    _lib.check(code, "cheb_poly_apply")


def set_fused_split(n: int, l: int, h: int = 0):
    """Choose how the fused FP32 step splits the n bits (11 + l + h = n); l = -1 resets."""
    _lib.check(_lib.lib().cheb_set_fused_split(int(n), int(l), int(h)), "cheb_set_fused_split")


def get_fused_split(n: int):
    l, h = ctypes.c_int(), ctypes.c_int()
    _lib.check(_lib.lib().cheb_get_fused_split(int(n), ctypes.byref(l), ctypes.byref(h)), "cheb_get_fused_split")
    return l.value, h.value


def set_fused_split_fp64(n: int, l: int, h: int = 0):
    """Split of the float-float fused FP64 step (10 + l + h = n); l = -1 resets."""
    _lib.check(_lib.lib().cheb_set_fused_split_fp64(int(n), int(l), int(h)), "cheb_set_fused_split_fp64")


def get_fused_split_fp64(n: int):
    l, h = ctypes.c_int(), ctypes.c_int()
    _lib.check(_lib.lib().cheb_get_fused_split_fp64(int(n), ctypes.byref(l), ctypes.byref(h)),
               "cheb_get_fused_split_fp64")
    return l.value, h.value


def set_programmatic_launch(on: bool):
    """Programmatic dependent launch of the fused step kernels (on by default)."""
    _lib.check(_lib.lib().cheb_set_programmatic_launch(1 if on else 0), "cheb_set_programmatic_launch")


def autotune(n: int, precision: str = "fp32", steps: int = 4, device=None):
    """Time the candidate step configurations for (n, precision) on the device and install
    the fastest (cheb_autotune); returns the result as a dict."""
    import torch

    need = int(_lib.lib().cheb_autotune_workspace_bytes(int(n), PREC[precision]))
    if need == 0:
        raise ValueError(f"unsupported n={n}")
    dev = torch.device(device if device is not None else "cuda")
    ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    p, nb = _ws_ptr(ws)
    res = _lib.TuneResult()
    code = _lib.lib().cheb_autotune(int(n), PREC[precision], int(steps), ctypes.c_void_p(p), nb, _stream_ptr(dev),
                                    ctypes.byref(res))
    _lib.check(code, "cheb_autotune")
    d = res.as_dict()
    d["path"] = {1: "plain", 2: "fused"}.get(d["path"], d["path"])
    return d


def autotune_load(path: str, device: Optional[str] = None) -> int:
    """Apply the lines of an autotuner cache file recorded for `device` (default: current)."""
    applied = ctypes.c_int(0)
    code = _lib.lib().cheb_autotune_load(path.encode(), device.encode() if device else None, ctypes.byref(applied))
    _lib.check(code, "cheb_autotune_load")
    return applied.value


def autotune_reset():
    _lib.check(_lib.lib().cheb_autotune_reset(), "cheb_autotune_reset")


def set_fused_blocking(mode):
    """L2-blocked launches of the fused step (cheb_set_fused_blocking): 0 / False
    separate launches, 1 / True the last strided pass and the low pass as one launch,
    2 the two strided passes as one launch, -1 / None automatic (the default: 2 from
    n = 26 on in FP32, from n = 28 on in FP64); results are identical."""
    _lib.check(_lib.lib().cheb_set_fused_blocking(-1 if mode is None else int(mode)), "cheb_set_fused_blocking")


def get_fused_blocking() -> int:
    return int(_lib.lib().cheb_get_fused_blocking())


def set_fused_compensated(on: bool):
    """Kahan-compensated flip sums in the fused FP32 passes (True) or plain FP32 adds."""
    _lib.check(_lib.lib().cheb_set_fused_compensated(1 if on else 0), "cheb_set_fused_compensated")


def get_fused_compensated() -> bool:
    return bool(_lib.lib().cheb_get_fused_compensated())


KERNEL_KIND = {"plain": 3, "adjoint_acc": 5, "low": 6, "high": 7, "tail": 8, "pair": 9}


def wait_selftest(device=None):
    """Run the library's two bounded device waits (an mbarrier wait, a team barrier) against
    waits nothing satisfies; raises ChebError with CHEB_ERR_TIMEOUT (the expected outcome)
    or returns if they did not both time out."""
    import torch

    buf = torch.zeros(64, dtype=torch.uint8, device=device if device is not None else "cuda")
    dev = buf.device
    _lib.check(_lib.lib().cheb_wait_selftest(ctypes.c_void_p(buf.data_ptr()), buf.numel(), _stream_ptr(dev)),
               "cheb_wait_selftest")


def launch_count() -> int:
    """Kernels launched by the CUDA library so far in this process."""
    return int(_lib.lib().cheb_launch_count())


def profile_enable(on: bool = True):
    _lib.check(_lib.lib().cheb_profile_enable(1 if on else 0), "cheb_profile_enable")


def profile_reset():
    _lib.check(_lib.lib().cheb_profile_reset(), "cheb_profile_reset")


def profile_read(kind: str):
    """(launches timed, total device ms) for 'plain', 'low', 'high', 'tail' or 'pair' step
    kernels or 'adjoint_acc' (the adjoint's per-step accumulation)."""
    c, ms = ctypes.c_longlong(), ctypes.c_double()
    _lib.check(_lib.lib().cheb_profile_read(KERNEL_KIND[kind], ctypes.byref(c), ctypes.byref(ms)),
               "cheb_profile_read")
    return int(c.value), float(ms.value)


def energy(h, J, psi):
    """(<psi|H_P|psi>, ||psi||^2) in FP64 on the GPU."""
    h, J = _f64(h), _f64(J)
    n = h.shape[0]
    _check_state(psi, n)
    prec = precision_of(psi)
    ws = workspace(n, prec, psi.device)
    p, nb = _ws_ptr(ws)
    e, nn = ctypes.c_double(), ctypes.c_double()
    code = _lib.lib().cheb_energy(n, _dp(h), _dp(J), ctypes.c_void_p(psi.data_ptr()), PREC[prec],
                                  ctypes.c_void_p(p), nb, _stream_ptr(psi.device), ctypes.byref(e), ctypes.byref(nn))
    _lib.check(code, "cheb_energy")
    return e.value, nn.value
