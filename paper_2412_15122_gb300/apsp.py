"""Python binding of the C ABI in include/apsp.h (ctypes, marshalling only).

Every function here has the name of the C entry point it calls and does no
compute of its own: it converts numpy arrays / torch tensors to pointers,
checks the returned status and raises ``ApspError`` on failure.  The CUDA
library must have been built (``paper_2412_15122_gb300.build.build()``);
loading fails loudly otherwise.

``Graph`` is a small object wrapper over the same calls.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapsp_gb300.so")

APSP_I32, APSP_F32 = 0, 1
APSP_DIRECTED, APSP_UNDIRECTED, APSP_D_GIVEN, APSP_DEVICE_INPUT, APSP_MINIMAX = 0, 1, 4, 8, 16
APSP_INF_I32 = 0x3FFFFFFF
APSP_MAX_CAPACITY = 18432

STATUS = {0: "APSP_OK", 1: "APSP_E_ARG", 2: "APSP_E_NODE", 3: "APSP_E_NEGATIVE", 4: "APSP_E_CAPACITY",
          5: "APSP_E_NOMEM", 6: "APSP_E_CUDA", 7: "APSP_E_TIMEOUT", 8: "APSP_E_BUSY", 9: "APSP_E_UNSUPPORTED"}
OPS = {0: "none", 1: "init", 2: "add", 3: "remove", 4: "decrease", 5: "increase", 6: "same", 7: "recompute"}
PATHS = {0: "none", 1: "sweep", 2: "trivial", 3: "warm", 4: "cold"}
DISPATCH = {"delta": 0, "warm": 1, "cold": 2, "model": 3}


class ApspError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_status_string(status)})")


class apsp_stats(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("path", ctypes.c_int32), ("node", ctypes.c_int32),
                ("node2", ctypes.c_int32), ("n_live", ctypes.c_int32), ("affected_rows", ctypes.c_int32),
                ("affected_pairs", ctypes.c_int64), ("sweep_rows", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("overflow", ctypes.c_int32), ("cold_reason", ctypes.c_int32), ("cost", ctypes.c_float),
                ("model_warm", ctypes.c_float), ("model_cold", ctypes.c_float),
                ("pairs_rechecked", ctypes.c_int64), ("warm_pass1_us", ctypes.c_float), ("warm_total_us", ctypes.c_float),
                ("grown_pairs", ctypes.c_int64), ("grown_rows", ctypes.c_int32), ("grown_cost", ctypes.c_float),
                ("reduce_rows", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["op"] = OPS.get(self.op, self.op)
        d["path"] = PATHS.get(self.path, self.path)
        return d


class apsp_batch_item(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("op", ctypes.c_int32), ("u", ctypes.c_int32), ("v", ctypes.c_int32),
                ("in_w", ctypes.c_void_p), ("out_w", ctypes.c_void_p), ("w", ctypes.c_double)]


BATCH_OPS = {"add": 0, "remove": 1, "edge": 2, "query": 3}


class apsp_request(ctypes.Structure):
    _fields_ = [("item", apsp_batch_item), ("arrival_s", ctypes.c_double)]


class apsp_request_result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("dist", ctypes.c_double),
                ("status", ctypes.c_int32), ("wave", ctypes.c_int32), ("new_id", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class apsp_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("small_max_slots", ctypes.c_int32),
                ("max_wave_requests", ctypes.c_int32)]


class apsp_batch_info(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("graph_captures", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("last_width", ctypes.c_int32), ("fixed_width", ctypes.c_int32)]


class apsp_info(ctypes.Structure):
    _fields_ = [("n_live", ctypes.c_int32), ("n_slots", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("ld", ctypes.c_int32), ("dtype", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("device_bytes", ctypes.c_int64)]


class apsp_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"the CUDA library {LIB_PATH} is not built; run paper_2412_15122_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "apsp_init": [ctypes.POINTER(P), P, I32, I32, I32, U32, P, P],
        "apsp_destroy": [P],
        "apsp_set_allocator": [ALLOC_FN, FREE_FN, P],
        "apsp_add_node": [P, P, P, ctypes.POINTER(I32)],
        "apsp_add_node_device": [P, P, P, ctypes.POINTER(I32)],
        "apsp_remove_node": [P, I32],
        "apsp_update_edge": [P, I32, I32, P],
        "apsp_recompute": [P],
        "apsp_query": [P, I32, I32, P],
        "apsp_query_batch": [P, P, I32, P],
        "apsp_query_paths": [P, P, I32, P, I32, P],
        "apsp_query_path": [P, I32, I32, P, I32, ctypes.POINTER(I32)],
        "apsp_query_all_paths": [P, I32, I32, P, I64, P, I32, ctypes.POINTER(I32), ctypes.POINTER(I64)],
        "apsp_probe_addmin_rate": [I32, ctypes.POINTER(ctypes.c_double)],
        "apsp_probe_l2_read_gbs": [ctypes.POINTER(ctypes.c_double)],
        "apsp_selftest_barrier_timeout": [I32, ctypes.POINTER(I32)],
        "apsp_copy_D": [P, P, I64, I32],
        "apsp_copy_W": [P, P, I64, I32],
        "apsp_copy_alive": [P, P],
        "apsp_info_get": [P, ctypes.POINTER(apsp_info)],
        "apsp_last_stats": [P, ctypes.POINTER(apsp_stats)],
        "apsp_copy_last_list": [P, P, I64, ctypes.POINTER(I64)],
        "apsp_next_hops": [P, P, I32, P, I64],
        "apsp_sync": [P],
        "apsp_set_dispatch": [P, I32, ctypes.c_double],
        "apsp_set_exact_list": [P, I32],
        "apsp_set_list_mode": [P, I32],
        "apsp_profile_enable": [P, I32],
        "apsp_profile_read": [P, ctypes.POINTER(apsp_profile_entry), I32, ctypes.POINTER(I32)],
        "apsp_profile_reset": [P],
        "apsp_add_node_noalloc": [P, I64, I32, P, I32, P, P, I32, P],
        "apsp_batch_create": [ctypes.POINTER(P), P],
        "apsp_batch_run": [P, ctypes.POINTER(P), I32, ctypes.POINTER(apsp_batch_item), I32, ctypes.POINTER(I32)],
        "apsp_batch_destroy": [P],
        "apsp_batch_set_width": [P, I32],
        "apsp_batch_info_get": [P, ctypes.POINTER(apsp_batch_info)],
        "apsp_batch_tuned_width": [I32, I32, ctypes.POINTER(I32)],
        "apsp_serve": [ctypes.POINTER(P), I32, ctypes.POINTER(apsp_request), I32, ctypes.POINTER(apsp_serve_config),
                       ctypes.POINTER(apsp_request_result)],
        "apsp_server_create": [ctypes.POINTER(P), ctypes.POINTER(P), I32, ctypes.POINTER(apsp_serve_config)],
        "apsp_server_submit": [P, ctypes.POINTER(apsp_batch_item), ctypes.POINTER(I64)],
        "apsp_server_poll": [P, I64, ctypes.POINTER(apsp_request_result), ctypes.POINTER(I32)],
        "apsp_server_wait": [P, I64, ctypes.c_double, ctypes.POINTER(apsp_request_result)],
        "apsp_server_destroy": [P],
        "apsp_set_model": [P, P],
        "apsp_model_loss_grad": [P, P, P, I32, P, P],
        "apsp_model_predict": [P, P, I32, P],
        "apsp_model_train": [P, P, I32, I32, I32, ctypes.c_float, ctypes.c_uint64, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.apsp_server_clock.argtypes = [P]
    lib.apsp_server_clock.restype = ctypes.c_double
    lib.apsp_launch_count.argtypes = [P]
    lib.apsp_launch_count.restype = I64
    lib.apsp_status_string.argtypes = [ctypes.c_int]
    lib.apsp_status_string.restype = ctypes.c_char_p
    lib.apsp_version.restype = ctypes.c_char_p
    lib.apsp_last_cuda_error.argtypes = [ctypes.POINTER(ctypes.c_char_p)]
    lib.apsp_last_cuda_error.restype = ctypes.c_int32
    _lib = lib
    return lib


def lib():
    return _load()


def _status_string(s: int) -> str:
    try:
        return _load().apsp_status_string(s).decode()
    except Exception:
        return "?"


def apsp_last_cuda_error():
    name = ctypes.c_char_p()
    code = int(_load().apsp_last_cuda_error(ctypes.byref(name)))
    return code, (name.value.decode() if name.value else "")


def _check(s: int, where: str):
    if s != 0:
        if STATUS.get(s) in ("APSP_E_CUDA", "APSP_E_NOMEM"):
            code, name = apsp_last_cuda_error()
            raise ApspError(s, f"{where} [{name} {code}]")
        raise ApspError(s, where)


def _np_dtype(dtype: int):
    return np.float32 if dtype == APSP_F32 else np.int32


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# one function per C entry point
# ---------------------------------------------------------------------------

def apsp_status_string(s: int) -> str:
    return _status_string(s)


def apsp_version() -> str:
    return _load().apsp_version().decode()


def apsp_init(W, n: int, capacity: int, dtype: int, flags: int = 0, D=None, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_load().apsp_init(ctypes.byref(h), _ptr(W), n, capacity, dtype, flags, _ptr(D), _stream_ptr(stream)),
           "apsp_init")
    return h.value


def apsp_destroy(g: int):
    _check(_load().apsp_destroy(g), "apsp_destroy")


def apsp_add_node(g: int, in_w, out_w) -> int:
    nid = ctypes.c_int32()
    _check(_load().apsp_add_node(g, _ptr(in_w), _ptr(out_w), ctypes.byref(nid)), "apsp_add_node")
    return nid.value


def apsp_add_node_device(g: int, in_w, out_w) -> int:
    nid = ctypes.c_int32()
    _check(_load().apsp_add_node_device(g, _ptr(in_w), _ptr(out_w), ctypes.byref(nid)), "apsp_add_node_device")
    return nid.value


def apsp_remove_node(g: int, v: int):
    _check(_load().apsp_remove_node(g, v), "apsp_remove_node")


def apsp_update_edge(g: int, u: int, v: int, w, dtype: int):
    buf = np.array([w], dtype=_np_dtype(dtype))
    _check(_load().apsp_update_edge(g, u, v, buf.ctypes.data), "apsp_update_edge")


def apsp_recompute(g: int):
    _check(_load().apsp_recompute(g), "apsp_recompute")


def apsp_query(g: int, u: int, v: int, dtype: int):
    buf = np.zeros(1, dtype=_np_dtype(dtype))
    _check(_load().apsp_query(g, u, v, buf.ctypes.data), "apsp_query")
    return buf[0]


def apsp_query_batch(g: int, uv: np.ndarray, dtype: int) -> np.ndarray:
    uv = np.ascontiguousarray(uv, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(uv), dtype=_np_dtype(dtype))
    _check(_load().apsp_query_batch(g, uv.ctypes.data, len(uv), out.ctypes.data), "apsp_query_batch")
    return out


def apsp_query_paths(g: int, uv: np.ndarray, stride: int):
    """Algorithm 7 for each pair: (paths count x stride, lens count)."""
    uv = np.ascontiguousarray(uv, dtype=np.int32).reshape(-1, 2)
    paths = np.full((len(uv), max(stride, 1)), -1, dtype=np.int32)
    lens = np.zeros(len(uv), dtype=np.int32)
    _check(_load().apsp_query_paths(g, uv.ctypes.data, len(uv), paths.ctypes.data, stride, lens.ctypes.data),
           "apsp_query_paths")
    return paths[:, :stride], lens


def apsp_query_path(g: int, u: int, v: int, cap: int) -> list:
    """Algorithm 7 for one pair: the slots of a shortest path (cut to cap; see apsp_query_paths for the full length)."""
    buf = np.zeros(max(cap, 1), dtype=np.int32)
    n = ctypes.c_int32()
    _check(_load().apsp_query_path(g, u, v, buf.ctypes.data, cap, ctypes.byref(n)), "apsp_query_path")
    return [int(x) for x in buf[:min(n.value, cap)]]


def apsp_query_all_paths(g: int, u: int, v: int) -> list:
    """Algorithm 8: list of shortest paths (lists of slots); sizes first, then the paths."""
    npaths, nnodes = ctypes.c_int32(), ctypes.c_int64()
    L = _load()
    _check(L.apsp_query_all_paths(g, u, v, None, 0, None, 0, ctypes.byref(npaths), ctypes.byref(nnodes)),
           "apsp_query_all_paths")
    nodes = np.zeros(max(nnodes.value, 1), dtype=np.int32)
    offs = np.zeros(npaths.value + 1, dtype=np.int64)
    _check(L.apsp_query_all_paths(g, u, v, nodes.ctypes.data, nnodes.value, offs.ctypes.data, npaths.value,
                                  ctypes.byref(npaths), ctypes.byref(nnodes)), "apsp_query_all_paths")
    return [[int(x) for x in nodes[offs[p]:offs[p + 1]]] for p in range(npaths.value)]


def apsp_probe_addmin_rate(dtype: int) -> float:
    """Min-plus steps per second of the CUDA cores (register-tile probe, current device)."""
    r = ctypes.c_double()
    _check(_load().apsp_probe_addmin_rate(dtype, ctypes.byref(r)), "apsp_probe_addmin_rate")
    return r.value


def apsp_probe_l2_read_gbs() -> float:
    """L2 read bandwidth of the current device in GB/s (probe kernel)."""
    r = ctypes.c_double()
    _check(_load().apsp_probe_l2_read_gbs(ctypes.byref(r)), "apsp_probe_l2_read_gbs")
    return r.value


def apsp_selftest_barrier_timeout(lose_cta: bool) -> int:
    """Status the bounded grid barrier reports when one CTA never arrives (or all do)."""
    st = ctypes.c_int32()
    _check(_load().apsp_selftest_barrier_timeout(1 if lose_cta else 0, ctypes.byref(st)),
           "apsp_selftest_barrier_timeout")
    return st.value


def apsp_copy_D(g: int, dst, ld: int, on_device: bool):
    _check(_load().apsp_copy_D(g, _ptr(dst), ld, 1 if on_device else 0), "apsp_copy_D")


def apsp_copy_W(g: int, dst, ld: int, on_device: bool):
    _check(_load().apsp_copy_W(g, _ptr(dst), ld, 1 if on_device else 0), "apsp_copy_W")


def apsp_copy_alive(g: int, capacity: int) -> np.ndarray:
    out = np.zeros(capacity, dtype=np.uint8)
    _check(_load().apsp_copy_alive(g, out.ctypes.data), "apsp_copy_alive")
    return out.astype(bool)


def apsp_info_get(g: int) -> dict:
    i = apsp_info()
    _check(_load().apsp_info_get(g, ctypes.byref(i)), "apsp_info_get")
    return {k: getattr(i, k) for k, _ in i._fields_}


def apsp_last_stats(g: int) -> dict:
    s = apsp_stats()
    _check(_load().apsp_last_stats(g, ctypes.byref(s)), "apsp_last_stats")
    return s.as_dict()


def apsp_copy_last_list(g: int) -> np.ndarray:
    """(count, 2) int32 array of the (i, j) pairs the last update listed."""
    cnt = ctypes.c_int64(0)
    _check(_load().apsp_copy_last_list(g, None, 0, ctypes.byref(cnt)), "apsp_copy_last_list")
    out = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
    _check(_load().apsp_copy_last_list(g, out.ctypes.data, cnt.value, ctypes.byref(cnt)), "apsp_copy_last_list")
    return out[: cnt.value]


def apsp_next_hops(g: int, rows, n_slots: int) -> np.ndarray:
    """(len(rows), n_slots) int32: next hops of the given live rows (-1: none)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)
    out = np.full((max(len(rows), 1), max(n_slots, 1)), -1, dtype=np.int32)
    _check(_load().apsp_next_hops(g, rows.ctypes.data, len(rows), out.ctypes.data, max(n_slots, 1)),
           "apsp_next_hops")
    return out[: len(rows), :n_slots]


def apsp_sync(g: int):
    _check(_load().apsp_sync(g), "apsp_sync")


def apsp_set_exact_list(g: int, on: bool):
    _check(_load().apsp_set_exact_list(g, 1 if on else 0), "apsp_set_exact_list")


LIST_MODES = {"corollary3": 0, "direct_edge": 1, "algorithm12": 2}


def apsp_set_list_mode(g: int, mode):
    m = LIST_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(_load().apsp_set_list_mode(g, m), "apsp_set_list_mode")


def apsp_set_dispatch(g: int, mode, delta: float = 1.0):
    m = DISPATCH[mode] if isinstance(mode, str) else int(mode)
    _check(_load().apsp_set_dispatch(g, m, float(delta)), "apsp_set_dispatch")


MODEL_NPARAM = 4750      # APSP_MODEL_NPARAM
MODEL_NTRAIN = 4738      # APSP_MODEL_NTRAIN


def _f32(a, shape_tail=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def apsp_set_model(g: int, params):
    """Install cost-model parameters (MODEL_NPARAM floats) on the handle; None removes it."""
    if params is None:
        _check(_load().apsp_set_model(g, None), "apsp_set_model")
        return
    p = _f32(params)
    if p.size != MODEL_NPARAM:
        raise ValueError(f"expected {MODEL_NPARAM} parameters, got {p.size}")
    _check(_load().apsp_set_model(g, p.ctypes.data), "apsp_set_model")


def apsp_model_loss_grad(params, X, Y):
    """(loss, grad[MODEL_NTRAIN]) of the model over samples X (n x 6), Y (n x 2)."""
    p, x, y = _f32(params), _f32(X), _f32(Y)
    n = x.shape[0]
    loss = np.zeros(1, np.float32)
    grad = np.zeros(MODEL_NTRAIN, np.float32)
    _check(_load().apsp_model_loss_grad(p.ctypes.data, x.ctypes.data, y.ctypes.data, n, loss.ctypes.data,
                                        grad.ctypes.data), "apsp_model_loss_grad")
    return float(loss[0]), grad


def apsp_model_predict(params, X):
    p, x = _f32(params), _f32(X)
    out = np.zeros((x.shape[0], 2), np.float32)
    _check(_load().apsp_model_predict(p.ctypes.data, x.ctypes.data, x.shape[0], out.ctypes.data), "apsp_model_predict")
    return out


def apsp_model_train(X, Y, epochs: int = 100, batch: int = 256, lr: float = 1e-3, seed: int = 1):
    """Train a cost model from scratch; returns (params[MODEL_NPARAM], final full-data loss)."""
    x, y = _f32(X), _f32(Y)
    out = np.zeros(MODEL_NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    _check(_load().apsp_model_train(x.ctypes.data, y.ctypes.data, x.shape[0], epochs, batch, float(lr), int(seed),
                                    out.ctypes.data, loss.ctypes.data), "apsp_model_train")
    return out, float(loss[0])


def apsp_batch_create(stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_load().apsp_batch_create(ctypes.byref(h), _stream_ptr(stream)), "apsp_batch_create")
    return h.value


def apsp_batch_destroy(b: int):
    _check(_load().apsp_batch_destroy(b), "apsp_batch_destroy")


def apsp_batch_set_width(b: int, threads: int):
    _check(_load().apsp_batch_set_width(b, threads), "apsp_batch_set_width")


def apsp_batch_info_get(b: int) -> dict:
    i = apsp_batch_info()
    _check(_load().apsp_batch_info_get(b, ctypes.byref(i)), "apsp_batch_info_get")
    return {k: getattr(i, k) for k, _ in i._fields_}


def apsp_batch_tuned_width(dtype: int, max_span: int) -> int:
    t = ctypes.c_int32()
    _check(_load().apsp_batch_tuned_width(dtype, max_span, ctypes.byref(t)), "apsp_batch_tuned_width")
    return t.value


def apsp_batch_run(b: int, graphs: Sequence[int], items) -> np.ndarray:
    """items: sequence of (graph index, op, ...): ("add", in_w, out_w), ("remove", u)
    or ("edge", u, v, w).  Returns the new slot of every add (-1 elsewhere)."""
    n = len(items)
    arr = (apsp_batch_item * max(1, n))()
    keep = []
    for q, it in enumerate(items):
        _fill_item(arr[q], it, keep)
    hs = (ctypes.c_void_p * len(graphs))(*graphs)
    ids = (ctypes.c_int32 * max(1, n))()
    _check(_load().apsp_batch_run(b, hs, len(graphs), arr, n, ids), "apsp_batch_run")
    return np.array(ids[:n], dtype=np.int32)


def _fill_item(e, it, keep):
    gi, op = it[0], it[1]
    e.graph = gi
    e.op = BATCH_OPS[op]
    if op == "add":
        a = np.ascontiguousarray(it[2])
        c = np.ascontiguousarray(it[3])
        keep += [a, c]
        e.in_w, e.out_w = a.ctypes.data, c.ctypes.data
    elif op == "remove":
        e.u = int(it[2])
    elif op == "query":
        e.u, e.v = int(it[2]), int(it[3])
    else:
        e.u, e.v, e.w = int(it[2]), int(it[3]), float(it[4])


def apsp_serve(graphs: Sequence[int], requests, arrivals, hbm_budget_bytes: float = 0.0, small_max_slots: int = 0,
               max_wave_requests: int = 0) -> dict:
    """Replays requests (items as for apsp_batch_run, plus ("query", u, v)) that
    arrive at `arrivals` (seconds, non-decreasing).  Returns numpy arrays:
    admit_s, done_s, dist, status, wave, new_id."""
    n = len(requests)
    arr = (apsp_request * max(1, n))()
    keep = []
    for q, it in enumerate(requests):
        _fill_item(arr[q].item, it, keep)
        arr[q].arrival_s = float(arrivals[q])
    cfg = apsp_serve_config(float(hbm_budget_bytes), int(small_max_slots), int(max_wave_requests))
    out = (apsp_request_result * max(1, n))()
    hs = (ctypes.c_void_p * len(graphs))(*graphs)
    _check(_load().apsp_serve(hs, len(graphs), arr, n, ctypes.byref(cfg), out), "apsp_serve")
    res = {k: np.array([getattr(out[q], k) for q in range(n)]) for k in ("admit_s", "done_s", "dist", "status", "wave", "new_id")}
    return res


def _result_dict(r) -> dict:
    return {k: getattr(r, k) for k in ("admit_s", "done_s", "dist", "status", "wave", "new_id")}


def apsp_server_create(graphs: Sequence[int], hbm_budget_bytes: float = 0.0, small_max_slots: int = 0,
                       max_wave_requests: int = 0) -> int:
    cfg = apsp_serve_config(float(hbm_budget_bytes), int(small_max_slots), int(max_wave_requests))
    hs = (ctypes.c_void_p * len(graphs))(*graphs)
    h = ctypes.c_void_p()
    _check(_load().apsp_server_create(ctypes.byref(h), hs, len(graphs), ctypes.byref(cfg)), "apsp_server_create")
    return h.value


def apsp_server_submit(s: int, item) -> int:
    e = apsp_batch_item()
    keep = []
    _fill_item(e, item, keep)
    t = ctypes.c_int64(-1)
    _check(_load().apsp_server_submit(s, ctypes.byref(e), ctypes.byref(t)), "apsp_server_submit")
    return t.value


def apsp_server_poll(s: int, ticket: int):
    """The request's result dict once it has completed, else None."""
    r = apsp_request_result()
    done = ctypes.c_int32(0)
    _check(_load().apsp_server_poll(s, ticket, ctypes.byref(r), ctypes.byref(done)), "apsp_server_poll")
    return _result_dict(r) if done.value else None


def apsp_server_wait(s: int, ticket: int, timeout_s: float = 60.0) -> dict:
    r = apsp_request_result()
    _check(_load().apsp_server_wait(s, ticket, float(timeout_s), ctypes.byref(r)), "apsp_server_wait")
    return _result_dict(r)


def apsp_server_clock(s: int) -> float:
    return float(_load().apsp_server_clock(s))


def apsp_server_destroy(s: int):
    _check(_load().apsp_server_destroy(s), "apsp_server_destroy")


class Server:
    """Online server over resident graphs (apsp_server_*): submit requests as
    they arrive, poll or wait for their results.  Requests are the items of
    apsp_batch_run plus ("query", u, v), each starting with its graph index."""

    def __init__(self, graphs, hbm_budget_bytes: float = 0.0, small_max_slots: int = 0, max_wave_requests: int = 0):
        self.h = apsp_server_create([g.h for g in graphs], hbm_budget_bytes, small_max_slots, max_wave_requests)

    def submit(self, item) -> int:
        return apsp_server_submit(self.h, item)

    def poll(self, ticket: int):
        return apsp_server_poll(self.h, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> dict:
        return apsp_server_wait(self.h, ticket, timeout_s)

    def clock(self) -> float:
        return apsp_server_clock(self.h)

    def close(self):
        if self.h:
            apsp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Executor that applies ordered updates to many graphs in one persistent launch."""

    def __init__(self, stream=None):
        self.h = apsp_batch_create(stream)

    def run(self, graphs, items) -> np.ndarray:
        return apsp_batch_run(self.h, [g.h for g in graphs], items)

    def set_width(self, threads: int):
        apsp_batch_set_width(self.h, threads)

    def info(self) -> dict:
        return apsp_batch_info_get(self.h)

    def close(self):
        if self.h:
            apsp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apsp_launch_count(g: int) -> int:
    return int(_load().apsp_launch_count(g))


def apsp_profile_enable(g: int, on: bool):
    _check(_load().apsp_profile_enable(g, 1 if on else 0), "apsp_profile_enable")


def apsp_profile_read(g: int) -> dict:
    cap = 64
    arr = (apsp_profile_entry * cap)()
    cnt = ctypes.c_int32()
    _check(_load().apsp_profile_read(g, arr, cap, ctypes.byref(cnt)), "apsp_profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(cnt.value, cap))}


def apsp_profile_reset(g: int):
    _check(_load().apsp_profile_reset(g), "apsp_profile_reset")


def apsp_add_node_noalloc(D, ld: int, n_slots: int, alive, dtype: int, in_w, out_w, p: int, stream=None):
    """Insertion on a caller-owned device matrix without any allocation (see apsp.h)."""
    _check(_load().apsp_add_node_noalloc(_ptr(D), ld, n_slots, _ptr(alive), dtype, _ptr(in_w), _ptr(out_w), p,
                                         _stream_ptr(stream)), "apsp_add_node_noalloc")


_torch_alloc_refs = None


def apsp_set_allocator_torch():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_refs
    import torch

    def _alloc(nbytes, stream, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _torch_alloc_refs = (a, f)
    _check(_load().apsp_set_allocator(a, f, None), "apsp_set_allocator")


def apsp_set_allocator_default():
    global _torch_alloc_refs
    _check(_load().apsp_set_allocator(ALLOC_FN(0), FREE_FN(0), None), "apsp_set_allocator")
    _torch_alloc_refs = None


# ---------------------------------------------------------------------------
# object wrapper
# ---------------------------------------------------------------------------

class Graph:
    """A device-resident graph and its APSP matrix (one C handle)."""

    def __init__(self, W, capacity: Optional[int] = None, *, undirected: bool = False, D=None,
                 stream=None, device_input: bool = False, minimax: bool = False):
        n = int(W.shape[0])
        if hasattr(W, "dtype") and str(W.dtype) in ("float32", "torch.float32"):
            self.dtype = APSP_F32
        else:
            self.dtype = APSP_I32
        flags = (APSP_UNDIRECTED if undirected else 0) | (APSP_D_GIVEN if D is not None else 0) | \
            (APSP_DEVICE_INPUT if device_input else 0) | (APSP_MINIMAX if minimax else 0)
        self.minimax = minimax
        self.capacity = int(capacity or n)
        self.undirected = undirected
        self.np_dtype = _np_dtype(self.dtype)
        if not device_input:
            W = np.ascontiguousarray(W, dtype=self.np_dtype)
            if D is not None:
                D = np.ascontiguousarray(D, dtype=self.np_dtype)
        self.h = apsp_init(W, n, self.capacity, self.dtype, flags, D, stream)

    def close(self):
        if self.h:
            apsp_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # updates
    def add_node(self, in_w, out_w) -> int:
        if hasattr(out_w, "data_ptr") and getattr(out_w, "is_cuda", False):
            return apsp_add_node_device(self.h, in_w, out_w)
        full_in = None if in_w is None else self._slot_vec(in_w)
        return apsp_add_node(self.h, full_in, self._slot_vec(out_w))

    def _slot_vec(self, w):
        w = np.asarray(w, dtype=self.np_dtype)
        if len(w) == self.capacity:
            return np.ascontiguousarray(w)
        out = np.full(self.capacity, self.inf, dtype=self.np_dtype)
        out[:len(w)] = w
        return out

    def remove_node(self, v: int):
        apsp_remove_node(self.h, v)

    def update_edge(self, u: int, v: int, w):
        apsp_update_edge(self.h, u, v, w, self.dtype)

    def recompute(self):
        apsp_recompute(self.h)

    # queries
    @property
    def inf(self):
        return np.float32(np.inf) if self.dtype == APSP_F32 else np.int32(APSP_INF_I32)

    def query(self, u: int, v: int):
        return apsp_query(self.h, u, v, self.dtype)

    def query_batch(self, uv):
        return apsp_query_batch(self.h, uv, self.dtype)

    def query_path(self, u: int, v: int, cap: Optional[int] = None) -> list:
        return apsp_query_path(self.h, u, v, self.capacity + 1 if cap is None else cap)

    def query_paths(self, uv, stride: Optional[int] = None):
        return apsp_query_paths(self.h, uv, self.capacity + 1 if stride is None else stride)

    def query_all_paths(self, u: int, v: int) -> list:
        return apsp_query_all_paths(self.h, u, v)

    def info(self) -> dict:
        return apsp_info_get(self.h)

    def D(self) -> np.ndarray:
        m = self.info()["n_slots"]
        out = np.empty((m, m), dtype=self.np_dtype)
        apsp_copy_D(self.h, out, m, False)
        return out

    def W(self) -> np.ndarray:
        m = self.info()["n_slots"]
        out = np.empty((m, m), dtype=self.np_dtype)
        apsp_copy_W(self.h, out, m, False)
        return out

    def alive(self) -> np.ndarray:
        return apsp_copy_alive(self.h, self.capacity)[: self.info()["n_slots"]]

    def stats(self) -> dict:
        return apsp_last_stats(self.h)

    def next_hops(self, rows) -> np.ndarray:
        return apsp_next_hops(self.h, rows, self.info()["n_slots"])

    def last_list(self) -> np.ndarray:
        return apsp_copy_last_list(self.h)

    def sync(self):
        apsp_sync(self.h)

    def set_dispatch(self, mode, delta: float = 1.0):
        apsp_set_dispatch(self.h, mode, delta)

    def set_list_mode(self, mode):
        apsp_set_list_mode(self.h, mode)

    def set_exact_list(self, on: bool = True):
        apsp_set_exact_list(self.h, on)

    def set_model(self, params):
        apsp_set_model(self.h, params)

    def launches(self) -> int:
        return apsp_launch_count(self.h)
