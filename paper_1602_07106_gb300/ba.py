"""Thin Python binding of libba (include/ba.h): argument marshalling only.

Every function named ``ba_*`` calls the C entry point of the same name; device buffers are
passed as torch CUDA tensors (or raw integer addresses) and streams as torch streams (or
raw ``cudaStream_t`` integers; None = torch's current stream).  Errors raise ``BAError``.
Importing this module raises ImportError when libba.so has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libba.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ba.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libba.so is not built ({LIB_PATH}); run "
                      "`python -m paper_1602_07106_gb300.build` (needs nvcc)")
_lib = ctypes.CDLL(LIB_PATH)

BA_OK, BA_ERR_INVALID_ARG, BA_ERR_RANGE, BA_ERR_OVERFLOW = 0, 1, 2, 3
BA_ERR_CUDA, BA_ERR_NOMEM, BA_ERR_TIMEOUT, BA_ERR_BUSY, BA_ERR_NOT_FOUND = 4, 5, 6, 7, 8
BA_KIND_GENERATE, BA_KIND_DEGREE, BA_KIND_BATCH = 0, 1, 2
BA_REQ_QUEUED, BA_REQ_RUNNING, BA_REQ_DONE, BA_REQ_FAILED = 0, 1, 2, 3
BA_VARIANT_CRC_HASH, BA_VARIANT_NO_SELF_LOOPS, BA_VARIANT_NO_PARALLEL_EDGES = 1, 2, 4

_u64, _u32, _i32, _i64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64
_vp = ctypes.c_void_p


class ba_tuning(ctypes.Structure):
    _fields_ = [("block", _i32), ("ctas_per_sm", _i32), ("tile", _i32), ("refill", _i32),
                ("hist_bins", _i32), ("hist_agg", _i32), ("chains", _i32),
                ("reserved", _i32)]

    def as_dict(self):
        return {k: getattr(self, k)
                for k in ("block", "ctas_per_sm", "tile", "refill", "hist_bins", "hist_agg",
                          "chains")}


class ba_graph_desc(ctypes.Structure):
    _fields_ = [("seed", _u64), ("n", _u64), ("n0", _u64), ("edge_begin", _u64),
                ("edge_end", _u64), ("d", _u32), ("reserved", _u32)]


class ba_server_config(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", _u64), ("chunk_edges", _u64), ("max_active", _i32),
                ("max_inflight_ticks", _i32), ("device", _i32), ("max_queued", _i32),
                ("tick_edges", _u64)]


class ba_server_stats(ctypes.Structure):
    _fields_ = [(k, _u64) for k in ("submitted", "admitted", "completed", "released",
                                    "rejected_busy", "ticks", "edges_done", "bytes_in_use",
                                    "queue_depth", "active", "cancelled")]


def _sig(name, restype, *argtypes):
    fn = getattr(_lib, name)
    fn.restype = restype
    fn.argtypes = list(argtypes)
    return fn


_sig("ba_status_string", ctypes.c_char_p, ctypes.c_int)
_sig("ba_last_error_message", ctypes.c_char_p)
_sig("ba_version", ctypes.c_int)
_sig("ba_num_edges", _u64, _u64, _u32, _u64)
_sig("ba_generate_edges", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _vp, _vp)
_sig("ba_generate_edges_host", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _vp, _vp)
_sig("ba_generate_edges32", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _vp, _vp)
_sig("ba_degree_count", ctypes.c_int, _u64, _u64, _u32, _u64, _vp, _vp)
_sig("ba_degree_count_range", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _u64, _vp,
     ctypes.c_int, _vp)
_sig("ba_generate_edges_variant", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _u32, _vp,
     _vp)
_sig("ba_degree_count_variant", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _u64, _u32,
     _vp, ctypes.c_int, _vp)
_sig("ba_set_tuning", ctypes.c_int, _i32, ctypes.POINTER(ba_tuning))
_sig("ba_get_tuning", ctypes.c_int, _i32, _u64, ctypes.POINTER(ba_tuning))
_sig("ba_tune", ctypes.c_int, _i32, _u64, _u64, _u32, _u64, _u64, _u64, _vp, _vp,
     ctypes.POINTER(ba_tuning))
_sig("ba_tune_save", ctypes.c_int, ctypes.c_char_p)
_sig("ba_tune_load", ctypes.c_int, ctypes.c_char_p)
_sig("ba_batch_plan_create", ctypes.c_int, ctypes.POINTER(ba_graph_desc), _i32, _vp,
     ctypes.POINTER(ba_tuning), ctypes.POINTER(_vp))
_sig("ba_batch_plan_total_edges", _u64, _vp)
_sig("ba_batch_plan_offsets", ctypes.c_int, _vp, _vp)
_sig("ba_batch_plan_launch", ctypes.c_int, _vp, _vp, _vp)
_sig("ba_batch_plan_destroy", ctypes.c_int, _vp)
_sig("ba_generate_batch", ctypes.c_int, ctypes.POINTER(ba_graph_desc), _i32, _vp, _vp,
     ctypes.POINTER(ba_tuning), _vp)
_sig("ba_generate_batch_noalloc", ctypes.c_int, ctypes.POINTER(ba_graph_desc), _i32, _vp, _vp,
     _vp)
_sig("ba_device_allocations", _u64)
_sig("ba_generate_edges_checked", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _vp, _u64, _vp,
     _vp)
_sig("ba_check_status", ctypes.c_int, _vp, _vp)
_sig("ba_chain_lengths", ctypes.c_int, _u64, _u64, _u32, _u64, _u64, _u64, _u32, _vp, ctypes.c_int,
     _vp)
_sig("ba_probe_hash", ctypes.c_int, _u64, _u64, _u64, _i32, _vp, _vp)
_sig("ba_probe_write", ctypes.c_int, _vp, _u64, _vp)
_sig("ba_server_create", ctypes.c_int, ctypes.POINTER(ba_server_config), ctypes.POINTER(_vp))
_sig("ba_server_submit", ctypes.c_int, _vp, ctypes.POINTER(ba_graph_desc), ctypes.POINTER(_u64))
_sig("ba_server_poll", ctypes.c_int, _vp, _u64, ctypes.POINTER(_i32), ctypes.POINTER(_u64))
_sig("ba_server_wait", ctypes.c_int, _vp, _u64, _i64)
_sig("ba_server_result", ctypes.c_int, _vp, _u64, ctypes.POINTER(_vp), ctypes.POINTER(_u64))
_sig("ba_server_copy_result", ctypes.c_int, _vp, _u64, _vp, _vp)
_sig("ba_server_release", ctypes.c_int, _vp, _u64)
_sig("ba_server_cancel", ctypes.c_int, _vp, _u64)
_sig("ba_server_stats_get", ctypes.c_int, _vp, ctypes.POINTER(ba_server_stats))
_sig("ba_server_destroy", ctypes.c_int, _vp)


class BAError(RuntimeError):
    def __init__(self, status: int, fn: str):
        self.status = status
        msg = _lib.ba_last_error_message().decode()
        super().__init__(f"{fn}: {_lib.ba_status_string(status).decode()}"
                         + (f" ({msg})" if msg else ""))


def _check(status: int, fn: str) -> None:
    if status != BA_OK:
        raise BAError(status, fn)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.data_ptr() if x.numel() else None
    return int(x)


def _stream(s) -> int | None:
    if s is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(s, torch.cuda.Stream):
        return s.cuda_stream
    return int(s)


def _need_cuda(t: torch.Tensor, dtype: torch.dtype, numel: int, what: str) -> None:
    if not isinstance(t, torch.Tensor):
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{what}: need a contiguous CUDA {dtype} tensor of >= {numel} elements")


# ------------------------------------------------------------------------- C names --

def ba_status_string(status: int) -> str:
    return _lib.ba_status_string(status).decode()


def ba_last_error_message() -> str:
    return _lib.ba_last_error_message().decode()


def ba_version() -> int:
    return _lib.ba_version()


def ba_num_edges(n: int, d: int, n0: int = 0) -> int:
    return int(_lib.ba_num_edges(n, d, n0))


def ba_generate_edges(seed, n, d, n0, edge_begin, edge_end, out, stream=None) -> None:
    _need_cuda(out, torch.int64, 2 * (edge_end - edge_begin), "ba_generate_edges out")
    _check(_lib.ba_generate_edges(seed, n, d, n0, edge_begin, edge_end, _ptr(out),
                                  _stream(stream)), "ba_generate_edges")


def ba_generate_edges32(seed, n, d, n0, edge_begin, edge_end, out, stream=None) -> None:
    _need_cuda(out, torch.int32, 2 * (edge_end - edge_begin), "ba_generate_edges32 out")
    _check(_lib.ba_generate_edges32(seed, n, d, n0, edge_begin, edge_end, _ptr(out),
                                    _stream(stream)), "ba_generate_edges32")


def ba_generate_edges_host(seed, n, d, n0, edge_begin, edge_end, host_out, stream=None) -> None:
    if isinstance(host_out, torch.Tensor):
        if host_out.is_cuda or host_out.dtype != torch.int64 or not host_out.is_contiguous() \
                or host_out.numel() < 2 * (edge_end - edge_begin):
            raise ValueError("ba_generate_edges_host: need a contiguous CPU int64 tensor")
    _check(_lib.ba_generate_edges_host(seed, n, d, n0, edge_begin, edge_end, _ptr(host_out),
                                       _stream(stream)), "ba_generate_edges_host")


def ba_degree_count(seed, n, d, node_limit, counts, stream=None) -> None:
    _need_cuda(counts, torch.int64, node_limit, "ba_degree_count counts")
    _check(_lib.ba_degree_count(seed, n, d, node_limit, _ptr(counts), _stream(stream)),
           "ba_degree_count")


def ba_degree_count_range(seed, n, d, n0, edge_begin, edge_end, node_limit, counts,
                          accumulate=0, stream=None) -> None:
    _need_cuda(counts, torch.int64, node_limit, "ba_degree_count_range counts")
    _check(_lib.ba_degree_count_range(seed, n, d, n0, edge_begin, edge_end, node_limit,
                                      _ptr(counts), int(accumulate), _stream(stream)),
           "ba_degree_count_range")


def ba_generate_edges_variant(seed, n, d, n0, edge_begin, edge_end, variant, out,
                              stream=None) -> None:
    _need_cuda(out, torch.int64, 2 * (edge_end - edge_begin), "ba_generate_edges_variant out")
    _check(_lib.ba_generate_edges_variant(seed, n, d, n0, edge_begin, edge_end, variant,
                                          _ptr(out), _stream(stream)),
           "ba_generate_edges_variant")


def ba_degree_count_variant(seed, n, d, n0, edge_begin, edge_end, node_limit, variant, counts,
                            accumulate=0, stream=None) -> None:
    _need_cuda(counts, torch.int64, node_limit, "ba_degree_count_variant counts")
    _check(_lib.ba_degree_count_variant(seed, n, d, n0, edge_begin, edge_end, node_limit,
                                        variant, _ptr(counts), int(accumulate),
                                        _stream(stream)), "ba_degree_count_variant")


def _tuning(t) -> ba_tuning | None:
    if t is None or isinstance(t, ba_tuning):
        return t
    x = ba_tuning()
    for k, v in dict(t).items():
        setattr(x, k, int(v))
    return x


def ba_set_tuning(kind: int, tune=None) -> None:
    t = _tuning(tune)
    _check(_lib.ba_set_tuning(kind, ctypes.byref(t) if t is not None else None), "ba_set_tuning")


def ba_get_tuning(kind: int, edge_end: int = 1) -> dict:
    t = ba_tuning()
    _check(_lib.ba_get_tuning(kind, edge_end, ctypes.byref(t)), "ba_get_tuning")
    return t.as_dict()


def ba_tune(kind, seed, n, d, n0, edge_begin, edge_end, scratch=None, stream=None) -> dict:
    t = ba_tuning()
    _check(_lib.ba_tune(kind, seed, n, d, n0, edge_begin, edge_end, _ptr(scratch),
                        _stream(stream), ctypes.byref(t)), "ba_tune")
    return t.as_dict()


def ba_tune_save(path: str | None = None) -> None:
    _check(_lib.ba_tune_save(path.encode() if path else None), "ba_tune_save")


def ba_tune_load(path: str | None = None) -> None:
    _check(_lib.ba_tune_load(path.encode() if path else None), "ba_tune_load")


def _descs(graphs) -> tuple[ctypes.Array, int]:
    """graphs: iterable of (seed, n, d, n0, edge_begin, edge_end) tuples or ba_graph_desc."""
    graphs = list(graphs)
    arr = (ba_graph_desc * max(len(graphs), 1))()
    for i, g in enumerate(graphs):
        if isinstance(g, ba_graph_desc):
            arr[i] = g
        else:
            seed, n, d, n0, a, b = g
            arr[i] = ba_graph_desc(seed, n, n0, a, b, d, 0)
    return arr, len(graphs)


def _offsets_arg(offsets, G: int):
    if offsets is None:
        return None, None
    if len(offsets) != G + 1:
        raise ValueError(f"offsets needs G + 1 = {G + 1} entries, got {len(offsets)}")
    arr = (ctypes.c_int64 * len(offsets))(*[int(x) for x in offsets])
    return arr, ctypes.addressof(arr)


def ba_batch_plan_create(graphs, offsets=None, tune=None) -> int:
    arr, G = _descs(graphs)
    keep, off = _offsets_arg(offsets, G)
    t = _tuning(tune)
    plan = _vp()
    _check(_lib.ba_batch_plan_create(arr, G, off, ctypes.byref(t) if t is not None else None,
                                     ctypes.byref(plan)), "ba_batch_plan_create")
    return plan.value


def ba_batch_plan_total_edges(plan: int) -> int:
    return int(_lib.ba_batch_plan_total_edges(plan))


def ba_batch_plan_offsets(plan: int, G: int) -> list[int]:
    arr = (ctypes.c_int64 * (G + 1))()
    _check(_lib.ba_batch_plan_offsets(plan, ctypes.addressof(arr)), "ba_batch_plan_offsets")
    return list(arr)


def ba_batch_plan_launch(plan: int, out, stream=None) -> None:
    _check(_lib.ba_batch_plan_launch(plan, _ptr(out), _stream(stream)), "ba_batch_plan_launch")


def ba_batch_plan_destroy(plan: int) -> None:
    _check(_lib.ba_batch_plan_destroy(plan), "ba_batch_plan_destroy")


def ba_generate_batch(graphs, out, offsets=None, tune=None, stream=None) -> None:
    arr, G = _descs(graphs)
    keep, off = _offsets_arg(offsets, G)
    t = _tuning(tune)
    _check(_lib.ba_generate_batch(arr, G, off, _ptr(out), ctypes.byref(t) if t is not None else None,
                                  _stream(stream)), "ba_generate_batch")


BA_NOALLOC_MAX_GRAPHS = 1024


def ba_generate_batch_noalloc(graphs, out, offsets=None, stream=None) -> None:
    """ba_generate_batch without any device allocation: scratch comes from the library's
    static device table (at most BA_NOALLOC_MAX_GRAPHS graphs); calls that overlap on the
    GPU share that table and must be serialised by the caller."""
    arr, G = _descs(graphs)
    keep, off = _offsets_arg(offsets, G)
    _check(_lib.ba_generate_batch_noalloc(arr, G, off, _ptr(out), _stream(stream)),
           "ba_generate_batch_noalloc")


def ba_chain_lengths(seed, n, d, n0, edge_begin, edge_end, bins, hist, accumulate=False,
                     stream=None) -> None:
    """Histogram of the chain lengths (draws per edge) of edges [edge_begin, edge_end) into
    the int64 device tensor hist (bins entries; the last one counts bins-1 draws or more)."""
    _check(_lib.ba_chain_lengths(seed, n, d, n0, edge_begin, edge_end, bins, _ptr(hist),
                                 int(bool(accumulate)), _stream(stream)), "ba_chain_lengths")


def ba_generate_edges_checked(seed, n, d, n0, edge_begin, edge_end, out, capacity, status,
                              stream=None) -> None:
    """ba_generate_edges with every store checked against `capacity` edges of `out`;
    `status` is a one-element int64 device tensor read by ba_check_status."""
    _check(_lib.ba_generate_edges_checked(seed, n, d, n0, edge_begin, edge_end, _ptr(out),
                                          capacity, _ptr(status), _stream(stream)),
           "ba_generate_edges_checked")


def ba_check_status(status, stream=None) -> None:
    """Raises BAError (BA_ERR_CUDA) if the checked launch behind `status` found a store
    beyond its capacity."""
    _check(_lib.ba_check_status(_ptr(status), _stream(stream)), "ba_check_status")


def ba_device_allocations() -> int:
    """Device allocations libba has made in this process so far."""
    return int(_lib.ba_device_allocations())


def ba_probe_hash(seed, base, edges, chains, sink, stream=None) -> None:
    """Two draws per edge with nothing else (the integer floor of the chain); sink is a
    one-element int64 device tensor that receives an XOR of the results."""
    _check(_lib.ba_probe_hash(seed, base, edges, chains, _ptr(sink), _stream(stream)),
           "ba_probe_hash")


def ba_probe_write(dst, nbytes=None, stream=None) -> None:
    """16-byte streaming stores over the device tensor dst (its first nbytes bytes)."""
    n = dst.numel() * dst.element_size() if nbytes is None else nbytes
    _check(_lib.ba_probe_write(_ptr(dst), n, _stream(stream)), "ba_probe_write")


def ba_server_create(memory_budget_bytes=0, chunk_edges=0, max_active=0, max_inflight_ticks=0,
                     device=-1, max_queued=0, tick_edges=0) -> int:
    cfg = ba_server_config(memory_budget_bytes, chunk_edges, max_active, max_inflight_ticks,
                           device, max_queued, tick_edges)
    srv = _vp()
    _check(_lib.ba_server_create(ctypes.byref(cfg), ctypes.byref(srv)), "ba_server_create")
    return srv.value


def ba_server_submit(server: int, seed, n, d, n0, edge_begin, edge_end) -> int:
    desc = ba_graph_desc(seed, n, n0, edge_begin, edge_end, d, 0)
    ticket = _u64()
    _check(_lib.ba_server_submit(server, ctypes.byref(desc), ctypes.byref(ticket)),
           "ba_server_submit")
    return ticket.value


def ba_server_poll(server: int, ticket: int) -> tuple[int, int]:
    state, lat = _i32(), _u64()
    _check(_lib.ba_server_poll(server, ticket, ctypes.byref(state), ctypes.byref(lat)),
           "ba_server_poll")
    return state.value, lat.value


def ba_server_wait(server: int, ticket: int, timeout_ms: int = 60_000) -> None:
    _check(_lib.ba_server_wait(server, ticket, timeout_ms), "ba_server_wait")


def ba_server_result(server: int, ticket: int) -> tuple[int, int]:
    ptr, n = _vp(), _u64()
    _check(_lib.ba_server_result(server, ticket, ctypes.byref(ptr), ctypes.byref(n)),
           "ba_server_result")
    return ptr.value or 0, n.value


def ba_server_release(server: int, ticket: int) -> None:
    _check(_lib.ba_server_release(server, ticket), "ba_server_release")


def ba_server_cancel(server: int, ticket: int) -> None:
    """Withdraws a request that is still waiting for admission."""
    _check(_lib.ba_server_cancel(server, ticket), "ba_server_cancel")


def ba_server_stats_get(server: int) -> dict:
    st = ba_server_stats()
    _check(_lib.ba_server_stats_get(server, ctypes.byref(st)), "ba_server_stats_get")
    return {k: getattr(st, k) for k, _ in ba_server_stats._fields_}


def ba_server_destroy(server: int) -> None:
    _check(_lib.ba_server_destroy(server), "ba_server_destroy")


# ------------------------------------------------------------------- conveniences --

def generate_edges(seed: int, n: int, d: int, n0: int = 0, edge_begin: int = 0,
                   edge_end: int | None = None, stream=None) -> torch.Tensor:
    """Edges [edge_begin, edge_end) as a (k, 2) int64 CUDA tensor on the current device."""
    m = ba_num_edges(n, d, n0)
    end = m if edge_end is None else edge_end
    out = torch.empty((max(end - edge_begin, 0), 2), dtype=torch.int64, device="cuda")
    ba_generate_edges(seed, n, d, n0, edge_begin, end, out, stream)
    return out


def degree_count(seed: int, n: int, d: int, node_limit: int, n0: int = 0, edge_begin: int = 0,
                 edge_end: int | None = None, stream=None) -> torch.Tensor:
    """Degrees of nodes 0..node_limit-1 over edges [edge_begin, edge_end) (int64 CUDA tensor)."""
    m = ba_num_edges(n, d, n0)
    end = m if edge_end is None else edge_end
    counts = torch.empty(node_limit, dtype=torch.int64, device="cuda")
    ba_degree_count_range(seed, n, d, n0, edge_begin, end, node_limit, counts, 0, stream)
    return counts


def ba_server_copy_result(server: int, ticket: int, dst, stream=None) -> None:
    _check(_lib.ba_server_copy_result(server, ticket, _ptr(dst), _stream(stream)),
           "ba_server_copy_result")


def server_result_tensor(server: int, ticket: int, stream=None) -> torch.Tensor:
    """Copies a DONE request's edges out of the server arena into a new (k, 2) CUDA tensor."""
    _, k = ba_server_result(server, ticket)
    out = torch.empty((k, 2), dtype=torch.int64, device="cuda")
    ba_server_copy_result(server, ticket, out, stream)
    return out


def declared_functions(header: str = HEADER) -> list[str]:
    """Names of the functions include/ba.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z0-9_]+)\s*\(", text)))
