"""The oracle -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``ba_oracle.c``, the plain single-threaded CPU statement of the
Batagelj-Brandes edge array (Sanders & Schulz, arXiv:1602.07106, section 2; seed graph
of section 4).  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA library.

Every function returns numpy arrays; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ba_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lib = None
_lock = threading.Lock()

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``ba_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                    "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.ora_hash_bits.restype = _u64
        lib.ora_hash_bits.argtypes = [_u64, _u64]
        lib.ora_hash.restype = _u64
        lib.ora_hash.argtypes = [_u64, _u64]
        lib.ora_num_edges.restype = _u64
        lib.ora_num_edges.argtypes = [_u64, _u32, _u64]
        lib.ora_bb_array.restype = ctypes.c_int
        lib.ora_bb_array.argtypes = [_u64, _u64, _u32, _u64, _ptr]
        for name in ("ora_edges_range", "ora_chain_lengths"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [_u64, _u64, _u32, _u64, _u64, _u64, _ptr]
        lib.ora_degrees_of_array.restype = None
        lib.ora_degrees_of_array.argtypes = [_ptr, _u64, _u64, _ptr]
        lib.ora_degree_count_range.restype = ctypes.c_int
        lib.ora_degree_count_range.argtypes = [_u64, _u64, _u32, _u64, _u64, _u64, _u64,
                                               _ptr]
        lib.ora_crc32c_update.restype = _u32
        lib.ora_crc32c_update.argtypes = [_u32, _ptr, _u64]
        lib.ora_crc32c_u64.restype = _u32
        lib.ora_crc32c_u64.argtypes = [_u32, _u64]
        lib.ora_hash_crc_bits.restype = _u64
        lib.ora_hash_crc_bits.argtypes = [_u64, _u64]
        lib.ora_draw.restype = _u64
        lib.ora_draw.argtypes = [ctypes.c_int, _u64, _u64, _u64]
        lib.ora_bb_array_variant.restype = ctypes.c_int
        lib.ora_bb_array_variant.argtypes = [_u64, _u64, _u32, _u64, ctypes.c_int,
                                             ctypes.c_int, _ptr]
        lib.ora_edges_range_variant.restype = ctypes.c_int
        lib.ora_edges_range_variant.argtypes = [_u64, _u64, _u32, _u64, ctypes.c_int,
                                                ctypes.c_int, _u64, _u64, _ptr]
        lib.ora_degree_count_range_variant.restype = ctypes.c_int
        lib.ora_degree_count_range_variant.argtypes = [_u64, _u64, _u32, _u64,
                                                       ctypes.c_int, ctypes.c_int, _u64,
                                                       _u64, _u64, _ptr]
        lib.ora_edges_simple.restype = ctypes.c_int
        lib.ora_edges_simple.argtypes = [_u64, _u64, _u32, _u64, ctypes.c_int, _ptr, _ptr]
        lib.ora_edges_range_simple.restype = ctypes.c_int
        lib.ora_edges_range_simple.argtypes = [_u64, _u64, _u32, _u64, ctypes.c_int, _u64,
                                               _u64, _ptr]
        lib.ora_degree_count_range_simple.restype = ctypes.c_int
        lib.ora_degree_count_range_simple.argtypes = [_u64, _u64, _u32, _u64, ctypes.c_int,
                                                      _u64, _u64, _u64, _ptr]
        _lib = lib
        return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def hash_bits(seed: int, r: int) -> int:
    """The 64 mixed bits z for position r (before reduction to 0..r-1)."""
    return int(_load().ora_hash_bits(seed, r))


def h(seed: int, r: int) -> int:
    """h(r) in 0..r-1 (section 2)."""
    return int(_load().ora_hash(seed, r))


def num_edges(n: int, d: int, n0: int = 0) -> int:
    """m = n0(n0-1)/2 + (n-n0) d; 0 when the parameters are not a graph."""
    return int(_load().ora_num_edges(n, d, n0))


def seed_edges(n0: int) -> int:
    return n0 * (n0 - 1) // 2 if n0 > 0 else 0


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid graph parameters or range")


def bb_array(seed: int, n: int, d: int, n0: int = 0) -> np.ndarray:
    """The full Batagelj-Brandes array E[0..2m-1] (int64)."""
    m = num_edges(n, d, n0)
    if m == 0:
        raise ValueError("oracle bb_array: invalid graph parameters")
    E = np.empty(2 * m, dtype=np.int64)
    _check(_load().ora_bb_array(seed, n, d, n0, _p(E)), "bb_array")
    return E


def edges_range(seed: int, n: int, d: int, n0: int, a: int, b: int) -> np.ndarray:
    """Edges a..b-1 as an int64 array of shape (b-a, 2), recomputed without the array."""
    out = np.empty((max(b - a, 0), 2), dtype=np.int64)
    _check(_load().ora_edges_range(seed, n, d, n0, a, b, _p(out)), "edges_range")
    return out


def chain_lengths(seed: int, n: int, d: int, n0: int, a: int, b: int) -> np.ndarray:
    """Hash evaluations spent on the second end point of each edge a..b-1."""
    out = np.empty(max(b - a, 0), dtype=np.uint64)
    _check(_load().ora_chain_lengths(seed, n, d, n0, a, b, _p(out)), "chain_lengths")
    return out


def degrees_of_array(E: np.ndarray, node_limit: int) -> np.ndarray:
    E = np.ascontiguousarray(E, dtype=np.int64)
    counts = np.zeros(node_limit, dtype=np.uint64)
    _load().ora_degrees_of_array(_p(E), E.size, node_limit, _p(counts))
    return counts


def degree_count_range(seed: int, n: int, d: int, n0: int, a: int, b: int,
                       node_limit: int, counts: np.ndarray | None = None) -> np.ndarray:
    """Degrees (end-point occurrences) of nodes 0..node_limit-1 over edges a..b-1."""
    if counts is None:
        counts = np.zeros(node_limit, dtype=np.uint64)
    assert counts.dtype == np.uint64 and counts.size == node_limit
    _check(_load().ora_degree_count_range(seed, n, d, n0, a, b, node_limit, _p(counts)),
           "degree_count_range")
    return counts


# ---------------------------------------------------------------- variants (section 4,
# Fig. 3).  family: HASH_SPLITMIX (the h above) or HASH_CRC (hash_crc of Fig. 3);
# no_self_loops: draw edge i's target only from the edges of earlier nodes.

HASH_SPLITMIX = 0
HASH_CRC = 1


def crc32c_update(crc: int, data: bytes) -> int:
    """CRC-32C advanced over ``data`` from the running value ``crc`` (no inversions)."""
    buf = np.frombuffer(bytes(data), dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    return int(_load().ora_crc32c_update(crc, _p(buf), len(data)))


def crc32c_u64(crc: int, v: int) -> int:
    """The 64-bit CRC32 instruction's update: the eight bytes of v, little-endian."""
    return int(_load().ora_crc32c_u64(crc, v))


def hash_crc_bits(seed: int, r: int) -> int:
    """hash_crc's 64 bits for key r (Fig. 3 for seed 0)."""
    return int(_load().ora_hash_crc_bits(seed, r))


def draw(family: int, seed: int, key: int, rng: int) -> int:
    """A draw in 0..rng-1 for ``key`` (h(r) is draw(HASH_SPLITMIX, seed, r, r))."""
    return int(_load().ora_draw(family, seed, key, rng))


def bb_array_variant(seed: int, n: int, d: int, n0: int, family: int,
                     no_self_loops: bool) -> np.ndarray:
    """The full variant array E[0..2m-1] (int64)."""
    m = num_edges(n, d, n0)
    if m == 0:
        raise ValueError("oracle bb_array_variant: invalid graph parameters")
    E = np.empty(2 * m, dtype=np.int64)
    _check(_load().ora_bb_array_variant(seed, n, d, n0, family, int(no_self_loops), _p(E)),
           "bb_array_variant")
    return E


def edges_range_variant(seed: int, n: int, d: int, n0: int, family: int,
                        no_self_loops: bool, a: int, b: int) -> np.ndarray:
    """Edges a..b-1 of the variant graph, shape (b-a, 2), recomputed without the array."""
    out = np.empty((max(b - a, 0), 2), dtype=np.int64)
    _check(_load().ora_edges_range_variant(seed, n, d, n0, family, int(no_self_loops), a,
                                           b, _p(out)), "edges_range_variant")
    return out


def degree_count_range_variant(seed: int, n: int, d: int, n0: int, family: int,
                               no_self_loops: bool, a: int, b: int, node_limit: int,
                               counts: np.ndarray | None = None) -> np.ndarray:
    """Degrees of nodes 0..node_limit-1 over edges a..b-1 of the variant graph."""
    if counts is None:
        counts = np.zeros(node_limit, dtype=np.uint64)
    assert counts.dtype == np.uint64 and counts.size == node_limit
    _check(_load().ora_degree_count_range_variant(seed, n, d, n0, family,
                                                  int(no_self_loops), a, b, node_limit,
                                                  _p(counts)), "degree_count_range_variant")
    return counts


# Graphs without parallel edges (section 4: a node's duplicate targets are rejected).
REDRAW_SALT = 0xD6E8FEB86659FD93
REDRAW_CAP = 65536


def edges_simple(seed: int, n: int, d: int, n0: int, no_self_loops: bool) -> np.ndarray:
    """All m edges, shape (m, 2), of the graph whose nodes reject duplicate targets, built
    on the stored array without rejection that the chains follow."""
    m = num_edges(n, d, n0)
    if m == 0:
        raise ValueError("oracle edges_simple: invalid graph parameters")
    E = np.empty(2 * m, dtype=np.int64)
    out = np.empty((m, 2), dtype=np.int64)
    _check(_load().ora_edges_simple(seed, n, d, n0, int(no_self_loops), _p(E), _p(out)),
           "edges_simple")
    return out


def edges_range_simple(seed: int, n: int, d: int, n0: int, no_self_loops: bool, a: int,
                       b: int) -> np.ndarray:
    """Edges a..b-1 of that graph, shape (b-a, 2), recomputed without the array."""
    out = np.empty((max(b - a, 0), 2), dtype=np.int64)
    _check(_load().ora_edges_range_simple(seed, n, d, n0, int(no_self_loops), a, b, _p(out)),
           "edges_range_simple")
    return out


def degree_count_range_simple(seed: int, n: int, d: int, n0: int, no_self_loops: bool, a: int,
                              b: int, node_limit: int,
                              counts: np.ndarray | None = None) -> np.ndarray:
    """Degrees of nodes 0..node_limit-1 over edges a..b-1 of that graph."""
    if counts is None:
        counts = np.zeros(node_limit, dtype=np.uint64)
    assert counts.dtype == np.uint64 and counts.size == node_limit
    _check(_load().ora_degree_count_range_simple(seed, n, d, n0, int(no_self_loops), a, b,
                                                 node_limit, _p(counts)),
           "degree_count_range_simple")
    return counts
