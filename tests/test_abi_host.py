"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/ba.h declares, and rejects malformed arguments before touching a GPU."""
import ctypes
import os

import pytest

from paper_1602_07106_gb300 import build as ba_build

LIB = ba_build.build()  # nvcc cross-compiles sm_103a without a GPU
from paper_1602_07106_gb300 import ba  # noqa: E402  (needs the built library)


def test_every_declared_function_is_exported():
    names = ba.declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(LIB)
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, missing


def test_library_targets_sm_103a_only():
    # the build passes exactly one -gencode (sm_103a); the binding loads that file
    assert ba_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.samefile(ba.LIB_PATH, LIB)


def test_num_edges_and_status_strings():
    assert ba.ba_num_edges(10**6, 4, 0) == 4 * 10**6
    assert ba.ba_num_edges(2**27, 16) == 2**31
    assert ba.ba_num_edges(10**10, 100) == 10**12
    assert ba.ba_num_edges(10, 3, 4) == 6 + 18
    assert ba.ba_num_edges(10, 0, 0) == 0
    assert ba.ba_num_edges(10, 1, 11) == 0
    assert ba.ba_num_edges(2**62 + 1, 1, 0) == 0
    assert ba.ba_status_string(0) == "ok"
    assert ba.ba_status_string(2).startswith("edge range")
    assert ba.ba_version() >= 10000


@pytest.mark.parametrize("args,status", [
    ((1, 10, 0, 0, 0, 1), ba.BA_ERR_INVALID_ARG),        # d = 0
    ((1, 0, 1, 0, 0, 0), ba.BA_ERR_INVALID_ARG),         # n = 0
    ((1, 10, 1, 11, 0, 1), ba.BA_ERR_INVALID_ARG),       # n0 > n
    ((1, 10, 1, 0, 0, 11), ba.BA_ERR_RANGE),             # end > m
    ((1, 10, 1, 0, 5, 4), ba.BA_ERR_RANGE),              # begin > end
    ((1, 2**62, 2, 0, 0, 1), ba.BA_ERR_OVERFLOW),        # m > 2^62
])
def test_generate_rejects_bad_arguments_before_any_launch(args, status):
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges(*args, out=0x1000, stream=0)
    assert e.value.status == status


def test_generate_rejects_null_or_misaligned_output_and_accepts_empty_range():
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges(1, 10, 1, 0, 0, 5, out=None, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges(1, 10, 1, 0, 0, 5, out=0x1008, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    ba.ba_generate_edges(1, 10, 1, 0, 3, 3, out=None, stream=0)   # empty: no launch, OK


def test_degree_count_argument_rules():
    with pytest.raises(ba.BAError) as e:
        ba.ba_degree_count_range(1, 10, 1, 0, 0, 11, 5, counts=0x1000, stream=0)
    assert e.value.status == ba.BA_ERR_RANGE
    with pytest.raises(ba.BAError) as e:
        ba.ba_degree_count_range(1, 10, 1, 0, 0, 10, 5, counts=0x1004, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    ba.ba_degree_count(1, 10, 1, 0, counts=None, stream=0)          # node_limit 0: no-op


def test_variant_argument_rules():
    V = ba.BA_VARIANT_NO_SELF_LOOPS
    for n0 in (0, 1):                      # the self-loop-free rule needs a seed edge
        with pytest.raises(ba.BAError) as e:
            ba.ba_generate_edges_variant(1, 10, 2, n0, 0, 5, V, out=0x1000, stream=0)
        assert e.value.status == ba.BA_ERR_INVALID_ARG
        with pytest.raises(ba.BAError) as e:
            ba.ba_degree_count_variant(1, 10, 2, n0, 0, 5, 8, V, counts=0x1000, stream=0)
        assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:   # unknown flag
        ba.ba_generate_edges_variant(1, 10, 2, 3, 0, 5, 8, out=0x1000, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    P = ba.BA_VARIANT_NO_PARALLEL_EDGES
    for d, v in ((1025, P), (2, P | ba.BA_VARIANT_CRC_HASH)):  # d <= 1024, SplitMix64 only
        with pytest.raises(ba.BAError) as e:
            ba.ba_generate_edges_variant(1, 10, d, 3, 0, 5, v, out=0x1000, stream=0)
        assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:   # the same limits for a degree count
        ba.ba_degree_count_variant(1, 10, 1025, 3, 0, 5, 8, P, counts=0x1000, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges_variant(1, 10, 2, 3, 0, 99, ba.BA_VARIANT_CRC_HASH, out=0x1000,
                                     stream=0)
    assert e.value.status == ba.BA_ERR_RANGE
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges_variant(1, 10, 2, 3, 0, 5, 3, out=0x1008, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    ba.ba_generate_edges_variant(1, 10, 2, 3, 4, 4, 3, out=None, stream=0)    # empty: OK
    ba.ba_degree_count_variant(1, 10, 2, 3, 0, 5, 0, 3, counts=None, stream=0)  # no counts


def test_default_shapes_leave_room_for_resident_warps():
    """The untuned shapes per position width: the staging rings (1024 positions per warp)
    and the degree count's hit buffers (512 per warp) plus its 8-byte bins must let at
    least 24 warps stay resident on an SM's 227 KB (8-byte rings allow 28 at most).  Asked
    in a fresh process so that no tuner cache loaded by another test shadows the defaults."""
    import json
    import subprocess
    import sys
    code = ("import json; from paper_1602_07106_gb300 import ba; "
            "print(json.dumps([ba.ba_get_tuning(k, e) for k in (0, 1, 2) for e in (2**31, 2**40)]))")
    env = {k: v for k, v in os.environ.items() if k != "BA_TUNE_CACHE"}
    out = subprocess.run([sys.executable, "-c", code], env=env, check=True, capture_output=True,
                         text=True, cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    shapes = json.loads(out.stdout.strip().splitlines()[-1])
    smem_sm = 227 * 1024
    for (kind, pos_bytes), s in zip([(k, w) for k in (0, 1, 2) for w in (4, 8)], shapes):
        warps = s["block"] // 32
        per_cta = warps * 1024 * pos_bytes if kind != 1 else \
            warps * 512 * pos_bytes + 8 * s["hist_bins"]
        resident = min(s["ctas_per_sm"], smem_sm // per_cta) * warps
        assert resident >= 24, (kind, pos_bytes, s)
    g32, g64, d32, d64 = shapes[0], shapes[1], shapes[2], shapes[3]
    assert d64["ctas_per_sm"] < d32["ctas_per_sm"] and g64["block"] < g32["block"]


def test_tuning_overrides_validate_and_round_trip(tmp_path):
    default = ba.ba_get_tuning(ba.BA_KIND_GENERATE)
    assert default["block"] % 32 == 0 and default["tile"] & (default["tile"] - 1) == 0
    for bad in ({"block": 100, "refill": 1}, {"tile": 100, "refill": 1}, {"refill": 3},
                {"block": 2048, "refill": 1}, {"refill": 1, "hist_agg": 2},
                {"refill": 1, "chains": 3}):
        with pytest.raises(ba.BAError):
            ba.ba_set_tuning(ba.BA_KIND_GENERATE, bad)
    ba.ba_set_tuning(ba.BA_KIND_GENERATE, {"block": 128, "ctas_per_sm": 8, "tile": 1024,
                                           "refill": 1})
    assert ba.ba_get_tuning(ba.BA_KIND_GENERATE)["tile"] == 1024
    ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)
    assert ba.ba_get_tuning(ba.BA_KIND_GENERATE) == default
    path = tmp_path / "tune.json"
    path.write_text('{"sm_count": 152, "entries": [\n  {"kind": 1, "r32": 0, "block": 256, '
                    '"ctas_per_sm": 4, "tile": 256, "refill": 1, "hist_bins": 8192, "hist_agg": 1}\n]}\n')
    ba.ba_tune_load(str(path))
    assert ba.ba_get_tuning(ba.BA_KIND_DEGREE, 2**40)["hist_bins"] == 8192
    assert ba.ba_get_tuning(ba.BA_KIND_DEGREE, 2**40)["hist_agg"] == 1
    assert ba.ba_get_tuning(ba.BA_KIND_DEGREE, 2**40)["chains"] == 1   # entry without "chains"
    out = tmp_path / "saved.json"
    ba.ba_tune_save(str(out))
    assert '"hist_bins": 8192' in out.read_text() and '"chains": 1' in out.read_text()
    ba.ba_set_tuning(ba.BA_KIND_GENERATE, {"refill": 1, "chains": 2})
    assert ba.ba_get_tuning(ba.BA_KIND_GENERATE)["chains"] == 2
    ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)
    with pytest.raises(ba.BAError):
        ba.ba_tune_load(str(tmp_path / "missing.json"))


def test_offsets_need_one_entry_per_graph_plus_one():
    graphs = [(1, 10, 1, 0, 0, 5), (2, 10, 1, 0, 0, 5)]
    for fn in (ba.ba_generate_batch, ba.ba_generate_batch_noalloc):
        with pytest.raises(ValueError):
            fn(graphs, out=0x1000, offsets=[0, 5], stream=0)      # G + 1 = 3 needed
    with pytest.raises(ValueError):
        ba.ba_batch_plan_create(graphs, offsets=[0, 5, 10, 15])
    assert ba.ba_device_allocations() >= 0


def test_checked_launch_argument_rules():
    with pytest.raises(ba.BAError) as e:
        ba.ba_check_status(None, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:                       # no status word
        ba.ba_generate_edges_checked(1, 10, 2, 0, 0, 5, 0x1000, 5, None, stream=0)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:                       # range beyond m, checked first
        ba.ba_generate_edges_checked(1, 10, 2, 0, 0, 21, 0x1000, 21, 0x2000, stream=0)
    assert e.value.status == ba.BA_ERR_RANGE


def test_chain_lengths_argument_rules():
    for bins, hist in ((1, 0x1000), (1025, 0x1000), (8, None), (8, 0x1004)):
        with pytest.raises(ba.BAError) as e:
            ba.ba_chain_lengths(1, 10, 2, 0, 0, 5, bins, hist, stream=0)
        assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_chain_lengths(1, 10, 2, 0, 0, 21, 8, 0x1000, stream=0)
    assert e.value.status == ba.BA_ERR_RANGE


def test_server_calls_reject_a_null_server():
    for call in (lambda: ba.ba_server_cancel(None, 1), lambda: ba.ba_server_release(None, 1)):
        with pytest.raises(ba.BAError) as e:
            call()
        assert e.value.status == ba.BA_ERR_INVALID_ARG


def test_probe_argument_rules():
    with pytest.raises(ba.BAError) as e:
        ba.ba_probe_hash(1, 0, 100, 1, None, stream=0)                 # no sink
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_probe_hash(1, 0, 100, 3, 0x1000, stream=0)               # chains 3
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_probe_hash(1, 2**60, 100, 1, 0x1000, stream=0)           # past 2^60
    assert e.value.status == ba.BA_ERR_RANGE
    ba.ba_probe_hash(1, 0, 0, 1, 0x1000, stream=0)                     # nothing to do
    for dst, n in ((0x1008, 64), (0x1000, 40), (None, 64)):
        with pytest.raises(ba.BAError) as e:
            ba.ba_probe_write(dst, n, stream=0)
        assert e.value.status == ba.BA_ERR_INVALID_ARG
    ba.ba_probe_write(None, 0, stream=0)                               # nothing to do


def test_batch_and_server_argument_rules():
    with pytest.raises(ba.BAError) as e:
        ba.ba_batch_plan_create([(1, 10, 0, 0, 0, 5)])                  # d = 0
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_batch([(1, 10, 1, 0, 0, 11)], out=0x1000, stream=0)
    assert e.value.status == ba.BA_ERR_RANGE
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_batch([(1, 10, 1, 0, 0, 5), (2, 10, 1, 0, 0, 5)], out=0x1000,
                             offsets=[0, 4, 9], stream=0)               # graph 0 does not fit
    assert e.value.status == ba.BA_ERR_INVALID_ARG
    ba.ba_generate_batch([], out=None, stream=0)                         # nothing to do
    for bad in ({"max_active": 65537}, {"max_inflight_ticks": 65}, {"max_queued": -1}):
        with pytest.raises(ba.BAError) as e:                             # before any CUDA call
            ba.ba_server_create(**bad)
        assert e.value.status == ba.BA_ERR_INVALID_ARG, bad
