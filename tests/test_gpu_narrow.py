"""GPU parity of ba_generate_edges32 (32-bit node IDs, 8 bytes per edge): the same values as
the oracle's int64 edges, on both position paths, with seed cliques, ragged tails and every
launch shape."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parallel as opar
from paper_1602_07106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu32(ba, seed, n, d, n0, a, b):
    out = torch.full((b - a, 2), -1, dtype=torch.int32, device="cuda")
    ba.ba_generate_edges32(seed, n, d, n0, a, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64)


CASES = [(1, 10**6, 4, 0, 0, 4 * 10**6), (3, 5000, 3, 0, 17, 14_983), (13, 1000, 4, 5, 0, 3990),
         (17, 500, 32, 33, 0, 528 + 467 * 32), (19, 200, 5, 1, 0, 995),
         (77, 2**29, 16, 0, 2**33 - 300_000, 2**33),            # 64-bit positions
         (79, 2**31, 2, 0, 2**32 - 5000, 2**32),                # node IDs up to 2^31 - 1
         (81, 2**29, 13, 0, 13 * 2**29 - 100_000, 13 * 2**29),  # 64-bit, d not a power of 2
         (83, 2**28, 24, 25, 300 + (2**28 - 25) * 24 - 100_000, 300 + (2**28 - 25) * 24)]


@pytest.mark.parametrize("seed,n,d,n0,a,b", CASES)
def test_int32_edges_match_oracle(ba, seed, n, d, n0, a, b):
    np.testing.assert_array_equal(_gpu32(ba, seed, n, d, n0, a, b),
                                  opar.edges_range(seed, n, d, n0, a, b))


@pytest.mark.parametrize("shape", [{"refill": 0, "block": 256, "ctas_per_sm": 8},
                                   {"refill": 1, "block": 64, "ctas_per_sm": 8, "tile": 64},
                                   {"refill": 1, "block": 256, "ctas_per_sm": 1, "tile": 2048},
                                   {"refill": 1, "block": 128, "ctas_per_sm": 2, "tile": 256,
                                    "chains": 2}])
def test_int32_output_does_not_depend_on_shape(ba, shape):
    try:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, shape)
        np.testing.assert_array_equal(_gpu32(ba, 31, 300_000, 3, 0, 5, 899_999),
                                      oracle.edges_range(31, 300_000, 3, 0, 5, 899_999))
    finally:
        ba.ba_set_tuning(ba.BA_KIND_GENERATE, None)


@pytest.mark.parametrize("seed,n,d,a,b", [(41, 10**6, 16, 3, 3_000_000),   # d = 2^4
                                           (43, 10**6, 12, 0, 2_500_001)])  # d not 2^l
def test_int32_output_8_byte_aligned_only(ba, seed, n, d, a, b):
    # The int32 entry point asks only for 8-byte alignment: an output 8 bytes past a
    # 16-byte boundary gives the same edges as an aligned one, and the oracle's.
    want = opar.edges_range(seed, n, d, 0, a, b)
    buf = torch.full((b - a + 1, 2), -1, dtype=torch.int32, device="cuda")
    for off in (0, 1):                      # byte offset 0 or 8 from a 16-byte boundary
        assert (buf.data_ptr() + 8 * off) % 16 == 8 * off
        view = buf[off:off + b - a]
        ba.ba_generate_edges32(seed, n, d, 0, a, b, view)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(view.cpu().numpy().astype(np.int64), want)


def test_int32_equals_int64_on_the_large_workload(ba):
    g = W.PLAIN_LARGE
    half = 2**30
    o32 = torch.empty((half, 2), dtype=torch.int32, device="cuda")
    o64 = torch.empty((half, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges32(g.seed, g.n, g.d, 0, half, g.m, o32)
    ba.ba_generate_edges(g.seed, g.n, g.d, 0, half, g.m, o64)
    torch.cuda.synchronize()
    assert torch.equal(o32.to(torch.int64), o64)


def test_int32_rejects_graphs_with_ids_beyond_2_31(ba):
    out = torch.empty((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ba.BAError) as e:
        ba.ba_generate_edges32(1, 2**31 + 1, 1, 0, 0, 4, out)
    assert e.value.status == ba.BA_ERR_INVALID_ARG
