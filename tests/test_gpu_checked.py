"""GPU tests of the checked launch (ba_generate_edges_checked + ba_check_status), the
library's debug aid while no sanitizer runs on this pool: every output store is compared
with a capacity the caller states.  A capacity smaller than the range makes the check fire
-- the output buffer is allocated larger than that capacity, so no access ever leaves it,
and the test checks that the slots beyond the capacity were not written."""
import pytest
import torch

pytestmark = pytest.mark.gpu

CASES = [(1, 10**6, 4, 0, 0, 4 * 10**6), (3, 50_000, 6, 7, 5, 21 + 49_993 * 6),
         (5, 2**29, 16, 0, 2**33 - 300_000, 2**33)]


def _plain(ba, seed, n, d, n0, a, b):
    out = torch.empty((b - a, 2), dtype=torch.int64, device="cuda")
    ba.ba_generate_edges(seed, n, d, n0, a, b, out)
    return out


@pytest.mark.parametrize("seed,n,d,n0,a,b", CASES)
def test_enough_capacity_is_clean_and_bit_identical(ba, seed, n, d, n0, a, b):
    out = torch.full((b - a, 2), -7, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_checked(seed, n, d, n0, a, b, out, b - a, status)
    ba.ba_check_status(status)
    assert torch.equal(out, _plain(ba, seed, n, d, n0, a, b))


@pytest.mark.parametrize("seed,n,d,n0,a,b", CASES)
def test_short_capacity_fires_and_writes_nothing_beyond(ba, seed, n, d, n0, a, b):
    cap = (b - a) * 3 // 5 + 1
    out = torch.full((b - a, 2), -7, dtype=torch.int64, device="cuda")   # room for all
    status = torch.zeros(1, dtype=torch.int64, device="cuda")
    ba.ba_generate_edges_checked(seed, n, d, n0, a, b, out, cap, status)
    with pytest.raises(ba.BAError) as e:
        ba.ba_check_status(status)
    assert e.value.status == ba.BA_ERR_CUDA and str(cap) in str(e.value)
    assert int(status.item()) == cap                  # the first slot past the capacity
    want = _plain(ba, seed, n, d, n0, a, b)
    assert torch.equal(out[:cap], want[:cap])
    assert bool((out[cap:] == -7).all())              # every store beyond it was skipped
    # the status word is reset by the next call
    ba.ba_generate_edges_checked(seed, n, d, n0, a, b, out, b - a, status)
    ba.ba_check_status(status)
    assert torch.equal(out, want)
