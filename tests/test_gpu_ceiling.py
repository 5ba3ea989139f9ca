"""The gather-rate diagnostic (pr_measure_gather_rate): it makes exactly the loads it
reports, at a positive rate, and loads that bypass L1 are not faster than a bound the
part cannot exceed (one 4-byte load per SM-cycle per SM, at the highest clock)."""
import pytest

pr = pytest.importorskip("paper_2109_09527_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


@pytest.mark.parametrize("cached", [0, 1])
@pytest.mark.parametrize("blocks_per_sm", [1, 4, 8])
def test_gather_rate_counts_and_bounds(cached, blocks_per_sm):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    chunks = 64
    r = pr.pr_measure_gather_rate(1 << 22, 1 << 20, cached, blocks_per_sm, chunks, seed=7)
    assert r["gathers"] == sms * blocks_per_sm * 256 * 16 * chunks
    assert r["ms"] > 0
    assert r["gathers_per_s"] == pytest.approx(r["gathers"] / (r["ms"] * 1e-3), rel=1e-9)
    if not cached:
        # at most a few loads per SM-cycle at 2.1 GHz: far above it, the loads were not made
        assert r["gathers_per_s"] < 4.0 * sms * 2.1e9


def test_gather_rate_small_vector_and_one_warp_of_chunks():
    # a vector of one element (every index 0) and the minimum index array
    r = pr.pr_measure_gather_rate(1, 1024, 0, 1, 1, seed=0)
    assert r["gathers"] > 0 and r["ms"] > 0
