"""skr_sort_noalloc, the sort entry point that allocates no device memory.

It serves callers that may not let a library allocate (an application that
owns all device memory through its own pool, or a latency-bound loop where
cudaMalloc/cudaFree would synchronise the device).  Its scratch is a fixed
array that the library keeps on every device, shared by all calls; this
file runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skr():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2401_09516_gb300 as m
    return m


def test_noalloc_sort_matches_allocating_sort_on_two_calls_in_a_row(skr):
    rng = np.random.default_rng(2024)
    # first call: a large N with real-valued parameters; second call: a
    # smaller N with many exact ties, so stale scratch from the first call
    # (distances, placed flags) would change the answer if it leaked through
    P1 = torch.tensor(rng.standard_normal((300, 2048)), device="cuda:0")
    P2 = torch.tensor(rng.integers(-2, 3, size=(41, 9)).astype(np.float64), device="cuda:0")
    from oracle import sort as osort
    for P, start in ((P1, 0), (P2, 7)):
        want = skr.skr_sort(P, start=start).cpu().numpy()
        got = skr.skr_sort_noalloc(P, start=start).cpu().numpy()
        np.testing.assert_array_equal(got, want)
        assert sorted(got.tolist()) == list(range(P.shape[0]))
        # and directly against the oracle's Algorithm 1
        assert got.tolist() == osort.greedy_sort(P.cpu().numpy(), start)


def test_noalloc_sort_rejects_oversize_and_host_input(skr):
    too_big = torch.zeros((skr._native.SKR_SORT_NOALLOC_MAX_N + 1, 3), dtype=torch.float64,
                          device="cuda:0")
    with pytest.raises(skr.SkrError) as e:
        skr.skr_sort_noalloc(too_big)
    assert "SKR_SORT_NOALLOC_MAX_N" in str(e.value)
    with pytest.raises(ValueError):
        skr.skr_sort_noalloc(np.zeros((4, 3)))
    # the entry point still works after the rejected calls
    P = torch.tensor(np.arange(12.0).reshape(6, 2)[::-1].copy(), device="cuda:0")
    np.testing.assert_array_equal(skr.skr_sort_noalloc(P).cpu().numpy(),
                                  skr.skr_sort(P).cpu().numpy())
