"""cdr_eval_predicates_noalloc against cdr_eval_predicates (needs a GPU).

The no-allocation entry point serves callers that cannot allocate device memory:
code that keeps kernels running on other streams, where cudaFree would wait for
the whole device, and processes whose device memory is held by a caching
allocator, where cudaMalloc can fail. It stages data in one fixed array of the
library instead. These checks call it through the C-ABI twice in a row, with
the second batch shorter than the first, so that what the first call left in
the shared array cannot leak into the second. Every kind must give the signs
and points of the allocating entry point, bit for bit (both run the same
formulas). They also check the size limit.

This file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


def _batch(rng, n):
    """Random, integer-grid (degenerate: exact paths) and 1-ulp-perturbed items."""
    it = np.zeros((n, 16))
    for i in range(n):
        k = i % 3
        if k == 0:
            P = rng.uniform(0, 1000, size=(5, 3))
        elif k == 1:
            P = rng.integers(-2, 3, size=(5, 3)).astype(np.float64)
        else:
            P = rng.integers(-2, 3, size=(5, 3)).astype(np.float64) * 0.1 + 0.3
            j, c = rng.integers(0, 5), rng.integers(0, 3)
            P[j, c] = np.nextafter(P[j, c], np.inf if rng.random() < 0.5 else -np.inf)
        it[i, :15] = P.reshape(-1)
    return it


def _same(a, b):
    return np.array_equal(a, b, equal_nan=True)


def test_noalloc_matches_allocating_entry_point(cdr):
    rng = np.random.default_rng(2024)
    first, second = _batch(rng, 3000), _batch(rng, 1100)
    for kind in range(12):
        f, s = first.copy(), second.copy()
        if kind == 7:  # the bound B of the bad-tetrahedron test
            f[:, 12] = 1.4
            s[:, 12] = 1.4
        sg1, pt1 = cdr.eval_predicates_noalloc(kind, f)
        sg2, pt2 = cdr.eval_predicates_noalloc(kind, s)
        rs1, rp1 = cdr.eval_predicates(kind, f)
        rs2, rp2 = cdr.eval_predicates(kind, s)
        assert np.array_equal(sg1, rs1), kind
        assert np.array_equal(sg2, rs2), kind
        assert _same(pt1, rp1), kind
        assert _same(pt2, rp2), kind


def test_noalloc_full_capacity_and_limit(cdr):
    rng = np.random.default_rng(2025)
    n = cdr.EVAL_NOALLOC_MAX_ITEMS
    items = rng.uniform(-1, 1, size=(n, 16))
    for _ in range(2):
        s_na, _ = cdr.eval_predicates_noalloc("insphere", items)
        s_ref, _ = cdr.eval_predicates("insphere", items)
        assert np.array_equal(s_na, s_ref)
    big = np.zeros((n + 1, 16))
    with pytest.raises(cdr.CdrError, match="at most %d" % n) as e:
        cdr.eval_predicates_noalloc("orient", big)
    assert e.value.status == -6
    # an empty batch is a no-op
    s0, p0 = cdr.eval_predicates_noalloc("orient", np.zeros((0, 16)))
    assert s0.shape == (0,) and p0.shape == (0, 3)


def test_noalloc_neither_allocates_nor_waits_for_other_streams(cdr):
    """What the entry point is for: while another stream is busy, a call on a
    stream of its own returns before that work ends (a cudaFree inside it would
    wait for the whole device), and the device's free memory does not move."""
    import torch
    rng = np.random.default_rng(2026)
    items = _batch(rng, 512)
    ref, _ = cdr.eval_predicates("orient", items)
    cdr.eval_predicates_noalloc("orient", items)  # loads the module on a fresh process
    torch.cuda.synchronize()
    busy, mine = torch.cuda.Stream(), torch.cuda.Stream()
    done = torch.cuda.Event()
    free_before = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(busy):
        torch.cuda._sleep(int(4e8))  # one thread spinning ~0.2 s at 2 GHz
        done.record(busy)
    sg, _ = cdr.eval_predicates_noalloc("orient", items, stream=mine)
    overlapped = not done.query()
    free_after = torch.cuda.mem_get_info()[0]
    torch.cuda.synchronize()
    assert overlapped, "the call waited for work on another stream"
    assert free_after == free_before
    assert np.array_equal(sg, ref)
