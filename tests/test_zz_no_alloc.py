"""sbd_sort_strings_noalloc: string ingestion without any device allocation.

The entry point serves callers that cannot let a library allocate device
memory for them (memory carved up in advance by their own allocator, plug-ins
that must not grow the host process's footprint).  Its output must be the
same as the allocating path's -- sbd_create followed by sbd_sorted_strings --
bit for bit, call after call, although every call reuses the same fixed work
space inside the library.
"""
import numpy as np
import pytest

from paper_2601_16637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_16637_gb300 import binding, build

    build.build()
    binding.load()
    return torch, binding


def _reference_sorted(binding, norb, nel, strings):
    # the allocating path: sbd_create sorts the alpha strings; a one-string beta set
    one = np.array([1], dtype=np.uint64)
    with binding.SBD(norb, nel, 1, np.zeros((norb, norb)), np.zeros((norb,) * 4), strings, one,
                     allocator="cuda") as g:
        return g.sorted_strings(0)


def test_noalloc_sort_matches_allocating_path_on_consecutive_calls(env):
    torch, B = env
    rng = np.random.default_rng(4)
    sets = [(40, 13, W.gumbel_top_k(40, 13, 50000, 0.1, rng)),     # many sort tiles, 5 radix digits
            (16, 5, W.config("cfg2").A),                           # the 2,000-string set
            (64, 3, W.gumbel_top_k(64, 3, 777, 0.05, rng))]       # bit 63 in use, ragged size
    refs = [_reference_sorted(B, norb, nel, s) for norb, nel, s in sets]
    # two calls in a row on the same set, then the other sets, then the first again:
    # the shared work space must not carry anything from one call into the next
    order = [0, 0, 1, 2, 0]
    for i in order:
        norb, nel, s = sets[i]
        keys = torch.from_numpy(s.view(np.int64)).cuda()
        out = torch.full_like(keys, -1)
        rc, bad = B.sbd_sort_strings_noalloc(keys, norb, nel, out)
        assert rc == 0 and bad == -1
        assert np.array_equal(out.cpu().numpy().view(np.uint64), refs[i])


def test_noalloc_sort_reports_the_same_errors(env):
    torch, B = env
    wl = W.make("t", 12, 4, 4, 300, 300, 0.3, seed=3)
    dup = wl.A.copy()
    dup[17] = dup[200]
    bad = wl.A.copy()
    bad[41] = np.uint64(0b111)  # three electrons instead of four
    for strings, code in ((dup, -3), (bad, -2)):
        with pytest.raises(B.SbdError) as e:
            _reference_sorted(B, 12, 4, strings)
        assert e.value.code == code
        keys = torch.from_numpy(strings.view(np.int64)).cuda()
        out = torch.empty_like(keys)
        for _ in range(2):
            rc, idx = B.sbd_sort_strings_noalloc(keys, 12, 4, out)
            assert rc == code
            if code == -2:
                assert idx == 41
            else:
                srt = np.sort(strings)
                assert srt[idx] == srt[idx - 1]
    # a clean call after the failing ones
    keys = torch.from_numpy(wl.A.view(np.int64)).cuda()
    out = torch.empty_like(keys)
    rc, idx = B.sbd_sort_strings_noalloc(keys, 12, 4, out)
    assert rc == 0 and idx == -1
    assert np.array_equal(out.cpu().numpy().view(np.uint64), np.sort(wl.A))


def test_noalloc_sort_rejects_sets_beyond_its_work_space(env):
    torch, B = env
    n = B.SBD_NOALLOC_MAX_STRINGS + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty_like(keys)
    with pytest.raises(B.SbdError) as e:
        B.sbd_sort_strings_noalloc(keys, 30, 3, out)
    assert e.value.code == -1
    assert "65536" in B.sbd_last_error()
    # empty input is a no-op
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    rc, idx = B.sbd_sort_strings_noalloc(empty, 30, 3, empty)
    assert rc == 0 and idx == -1
