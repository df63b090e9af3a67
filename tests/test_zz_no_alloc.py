"""The no-allocation Philox entry point (requires a GB300).

vegas_rng_words_noalloc serves callers that cannot allocate device memory
(a process whose memory a caching allocator holds, or code that cannot take
cudaFree's synchronisation).  Through the library's fixed device buffer it
returns the same words as the allocating entry point, on consecutive calls;
it refuses requests beyond the buffer; and once set up, its calls leave the
device's free memory unchanged.  Named to be collected last, so it also runs
after every other test.
"""
import numpy as np
import pytest

from paper_1503_06182_gb300 import vegas as v

pytestmark = pytest.mark.gpu

CASES = [
    (1234, 3, 0, 0, 4096, 4),
    (2**63 + 5, 7, 3, 2**32 - 100, 5000, 13),
    (99, 2**31, 63, 10**9, v.VEGAS_NOALLOC_MAX_WORDS // 16, 16),  # the whole buffer
]


def test_noalloc_words_equal_allocating_entry_point_on_consecutive_calls():
    v.vegas_rng_words_noalloc(1, 0, 0, 0, 0, 4)  # set-up only
    for args in CASES:
        got = v.vegas_rng_words_noalloc(*args)
        again = v.vegas_rng_words_noalloc(*args)
        want = v.vegas_rng_words(*args)
        assert np.array_equal(got, want), args
        assert np.array_equal(again, want), args


def test_noalloc_refuses_requests_beyond_the_buffer():
    n = v.VEGAS_NOALLOC_MAX_WORDS // 4 + 1
    with pytest.raises(v.VegasError, match="exceeds the fixed buffer"):
        v.vegas_rng_words_noalloc(1, 0, 0, 0, n, 4)
    # a refused call leaves the buffer usable
    assert np.array_equal(v.vegas_rng_words_noalloc(5, 1, 0, 7, 100, 4),
                          v.vegas_rng_words(5, 1, 0, 7, 100, 4))


def test_noalloc_calls_leave_free_device_memory_unchanged():
    torch = pytest.importorskip("torch")
    v.vegas_rng_words_noalloc(1, 0, 0, 0, 0, 4)  # set-up
    v.vegas_rng_words_noalloc(*CASES[0])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    outs = [v.vegas_rng_words_noalloc(*args) for args in CASES for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.array_equal(outs[0], outs[1])
