"""The no-allocation Philox entry point (requires a GB300): through the
library's fixed device buffer it returns the same words as the allocating
entry point, on consecutive calls, and refuses requests beyond the buffer.
Named to be collected last, so it also runs after every other test."""
import numpy as np
import pytest

from paper_1503_06182_gb300 import vegas as v

pytestmark = pytest.mark.gpu


def test_noalloc_words_equal_allocating_entry_point_on_consecutive_calls():
    v.vegas_rng_words_noalloc(1, 0, 0, 0, 0, 4)  # set-up only
    cases = [
        (1234, 3, 0, 0, 4096, 4),
        (2**63 + 5, 7, 3, 2**32 - 100, 5000, 13),
        (99, 2**31, 63, 10**9, v.VEGAS_NOALLOC_MAX_WORDS // 16, 16),  # the whole buffer
    ]
    for args in cases:
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
