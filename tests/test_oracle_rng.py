"""Pins for the oracle's random-number path (Section 2.2: every event gets its
own group of pseudo-random numbers, whatever the thread count).

Philox4x32-10 is checked against an independent implementation (the one in
the Triton library, run by its CPU interpreter in a subprocess); the
uniform -> bin map is checked by exact integer arithmetic in Python.
"""
import json
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c_ptr, key_ptr, out_ptr, n, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
    seed = tl.load(key_ptr)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a, mask=m)
    tl.store(out_ptr + 4 * i + 1, b, mask=m)
    tl.store(out_ptr + 4 * i + 2, c, mask=m)
    tl.store(out_ptr + 4 * i + 3, d, mask=m)

cases = json.loads(sys.stdin.read())
res = []
for ctr, key in cases:
    c = torch.from_numpy(np.array(ctr, dtype=np.uint32).view(np.int32).copy())
    seed = (key[1] << 32) | key[0]
    if seed >= 1 << 63:
        seed -= 1 << 64
    kk = torch.tensor([seed], dtype=torch.int64)
    out = torch.zeros(4, dtype=torch.int32)
    k[(1,)](c, kk, out, 1, BLOCK=2)
    res.append([int(v) for v in out.numpy().view(np.uint32)])
print(json.dumps(res))
"""


def _triton_philox(cases):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_philox_matches_independent_implementation(oracle_mod):
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xFFFFFFFF] * 4, [0xFFFFFFFF, 0xFFFFFFFF])]
    for _ in range(40):
        cases.append(([int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)],
                      [int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)]))
    # the counter layout used for events: (event lo, event hi, iteration, batch<<8|j)
    seed = 1234
    for ev, it, batch, j in [(0, 0, 0, 0), (5, 3, 0, 1), (2**32 + 17, 9, 63, 2), (123456789, 1, 7, 3)]:
        cases.append(([ev & 0xFFFFFFFF, ev >> 32, it, (batch << 8) | j], [seed & 0xFFFFFFFF, seed >> 32]))
    ref = _triton_philox(cases)
    for (ctr, key), want in zip(cases, ref):
        got = oracle_mod.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want, (ctr, key)


def test_event_words_layout(oracle_mod):
    """Word 4j+k of an event is word k of Philox block j."""
    seed, it, batch = 0x1234_5678_9ABC_DEF0, 11, 5
    for ev in (0, 1, 4095, 2**33 + 3):
        w = oracle_mod.event_words(seed, it, batch, ev, 13)
        for j in range(4):
            blk = oracle_mod.philox4x32_10(
                [ev & 0xFFFFFFFF, ev >> 32, it, (batch << 8) | j],
                [seed & 0xFFFFFFFF, seed >> 32])
            for k in range(4):
                if 4 * j + k < 13:
                    assert w[4 * j + k] == blk[k]
    # distinct events, iterations and batches give distinct groups
    a = oracle_mod.event_words(1234, 0, 0, 10, 4)
    assert not np.array_equal(a, oracle_mod.event_words(1234, 1, 0, 10, 4))
    assert not np.array_equal(a, oracle_mod.event_words(1234, 0, 1, 10, 4))
    assert not np.array_equal(a, oracle_mod.event_words(1234, 0, 0, 11, 4))


@pytest.mark.parametrize("nbins", [2, 3, 7, 50, 100, 1000, 1024])
def test_bin_map_boundaries_exact(oracle_mod, nbins):
    """Bin i holds exactly the words r with i*2^32 <= r*N < (i+1)*2^32."""
    for i in range(nbins):
        lo = -((-i * 2**32) // nbins)  # ceil(i 2^32 / N): first word of bin i
        b, f = oracle_mod.bin_map(lo, nbins)
        assert b == i
        assert Fraction(f) == Fraction((lo * nbins) % 2**32) / 2**32 + Fraction(1, 2**33)
        if i > 0:
            b, f = oracle_mod.bin_map(lo - 1, nbins)
            assert b == i - 1
    b, f = oracle_mod.bin_map(2**32 - 1, nbins)
    assert b == nbins - 1 and 0.0 < f < 1.0


def test_bin_map_subsampled_brute_force(oracle_mod):
    """N = 3 over a 2^16-spaced subsample of all words (plus offsets)."""
    nbins = 3
    counts = np.zeros(nbins, int)
    for r in list(range(0, 2**32, 2**16)) + [2**32 - 1, 1, 2**31, 1431655765, 1431655766]:
        b, f = oracle_mod.bin_map(r, nbins)
        assert b == (r * nbins) >> 32
        assert 0.0 < f < 1.0
        assert abs(f - (((r * nbins) % 2**32) + 0.5) / 2**32) == 0.0
        counts[b] += 1
    assert abs(counts[0] - counts[2]) <= 3


def test_grid_map_preserves_integrals(oracle_mod):
    """Importance-sampling identity of the adaptive map: averaging J(u) h(x(u))
    over all words u equals int_0^1 h(x) dx for any grid.  With the bins
    aligned to the sampling cells, a midpoint sum over the words integrates
    each bin's linear piece exactly for linear h, and to O(cell^2) for cubic h."""
    rng = np.random.default_rng(3)
    nbins = 8
    cuts = np.sort(rng.uniform(0, 1, nbins - 1))
    edges = np.concatenate([[0.0], cuts, [1.0]])
    M = 2**14
    acc_lin = acc_cub = 0.0
    for k in range(M):
        r = (k * 2**32) // M + 2**32 // (2 * M)
        x, jac = oracle_mod.grid_map(edges, nbins, r)
        assert 0.0 < x < 1.0
        acc_lin += jac * (3.0 * x + 1.0)
        acc_cub += jac * (x ** 3 - 2.0 * x)
    # the half-word offset of f shifts x by 2^-33 of a bin width: < 1e-9 here
    assert abs(acc_lin / M - 2.5) < 1e-9
    assert abs(acc_cub / M - (0.25 - 1.0)) < 1e-6
