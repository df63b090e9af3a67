"""Pins for the oracle's VEGAS+ (adaptive stratified sampling on the VEGAS map).

VEGAS+ (Lepage 2021) is a later form of the VEGAS method the paper cites
(Section 2.1).  Its pieces are pinned from outside the stage: the strata
count and the stratified word by their integer definitions and densities,
the allocation weight against v^(beta/2) and exact powers of two, the
allocation on hand values, a direct Python loop over the events built from
the already pinned Philox words, grid map and integrands, the reduction to
plain VEGAS with one stratum, unbiasedness against closed forms and
quadrature, and the variance reduction that is the method's purpose.
"""
import math

import numpy as np
import pytest

import refs
from paper_1503_06182_gb300.workloads import DY_PARAMS, GAUSS_PARAMS, GAUSS_SHIFTED_PARAMS


# ------------------------------------------------------------- strata
@pytest.mark.parametrize("ndim,ncall", [(1, 100), (2, 150), (2, 200_000), (4, 1_000_000),
                                        (5, 10_000_000), (13, 1_000_000), (3, 4 * 27)])
def test_plus_nstrat_is_the_largest_admissible(oracle_mod, ndim, ncall):
    s = oracle_mod.plus_nstrat(ndim, ncall)
    assert s >= 1
    assert 4 * s ** ndim <= ncall and s ** ndim <= 2 ** 22
    assert 4 * (s + 1) ** ndim > ncall or (s + 1) ** ndim > 2 ** 22


def test_plus_nstrat_capped(oracle_mod):
    s = oracle_mod.plus_nstrat(2, 10 ** 9)
    assert s == 2048  # 2048^2 = 2^22 hypercubes


def test_plus_word_lies_in_its_stratum_with_uniform_density(oracle_mod):
    """y = r'/2^32 stays inside [c/s, (c+1)/s], is non-decreasing in r, and
    consecutive words r hit each r' s times (uniform density), except at the
    ends of a stratum."""
    for s in (3, 7, 22, 1000):
        for c in (0, 1, s // 2, s - 1):
            lo = oracle_mod.plus_word(0, c, s)
            hi = oracle_mod.plus_word(2 ** 32 - 1, c, s)
            assert lo * s >= c * 2 ** 32 - s and lo * s <= c * 2 ** 32
            assert hi * s <= (c + 1) * 2 ** 32 and (hi + 1) * s > (c + 1) * 2 ** 32 - s
            r0 = 12345 * s
            ws = [oracle_mod.plus_word(r0 + i, c, s) for i in range(20 * s)]
            assert all(b >= a for a, b in zip(ws, ws[1:]))
            vals, counts = np.unique(ws, return_counts=True)
            assert np.all(counts[1:-1] == s)


# ------------------------------------------------------------- allocation
def test_plus_weight_matches_power(oracle_mod):
    rng = np.random.default_rng(5)
    for beta in (0.25, 0.5, 0.75, 1.0):
        for v in 10.0 ** rng.uniform(-300, 300, 200):
            w = oracle_mod.plus_weight(v, beta)
            want = math.exp(beta / 2 * math.log(v))
            assert abs(w - want) <= 5e-7 * want, (v, beta)
        # powers 2^(8q) go through exactly
        for q in (-40, -1, 0, 1, 37):
            assert oracle_mod.plus_weight(2.0 ** (8 * q), beta) == 2.0 ** (q * 4 * beta)
    assert oracle_mod.plus_weight(0.0, 0.75) == 0.0
    assert oracle_mod.plus_weight(7.0, 0.0) == 1.0 and oracle_mod.plus_weight(0.0, 0.0) == 1.0
    with pytest.raises(ValueError):
        oracle_mod.plus_weight(1.0, 0.3)


def test_plus_allocate_hand_values(oracle_mod):
    # beta = 1: d = sqrt(v) = 1, 2, 0, 4; D = 7; C = 75: 75 d / 7 = 10.7, 21.4, 0, 42.9
    n = oracle_mod.plus_allocate(75, [1.0, 4.0, 0.0, 16.0], beta=1.0)
    assert list(n) == [10, 21, 2, 42]
    # no variance anywhere: uniform floor(C / NH)
    assert list(oracle_mod.plus_allocate(75, [0.0] * 4)) == [18] * 4
    # beta = 0: every hypercube weighs the same
    assert list(oracle_mod.plus_allocate(75, [1.0, 4.0, 0.0, 16.0], beta=0.0)) == [18] * 4


# ------------------------------------------------------------- the stage
def test_plus_matches_direct_event_loop(oracle_mod):
    """One iteration on a non-uniform grid and a non-uniform allocation,
    rebuilt event by event in Python from the pinned pieces: Philox words,
    the stratified word in integer arithmetic, the grid map, the integrand."""
    nd, nb, ncall, seed, it = 2, 8, 600, 17, 3
    s = oracle_mod.plus_nstrat(nd, ncall)
    nh = s ** nd
    e = oracle_mod.uniform_edges(nd, nb)
    e[:, 1:-1] += 0.04 * np.cos(np.arange(1, nb))[None, :] / nb
    alloc = np.array([2 + (h * 7) % 5 for h in range(nh)], np.int32)
    r = oracle_mod.iterate_plus(nd, nb, seed, ncall, 1, oracle_mod.GAUSS, GAUSS_PARAMS, edges=e,
                                alloc=alloc, iteration=it, adapt=False)
    off = np.concatenate([[0], np.cumsum(alloc)])
    m, v, S1 = [], [], []
    dl = [[[] for _ in range(nb)] for _ in range(nd)]
    for h in range(nh):
        coords = [(h // s ** a) % s for a in range(nd)]
        fh = []
        for ev in range(off[h], off[h + 1]):
            words = oracle_mod.event_words(seed, it, 0, int(ev), nd)
            x, J, bins = [], 1.0, []
            for a in range(nd):
                rw = ((coords[a] << 32) + int(words[a])) // s
                xa, ja = oracle_mod.grid_map(e[a], nb, rw)
                x.append(xa)
                J *= ja
                bins.append((rw * nb) >> 32)
            F = J * oracle_mod.integrand(oracle_mod.GAUSS, np.array(x), GAUSS_PARAMS)
            fh.append(F)
            q = F * math.sqrt(1.0 / (nh * alloc[h]))
            for a in range(nd):
                dl[a][bins[a]].append(q * q)
            S1.append(F * ncall / (nh * alloc[h]))
        n = len(fh)
        mh = math.fsum(fh) / n
        vh = max((math.fsum(f * f for f in fh) - math.fsum(fh) ** 2 / n) / (n - 1), 0.0)
        m.append(mh)
        v.append(vh)
    I = math.fsum(S1) / ncall
    sig = math.sqrt(math.fsum(vh / nn for vh, nn in zip(v, alloc)) / nh ** 2)
    assert abs(r.per_iter[0, 0] - I) <= 1e-14 * abs(I)
    assert abs(r.per_iter[0, 0] - math.fsum(m) / nh) <= 1e-13 * abs(I)
    assert abs(r.per_iter[0, 1] - sig) <= 1e-12 * sig
    assert np.allclose(r.var, v, rtol=1e-11, atol=0)
    for a in range(nd):
        for i in range(nb):
            want = math.fsum(dl[a][i])
            assert abs(r.sums[2 + a * nb + i] - want) <= 1e-15 * want
    assert r.calls[0] == off[-1]


def test_plus_with_one_stratum_is_vegas(oracle_mod):
    """With one hypercube every event has a_h = 1: the estimate, its error and
    the refined grid are plain VEGAS's (the bin sums are VEGAS's over C,
    which the refinement does not see)."""
    for iid, params in [(oracle_mod.GAUSS, GAUSS_PARAMS), (oracle_mod.DY, DY_PARAMS)]:
        nd = 4
        a = oracle_mod.iterate(nd, 40, 9, 30_000, 3, iid, params, want_sums=True)
        b = oracle_mod.iterate_plus(nd, 40, 9, 30_000, 3, iid, params, nstrat=1)
        assert np.max(np.abs(a.per_iter - b.per_iter) / np.abs(a.per_iter)) < 1e-12
        assert np.max(np.abs(a.edges - b.edges)) < 1e-12
        assert np.allclose(b.sums[2:] * 30_000, a.sums[2:], rtol=1e-12, atol=0)
        assert list(b.calls) == [30_000] * 3 and list(b.alloc) == [30_000]


def test_plus_calls_and_allocation_bounds(oracle_mod):
    r = oracle_mod.iterate_plus(3, 30, 4, 50_000, 4, oracle_mod.GAUSS, GAUSS_PARAMS)
    nh = r.nstrat ** 3
    assert np.all(r.alloc >= 2)
    assert np.all(r.calls <= 50_000 + 2 * nh) and np.all(r.calls >= 2 * nh)
    assert r.calls[0] == (50_000 // nh) * nh


def test_plus_frozen_stage_keeps_grid_and_allocation(oracle_mod):
    r0 = oracle_mod.iterate_plus(2, 20, 4, 20_000, 2, oracle_mod.GAUSS, GAUSS_PARAMS)
    r1 = oracle_mod.iterate_plus(2, 20, 4, 20_000, 3, oracle_mod.GAUSS, GAUSS_PARAMS,
                                 edges=r0.edges, alloc=r0.alloc, iteration=r0.iteration,
                                 adapt=False)
    assert np.array_equal(r1.edges, r0.edges) and np.array_equal(r1.alloc, r0.alloc)
    assert len(set(r1.calls)) == 1


def test_plus_independent_of_thread_count(oracle_mod):
    n0 = oracle_mod.get_threads()
    try:
        outs = []
        for t in (1, 3, max(n0, 2)):
            oracle_mod.set_threads(t)
            outs.append(oracle_mod.iterate_plus(4, 50, 2, 60_000, 3, oracle_mod.DY, DY_PARAMS))
    finally:
        oracle_mod.set_threads(n0)
    for o in outs[1:]:
        for key in ("per_iter", "edges", "alloc", "sums", "var", "calls"):
            assert np.array_equal(o[key], outs[0][key]), key


# ------------------------------------------------------------- statistics
def _two_stage_plus(o, ndim, nbins, iid, params, ncall, warm, prod, seed):
    r = o.iterate_plus(ndim, nbins, seed, ncall // 4, warm, iid, params)
    # a new call count means new strata: the production stage restarts the allocation
    return o.iterate_plus(ndim, nbins, seed, ncall, prod, iid, params, edges=r.edges,
                          iteration=r.iteration)


def test_plus_gauss_pulls_over_seeds(oracle_mod):
    exact = refs.gauss_exact(4, GAUSS_PARAMS[0])
    pulls = []
    for seed in range(20):
        r = _two_stage_plus(oracle_mod, 4, 50, oracle_mod.GAUSS, GAUSS_PARAMS, 40_000, 3, 5, seed)
        pulls.append((r.integral - exact) / r.error)
    pulls = np.array(pulls)
    assert np.max(np.abs(pulls)) < 4.0
    assert abs(np.mean(pulls)) < 1.0 and 0.4 < np.std(pulls) < 1.8


@pytest.mark.parametrize("params,ndim", [(GAUSS_PARAMS, 2), (GAUSS_SHIFTED_PARAMS, 2),
                                         (GAUSS_PARAMS, 6)])
def test_plus_gauss_closed_forms(oracle_mod, params, ndim):
    exact = refs.gauss_exact(ndim, params[0]) - (params[1] if len(params) > 1 else 0.0)
    r = _two_stage_plus(oracle_mod, ndim, 50, oracle_mod.GAUSS, params, 100_000, 3, 5, 1234)
    assert abs(r.integral - exact) < 4.5 * r.error


def test_plus_dy_cross_section(oracle_mod):
    exact = refs.dy_sigma_quadrature(DY_PARAMS)
    r = _two_stage_plus(oracle_mod, 4, 100, oracle_mod.DY, DY_PARAMS, 400_000, 4, 5, 1234)
    assert abs(r.integral - exact) < 4.5 * r.error


def test_plus_reduces_the_variance(oracle_mod):
    """Stratification's purpose: at the same number of events per iteration,
    the d = 2 Gaussian's error shrinks several-fold against plain VEGAS."""
    a = oracle_mod.iterate(2, 50, 3, 100_000, 4, oracle_mod.GAUSS, GAUSS_PARAMS)
    a = oracle_mod.iterate(2, 50, 3, 100_000, 5, oracle_mod.GAUSS, GAUSS_PARAMS, edges=a.edges,
                           iteration=a.iteration)
    b = oracle_mod.iterate_plus(2, 50, 3, 100_000, 4, oracle_mod.GAUSS, GAUSS_PARAMS)
    b = oracle_mod.iterate_plus(2, 50, 3, 100_000, 5, oracle_mod.GAUSS, GAUSS_PARAMS,
                                edges=b.edges, alloc=b.alloc, iteration=b.iteration)
    assert b.error * 3 < a.error
