"""Pins for the oracle's histograms during integration.

The paper shows differential distributions filled while integrating (the
di-jet mass plots of Section 3.2).  Here each event's weight also goes into
the bin of one observable: Gauss x_0, Drell-Yan m_ll, 3-jet thrust.  The
pins come from outside the oracle: closed forms (erf, the leading-order
thrust distribution), quadrature of the Drell-Yan mass spectrum, the
invariant mass and thrust recomputed from the oracle's four-momenta, a
direct event loop, and the sum rule that the bins add up to the integral.
"""
import math

import numpy as np
import pytest

import refs
from paper_1503_06182_gb300.workloads import (DY_PARAMS, DYNLO_PARAMS, EE3J_PARAMS, GAUSS_PARAMS,
                                              GAUSS_SHIFTED_PARAMS)


def _two_stage(o, ndim, nbins, iid, params, ncall, warm, prod, seed, hist):
    r = o.iterate(ndim, nbins, seed, ncall // 4, warm, iid, params)
    return o.iterate(ndim, nbins, seed, ncall, prod, iid, params, edges=r.edges,
                     iteration=r.iteration, hist=hist)


def _pulls_ok(val, err, exact, limit=4.5):
    """Every bin within `limit` standard errors; bins whose exact value is 0
    are exactly 0 with error 0."""
    for v, e, x in zip(val, err, exact):
        if x == 0.0:
            assert v == 0.0 and e == 0.0
        else:
            assert abs(v - x) < limit * e, (v, x, e)


# ------------------------------------------------------------- bin rule
def test_hist_bin_rule_edges_and_specials(oracle_mod):
    nh, lo, hi = 12, 60.0, 120.0
    assert oracle_mod.hist_bin(lo, nh, lo, hi) == 1
    assert oracle_mod.hist_bin(np.nextafter(lo, -np.inf), nh, lo, hi) == 0
    assert oracle_mod.hist_bin(hi, nh, lo, hi) == nh + 1
    assert oracle_mod.hist_bin(np.nextafter(hi, -np.inf), nh, lo, hi) == nh
    assert oracle_mod.hist_bin(float("nan"), nh, lo, hi) == 0
    assert oracle_mod.hist_bin(float("inf"), nh, lo, hi) == nh + 1
    assert oracle_mod.hist_bin(-float("inf"), nh, lo, hi) == 0


def test_hist_bin_rule_against_edge_search(oracle_mod):
    """Away from the edges (closer than 1e-9 of a bin width: skipped), the bin
    equals the position among the edges lo + j (hi - lo)/nh by binary search."""
    rng = np.random.default_rng(3)
    for nh, lo, hi in [(7, 0.0, 1.0), (60, 60.0, 120.0), (10, 2 / 3, 1.0)]:
        edges = lo + (hi - lo) * np.arange(nh + 1) / nh
        vals = rng.uniform(lo - 0.2 * (hi - lo), hi + 0.2 * (hi - lo), 3000)
        width = (hi - lo) / nh
        for v in vals:
            if np.min(np.abs(edges - v)) < 1e-9 * width:
                continue
            want = int(np.searchsorted(edges, v, side="right"))  # 0 below lo, nh+1 above hi
            assert oracle_mod.hist_bin(v, nh, lo, hi) == want, (v, nh, lo, hi)


# ------------------------------------------------------------- observables
def test_dy_observable_is_dilepton_mass(oracle_mod):
    rng = np.random.default_rng(11)
    for params in (DY_PARAMS, DYNLO_PARAMS):
        iid = oracle_mod.DY if params is DY_PARAMS else oracle_mod.DYNLO
        for _ in range(100):
            x = rng.uniform(0, 1, 4 if iid == oracle_mod.DY else 6)
            _, mom = oracle_mod.integrand(iid, x, params, mom=True)
            p = mom[2] + mom[3]  # the two leptons
            m = math.sqrt(p[0] ** 2 - p[1] ** 2 - p[2] ** 2 - p[3] ** 2)
            assert abs(oracle_mod.observable(iid, x, params) - m) < 1e-9 * m
            assert params[5] <= m <= params[6] * (1 + 1e-12)


def test_ee3j_observable_is_thrust(oracle_mod):
    """Thrust from the momenta: max over directions n of sum |p_i.n| / sum |p_i|,
    which for three massless partons is attained along the hardest parton;
    checked against a search over the parton directions and random ones."""
    rng = np.random.default_rng(12)
    Q = EE3J_PARAMS[1]
    n_ok = 0
    while n_ok < 60:
        x = rng.uniform(0, 1, 5)
        g, mom = oracle_mod.integrand(oracle_mod.EE3J, x, EE3J_PARAMS, mom=True)
        if g == 0.0:
            continue
        n_ok += 1
        ps = mom[:3, 1:]
        norm = np.sum(np.linalg.norm(ps, axis=1))
        cand = [p / np.linalg.norm(p) for p in ps]
        rnd = rng.normal(size=(400, 3))
        cand += list(rnd / np.linalg.norm(rnd, axis=1)[:, None])
        best = max(np.sum(np.abs(ps @ n)) for n in cand) / norm
        T = oracle_mod.observable(oracle_mod.EE3J, x, EE3J_PARAMS)
        assert abs(T - best) < 1e-12
        assert abs(T - 2 * max(np.linalg.norm(ps, axis=1)) / Q) < 1e-12


def test_gauss_observable_is_first_axis(oracle_mod):
    x = np.array([0.123, 0.9, 0.4, 0.7])
    assert oracle_mod.observable(oracle_mod.GAUSS, x, GAUSS_PARAMS) == 0.123


# ------------------------------------------------------------- combination
def test_hist_combine_hand_values(oracle_mod):
    sk = np.array([1.0, 2.0])
    H = np.array([[1.0, 3.0], [2.0, 5.0]])
    V = np.array([[0.25, 1.0], [4.0, 0.0]])
    val, err = oracle_mod.hist_combine(sk, H, V)
    # weights 1 and 1/4, W = 5/4
    assert np.allclose(val, [(1.0 + 0.5) / 1.25, (3.0 + 1.25) / 1.25], rtol=0, atol=1e-15)
    assert np.allclose(err, [math.sqrt(0.25 + 4.0 / 16) / 1.25, math.sqrt(1.0) / 1.25],
                       rtol=0, atol=1e-15)
    # a zero-variance iteration: it alone, with its own variance
    val, err = oracle_mod.hist_combine(np.array([0.0, 2.0]), H, V)
    assert np.array_equal(val, [1.0, 3.0]) and np.array_equal(err, [0.5, 1.0])


# ------------------------------------------------------------- sums
@pytest.mark.parametrize("iid,params,ndim,hist", [
    (0, GAUSS_PARAMS, 4, (20, 0.0, 1.0)),
    (0, GAUSS_PARAMS, 3, (12, 0.2, 0.8)),
    (1, DY_PARAMS, 4, (30, 70.0, 110.0)),
    (2, EE3J_PARAMS, 5, (10, 2 / 3, 1.0)),
    (3, DYNLO_PARAMS, 7, (12, 60.0, 120.0)),
    (0, GAUSS_SHIFTED_PARAMS, 2, (16, 0.1, 0.9)),
])
def test_hist_adds_up_to_the_integral(oracle_mod, iid, params, ndim, hist):
    """Bins including underflow and overflow add up to the combined integral
    (the histogram is combined with the integral's weights), and the last
    iteration's bin sums add up to its sum w and sum w^2."""
    r = oracle_mod.iterate(ndim, 40, 7, 30_000, 4, iid, params, want_sums=True, hist=hist)
    assert abs(math.fsum(r.hist_value) - r.integral) <= 1e-12 * abs(r.integral)
    assert abs(math.fsum(r.hist_last[0]) - r.sums[0]) <= 1e-13 * abs(r.sums[0])
    assert abs(math.fsum(r.hist_last[1]) - r.sums[1]) <= 1e-13 * abs(r.sums[1])
    assert np.all(r.hist_error >= 0)


def test_hist_matches_direct_event_loop(oracle_mod):
    """One iteration on a fixed non-uniform grid: the per-bin sums equal a
    plain math.fsum over the events, each binned by its observable."""
    nd, nb, ncall, nh, lo, hi = 4, 10, 6000, 9, 65.0, 115.0
    e = oracle_mod.uniform_edges(nd, nb)
    e[:, 1:-1] += 0.03 * np.sin(np.arange(1, nb))[None, :] / nb
    r = oracle_mod.iterate(nd, nb, 21, ncall, 1, oracle_mod.DY, DY_PARAMS, edges=e, adapt=False,
                           want_sums=True, hist=(nh, lo, hi))
    sw = [[] for _ in range(nh + 2)]
    for ev in range(ncall):
        w, _, x = oracle_mod.event(oracle_mod.DY, nd, nb, e, DY_PARAMS, 21, 0, 0, ev)
        b = oracle_mod.hist_bin(oracle_mod.observable(oracle_mod.DY, x, DY_PARAMS), nh, lo, hi)
        sw[b].append(w)
    for b in range(nh + 2):
        ws = np.array(sw[b])
        want1, want2 = math.fsum(ws), math.fsum(ws * ws)
        assert abs(r.hist_last[0, b] - want1) <= 4e-16 * abs(want1)
        assert abs(r.hist_last[1, b] - want2) <= 4e-16 * want2
        h = want1 / ncall
        v = max((want2 / ncall - h * h) / (ncall - 1), 0.0)
        assert abs(r.hist_value[b] - h) <= 1e-14 * abs(h)
        assert abs(r.hist_error[b] - math.sqrt(v)) <= 1e-12 * math.sqrt(v)
    assert len(sw[0]) > 0 and len(sw[nh + 1]) > 0  # m_ll outside [65, 115) GeV


def test_hist_leaves_the_integration_unchanged(oracle_mod):
    a = oracle_mod.iterate(4, 50, 3, 20_000, 3, oracle_mod.DY, DY_PARAMS)
    b = oracle_mod.iterate(4, 50, 3, 20_000, 3, oracle_mod.DY, DY_PARAMS, hist=(25, 60.0, 120.0))
    assert np.array_equal(a.per_iter, b.per_iter) and np.array_equal(a.edges, b.edges)
    assert a.integral == b.integral and a.error == b.error


def test_hist_independent_of_thread_count(oracle_mod):
    n0 = oracle_mod.get_threads()
    try:
        outs = []
        for t in (1, 3, max(n0, 2)):
            oracle_mod.set_threads(t)
            outs.append(oracle_mod.iterate(5, 30, 9, 30_000, 2, oracle_mod.EE3J, EE3J_PARAMS,
                                           hist=(15, 2 / 3, 1.0)))
    finally:
        oracle_mod.set_threads(n0)
    for o in outs[1:]:
        assert np.array_equal(o.hist_value, outs[0].hist_value)
        assert np.array_equal(o.hist_error, outs[0].hist_error)
        assert np.array_equal(o.hist_last, outs[0].hist_last)


# ------------------------------------------------------------- physics
def test_gauss_hist_closed_form(oracle_mod):
    """x_0 histogram of the d=4 Gaussian against erf, bin by bin; over [0.2,
    0.8) the tails land in the underflow and overflow bins."""
    nh, lo, hi = 12, 0.2, 0.8
    r = _two_stage(oracle_mod, 4, 50, oracle_mod.GAUSS, GAUSS_PARAMS, 200_000, 3, 5, 1234,
                   (nh, lo, hi))
    w = (hi - lo) / nh
    exact = [refs.gauss_bin(0.0, lo, 4)]
    exact += [refs.gauss_bin(lo + j * w, lo + (j + 1) * w, 4) for j in range(nh)]
    exact += [refs.gauss_bin(hi, 1.0, 4)]
    _pulls_ok(r.hist_value, r.hist_error, exact)
    assert max(r.hist_error[1:-1] / np.array(exact[1:-1])) < 0.03  # the pins have power


def test_dy_mass_spectrum_against_quadrature(oracle_mod):
    """dsigma/dm_ll in 12 bins over the generated 60-120 GeV against 2-D
    quadrature of lumi x sigmahat over each bin; nothing outside the range."""
    nh, lo, hi = 12, 60.0, 120.0
    r = _two_stage(oracle_mod, 4, 100, oracle_mod.DY, DY_PARAMS, 200_000, 3, 5, 1234,
                   (nh, lo, hi))
    w = (hi - lo) / nh
    exact = [0.0] + [refs.dy_sigma_quadrature(DY_PARAMS, epsrel=1e-9,
                                              m_range=(lo + j * w, lo + (j + 1) * w))
                     for j in range(nh)] + [0.0]
    _pulls_ok(r.hist_value, r.hist_error, exact)
    # the Z peak: the bin holding M_Z is the largest
    assert int(np.argmax(r.hist_value)) == 1 + int((DY_PARAMS[1] - lo) / w)


def test_ee3j_thrust_against_closed_form(oracle_mod):
    """Thrust histogram of e+e- -> q qbar g against the leading-order thrust
    distribution integrated over each bin (the cut leaves T < 1 - y_cut); no
    event has T < 2/3 or T >= 1."""
    y = EE3J_PARAMS[0]
    nh, lo, hi = 10, 2 / 3, 1.0
    r = _two_stage(oracle_mod, 5, 100, oracle_mod.EE3J, EE3J_PARAMS, 200_000, 3, 5, 1234,
                   (nh, lo, hi))
    w = (hi - lo) / nh
    exact = [0.0] + [refs.ee3j_thrust_bin(lo + j * w, lo + (j + 1) * w, y)
                     for j in range(nh)] + [0.0]
    _pulls_ok(r.hist_value, r.hist_error, exact)


def test_shifted_gauss_signed_weights(oracle_mod):
    """The Gaussian minus a constant: mostly negative weights.  The integral
    is the closed form minus the constant; each x_0 bin is its erf integral
    minus the constant times the bin width; negative bins come out negative."""
    sigma, shift = GAUSS_SHIFTED_PARAMS
    nh, lo, hi = 10, 0.0, 1.0
    r = _two_stage(oracle_mod, 2, 50, oracle_mod.GAUSS, GAUSS_SHIFTED_PARAMS, 200_000, 3, 5,
                   1234, (nh, lo, hi))
    exact = refs.gauss_exact(2, sigma) - shift
    assert exact < 0 and abs(r.integral - exact) < 4.5 * r.error
    w = (hi - lo) / nh
    bins = [0.0] + [refs.gauss_bin(lo + j * w, lo + (j + 1) * w, 2, sigma) - shift * w
                    for j in range(nh)] + [0.0]
    _pulls_ok(r.hist_value, r.hist_error, bins)
    assert r.hist_value[1] < 0 < r.hist_value[5]
