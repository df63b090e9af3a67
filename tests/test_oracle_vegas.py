"""Pins for the oracle's VEGAS iteration, combination and grid refinement.

Section 2.1: iterations of event sets, all events combined, the grid optimised
serially after each iteration.  Section 2.2: results independent of the
number of threads (made bit-exact here).  The refinement steps follow
Lepage's VEGAS, which the paper cites.
"""
import math

import numpy as np
import pytest

import refs
from paper_1503_06182_gb300.workloads import DY_PARAMS, EE3J_PARAMS, GAUSS_PARAMS


# ---------------------------------------------------------------- combination
def test_combine_hand_values(oracle_mod):
    I, e, c = oracle_mod.combine([1.0, 2.0], [1.0, 1.0])
    assert I == 1.5 and abs(e - 1 / math.sqrt(2)) < 1e-16 and abs(c - 0.5) < 1e-16
    I, e, c = oracle_mod.combine([1.0, 4.0], [1.0, 2.0])
    # weights 1 and 1/4: mean = (1 + 1) / 1.25 = 1.6; err = 1/sqrt(1.25)
    assert abs(I - 1.6) < 1e-15 and abs(e - 1 / math.sqrt(1.25)) < 1e-15
    assert abs(c - ((1 - 1.6) ** 2 + (4 - 1.6) ** 2 / 4)) < 1e-14
    I, e, c = oracle_mod.combine([3.0], [0.5])
    assert (I, e, c) == (3.0, 0.5, 0.0)
    # zero-variance iterations: plain mean of those, error 0
    I, e, c = oracle_mod.combine([2.0, 5.0, 4.0], [0.0, 1.0, 0.0])
    assert (I, e, c) == (3.0, 0.0, 0.0)


# ------------------------------------------------------------------ refinement
def _step_mass(edges_old, r, a, b):
    """Integral over [a, b] of the density that puts r_i uniformly on old bin i."""
    tot = 0.0
    for i in range(len(r)):
        lo, hi = max(a, edges_old[i]), min(b, edges_old[i + 1])
        if hi > lo:
            tot += r[i] * (hi - lo) / (edges_old[i + 1] - edges_old[i])
    return tot


def test_refine_uniform_sums_keep_any_grid(oracle_mod):
    rng = np.random.default_rng(1)
    for nbins in (2, 3, 10, 64):
        e = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, nbins - 1)), [1.0]])[None, :]
        out = oracle_mod.refine(np.full((1, nbins), 7.25), e)
        assert np.max(np.abs(out - e)) < 1e-14


def test_refine_zero_sums_and_alpha_zero_leave_grid(oracle_mod):
    rng = np.random.default_rng(2)
    e = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, 9)), [1.0]])[None, :]
    assert np.array_equal(oracle_mod.refine(np.zeros((1, 10)), e), e)
    d = rng.uniform(0.1, 5, (1, 10))
    assert np.max(np.abs(oracle_mod.refine(d, e, alpha=0.0) - e)) < 1e-14


def test_refine_scale_invariant_and_monotone(oracle_mod):
    rng = np.random.default_rng(4)
    d = rng.exponential(1.0, (3, 40)) ** 3
    d[1, 10:20] = 0.0
    e = oracle_mod.uniform_edges(3, 40)
    a = oracle_mod.refine(d, e)
    b = oracle_mod.refine(d * 1024.0, e)
    assert np.array_equal(a, b)
    assert np.all(a[:, 0] == 0.0) and np.all(a[:, -1] == 1.0)
    assert np.all(np.diff(a, axis=1) > 0)


def test_refine_equal_share_property(oracle_mod):
    """Each new bin carries exactly 1/N of the compressed, smoothed mass.  The
    smoothing and compression are the definitions of the step; the test checks
    the redistribution (the interpolation) by integrating the step density."""
    rng = np.random.default_rng(5)
    N, alpha = 25, 1.5
    d = rng.gamma(0.5, 1.0, N)
    d[3] = 0.0
    d[4] = 0.0
    d[5] = 0.0
    e = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, N - 1)), [1.0]])
    new = oracle_mod.refine(d[None, :], e[None, :], alpha)[0]
    sm = np.empty(N)
    sm[0] = (d[0] + d[1]) / 2
    sm[-1] = (d[-2] + d[-1]) / 2
    sm[1:-1] = (d[:-2] + d[1:-1] + d[2:]) / 3
    rho = sm / sm.sum()
    r = np.where(rho > 0, ((1 - rho) / -np.log(np.where(rho > 0, rho, 0.5))) ** alpha, 0.0)
    share = r.sum() / N
    for j in range(N):
        m = _step_mass(e, r, new[j], new[j + 1])
        assert abs(m - share) < 1e-12 * r.sum()


def test_refine_two_bins_hand_value(oracle_mod):
    """N = 2, worked by hand: both bins smooth to (d_0 + d_1)/2, so rho = 1/2
    for each, both compress to the same r, and the one inner edge sits where
    the cumulative mass reaches R/2 = r: at the end of old bin 0, i.e. the
    old edge.  Any sums, any edge: the grid is unchanged (a different end
    rule of the smoothing would move it)."""
    for e1, d in ((0.3, (5.0, 1.0)), (0.9, (1e-30, 7.0)), (0.125, (2.0, 0.0))):
        e = np.array([[0.0, e1, 1.0]])
        for alpha in (0.5, 1.0, 1.5):
            assert np.array_equal(oracle_mod.refine(np.array([d]), e, alpha), e)


def test_refine_three_bins_hand_values(oracle_mod):
    """N = 3, worked by hand (values to 16 digits from the closed forms).

    (a) d = (0, 0, 6), edges (0, 1/2, 3/4, 1), alpha = 1:
        smoothed (d0+d1)/2, (d0+d1+d2)/3, (d1+d2)/2 = (0, 2, 3), total 5,
        rho = (0, 2/5, 3/5), r = (0, (3/5)/ln(5/2), (2/5)/ln(5/3))
          = (0, 0.6548140007623749, 0.7830460755884871),
        R/3 = 0.4792866921169540.
        Edge 1: bin 0 holds nothing, bin 1 holds r_1 > R/3, so
          e'_1 = 1/2 + (R/3)/r_1 * (3/4 - 1/2) = 0.6829858141239111.
        Edge 2: 2R/3 > r_1, so it lies in bin 2:
          e'_2 = 3/4 + (2R/3 - r_1)/r_2 * (1 - 3/4) = 0.8469800478353867.
    (b) d = (0, 6, 0), uniform edges, alpha = 3/2:
        smoothed (3, 2, 3), total 8, rho = (3/8, 1/4, 3/8),
        r_0 = r_2 = ((5/8)/ln(8/3))^(3/2) = 0.5086627218742808,
        r_1 = ((3/4)/ln 4)^(3/2) = 0.3979318583048829,
        R/3 = 0.4717524340178148 < r_0, so
          e'_1 = (R/3)/r_0 * (1/3) = 0.3091455390319268, and by symmetry
          e'_2 = 1 - e'_1 = 0.6908544609680732."""
    a = oracle_mod.refine(np.array([[0.0, 0.0, 6.0]]), np.array([[0.0, 0.5, 0.75, 1.0]]), 1.0)
    assert np.max(np.abs(a - [[0.0, 0.6829858141239111, 0.8469800478353867, 1.0]])) < 2e-16
    b = oracle_mod.refine(np.array([[0.0, 6.0, 0.0]]), oracle_mod.uniform_edges(1, 3), 1.5)
    assert np.max(np.abs(b - [[0.0, 0.3091455390319268, 0.6908544609680732, 1.0]])) < 2e-16


def test_refine_concentrates_bins_on_peak(oracle_mod):
    d = np.zeros((1, 20))
    d[0, 9] = 1.0
    d[0, 10] = 1.0
    new = oracle_mod.refine(d, oracle_mod.uniform_edges(1, 20))[0]
    inside = np.sum((new > 0.39) & (new < 0.61))
    assert inside >= 15  # almost all edges move into the smoothed peak


def test_refine_alternating_widths_grow_on_flat_axis(oracle_mod):
    """First-order response of one refinement on an axis the integrand does
    not depend on, worked out by hand.  There d_i is proportional to the
    squared Jacobian factor Delta_i^2; take widths Delta_i = (1 + eps
    (-1)^i)/N, N even, so d_i = (1 + 2 eps (-1)^i)/N^2 + O(eps^2).
    - The 3-point mean of the interior gives the alternating part (2 eps/3)
      (1 - 2)(-1)^i = -(2 eps/3)(-1)^i: the wider bins get the smaller smoothed
      sums.  The ends' 2-point means have no first-order part, and the total
      is 1/N.
    - The compression m(rho) = ((1 - rho)/ln(1/rho))^alpha has the logarithmic
      slope kappa = alpha (1/ln(1/rho) - rho/(1 - rho)) at rho = 1/N, so
      inside m_i = mbar (1 - kappa (2 eps/3)(-1)^i), and m_0 = m_{N-1} = mbar.
    - The sum of m up to old edge j exceeds j mbar by mbar kappa (2 eps/3) for
      even j >= 2 and equals it for odd j; the N equal shares therefore move
      each even edge left by kappa (2 eps/3)/N and keep the odd ones.
    So bin i's new width is (1 + (1 + 2 kappa/3) eps (-1)^i)/N for 1 <= i <=
    N - 2, and bins 0 and N - 1 keep theirs.  The alternation grows by
    1 + 2 kappa/3 (1.207 at N = 100) per refinement: the reason a long run of
    adapting iterations roughens the grid along such an axis."""
    N, eps, alpha = 100, 1e-5, 1.5
    sgn = (-1.0) ** np.arange(N)
    w = (1.0 + eps * sgn) / N
    edges = np.concatenate([[0.0], np.cumsum(w)])
    edges[-1] = 1.0
    new = oracle_mod.refine((w ** 2)[None, :], edges[None, :], alpha)[0]
    rho = 1.0 / N
    kappa = alpha * (1.0 / math.log(1.0 / rho) - rho / (1.0 - rho))
    g = (np.diff(new) * N - 1.0) / (eps * sgn)  # each width's deviation in units of eps
    # second-order terms are O(eps) of these
    assert np.max(np.abs(g[1:-1] - (1.0 + 2.0 * kappa / 3.0))) < 1e-4
    assert abs(g[0] - 1.0) < 1e-4 and abs(g[-1] - 1.0) < 1e-4


# ----------------------------------------------------------- VEGAS estimates
def _two_stage(oracle_mod, ndim, nbins, iid, params, ncall, warm, prod, seed):
    r = oracle_mod.iterate(ndim, nbins, seed, ncall // 4, warm, iid, params)
    return oracle_mod.iterate(ndim, nbins, seed, ncall, prod, iid, params,
                              edges=r.edges, iteration=r.iteration)


def test_gauss_pulls_over_seeds(oracle_mod):
    """20 seeds of the d=4 Gaussian: pulls against the closed form ~ N(0,1)."""
    exact = refs.gauss_exact(4, GAUSS_PARAMS[0])
    vals, errs = [], []
    for seed in range(20):
        r = _two_stage(oracle_mod, 4, 50, oracle_mod.GAUSS, GAUSS_PARAMS, 40_000, 3, 5, seed)
        vals.append(r.integral)
        errs.append(r.error)
    p = refs.pulls(vals, errs, exact)
    assert np.all(np.abs(p) < 4.5)
    assert abs(np.mean(p)) < 1.0
    assert 0.4 < np.std(p) < 1.8


@pytest.mark.parametrize("ndim", [1, 2, 7])
def test_gauss_other_dims(oracle_mod, ndim):
    r = _two_stage(oracle_mod, ndim, 30, oracle_mod.GAUSS, GAUSS_PARAMS, 40_000, 3, 5, 99)
    assert abs(r.integral - refs.gauss_exact(ndim)) < 4.5 * r.error


def test_ee3j_closed_form_and_estimate(oracle_mod):
    y = EE3J_PARAMS[0]
    exact = refs.ee3j_exact(y)
    assert abs(exact - refs.ee3j_quadrature(y)) < 1e-10 * exact
    r = _two_stage(oracle_mod, 5, 100, oracle_mod.EE3J, EE3J_PARAMS, 400_000, 4, 5, 1234)
    assert abs(r.integral - exact) < 4.5 * r.error
    assert r.error < 2e-3 * exact


def test_ee3j_momenta_and_matrix_element(oracle_mod):
    """Momenta conserve four-momentum, are massless, carry E_i = x_i Q/2, and
    |M|^2 evaluated through them equals (x1^2+x2^2)/((1-x1)(1-x2))."""
    rng = np.random.default_rng(8)
    Q = EE3J_PARAMS[1]
    n = 0
    while n < 200:
        x = rng.uniform(0, 1, 5)
        g, mom = oracle_mod.integrand(oracle_mod.EE3J, x, EE3J_PARAMS, mom=True)
        x1, x2 = x[0], x[1]
        y = EE3J_PARAMS[0]
        if not (1 - x1 > y and 1 - x2 > y and x1 + x2 - 1 > y):
            assert g == 0.0
            continue
        n += 1
        p = mom[:3]
        tot = p.sum(axis=0)
        assert np.allclose(tot, [Q, 0, 0, 0], atol=1e-11 * Q)
        for v in p:
            assert abs(v[0] ** 2 - v[1] ** 2 - v[2] ** 2 - v[3] ** 2) < 1e-10 * Q * Q
        assert abs(p[0, 0] - x1 * Q / 2) < 1e-13 * Q and abs(p[1, 0] - x2 * Q / 2) < 1e-13 * Q
        want = (x1 * x1 + x2 * x2) / ((1 - x1) * (1 - x2))
        assert abs(g - want) < 1e-10 * want


def test_dy_partonic_matches_helicity_amplitudes(oracle_mod):
    p = DY_PARAMS
    rng = np.random.default_rng(9)
    for _ in range(200):
        m = rng.uniform(60, 120)
        c = rng.uniform(-1, 1)
        for up, fq in ((1, refs.UP), (0, refs.DOWN)):
            got = oracle_mod.dy_dsigma_domega(up, m * m, c, p)
            want = refs.dy_dsigma_domega_helicity(fq, m * m, c, p[1], p[2], p[3], p[4])
            assert abs(got - want) < 1e-12 * abs(want)


def test_dy_forward_backward_sign(oracle_mod):
    """Above the Z pole the gamma-Z interference makes mu- follow the quark."""
    p = DY_PARAMS
    s = 110.0 ** 2
    assert oracle_mod.dy_dsigma_domega(1, s, 0.5, p) > oracle_mod.dy_dsigma_domega(1, s, -0.5, p)
    s = 70.0 ** 2
    assert oracle_mod.dy_dsigma_domega(1, s, 0.5, p) < oracle_mod.dy_dsigma_domega(1, s, -0.5, p)


def test_dy_momenta_and_symmetry(oracle_mod):
    p = DY_PARAMS
    s = p[0] ** 2
    rng = np.random.default_rng(10)
    for _ in range(200):
        x = rng.uniform(0, 1, 4)
        g, mom = oracle_mod.integrand(oracle_mod.DY, x, p, mom=True)
        p1, p2, p3, p4 = mom
        tot_in, tot_out = p1 + p2, p3 + p4
        scale = tot_in[0]
        assert np.allclose(tot_in, tot_out, atol=1e-12 * scale)
        for v in mom:
            assert abs(v[0] ** 2 - v[1] ** 2 - v[2] ** 2 - v[3] ** 2) < 1e-9 * v[0] ** 2
        mll2 = (p3 + p4)[0] ** 2 - np.sum((p3 + p4)[1:] ** 2)
        tau = (p[5] / p[0]) ** 2 * (p[6] / p[5]) ** (2 * x[0])
        assert abs(mll2 - tau * s) < 1e-6 * tau * s
        # pp is symmetric under z -> -z: (y, cos theta) -> (-y, -cos theta)
        xr = x.copy()
        xr[1] = 1 - x[1]
        xr[2] = 1 - x[2]
        assert abs(oracle_mod.integrand(oracle_mod.DY, xr, p) - g) < 1e-11 * g


def test_dy_total_cross_section(oracle_mod):
    exact = refs.dy_sigma_quadrature(DY_PARAMS)
    assert abs(exact - 5.5962) < 1e-3
    r = _two_stage(oracle_mod, 4, 100, oracle_mod.DY, DY_PARAMS, 400_000, 4, 5, 1234)
    assert abs(r.integral - exact) < 4.5 * r.error
    assert r.error < 1e-3 * exact


# ------------------------------------------------- NLO-shaped stand-in (id 3)
DYNLO_BETA = 0.5


def test_dynlo_extra_factor_integrates_to_one(oracle_mod):
    """Along one extra axis the weight is the Drell-Yan weight times
    exp(beta cos 2 pi u) / I0(beta); quadrature of that factor (no Bessel
    function involved) gives 1."""
    from scipy.integrate import quad

    x = np.array([0.3, 0.6, 0.2, 0.7, 0.0])
    g_dy = oracle_mod.integrand(oracle_mod.DY, x, DY_PARAMS)
    for beta in (0.3, 1.0, 2.5):
        p = tuple(DY_PARAMS) + (beta,)

        def f(u):
            xx = x.copy()
            xx[4] = u
            return oracle_mod.integrand(oracle_mod.DYNLO, xx, p) / g_dy

        val, err = quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert abs(val - 1.0) < 1e-12, (beta, val)


def test_dynlo_beta_zero_is_drell_yan(oracle_mod):
    """beta = 0 makes every extra factor exactly 1: the events' weights are the
    Drell-Yan ones bit for bit (13 axes, the same Philox streams and bins)."""
    edges = oracle_mod.uniform_edges(13, 50)
    p = tuple(DY_PARAMS) + (0.0,)
    for ev in (0, 17, 123_456):
        w0, b0, _ = oracle_mod.event(oracle_mod.DY, 13, 50, edges, DY_PARAMS, 1234, 2, 0, ev)
        w1, b1, _ = oracle_mod.event(oracle_mod.DYNLO, 13, 50, edges, p, 1234, 2, 0, ev)
        assert w0 == w1 and np.array_equal(b0, b1)


def test_dynlo_total_is_drell_yan_cross_section(oracle_mod):
    """13 axes, beta = 0.5: the integral is the Drell-Yan cross section."""
    exact = refs.dy_sigma_quadrature(DY_PARAMS)
    p = tuple(DY_PARAMS) + (DYNLO_BETA,)
    r = _two_stage(oracle_mod, 13, 50, oracle_mod.DYNLO, p, 200_000, 4, 5, 1234)
    assert abs(r.integral - exact) < 4.5 * r.error
    assert r.error < 3e-3 * exact


# --------------------------------------------------------- thread invariance
def test_results_independent_of_thread_count(oracle_mod):
    """Section 2.2's validation invariant, bit-exact: 1, 2, 3 and 8 threads."""
    outs = []
    try:
        for nt in (1, 2, 3, 8):
            oracle_mod.set_threads(nt)
            r = oracle_mod.iterate(4, 50, 1234, 30_001, 3, oracle_mod.DY, DY_PARAMS, want_sums=True)
            outs.append(r)
    finally:
        oracle_mod.set_threads(0)
    for r in outs[1:]:
        assert np.array_equal(r.per_iter, outs[0].per_iter)
        assert np.array_equal(r.edges, outs[0].edges)
        assert np.array_equal(r.sums, outs[0].sums)
        assert r.integral == outs[0].integral


def test_stage_split_is_seamless(oracle_mod):
    """5 iterations in one call equal 2 + 3 iterations with the grid and the
    iteration counter carried over (the checkpoint state)."""
    a = oracle_mod.iterate(4, 50, 7, 20_000, 5, oracle_mod.GAUSS, GAUSS_PARAMS)
    b = oracle_mod.iterate(4, 50, 7, 20_000, 2, oracle_mod.GAUSS, GAUSS_PARAMS)
    c = oracle_mod.iterate(4, 50, 7, 20_000, 3, oracle_mod.GAUSS, GAUSS_PARAMS,
                           edges=b.edges, iteration=b.iteration)
    assert np.array_equal(a.per_iter, np.concatenate([b.per_iter, c.per_iter]))
    assert np.array_equal(a.edges, c.edges)
    assert c.iteration == 5


def test_sums_match_direct_event_loop(oracle_mod):
    """The chunked compensated sums equal a plain math.fsum over the events."""
    nd, nb, ncall = 3, 10, 9000
    e = oracle_mod.uniform_edges(nd, nb)
    r = oracle_mod.iterate(nd, nb, 5, ncall, 1, oracle_mod.GAUSS, GAUSS_PARAMS, adapt=False,
                           want_sums=True)
    ws, bins = [], []
    for ev in range(ncall):
        w, b, _ = oracle_mod.event(oracle_mod.GAUSS, nd, nb, e, GAUSS_PARAMS, 5, 0, 0, ev)
        ws.append(w)
        bins.append(b)
    ws = np.array(ws)
    bins = np.array(bins)
    assert abs(r.sums[0] - math.fsum(ws)) <= 2e-16 * abs(r.sums[0])
    assert abs(r.sums[1] - math.fsum(ws * ws)) <= 2e-16 * r.sums[1]
    d = r.sums[2:].reshape(nd, nb)
    for a in range(nd):
        for i in range(nb):
            want = math.fsum(ws[bins[:, a] == i] ** 2)
            assert abs(d[a, i] - want) <= 4e-16 * want
    I = r.per_iter[0, 0]
    assert abs(I - math.fsum(ws) / ncall) <= 2e-16 * I
    var = (math.fsum(ws * ws) / ncall - I * I) / (ncall - 1)
    assert abs(r.per_iter[0, 1] - math.sqrt(var)) <= 1e-12 * r.per_iter[0, 1]


def test_zero_weight_iteration_keeps_grid(oracle_mod):
    """y_cut = 0.4 leaves no phase space: every weight is 0, I = 0, grid unchanged."""
    r = oracle_mod.iterate(5, 20, 3, 5000, 2, oracle_mod.EE3J, (0.4, 91.1876))
    assert r.integral == 0.0 and r.error == 0.0
    assert np.array_equal(r.edges, oracle_mod.uniform_edges(5, 20))


def test_nonfinite_weights_are_counted(oracle_mod):
    p = list(DY_PARAMS)
    p[9] = float("inf")
    r = oracle_mod.iterate(4, 10, 3, 5000, 1, oracle_mod.DY, p)
    assert r.nonfinite == 5000
