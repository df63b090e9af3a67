"""Pins for the oracle's Drell-Yan gradient d sigma / d(M_Z, Gamma_Z, sw2, a, b).

The analytic derivative of the event weight is checked against central
differences of the weight; the frozen-grid gradient estimate against central
differences of the frozen-grid VEGAS estimate on the same events; and the
estimate against the derivative of the quadrature value of sigma.
"""
import numpy as np

import refs
from paper_1503_06182_gb300.workloads import DY_GRAD_INDEX, DY_PARAMS


def test_event_gradient_matches_finite_differences(oracle_mod):
    rng = np.random.default_rng(11)
    p0 = np.array(DY_PARAMS)
    for _ in range(40):
        x = rng.uniform(0.02, 0.98, 4)
        g, grad = oracle_mod.integrand(oracle_mod.DY, x, p0, grad=True)
        for k, idx in enumerate(DY_GRAD_INDEX):
            h = 1e-6 * max(abs(p0[idx]), 1e-3)
            pp, pm = p0.copy(), p0.copy()
            pp[idx] += h
            pm[idx] -= h
            fd = (oracle_mod.integrand(oracle_mod.DY, x, pp) -
                  oracle_mod.integrand(oracle_mod.DY, x, pm)) / (2 * h)
            assert abs(grad[k] - fd) <= 1e-6 * max(abs(fd), 1e-9 * abs(g) / max(abs(p0[idx]), 1e-3))


def test_gradient_estimate_matches_fd_of_estimate(oracle_mod):
    """Same events, same frozen grid, single iteration: the estimate of
    E[dw/dtheta] equals the central difference of the estimate of E[w]."""
    nd, nb, ncall = 4, 50, 20_000
    warm = oracle_mod.iterate(nd, nb, 1234, ncall, 3, oracle_mod.DY, DY_PARAMS)
    edges, it0 = warm.edges, warm.iteration
    adj = oracle_mod.adjoint(nd, nb, 1234, ncall, 1, DY_PARAMS, edges=edges, iteration=it0)
    p0 = np.array(DY_PARAMS)
    for k, idx in enumerate(DY_GRAD_INDEX):
        h = 1e-4 * abs(p0[idx])
        pp, pm = p0.copy(), p0.copy()
        pp[idx] += h
        pm[idx] -= h
        fp = oracle_mod.iterate(nd, nb, 1234, ncall, 1, oracle_mod.DY, pp, edges=edges,
                                iteration=it0, adapt=False).integral
        fm = oracle_mod.iterate(nd, nb, 1234, ncall, 1, oracle_mod.DY, pm, edges=edges,
                                iteration=it0, adapt=False).integral
        fd = (fp - fm) / (2 * h)
        assert abs(adj.grad[k] - fd) <= 1e-4 * abs(fd), (k, adj.grad[k], fd)
    assert abs(adj.integral - oracle_mod.iterate(nd, nb, 1234, ncall, 1, oracle_mod.DY, p0,
                                                 edges=edges, iteration=it0,
                                                 adapt=False).integral) == 0.0


def test_gradient_estimate_matches_quadrature_derivative(oracle_mod):
    nd, nb = 4, 100
    warm = oracle_mod.iterate(nd, nb, 77, 100_000, 5, oracle_mod.DY, DY_PARAMS)
    adj = oracle_mod.adjoint(nd, nb, 77, 200_000, 5, DY_PARAMS, edges=warm.edges,
                             iteration=warm.iteration)
    p0 = np.array(DY_PARAMS)
    for k, idx in enumerate(DY_GRAD_INDEX):
        h = 1e-3 * abs(p0[idx])
        pp, pm = p0.copy(), p0.copy()
        pp[idx] += h
        pm[idx] -= h
        d = (refs.dy_sigma_quadrature(pp, 1e-11) - refs.dy_sigma_quadrature(pm, 1e-11)) / (2 * h)
        assert abs(adj.grad[k] - d) < 5.0 * adj.grad_err[k] + 1e-5 * abs(d), (k, adj.grad[k], d)
