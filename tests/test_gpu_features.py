"""GPU path: adjoint gradient, autograd, checkpoint/resume, grid validation,
non-finite weights, edge sizes and argument errors (requires a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import DY_GRAD_INDEX, DY_PARAMS, EE3J_PARAMS, GAUSS_PARAMS

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def warm_dy(precision="fp64", ncall=20_000, itmx=3, nbins=50):
    g = v.Vegas(4, nbins, 1234, precision=precision)
    g.iterate(ncall, itmx, v.VEGAS_DY, DY_PARAMS)
    return g


# ------------------------------------------------------------------ adjoint
def test_adjoint_fp64_matches_oracle():
    g = warm_dy()
    try:
        edges = g.grid
        grad, gerr, I, e, per = g.adjoint(30_000 + 11, 3, DY_PARAMS)
    finally:
        g.close()
    # the counter after 3 warm-up iterations is 3
    ref = oracle.adjoint(4, 50, 1234, 30_011, 3, DY_PARAMS, edges=edges, iteration=3)
    for k in range(3):
        for p in range(5):
            G, sG = per[k, p]
            Go, sGo = ref.per_iter_grad[k, p]
            assert abs(G - Go) <= 1e-10 * (abs(Go) + sGo)
            assert abs(sG - sGo) <= 1e-9 * sGo
    assert np.all(np.abs(grad - ref.grad) <= 1e-10 * (np.abs(ref.grad) + ref.grad_err))
    assert rel(I, ref.integral) < 1e-12
    assert rel(e, ref.error) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ndim", [4, 6])
def test_adjoint_identical_across_events_per_thread(precision, ndim):
    """Exact tile sums: the gradient stage gives the same bits whatever the
    events per thread (block size), for a ragged call count and for the
    kernels of up to 4 and of up to 16 axes."""
    outs = []
    for ept in (1, 2, 4):
        g = v.Vegas(ndim, 50, 1234, precision=precision)
        try:
            g.iterate(20_000, 2, v.VEGAS_DY, DY_PARAMS)
            g.set(v.VEGAS_OPT_EPT, ept)
            outs.append(g.adjoint(30_011, 2, DY_PARAMS))
        finally:
            g.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(np.asarray(a), np.asarray(b))


def test_adjoint_fp64_matches_oracle_six_axes():
    """Two flat extra axes: the same gradient, from the 16-axis kernel."""
    g = v.Vegas(6, 40, 77, precision="fp64")
    try:
        g.iterate(20_000, 2, v.VEGAS_DY, DY_PARAMS)
        edges = g.grid
        g.set(v.VEGAS_OPT_EPT, 1)
        grad, gerr, I, e, per = g.adjoint(25_000 + 7, 2, DY_PARAMS)
    finally:
        g.close()
    ref = oracle.adjoint(6, 40, 77, 25_007, 2, DY_PARAMS, edges=edges, iteration=2)
    assert np.all(np.abs(grad - ref.grad) <= 1e-10 * (np.abs(ref.grad) + ref.grad_err))
    assert np.all(np.abs(gerr - ref.grad_err) <= 1e-9 * ref.grad_err)
    assert rel(I, ref.integral) < 1e-12
    assert rel(e, ref.error) < 1e-12


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("ept", [4, 8])
def test_sums_equal_exact_sums_of_event_weights_with_subnormal_products(precision, ept):
    """The fill's once-rounded sums against the exact sums of its own weights
    (the per-event diagnostics form each weight as a double).  A narrow
    Gaussian minus 1e-40: almost every event's FP32 product is subnormal, so
    the FP32 fill takes its general route for it (the bins far from the peak
    hold nothing else), the few central events its direct route."""
    from fractions import Fraction

    ndim, nbins, ncall = 4, 50, 200_003
    params = (0.01, 1e-40)
    g = v.Vegas(ndim, nbins, 4242, precision=precision)
    try:
        g.set(v.VEGAS_OPT_EPT, ept)
        w, bins = g.eval_events(v.VEGAS_GAUSS, params, 0, np.arange(ncall, dtype=np.int64))
        g.iterate(ncall, 1, v.VEGAS_GAUSS, params)
        sums = g.last_sums()
    finally:
        g.close()
    tiny = (w != 0.0) & (np.abs(w) < 2.0**-120)
    assert tiny.sum() > 100_000 and (np.abs(w) > 2.0**-100).sum() > 100
    # exact sums as integers: w = mi 2^(e - 53) = mi 2^sh / 2^1200
    m, e = np.frexp(w)
    mi = (m * 2.0**53).astype(np.int64)
    sh = e.astype(np.int64) - 53 + 1200
    assert sh[w != 0].min() >= 0
    s1, s2 = 0, 0
    d = [0] * (ndim * nbins)
    dmax = np.zeros(ndim * nbins)
    for j in np.flatnonzero(w):
        x = int(mi[j]) << int(sh[j])
        xx = x * x  # over 2^2400
        s1 += x
        s2 += xx
        for ax in range(ndim):
            k = ax * nbins + int(bins[j, ax])
            d[k] += xx
            dmax[k] = max(dmax[k], abs(w[j]))
    S1, S2 = float(Fraction(s1, 1 << 1200)), float(Fraction(s2, 1 << 2400))
    assert abs(sums[0] - S1) <= 1e-15 * abs(S1)
    assert abs(sums[1] - S2) <= 1e-15 * S2
    dref = np.array([float(Fraction(x, 1 << 2400)) for x in d])
    nz = dref != 0
    assert np.array_equal(sums[2:] != 0, nz)
    assert rel(sums[2:][nz], dref[nz]) < 1e-13
    # bins whose every event came through the general route
    assert np.count_nonzero(nz & (dmax < 2.0**-120)) >= 10


def test_adjoint_matches_central_differences_on_gpu():
    """Frozen grid, one iteration, the same events: the adjoint estimate equals
    the central difference of the forward estimate (h = 1e-4 theta)."""
    g = warm_dy()
    try:
        g.set(v.VEGAS_OPT_ADAPT, 0)
        st = g.state()
        grad, _, _, _, _ = g.adjoint(20_000, 1, DY_PARAMS)
        p0 = np.array(DY_PARAMS)
        for k, idx in enumerate(DY_GRAD_INDEX):
            h = 1e-4 * abs(p0[idx])
            pp, pm = p0.copy(), p0.copy()
            pp[idx] += h
            pm[idx] -= h
            g.restore(st)
            fp = g.iterate(20_000, 1, v.VEGAS_DY, pp)[0]
            g.restore(st)
            fm = g.iterate(20_000, 1, v.VEGAS_DY, pm)[0]
            fd = (fp - fm) / (2 * h)
            assert abs(grad[k] - fd) <= 1e-4 * abs(fd), (k, grad[k], fd)
    finally:
        g.close()


def test_autograd_function_gives_adjoint():
    torch = pytest.importorskip("torch")
    from paper_1503_06182_gb300.autograd import DrellYanIntegral

    integ = DrellYanIntegral(ncall=20_000, itmx=2, nbins=50)
    try:
        integ.warmup(20_000, 3)
        st = integ.g.state()
        theta = torch.tensor([DY_PARAMS[i] for i in DY_GRAD_INDEX], dtype=torch.float64,
                             requires_grad=True)
        sigma = integ(theta)
        (2.0 * sigma).backward()
        after = integ.g.state()
        integ.g.restore(st)
        grad, _, I, _, _ = integ.g.adjoint(20_000, 2, DY_PARAMS)
        assert sigma.item() == I
        assert np.array_equal(theta.grad.numpy(), 2.0 * grad)
        assert after != st  # the forward advanced the iteration counter
    finally:
        integ.close()


def test_fp32_adjoint_error_vs_oracle():
    g = warm_dy("fp32")
    try:
        edges = g.grid
        grad, gerr, I, e, per = g.adjoint(50_000, 2, DY_PARAMS)
    finally:
        g.close()
    ref = oracle.adjoint(4, 50, 1234, 50_000, 2, DY_PARAMS, edges=edges, iteration=3)
    err = np.abs(grad - ref.grad) / (np.abs(ref.grad) + ref.grad_err)
    print("fp32 adjoint: max |dG|/(|G|+sigma_G) =", err.max())
    assert err.max() < 1e-4
    assert rel(I, ref.integral) < 2e-5


# ------------------------------------------------------------ checkpointing
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_bit_exact(precision):
    a = v.Vegas(4, 50, 99, precision=precision)
    b = v.Vegas(4, 50, 99, precision=precision)
    c = v.Vegas(4, 50, 7, precision="fp64")
    try:
        straight = [a.iterate(5000, 1, v.VEGAS_DY, DY_PARAMS)[3] for _ in range(5)]
        first = [b.iterate(5000, 1, v.VEGAS_DY, DY_PARAMS)[3] for _ in range(2)]
        blob = b.state()
        c.restore(blob)  # another context, other seed and precision: all restored
        rest = [c.iterate(5000, 1, v.VEGAS_DY, DY_PARAMS)[3] for _ in range(3)]
        assert np.array_equal(np.concatenate(straight), np.concatenate(first + rest))
        assert np.array_equal(a.grid, c.grid)
    finally:
        a.close()
        b.close()
        c.close()


def test_state_blob_rejected_for_other_shape():
    a = v.Vegas(4, 50, 1)
    b = v.Vegas(4, 40, 1)
    try:
        with pytest.raises(v.VegasError) as ei:
            b.restore(a.state())
        assert ei.value.status == v.VEGAS_ESTATE
        with pytest.raises(v.VegasError):
            b.restore(b.state()[:10])
    finally:
        a.close()
        b.close()


# ------------------------------------------------------------------- grids
def test_grid_set_get_and_validation():
    g = v.Vegas(3, 10, 1)
    try:
        rng = np.random.default_rng(0)
        e = np.concatenate([np.zeros((3, 1)), np.sort(rng.uniform(0, 1, (3, 9)), axis=1),
                            np.ones((3, 1))], axis=1)
        g.grid = e
        assert np.array_equal(g.grid, e)
        bad = e.copy()
        bad[1, 4] = bad[1, 5]  # not strictly increasing
        with pytest.raises(v.VegasError) as ei:
            g.grid = bad
        assert ei.value.status == v.VEGAS_EGRID
        bad = e.copy()
        bad[2, -1] = 0.999
        with pytest.raises(v.VegasError):
            g.grid = bad
        assert np.array_equal(g.grid, e)  # unchanged after an error
        # the set grid is used: one frozen iteration equals the oracle on it
        g.set(v.VEGAS_OPT_ADAPT, 0)
        per = g.iterate(4096 + 3, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)[3]
        ref = oracle.iterate(3, 10, 1, 4099, 1, oracle.GAUSS, GAUSS_PARAMS, edges=e, adapt=False)
        assert rel(per, ref.per_iter) < 1e-12
    finally:
        g.close()


# --------------------------------------------------------- special values
def test_nonfinite_weights_counted_and_reported():
    p = list(DY_PARAMS)
    p[9] = 1e300  # N^2 overflows: every weight is infinite
    g = v.Vegas(4, 20, 3)
    try:
        with pytest.raises(v.VegasError) as ei:
            g.iterate(3000, 1, v.VEGAS_DY, p)
        assert ei.value.status == v.VEGAS_ENONFINITE
        g.set(v.VEGAS_OPT_NONFINITE, 1)
        I, e, c, per, st = g.iterate(3000, 1, v.VEGAS_DY, p)
        assert st == v.VEGAS_OK and I == 0.0
        v.vegas_launch(g.h, 3000, 2, v.VEGAS_DY, p)
        out = v.vegas_fetch(g.h, 2, allow_nonfinite=True)
        assert out[4] == 6000
    finally:
        g.close()
    ref = oracle.iterate(4, 20, 3, 3000, 1, oracle.DY, p)
    assert ref.nonfinite == 3000


def test_zero_weights_leave_grid():
    g = v.Vegas(5, 20, 3)
    try:
        I, e, c, per, _ = g.iterate(5000, 2, v.VEGAS_EE3J, (0.4, 91.1876))
        assert I == 0.0 and e == 0.0 and c == 0.0
        assert np.array_equal(g.grid, oracle.uniform_edges(5, 20))
    finally:
        g.close()


@pytest.mark.parametrize("ndim,nbins,ncall,iid,params", [
    (1, 7, 2, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (1, 2, 3000, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (2, 3, 1023, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (4, 1024, 1024, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (16, 256, 1025, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (13, 50, 4100, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (7, 31, 3000, v.VEGAS_DY, DY_PARAMS),
    (12, 100, 2500, v.VEGAS_EE3J, EE3J_PARAMS),
])
def test_edge_sizes_match_oracle(ndim, nbins, ncall, iid, params):
    """Each iteration against the oracle started from the same grid.  Sparse
    sampling of a peaked integrand shrinks some bins to ~1e-6 of the unit
    interval; the next iteration's Jacobian then magnifies an edge's last-bit
    difference by 1/width, so results are compared iteration by iteration
    (each from the GPU's grid) rather than through a chain of refinements."""
    g = v.Vegas(ndim, nbins, 5)
    try:
        I, e, c, per, _ = g.iterate(ncall, 3, iid, params)
    finally:
        g.close()
    g = v.Vegas(ndim, nbins, 5)
    try:
        grids, steps = [g.grid], []
        for _ in range(3):
            steps.append(g.iterate(ncall, 1, iid, params)[3][0])
            grids.append(g.grid)
    finally:
        g.close()
    # a stage equals the same iterations one at a time, bit for bit
    assert np.array_equal(per, np.array(steps))
    for k in range(3):
        ref = oracle.iterate(ndim, nbins, 5, ncall, 1, iid, params, edges=grids[k], iteration=k)
        assert rel(per[k], ref.per_iter[0]) < 1e-12, k
        assert np.max(np.abs(grids[k + 1] - ref.edges)) < 1e-12, k
    Io, eo, co = oracle.combine(per[:, 0], per[:, 1])
    assert rel(I, Io) < 1e-12 and rel(e, eo) < 1e-12
    assert abs(c - co) <= 1e-10 * max(1.0, co)


def test_bin_sums_keep_relative_precision_over_wide_range():
    """A narrow Gaussian sampled sparsely: its bin sums of w^2 span far more
    than any fixed-point window, yet each must keep its relative precision --
    the compression of the refinement gives even a bin with rho = 1e-100 a
    visible share of the new grid."""
    ndim, nbins, ncall, params = 6, 400, 3000, (0.05,)
    g = v.Vegas(ndim, nbins, 77)
    try:
        g.iterate(ncall, 1, v.VEGAS_GAUSS, params)
        sums, edges = g.last_sums(), g.grid
    finally:
        g.close()
    ref = oracle.iterate(ndim, nbins, 77, ncall, 1, v.VEGAS_GAUSS, params, want_sums=True)
    d_ref, d_gpu = ref.sums[2:], sums[2:]
    nz = d_ref != 0
    assert d_ref[nz].max() / d_ref[nz].min() > 1e60
    assert np.array_equal(d_gpu == 0, ~nz)
    assert rel(d_gpu[nz], d_ref[nz]) < 1e-12
    assert np.max(np.abs(edges - ref.edges)) < 1e-12


def test_invalid_arguments():
    with pytest.raises(v.VegasError):
        v.vegas_init(0, 10, 1)
    with pytest.raises(v.VegasError):
        v.vegas_init(17, 10, 1)
    with pytest.raises(v.VegasError):
        v.vegas_init(4, 1, 1)
    with pytest.raises(v.VegasError):
        v.vegas_init(8, 1000, 1)  # 8000 > 4096 bins in total
    g = v.Vegas(4, 10, 1)
    try:
        for args in [(1, 1, v.VEGAS_GAUSS, GAUSS_PARAMS), (100, 0, v.VEGAS_GAUSS, GAUSS_PARAMS),
                     (100, 1, 9, GAUSS_PARAMS), (100, 1, v.VEGAS_GAUSS, (0.1, 0.2, 0.3)),
                     (100, 1, v.VEGAS_GAUSS, (-0.1,)), (100, 1, v.VEGAS_EE3J, EE3J_PARAMS),
                     (100, 1, v.VEGAS_DY, DY_PARAMS[:9])]:
            with pytest.raises(v.VegasError) as ei:
                g.iterate(*args)
            assert ei.value.status == v.VEGAS_EINVAL
        with pytest.raises(v.VegasError):
            g.adjoint(100, 1, GAUSS_PARAMS, v.VEGAS_GAUSS)
        with pytest.raises(v.VegasError):
            g.set(v.VEGAS_OPT_EPT, 3)
        # the context still works after the errors
        g.iterate(1000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)
    finally:
        g.close()


# ---------------------------------------------------------- other features
def test_fp32_single_events_close_to_fp64():
    g = v.Vegas(4, 100, 1234, precision="fp32")
    try:
        g.iterate(20_000, 2, v.VEGAS_DY, DY_PARAMS)
        edges = g.grid
        ev = np.arange(0, 100_000, 37, dtype=np.int64)
        w, bins = g.eval_events(v.VEGAS_DY, DY_PARAMS, 9, ev)
    finally:
        g.close()
    for j, e in enumerate(ev[:300]):
        wo, bo, _ = oracle.event(oracle.DY, 4, 100, edges, DY_PARAMS, 1234, 9, 0, int(e))
        assert np.array_equal(bins[j], bo)
        assert abs(w[j] - wo) <= 5e-5 * abs(wo) + 1e-30


def test_batch_id_and_seed_change_events():
    outs = {}
    for seed, batch in [(1, 0), (1, 0), (2, 0), (1, 5)]:
        g = v.Vegas(4, 20, seed)
        try:
            g.set(v.VEGAS_OPT_BATCH_ID, batch)
            outs.setdefault((seed, batch), []).append(g.iterate(3000, 1, v.VEGAS_GAUSS,
                                                                GAUSS_PARAMS)[3])
        finally:
            g.close()
    a, b = outs[(1, 0)]
    assert np.array_equal(a, b)
    assert not np.array_equal(a, outs[(2, 0)][0])
    assert not np.array_equal(a, outs[(1, 5)][0])
    ref = oracle.iterate(4, 20, 1, 3000, 1, oracle.GAUSS, GAUSS_PARAMS, batch=5)
    assert rel(outs[(1, 5)][0], ref.per_iter) < 1e-12


def test_torch_workspace_and_stream_give_same_results():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    a = v.Vegas(4, 50, 11)
    b = v.Vegas(4, 50, 11, torch_workspace=True, stream=s.cuda_stream)
    try:
        ra = a.iterate(30_000, 3, v.VEGAS_DY, DY_PARAMS)
        with torch.cuda.stream(s):
            rb = b.iterate(30_000, 3, v.VEGAS_DY, DY_PARAMS)
        assert np.array_equal(ra[3], rb[3])
        assert np.array_equal(a.grid, b.grid)
    finally:
        a.close()
        b.close()


def test_launch_fetch_and_kernel_timing():
    g = v.Vegas(4, 50, 3)
    try:
        g.set(v.VEGAS_OPT_TIMING, 1)
        v.vegas_launch(g.h, 50_000, 4, v.VEGAS_DY, DY_PARAMS)
        I, e, c, per, nf, st = v.vegas_fetch(g.h, 4)
        assert st == v.VEGAS_OK and nf == 0 and per.shape == (4, 2)
        for kid in (v.VEGAS_KERNEL_FILL, v.VEGAS_KERNEL_REDUCE):
            ms, n = v.vegas_kernel_time(g.h, kid, reset=True)
            assert n == 4 and ms > 0.0
        # the grid refinement runs inside the reduce kernel
        assert v.vegas_kernel_time(g.h, v.VEGAS_KERNEL_REFINE) == (0.0, 0)
        assert v.vegas_get_ept(g.h) in (1, 2, 4, 8)
    finally:
        g.close()
