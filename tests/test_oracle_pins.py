"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU. Each test names the passage it follows. None of them re-types the
oracle's own formula: they use hand-worked fixtures (tests/golden), an
independently assembled sparse D, closed-form spectra, textbook special cases
(1-D Newton, closed-form lasso), generic optimisers (L-BFGS-B, subgradient),
invariances and finite differences.
"""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import brute
from paper_1905_13408_gb300 import synth


def P(orc, shape, **kw):
    return orc.Params(tuple(shape), **kw)


# ---------- closed forms (Eq. 14, 16, 21) ----------

def test_soft_threshold_table(orc):
    """Eq. 21: hand-worked cases in tests/golden/soft_threshold.txt."""
    for z, t, want in golden("soft_threshold.txt"):
        assert orc.soft(z, t) == pytest.approx(want, abs=1e-15), (z, t)


def test_huber_table(orc):
    """Eq. 14 closed form and Eq. 16 gradient: tests/golden/huber.txt."""
    for z0, z1, z2, mu, val, g0, g1, g2 in golden("huber.txt"):
        assert orc.huber((z0, z1, z2), mu) == pytest.approx(val, rel=1e-14, abs=1e-18)
        np.testing.assert_allclose(orc.huber_grad((z0, z1, z2), mu), [g0, g1, g2], rtol=1e-14, atol=1e-15)


def test_huber_properties(orc):
    """Eq. 14/16: continuity at |z| = mu, gradient equals a central difference of
    the value, gradient inside the unit ball (the dual set Q_d of Eq. 13)."""
    rng = np.random.default_rng(0)
    mu = 1e-3
    for _ in range(200):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        lo = orc.huber(d * mu * (1 - 1e-12), mu)
        hi = orc.huber(d * mu * (1 + 1e-12), mu)
        assert abs(lo - hi) < 1e-14
        z = rng.standard_normal(3) * 10 ** rng.uniform(-4.5, 0)
        g = orc.huber_grad(z, mu)
        assert np.linalg.norm(g) <= 1 + 1e-15
        h = 1e-7 * max(np.linalg.norm(z), mu)
        fd = [(orc.huber(z + h * e, mu) - orc.huber(z - h * e, mu)) / (2 * h) for e in np.eye(3)]
        np.testing.assert_allclose(g, fd, atol=1e-6)


# ---------- linear operators (Eq. 12, 17) ----------

def test_grad_hand_example(orc):
    """Eq. 12 on a 2x2x2 volume, differences worked by hand."""
    rows = golden("grad_2x2x2.txt")
    x = np.zeros((2, 2, 2))
    want = np.zeros((3, 2, 2, 2))
    for z, y, xx, val, dx, dy, dz in rows:
        z, y, xx = int(z), int(y), int(xx)
        x[z, y, xx] = val
        want[:, z, y, xx] = (dx, dy, dz)
    np.testing.assert_array_equal(orc.grad(x), want)


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 7, 9), (1, 6, 2), (4, 4, 4)])
def test_grad_matches_kronecker_matrix(orc, shape):
    """Eq. 12 from index loops equals the Kronecker-assembled sparse D."""
    x = synth.random_volume(shape, 1)
    D = brute.d_matrix(shape)
    np.testing.assert_allclose(orc.grad(x).ravel(), D @ x.ravel(), rtol=0, atol=1e-14)
    u = synth.random_volume((3,) + shape, 2)
    np.testing.assert_allclose(orc.div(u).ravel(), D.T @ u.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(5, 7, 9), (33, 17, 6), (2, 3, 1)])
def test_adjoint_identity(orc, shape):
    """Eq. 17 is the adjoint of Eq. 12: <Dx, u> = <x, D^T u>."""
    x = synth.random_volume(shape, 3)
    u = synth.random_volume((3,) + shape, 4)
    lhs = float((orc.grad(x) * u).sum())
    rhs = float((x * orc.div(u)).sum())
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.abs(x).sum())


def test_constant_has_zero_gradient_and_tv(orc):
    """A constant volume has D x = 0, so its smoothed TV (Eq. 14) is zero."""
    x = np.full((6, 5, 4), 3.25)
    assert np.abs(orc.grad(x)).max() == 0.0
    p = P(orc, x.shape, lambda_l1=0.0, lambda_tv=1.0)
    obj = orc.objective(x, x, np.ones_like(x), None, None, p)
    assert obj[2] == 0.0 and obj[0] == 0.0


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 7), (8, 2, 6)])
def test_spectrum_of_DtD(orc, shape):
    """D^T D is the Neumann grid Laplacian; its largest eigenvalue is
    sum_a 4 sin^2(pi (n_a - 1) / (2 n_a)) < 12 (the bound behind L)."""
    want = sum(4 * math.sin(math.pi * (n - 1) / (2 * n)) ** 2 for n in shape if n > 1)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(shape)
    lam = 0.0
    for _ in range(3000):
        v = orc.div(orc.grad(v))
        lam = np.linalg.norm(v)
        v /= lam
    assert lam == pytest.approx(want, rel=1e-6)
    assert lam < 12.0


def test_tv_of_ramp_and_spike(orc):
    """Eq. 14 objective on hand-analysable volumes."""
    nz, ny, nx = 3, 4, 5
    s, mu = 0.5, 1e-3
    ramp = np.broadcast_to(s * np.arange(nx)[None, None, :], (nz, ny, nx)).copy()
    p = P(orc, (nz, ny, nx), lambda_l1=0.0, lambda_tv=1.0, mu=mu)
    tv = orc.objective(ramp, ramp, np.ones_like(ramp), None, None, p)[2]
    assert tv == pytest.approx((nx - 1) * ny * nz * (s - mu / 2), rel=1e-14)
    # single interior spike of height h: |Dx| = h sqrt(3) at the spike and h
    # at its three forward neighbours
    h = 2.0
    spike = np.zeros((nz, ny, nx))
    spike[1, 1, 1] = h
    tv = orc.objective(spike, spike, np.ones_like(spike), None, None, p)[2]
    assert tv == pytest.approx((h * math.sqrt(3) - mu / 2) + 3 * (h - mu / 2), rel=1e-14)


def test_objective_hand_example(orc):
    """Eq. 11 objective (data term of Eq. 28/31, weighted l1, weighted smoothed
    TV of Eq. 14) with non-uniform om1 and omtv on a 2x1x2 volume worked by
    hand (tests/golden/objective_2x1x2.txt)."""
    rows = golden("objective_2x1x2.txt")
    vox = [r for r in rows if len(r) == 8]
    (lam1, lamtv, mu, data, l1, tv, total), = [r for r in rows if len(r) == 7]
    shape = (2, 1, 2)
    x, b, w, om1, omtv = (np.zeros(shape) for _ in range(5))
    for z, y, xx, xv, bv, wv, o1, ot in vox:
        q = (int(z), int(y), int(xx))
        x[q], b[q], w[q], om1[q], omtv[q] = xv, bv, wv, o1, ot
    p = P(orc, shape, lambda_l1=lam1, lambda_tv=lamtv, mu=mu)
    got = orc.objective(x, b, w, om1, omtv, p)
    np.testing.assert_allclose(got, [data, l1, tv, total], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("shape", [(4, 5, 6), (7, 3, 2), (1, 9, 4)])
def test_objective_parts_match_sparse_evaluation(orc, shape):
    """Each part of the Eq. 11 objective (data, om1-weighted l1, omtv-weighted
    smoothed TV) against a separate evaluation from the Kronecker-assembled D,
    on random x straddling mu and random non-uniform weights (as in rounds
    2 and 3, where Eq. 11's weights come from the previous round's iterate)."""
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) * 10 ** rng.uniform(-3.5, 0, shape)
    b = rng.standard_normal(shape)
    w = rng.uniform(0.3, 4, shape)
    om1 = rng.uniform(0.01, 1, shape)
    omtv = rng.uniform(0.01, 1, shape)
    p = P(orc, shape, lambda_l1=0.07, lambda_tv=0.13, mu=1e-3)
    got = orc.objective(x, b, w, om1, omtv, p)
    want = brute.Problem(b, w, om1, omtv, p.lambda_l1, p.lambda_tv, p.mu).parts(x)
    np.testing.assert_allclose(got[:3], want, rtol=1e-12, atol=0)
    assert got[3] == pytest.approx(sum(want), rel=1e-12)
    # the weights matter: dropping either one changes its part
    unw = brute.Problem(b, w, None, None, p.lambda_l1, p.lambda_tv, p.mu).parts(x)
    assert abs(unw[1] - got[1]) > 1e-3 * got[1] and abs(unw[2] - got[2]) > 1e-3 * got[2]


def test_reweight_spike(orc):
    """Eq. 11 weights scaled by eps (Sec. 2.5) on a single spike."""
    eps, eps_tv, h = 1e-3, 2e-3, 0.7
    x = np.zeros((4, 4, 4))
    x[2, 1, 2] = -h
    p = P(orc, x.shape, eps=eps, eps_tv=eps_tv)
    om1, omtv, st = orc.reweight(x, p)
    assert om1[2, 1, 2] == pytest.approx(eps / (h + eps), rel=1e-15)
    assert np.all(np.delete(om1.ravel(), np.ravel_multi_index((2, 1, 2), x.shape)) == 1.0)
    assert omtv[2, 1, 2] == pytest.approx(eps_tv / (h * math.sqrt(3) + eps_tv), rel=1e-14)
    for q in [(2, 1, 3), (2, 2, 2), (3, 1, 2)]:
        assert omtv[q] == pytest.approx(eps_tv / (h + eps_tv), rel=1e-14)
    assert st[0] == 1.0 and st[1] == 1.0
    assert st[2] == pytest.approx(63 + eps / (h + eps), rel=1e-14)


def test_lipschitz_bound_holds(orc):
    """|grad f(x) - grad f(y)| <= L |x - y| with L = max w + 12 lambda_tv max omtv / mu."""
    rng = np.random.default_rng(7)
    shape = (6, 5, 7)
    w = synth.random_volume(shape, 8, positive=True)
    b = synth.random_volume(shape, 9)
    omtv = rng.uniform(0.1, 1.0, shape)
    p = P(orc, shape, lambda_tv=0.3, mu=0.05)
    L = orc.lipschitz(w, omtv.max(), p)
    for _ in range(20):
        x = rng.standard_normal(shape) * 0.1
        y = x + rng.standard_normal(shape) * 1e-3
        d = np.linalg.norm(orc.grad_f(x, b, w, omtv, p) - orc.grad_f(y, b, w, omtv, p))
        assert d <= L * np.linalg.norm(x - y) * (1 + 1e-12)


def test_lipschitz_bound_is_valid_and_tight(orc):
    """Where every |Dx| < mu the smooth part is quadratic with Hessian
    diag(w) + lambda_tv/mu D^T diag(omtv) D. Power iteration on finite
    differences of grad f around x = 0 finds its top eigenvalue, which must
    not exceed L, and for uniform weights on 8^3 is within 5% of it
    (sum_a 4 sin^2(7 pi / 16) = 11.54 of the bound's 12)."""
    shape = (8, 8, 8)
    b = np.zeros(shape)
    w = np.full(shape, 1.5)
    p = P(orc, shape, lambda_tv=0.2, mu=0.01)
    L = orc.lipschitz(w, 1.0, p)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(shape)
    h = 1e-6 * p.mu
    g0 = orc.grad_f(np.zeros(shape), b, w, None, p)
    lam = 0.0
    for _ in range(2000):
        v /= np.linalg.norm(v)
        hv = (orc.grad_f(h * v, b, w, None, p) - g0) / h
        lam = float((v * hv).sum())
        v = hv
    assert lam <= L * (1 + 1e-6)
    assert lam >= 0.95 * L


def test_grad_f_matches_finite_difference_of_objective(orc):
    """The smooth part's gradient (Eq. 15-17 plus the data term) against a
    central difference of the objective value."""
    shape = (4, 5, 3)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(shape)
    w = rng.uniform(0.5, 2, shape)
    omtv = rng.uniform(0.2, 1, shape)
    p = P(orc, shape, lambda_l1=0.0, lambda_tv=0.4, mu=0.3)
    x = rng.standard_normal(shape)
    g = orc.grad_f(x, b, w, omtv, p)
    h = 1e-6
    for v in range(0, x.size, 7):
        e = np.zeros(x.size)
        e[v] = h
        e = e.reshape(shape)
        fp = orc.objective(x + e, b, w, None, omtv, p)[3]
        fm = orc.objective(x - e, b, w, None, omtv, p)[3]
        assert g.ravel()[v] == pytest.approx((fp - fm) / (2 * h), abs=2e-7)


# ---------- special cases of the solve ----------

def test_data_only_closed_form(orc):
    """lambda_tv = 0, uniform w, tau = 1/w: one plain step from any x gives the
    weighted lasso solution sign(b) max(|b| - lambda_l1 om1 / w, 0)."""
    shape = (5, 6, 7)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(shape)
    wv = 2.5
    w = np.full(shape, wv)
    om1 = rng.uniform(0.1, 1, shape)
    p = P(orc, shape, lambda_l1=0.3, lambda_tv=0.0, momentum="ista")
    x0 = rng.standard_normal(shape)
    x1 = orc.step(x0, x0, 0.0, 1.0 / wv, b, w, om1, None, p)
    want = np.sign(b) * np.maximum(np.abs(b) - 0.3 * om1 / wv, 0)
    np.testing.assert_allclose(x1, want, rtol=0, atol=1e-15)


def test_no_regularisation_converges_to_b(orc):
    """lambda_l1 = lambda_tv = 0: the minimiser is b."""
    shape = (6, 6, 6)
    rng = np.random.default_rng(13)
    b = rng.standard_normal(shape)
    w = rng.uniform(0.5, 3, shape)
    p = P(orc, shape, lambda_l1=0.0, lambda_tv=0.0)
    r = orc.solve(b, w, p, rounds=1, iters=300)
    np.testing.assert_allclose(r.x, b, atol=1e-12)


def test_tv_1d_reducible_matches_newton(orc):
    """b, w constant along y and z: the 3-D problem is ny*nz copies of a 1-D
    Huber-TV problem (lambda_l1 = 0), solved independently by Newton."""
    nz, ny, nx = 3, 2, 24
    rng = np.random.default_rng(14)
    b1 = np.cumsum(rng.standard_normal(nx)) * 0.3
    w1 = rng.uniform(0.5, 2.0, nx)
    b = np.broadcast_to(b1, (nz, ny, nx)).copy()
    w = np.broadcast_to(w1, (nz, ny, nx)).copy()
    mu, lam = 0.05, 0.2
    p = P(orc, b.shape, lambda_l1=0.0, lambda_tv=lam, mu=mu, eps=1e30, eps_tv=1e30)
    r = orc.solve(b, w, p, rounds=1, iters=20000, with_hist=False)
    want = brute.tv1d_newton(b1, w1, None, lam, mu)
    for z in range(nz):
        for y in range(ny):
            np.testing.assert_allclose(r.x[z, y], want, atol=1e-11)


def test_axis_permutation_symmetry(orc):
    """The three axes enter Eq. 12/17 the same way: transposing b and w
    transposes the result."""
    vol = synth.make_volume((6, 7, 8), blobs=6, radius=2.5, seed=15)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    p = P(orc, b.shape, mu=0.02)
    x = orc.solve(b, w, p, rounds=2, iters=40, with_hist=False).x
    for perm in [(2, 1, 0), (1, 0, 2), (0, 2, 1)]:
        bt, wt = np.ascontiguousarray(b.transpose(perm)), np.ascontiguousarray(w.transpose(perm))
        xt = orc.solve(bt, wt, P(orc, bt.shape, mu=0.02), rounds=2, iters=40, with_hist=False).x
        np.testing.assert_allclose(xt, x.transpose(perm), atol=1e-12)


def test_scaling_invariance(orc):
    """Scaling b by c and (mu, eps, eps_tv, lambda_l1, lambda_tv) by c scales
    every iterate by c and F by c^2 with tau unchanged (Eq. 11, 14, 16, 21);
    c = 2 is exact in binary floating point."""
    vol = synth.make_volume((8, 8, 8), blobs=5, radius=2.0, seed=16)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    p1 = P(orc, b.shape)
    c = 2.0
    p2 = P(orc, b.shape, lambda_l1=p1.lambda_l1 * c, lambda_tv=p1.lambda_tv * c, mu=p1.mu * c,
           eps=p1.eps * c, eps_tv=p1.eps_tv * c)
    r1 = orc.solve(b, w, p1, rounds=2, iters=25)
    r2 = orc.solve(b * c, w, p2, rounds=2, iters=25)
    np.testing.assert_array_equal(r2.x, c * r1.x)
    np.testing.assert_array_equal(r2.hist, c * c * r1.hist)
    np.testing.assert_array_equal(r2.rstats[:, 5], r1.rstats[:, 5])


def test_ista_is_monotone(orc):
    """With beta = 0 (the paper's plain Eq. 20-21 update) and step 1/L, the
    round objective never increases."""
    vol = synth.make_volume((12, 12, 12), blobs=8, radius=4, seed=17)
    p = P(orc, vol.b.shape, momentum="ista")
    r = orc.solve(vol.b, vol.w, p, rounds=3, iters=60)
    tot = r.hist[:, :, 3]
    assert np.all(np.diff(tot, axis=1) <= 1e-12 * np.abs(tot[:, 1:]))


def test_fista_rate_bound(orc):
    """FISTA: F(x_k) - F* <= 2 L |x_0 - x*|^2 / (k+1)^2 (Beck-Teboulle)."""
    vol = synth.make_volume((4, 4, 4), blobs=3, radius=1.0, seed=18)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    p = P(orc, b.shape, mu=0.01, lambda_tv=0.05)
    r = orc.solve(b, w, p, rounds=1, iters=400)
    prob = brute.Problem(b, w, r.om1, r.omtv, p.lambda_l1, p.lambda_tv, p.mu)
    xs, fs = prob.lbfgs()
    L = r.rstats[0, 4]
    k = np.arange(400)
    bound = 2 * L * (xs ** 2).sum() / (k + 1) ** 2
    assert np.all(r.hist[0, :, 3] - fs <= bound + 1e-12)


def _tiny_problem(orc, seed=19, mu=1e-3, lam_tv=0.1, lam_l1=0.05):
    vol = synth.make_volume((4, 4, 4), blobs=3, radius=1.0, seed=seed)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    p = P(orc, b.shape, mu=mu, lambda_tv=lam_tv, lambda_l1=lam_l1)
    return b, w, p


def test_4cubed_optimality_lbfgs_kkt(orc):
    """4^3 round-1 problem at the paper-scale parameters: the oracle run long
    reaches the L-BFGS-B minimiser of the split problem and satisfies the KKT
    conditions of the weighted lasso + smoothed TV objective."""
    b, w, p = _tiny_problem(orc)
    r = orc.solve(b, w, p, rounds=1, iters=60000, with_hist=False)
    prob = brute.Problem(b, w, r.om1, r.omtv, p.lambda_l1, p.lambda_tv, p.mu)
    xs, fs = prob.lbfgs()
    f_orc = prob.F(r.x)
    assert abs(f_orc - fs) <= 1e-10 * abs(fs)
    assert np.abs(r.x - xs).max() <= 1e-5
    assert prob.kkt_residual(r.x) <= 1e-9


def test_4cubed_subgradient_long_run(orc):
    """North-star pin: a long-run brute-force subgradient solve of the same
    4^3 problem agrees with the oracle's solution (moderate mu so the
    subgradient method converges in reasonable time)."""
    b, w, p = _tiny_problem(orc, mu=0.05)
    r = orc.solve(b, w, p, rounds=1, iters=20000, with_hist=False)
    prob = brute.Problem(b, w, r.om1, r.omtv, p.lambda_l1, p.lambda_tv, p.mu)
    xg, fg = prob.subgradient(iters=60000)
    f_orc = prob.F(r.x)
    assert f_orc <= fg + 1e-12
    assert fg - f_orc <= 1e-6 * abs(f_orc)
    assert np.abs(xg - r.x).max() <= 2e-3


def test_certificate_bounds_gap(orc):
    """Strong convexity (m = min w): F(x+) - F* <= |r|^2 / (2 m), r the
    subgradient at x+ built from the prox step."""
    b, w, p = _tiny_problem(orc, mu=0.01)
    r = orc.solve(b, w, p, rounds=1, iters=30, with_hist=False)
    prob = brute.Problem(b, w, r.om1, r.omtv, p.lambda_l1, p.lambda_tv, p.mu)
    _, fs = prob.lbfgs()
    tau = r.rstats[0, 5]
    y = r.x
    xplus = orc.step(y, y, 0.0, tau, b, w, r.om1, r.omtv, p)
    cert = orc.certificate(y, xplus, tau, b, w, r.omtv, p)
    gap = prob.F(xplus) - fs
    assert 0 <= gap <= cert / (2 * w.min()) * (1 + 1e-9) + 1e-14


def test_certificate_is_the_norm_of_a_subgradient(orc):
    """The certificate is |r|^2 for the r that the prox step makes a
    subgradient of F at x+: r - grad f(x+) = grad f(y) -> (y - x+)/tau - grad
    f(y) lies in lambda_l1 om1 d|x+| (equal to lambda_l1 om1 sign x+ where x+
    is non-zero, within that bound where it is zero), from the soft-threshold's
    optimality condition (Eq. 21), with grad f pinned on its own by finite
    differences. A random y (not a fixed point) keeps r far from zero; a large
    lambda_l1 makes the threshold zero a part of the voxels."""
    b, w, p = _tiny_problem(orc, mu=0.01, lam_l1=30.0)
    rng = np.random.default_rng(23)
    y = rng.standard_normal(b.shape)
    om1 = rng.uniform(0.3, 1.0, b.shape)
    omtv = rng.uniform(0.3, 1.0, b.shape)
    tau = 1.0 / orc.lipschitz(w, omtv.max(), p)
    xplus = orc.step(y, y, 0.0, tau, b, w, om1, omtv, p)
    assert np.count_nonzero(xplus) > 5 and np.count_nonzero(xplus == 0) > 5
    s = (y - xplus) / tau - orc.grad_f(y, b, w, omtv, p)   # the l1 part of r
    t = p.lambda_l1 * om1
    nz = xplus != 0
    np.testing.assert_allclose(s[nz], t[nz] * np.sign(xplus[nz]), rtol=1e-9, atol=1e-9)
    assert np.all(np.abs(s[~nz]) <= t[~nz] * (1 + 1e-9) + 1e-12)
    r = orc.grad_f(xplus, b, w, omtv, p) + s
    cert = orc.certificate(y, xplus, tau, b, w, omtv, p)
    assert cert == pytest.approx(float((r * r).sum()), rel=1e-12)
    assert cert > 1e-3


def test_reweighting_majorises_log_penalty(orc):
    """Sec. 2.1 (tangent majoriser of the log penalty, Eq. 9/11): with the TV
    term off, each fully solved round does not increase
    1/2 sum w (x-b)^2 + lambda_l1 eps sum log(|x| + eps)."""
    vol = synth.make_volume((6, 6, 6), blobs=4, radius=1.5, seed=20)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    eps = 0.05
    p = P(orc, b.shape, lambda_tv=0.0, lambda_l1=0.2, eps=eps)

    def phi(x):
        return 0.5 * (w * (x - b) ** 2).sum() + p.lambda_l1 * eps * np.log(np.abs(x) + eps).sum()

    x = np.zeros_like(b)
    prev = phi(x)
    for _ in range(5):
        x = orc.solve(b, w, p, rounds=1, iters=400, x0=x, with_hist=False).x
        cur = phi(x)
        assert cur <= prev + 1e-12
        prev = cur


def test_sampled_step_equals_full_step(orc):
    """The one-voxel evaluation used for sampled checks at full size agrees
    with the whole-volume step (same definitions, evaluated locally)."""
    vol = synth.make_volume((9, 10, 11), blobs=5, radius=3, seed=21)
    p = P(orc, vol.b.shape)
    rng = np.random.default_rng(22)
    xk = rng.standard_normal(vol.b.shape) * 0.3
    xkm1 = rng.standard_normal(vol.b.shape) * 0.3
    om1 = rng.uniform(0.1, 1, vol.b.shape)
    omtv = rng.uniform(0.1, 1, vol.b.shape)
    full = orc.step(xk, xkm1, 0.37, 8e-4, vol.b, vol.w, om1, omtv, p)
    idx = np.arange(vol.b.size)
    samp = orc.step_sampled(xk, xkm1, 0.37, 8e-4, vol.b, vol.w, om1, omtv, p, idx)
    np.testing.assert_allclose(samp, full.ravel(), rtol=0, atol=1e-15)


def test_beta_table(orc):
    """FISTA t-sequence: t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2; beta_0 = 0,
    beta_k -> 1, beta_k = (t_k - 1)/t_{k+1} ~ (k - 1)/(k + 2) asymptotically."""
    bt = orc.beta_table(2000)
    assert bt[0] == 0.0
    assert bt[1] == pytest.approx(((1 + math.sqrt(5)) / 2 - 1) / ((1 + math.sqrt(1 + (1 + math.sqrt(5)) ** 2)) / 2))
    assert np.all(np.diff(bt) > 0) and bt[-1] < 1
    assert bt[1999] == pytest.approx(1998 / 2001, rel=2e-3)
    assert np.all(orc.beta_table(10, "ista") == 0)


# ---------- differentiation (adjoint of K unrolled steps) ----------

def _adjoint_case(orc, shape=(8, 9, 10), K=10, seed=31):
    vol = synth.make_volume(shape, blobs=5, radius=2.5, seed=seed)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    p = P(orc, shape, mu=0.02, lambda_tv=0.1, lambda_l1=0.05)
    tau = 1.0 / orc.lipschitz(w, 1.0, p)
    x0 = np.zeros(shape)
    return vol, b, w, p, tau, x0, K


def test_adjoint_matches_central_differences(orc):
    """The FP64 adjoint of K unrolled steps (tau and weights fixed) agrees with
    central differences (step 1e-4) of L = |x_K - phantom|^2 in 64 random
    single-voxel directions of b and w and in both scalars; directions whose
    perturbed runs cross a soft-threshold kink in a different place are left
    out, as the map is not differentiable across them."""
    vol, b, w, p, tau, x0, K = _adjoint_case(orc)
    ph = vol.phantom.astype(np.float64)

    def loss(bb, ww, pp):
        xk, act = orc.unrolled_active(bb, ww, None, None, tau, K, x0, pp)
        return float(((xk - ph) ** 2).sum()), act

    L0, act0 = loss(b, w, p)
    xK = orc.unrolled(b, w, None, None, tau, K, x0, p)
    gb, gw, gs = orc.backward(b, w, None, None, tau, K, x0, 2 * (xK - ph), p)
    rng = np.random.default_rng(32)
    h = 1e-4
    checked = 0
    for which, grad, base in (("b", gb, b), ("w", gw, w)):
        for v in rng.choice(b.size, 32, replace=False):
            e = np.zeros(b.size)
            e[v] = h
            e = e.reshape(b.shape)
            if which == "b":
                (lp, ap), (lm, am) = loss(b + e, w, p), loss(b - e, w, p)
            else:
                (lp, ap), (lm, am) = loss(b, w + e, p), loss(b, w - e, p)
            if ap != act0 or am != act0:
                continue
            fd = (lp - lm) / (2 * h)
            assert grad.ravel()[v] == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, v)
            checked += 1
    assert checked >= 48
    # a scalar moves every threshold at once, so a step of 1e-4 may cross a
    # kink somewhere; the step is shrunk until the active set is unchanged
    for i, name in enumerate(("lambda_l1", "lambda_tv")):
        done = False
        for hs in (1e-4, 1e-5, 1e-6, 1e-7):
            hp = P(orc, b.shape, mu=p.mu, lambda_tv=p.lambda_tv, lambda_l1=p.lambda_l1)
            hm = P(orc, b.shape, mu=p.mu, lambda_tv=p.lambda_tv, lambda_l1=p.lambda_l1)
            setattr(hp, name, getattr(p, name) + hs)
            setattr(hm, name, getattr(p, name) - hs)
            (lp, ap), (lm, am) = loss(b, w, hp), loss(b, w, hm)
            if ap == act0 and am == act0:
                assert gs[i] == pytest.approx((lp - lm) / (2 * hs), rel=1e-6), name
                done = True
                break
        assert done, name


def test_unrolled_kink_counts(orc):
    """The counting run used to exclude kink-crossing directions: same x_K and
    threshold count as the plain unrolled run; on a constant problem every
    difference is 0, so every voxel-step is on the quadratic branch of the
    smoothed norm (Eq. 14/16), and with a large threshold none passes."""
    vol, b, w, p, tau, x0, K = _adjoint_case(orc)
    xa, act = orc.unrolled_active(b, w, None, None, tau, K, x0, p)
    xc, (passes, quad) = orc.unrolled_counts(b, w, None, None, tau, K, x0, p)
    np.testing.assert_array_equal(xa, xc)
    assert passes == act and 0 < quad < b.size * K
    shape = b.shape
    pc = P(orc, shape, mu=0.02, lambda_tv=0.1, lambda_l1=10.0)
    _, (passes, quad) = orc.unrolled_counts(np.full(shape, 0.7), np.full(shape, 2.0), None, None, 0.1, K,
                                            x0, pc)
    assert quad == b.size * K and passes == 0


def test_adjoint_identity_of_one_linear_step(orc):
    """With lambda_l1 = 0 and every |Dy| below mu one step is linear in
    (x_k, x_{k-1}, b): the adjoint's b-gradient equals tau w g for a loss
    <g, x_1> (transposed-operand check)."""
    shape = (5, 6, 7)
    rng = np.random.default_rng(33)
    b = 1e-5 * rng.standard_normal(shape)
    w = rng.uniform(0.5, 2, shape)
    p = P(orc, shape, mu=1.0, lambda_tv=0.3, lambda_l1=0.0)
    tau = 1.0 / orc.lipschitz(w, 1.0, p)
    g = rng.standard_normal(shape)
    gb, gw, gs = orc.backward(b, w, None, None, tau, 1, np.zeros(shape), g, p)
    np.testing.assert_allclose(gb, tau * w * g, rtol=1e-12, atol=1e-15)


def test_gradient_restart_converges_faster(orc):
    """Gradient restart of the extrapolation (O'Donoghue-Candes): the solve
    reaches the same L-BFGS-B minimiser, in fewer steps than plain FISTA on an
    ill-conditioned 6^3 problem (a restart test with the wrong sign restarts
    every step and is slower)."""
    vol = synth.make_volume((6, 6, 6), blobs=4, radius=1.5, seed=34)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    base = dict(mu=0.005, lambda_tv=0.1, lambda_l1=0.05)
    plain = orc.solve(b, w, P(orc, b.shape, **base), 1, 1500)
    rst = orc.solve(b, w, P(orc, b.shape, restart=True, **base), 1, 1500)
    prob = brute.Problem(b, w, rst.om1, rst.omtv, base["lambda_l1"], base["lambda_tv"], base["mu"])
    _, fs = prob.lbfgs()
    assert prob.F(rst.x) - fs <= 1e-9 * abs(fs)

    def first_within(h, tol):
        gap = (h[0, :, 3] - fs) / abs(fs)
        idx = np.nonzero(gap <= tol)[0]
        return idx[0] if len(idx) else 10 ** 9

    assert first_within(rst.hist, 1e-6) < first_within(plain.hist, 1e-6)


# ---------- implicit-gradient term (Eq. 22 / Eq. 31) ----------

def test_gamma_term_folds_into_data_and_weight(orc):
    """gamma |x - a|^2 added to 1/2 w (x - b)^2 equals 1/2 w' (x - b')^2 + const
    with w' = w + 2 gamma, b' = (w b + 2 gamma a)/w': the oracle's direct
    implementation of Eq. 22 and a gamma-free solve on (b', w') produce the
    same iterates and objective differences."""
    shape = (7, 8, 9)
    vol = synth.make_volume(shape, blobs=5, radius=2.5, seed=35)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)
    a = np.random.default_rng(36).standard_normal(shape) * 0.3
    g = 0.7
    pg = P(orc, shape, mu=0.02, gamma=g, anchor=a)
    r1 = orc.solve(b, w, pg, 2, 40)
    w2 = w + 2 * g
    b2 = (w * b + 2 * g * a) / w2
    r2 = orc.solve(b2, w2, P(orc, shape, mu=0.02), 2, 40)
    np.testing.assert_allclose(r1.x, r2.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.diff(r1.hist[..., 3], axis=1), np.diff(r2.hist[..., 3], axis=1), atol=1e-9)


def test_gamma_to_infinity_pins_the_anchor(orc):
    """As gamma grows the minimiser approaches the anchor (the quadratic
    term dominates): |x* - a| = O(1/gamma)."""
    shape = (5, 6, 7)
    vol = synth.make_volume(shape, blobs=4, radius=2, seed=37)
    a = np.random.default_rng(38).standard_normal(shape)
    errs = []
    for g in (1e2, 1e3):
        r = orc.solve(vol.b, vol.w, P(orc, shape, mu=0.02, gamma=g, anchor=a), 1, 400, with_hist=False)
        errs.append(np.abs(r.x - a).max())
    assert errs[1] < errs[0] / 5 and errs[1] < 1e-2
