"""Pins of the alternative readings of the paper that the oracle carries as
flags (no GPU): forward instead of backward differences (Eq. 12), a periodic
instead of a Neumann boundary (the paper is silent), and the TV weight after
the divergence as Eq. 20 prints it instead of inside it.

Each pin is a property that the mathematics fixes for that reading, not a
restatement of the code: adjointness of D and D^T, the exact symmetries that
relate the readings (reversing the axes turns forward differences into
backward ones; a periodic solve commutes with circular shifts), the spectral
norm of the periodic D^T D, and whether the TV "gradient" is a gradient at
all (symmetric Jacobian) under each weighting.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1905_13408_gb300 import synth

READINGS = list(itertools.product(("backward", "forward"), ("neumann", "periodic")))
HYPER = dict(lambda_l1=0.05, lambda_tv=0.1, mu=0.02, eps=1e-3, eps_tv=1e-3)


def params(shape, difference="backward", boundary="neumann", tv_weight="inside", **kw):
    return oracle.Params(tuple(shape), difference=difference, boundary=boundary, tv_weight=tv_weight,
                         **dict(HYPER, **kw))


@pytest.mark.parametrize("difference,boundary", READINGS)
@pytest.mark.parametrize("shape", [(5, 7, 9), (1, 4, 6), (2, 1, 3), (4, 4, 4)])
def test_div_is_the_adjoint_of_grad(difference, boundary, shape):
    """<D x, u> = <x, D^T u> for every reading and odd/degenerate extents."""
    rng = np.random.default_rng(31)
    x = rng.standard_normal(shape)
    u = rng.standard_normal((3,) + shape)
    p = params(shape, difference, boundary)
    lhs = float((oracle.grad(x, p) * u).sum())
    rhs = float((x * oracle.div(u, p)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("difference,boundary", READINGS)
def test_constants_have_zero_tv(difference, boundary):
    shape = (6, 5, 7)
    p = params(shape, difference, boundary)
    g = oracle.grad(np.full(shape, 2.5), p)
    assert np.abs(g).max() == 0.0


def test_forward_differences_are_reversed_backward_ones():
    """With every axis reversed, x_{v+e} - x_v becomes -(x'_v - x'_{v-e}) and
    the Neumann edge moves to the other face: D_f x = -R D_b R x, exactly."""
    shape = (6, 7, 8)
    x = np.random.default_rng(32).standard_normal(shape)
    R = lambda a: a[..., ::-1, ::-1, ::-1]
    gf = oracle.grad(x, params(shape, "forward"))
    gb = oracle.grad(np.ascontiguousarray(R(x)), params(shape, "backward"))
    np.testing.assert_array_equal(gf, -R(gb))


@pytest.mark.parametrize("boundary", ["neumann", "periodic"])
def test_forward_solve_is_the_mirrored_backward_solve(boundary):
    """The whole reweighted solve (weights, TV, steps) under forward differences
    equals the backward-difference solve of the mirrored data, mirrored back:
    |D_f x| at v is |D_b Rx| at the mirrored voxel, and h_mu is even."""
    shape = (10, 12, 14)
    vol = synth.make_volume(shape, blobs=6, radius=4, seed=33)
    R = lambda a: np.ascontiguousarray(np.asarray(a)[..., ::-1, ::-1, ::-1])
    rf = oracle.solve(vol.b, vol.w, params(shape, "forward", boundary), 2, 25)
    rb = oracle.solve(R(vol.b), R(vol.w), params(shape, "backward", boundary), 2, 25)
    np.testing.assert_allclose(rf.x, R(rb.x), rtol=0, atol=1e-12)
    np.testing.assert_allclose(rf.hist, rb.hist, rtol=1e-12)


def test_periodic_solve_commutes_with_circular_shifts():
    """A periodic boundary makes D shift-invariant, so rolling the data rolls
    the solution; the Neumann solve does not commute (the flag is live)."""
    shape = (8, 10, 12)
    vol = synth.make_volume(shape, blobs=6, radius=4, seed=34)
    sh = (3, -4, 5)
    roll = lambda a: np.ascontiguousarray(np.roll(a, sh, axis=(0, 1, 2)))
    for boundary, expect_equal in (("periodic", True), ("neumann", False)):
        p = params(shape, boundary=boundary)
        r0 = oracle.solve(vol.b, vol.w, p, 2, 25, with_hist=False)
        r1 = oracle.solve(roll(vol.b), roll(vol.w), p, 2, 25, with_hist=False)
        d = np.abs(r1.x - roll(r0.x)).max()
        if expect_equal:
            assert d <= 1e-12
        else:
            assert d > 1e-3


@pytest.mark.parametrize("boundary,expect", [("periodic", 12.0), ("neumann", None)])
def test_spectral_norm_of_dtd(boundary, expect):
    """|D|^2 = 12 exactly for a periodic boundary on even extents (the
    alternating volume is an eigenvector of each 1-D periodic Laplacian with
    eigenvalue 4), and below 12 for Neumann: the Lipschitz bound L = max w +
    12 lambda_tv max(omtv) / mu holds for both."""
    shape = (6, 8, 10)
    p = params(shape, boundary=boundary)
    i = np.indices(shape).sum(0)
    alt = (-1.0) ** i
    rq = float((oracle.div(oracle.grad(alt, p), p) * alt).sum() / (alt * alt).sum())
    x = np.random.default_rng(35).standard_normal(shape)
    for _ in range(400):
        x = oracle.div(oracle.grad(x, p), p)
        x /= np.linalg.norm(x)
    lam = float((oracle.div(oracle.grad(x, p), p) * x).sum())
    if expect is not None:
        assert abs(rq - expect) <= 1e-12
        assert abs(lam - expect) <= 1e-6
    else:
        assert lam < 12.0 and rq < 12.0


def _jacobian_asymmetry(p, x, omtv, h=1e-6, pairs=12, seed=36):
    """max |<e_j, J e_i> - <e_i, J e_j>| / scale over random voxel pairs, J the
    Jacobian of x -> tv_grad(x) by central differences."""
    rng = np.random.default_rng(seed)
    n = x.size
    worst, scale = 0.0, 0.0

    def col(i):
        e = np.zeros(n)
        e[i] = h
        e = e.reshape(x.shape)
        return ((oracle.tv_grad(x + e, omtv, p) - oracle.tv_grad(x - e, omtv, p)) / (2 * h)).ravel()

    for _ in range(pairs):
        # neighbouring voxels, so the entries are non-zero
        i = int(rng.integers(n))
        j = (i + 1) % n
        ci, cj = col(i), col(j)
        worst = max(worst, abs(ci[j] - cj[i]))
        scale = max(scale, abs(ci[i]), abs(cj[j]))
    return worst / scale


def test_tv_weight_inside_is_a_gradient_and_post_div_is_not():
    """D^T(omtv grad h(Dx)) is the gradient of sum omtv h(Dx): its Jacobian is
    symmetric. omtv * D^T(grad h(Dx)) (Eq. 20 as printed) has a non-symmetric
    Jacobian when omtv varies, so it is the gradient of no objective; with
    omtv constant the two readings coincide (up to rounding order)."""
    shape = (5, 6, 7)
    rng = np.random.default_rng(37)
    x = 0.05 * rng.standard_normal(shape)  # |Dx| of the order of mu: the smooth branch
    omtv = rng.uniform(0.2, 1.0, shape)
    inside = _jacobian_asymmetry(params(shape), x, omtv)
    post = _jacobian_asymmetry(params(shape, tv_weight="post_div"), x, omtv)
    assert inside < 1e-6
    assert post > 1e-2
    one = np.full(shape, 0.7)
    np.testing.assert_allclose(oracle.tv_grad(x, one, params(shape)),
                               oracle.tv_grad(x, one, params(shape, tv_weight="post_div")), rtol=1e-14, atol=1e-14)


def test_adopted_only_functions_reject_other_readings():
    shape = (4, 4, 4)
    z = np.zeros(shape)
    with pytest.raises(ValueError):
        oracle.step_sampled(z, z, 0.0, 0.1, z, z + 1, None, None, params(shape, "forward"), np.array([0]))
