"""Pins for the oracle's spline transform and advection A(tau) (Sec. 2.2, Sec. 3)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle import chasm_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_bspline_node_values_and_partition_of_unity():
    g = GOLDEN["bspline_node_values"]
    assert O.bspline(np.array([0.0]))[0] == pytest.approx(g["B_center"], abs=1e-15)
    assert O.bspline(np.array([1.0]))[0] == pytest.approx(g["B_neighbour"], abs=1e-15)
    assert O.bspline(np.array([-1.0]))[0] == pytest.approx(g["B_neighbour"], abs=1e-15)
    # sum_nu B_nu(x) = 1 anywhere in the interior of the knot range
    x = np.linspace(0.0, 10.0, 997)
    s = sum(O.bspline(x - nu) for nu in range(-3, 14))
    assert np.max(np.abs(s - 1.0)) < 1e-14
    # C2 continuity at the knots: left and right second differences agree
    e = 1e-5
    for t in (-2.0, -1.0, 0.0, 1.0, 2.0):
        d2l = (O.bspline(np.array([t])) - 2 * O.bspline(np.array([t - e])) + O.bspline(np.array([t - 2 * e]))) / e**2
        d2r = (O.bspline(np.array([t + 2 * e])) - 2 * O.bspline(np.array([t + e])) + O.bspline(np.array([t]))) / e**2
        assert abs(d2l[0] - d2r[0]) < 1e-3


def _spline_eval(eta, h, y, x0=0.0):
    n3 = eta.shape[0]
    return sum(eta[nu + 1] * O.bspline((y - x0 - nu * h) / h) for nu in range(-1, n3 - 1))


@pytest.mark.parametrize("n,h", [(9, 0.7), (17, 0.5), (33, 0.25)])
def test_full_stencil_pmbc_equals_textbook_natural_spline(n, h):
    """With n_nb >= N the PMBC closure reproduces the global natural spline exactly; compare the
    interpolant with scipy's natural cubic spline (a library routine)."""
    xs = O.x_nodes(n, -1.0, -1.0 + (n - 1) * h)
    phi = np.sin(1.3 * xs) + 0.2 * xs**3 - xs
    eta = O.spline_coeffs_1d(phi[:, None], 0, h, n_nb=n + 5)[:, 0]
    y = np.linspace(xs[0], xs[-1], 301)
    s = _spline_eval(eta, h, y, x0=xs[0])
    ref = CubicSpline(xs, phi, bc_type="natural")(y)
    assert np.max(np.abs(s - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    # natural end conditions s''(x_0) = s''(x_N) = 0 (Eq. 2.13) on eta
    assert abs(eta[0] - 2 * eta[1] + eta[2]) < 1e-12
    assert abs(eta[-3] - 2 * eta[-2] + eta[-1]) < 1e-12


def test_pmbc_stencil_decay_and_symmetry():
    """The end stencils decay geometrically with ratio lambda = sqrt(3) - 2, the decay rate of the
    inverse of the (1/6, 2/3, 1/6) Toeplitz matrix (Sec. 3.1.1); by reflection c- = -c+."""
    cp, cm = O.pmbc_end_stencils(60, 0.8, 40)
    lam = math.sqrt(3.0) - 2.0
    r = cp[5:30] / cp[4:29]
    assert np.max(np.abs(r - lam)) < 1e-10
    assert np.max(np.abs(cm + cp)) < 1e-14
    # the closure is a derivative: it annihilates constants and maps a linear ramp to its slope
    n, h = 60, 0.8
    xs = O.x_nodes(n, 0.0, (n - 1) * h)
    cp_full, _ = O.pmbc_end_stencils(n, h, n)
    assert abs(np.dot(cp_full, np.ones(n))) < 1e-12
    assert abs(np.dot(cp_full, 2.5 * xs + 1.0) - 2.5) < 1e-11


def test_truncated_stencil_error_is_small():
    """n_nb = 10 perturbs the coefficients at the ~1e-5 level, n_nb >= 20 is negligible
    (Sec. 5.1 observations)."""
    n, h = 64, 0.5
    xs = O.x_nodes(n, -16.0, 15.5)
    phi = np.sin(0.37 * xs) + 0.5 * np.cos(0.11 * xs)  # data reaching beyond the stencil
    full = O.spline_coeffs_1d(phi[:, None], 0, h, n)[:, 0]
    e10 = np.max(np.abs(O.spline_coeffs_1d(phi[:, None], 0, h, 10)[:, 0] - full))
    e20 = np.max(np.abs(O.spline_coeffs_1d(phi[:, None], 0, h, 20)[:, 0] - full))
    assert 1e-8 < e10 < 1e-4
    assert e20 < 1e-10


def _prob(nx, nk, L, lk, **kw):
    return O.Problem(nx=(nx,) * 3, nk=nk, x_lo=(-L,) * 3, x_hi=(L,) * 3, lk=lk, **kw)


def test_advect_zero_shift_is_identity():
    prob = _prob(7, 4, 3.0, 2.0)
    f = np.random.default_rng(1).standard_normal(prob.shape)
    assert np.max(np.abs(O.advect(f, prob, 0.0) - f)) < 1e-13


def test_advect_integer_shift_is_exact_index_shift():
    """tau = h/dk makes alpha = k tau / h = j - N_k/2 an integer for every k; an interpolating
    spline then reproduces grid values: f_new(x_j, k) = f(x_{j-alpha}, k) where the foot is on
    the grid (Eq. 2.6 with A_tau(x, k) = (x - hbar k tau / m, k))."""
    prob = _prob(9, 4, 4.0, 2.0)
    h = prob.hs(0)
    tau = h / prob.dk
    f = np.random.default_rng(2).standard_normal(prob.shape)
    g = O.advect(f, prob, tau)
    nk = prob.nk
    for k1 in range(nk):
        for k2 in range(nk):
            for k3 in range(nk):
                a = [k1 - nk // 2, k2 - nk // 2, k3 - nk // 2]
                for j in [(4, 4, 4), (3, 5, 2), (6, 2, 5)]:
                    src = [j[d] - a[d] for d in range(3)]
                    if all(0 <= s < 9 for s in src):
                        assert g[j + (k1, k2, k3)] == pytest.approx(
                            f[tuple(src) + (k1, k2, k3)], abs=1e-12)


def test_advect_64_tap_equals_three_directional_passes():
    """Sum factorisation: the literal 64-term sum of Eq. 3.10 equals three successive 1-D
    spline-and-shift passes along x1, x2, x3 (the tensor-product operators commute)."""
    prob = _prob(8, 4, 3.0, 2.0)
    f = np.random.default_rng(3).standard_normal(prob.shape)
    tau = 0.37
    g = O.advect(f, prob, tau)
    ks = prob.ks()
    h = f
    for d in range(3):
        alpha = prob.hbar * ks * tau / (prob.m * prob.hs(d))
        h = O.advect_1d(h, d, prob.hs(d), prob.n_nb, alpha, 3 + d)
    assert np.max(np.abs(g - h)) < 1e-12


def test_advect_reproduces_linear_functions_in_the_interior():
    """Natural cubic splines reproduce linear data exactly; feet inside the domain are exact."""
    prob = _prob(9, 4, 4.0, 2.0)
    xs = prob.xs(0)
    X1, X2, X3 = np.meshgrid(xs, xs, xs, indexing="ij")
    lin = 0.3 + 0.5 * X1 - 0.25 * X2 + 0.125 * X3
    f = np.broadcast_to(lin[..., None, None, None], prob.shape).copy()
    tau = 0.2
    g = O.advect(f, prob, tau)
    ks = prob.ks()
    for (k1, k2, k3) in [(0, 1, 2), (3, 3, 0), (2, 0, 1)]:
        sh = np.array([ks[k1], ks[k2], ks[k3]]) * tau
        ex = 0.3 + 0.5 * (X1 - sh[0]) - 0.25 * (X2 - sh[1]) + 0.125 * (X3 - sh[2])
        inner = (slice(1, -1),) * 3
        assert np.max(np.abs(g[inner + (k1, k2, k3)] - ex[inner])) < 1e-12


def test_advect_gaussian_converges_at_fourth_order():
    """Translating a smooth packet: the error falls ~ h^4 (Sec. 5.1: fourth order in dx)."""
    errs = []
    for nx in (17, 33):
        prob = _prob(nx, 4, 6.0, 2.0, n_nb=40)
        xs = prob.xs(0)
        ks = prob.ks()
        tau = 0.3
        G = lambda x: np.exp(-(x**2) / 4.0)
        f = (G(xs)[:, None, None] * G(xs)[None, :, None] * G(xs)[None, None, :])[..., None, None, None]
        f = np.broadcast_to(f, prob.shape).copy()
        g = O.advect(f, prob, tau)
        k1, k2, k3 = 3, 1, 2
        ex = (G(xs - ks[k1] * tau)[:, None, None] * G(xs - ks[k2] * tau)[None, :, None]
              * G(xs - ks[k3] * tau)[None, None, :])
        errs.append(np.max(np.abs(g[..., k1, k2, k3] - ex)))
    order = math.log2(errs[0] / errs[1])
    assert order > 3.5, errs
