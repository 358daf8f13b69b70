"""Pins of the LPC1 oracle (Sec. 2.2) and of Theta for the quadratic potential (Eq. 5.1),
against closed forms, the already-pinned exact k-shift, the matrix exponential and invariants."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import synth
from oracle import chasm_oracle as O


def _prob(nx, nk, L, lk, **kw):
    return O.Problem(nx=(nx,) * 3 if isinstance(nx, int) else nx, nk=nk, x_lo=(-L,) * 3,
                     x_hi=(L,) * 3, lk=lk, **kw)


def test_theta_harmonic_of_a_gaussian_matches_the_closed_form():
    """Theta f = sum_d kappa (x_d - c_d)/hbar df/dk_d; for f = exp(-a|x-x0|^2 - b|k-k0|^2) the
    k-derivative is -2 b (k_d - k0_d) f.  The packet's spectrum beyond the grid's Nyquist
    frequency pi/dk is ~exp(-(pi/dk)^2 / 4b) = 3e-9 of its peak, which bounds the agreement."""
    prob = _prob((4, 5, 3), 32, 3.0, 4.0, kappa=0.7, center=(0.2, -0.1, 0.3), hbar=1.3)
    x0, k0, a, b = (0.3, -0.2, 0.1), (0.4, -0.3, 0.2), 0.5, 2.0
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk,
                               [{"w": 1.0, "x0": x0, "k0": k0, "ax": a, "ak": b}])
    X = np.meshgrid(prob.xs(0), prob.xs(1), prob.xs(2), indexing="ij")
    K = np.meshgrid(prob.ks(), prob.ks(), prob.ks(), indexing="ij")
    ref = np.zeros_like(f)
    for d in range(3):
        rate = prob.kappa * (X[d] - prob.center[d]) / prob.hbar
        ref += rate[:, :, :, None, None, None] * (-2.0 * b * (K[d] - k0[d]))[None, None, None] * f
    got = O.theta_harmonic(f, prob)
    assert O.rel_l2(got, ref) < 1e-7


def test_theta_harmonic_is_the_rate_of_the_exact_k_shift():
    """For any grid function the spectral shift P(s) of pflow_harmonic is exp(s Theta), so the
    central difference (P(e) - P(-e)) / 2e approaches Theta f at second order in e."""
    prob = _prob((3, 4, 3), 16, 2.0, 3.0, kappa=1.1, center=(0.1, 0.2, -0.3))
    rng = np.random.default_rng(3)
    f = rng.standard_normal(prob.shape)
    th = O.theta_harmonic(f, prob)
    errs = []
    for e in (1e-2, 5e-3, 2.5e-3):
        fd = (O.pflow_harmonic(f, prob, e) - O.pflow_harmonic(f, prob, -e)) / (2 * e)
        errs.append(O.rel_l2(fd, th))
    assert errs[-1] < 1e-3          # random data: the top modes carry most of the O(e^2) error
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def test_lpc1_without_a_potential_is_the_advection():
    prob = _prob((7, 6, 8), 8, 3.0, 3.0, kappa=0.0)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(prob.shape)
    assert np.array_equal(O.lpc1_step(f, prob, 0.07), O.advect(f, prob, 0.07))


@pytest.mark.parametrize("potential", ["coulomb", "harmonic"])
def test_lpc1_without_advection_is_second_order_in_time(potential):
    """With hbar/m -> 0 the feet stay on the nodes and LPC1 is the predictor-corrector for
    df/dt = Theta f at each x point: local error O(dt^3) against the matrix exponential of Theta
    (a wrong corrector weight leaves an O(dt^2) error)."""
    kw = dict(nuclei=[((0.2, -0.3, 0.1), 1.0)]) if potential == "coulomb" else \
        dict(kappa=0.9, center=(0.1, 0.0, -0.2))
    prob = _prob(4, 8, 2.0, 3.0, m=1e15, **kw)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(prob.shape)
    ix = (1, 2, 0)
    xpt = np.array([[prob.xs(d)[ix[d]] for d in range(3)]])
    n = prob.nk ** 3
    basis = np.eye(n).reshape(n, prob.nk, prob.nk, prob.nk)
    one = O.Problem(nx=(1, 1, 1), nk=prob.nk, x_lo=tuple(xpt[0]), x_hi=tuple(xpt[0] + 1.0),
                    lk=prob.lk, **kw)
    if potential == "coulomb":
        M = O.theta_coulomb(basis, one, xpts=np.repeat(xpt, n, axis=0)).reshape(n, n).T
    else:
        M = np.stack([O.theta_harmonic(b[None, None, None], one).reshape(n) for b in basis], axis=1)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        got = O.lpc1_step(f, prob, dt)[ix].reshape(n)
        ref = expm(dt * M) @ f[ix].reshape(n)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[-1] < 1e-3
    assert 7.0 < errs[1] / errs[2] < 9.0, errs


def test_theta_harmonic_moves_no_mass_between_x_points():
    """The spectral k-derivative of periodic data has no mean, so sum_k Theta f = 0 at every x
    point (Theta only moves mass along k): the operator part of LPC1 conserves mass exactly."""
    prob = _prob((5, 4, 6), 16, 3.0, 3.0, kappa=0.8, center=(0.3, -0.2, 0.1))
    f = np.random.default_rng(9).standard_normal(prob.shape)
    th = O.theta_harmonic(f, prob)
    per_x = th.sum(axis=(3, 4, 5))
    assert np.max(np.abs(per_x)) < 1e-12 * np.max(np.abs(th)) * prob.nk ** 3


def test_lpc1_plane_converges_at_second_order_to_the_exact_rotation():
    """1-D harmonic oscillator (hbar = m = kappa = 1): the Wigner function rotates rigidly in the
    (x, k) plane (Sec. 5.1).  On a fine plane grid the spatial error is negligible and the global
    error of LPC1 at fixed T falls by 4 per halving of dt.  Misplacing the advection of Theta f
    (or a wrong corrector weight) in lpc1_combine, which the 6-D step shares, leaves a
    first-order scheme."""
    prob = O.Problem(nx=(256, 4, 4), nk=64, x_lo=(-8.0,) * 3, x_hi=(8.0,) * 3, lk=8.0, kappa=1.0)
    x, k = prob.xs(0), prob.ks()
    X, K = np.meshgrid(x, k, indexing="ij")
    x0, k0, T = 1.0, 0.5, 0.4

    def g0(xx, kk):
        return np.exp(-(xx - x0) ** 2 - (kk - k0) ** 2) / math.pi

    errs = []
    for n in (8, 16, 32):
        dt = T / n
        g = g0(X, K)
        for _ in range(n):
            g = O.lpc1_step_plane(g, prob, 0, dt)
        Xr, Kr = O.harmonic_rotation(X, K, T, 1.0)
        errs.append(np.linalg.norm(g - g0(Xr, Kr)) / np.linalg.norm(g0(Xr, Kr)))
    assert errs[-1] < 1e-3
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs
