"""Pins of the PMBC patch decomposition of the oracle (Sec. 3.1.2-3.1.3)."""
import numpy as np
import pytest

from oracle import chasm_oracle as O


def _line(n, seed, m=3):
    rng = np.random.default_rng(seed)
    x = np.linspace(-1, 1, n)
    return np.exp(-3 * x ** 2)[:, None] + 0.1 * rng.standard_normal((n, m))


@pytest.mark.parametrize("n,p", [(13, 2), (13, 3), (13, 4), (16, 3), (16, 5), (17, 4)])
def test_patches_with_full_stencils_reproduce_the_global_spline(n, p):
    """With n_nb >= N every closure value is the exact end derivative of the global natural
    spline, so each patch's Hermite-closed spline is the global spline on that patch (a cubic
    spline is fixed by its node values and end slopes): p patches equal one patch to rounding,
    for feet inside, on the nodes of, and outside the domain."""
    h = 0.3
    phi = _line(n, n + p)
    alpha = np.array([0.0, 0.37, -0.61, 1.0, -1.0, 2.3, -1.8])
    phi_k = np.repeat(phi[:, None, :], len(alpha), axis=1)
    ref = O.advect_1d(phi_k, 0, h, n, alpha, 1)
    got = O.advect_1d_patches(phi_k, 0, h, n, alpha, 1, p)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_truncated_patch_stencils_decay_geometrically():
    """Truncated stencils (Eq. 3.3): the departure of p > 1 from p = 1 falls like |lambda|^n_nb,
    lambda = sqrt(3) - 2 (the decay of the inverse spline matrix, Sec. 3.1.1): about 700x per
    five more taps.  Per step it stays below the ~1e-5 the paper reports for whole runs at
    n_nb = 10 (Sec. 5.1)."""
    n, p, h = 61, 4, 0.3
    x = np.linspace(-9, 9, n)
    phi = (np.sin(1.3 * x) + 0.2 * x)[:, None]
    alpha = np.array([0.41])
    phi_k = phi[:, None, :]
    errs = {}
    for nb in (10, 15, 20):
        a = O.advect_1d(phi_k, 0, h, nb, alpha, 1)
        b = O.advect_1d_patches(phi_k, 0, h, nb, alpha, 1, p)
        errs[nb] = np.max(np.abs(a - b))
    assert 1e-9 < errs[10] < 1e-5
    assert errs[15] < errs[10] / 100 and errs[20] < errs[15] / 100


def test_one_patch_is_the_single_patch_transform():
    phi = _line(12, 1)
    alpha = np.array([0.2, -0.7])
    phi_k = np.repeat(phi[:, None, :], 2, axis=1)
    assert np.allclose(O.advect_1d_patches(phi_k, 0, 0.5, 20, alpha, 1, 1),
                       O.advect_1d(phi_k, 0, 0.5, 20, alpha, 1), rtol=0, atol=1e-13)


def test_3d_patch_advection_with_one_patch_equals_the_64_term_sum():
    prob = O.Problem(nx=(7, 6, 8), nk=4, x_lo=(-2.0,) * 3, x_hi=(2.0, 2.5, 1.5), lk=2.0)
    f = np.random.default_rng(3).standard_normal(prob.shape)
    a = O.advect(f, prob, 0.3)
    b = O.advect_patches(f, prob, 0.3, (1, 1, 1))
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_plane_step_with_patches():
    """The plane step with p PMBC patches (Sec. 3.1.2-3.1.3): with full stencils (n_nb >= N) it
    equals the one-patch plane step (each patch spline is the global spline); with truncated
    stencils it departs from it (so the patches are applied), by less at n_nb = 15 than at
    n_nb = 10."""
    base = dict(nx=(33, 4, 4), nk=8, x_lo=(-8.0, -1.0, -1.0), x_hi=(8.0, 1.0, 1.0), lk=3.0,
                nuclei=[], kappa=0.4)
    full = O.Problem(n_nb=40, **base)
    xs, ks = full.xs(0), full.ks()
    g = np.exp(-0.5 * (xs[:, None] - 1.0) ** 2 - 2.0 * ks[None, :] ** 2) / np.pi
    one = O.strang_step_plane(g, full, 0, 0.2)
    four = O.strang_step_plane(g, full, 0, 0.2, p=4)
    assert np.max(np.abs(four - one)) <= 1e-13 * np.max(np.abs(one))
    dev = {}
    for nb in (10, 15):
        P = O.Problem(n_nb=nb, **base)
        dev[nb] = np.max(np.abs(O.strang_step_plane(g, P, 0, 0.2, p=4) - O.strang_step_plane(g, P, 0, 0.2)))
    assert 0 < dev[15] < dev[10]
