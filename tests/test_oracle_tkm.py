"""Pins for the oracle's truncated-kernel-method Coulomb operator Theta^T (Sec. 4)."""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.linalg import expm
from scipy.special import dawsn

from oracle import chasm_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_constants_and_kernel_small_xi_asymptotics():
    assert O.c_n_alpha(3, 1) == pytest.approx(GOLDEN["c_3_1"]["value"], rel=1e-14)
    g = GOLDEN["truncated_kernel_small_xi"]
    D = 3.7
    xi = np.array([1e-3, 2e-3])
    U = O.truncated_kernel_hat(xi, D)
    approx = g["c0_over_D"] * D + g["c2_over_D3"] * D**3 * xi**2
    assert np.max(np.abs(U - approx)) < 5 * D**5 * xi.max() ** 4
    assert O.truncated_kernel_hat(np.array([0.0]), D)[0] == pytest.approx(4 * math.pi * D)
    # Si against its defining integral by Gauss-Legendre at a few points
    x, w = leggauss(60)
    for b in (0.3, 2.0, 9.5):
        t = 0.5 * b * (x + 1)
        ref = 0.5 * b * np.sum(w * np.sin(t) / t)
        assert O.si(np.array([b]))[0] == pytest.approx(ref, abs=1e-13)


@pytest.mark.parametrize("p", [(0, 0, 0), (1, 2, 3), (-3, 1, 0), (2, -2, -1)])
def test_tensor_matches_its_defining_sum(p):
    """T from one (3N_k)^3 backward FFT equals the brute-force sum of Eq. 4.7."""
    nk, lk = 4, 2.0
    T = O.tkm_tensor(nk, lk)
    ref = O.tkm_tensor_direct(nk, lk, p)
    assert abs(ref.imag) < 1e-13
    assert T[p[0] + nk - 1, p[1] + nk - 1, p[2] + nk - 1] == pytest.approx(ref.real, abs=1e-13)


def test_tensor_is_even_in_each_direction():
    T = O.tkm_tensor(8, 3.0)
    assert np.max(np.abs(T - T[::-1, :, :])) < 1e-13
    assert np.max(np.abs(T - T[:, ::-1, :])) < 1e-13
    assert np.max(np.abs(T - T[:, :, ::-1])) < 1e-13
    assert np.max(np.abs(T - T.transpose(1, 0, 2))) < 1e-13


def test_fft_convolution_equals_direct_sum():
    """Twofold zero padding reproduces the linear convolution of Eq. 4.6 exactly."""
    nk = 6
    rng = np.random.default_rng(5)
    T = O.tkm_tensor(nk, 2.5)
    fs = rng.standard_normal((2, nk, nk, nk)) + 1j * rng.standard_normal((2, nk, nk, nk))
    a = O.tkm_convolve(fs, T)
    b = O.tkm_convolve_direct(fs, T)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_dawson_closed_form_spectral_convergence():
    """Example 4.1: Phi = |k|^-2 * exp(-|k|^2) = 2 pi^{3/2} F(k)/k (F = Dawson).  The TKM error
    falls spectrally with N_k (Table 2 trend) until the tail exp(-L_k^2) is reached."""
    assert 2 * math.pi ** 1.5 == pytest.approx(GOLDEN["dawson_origin"]["value"], rel=1e-14)
    errs = []
    lk = 4.0
    for nk in (8, 16, 32):
        ks = O.k_nodes(nk, lk)
        T = O.tkm_tensor(nk, lk)
        K = np.sqrt(ks[:, None, None] ** 2 + ks[None, :, None] ** 2 + ks[None, None, :] ** 2)
        Phi = O.tkm_convolve(np.exp(-K**2).astype(complex), T).real
        Kp = np.where(K > 0, K, 1.0)
        ex = np.where(K > 0, 2 * math.pi ** 1.5 * dawsn(Kp) / Kp, 2 * math.pi ** 1.5)
        errs.append(np.max(np.abs(Phi - ex)) / np.max(ex))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-5 and errs[2] < 1e-7, errs


def theta_quadrature(k, k0, xt, Z=1.0, hbar=1.0, nr=96, nmu=96, nphi=192):
    """Continuous Coulomb operator of a Gaussian f = exp(-|k - k0|^2), from Eq. 2.3 rewritten as
    Theta(k) = -(2Z/(pi^2 hbar)) int sin(2 xt.q) |q|^-2 f(k - q) dq and integrated in spherical
    coordinates about q = 0 (|q|^-2 cancels the Jacobian): Gauss-Legendre in r and cos(theta),
    trapezoid in phi."""
    th = 2 * np.asarray(xt, dtype=float)
    d = np.asarray(k, dtype=float) - np.asarray(k0, dtype=float)
    R = np.linalg.norm(d) + 7.0
    xr, wr = leggauss(nr)
    r = 0.5 * R * (xr + 1)
    wr = 0.5 * R * wr
    mu, wmu = leggauss(nmu)
    ph = np.arange(nphi) * 2 * math.pi / nphi
    st = np.sqrt(1 - mu**2)
    w = np.stack([st[:, None] * np.cos(ph)[None, :], st[:, None] * np.sin(ph)[None, :],
                  np.broadcast_to(mu[:, None], (nmu, nphi))], -1)
    tw = w @ th
    dw = w @ d
    val = np.sin(r[:, None, None] * tw[None]) * np.exp(
        -(d @ d - 2 * r[:, None, None] * dw[None] + r[:, None, None] ** 2))
    integral = np.einsum("r,m,rmp->", wr, wmu, val) * (2 * math.pi / nphi)
    return -(2 * Z / (math.pi**2 * hbar)) * integral


def test_theta_matches_continuous_operator_with_spectral_convergence():
    """Theta^T of a Gaussian at xt != 0 against the continuous pseudodifferential operator
    (independent quadrature).  Pins the sign of Eq. 2.3, the 1/pi^2 prefactor and the Delta-k^3
    normalisation folded into T; the error decays as in Theorem 4.1."""
    xt = np.array([0.7, -0.4, 0.5])
    k0 = np.array([0.3, 0.0, -0.2])
    assert theta_quadrature((0.5, 0.25, 0), k0, xt) == pytest.approx(
        theta_quadrature((0.5, 0.25, 0), k0, xt, nr=140, nmu=140, nphi=280), abs=1e-12)
    errs = []
    for nk in (8, 16, 32):
        lk = 4.0
        ks = O.k_nodes(nk, lk)
        T = O.tkm_tensor(nk, lk)
        K1, K2, K3 = np.meshgrid(ks, ks, ks, indexing="ij")
        f = np.exp(-((K1 - k0[0]) ** 2 + (K2 - k0[1]) ** 2 + (K3 - k0[2]) ** 2))
        th = O.theta_coulomb_point(f, xt, 1.0, 1.0, ks, T)
        rng = np.random.default_rng(0)
        e = 0.0
        for _ in range(5):
            i = tuple(rng.integers(nk // 4, 3 * nk // 4, 3))
            e = max(e, abs(th[i] - theta_quadrature((ks[i[0]], ks[i[1]], ks[i[2]]), k0, xt)))
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-4 and errs[2] < 1e-7, errs


def test_theta_scales_with_charge_and_hbar_and_is_zero_at_the_nucleus():
    nk, lk = 8, 3.0
    ks = O.k_nodes(nk, lk)
    T = O.tkm_tensor(nk, lk)
    f = np.random.default_rng(7).standard_normal((nk, nk, nk))
    xt = np.array([0.4, 0.1, -0.3])
    a = O.theta_coulomb_point(f, xt, 1.0, 1.0, ks, T)
    b = O.theta_coulomb_point(f, xt, 2.5, 0.5, ks, T)
    assert np.max(np.abs(b - 5.0 * a)) < 1e-12 * np.max(np.abs(b))
    z = O.theta_coulomb_point(f, np.zeros(3), 1.0, 1.0, ks, T)
    assert np.max(np.abs(z)) < 1e-13


def _theta_matrix(nk, lk, xt):
    ks = O.k_nodes(nk, lk)
    T = O.tkm_tensor(nk, lk)
    n = nk**3
    E = np.eye(n).reshape(n, nk, nk, nk)
    M = O.theta_coulomb_point(E, np.broadcast_to(xt, (n, 3)), 1.0, 1.0, ks, T)
    return M.reshape(n, n).T   # column j = Theta[e_j]


def test_theta_is_an_antisymmetric_real_operator():
    """Theta^T = C sum_q T_{p-q} sin(2 xt.(k_p - k_q)) f_q with T even: an antisymmetric matrix."""
    M = _theta_matrix(4, 2.0, np.array([0.6, -0.2, 0.35]))
    assert np.max(np.abs(M + M.T)) < 1e-12 * np.max(np.abs(M))


def test_coulomb_pflow_is_the_fourth_order_taylor_polynomial():
    """P(dt) in Horner form equals I + dt M + ... + (dt M)^4/4! exactly, and differs from
    exp(dt M) by O(dt^5)."""
    nk, lk = 4, 2.0
    xt = np.array([0.6, -0.2, 0.35])
    M = _theta_matrix(nk, lk, xt)
    prob = O.Problem(nx=(1, 1, 1), nk=nk, x_lo=(0.6, -0.2, 0.35), x_hi=(1.6, 0.8, 1.35), lk=lk,
                     nuclei=[((0.0, 0.0, 0.0), 1.0)])
    f = np.random.default_rng(8).standard_normal(prob.shape)
    v = f.reshape(-1)
    for dt in (0.05, 0.1):
        taylor = v.copy()
        term = v.copy()
        for n in range(1, 5):
            term = dt * (M @ term) / n
            taylor = taylor + term
        P = O.pflow_coulomb(f, prob, dt).reshape(-1)
        assert np.max(np.abs(P - taylor)) < 1e-12 * np.max(np.abs(v))
    e1 = np.max(np.abs(O.pflow_coulomb(f, prob, 0.1).reshape(-1) - expm(0.1 * M) @ v))
    e2 = np.max(np.abs(O.pflow_coulomb(f, prob, 0.05).reshape(-1) - expm(0.05 * M) @ v))
    assert e1 / e2 > 20.0   # ~2^5


def test_theta_approaches_the_classical_force_term_far_from_the_nucleus():
    """Classical limit: far from the nucleus Theta^T[f] -> (1/hbar) grad V . grad_k f with
    V = -Z/|x| (the sign of Eq. 2.3; Eq. 5.1 for the quadratic case), the first quantum correction
    (hbar^2/24) d^3V d^3_k f being O(|x|^-2) relative.  The relative deviation times |x|^2 stays
    constant while it falls 16-fold from |x| = 2 to 8 (a wrong sign leaves it near 2, a wrong
    prefactor leaves a constant).  The k-grid must resolve the modulation: 2 |x| dk < pi."""
    nk, lk = 32, 3.0
    prob = O.Problem(nx=(1, 1, 1), nk=nk, x_lo=(0.0,) * 3, x_hi=(1.0,) * 3, lk=lk,
                     nuclei=[((0.0, 0.0, 0.0), 1.0)])
    ks = prob.ks()
    K = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), -1)
    b, k0 = 2.0, np.array([0.3, -0.2, 0.1])
    f = np.exp(-b * np.sum((K - k0) ** 2, -1))
    grad = -2 * b * (K - k0) * f[..., None]
    T = O.tkm_tensor(nk, lk)
    scaled = []
    for r in (2.0, 4.0, 8.0):
        x = np.array([[0.6 * r, 0.8 * r, 0.0]])
        th = O.theta_coulomb(f[None], prob, T, xpts=x)[0]
        classical = np.tensordot(grad, x[0] / np.linalg.norm(x[0]) ** 3, axes=([3], [0]))
        e = np.linalg.norm(th - classical) / np.linalg.norm(classical)
        scaled.append(e * r * r)
    assert e < 0.05
    assert max(scaled) / min(scaled) < 1.3, scaled
