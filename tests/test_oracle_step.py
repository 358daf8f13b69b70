"""Pins for the oracle's full Strang step, its P-flows, diagnostics and the input generators."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_paper_grid_conventions():
    g = GOLDEN["x_grid_1s"]
    xs = O.x_nodes(g["n"], g["lo"], g["hi"])
    assert xs[1] - xs[0] == pytest.approx(g["h"], rel=1e-12)
    assert xs[-1] == pytest.approx(g["hi"], rel=1e-14)
    g = GOLDEN["k_grids_1s"]
    for nk, dk in zip(g["nk"], g["dk"]):
        ks = O.k_nodes(nk, g["lk"])
        assert ks[1] - ks[0] == pytest.approx(dk, rel=1e-12)
        assert ks[0] == pytest.approx(-g["lk"]) and ks[nk // 2] == 0.0
    g = GOLDEN["memory_81_64"]
    assert g["nx"] ** 3 * g["nk"] ** 3 * g["bytes_per_cell"] / 1e9 == pytest.approx(g["gb"], rel=2e-3)


def test_harmonic_rotation_period():
    g = GOLDEN["harmonic_period"]
    x, k = O.harmonic_rotation(np.array([1.0]), np.array([0.3]), g["T"], kappa=g["omega"])
    assert x[0] == pytest.approx(1.0, abs=1e-12) and k[0] == pytest.approx(0.3, abs=1e-12)


def test_wigner_1s_generator_peak_and_mass():
    """max f_1s = 1/pi^3 (Sec. 5.2) and unit mass, from the discrete Fourier sum."""
    nk, lk = 16, 8.0
    f = synth.wigner_1s((3, 3, 3), nk, (-1, -1, -1), (1, 1, 1), lk, n_y=64)
    assert f[1, 1, 1, nk // 2, nk // 2, nk // 2] == pytest.approx(1 / math.pi ** 3, rel=1e-3)
    assert f[1, 1, 1, nk // 2, nk // 2, nk // 2] == pytest.approx(
        GOLDEN["wigner_1s_max"]["value"], rel=2e-3)
    # integral over k of f(x, k) equals (2 pi)^3 phi_1s(x)^2 (up to y-images at 2 pi / dk)
    lk = 4.0
    f = synth.wigner_1s((3, 3, 3), nk, (-1, -1, -1), (1, 1, 1), lk, n_y=64)
    dk = 2 * lk / nk
    rho = f[1, 1, 1].sum() * dk ** 3
    assert rho == pytest.approx((2 * math.pi) ** 3 * synth.phi_1s(0.0) ** 2, rel=1e-4)


def test_mass_and_energy_of_a_packet_match_closed_forms():
    """Unit-mass packet pi^-3 exp(-|x-x0|^2/2 - 2|k-k0|^2) in V = |x|^2/2:
    <|k|^2>/2 = (3/8 + |k0|^2)/2 ... and <|x|^2>/2 = (3 + |x0|^2)/2."""
    x0, k0 = (0.5, -0.25, 0.0), (0.2, 0.0, -0.1)
    # steps dx = 1, dk = 1/2: the Riemann-sum (Poisson) error of these Gaussians is ~1e-8
    prob = O.Problem(nx=(19,) * 3, nk=20, x_lo=(-9,) * 3, x_hi=(9,) * 3, lk=5.0, kappa=1.0)
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk,
                               [synth.packet(x0, k0)])
    assert O.mass(f, prob) == pytest.approx(1.0, rel=1e-7)
    e_kin = 0.5 * (3 * 0.25 + sum(c * c for c in k0))
    e_pot = 0.5 * (3 * 1.0 + sum(c * c for c in x0))
    assert O.energy(f, prob) == pytest.approx(e_kin + e_pot, rel=1e-6)


def test_harmonic_pflow_is_an_exact_spectral_shift():
    """For band-limited periodic data the spectral k-shift is exact: f(x, k + s)."""
    nk, lk = 8, 2.0
    prob = O.Problem(nx=(3, 2, 2), nk=nk, x_lo=(-1, -1, -1), x_hi=(1, 1, 1), lk=lk, kappa=0.7)
    ks = prob.ks()
    w = math.pi / lk  # fundamental of the period 2 lk
    def fk(a, b, c):
        return (1.0 + 0.3 * np.cos(w * a) + 0.2 * np.sin(2 * w * b)) * (0.5 + np.cos(3 * w * c))
    K1, K2, K3 = np.meshgrid(ks, ks, ks, indexing="ij")
    f = np.broadcast_to(fk(K1, K2, K3), prob.shape).copy()
    dt = 0.37
    g = O.pflow_harmonic(f, prob, dt)
    for i1 in range(3):
        for i2 in range(2):
            for i3 in range(2):
                s = [dt * prob.kappa * prob.xs(d)[i] for d, i in zip(range(3), (i1, i2, i3))]
                ex = fk(K1 + s[0], K2 + s[1], K3 + s[2])
                assert np.max(np.abs(g[i1, i2, i3] - ex)) < 1e-12


def _harmonic_reference(prob, pk, dt, n, which):
    """Exact solution transported along the exact Strang map (which='map') or along the exact
    rotation of Eq. 5.2 (which='rot'), evaluated on the grid."""
    X = np.meshgrid(prob.xs(0), prob.xs(1), prob.xs(2), indexing="ij")
    ks = prob.ks()
    fx = [np.broadcast_to(X[d][..., None, None, None], prob.shape) for d in range(3)]
    kk = [np.broadcast_to(ks.reshape([1] * (3 + d) + [-1] + [1] * (2 - d)), prob.shape)
          for d in range(3)]
    if which == "map":
        ft = [O.strang_discrete_map(fx[d], kk[d], dt, n, prob.kappa) for d in range(3)]
    else:
        ft = [O.harmonic_rotation(fx[d], kk[d], dt * n, prob.kappa) for d in range(3)]
    p = pk[0]
    return p["w"] * np.exp(-p["ax"] * sum((ft[d][0] - p["x0"][d]) ** 2 for d in range(3))
                           - p["ak"] * sum((ft[d][1] - p["k0"][d]) ** 2 for d in range(3)))


@pytest.mark.slow
def test_harmonic_strang_follows_the_discrete_map_and_the_rotation():
    """Quadratic V: Strang with the exact P-flow is a composition of exact linear maps, so the
    oracle must follow the exact Strang characteristic map up to the spline error, and the exact
    rotation of Eq. 5.2 up to O(dt^2).  A planted mistake (P shifting k the wrong way) must fail
    the same check by a wide margin."""
    prob = O.Problem(nx=(13, 9, 9), nk=12, x_lo=(-6.0, -4.0, -4.0), x_hi=(6.0, 4.0, 4.0),
                     lk=4.0, kappa=1.0, n_nb=20)
    pk = [synth.packet((1.0, 0.0, 0.0), (0.0, 0.5, 0.0), ax=0.5, ak=0.5)]
    f0 = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    dt, n = 0.1, 2
    f = O.run(f0, prob, dt, n)
    f_map = _harmonic_reference(prob, pk, dt, n, "map")
    f_rot = _harmonic_reference(prob, pk, dt, n, "rot")
    e_map = np.max(np.abs(f - f_map)) / np.max(f_map)
    e_rot = np.max(np.abs(f - f_rot)) / np.max(f_rot)
    assert e_map < 1e-2, e_map
    assert e_rot < 1e-2, e_rot
    # mass of a packet inside the box is conserved up to leakage through the x-boundary
    assert O.mass(f, prob) == pytest.approx(O.mass(f0, prob), rel=1e-3)
    good1 = np.max(np.abs(O.run(f0, prob, dt, 1) - _harmonic_reference(prob, pk, dt, 1, "map")))
    bad = O.Problem(**{**prob.__dict__, "kappa": -1.0})
    bad1 = np.max(np.abs(O.run(f0, bad, dt, 1) - _harmonic_reference(prob, pk, dt, 1, "map")))
    assert bad1 > 10 * good1, (bad1, good1)


def test_hydrogen_1s_is_stationary_and_the_sign_matters():
    """The Wigner transform of an eigenstate is stationary (Sec. 2.1): at points away from the
    nucleus, -k . grad_x f_1s + Theta^T[f_1s] must nearly vanish.  grad_x f comes from central
    differences of the 1s generator; Theta^T from the oracle.  With the operator's sign flipped
    (the sign printed in Eq. 2.4) the two terms add instead of cancelling."""
    nk, lk, ny = 16, 4.0, 64
    ks = O.k_nodes(nk, lk)
    T = O.tkm_tensor(nk, lk)
    K = np.meshgrid(ks, ks, ks, indexing="ij")
    def f1s(p):
        return synth.wigner_1s((2, 2, 2), nk, tuple(p), tuple(p + 1.0), lk, n_y=ny)[0, 0, 0]
    for x in [(1.5, 0.5, -0.7), (2.2, -1.0, 0.3), (0.6, 0.4, 0.2)]:
        x = np.array(x)
        d = 1e-3
        grad = [(f1s(x + d * e) - f1s(x - d * e)) / (2 * d) for e in np.eye(3)]
        adv = -(K[0] * grad[0] + K[1] * grad[1] + K[2] * grad[2])
        th = O.theta_coulomb_point(f1s(x), x, 1.0, 1.0, ks, T)
        r_good = np.linalg.norm(adv + th) / np.linalg.norm(adv)
        r_flip = np.linalg.norm(adv - th) / np.linalg.norm(adv)
        assert r_good < 0.2, (x, r_good)
        assert r_flip > 1.8, (x, r_flip)


def test_splitmix64_reference_values():
    """First outputs of SplitMix64 seeded with 1234567 (published test vector of the reference
    implementation)."""
    g = synth.SplitMix64(1234567)
    got = [g.next_u64() for _ in range(3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_plane_step_factors_the_quadratic_potential_step():
    """For V = kappa/2 |x - c|^2 the Strang step maps a product f = prod_d g_d(x_d, k_d) factor by
    factor (A is a tensor product of 1-D interpolations along x_d with shifts set by k_d; P a
    product of shifts along k_d set by x_d).  The plane map must reproduce the 6-D step exactly,
    on an anisotropic grid with an off-centre potential; a plane map on the wrong axis or with the
    wrong shift sign fails."""
    P = O.Problem(nx=(7, 8, 9), nk=8, x_lo=(-3.0, -2.5, -3.5), x_hi=(3.0, 3.5, 2.5), lk=3.0,
                  nuclei=[], kappa=0.8, center=(0.2, -0.1, 0.3))
    ks = P.ks()
    g = synth.SplitMix64(77)
    gs = []
    for d in range(3):
        xs = P.xs(d)
        base = np.exp(-0.6 * (xs[:, None] - 0.3 * d) ** 2 - 0.7 * (ks[None, :] + 0.2 * d) ** 2)
        noise = np.array([[g.uniform(-1.0, 1.0) for _ in ks] for _ in xs])
        gs.append(base * (1.0 + 0.01 * noise))
    f = np.einsum("ai,bj,ck->abcijk", *gs)
    want = O.strang_step(f, P, 0.13)
    got = np.einsum("ai,bj,ck->abcijk", *[O.strang_step_plane(gs[d], P, d, 0.13) for d in range(3)])
    assert O.rel_l2(got, want) < 1e-13
    # the same factor maps with the k-shift reversed do not reproduce the step
    Pm = O.Problem(nx=P.nx, nk=P.nk, x_lo=P.x_lo, x_hi=P.x_hi, lk=P.lk, nuclei=[], kappa=-0.8,
                   center=P.center)
    bad = np.einsum("ai,bj,ck->abcijk", *[O.strang_step_plane(gs[d], Pm, d, 0.13) for d in range(3)])
    assert O.rel_l2(bad, want) > 1e-3
