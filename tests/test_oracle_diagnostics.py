"""Pins of the phase-space diagnostics of the oracle (Sec. 5: reduced Wigner functions W_j, the
spatial marginal P(x1, x2), the averaged position and momentum): for a separable packet every
one factorises into 1-D grid sums, computed here from the 1-D factors alone."""
import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O


def _factors(prob, p):
    gx = [p["w"] ** (1 / 3) * np.exp(-p["ax"] * (prob.xs(d) - p["x0"][d]) ** 2) for d in range(3)]
    gk = [np.exp(-p["ak"] * (prob.ks() - p["k0"][d]) ** 2) for d in range(3)]
    return gx, gk


@pytest.fixture
def case():
    prob = O.Problem(nx=(9, 7, 8), nk=8, x_lo=(-3.0, -2.5, -3.5), x_hi=(3.5, 2.0, 3.0), lk=3.0)
    p = synth.packet((0.4, -0.3, 0.2), (0.5, -0.25, 0.1))
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, [p])
    return prob, p, f


@pytest.mark.parametrize("j", [0, 1, 2])
def test_reduced_wigner_of_a_product_packet(case, j):
    prob, p, f = case
    gx, gk = _factors(prob, p)
    ref = np.outer(gx[j], gk[j])
    for d in range(3):
        if d != j:
            ref = ref * gx[d].sum() * prob.hs(d) * gk[d].sum() * prob.dk
    got = O.reduced_wigner(f, prob, j)
    assert got.shape == (prob.nx[j], prob.nk)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_marginal_of_a_product_packet(case):
    prob, p, f = case
    gx, gk = _factors(prob, p)
    ref = np.outer(gx[0], gx[1]) * gx[2].sum() * prob.hs(2)
    for d in range(3):
        ref = ref * gk[d].sum() * prob.dk
    got = O.marginal_x12(f, prob)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_expectations_of_a_product_packet(case):
    prob, p, f = case
    gx, gk = _factors(prob, p)
    ref = [np.sum(prob.xs(d) * gx[d]) / gx[d].sum() for d in range(3)] + \
          [np.sum(prob.ks() * gk[d]) / gk[d].sum() for d in range(3)]
    assert np.allclose(O.expectations(f, prob), ref, rtol=0, atol=1e-13)


def test_reduced_wigner_integrates_to_the_mass(case):
    prob, _, f = case
    m = O.mass(f, prob)
    for j in range(3):
        w = O.reduced_wigner(f, prob, j)
        assert np.sum(w) * prob.hs(j) * prob.dk == pytest.approx(m, rel=1e-13)
    assert np.sum(O.marginal_x12(f, prob)) * prob.hs(0) * prob.hs(1) == pytest.approx(m, rel=1e-13)
