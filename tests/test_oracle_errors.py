"""Pins of the error metrics of Sec. 5 in the oracle: eps_inf (largest pointwise deviation),
eps_2 (square root of the integral of the squared deviation, the integral as the grid sum times
the cell volume) and eps_mass (|integral of f_num(t) - f_ref(0)|), on inputs whose values follow
by hand: a constant offset, isolated perturbed cells, and a cell volume built from the grid
spacings written out here."""
import math

import numpy as np
import pytest

from oracle import chasm_oracle as O


@pytest.fixture
def prob():
    # unequal spacings in every x-dimension, so a dropped or repeated factor of the volume shows
    return O.Problem(nx=(5, 6, 7), nk=4, x_lo=(-2.0, -3.0, -1.0), x_hi=(1.0, 2.5, 2.6), lk=1.4)


def _vol():
    # h = (hi - lo)/(n - 1) per dimension and dk = 2 L_k / N_k, by hand for the fixture
    h1, h2, h3 = 3.0 / 4, 5.5 / 5, 3.6 / 6
    dk = 2 * 1.4 / 4
    return h1 * h2 * h3 * dk ** 3


def test_cell_volume_by_hand(prob):
    assert [prob.hs(d) for d in range(3)] == pytest.approx([0.75, 1.1, 0.6], rel=1e-15)
    assert O.cell_volume(prob) == pytest.approx(_vol(), rel=1e-15)


def test_errors_of_a_constant_offset(prob):
    rng = np.random.default_rng(3)
    f_ref = rng.standard_normal(prob.shape)
    c = -0.37
    e_inf, e2 = O.errors(f_ref, f_ref + c, prob)
    n_cells = 5 * 6 * 7 * 4 ** 3
    assert e_inf == pytest.approx(abs(c), rel=1e-12)
    assert e2 == pytest.approx(abs(c) * math.sqrt(n_cells * _vol()), rel=1e-12)


def test_errors_of_isolated_cells_take_the_absolute_maximum(prob):
    """Two perturbed cells of opposite sign: the larger magnitude is the negative one (a signed
    maximum would return 0.2), and eps_2 is sqrt((0.5^2 + 0.2^2) vol)."""
    rng = np.random.default_rng(4)
    f_ref = rng.standard_normal(prob.shape)
    f_num = f_ref.copy()
    f_num[1, 2, 3, 0, 1, 2] += 0.5       # f_ref - f_num = -0.5 there
    f_num[4, 0, 6, 3, 3, 3] -= 0.2       # +0.2 there
    e_inf, e2 = O.errors(f_ref, f_num, prob)
    assert e_inf == pytest.approx(0.5, rel=1e-12)
    assert e2 == pytest.approx(math.sqrt((0.25 + 0.04) * _vol()), rel=1e-12)
    # symmetric in its arguments
    assert O.errors(f_num, f_ref, prob) == pytest.approx((e_inf, e2), rel=1e-15)


def test_errors_with_a_plain_cell_volume():
    """Functions of k alone (Example 4.1): the cell volume is dk^3."""
    a = np.zeros((8, 8, 8))
    b = a.copy()
    b[2, 3, 4] = 3.0
    dk = 0.25
    assert O.errors(a, b, dk ** 3) == pytest.approx((3.0, 3.0 * dk ** 1.5), rel=1e-14)


def test_mass_error(prob):
    rng = np.random.default_rng(5)
    f0 = rng.random(prob.shape)
    f1 = f0.copy()
    f1[0, 0, 0, 0, 0, 0] -= 0.125
    f1[2, 3, 4, 1, 2, 3] += 0.5
    assert O.mass_error(f1, f0, prob) == pytest.approx(0.375 * _vol(), rel=1e-12)
    f1[2, 3, 4, 1, 2, 3] -= 1.0          # net -0.625: eps_mass takes the absolute value
    assert O.mass_error(f1, f0, prob) == pytest.approx(0.625 * _vol(), rel=1e-12)
