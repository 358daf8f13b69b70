"""The PMBC closure (Eq. 3.5) of the FP32-mixed form with long stencils on steep boundary data.

The FP32-mixed advection accumulates the closure dot products phi_L = sum_j c+_j phi_j and phi_R
in compensated FP32 pairs (error-free products by FMA, two-sum; about 48 significant bits) and
runs the rest of the pass in FP32.  Here n_nb = 40 (41 taps per end on a 48-point line, the
register kernel's longest closure), with data whose values near the ends are large against their
derivative (a spike at the left end, a large offset, a steep ramp): the advected values at the
four nodes next to each end, where the closure enters, must match the FP64 oracle to within
1e-6 of the data's scale (a few FP32 units in the last place: the spline of the under-resolved
spike has coefficients of alternating sign larger than the data), for shifts of both signs (all
eight k values of the grid).  A closure accumulated in plain FP32 stays within about 8e-8 on
these data (its rounding reaches f through the end coefficients at the size of FP32 rounding),
so the bound holds the pass as a whole to FP32 rounding at the ends; the closure's own precision
is not observable through f."""
import numpy as np
import pytest

from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available()
    return pkg


def _profile(kind, x, L0):
    if kind == "spike":
        return 1e3 * np.exp(-(x + L0) ** 2 / 0.05) + np.exp(-x ** 2)
    if kind == "offset":
        return 1e4 + np.exp(-x ** 2) + 50 * np.sin(3 * x)
    return 1e4 * (x + L0) + 3e3 * np.cos(2.5 * x)


@pytest.mark.parametrize("kind", ["spike", "offset", "ramp"])
@pytest.mark.parametrize("tau", [0.31, -0.47])
def test_fp32_closure_with_long_stencils_at_the_ends(ch, kind, tau):
    L0, nk, lk = 6.0, 8, 2.0
    prob = O.Problem(nx=(48, 4, 4), nk=nk, x_lo=(-L0, -1.5, -1.5), x_hi=(L0, 1.5, 1.5), lk=lk,
                     nuclei=[], kappa=0.0, n_nb=40)
    x1 = prob.xs(0)
    rng = np.random.default_rng(3)
    side = 1.0 + 0.1 * rng.standard_normal((4, 4, nk, nk, nk))
    f = _profile(kind, x1, L0)[:, None, None, None, None, None] * side[None]
    f32 = f.astype(np.float32)
    with ch.Solver(prob.nx, nk, prob.x_lo, prob.x_hi, lk, nuclei=[], kappa=0.0,
                   precision=ch.FP32_MIXED, n_nb=40) as s:
        fd = torch.from_numpy(f32).to("cuda")
        s.advect(fd, tau)
        s.sync()
        got = fd.double().cpu().numpy()
    ref = O.advect(f32.astype(np.float64), prob, tau)
    scale = np.max(np.abs(ref))
    ends = np.r_[0:4, 44:48]
    assert np.max(np.abs(got[ends] - ref[ends])) <= 1e-6 * scale, np.max(np.abs(got[ends] - ref[ends])) / scale
    assert O.rel_l2(got, ref) <= 1e-6, O.rel_l2(got, ref)
