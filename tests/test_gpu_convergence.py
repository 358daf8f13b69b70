"""Spatial convergence study of the GPU steps (Sec. 5.1): the 6-D quantum harmonic oscillator
(hbar = m = kappa = 1) rotates every (x_d, k_d) phase plane rigidly, so the exact solution of a
product of Gaussians is known in closed form.  With a small time step the error is dominated by
the cubic-spline interpolation in x, which the paper observes to converge at fourth order in
the grid spacing; the oracle's plane step shows the same (errors 2.7e-2, 4.6e-3, 1.2e-3 at
N_x = 16, 24, 32 on [-6, 6] for Strang, dt = 0.0125, T = 0.5)."""
import math

import numpy as np
import pytest

from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

X0, K0 = (1.0, -0.5, 0.3), (0.5, 0.2, -0.4)


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def _exact_slab(prob, t, i1):
    """f0(R(-t)(x, k)) at x1 index i1 for f0 = pi^-3 exp(-|x - X0|^2 - |k - K0|^2): the product over
    d of the rotated (x_d, k_d) Gaussians.  Shape (nx2, nx3, N, N, N)."""
    g = []
    for d in range(3):
        X, K = np.meshgrid(prob.xs(d), prob.ks(), indexing="ij")
        Xr, Kr = O.harmonic_rotation(X, K, t, 1.0)
        g.append(np.exp(-(Xr - X0[d]) ** 2 - (Kr - K0[d]) ** 2) / math.pi)
    return (g[0][i1][None, None, :, None, None] * g[1][:, None, None, :, None]
            * g[2][None, :, None, None, :])


def _run(ch, nx, integrator, dt, T, name="fp64"):
    prob = O.Problem(nx=(nx,) * 3, nk=32, x_lo=(-6.0,) * 3, x_hi=(6.0,) * 3, lk=4.0, kappa=1.0)
    with ch.Solver(nx, 32, -6.0, 6.0, 4.0, kappa=1.0, integrator=integrator,
                   precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED) as s:
        f = torch.empty(prob.shape, device="cuda",
                        dtype=torch.float64 if name == "fp64" else torch.float32)
        s.init_gaussians(f, [{"w": math.pi ** -3, "x0": X0, "k0": K0, "ax": 1.0, "ak": 1.0}])
        s.step(f, dt, int(round(T / dt)))
        s.sync()
        num = den = 0.0
        for i1 in range(nx):        # slab by slab against the closed form
            ref = _exact_slab(prob, T, i1)
            got = f[i1].double().cpu().numpy()
            num += float(np.sum((got - ref) ** 2))
            den += float(np.sum(ref ** 2))
    return math.sqrt(num / den)


@pytest.mark.parametrize("integrator,dt", [("strang", 0.0125), ("lpc1", 0.004)])
def test_harmonic_oscillator_converges_at_fourth_order_in_h(ch, integrator, dt):
    integ = ch.STRANG if integrator == "strang" else ch.LPC1
    errs = {nx: _run(ch, nx, integ, dt, 0.5, "fp32") for nx in (16, 24, 32)}
    h = {nx: 12.0 / (nx - 1) for nx in errs}
    order = math.log(errs[16] / errs[32]) / math.log(h[16] / h[32])
    print(integrator, errs, "order", order)
    assert errs[32] < 3e-3
    assert errs[16] > errs[24] > errs[32]
    assert 3.5 < order < 5.0, (errs, order)
