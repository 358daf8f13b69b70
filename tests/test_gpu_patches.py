"""GPU parity of the PMBC patch decomposition (p > 1 patches per x-dimension, Sec. 3.1.2-3.1.3)
through the C ABI against the oracle's patch transform (FP64 <= 1e-12, FP32-mixed <= 1e-5)."""
import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def _solver(ch, prob, name, patches):
    return ch.Solver(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, kappa=prob.kappa,
                     precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED, n_nb=prob.n_nb,
                     patches=patches)


def _input(prob, seed):
    rng = np.random.default_rng(seed)
    pk = [synth.packet(rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 3)) for _ in range(2)]
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    return f + 1e-3 * rng.standard_normal(f.shape) * f.max()


def _dev(a, name):
    return torch.from_numpy(np.ascontiguousarray(a)).to(
        device="cuda", dtype=torch.float64 if name == "fp64" else torch.float32)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("patches,n_nb,tau", [((3, 2, 4), 5, 0.23), ((3, 2, 4), 20, -0.41),
                                              ((4, 1, 2), 3, 1.7), ((2, 4, 1), 8, 0.0)])
def test_patch_advection_matches_oracle(ch, name, patches, n_nb, tau):
    prob = O.Problem(nx=(13, 9, 17), nk=8, x_lo=(-3.0, -2.0, -3.5), x_hi=(3.0, 2.5, 3.0), lk=3.0,
                     n_nb=n_nb)
    f0 = _input(prob, 5)
    with _solver(ch, prob, name, patches) as s:
        f = _dev(f0, name)
        s.advect(f, tau)
        s.sync()
        got = f.double().cpu().numpy()
    fo = f0.astype(np.float32).astype(np.float64) if name == "fp32" else f0
    ref = O.advect_patches(fo, prob, tau, patches)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


def test_patches_with_full_stencils_equal_one_patch(ch):
    """n_nb >= N: every patch spline is the global one, so p > 1 reproduces p = 1 on the GPU."""
    prob = O.Problem(nx=(13, 9, 17), nk=8, x_lo=(-3.0,) * 3, x_hi=(3.0,) * 3, lk=3.0, n_nb=20)
    f0 = _input(prob, 9)
    outs = []
    for patches in ((1, 1, 1), (4, 2, 4)):
        with _solver(ch, prob, "fp64", patches) as s:
            f = _dev(f0, "fp64")
            s.advect(f, 0.37)
            s.sync()
            outs.append(f.cpu().numpy())
    assert O.rel_l2(outs[1], outs[0]) <= 1e-12


def test_patch_strang_steps_run_and_conserve_mass_like_one_patch(ch):
    """Full Strang steps with patches (harmonic potential): the result stays within the
    truncation error of one patch at n_nb = 10."""
    prob = O.Problem(nx=(13, 13, 13), nk=8, x_lo=(-4.0,) * 3, x_hi=(4.0,) * 3, lk=4.0, kappa=1.0,
                     n_nb=10)
    pk = [synth.packet((0.5, -0.2, 0.1), (0.3, 0.0, -0.2))]
    f0 = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    outs, masses = [], []
    for patches in ((1, 1, 1), (3, 4, 2)):
        with _solver(ch, prob, "fp64", patches) as s:
            f = _dev(f0, "fp64")
            s.step(f, 0.05, 4)
            s.sync()
            outs.append(f.cpu().numpy())
            masses.append(s.mass(f))
    assert O.rel_l2(outs[1], outs[0]) < 1e-4
    assert abs(masses[1] - masses[0]) < 1e-4 * masses[0]
