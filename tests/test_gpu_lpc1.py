"""GPU parity of the LPC1 integrator (Sec. 2.2) and of Theta for the quadratic potential (Eq. 5.1),
through the C ABI, against the FP64 oracle (relative L2: FP64 <= 1e-12, FP32-mixed <= 1e-5; mass
<= 1e-6 relative)."""
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


def to_dev(a, name):
    return torch.from_numpy(np.ascontiguousarray(a)).to(
        device="cuda", dtype=torch.float64 if name == "fp64" else torch.float32)


def oracle_input(a, name):
    return a.astype(np.float32).astype(np.float64) if name == "fp32" else a


def solver(ch, prob, name, form="auto", integrator=None, **kw):
    tf = {"table": ch.THETA_TABLE, "modulated": ch.THETA_MODULATED, "auto": ch.THETA_AUTO}[form]
    return ch.Solver(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, nuclei=prob.nuclei,
                     kappa=prob.kappa, center=prob.center, hbar=prob.hbar, m=prob.m,
                     precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED, n_nb=prob.n_nb,
                     theta_form=tf, integrator=ch.LPC1 if integrator is None else integrator, **kw)


def rough_input(prob, seed):
    rng = np.random.default_rng(seed)
    pk = [synth.packet(rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 3)) for _ in range(2)]
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    return f + 1e-3 * rng.standard_normal(f.shape) * f.max()


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk,nx", [(8, (5, 4, 6)), (16, (4, 5, 4)), (32, (4, 4, 5))])
def test_theta_harmonic_matches_oracle(ch, name, nk, nx):
    prob = O.Problem(nx=nx, nk=nk, x_lo=(-2.0, -1.5, -2.5), x_hi=(2.5, 1.0, 2.0), lk=4.0,
                     kappa=0.9, center=(0.2, -0.1, 0.3), hbar=1.2)
    f0 = rough_input(prob, 2)
    with solver(ch, prob, name) as s:
        u = to_dev(f0, name)
        out = torch.empty_like(u)
        s.theta(u, out)
        s.sync()
        got = out.double().cpu().numpy()
    ref = O.theta_harmonic(oracle_input(f0, name), prob)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["coulomb-table", "coulomb2-modulated", "harmonic"])
def test_lpc1_steps_match_oracle(ch, name, case):
    if case == "harmonic":
        prob = O.Problem(nx=(9, 8, 7), nk=8, x_lo=(-4.0,) * 3, x_hi=(4.0,) * 3, lk=4.0, kappa=1.0)
        nsteps, dt, form = 3, 0.02, "auto"
    else:
        nuc = [((0.2, 0.1, -0.1), 1.0)] if case == "coulomb-table" else \
              [((0.7, 0.0, 0.0), 1.0), ((-0.7, 0.0, 0.0), 1.0)]
        prob = O.Problem(nx=(7, 6, 8), nk=8, x_lo=(-4.0, -3.0, -4.0), x_hi=(4.0, 3.5, 3.5), lk=4.0,
                         nuclei=nuc)
        nsteps, dt = 2, 0.02            # dt rho <= 0.92 with two nuclei
        form = "table" if case == "coulomb-table" else "modulated"
    pk = [synth.packet((0.5, -0.2, 0.1), (0.3, 0.0, -0.2))]
    f0 = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    with solver(ch, prob, name, form) as s:
        f = to_dev(f0, name)
        s.step(f, dt, nsteps)
        s.sync()
        got = f.double().cpu().numpy()
        m_gpu = s.mass(f)
    ref = O.run_lpc1(oracle_input(f0, name), prob, dt, nsteps)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)
    m_ref = O.mass(ref, prob)
    assert abs(m_gpu - m_ref) <= 1e-6 * abs(m_ref)


def test_lpc1_many_points_three_nuclei(ch):
    """Table form, N_k = 32, more x points than one wave of CTAs, three nuclei, one LPC1 step."""
    prob = O.Problem(nx=(5, 6, 7), nk=32, x_lo=(-3.0, -2.5, -3.5), x_hi=(3.5, 2.0, 3.0), lk=4.0,
                     nuclei=[((0.3, -0.2, 0.1), 1.0), ((-0.4, 0.25, -0.3), 0.7),
                             ((1.1, 0.6, -0.9), 2.0)])
    f0 = rough_input(prob, 8)
    with solver(ch, prob, "fp32", "table") as s:
        f = to_dev(f0, "fp32")
        s.step(f, 0.01, 1)
        s.sync()
        got = f.double().cpu().numpy()
    ref = O.lpc1_step(oracle_input(f0, "fp32"), prob, 0.01)
    assert O.rel_l2(got, ref) <= TOL["fp32"], O.rel_l2(got, ref)


def test_lpc1_graph_replay_equals_direct_launches(ch):
    prob = O.Problem(nx=(6, 5, 7), nk=8, x_lo=(-3.0,) * 3, x_hi=(3.0,) * 3, lk=3.0,
                     nuclei=[((0.1, 0.0, 0.2), 1.0)])
    f0 = rough_input(prob, 21)
    outs = []
    for graphs in (True, False):
        with solver(ch, prob, "fp32", use_graphs=graphs) as s:
            f = to_dev(f0, "fp32")
            s.step(f, 0.02, 3)
            s.sync()
            outs.append(f.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_lpc1_stability_limit_is_enforced(ch):
    prob = O.Problem(nx=(6, 6, 6), nk=16, x_lo=(-6.0,) * 3, x_hi=(6.0,) * 3, lk=4.0, kappa=1.0)
    with solver(ch, prob, "fp32") as s:
        f = torch.zeros(prob.shape, device="cuda", dtype=torch.float32)
        with pytest.raises(ch.ChasmError) as e:
            s.step(f, 0.05, 1)            # dt rho = 5 for this grid (the Sec. 5.1 stiffness)
        assert e.value.code == ch.chasm.EUNSTABLE
        s.step(f, 0.005, 1)               # within the limit; the handle is still usable
        s.sync()


# ------------------------------------------------------------------------------------------------
# Phase-space diagnostics (Sec. 5)
@pytest.mark.parametrize("name,nk,nx", [("fp64", 8, (7, 5, 6)), ("fp32", 16, (6, 7, 5)),
                                        ("fp32", 32, (4, 5, 6))])
def test_diagnostics_match_oracle_and_are_reproducible(ch, name, nk, nx):
    prob = O.Problem(nx=nx, nk=nk, x_lo=(-3.0, -2.5, -2.0), x_hi=(2.5, 3.0, 2.0), lk=3.5,
                     nuclei=[((0.1, 0.2, -0.1), 1.0)])
    f0 = rough_input(prob, 12)
    fo = oracle_input(f0, name)
    tol = 1e-12
    with solver(ch, prob, name, integrator=ch.STRANG) as s:
        f = to_dev(f0, name)
        for j in range(3):
            w = s.reduced_wigner(f, j)
            ref = O.reduced_wigner(fo, prob, j)
            assert np.max(np.abs(w - ref)) <= tol * np.max(np.abs(ref))
            assert np.array_equal(w, s.reduced_wigner(f, j))
        p = s.marginal_x12(f)
        ref = O.marginal_x12(fo, prob)
        assert np.max(np.abs(p - ref)) <= tol * np.max(np.abs(ref))
        e = np.array(s.expectations(f))
        assert np.allclose(e, O.expectations(fo, prob), rtol=0, atol=1e-12)
        assert np.array_equal(e, np.array(s.expectations(f)))


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk", [16, 32])
def test_lpc1_table_form_with_patches_matches_oracle(ch, name, nk):
    """LPC1 in the table form at N_k = 16 and 32 (the Theta kernel forms the predictor and the
    corrector base itself) with p > 1 PMBC patches in two x-dimensions: steps against the
    oracle's LPC1 combination (Sec. 2.2) of its patch advection and Theta."""
    patches = (3, 2, 1)
    prob = O.Problem(nx=(7, 5, 4), nk=nk, x_lo=(-3.0, -2.5, -2.0), x_hi=(3.5, 2.0, 2.5), lk=4.0,
                     nuclei=[((0.35, -0.2, 0.15), 1.0)], n_nb=4)
    f0 = rough_input(prob, 31)
    dt, nsteps = 0.015, (2 if nk == 16 else 1)   # the oracle's N_k = 32 Theta takes seconds
    with solver(ch, prob, name, "table", patches=patches) as s:
        f = to_dev(f0, name)
        s.step(f, dt, nsteps)
        s.sync()
        got = f.double().cpu().numpy()
    T = O.tkm_tensor(prob.nk, prob.lk)
    ref = oracle_input(f0, name)
    for _ in range(nsteps):
        ref = O.lpc1_combine(ref, lambda u: O.advect_patches(u, prob, dt, patches),
                             lambda u: O.theta(u, prob, T), dt)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)
