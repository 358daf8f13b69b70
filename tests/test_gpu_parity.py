"""GPU parity: every substep and the full Strang step through the C ABI against the FP64 oracle.

Tolerances (relative L2 against the FP64 oracle on the same seeded input):
  FP64 form           <= 1e-12
  FP32-mixed form     <= 1e-5   (FP32 storage/FFT arithmetic; the input handed to the oracle is the
                                 same FP32-rounded array, promoted to FP64)
Mass agrees with the oracle's to 1e-6 relative in both forms.
"""
import math

import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
FORMS = ["table", "modulated"]


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()   # fails loudly if the library is missing
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def prec(ch, name):
    return ch.FP64 if name == "fp64" else ch.FP32_MIXED


def dtype(name):
    return torch.float64 if name == "fp64" else torch.float32


def to_dev(a, name):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype(name))


def oracle_input(a, name):
    """The array the oracle sees: the same values the GPU received (FP32-rounded for fp32)."""
    return a.astype(np.float32).astype(np.float64) if name == "fp32" else a


def problem(nx, nk, lo, hi, lk, **kw):
    nx = tuple(nx) if hasattr(nx, "__len__") else (nx,) * 3
    lo = tuple(lo) if hasattr(lo, "__len__") else (lo,) * 3
    hi = tuple(hi) if hasattr(hi, "__len__") else (hi,) * 3
    return O.Problem(nx=nx, nk=nk, x_lo=lo, x_hi=hi, lk=lk, **kw)


def theta_form(ch, form):
    return {"table": ch.THETA_TABLE, "modulated": ch.THETA_MODULATED, "auto": ch.THETA_AUTO}[form]


def solver(ch, prob, name, form="auto", **kw):
    kw.setdefault("theta_form", theta_form(ch, form))
    return ch.Solver(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, nuclei=prob.nuclei,
                     kappa=prob.kappa, center=prob.center, hbar=prob.hbar, m=prob.m,
                     precision=prec(ch, name), n_nb=prob.n_nb, **kw)


def rough_input(prob, seed):
    """Seeded smooth packets plus a small seeded perturbation (exercises every stencil tap)."""
    rng = np.random.default_rng(seed)
    pk = [synth.packet(rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 3)) for _ in range(2)]
    f = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    return f + 1e-3 * rng.standard_normal(f.shape) * f.max()


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nk", [8, 16, 32])
def test_symbol_tensor_matches_oracle(ch, nk):
    prob = problem(5, nk, -2, 2, 4.0, nuclei=[((0.0, 0.0, 0.0), 1.0)])
    with solver(ch, prob, "fp64") as s:
        out = np.zeros((2 * nk - 1,) * 3)
        s.tkm_tensor(out.ctypes.data)
    ref = O.tkm_tensor(nk, 4.0)
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk,nx", [(8, (5, 4, 6)), (16, (4, 5, 4)), (32, (4, 4, 5))])
def test_theta_matches_oracle(ch, name, nk, nx, form):
    prob = problem(nx, nk, (-2.0, -1.5, -2.5), (2.5, 1.0, 2.0), 4.0,
                   nuclei=[((0.3, -0.2, 0.1), 1.0), ((-0.4, 0.25, -0.3), 0.7)])
    f0 = rough_input(prob, 11)
    with solver(ch, prob, name, form) as s:
        u = to_dev(f0, name)
        out = torch.empty_like(u)
        s.theta(u, out)
        s.sync()
        got = out.double().cpu().numpy()
    ref = O.theta_coulomb(oracle_input(f0, name), prob)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", [0.0, 0.23, -0.41, 1.7])
def test_advect_matches_oracle(ch, name, tau):
    prob = problem((9, 7, 8), 8, (-3.0, -2.0, -3.5), (3.0, 2.5, 3.0), 3.0, kappa=0.0, n_nb=20)
    f0 = rough_input(prob, 5)
    with solver(ch, prob, name) as s:
        f = to_dev(f0, name)
        s.advect(f, tau)
        s.sync()
        got = f.double().cpu().numpy()
    ref = O.advect(oracle_input(f0, name), prob, tau)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("n_nb", [3, 10, 40])
def test_advect_truncated_stencils_match_oracle(ch, n_nb):
    prob = problem((12, 5, 6), 8, -4.0, 4.0, 3.0, n_nb=n_nb)
    f0 = rough_input(prob, 7)
    with solver(ch, prob, "fp64") as s:
        f = to_dev(f0, "fp64")
        s.advect(f, 0.3)
        s.sync()
        got = f.cpu().numpy()
    assert O.rel_l2(got, O.advect(f0, prob, 0.3)) <= 1e-12


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", ["fp64", "fp32"])
def test_pflow_coulomb_matches_oracle(ch, name, form):
    prob = problem((4, 5, 4), 16, (-2.0, -1.5, -2.0), (2.0, 1.5, 2.5), 4.0,
                   nuclei=[((0.1, 0.2, -0.1), 1.0)])
    f0 = rough_input(prob, 3)
    with solver(ch, prob, name, form) as s:
        f = to_dev(f0, name)
        s.pflow(f, 0.05)
        s.sync()
        got = f.double().cpu().numpy()
    ref = O.pflow_coulomb(oracle_input(f0, name), prob, 0.05)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk", [8, 16])
def test_pflow_harmonic_matches_oracle(ch, name, nk):
    prob = problem((5, 4, 6), nk, -2.0, 2.0, 3.0, kappa=0.8, center=(0.1, -0.2, 0.3))
    f0 = rough_input(prob, 9)
    with solver(ch, prob, name) as s:
        f = to_dev(f0, name)
        s.pflow(f, 0.17)
        s.sync()
        got = f.double().cpu().numpy()
    ref = O.pflow_harmonic(oracle_input(f0, name), prob, 0.17)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["coulomb1", "coulomb2", "coulomb2-modulated", "harmonic"])
def test_strang_steps_match_oracle(ch, name, case):
    form = "modulated" if case.endswith("modulated") else "table"
    if case == "harmonic":
        prob = problem((9, 8, 7), 8, -4.0, 4.0, 4.0, kappa=1.0)
        nsteps, dt = 3, 0.05
    else:
        nuc = [((0.2, 0.1, -0.1), 1.0)] if case == "coulomb1" else \
              [((0.7, 0.0, 0.0), 1.0), ((-0.7, 0.0, 0.0), 1.0)]
        prob = problem((7, 6, 8), 8, (-4.0, -3.0, -4.0), (4.0, 3.5, 3.5), 4.0, nuclei=nuc)
        nsteps, dt = 2, 0.025
    pk = [synth.packet((0.5, -0.2, 0.1), (0.3, 0.0, -0.2))]
    f0 = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    with solver(ch, prob, name, "auto" if case == "harmonic" else form) as s:
        f = to_dev(f0, name)
        s.step(f, dt, nsteps)
        s.sync()
        got = f.double().cpu().numpy()
        m_gpu = s.mass(f)
    ref = O.run(oracle_input(f0, name), prob, dt, nsteps)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)
    m_ref = O.mass(ref, prob)
    assert abs(m_gpu - m_ref) <= 1e-6 * abs(m_ref)


def test_graph_replay_equals_direct_launches(ch):
    prob = problem((6, 5, 7), 8, -3.0, 3.0, 3.0, nuclei=[((0.1, 0.0, 0.2), 1.0)])
    f0 = rough_input(prob, 21)
    outs = []
    for graphs in (True, False):
        with solver(ch, prob, "fp32", use_graphs=graphs) as s:
            f = to_dev(f0, "fp32")
            s.step(f, 0.02, 3)
            s.sync()
            outs.append(f.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("name", ["fp64", "fp32"])
def test_moments_match_oracle_and_are_reproducible(ch, name):
    prob = problem((7, 9, 6), 16, -3.0, 3.0, 4.0, nuclei=[((0.15, 0.05, 0.0), 1.0)])
    f0 = rough_input(prob, 4)
    with solver(ch, prob, name) as s:
        f = to_dev(f0, name)
        m1, e1 = s.moments(f)
        m2, e2 = s.moments(f)
    fo = oracle_input(f0, name)
    assert m1 == m2 and e1 == e2
    assert m1 == pytest.approx(O.mass(fo, prob), rel=1e-12)
    assert e1 == pytest.approx(O.energy(fo, prob), rel=1e-12)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk,npk", [(8, 2), (16, 5), (32, 16)])
def test_init_gaussians_matches_generator(ch, name, nk, npk):
    prob = problem((5, 6, 7) if nk < 32 else (4, 5, 4), nk, -3.0, 3.0, 3.0)
    rng = np.random.default_rng(nk + npk)
    pk = [synth.packet((0.5, -0.2, 0.1), (0.3, 0.0, -0.2)), synth.packet((-1, 1, 0), (0, 0, 0.5))]
    pk += [synth.packet(rng.uniform(-2, 2, 3), rng.uniform(-1, 1, 3), ax=rng.uniform(0.2, 1.0),
                        ak=rng.uniform(0.5, 3.0), w=rng.uniform(-0.5, 1.0)) for _ in range(npk - 2)]
    with solver(ch, prob, name) as s:
        f = torch.empty(prob.shape, device="cuda", dtype=dtype(name))
        s.init_gaussians(f, pk)
        s.sync()
        got = f.double().cpu().numpy()
    ref = synth.gaussian_packets(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, pk)
    assert O.rel_l2(got, ref) <= (1e-14 if name == "fp64" else 1e-7)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
def test_init_hydrogen_1s_matches_generator(ch, name):
    # The FP32-mixed form sums the 1s samples in FP32 before the FP64 DFT.
    prob = problem((4, 5, 4), 8, (-2.0, -1.5, -1.0), (2.0, 1.5, 1.0), 4.0)
    with solver(ch, prob, name) as s:
        f = torch.empty(prob.shape, device="cuda", dtype=dtype(name))
        s.init_hydrogen_1s(f, n_y=32)
        s.sync()
        got = f.double().cpu().numpy()
    ref = synth.wigner_1s(prob.nx, prob.nk, prob.x_lo, prob.x_hi, prob.lk, n_y=32)
    assert O.rel_l2(got, ref) <= (1e-12 if name == "fp64" else 1e-6)


def test_errors_are_reported_not_raised_on_device(ch):
    prob = problem(6, 8, -3.0, 3.0, 3.0, nuclei=[((0.0, 0.0, 0.0), 1.0)])
    with solver(ch, prob, "fp32") as s:
        f = torch.zeros(prob.shape, device="cuda", dtype=torch.float32)
        with pytest.raises(ch.ChasmError) as e:
            s.step(f, 10.0, 1)            # far beyond the Taylor-4 stability bound
        assert e.value.code == ch.chasm.EUNSTABLE
        with pytest.raises(ch.ChasmError) as e:
            s.step(f, -0.1, 1)
        assert e.value.code == ch.chasm.EINVAL
        with pytest.raises(ch.ChasmError):
            s.theta(f, f)                 # aliasing is rejected
        s.step(f, 0.01, 1)                # the handle is still usable
        s.sync()


@pytest.mark.parametrize("variant", ["global", "cluster"])
@pytest.mark.parametrize("name,nk,nx", [("fp32", 32, (4, 5, 4)), ("fp32", 16, (6, 5, 4)),
                                        ("fp64", 16, (4, 5, 6)), ("fp32", 8, (7, 5, 6))])
def test_theta_kernel_variants_match_oracle(ch, monkeypatch, variant, name, nk, nx):
    """Both implementations of the modulated-form Theta kernel (per-CTA global scratch, and the
    spectrum held in the shared memory of one CTA or of a thread-block cluster) against the
    oracle, with two nuclei so the per-nucleus accumulation is exercised."""
    monkeypatch.setenv("CHASM_THETA_VARIANT", variant)
    prob = problem(nx, nk, (-2.0, -1.5, -2.5), (2.5, 1.0, 2.0), 4.0,
                   nuclei=[((0.3, -0.2, 0.1), 1.0), ((-0.4, 0.25, -0.3), 0.7)])
    f0 = rough_input(prob, 13)
    with solver(ch, prob, name, "modulated") as s:
        u = to_dev(f0, name)
        out = torch.empty_like(u)
        s.theta(u, out)
        base = to_dev(f0 * 0.5, name)
        s.pflow(base, 0.02)
        s.sync()
        got = out.double().cpu().numpy()
        got_p = base.double().cpu().numpy()
    ref = O.theta_coulomb(oracle_input(f0, name), prob)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)
    ref_p = O.pflow_coulomb(oracle_input(f0 * 0.5, name), prob, 0.02)
    assert O.rel_l2(got_p, ref_p) <= TOL[name], O.rel_l2(got_p, ref_p)


@pytest.mark.parametrize("name,nk,nx", [("fp32", 32, (5, 7, 9)), ("fp64", 32, (4, 4, 5)),
                                        ("fp32", 16, (11, 9, 7)), ("fp64", 8, (9, 8, 7))])
def test_table_form_many_points_three_nuclei(ch, name, nk, nx):
    """Table form with more x points than one wave of CTAs covers (ragged last wave), three
    nuclei folded into one symbol, Theta out of place and P(dt) in place."""
    prob = problem(nx, nk, (-3.0, -2.5, -3.5), (3.5, 2.0, 3.0), 4.0,
                   nuclei=[((0.3, -0.2, 0.1), 1.0), ((-0.4, 0.25, -0.3), 0.7),
                           ((1.1, 0.6, -0.9), 2.0)])
    f0 = rough_input(prob, 17)
    with solver(ch, prob, name, "table") as s:
        u = to_dev(f0, name)
        out = torch.empty_like(u)
        s.theta(u, out)
        s.pflow(u, 0.01)
        s.sync()
        got = out.double().cpu().numpy()
        got_p = u.double().cpu().numpy()
    fo = oracle_input(f0, name)
    ref = O.theta_coulomb(fo, prob)
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)
    ref_p = O.pflow_coulomb(fo, prob, 0.01)
    assert O.rel_l2(got_p, ref_p) <= TOL[name], O.rel_l2(got_p, ref_p)


def test_table_and_modulated_forms_agree(ch):
    """The two evaluations of the same operator on the same FP64 input agree to rounding."""
    prob = problem((6, 5, 7), 16, -3.0, 3.0, 4.0, nuclei=[((0.2, -0.1, 0.3), 1.0),
                                                          ((-0.6, 0.4, 0.0), 1.0)])
    f0 = rough_input(prob, 23)
    outs = []
    for form in FORMS:
        with solver(ch, prob, "fp64", form) as s:
            f = to_dev(f0, "fp64")
            s.step(f, 0.02, 2)
            s.sync()
            outs.append(f.cpu().numpy())
    assert O.rel_l2(outs[0], outs[1]) <= 1e-13


@pytest.mark.parametrize("form", FORMS)
def test_nucleus_on_a_grid_node(ch, form):
    """Degenerate x point: at x = x_A the modulation is 1 (the per-x kernel sin(2 (x - x_A).m dk)
    vanishes), so Theta^T is zero there up to rounding; elsewhere it matches the oracle."""
    prob = problem((5, 5, 5), 16, -2.0, 2.0, 4.0, nuclei=[((0.0, 1.0, -1.0), 1.0)])
    f0 = rough_input(prob, 41)
    with solver(ch, prob, "fp64", form) as s:
        u = to_dev(f0, "fp64")
        out = torch.empty_like(u)
        s.theta(u, out)
        s.sync()
        got = out.cpu().numpy()
    assert np.max(np.abs(got[2, 3, 1])) <= 1e-13 * np.max(np.abs(got))   # x_A is node (2, 3, 1)
    ref = O.theta_coulomb(f0, prob)
    assert O.rel_l2(got, ref) <= TOL["fp64"]


@pytest.mark.parametrize("name", ["fp64", "fp32"])
def test_zero_data_and_zero_steps(ch, name):
    prob = problem((6, 5, 4), 8, -3.0, 3.0, 3.0, nuclei=[((0.1, 0.0, 0.2), 1.0)])
    f0 = rough_input(prob, 43)
    with solver(ch, prob, name) as s:
        z = torch.zeros(prob.shape, device="cuda", dtype=dtype(name))
        s.step(z, 0.02, 2)
        f = to_dev(f0, name)
        before = f.clone()
        s.step(f, 0.02, 0)
        s.sync()
        assert int(torch.count_nonzero(z)) == 0
        assert torch.equal(f, before)


@pytest.mark.parametrize("graphs", [True, False])
def test_launch_count_counts_the_step_kernels(ch, graphs):
    """chasm_launch_count: a Strang step is 6 advection passes and one P(dt) launch in the table
    form (P(dt) as four Theta launches in the modulated form); a graph replay counts its kernels;
    an LPC1 step in the table form is Theta, two advections and the corrector launch."""
    prob = problem((6, 5, 7), 8, -3.0, 3.0, 3.0, nuclei=[((0.1, 0.0, 0.2), 1.0)])
    f0 = rough_input(prob, 23)
    cases = [("table", ch.STRANG, 7), ("modulated", ch.STRANG, 10), ("table", ch.LPC1, 8)]
    for form, integ, per_step in cases:
        with solver(ch, prob, "fp32", form, use_graphs=graphs, integrator=integ) as s:
            f = to_dev(f0, "fp32")
            for n in (1, 3):
                c0 = s.launch_count()
                s.step(f, 0.02, n)
                assert s.launch_count() - c0 == per_step * n, (form, integ, n)
            c0 = s.launch_count()
            s.advect(f, 0.01)
            assert s.launch_count() - c0 == 3
            s.sync()
