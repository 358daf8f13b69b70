"""Parity at the full benchmark size (32^3 x 32^3 on [-12,12]^3 x [-4,4)^3, Coulomb nucleus at the
origin), in the launch configuration the benchmark times.

The oracle cannot run the whole 1.07e9-cell step, so each substep is checked on samples it can
compute one at a time: A(tau) is independent per k point (the full x-cube at a sampled k), P(dt)
is independent per x point (the full k-cube at a sampled x).  The input is a seeded separable
wavepacket, built on the device with torch from 1-D factors and rebuilt in numpy for the oracle.
The accumulated multi-step result of the FP32-mixed form is compared with the FP64 form, which is
itself pinned to the oracle above and in test_gpu_parity.py.
"""
import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NX, NK, L, LK, DT = 32, 32, 12.0, 4.0, 0.025
NUC = [((0.0, 0.0, 0.0), 1.0)]
TOL = {"fp64": 1e-12, "fp32": 1e-5}
PACKET = synth.packet((-1.5, 0.75, 0.5), (0.4, -0.2, 0.1), ax=0.25, ak=1.0)


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available()
    return pkg


def prob():
    return O.Problem(nx=(NX,) * 3, nk=NK, x_lo=(-L,) * 3, x_hi=(L,) * 3, lk=LK, nuclei=NUC)


def factors():
    xs, ks = synth.axes((NX,) * 3, NK, (-L,) * 3, (L,) * 3, LK)
    p = PACKET
    gx = [np.exp(-p["ax"] * (xs[d] - p["x0"][d]) ** 2) for d in range(3)]
    gk = [np.exp(-p["ak"] * (ks - p["k0"][d]) ** 2) for d in range(3)]
    return p["w"], gx, gk


def device_input(name):
    w, gx, gk = factors()
    t = [torch.from_numpy(a).cuda() for a in gx + gk]
    f = (w * t[0][:, None, None, None, None, None] * t[1][None, :, None, None, None, None]
         * t[2][None, None, :, None, None, None] * t[3][None, None, None, :, None, None]
         * t[4][None, None, None, None, :, None] * t[5][None, None, None, None, None, :])
    return f if name == "fp64" else f.float()


def host_at_k(k, name):
    w, gx, gk = factors()
    cube = w * gx[0][:, None, None] * gx[1][None, :, None] * gx[2][None, None, :]
    c = cube * gk[0][k[0]] * gk[1][k[1]] * gk[2][k[2]]
    c = c.astype(np.float32).astype(np.float64) if name == "fp32" else c
    return c[..., None, None, None]


def host_at_x(i, name):
    w, gx, gk = factors()
    kc = gk[0][:, None, None] * gk[1][None, :, None] * gk[2][None, None, :]
    c = w * gx[0][i[0]] * gx[1][i[1]] * gx[2][i[2]] * kc
    return c.astype(np.float32).astype(np.float64) if name == "fp32" else c


def solver(ch, name):
    return ch.Solver(NX, NK, -L, L, LK, nuclei=NUC,
                     precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED)


@pytest.mark.parametrize("name", ["fp32", "fp64"])
def test_fullsize_advection_sampled_k(ch, name):
    P = prob()
    ks = P.ks()
    with solver(ch, name) as s:
        f = device_input(name)
        s.advect(f, 0.5 * DT)
        s.sync()
        for k in [(3, 17, 29), (16, 16, 16), (31, 0, 9)]:
            got = f[:, :, :, k[0], k[1], k[2]].double().cpu().numpy()
            ref = O.advect(host_at_k(k, name), P, 0.5 * DT,
                           kaxes=(ks[k[0]:k[0] + 1], ks[k[1]:k[1] + 1], ks[k[2]:k[2] + 1]))[..., 0, 0, 0]
            assert O.rel_l2(got, ref) <= TOL[name], (k, O.rel_l2(got, ref))


@pytest.mark.parametrize("name", ["fp32", "fp64"])
def test_fullsize_pflow_sampled_x(ch, name):
    P = prob()
    xs = P.xs(0)
    T = O.tkm_tensor(NK, LK)
    with solver(ch, name) as s:
        f = device_input(name)
        s.pflow(f, DT)
        s.sync()
        for i in [(15, 16, 15), (0, 31, 7), (20, 9, 27)]:
            got = f[i[0], i[1], i[2]].double().cpu().numpy()
            x = np.array([[xs[i[0]], xs[i[1]], xs[i[2]]]])
            ref = O.pflow_coulomb(host_at_x(i, name)[None], P, DT, T, xpts=x)[0]
            assert O.rel_l2(got, ref) <= TOL[name], (i, O.rel_l2(got, ref))


def test_fullsize_mixed_form_tracks_fp64_over_steps(ch):
    out = {}
    mass = {}
    for name in ("fp64", "fp32"):
        with solver(ch, name) as s:
            f = device_input(name)
            s.step(f, DT, 4)
            s.sync()
            mass[name] = s.mass(f)
            out[name] = f.double()
            del f
    diff = torch.linalg.vector_norm(out["fp32"] - out["fp64"]) / torch.linalg.vector_norm(out["fp64"])
    assert float(diff) <= 1e-5, float(diff)
    assert abs(mass["fp32"] - mass["fp64"]) <= 1e-6 * abs(mass["fp64"])


def test_fullsize_lpc1_mixed_form_tracks_fp64(ch):
    """The LPC1 integrator at the full size (the bench's lpc1 section): FP32-mixed against FP64
    over two steps (LPC1's FP64 form is pinned to the oracle in test_gpu_lpc1.py)."""
    out = {}
    mass = {}
    for name in ("fp64", "fp32"):
        with ch.Solver(NX, NK, -L, L, LK, nuclei=NUC, integrator=ch.LPC1,
                       precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED) as s:
            f = device_input(name)
            s.step(f, DT, 2)
            s.sync()
            mass[name] = s.mass(f)
            out[name] = f.double()
            del f
    diff = torch.linalg.vector_norm(out["fp32"] - out["fp64"]) / torch.linalg.vector_norm(out["fp64"])
    assert float(diff) <= 1e-5, float(diff)
    assert abs(mass["fp32"] - mass["fp64"]) <= 1e-6 * abs(mass["fp64"])
