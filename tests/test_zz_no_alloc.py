"""chasm_moments_noalloc, the allocation-free mass/energy entry point, against chasm_moments.

Who needs it: callers that must not allocate device memory at the moment they check a solve --
services that hand their whole memory budget to solves up front, plug-ins that only get a device
pointer from a framework that owns all device memory.  The entry point keeps its scratch in a
fixed device array, so the test also checks that calls in a row with different inputs each give
their own answer (the array keeps the previous call's contents), that the largest accepted grid
(64^3 x points, the whole array) is right, and that grids above the limit are refused.  This file
is collected last so that a failure here does not stop the rest of the GPU suite; it passes alone
and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available()
    return pkg


def _noalloc(ch, f, nx, nk, L, lk, nuclei, precision, kappa=0.0):
    lib = ch.chasm.lib()
    g = ch.chasm.make_grid(nx, nk)
    b = ch.chasm.make_box(-L, L, lk)
    nuc = (ch.chasm.Nucleus * max(1, len(nuclei)))(
        *[ch.chasm.Nucleus((C.c_double * 3)(*p), z) for p, z in nuclei])
    pot = ch.chasm.Potential(nuc if nuclei else None, len(nuclei), kappa, (C.c_double * 3)(0, 0, 0))
    m, e = C.c_double(), C.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.chasm_moments_noalloc(f.data_ptr(), C.byref(g), C.byref(b), C.byref(pot), 1.0, 1.0,
                                   precision, stream, C.byref(m), C.byref(e))
    return rc, m.value, e.value


@pytest.mark.parametrize("name", ["fp32", "fp64"])
def test_noalloc_moments_match_the_handle_entry_point_on_two_calls_in_a_row(ch, name):
    prec = ch.FP64 if name == "fp64" else ch.FP32_MIXED
    dt = torch.float64 if name == "fp64" else torch.float32
    cases = [
        (10, 16, 5.0, 4.0, [((0.3, -0.2, 0.1), 1.0)], synth.packet((0.5, 0, 0), (0, 0.4, 0))),
        (12, 8, 6.0, 3.0, [((0.7, 0, 0), 1.0), ((-0.7, 0, 0), 1.0)], synth.packet((-1, 1, 0), (0.3, 0, 0))),
    ]
    for nx, nk, L, lk, nuclei, pk in cases:
        with ch.Solver(nx, nk, -L, L, lk, nuclei=nuclei, precision=prec) as s:
            f = torch.empty((nx,) * 3 + (nk,) * 3, device="cuda", dtype=dt)
            s.init_gaussians(f, [pk])
            m_ref, e_ref = s.moments(f)
            rc, m, e = _noalloc(ch, f, nx, nk, L, lk, nuclei, prec)
            fh = f.double().cpu().numpy()
        assert rc == 0, ch.chasm.lib().chasm_last_error(None)
        assert m == pytest.approx(m_ref, rel=1e-12)
        assert e == pytest.approx(e_ref, rel=1e-12)
        # and the definitions themselves (the FP64 oracle on the same stored values)
        prob = O.Problem(nx=(nx,) * 3, nk=nk, x_lo=(-L,) * 3, x_hi=(L,) * 3, lk=lk, nuclei=nuclei)
        assert m == pytest.approx(O.mass(fh, prob), rel=1e-12)
        assert e == pytest.approx(O.energy(fh, prob), rel=1e-12)


def test_noalloc_at_the_largest_accepted_grid(ch):
    """64^3 x points fill the whole scratch array (its results sit right behind the last
    partial-sum triple): compared with chasm_moments twice in a row, FP32-mixed, N_k = 8."""
    nx, nk, L, lk = 64, 8, 8.0, 3.0
    nuclei = [((0.21, -0.13, 0.05), 1.0)]
    with ch.Solver(nx, nk, -L, L, lk, nuclei=nuclei, precision=ch.FP32_MIXED) as s:
        f = torch.empty((nx,) * 3 + (nk,) * 3, device="cuda", dtype=torch.float32)
        for pk in (synth.packet((1.0, -0.5, 0.0), (0.2, 0.0, -0.3)),
                   synth.packet((-2.0, 0.5, 1.0), (0.0, 0.4, 0.1))):
            s.init_gaussians(f, [pk])
            m_ref, e_ref = s.moments(f)
            rc, m, e = _noalloc(ch, f, nx, nk, L, lk, nuclei, ch.FP32_MIXED)
            assert rc == 0, ch.chasm.lib().chasm_last_error(None)
            assert m == pytest.approx(m_ref, rel=1e-12)
            assert e == pytest.approx(e_ref, rel=1e-12)
        del f


def test_noalloc_refuses_grids_beyond_its_scratch(ch):
    lib = ch.chasm.lib()
    f = torch.zeros(8, device="cuda")
    rc, _, _ = _noalloc(ch, f, 65, 8, 5.0, 4.0, [((0.0, 0.0, 0.0), 1.0)], ch.FP32_MIXED)
    assert rc == ch.chasm.EINVAL
    assert b"x points" in lib.chasm_last_error(None)
    # one x point above the limit: 5 x 13 x 4033 = 262145
    g = ch.chasm.make_grid(5, 8)
    g.nx[1], g.nx[2] = 13, 4033
    b = ch.chasm.make_box(-5.0, 5.0, 4.0)
    nuc = (ch.chasm.Nucleus * 1)(ch.chasm.Nucleus((C.c_double * 3)(0, 0, 0), 1.0))
    pot = ch.chasm.Potential(nuc, 1, 0.0, (C.c_double * 3)(0, 0, 0))
    m = C.c_double()
    rc = lib.chasm_moments_noalloc(f.data_ptr(), C.byref(g), C.byref(b), C.byref(pot), 1.0, 1.0,
                                   ch.FP32_MIXED, None, C.byref(m), None)
    assert rc == ch.chasm.EINVAL
    assert b"262145" in lib.chasm_last_error(None)
    # the checks of chasm_create apply as well (a non-finite nucleus)
    nuc[0].charge = float("inf")
    g2 = ch.chasm.make_grid(8, 8)
    rc = lib.chasm_moments_noalloc(f.data_ptr(), C.byref(g2), C.byref(b), C.byref(pot), 1.0, 1.0,
                                   ch.FP32_MIXED, None, C.byref(m), None)
    assert rc == ch.chasm.EINVAL
