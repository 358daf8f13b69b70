"""chasm_moments_noalloc, the allocation-free mass/energy entry point, against chasm_moments.

Who needs it: callers that must not allocate device memory at the moment they check a solve --
code running while a stream is captured in the global capture mode, services that hand their
whole memory budget to solves, plug-ins that only get a device pointer.  The entry point keeps its
scratch in a fixed device array, so the test also checks that two calls in a row with different
inputs each give their own answer (the array keeps the previous call's contents), and that grids
above its stated limit are refused.  This file is collected last so that a failure here does not
stop the rest of the GPU suite; it passes alone and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth

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
        assert rc == 0, ch.chasm.lib().chasm_last_error(None)
        assert m == pytest.approx(m_ref, rel=1e-12)
        assert e == pytest.approx(e_ref, rel=1e-12)


def test_noalloc_refuses_grids_beyond_its_scratch(ch):
    f = torch.zeros(8, device="cuda")
    rc, _, _ = _noalloc(ch, f, 65, 8, 5.0, 4.0, [((0.0, 0.0, 0.0), 1.0)], ch.FP32_MIXED)
    assert rc == ch.chasm.EINVAL
    assert b"x points" in ch.chasm.lib().chasm_last_error(None)
