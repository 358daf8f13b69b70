"""CPU-only checks of the C ABI: the library loads, exports every function that include/chasm.h
declares, and validates arguments on the host without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chasm.h")


@pytest.fixture(scope="module")
def ch():
    from paper_2205_02380_gb300 import build
    build.build()
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    return pkg.chasm


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chasm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("chasm_create", "chasm_step", "chasm_mass", "chasm_energy", "chasm_submit",
                     "chasm_poll", "chasm_destroy", "chasm_workspace_bytes"):
        assert required in names


def test_library_exports_every_declared_symbol(ch):
    L = ch.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    bound = {n for n, _, _ in ch._SIGS}
    assert set(declared_functions()) == bound


def test_struct_layouts_match_the_header(ch):
    assert C.sizeof(ch.Grid) == 24
    assert C.sizeof(ch.Box) == 72
    assert C.sizeof(ch.Nucleus) == 32
    assert C.sizeof(ch.Gaussian) == 72
    assert C.sizeof(ch.Options) == 40


def test_options_default(ch):
    o = ch.Options()
    assert ch.lib().chasm_options_default(C.byref(o)) == 0
    assert (o.precision, o.n_nb, list(o.patches), o.use_graphs) == (ch.FP32_MIXED, 20, [1, 1, 1], 1)
    assert o.theta_form == ch.THETA_AUTO and o.integrator == ch.STRANG
    assert ch.lib().chasm_options_default(None) == ch.EINVAL


def _create(ch, nx=(8, 8, 8), nk=16, lo=-4.0, hi=4.0, lk=4.0, nuclei=(), hbar=1.0, m=1.0,
            precision=0, n_nb=20, patches=(1, 1, 1), theta_form=0, integrator=0):
    L = ch.lib()
    g = ch.make_grid(list(nx), nk) if not isinstance(nk, tuple) else ch.Grid(
        (C.c_int32 * 3)(*nx), (C.c_int32 * 3)(*nk))
    b = ch.make_box(lo, hi, lk)
    nuc = (ch.Nucleus * max(1, len(nuclei)))(*[ch.Nucleus((C.c_double * 3)(*p), z) for p, z in nuclei])
    pot = ch.Potential(nuc if nuclei else None, len(nuclei), 0.0, (C.c_double * 3)(0, 0, 0))
    o = ch.Options()
    L.chasm_options_default(C.byref(o))
    o.precision = precision
    o.n_nb = n_nb
    o.patches = (C.c_int32 * 3)(*patches)
    o.theta_form = theta_form
    o.integrator = integrator
    h = C.c_void_p()
    rc = L.chasm_create(C.byref(g), C.byref(b), C.byref(pot), hbar, m, C.byref(o), C.byref(h))
    return rc, L.chasm_last_error(None).decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(nk=12), "nk"),
    (dict(nk=(16, 16, 8)), "nk"),
    (dict(nx=(3, 8, 8)), "nx"),
    (dict(lo=4.0, hi=-4.0), "x_hi"),
    (dict(lk=0.0), "k_half"),
    (dict(hbar=0.0), "hbar"),
    (dict(m=-1.0), "m must"),
    (dict(precision=7), "precision"),
    (dict(n_nb=0), "n_nb"),
    (dict(patches=(2, 1, 1), nx=(8, 8, 8)), "divide"),
    (dict(patches=(7, 1, 1), nx=(8, 8, 8)), "patches"),
    (dict(patches=(1, 4, 1), nx=(8, 5, 8)), "intervals per patch"),
    (dict(nuclei=[((float("nan"), 0, 0), 1.0)]), "nucleus"),
    (dict(theta_form=3), "theta_form"),
    (dict(integrator=2), "integrator"),
])
def test_create_rejects_invalid_arguments_on_the_host(ch, kw, needle):
    rc, msg = _create(ch, **kw)
    assert rc == ch.EINVAL
    assert needle in msg


def test_workspace_bytes(ch):
    L = ch.lib()
    g = ch.make_grid([16, 16, 16], 16)
    pot = ch.Potential(None, 0, 0.5, (C.c_double * 3)(0, 0, 0))
    w32 = L.chasm_workspace_bytes(C.byref(g), C.byref(pot), None)
    assert 0 < w32 < 16 ** 6 * 4 // 10        # the harmonic form needs only small tables
    bad = ch.make_grid([16, 16, 16], 12)
    assert L.chasm_workspace_bytes(C.byref(bad), C.byref(pot), None) == 0


def test_workspace_bytes_of_the_two_theta_forms(ch):
    """Coulomb workspace: the table form holds 4 N_k^3 values per x point (four copies of f) and
    no Horner buffers; the modulated form two Horner buffers; AUTO picks the table when it needs
    at most half of the device's memory (64 GiB when no device can be queried, as here)."""
    nuc = [((0.0, 0.0, 0.0), 1.0)]
    f = 16 ** 6 * 4
    w_tab = ch.workspace_bytes(16, 16, nuclei=nuc, theta_form=ch.THETA_TABLE)
    w_mod = ch.workspace_bytes(16, 16, nuclei=nuc, theta_form=ch.THETA_MODULATED)
    w_auto = ch.workspace_bytes(16, 16, nuclei=nuc)
    assert 4 * f <= w_tab < 5 * f
    assert 2 * f <= w_mod < 4 * f
    assert w_auto == w_tab
    # 128^3 x 32^3 FP32: a 1.1 TB table is above the AUTO limit on any device
    big_tab = ch.workspace_bytes(128, 32, nuclei=nuc, theta_form=ch.THETA_TABLE)
    assert big_tab >= 4 * 128 ** 3 * 32 ** 3 * 4
    assert ch.workspace_bytes(128, 32, nuclei=nuc) < big_tab
    # LPC1 adds one work copy of f to the table form (Theta f; the predictor is formed inside the
    # Theta kernel) and two to the quadratic potential
    assert ch.workspace_bytes(16, 16, nuclei=nuc, theta_form=ch.THETA_TABLE,
                              integrator=ch.LPC1) == w_tab + f
    assert ch.workspace_bytes(16, 16, nuclei=nuc, theta_form=ch.THETA_MODULATED,
                              integrator=ch.LPC1) == w_mod
    w_h = ch.workspace_bytes(16, 16, kappa=1.0)
    assert ch.workspace_bytes(16, 16, kappa=1.0, integrator=ch.LPC1) == w_h + 2 * f


def test_null_handles_are_rejected(ch):
    L = ch.lib()
    assert L.chasm_step(None, None, 0.1, 1) == ch.EINVAL
    assert L.chasm_sync(None) == ch.EINVAL
    assert L.chasm_destroy(None) == ch.OK
    m = C.c_double()
    assert L.chasm_mass(None, None, C.byref(m)) == ch.EINVAL


def test_server_validates_on_the_host(ch):
    L = ch.lib()
    s = C.c_void_p()
    assert L.chasm_server_create(0, 4, 1, 8, C.byref(s)) == ch.EINVAL
    assert L.chasm_server_create(1 << 30, 0, 1, 8, C.byref(s)) == ch.EINVAL
    assert L.chasm_server_create(1 << 20, 2, 1, 8, C.byref(s)) == ch.OK
    try:
        pk = [dict(w=1.0, x0=(0, 0, 0), k0=(0, 0, 0), ax=0.5, ak=2.0)]
        t = C.c_uint64()
        bad = ch.make_request(16, 16, -4, 4, 4.0, dt=-0.1, nsteps=3, kappa=1.0, packets=pk)
        assert L.chasm_submit(s, C.byref(bad), C.byref(t)) == ch.EINVAL
        nopk = ch.make_request(16, 16, -4, 4, 4.0, dt=0.1, nsteps=3, kappa=1.0, packets=[])
        assert L.chasm_submit(s, C.byref(nopk), C.byref(t)) == ch.EINVAL
        huge = ch.make_request(64, 32, -4, 4, 4.0, dt=0.1, nsteps=3, kappa=1.0, packets=pk)
        assert L.chasm_submit(s, C.byref(huge), C.byref(t)) == ch.EBUSY   # 1 MiB budget
        r = ch.Result()
        assert L.chasm_poll(s, 12345, C.byref(r)) == ch.ENOTFOUND
    finally:
        assert L.chasm_server_destroy(s) == ch.OK
