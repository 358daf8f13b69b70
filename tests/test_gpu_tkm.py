"""chasm_tkm_convolve: the truncated-kernel convolution phi = T * g of Sec. 4 on the GPU (the
table-form kernels with the real spectrum of T), against the oracle's tkm_convolve on seeded data
and against the Dawson closed form of Example 4.1 (Phi = |k|^-2 * exp(-|k|^2) =
2 pi^{3/2} F(k)/k), for N_k = 8, 16, 32 in both forms."""
import math

import numpy as np
import pytest
from scipy.special import dawsn

import synth
from oracle import chasm_oracle as O

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available()
    return pkg


def _solver(ch, nx, nk, lk, name):
    return ch.Solver(nx, nk, (-2.0, -1.5, -2.5), (2.5, 1.0, 2.0), lk,
                     nuclei=[((0.3, -0.2, 0.1), 1.0)], theta_form=ch.THETA_TABLE,
                     precision=ch.FP64 if name == "fp64" else ch.FP32_MIXED)


def _dtype(name):
    return torch.float64 if name == "fp64" else torch.float32


@pytest.mark.parametrize("name", ["fp64", "fp32"])
@pytest.mark.parametrize("nk,nx", [(8, (5, 4, 6)), (16, (4, 5, 4)), (32, (4, 4, 5))])
def test_tkm_convolve_matches_the_oracle(ch, name, nk, nx):
    lk = 4.0
    rng = np.random.default_rng(nk)
    pk = [synth.packet(rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)) for _ in range(2)]
    g = synth.gaussian_packets(nx, nk, (-2.0, -1.5, -2.5), (2.5, 1.0, 2.0), lk, pk)
    g = g + 1e-3 * rng.standard_normal(g.shape) * g.max()
    with _solver(ch, nx, nk, lk, name) as s:
        gd = torch.from_numpy(g).to("cuda", _dtype(name))
        out = torch.empty_like(gd)
        s.tkm_convolve(gd, out)
        s.tkm_convolve(gd, out)   # a second call reuses the table
        s.sync()
        got = out.double().cpu().numpy()
        src = gd.double().cpu().numpy()
    ref = O.tkm_convolve(src.astype(complex), O.tkm_tensor(nk, lk)).real
    assert O.rel_l2(got, ref) <= TOL[name], O.rel_l2(got, ref)


@pytest.mark.parametrize("name", ["fp64", "fp32"])
def test_tkm_convolve_dawson_example(ch, name):
    """Example 4.1 at every x point: the error against the closed form falls with N_k (spectral
    convergence of the TKM until the tail exp(-L_k^2))."""
    lk = 4.0
    errs = []
    for nk in (8, 16, 32):
        ks = O.k_nodes(nk, lk)
        K = np.sqrt(ks[:, None, None] ** 2 + ks[None, :, None] ** 2 + ks[None, None, :] ** 2)
        Kp = np.where(K > 0, K, 1.0)
        ex = np.where(K > 0, 2 * math.pi ** 1.5 * dawsn(Kp) / Kp, 2 * math.pi ** 1.5)
        with _solver(ch, 4, nk, lk, name) as s:
            gd = torch.from_numpy(np.exp(-K ** 2)).to("cuda", _dtype(name))
            gd = gd.expand((4, 4, 4) + gd.shape).contiguous()
            out = torch.empty_like(gd)
            s.tkm_convolve(gd, out)
            s.sync()
            got = out.double().cpu().numpy()
        assert np.max(np.abs(got - got[:1, :1, :1])) <= (1e-13 if name == "fp64" else 1e-6) * ex.max()
        errs.append(np.max(np.abs(got[0, 0, 0] - ex)) / ex.max())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[1] < 1e-5 and errs[2] < (1e-7 if name == "fp64" else 1e-5), errs
