"""Spherical-harmonic synthesis (hpx_sh_synthesis) through the C ABI against the
oracle's plain sum of a_lm Y_lm at the pixel centres."""

import numpy as np
import pytest

from oracle import hp2sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# max |f_gpu - f_oracle| / max |f_oracle|
TOL = {"fp64": 1e-11, "fp32": 1e-5}


@pytest.fixture(scope="module")
def hp():
    import os
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    assert torch.cuda.is_available()
    return hp


def _random_alm(L, B, seed, alpha=1.0):
    rng = np.random.default_rng(seed)
    n = hp2sph.n_alm(L)
    a = rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n))
    for m in range(L + 1):
        i0 = hp2sph.alm_index(m, m, L)
        l = np.arange(m, L + 1)
        a[:, i0:i0 + L - m + 1] *= (1.0 + l) ** -alpha
    return a


@pytest.mark.parametrize("sweeps", [False, True], ids=["operators", "sweeps"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nside,lmax,B", [(2, 4, 2), (4, 8, 3), (8, 16, 2), (8, 11, 2), (16, 32, 3), (64, 128, 2),
                                          (128, 256, 17), (32, 57, 33)])
def test_synthesis_matches_oracle(hp, prec, nside, lmax, B, sweeps):
    """operators: per-order synthesis operators R_{m,c} Es built at plan time
    (FP32 plans of more than 8 maps: on the tensor cores; 33 maps span two
    32-map column tiles); sweeps: transposed sweeps and the Legendre-to-Fourier
    table per call."""
    a = _random_alm(lmax, B, seed=nside + lmax)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    a = a.astype(cdt)
    plan = hp.Plan(nside, lmax, B, prec, synthesis=True, sweeps=sweeps)
    f = plan.sh_synthesis(torch.as_tensor(a, device="cuda"))
    plan.sync()
    ref = hp2sph.synthesize(a.astype(np.complex128), nside, lmax)
    err = np.max(np.abs(f.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < TOL[prec], err


def test_synthesis_needs_the_flag(hp):
    plan = hp.Plan(8, -1, 1, "fp32")
    a = torch.zeros((1, plan.nalm), dtype=torch.complex64, device="cuda")
    with pytest.raises(hp.HpxError):
        plan.sh_synthesis(a)


def test_synthesis_uneven_batch(hp):
    nsides = [8, 16, 8]
    plan = hp.Plan(nsides=nsides, precision="fp64", synthesis=True)
    parts, refs = [], []
    for k, ns in enumerate(nsides):
        a = _random_alm(2 * ns, 1, seed=900 + k)[0]
        parts.append(a)
        refs.append(hp2sph.synthesize(a, ns, 2 * ns))
    f = plan.sh_synthesis(torch.as_tensor(np.concatenate(parts), device="cuda")).cpu().numpy()
    ref = np.concatenate(refs)
    assert np.max(np.abs(f - ref)) / np.max(np.abs(ref)) < TOL["fp64"]


def test_analysis_of_synthesis_on_exact_subspace(hp):
    """hpx_analyze inverts hpx_sh_synthesis on span{Y_0^0, Y_2^0, Y_l^{+-1}}."""
    ns, L = 32, 64
    rng = np.random.default_rng(3)
    a = np.zeros((1, hp2sph.n_alm(L)), dtype=np.complex128)
    a[0, hp2sph.alm_index(0, 0, L)] = 1.1
    a[0, hp2sph.alm_index(2, 0, L)] = 0.4
    for l in range(1, L + 1):
        a[0, hp2sph.alm_index(l, 1, L)] = rng.standard_normal() + 1j * rng.standard_normal()
    plan = hp.Plan(ns, L, 1, "fp64", synthesis=True)
    f = plan.sh_synthesis(torch.as_tensor(a, device="cuda"))
    back = plan.analyze(f)
    plan.sync()
    np.testing.assert_allclose(back.cpu().numpy(), a, atol=1e-10)
