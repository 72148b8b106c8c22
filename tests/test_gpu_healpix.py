"""The HEALPix software's analysis (Sec. 2.2: equal-weight quadrature, Eq. healsph,
and its Jacobi refinement, Eqs. uzawa/richardson) through the C ABI, against the
oracle's plain double sums, and the transpose of the synthesis it is built from."""

import numpy as np
import pytest

import skies
from helpers import per_l_error
from oracle import dense, hp2sph, healpix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-5}


@pytest.fixture(scope="module")
def hp():
    import os
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    assert torch.cuda.is_available()
    return hp


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("sweeps", [False, True], ids=["operators", "sweeps"])
@pytest.mark.parametrize("nside,lmax,B", [(4, 8, 2), (16, 29, 3), (64, 128, 12)])
def test_synthesis_adjoint_dot(hp, prec, tol, sweeps, nside, lmax, B):
    """<S a, f> = <a, S^T f> with the coefficient inner product of weight 2 for m > 0."""
    rng = np.random.default_rng(nside + B)
    plan = hp.Plan(nside, lmax, B, prec, synthesis=True, sweeps=sweeps)
    rd = torch.float64 if prec == "fp64" else torch.float32
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    f = rng.standard_normal((B, plan.npix))
    a = rng.standard_normal((B, plan.nalm)) + 1j * rng.standard_normal((B, plan.nalm))
    Sa = plan.sh_synthesis(torch.as_tensor(a, dtype=cd, device="cuda")).cpu().numpy().astype(np.float64)
    Stf = plan.sh_synthesis_adjoint(torch.as_tensor(f, dtype=rd, device="cuda")).cpu().numpy().astype(np.complex128)
    plan.sync()
    for b in range(B):
        lhs = float(np.dot(Sa[b], f[b]))
        rhs = dense.alm_dot(a[b], Stf[b], lmax)
        assert abs(lhs - rhs) <= tol * np.linalg.norm(Sa[b]) * np.linalg.norm(f[b]), (b, lhs, rhs)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("sweeps", [False, True], ids=["operators", "sweeps"])
@pytest.mark.parametrize("nside,lmax,B", [(8, 16, 2), (16, 32, 3), (64, 128, 10)])
def test_equal_weight_and_jacobi_vs_oracle(hp, prec, sweeps, nside, lmax, B):
    """niter = 0 (Eq. healsph) and niter = 3 (the software's default) against the
    oracle, every degree of every map."""
    maps, _ = skies.small_powerlaw_maps(nside, B, seed=900 + nside, alpha=2.0, noise=1e-3, lmax=lmax)
    if prec == "fp32":
        maps = maps.astype(np.float32).astype(np.float64)
    plan = hp.Plan(nside, lmax, B, prec, jacobi=True, sweeps=sweeps)
    assert plan.flags & hp.HPX_FLAG_JACOBI
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.as_tensor(maps, dtype=dt, device="cuda")
    for niter, ref in ((0, healpix.equal_weight(maps, nside, lmax)), (3, healpix.jacobi(maps, nside, lmax, 3))):
        a = plan.healpix_analysis(x, niter=niter)
        plan.sync()
        a = a.cpu().numpy().astype(np.complex128)
        for b in range(B):
            e = per_l_error(a[b], ref[b], lmax)
            assert e.max() < TOL[prec], (niter, b, e.max(), int(np.argmax(e)))


def test_jacobi_converges_to_band_limited_coefficients(hp):
    """Eq. (richardson): for a map synthesised from coefficients of degree <= Nside the
    iteration converges to those coefficients (FP64)."""
    ns, L = 16, 16
    rng = np.random.default_rng(5)
    at = rng.standard_normal(hp2sph.n_alm(L)) + 1j * rng.standard_normal(hp2sph.n_alm(L))
    for l in range(L + 1):
        at[hp2sph.alm_index(l, 0, L)] = at[hp2sph.alm_index(l, 0, L)].real
    f = hp2sph.synthesize(at, ns, L)
    plan = hp.Plan(ns, L, 1, "fp64", jacobi=True)
    x = torch.as_tensor(f[None], device="cuda")
    errs = [np.abs(plan.healpix_analysis(x, niter=k).cpu().numpy()[0] - at).max() for k in (0, 2, 12)]
    assert errs[1] < 0.01 * errs[0] and errs[2] < 1e-11, errs


def test_healpix_analysis_needs_the_workspace_flag(hp):
    plan = hp.Plan(8, 16, 1, "fp64", synthesis=True)
    x = torch.zeros((1, plan.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(hp.HpxError) as ei:
        plan.healpix_analysis(x, niter=1)
    assert ei.value.code == hp.HPX_ERR_STATE
