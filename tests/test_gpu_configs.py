"""The remaining workload configurations at their full sizes, through the C ABI:
64 maps at Nside 512 (two 32-map column tiles of the tensor-core kernel), an
uneven batch of 200 maps with Nside drawn from {64, ..., 1024} replayed as one
CUDA graph, and 8 maps at Nside 2048 (checked through properties that hold at
any size, since the oracle's dense least squares at that size takes too long)."""

import numpy as np
import pytest

import skies
from helpers import per_l_error, per_l_norms, sampled_per_l_error
from oracle import geometry, hp2sph
from oracle.legendre import pbar_table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5   # FP32 per-degree relative error


@pytest.fixture(scope="module")
def hp():
    import os
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    assert torch.cuda.is_available()
    return hp


def _sampled_check(a, maps_b, alm_b, ns, L, norms=None):
    strat = [int((k + 0.5) * (L + 1) / 8) for k in range(8)]
    low = [0, 1, L]
    ref = hp2sph.analyze_columns(maps_b.astype(np.float64), ns, L, strat + low)
    got = {m: a[hp2sph.alm_index(m, m, L):hp2sph.alm_index(m, m, L) + L - m + 1] for m in strat + low}
    norms = per_l_norms(alm_b, L) if norms is None else norms
    err = sampled_per_l_error({m: got[m] for m in strat}, {m: ref[m][0] for m in strat}, norms, L)
    assert err < TOL, err
    for m in low:
        l = np.arange(max(m, 2), L + 1)
        d = np.abs(got[m][l - m] - ref[m][0][l - m]) / norms[l]
        assert d.max() < TOL, (m, d.max())


@pytest.mark.slow
def test_nside512_64_maps(hp):
    """64 FP32 maps at Nside 512, lmax 1024, power-law skies with noise; maps 0,
    31, 32 and 63 (both column tiles, both edges) on a sample of orders."""
    maps, alms = skies.workload_maps("w3_nside512x64", dtype=np.float32, return_alm=True)
    plan = hp.Plan(512, 1024, 64, "fp32")
    x = torch.as_tensor(maps, device="cuda")
    a = plan.analyze(x)
    cl = plan.cl(a)
    plan.sync()
    a = a.cpu().numpy().astype(np.complex128)
    for b in (0, 31, 32, 63):
        _sampled_check(a[b], maps[b], alms[b], 512, 1024)
    assert np.all(np.isfinite(cl.cpu().numpy()))


@pytest.mark.slow
def test_uneven_200_maps_graph(hp):
    """200 maps with Nside drawn from {64, 128, 256, 512, 1024} (probabilities
    .40/.30/.15/.10/.05), lmax = 2 Nside, one plan replayed as a CUDA graph; the
    first map of every Nside against the oracle (full below 512, sampled above)."""
    nsides = [int(v) for v in skies.uneven_nsides(200)]
    maps, alms = [], []
    for k, ns in enumerate(nsides):
        mp, al = skies.small_powerlaw_maps(ns, 1, seed=7000 + k, alpha=2.0, noise=1e-3)
        maps.append(mp[0].astype(np.float32))
        alms.append(al[0])
    plan = hp.Plan(nsides=nsides, precision="fp32", graph=True)
    x = torch.as_tensor(np.concatenate(maps), device="cuda")
    for _ in range(2):
        a = plan.analyze(x)
        plan.sync()
    a = a.cpu().numpy().astype(np.complex128)
    offs = np.cumsum([0] + [hp2sph.n_alm(2 * ns) for ns in nsides])
    seen = set()
    for k, ns in enumerate(nsides):
        if ns in seen:
            continue
        seen.add(ns)
        L = 2 * ns
        ak = a[offs[k]:offs[k + 1]]
        if ns <= 256:
            ref = hp2sph.analyze(maps[k].astype(np.float64), ns, L)
            assert per_l_error(ak, ref, L).max() < TOL, ns
        else:
            _sampled_check(ak, maps[k], alms[k], ns, L)
    assert seen == {64, 128, 256, 512, 1024}


def _ring_perm(nside, quarter):
    """Pixel permutation of a quarter turn (lambda -> lambda + pi/2: every ring
    shifts by nphi/4 pixels) or of the north-south mirror."""
    rings = geometry.ring_table(nside)
    perm = np.empty(geometry.npix(nside), dtype=np.int64)
    R = len(rings)
    for i, r in enumerate(rings):
        k = np.arange(r["nphi"])
        if quarter:
            perm[r["start"] + k] = r["start"] + (k + r["nphi"] // 4) % r["nphi"]
        else:
            perm[r["start"] + k] = rings[R - 1 - i]["start"] + k
    return perm


@pytest.mark.slow
def test_nside2048_properties(hp):
    """8 FP32 maps at Nside 2048, lmax 4096 (the plan takes the sweeps: the
    operators would need 69 GB): (1) white-noise maps turned by a quarter turn
    give a_lm e^{i m pi/2}, mirrored north-south give (-1)^{l+m} a_lm;
    (2) a map in span{Y_0^0, Y_2^0, Y_l^{+-1}} is analysed exactly."""
    ns, L, B = 2048, 4096, 8
    npix = geometry.npix(ns)
    rng = np.random.default_rng(2048)
    f = rng.standard_normal((B, npix)).astype(np.float32)
    plan = hp.Plan(ns, L, B, "fp32")
    assert plan.flags & hp.HPX_FLAG_SWEEPS
    a0 = plan.analyze(torch.as_tensor(f, device="cuda")).cpu().numpy().astype(np.complex128)
    m = np.concatenate([np.full(L - mm + 1, mm) for mm in range(L + 1)])
    l = np.concatenate([np.arange(mm, L + 1) for mm in range(L + 1)])
    scale = np.sqrt(np.mean(np.abs(a0[:2]) ** 2))
    for quarter, factor in ((True, np.exp(0.5j * np.pi * m)), (False, (-1.0) ** (l + m))):
        perm = _ring_perm(ns, quarter)
        g = f[:2][:, perm]
        a1 = plan.analyze(torch.as_tensor(np.ascontiguousarray(np.concatenate([g, f[2:]])), device="cuda"))
        a1 = a1.cpu().numpy().astype(np.complex128)[:2]
        assert np.max(np.abs(a1 - a0[:2] * factor)) < 1e-4 * scale, quarter
    # exact subspace: F_0 from Y_0^0 and Y_2^0, F_1 from Y_l^1 (l = 1..L)
    coef = np.zeros(hp2sph.n_alm(L), dtype=np.complex128)
    coef[hp2sph.alm_index(0, 0, L)] = 1.0
    coef[hp2sph.alm_index(2, 0, L)] = -0.5
    # unit-variance coefficients at every degree: with a steep spectrum the
    # high degrees would sit below the FP32 rounding of the low-degree signal
    c1 = (rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(2.0)
    coef[hp2sph.alm_index(1, 1, L):hp2sph.alm_index(1, 1, L) + L] = c1
    rings = geometry.ring_table(ns)
    th = np.array([r["theta"] for r in rings])
    p0 = pbar_table(0, 2, np.cos(th), np.sin(th))
    p1 = pbar_table(1, L, np.cos(th), np.sin(th))
    F0 = (coef[0] * p0[0] - 0.5 * p0[2]) / np.sqrt(2 * np.pi)
    F1 = (c1 @ p1) / np.sqrt(2 * np.pi)
    fm = np.zeros(npix)
    for i, r in enumerate(rings):
        phi = r["phi0"] + 2 * np.pi * np.arange(r["nphi"]) / r["nphi"]
        fm[r["start"]:r["start"] + r["nphi"]] = F0[i].real + 2 * (F1[i] * np.exp(1j * phi)).real
    batch = np.concatenate([fm[None].astype(np.float32), f[1:]])
    a2 = plan.analyze(torch.as_tensor(batch, device="cuda")).cpu().numpy().astype(np.complex128)[0]
    e = per_l_error(a2, coef, L)
    assert e.max() < TOL, (e.max(), int(np.argmax(e)))
