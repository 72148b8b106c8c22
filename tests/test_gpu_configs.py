"""The remaining workload configurations at their full sizes, through the C ABI:
64 maps at Nside 512 (two 32-map column tiles of the tensor-core kernel), an
uneven batch of 200 maps with Nside drawn from {64, ..., 1024} replayed as one
CUDA graph, and 8 maps at Nside 2048 (the run-time Givens sweeps): against the
oracle on a sample of orders, through a full-size dot test of the adjoint and
the gradient of a C_l loss, and through properties that hold at any size."""

import numpy as np
import pytest

import skies
from helpers import per_l_error, per_l_norms, ring_perm, sampled_per_l_error
from oracle import dense, geometry, hp2sph
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
        perm = ring_perm(ns, quarter)
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


@pytest.mark.slow
def test_nside2048_workload_oracle_adjoint_gradient(hp):
    """The differentiation workload: 8 FP32 maps at Nside 2048, lmax 4096 (the plan
    runs the Givens sweeps per call).  Maps 0 and 7 are the workload's seeded
    power-law skies; maps 1-6 are quarter turns and north-south mirrors of them
    (the same spectra, without synthesising six more 50M-pixel skies).
    (1) Maps 0 and 7 against the oracle on 12 orders spread over 0..L plus the
        edge orders 0, 1, 2, L-1, L (per-degree estimate and element checks).
    (2) Full-size dot test <A f, a> = <f, A^T a> of hpx_synthesize.
    (3) One backward() of the loss sum_l w_l (C_l - C*_l)^2 (w_l = 1/l, l >= 2,
        C*_l a seeded power law): its directional derivative along a random map d
        equals the one computed from the forward analysis of d."""
    ns, L, B = 2048, 4096, 8
    m0, a0 = skies.workload_maps("w5_nside2048x8", nmaps=1, first=0, dtype=np.float32, return_alm=True)
    m7, a7 = skies.workload_maps("w5_nside2048x8", nmaps=1, first=7, dtype=np.float32, return_alm=True)
    q, mir = ring_perm(ns, True), ring_perm(ns, False)
    maps = np.stack([m0[0], m0[0][q], m0[0][mir], m0[0][q][q], m7[0][q], m7[0][mir], m7[0][q][mir], m7[0]])
    plan = hp.Plan(ns, L, B, "fp32")
    assert plan.flags & hp.HPX_FLAG_SWEEPS
    x = torch.as_tensor(maps, device="cuda")
    a = plan.analyze(x)
    plan.sync()
    a_np = a.cpu().numpy().astype(np.complex128)

    # (1) oracle on sampled orders
    strat = [int((k + 0.5) * (L + 1) / 12) for k in range(12)]
    low = [0, 1, 2, L - 1, L]
    ref = hp2sph.analyze_columns(np.stack([m0[0], m7[0]]).astype(np.float64), ns, L, strat + low)
    for k, (b, alms) in enumerate(((0, a0[0]), (7, a7[0]))):
        got = {m: a_np[b][hp2sph.alm_index(m, m, L):hp2sph.alm_index(m, m, L) + L - m + 1] for m in strat + low}
        norms = per_l_norms(alms, L)
        err = sampled_per_l_error({m: got[m] for m in strat}, {m: ref[m][k] for m in strat}, norms, L)
        assert err < TOL, (b, err)
        for m in low:
            l = np.arange(max(m, 2), L + 1)
            d = np.abs(got[m][l - m] - ref[m][k][l - m]) / norms[l]
            assert d.max() < TOL, (b, m, d.max())

    # (2) full-size dot test of the adjoint
    rng = np.random.default_rng(2049)
    coef = (rng.standard_normal((B, plan.nalm)) + 1j * rng.standard_normal((B, plan.nalm))).astype(np.complex64)
    Ata = plan.synthesize(torch.as_tensor(coef, device="cuda")).cpu().numpy().astype(np.float64)
    plan.sync()
    for b in (0, 7):
        lhs = dense.alm_dot(a_np[b], coef[b].astype(np.complex128), L)
        rhs = float(np.dot(maps[b].astype(np.float64), Ata[b]))
        assert abs(lhs - rhs) <= 2e-5 * np.linalg.norm(maps[b]) * np.linalg.norm(Ata[b]), (b, lhs, rhs)

    # (3) gradient of a C_l loss through autograd (hpx_cl_vjp, hpx_analyze_vjp)
    w = np.zeros(L + 1)
    w[2:] = 1.0 / np.arange(2, L + 1)
    cstar = skies.power_law(L, 2.0) * rng.uniform(0.5, 1.5, L + 1)
    wl, cs = torch.as_tensor(w, device="cuda"), torch.as_tensor(cstar, device="cuda")
    xg = x.clone().requires_grad_(True)
    c = hp.cl(hp.analyze(xg, plan), plan)
    loss = torch.sum(wl * (c - cs) ** 2)
    loss.backward()
    g = xg.grad.detach().double()
    d = torch.as_tensor(rng.standard_normal(maps.shape).astype(np.float32), device="cuda")
    ad = plan.analyze(d).cpu().numpy().astype(np.complex128)
    cl_np = c.detach().cpu().numpy()
    m_idx = np.concatenate([np.full(L - mm + 1, mm) for mm in range(L + 1)])
    l_idx = np.concatenate([np.arange(mm, L + 1) for mm in range(L + 1)])
    wm = np.where(m_idx == 0, 1.0, 2.0)
    expect, size = 0.0, 0.0
    for b in range(B):
        dcl = np.bincount(l_idx, weights=wm * 2.0 * np.real(np.conj(a_np[b]) * ad[b]), minlength=L + 1)
        dcl /= 2.0 * np.arange(L + 1) + 1.0
        terms = 2.0 * w * (cl_np[b] - cstar) * dcl
        expect += float(np.sum(terms))
        size += float(np.sum(np.abs(terms)))
    got = float(torch.sum(g * d.double()).item())
    # FP32 products: the tolerance is relative to the sum of the terms' magnitudes
    assert abs(got - expect) <= 1e-4 * size, (got, expect, size)
