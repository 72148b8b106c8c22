"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (per-degree relative l2 error e_l, see helpers.per_l_error):
FP64 plans 1e-11, FP32 plans 1e-5 -- the accuracy targets of the method's
FP64 and FP32 forms.  Inputs are seeded skies from `skies`."""

import numpy as np
import pytest

import skies
from helpers import per_l_error, per_l_norms, ring_perm, sampled_per_l_error, sampled_per_l_errors
from oracle import hp2sph

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


def _run(hp, maps, nside, lmax, prec, sweeps=False, simt=False):
    B = maps.shape[0]
    plan = hp.Plan(nside, lmax, B, prec, sweeps=sweeps, simt=simt)
    assert bool(plan.flags & hp.HPX_FLAG_SWEEPS) == sweeps
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.as_tensor(maps, dtype=dt, device="cuda")
    alm = plan.analyze(x)
    cl = plan.cl(alm)
    plan.sync()
    return alm.cpu().numpy().astype(np.complex128), cl.cpu().numpy(), plan


@pytest.mark.parametrize("path", ["fused", "sweeps", "simt"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nside,lmax,B", [(2, 4, 3), (4, 8, 3), (4, 5, 3), (8, 16, 3), (16, 32, 3), (16, 29, 17),
                                          (32, 64, 3), (64, 128, 33), (128, 256, 20), (64, 117, 6)])
def test_parity_full(hp, prec, nside, lmax, B, path):
    """fused: per-order operators (tensor cores for FP32 batches of 9+ maps);
    simt: the same on the FP32 pipes; sweeps: D and the Givens sweeps at run time
    (FP32 from 4 maps: D on the tensor cores and the staged sweep kernel)."""
    if path == "simt" and (prec == "fp64" or B <= 8):
        pytest.skip("the tensor-core variant only exists for FP32 batches of 9+ maps")
    maps, _ = skies.small_powerlaw_maps(nside, B, seed=100 + nside, alpha=2.0, noise=1e-3, lmax=2 * nside)
    if prec == "fp32":
        maps = maps.astype(np.float32).astype(np.float64)   # the oracle sees the same inputs
    a, cl, _ = _run(hp, maps, nside, lmax, prec, path == "sweeps", path == "simt")
    ref = hp2sph.analyze(maps, nside, lmax)
    for b in range(maps.shape[0]):
        e = per_l_error(a[b], ref[b], lmax)
        assert e.max() < TOL[prec], (b, e.max(), int(np.argmax(e)))
        clr = hp2sph.cl(ref[b], lmax)
        rel = np.abs(cl[b] - clr) / np.maximum(clr, 1e-300)
        assert rel[2:].max() < 2.5 * TOL[prec], rel.max()


def test_workload1_nside16_fp64(hp):
    maps = skies.workload_maps("w1_nside16")
    a, cl, _ = _run(hp, maps, 16, 32, "fp64")
    ref = hp2sph.analyze(maps, 16, 32)
    assert per_l_error(a[0], ref[0], 32).max() < TOL["fp64"]


def test_zero_and_constant_maps(hp):
    ns = 8
    z = np.zeros((2, 12 * ns * ns))
    z[1] = 3.5
    a, cl, _ = _run(hp, z, ns, 16, "fp64")
    assert np.all(a[0] == 0)
    ref = hp2sph.analyze(z[1], ns, 16)
    np.testing.assert_allclose(a[1], ref, atol=1e-12)
    assert abs(a[1][0] - 3.5 * np.sqrt(4 * np.pi)) < 1e-12


def test_batch_position_independent(hp):
    """A map gives bit-identical coefficients wherever it sits in a batch."""
    ns = 16
    maps, _ = skies.small_powerlaw_maps(ns, 5, seed=9)
    a5, _, _ = _run(hp, maps.astype(np.float32), ns, 32, "fp32")
    a1, _, _ = _run(hp, maps[3:4].astype(np.float32), ns, 32, "fp32")
    assert np.array_equal(a5[3], a1[0])


def test_lmax_zero(hp):
    ns = 4
    maps, _ = skies.small_powerlaw_maps(ns, 1, seed=2)
    a, cl, _ = _run(hp, maps, ns, 0, "fp64")
    ref = hp2sph.analyze(maps, ns, 0)
    np.testing.assert_allclose(a, ref, atol=1e-13)


_W2 = {}


def _w2_reference(prec):
    """Oracle coefficients (all orders) of the Nside-256 sky, computed once per
    input precision."""
    if prec not in _W2:
        maps, alms = skies.workload_maps("w2_nside256", return_alm=True)
        if prec == "fp32":
            maps = maps.astype(np.float32).astype(np.float64)
        _W2[prec] = (maps, hp2sph.analyze(maps, 256, 512))
    return _W2[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("sweeps", [False, True], ids=["fused", "sweeps"])
def test_workload2_nside256(hp, prec, sweeps):
    """Nside 256, lmax 512, FP64 and FP32 side by side; every degree."""
    maps, ref = _w2_reference(prec)
    a, cl, _ = _run(hp, maps, 256, 512, prec, sweeps)
    e = per_l_error(a[0], ref[0], 512)
    assert e.max() < TOL[prec], (e.max(), int(np.argmax(e)))
    clr = hp2sph.cl(ref[0], 512)
    assert (np.abs(cl[0] - clr) / clr)[2:].max() < 2.5 * TOL[prec]


@pytest.mark.slow
def test_bench_workload_sampled(hp):
    """The benchmark's workload (32 FP32 maps, Nside 1024, lmax 2048) in the
    launch configuration the benchmark times; the oracle checks maps 0 and 31
    on a sample of orders."""
    maps, alms = skies.workload_maps("bench_nside1024x32", dtype=np.float32, return_alm=True)
    a, _, _ = _run(hp, maps, 1024, 2048, "fp32")
    L = 2048
    strat = [int((k + 0.5) * (L + 1) / 12) for k in range(12)]     # uniform over orders
    low = [0, 1, 2, L - 1, L]
    for b in (0, 31):
        ref = hp2sph.analyze_columns(maps[b].astype(np.float64), 1024, L, strat + low)
        got = {m: a[b][hp2sph.alm_index(m, m, L):hp2sph.alm_index(m, m, L) + L - m + 1] for m in strat + low}
        norms = per_l_norms(alms[b], L)
        # e_l estimated from a uniform sample of orders
        err = sampled_per_l_error({m: got[m] for m in strat}, {m: ref[m][0] for m in strat}, norms, L)
        assert err < TOL["fp32"], (b, err)
        # single elements of the edge orders: |da_lm| <= tol ||a_l|| is necessary for e_l <= tol
        for m in low:
            l = np.arange(max(m, 2), L + 1)
            d = np.abs(got[m][l - m] - ref[m][0][l - m]) / norms[l]
            assert d.max() < TOL["fp32"], (b, m, d.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_uneven_batch(hp, prec, graph):
    """Maps of different nside in one plan (concatenated layout), gathered
    (interleaved nsides) and in place (adjacent runs), optionally replayed as
    one CUDA graph; every map against the oracle."""
    nsides = [8, 4, 16, 8, 32, 4, 4, 16]
    maps = []
    for k, ns in enumerate(nsides):
        mp, _ = skies.small_powerlaw_maps(ns, 1, seed=300 + k, alpha=2.0, noise=1e-3)
        maps.append(mp[0].astype(np.float32).astype(np.float64) if prec == "fp32" else mp[0])
    plan = hp.Plan(nsides=nsides, precision=prec, graph=graph)
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.as_tensor(np.concatenate(maps), dtype=dt, device="cuda")
    for rep in range(2):            # the second call replays the captured graph
        alm = plan.analyze(x)
        cl = plan.cl(alm)
        plan.sync()
    a = alm.cpu().numpy().astype(np.complex128)
    c = cl.cpu().numpy()
    oa = oc = 0
    for ns, mp in zip(nsides, maps):
        L = 2 * ns
        na = (L + 1) * (L + 2) // 2
        ref = hp2sph.analyze(mp, ns, L)
        assert per_l_error(a[oa:oa + na], ref, L).max() < TOL[prec]
        clr = hp2sph.cl(ref, L)
        assert (np.abs(c[oc:oc + L + 1] - clr) / clr)[2:].max() < 2.5 * TOL[prec]
        oa += na
        oc += L + 1
    assert oa == plan.nalm and oc == plan.ncl


def test_graph_uniform_plan_matches_eager(hp):
    ns = 32
    maps, _ = skies.small_powerlaw_maps(ns, 4, seed=41)
    x = torch.as_tensor(maps.astype(np.float32), device="cuda")
    eager = hp.Plan(ns, -1, 4, "fp32").analyze(x)
    gp = hp.Plan(ns, -1, 4, "fp32", graph=True)
    out1 = gp.analyze(x)
    out2 = torch.empty_like(out1)
    gp.analyze(x, out=out2)          # new output pointer: a second capture
    gp.analyze(x, out=out1)          # replay of the first graph
    torch.cuda.synchronize()
    assert torch.equal(eager, out1) and torch.equal(eager, out2)


@pytest.mark.parametrize("nside,B", [(128, 33), (256, 32)])
def test_operator_paths_deterministic(hp, nside, B):
    """Repeated analyses are bit-identical on the tensor-core path, and the
    tensor-core and FP32-pipe kernels agree to FP32 accuracy."""
    maps, _ = skies.small_powerlaw_maps(nside, B, seed=77, alpha=2.0, noise=1e-3)
    x = torch.as_tensor(maps.astype(np.float32), device="cuda")
    tc = hp.Plan(nside, -1, B, "fp32")
    a1 = tc.analyze(x)
    a2 = tc.analyze(x)
    tc.sync()
    assert torch.equal(a1, a2)
    a3 = hp.Plan(nside, -1, B, "fp32", simt=True).analyze(x)
    torch.cuda.synchronize()
    L = 2 * nside
    for b in (0, B - 1):
        e = per_l_error(a1[b].cpu().numpy().astype(np.complex128), a3[b].cpu().numpy().astype(np.complex128), L)
        assert e.max() < TOL["fp32"], (b, e.max())


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_cl_same_coefficients(hp, prec, tol):
    """hpx_cl on given coefficients against Eq. (APS) evaluated by the oracle
    (FP64, compensated) on the same coefficients: degrees 0..1024 of 3 maps,
    with a dynamic range of 1e6 between degrees."""
    ns, L, B = 512, 1024, 3
    plan = hp.Plan(ns, L, B, prec, sweeps=True)
    rng = np.random.default_rng(5)
    cdt = np.complex64 if prec == "fp32" else np.complex128
    a = np.zeros((B, plan.nalm), dtype=cdt)
    for b in range(B):
        for m in range(L + 1):
            i0 = hp2sph.alm_index(m, m, L)
            l = np.arange(m, L + 1)
            amp = (1.0 + l) ** -2.0
            v = amp * (rng.standard_normal(L - m + 1) + 1j * rng.standard_normal(L - m + 1))
            if m == 0:
                v = v.real
            a[b, i0:i0 + L - m + 1] = v
    got = plan.cl(torch.as_tensor(a, device="cuda")).cpu().numpy()
    for b in range(B):
        ref = hp2sph.cl(a[b].astype(np.complex128), L)
        assert np.max(np.abs(got[b] - ref) / ref) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_per_map_lmax(hp, prec, graph):
    """Per-map degrees (descriptor field lmaxs), with and without per-map nside:
    one sub-plan per (nside, lmax); every map against the oracle at its lmax."""
    cases = [([8, 16, 8, 16, 4], [5, -1, 16, 7, -1]), (None, [3, 32, -1, 3])]
    for nsides, lmaxs in cases:
        ns_list = nsides if nsides is not None else [16] * len(lmaxs)
        maps = []
        for k, ns in enumerate(ns_list):
            mp, _ = skies.small_powerlaw_maps(ns, 1, seed=500 + k, alpha=2.0, noise=1e-3)
            maps.append(mp[0].astype(np.float32).astype(np.float64) if prec == "fp32" else mp[0])
        plan = hp.Plan(16 if nsides is None else None, -1, precision=prec, graph=graph, nsides=nsides,
                       lmaxs=lmaxs)
        dt = torch.float64 if prec == "fp64" else torch.float32
        x = torch.as_tensor(np.concatenate(maps), dtype=dt, device="cuda")
        for _ in range(2):
            alm = plan.analyze(x)
            cl = plan.cl(alm)
            plan.sync()
        a = alm.cpu().numpy().astype(np.complex128)
        c = cl.cpu().numpy()
        oa = oc = 0
        for i, (ns, mp) in enumerate(zip(ns_list, maps)):
            L = plan.map_lmax(i)
            na = (L + 1) * (L + 2) // 2
            ref = hp2sph.analyze(mp, ns, L)
            assert per_l_error(a[oa:oa + na], ref, L).max() < TOL[prec], (nsides, lmaxs, i)
            clr = hp2sph.cl(ref, L)
            if L >= 2:
                assert (np.abs(c[oc:oc + L + 1] - clr) / clr)[2:].max() < 2.5 * TOL[prec]
            oa += na
            oc += L + 1
        assert oa == plan.nalm and oc == plan.ncl


@pytest.mark.parametrize("uneven", [False, True], ids=["uniform", "group"])
def test_checked_flag(hp, uneven):
    """HPX_FLAG_CHECKED: a NaN or an infinity in the input is reported by the next
    hpx_sync as HPX_ERR_NONFINITE (once); host pointers are refused before any
    launch; clean inputs analyse as without the flag."""
    ns = 16
    nsides = [16, 8] if uneven else None
    plan = hp.Plan(None if uneven else ns, -1, 2, "fp32", nsides=nsides, checked=True)
    ref_plan = hp.Plan(None if uneven else ns, -1, 2, "fp32", nsides=nsides)
    npix = plan.npix
    rng = np.random.default_rng(1)
    clean = rng.standard_normal(npix if uneven else (2, 12 * ns * ns)).astype(np.float32)
    x = torch.as_tensor(clean, device="cuda")
    a = plan.analyze(x)
    plan.sync()
    assert torch.equal(a, ref_plan.analyze(x))
    for bad in (np.nan, np.inf, -np.inf):
        y = x.clone()
        y.view(-1)[y.numel() // 3] = float(bad)
        plan.analyze(y)
        with pytest.raises(hp.HpxError) as ei:
            plan.sync()
        assert ei.value.code == hp.HPX_ERR_NONFINITE
        plan.sync()                      # reported once
    # adjoint input checked too
    g = torch.zeros_like(a)
    g.view(-1)[5] = complex(float("nan"), 0.0)
    plan.synthesize(g)
    with pytest.raises(hp.HpxError):
        plan.sync()
    # host memory is refused before anything is launched
    host_maps = np.zeros(x.numel(), dtype=np.float32)
    host_alm = np.zeros(2 * a.numel(), dtype=np.float32)
    rc = hp.lib().hpx_analyze(plan.handle, host_maps.ctypes.data, host_alm.ctypes.data)
    assert rc == hp.HPX_ERR_ARG
    rc = hp.lib().hpx_analyze(plan.handle, x.data_ptr(), host_alm.ctypes.data)
    assert rc == hp.HPX_ERR_ARG
    plan.sync()


@pytest.mark.parametrize("prec,nside,B", [("fp32", 32, 12), ("fp64", 16, 1)])
def test_autotune_keeps_a_correct_path(hp, prec, nside, B):
    """HPX_FLAG_AUTOTUNE picks the operators or the sweeps; either way the
    result matches the oracle."""
    maps, _ = skies.small_powerlaw_maps(nside, B, seed=61, alpha=2.0, noise=1e-3)
    if prec == "fp32":
        maps = maps.astype(np.float32).astype(np.float64)
    plan = hp.Plan(nside, -1, B, prec, autotune=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    a = plan.analyze(torch.as_tensor(maps, dtype=dt, device="cuda"))
    plan.sync()
    a = a.cpu().numpy().astype(np.complex128)
    ref = hp2sph.analyze(maps, nside, 2 * nside)
    for b in range(B):
        assert per_l_error(a[b], ref[b], 2 * nside).max() < TOL[prec]


def test_launch_shapes_give_identical_results(hp):
    """The ring-FFT and grid-FFT kernels with 16 or 32 elements per thread run the
    same radix passes in the same order, the three forms of the run-time sweeps
    (complex lanes with 32 or 16 stages per pass, real lanes) the same rotations
    on the same values, and both placements of the
    FP16-pair packing of b the same scalings and roundings, so every launch shape
    (and whatever HPX_FLAG_AUTOTUNE picks) gives bit-identical coefficients, on the
    run-time sweeps (FP32 pipes, 2 maps) and on the tensor-core D (4 maps); other
    values are refused."""
    ns = 1024
    rng = np.random.default_rng(71)
    for B in (2, 4):
        x = torch.as_tensor(rng.standard_normal((B, 12 * ns * ns)).astype(np.float32), device="cuda")
        plan = hp.Plan(ns, -1, B, "fp32", sweeps=True, autotune=True)
        t = plan.tuning
        assert t[0] in (16, 32) and t[1] in (16, 32) and t[2] in (0, 1, 2) and t[3] in (0, 1) and t[4] in (0, 1)
        tuned = plan.analyze(x).clone()
        outs = []
        rf = t[4]   # the ring form changes the roundings; the other choices must not
        for shapes in ((16, 16, 0, 0, rf), (32, 32, 1, 1, rf), (16, 32, 2, 0, rf), (32, 16, 2, 1, rf)):
            plan.tuning = shapes
            assert plan.tuning == shapes
            outs.append(plan.analyze(x).clone())
        torch.cuda.synchronize()
        for o in outs:
            assert torch.equal(o, tuned)
        for bad in ((8, 16, 0, 0, 0), (16, 64, 0, 0, 0), (16, 16, 3, 0, 0), (16, 16, 0, 2, 0), (16, 16, 0, 0, 2)):
            with pytest.raises(hp.HpxError):
                plan.tuning = bad
        plan.close()


def test_quarter_length_bluestein_rings(hp):
    """Ring form 1 (the Bluestein rings of 4096 points and more as four
    quarter-length Bluestein transforms and a radix-4 step) on maps 0 and 1 of
    the benchmark workload at Nside 1024: against the oracle on a sample of
    orders plus the edge orders (the parity gate), and per degree within half the
    gate of ring form 0 (both are FP32 evaluations of the same DFTs)."""
    ns, L = 1024, 2048
    maps, alms = skies.workload_maps("bench_nside1024x32", nmaps=2, dtype=np.float32, return_alm=True)
    x = torch.as_tensor(maps, device="cuda")
    plan = hp.Plan(ns, L, 2, "fp32")
    t = list(plan.tuning)
    res = {}
    for rf in (0, 1):
        t[4] = rf
        plan.tuning = tuple(t)
        res[rf] = plan.analyze(x).cpu().numpy().astype(np.complex128)
    plan.close()
    assert not np.array_equal(res[0], res[1])   # the other form did run
    strat = [int((k + 0.5) * (L + 1) / 6) for k in range(6)]
    low = [0, 1, 2, L]
    ref = hp2sph.analyze_columns(maps[0].astype(np.float64), ns, L, strat + low)
    norms = per_l_norms(alms[0], L)
    got = {m: res[1][0][hp2sph.alm_index(m, m, L):hp2sph.alm_index(m, m, L) + L - m + 1] for m in strat + low}
    err = sampled_per_l_error({m: got[m] for m in strat}, {m: ref[m][0] for m in strat}, norms, L)
    assert err < TOL["fp32"], err
    for m in low:
        l = np.arange(max(m, 2), L + 1)
        d = np.abs(got[m][l - m] - ref[m][0][l - m]) / norms[l]
        assert d.max() < TOL["fp32"], (m, d.max())
    for b in range(2):
        assert per_l_error(res[1][b], res[0][b], L)[2:].max() < 0.5 * TOL["fp32"]


def test_graph_tensor_core_path_matches_eager(hp):
    """The tensor-core path overlaps grid FFTs and operators on two streams; a
    graph capture of it replays to the same coefficients as eager calls."""
    ns, B = 64, 12
    maps, _ = skies.small_powerlaw_maps(ns, B, seed=44)
    x = torch.as_tensor(maps.astype(np.float32), device="cuda")
    eager = hp.Plan(ns, -1, B, "fp32").analyze(x)
    gp = hp.Plan(ns, -1, B, "fp32", graph=True)
    out = gp.analyze(x)
    out = gp.analyze(x, out=out)      # replay
    torch.cuda.synchronize()
    assert torch.equal(eager, out)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nside,lmax,B", [(4, 8, 2), (16, 32, 3), (16, 29, 2), (64, 128, 3), (256, 512, 2)])
def test_cg_latitude_solve(hp, prec, nside, lmax, B):
    """HPX_FLAG_CG: conjugate gradients on the normal equations of every column
    (the paper's form of the latitude solve) give the oracle's exact least-squares
    coefficients to the same tolerance as the premultiplied operators."""
    maps, _ = skies.small_powerlaw_maps(nside, B, seed=800 + nside, alpha=2.0, noise=1e-3)
    if prec == "fp32":
        maps = maps.astype(np.float32).astype(np.float64)
    plan = hp.Plan(nside, lmax, B, prec, cg=True)
    assert plan.flags & hp.HPX_FLAG_SWEEPS
    dt = torch.float64 if prec == "fp64" else torch.float32
    a = plan.analyze(torch.as_tensor(maps, dtype=dt, device="cuda"))
    plan.sync()
    a = a.cpu().numpy().astype(np.complex128)
    ref = hp2sph.analyze(maps, nside, lmax)
    for b in range(B):
        e = per_l_error(a[b], ref[b], lmax)
        assert e.max() < TOL[prec], (b, e.max(), int(np.argmax(e)))


def _damped_maps(nside, lmax, seeds):
    """Noise-free skies with the damped spectrum C_l = l^-2 exp(-(l/400)^2)."""
    alms = np.stack([skies.gaussian_alm(skies.cl_workload2(lmax), lmax, np.random.Generator(np.random.PCG64(s)))
                     for s in seeds])
    return skies.synthesize(alms, nside, lmax), alms


@pytest.mark.parametrize("sweeps", [False, True], ids=["operators", "sweeps"])
def test_tensor_core_damped_spectrum_nside256(hp, sweeps):
    """The FP16-pair tensor-core kernels (FP32 plan, 10 maps: the per-order
    operators, or D ahead of the run-time sweeps) on noise-free skies whose
    spectrum falls by exp(-(l/400)^2): every degree of every map within 1e-5 of
    the oracle, like the FP32-pipe kernels (which give other bits)."""
    ns, L, B = 256, 512, 10
    maps, _ = _damped_maps(ns, L, range(9100, 9100 + B))
    maps = maps.astype(np.float32).astype(np.float64)
    x = torch.as_tensor(maps, dtype=torch.float32, device="cuda")
    plan = hp.Plan(ns, L, B, "fp32", sweeps=sweeps)
    assert bool(plan.flags & hp.HPX_FLAG_SWEEPS) == sweeps
    a = plan.analyze(x)
    a_simt = hp.Plan(ns, L, B, "fp32", sweeps=sweeps, simt=True).analyze(x)
    plan.sync()
    assert not torch.equal(a, a_simt)
    a = a.cpu().numpy().astype(np.complex128)
    ref = hp2sph.analyze(maps, ns, L)
    for b in range(B):
        e = per_l_error(a[b], ref[b], L)
        assert e.max() < TOL["fp32"], (b, e.max(), int(np.argmax(e)))


@pytest.mark.slow
def test_tensor_core_damped_spectrum_nside1024(hp):
    """32 FP32 maps at Nside 1024 with the damped, noise-free spectrum, where the
    high degrees lie up to 1e-9 below the low ones (the range the FP16 pairs of
    the tensor-core kernel have to carry).  Maps 0 and 31 are seeded skies; maps
    1-30 are quarter turns and mirrors of them.  On a sample of orders, per
    degree: the tensor-core path meets 1e-5 wherever the FP32-pipe path (the
    same stages with the contraction in FP32 FMAs) meets it with a margin of 2,
    and is never worse than twice its error (or half the gate): the degrees that
    miss 1e-5 on both are those whose power lies below the FP32 rounding of the
    map (white error floor of FP32 arithmetic)."""
    ns, L, B = 1024, 2048, 32
    base, alms = _damped_maps(ns, L, [9200, 9231])
    q, mir = ring_perm(ns, True), ring_perm(ns, False)
    perms = [np.arange(base.shape[1]), q, mir, q[q], q[mir], q[q][q], q[q][mir], q[q][q][mir]]
    maps = np.empty((B, base.shape[1]), dtype=np.float32)
    for b in range(B):
        src = base[0] if b < B // 2 else base[1]
        maps[b] = src[perms[(b if b < B // 2 else B - 1 - b) % len(perms)]]
    assert np.array_equal(maps[0], base[0].astype(np.float32))
    assert np.array_equal(maps[B - 1], base[1].astype(np.float32))
    x = torch.as_tensor(maps, device="cuda")
    tc = hp.Plan(ns, L, B, "fp32")
    a_tc = tc.analyze(x).cpu().numpy().astype(np.complex128)
    tc.close()
    simt = hp.Plan(ns, L, B, "fp32", simt=True)
    a_si = simt.analyze(x).cpu().numpy().astype(np.complex128)
    simt.close()
    strat = [int((k + 0.5) * (L + 1) / 12) for k in range(12)]
    ref = hp2sph.analyze_columns(np.stack([maps[0], maps[B - 1]]).astype(np.float64), ns, L, strat)
    for k, b in enumerate((0, B - 1)):
        norms = per_l_norms(alms[k], L)
        cols = lambda a: {m: a[b][hp2sph.alm_index(m, m, L):hp2sph.alm_index(m, m, L) + L - m + 1] for m in strat}
        rk = {m: ref[m][k] for m in strat}
        e_tc = sampled_per_l_errors(cols(a_tc), rk, norms, L)
        e_si = sampled_per_l_errors(cols(a_si), rk, norms, L)
        assert (e_si[2:800] < TOL["fp32"]).all(), (b, e_si[2:800].max())     # FP32 resolves these degrees
        clear = e_si < 0.5 * TOL["fp32"]                                      # ... with a margin of 2
        assert (e_tc[clear] < TOL["fp32"]).all(), (b, e_tc[clear].max())
        assert (e_tc <= np.maximum(2.0 * e_si, 0.5 * TOL["fp32"])).all(), (b, np.max(e_tc / np.maximum(e_si, 1e-30)))
