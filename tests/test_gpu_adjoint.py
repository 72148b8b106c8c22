"""hpx_synthesize is the exact adjoint of hpx_analyze (P8), and the map gradient
of a C_l loss through it matches finite differences (P9)."""

import numpy as np
import pytest

import skies
from oracle import dense, hp2sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hp():
    import os
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    return hp


def _alm_dot(a, b, lmax):
    return dense.alm_dot(a, b, lmax)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("nside,lmax,B", [(2, 4, 2), (4, 8, 3), (8, 13, 2), (32, 64, 3), (64, 128, 17)])
def test_dot_test(hp, prec, tol, nside, lmax, B):
    """<A f, a> = <f, A^T a> with the stated inner products."""
    rng = np.random.default_rng(nside + B)
    plan = hp.Plan(nside, lmax, B, prec)
    rd = torch.float64 if prec == "fp64" else torch.float32
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    f = torch.as_tensor(rng.standard_normal((B, plan.npix)), dtype=rd, device="cuda")
    a_np = rng.standard_normal((B, plan.nalm)) + 1j * rng.standard_normal((B, plan.nalm))
    a = torch.as_tensor(a_np, dtype=cd, device="cuda")
    Af = plan.analyze(f).cpu().numpy()
    Ata = plan.synthesize(a).cpu().numpy()
    plan.sync()
    fn = f.cpu().numpy().astype(np.float64)
    for b in range(B):
        lhs = _alm_dot(Af[b].astype(np.complex128), a_np[b], lmax)
        rhs = float(np.dot(fn[b], Ata[b].astype(np.float64)))
        scale = np.linalg.norm(fn[b]) * np.linalg.norm(Ata[b])
        assert abs(lhs - rhs) <= tol * scale, (b, lhs, rhs)


@pytest.mark.parametrize("nside,lmax", [(2, 4), (4, 8), (4, 6)])
def test_synthesize_matches_oracle_transpose(hp, nside, lmax):
    """GPU A^T against the transpose of the oracle's dense analysis matrix."""
    A = dense.analysis_matrix(nside, lmax)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, hp2sph.n_alm(lmax))) + 1j * rng.standard_normal((2, hp2sph.n_alm(lmax)))
    ref = dense.transpose_apply(A, a, lmax)
    plan = hp.Plan(nside, lmax, 2, "fp64")
    got = plan.synthesize(torch.as_tensor(a, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


def test_imaginary_m0_ignored(hp):
    ns, L = 8, 16
    plan = hp.Plan(ns, L, 1, "fp64")
    a = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    a[0, : L + 1] = 1j          # purely imaginary a_l0
    out = plan.synthesize(a)
    assert torch.count_nonzero(out).item() == 0


def test_cl_loss_gradient_finite_differences(hp):
    """P9: loss = sum_l w_l (C_l - C*_l)^2, w_l = 1/l (l >= 2), C*_l a seeded power
    law; the gradient through the adjoint against central differences (FP64)."""
    ns, L = 16, 32
    maps, _ = skies.small_powerlaw_maps(ns, 1, seed=5)
    rng = np.random.default_rng(8)
    cstar = torch.as_tensor(skies.power_law(L, 2.2) * rng.uniform(0.5, 1.5, L + 1), device="cuda")
    wl = torch.zeros(L + 1, dtype=torch.float64, device="cuda")
    wl[2:] = 1.0 / torch.arange(2, L + 1, dtype=torch.float64, device="cuda")
    plan = hp.Plan(ns, L, 1, "fp64")

    def loss(x):
        c = hp.cl(hp.analyze(x, plan), plan)
        return torch.sum(wl * (c[0] - cstar) ** 2)

    x = torch.as_tensor(maps, device="cuda").requires_grad_(True)
    L0 = loss(x)
    L0.backward()
    g = x.grad.detach()
    for k in range(4):
        d = torch.as_tensor(rng.standard_normal(maps.shape), device="cuda")
        eps = 1e-4
        with torch.no_grad():
            fd = (loss(x + eps * d) - loss(x - eps * d)) / (2 * eps)
        an = torch.sum(g * d)
        assert abs(fd.item() - an.item()) <= 1e-7 * max(abs(an.item()), 1e-30), (fd.item(), an.item())


def _euclid(a, b):
    """Plain real inner product of packed complex arrays read as (re, im) pairs."""
    return float(np.sum(a.real * b.real + a.imag * b.imag))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("kind", ["uniform", "uneven"])
def test_analyze_vjp_is_euclidean_transpose(hp, prec, tol, kind):
    """hpx_analyze_vjp: <A f, g> = <f, vjp(g)> with the plain inner product on the
    packed (re, im) array, for a uniform plan and for an uneven (nsides) plan
    whose layouts are concatenated; the imaginary parts of a_l0 are dropped."""
    rng = np.random.default_rng(31)
    if kind == "uniform":
        plan = hp.Plan(8, 16, 3, prec)
        shape_f, shape_a = (3, plan.npix), (3, plan.nalm)
    else:
        plan = hp.Plan(nsides=[8, 4, 8, 16], precision=prec)
        shape_f, shape_a = (plan.npix,), (plan.nalm,)
    rd = torch.float64 if prec == "fp64" else torch.float32
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    f = rng.standard_normal(shape_f)
    g = rng.standard_normal(shape_a) + 1j * rng.standard_normal(shape_a)
    Af = plan.analyze(torch.as_tensor(f, dtype=rd, device="cuda")).cpu().numpy().astype(np.complex128)
    vg = plan.analyze_vjp(torch.as_tensor(g, dtype=cd, device="cuda")).cpu().numpy().astype(np.float64)
    plan.sync()
    lhs = _euclid(Af.ravel(), g.ravel())
    rhs = float(np.dot(f.ravel(), vg.ravel()))
    assert abs(lhs - rhs) <= tol * np.linalg.norm(f) * np.linalg.norm(vg), (lhs, rhs)


@pytest.mark.parametrize("kind", ["uniform", "uneven"])
def test_cl_vjp_formula(hp, kind):
    """hpx_cl_vjp: dL/da_lm = g_l 2 w_m a_lm / (2l+1) (w_0 = 1, w_m = 2), with the
    degree of every packed coefficient found from the layout on the host."""
    rng = np.random.default_rng(7)
    if kind == "uniform":
        plan = hp.Plan(8, 13, 2, "fp64")
        lmaxs = [13, 13]
    else:
        plan = hp.Plan(nsides=[4, 8, 4], lmaxs=[8, 11, 5], precision="fp64")
        lmaxs = [8, 11, 5]
    a_parts, g_parts, want = [], [], []
    for L in lmaxs:
        n = hp2sph.n_alm(L)
        a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        g = rng.standard_normal(L + 1)
        w = np.zeros(n)
        for m in range(L + 1):
            for l in range(m, L + 1):
                w[hp2sph.alm_index(l, m, L)] = g[l] * 2.0 * (1.0 if m == 0 else 2.0) / (2 * l + 1)
        a_parts.append(a)
        g_parts.append(g)
        want.append(w * a)
    shape = (len(lmaxs), -1) if kind == "uniform" else (-1,)
    a_t = torch.as_tensor(np.concatenate(a_parts).reshape(shape), device="cuda")
    g_t = torch.as_tensor(np.concatenate(g_parts).reshape(shape), device="cuda")
    got = plan.cl_vjp(a_t, g_t).cpu().numpy().ravel()
    np.testing.assert_allclose(got, np.concatenate(want), rtol=1e-14, atol=0)


def test_cl_loss_gradient_uneven_plan(hp):
    """P9 for an uneven batch (nsides 8, 16, 8; concatenated 1-D layouts): the
    autograd gradient of sum_i sum_l w_l (C_l^(i) - C*_l)^2 against central
    finite differences (FP64)."""
    nsides = [8, 16, 8]
    maps = [skies.small_powerlaw_maps(ns, 1, seed=40 + k)[0][0] for k, ns in enumerate(nsides)]
    plan = hp.Plan(nsides=nsides, precision="fp64")
    rng = np.random.default_rng(9)
    targets, weights = [], []
    for ns in nsides:
        L = 2 * ns
        targets.append(skies.power_law(L, 2.1) * rng.uniform(0.5, 1.5, L + 1))
        w = np.zeros(L + 1)
        w[2:] = 1.0 / np.arange(2, L + 1)
        weights.append(w)
    cstar = torch.as_tensor(np.concatenate(targets), device="cuda")
    wl = torch.as_tensor(np.concatenate(weights), device="cuda")

    def loss(x):
        c = hp.cl(hp.analyze(x, plan), plan)
        return torch.sum(wl * (c - cstar) ** 2)

    x = torch.as_tensor(np.concatenate(maps), device="cuda").requires_grad_(True)
    loss(x).backward()
    g = x.grad.detach()
    for _ in range(3):
        d = torch.as_tensor(rng.standard_normal(x.shape), device="cuda")
        eps = 1e-4
        with torch.no_grad():
            fd = (loss(x + eps * d) - loss(x - eps * d)) / (2 * eps)
        an = torch.sum(g * d)
        assert abs(fd.item() - an.item()) <= 1e-7 * max(abs(an.item()), 1e-30), (fd.item(), an.item())
