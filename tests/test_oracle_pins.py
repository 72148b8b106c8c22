"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own formulas (closed forms, textbook values, a
third-party spherical-harmonic routine, brute-force quadrature, symmetries,
the paper's potential-spline test with its exact coefficients)."""

import os

import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import dense, geometry, hp2sph
from oracle.legendre import pbar_table, ylm

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------- geometry
def test_geometry_nside2_golden(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "healpix_nside2_rings.txt"))
    rings = geometry.ring_table(2)
    assert len(rings) == rows.shape[0] == 7
    for r, row in zip(rings, rows):
        assert r["z"] == pytest.approx(row[1] / row[2], abs=1e-15)
        assert np.cos(r["theta"]) == pytest.approx(row[1] / row[2], abs=1e-15)
        assert r["nphi"] == int(row[3])
        assert r["phi0"] == pytest.approx(np.pi * row[4] / row[5], abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 64])
def test_geometry_counts_and_symmetry(nside):
    rings = geometry.ring_table(nside)
    assert len(rings) == 4 * nside - 1
    assert sum(r["nphi"] for r in rings) == 12 * nside * nside
    th = np.array([r["theta"] for r in rings])
    assert np.all(np.diff(th) > 0)
    np.testing.assert_allclose(th + th[::-1], np.pi, atol=1e-14)
    # equal area: the rings split the sphere into bands whose pixel counts are
    # proportional to area; between ring centres the z-spacing in the equatorial
    # belt is the constant 2/(3 Nside)
    z = np.array([r["z"] for r in rings])
    if nside > 1:
        eq = z[nside - 1:3 * nside]
        np.testing.assert_allclose(-np.diff(eq), 2.0 / (3 * nside), atol=1e-14)
    # standard HEALPix: an equatorial ring j is shifted iff (j - Nside) is even;
    # Eq. (healpts) agrees with that for every Nside = 2^t >= 2
    for j in range(nside, 3 * nside + 1 if nside >= 2 else 0):
        assert rings[j - 1]["shifted"] == ((j - nside) % 2 == 0)


# ----------------------------------------------------------------- Y_l^m
def test_ylm_textbook_closed_forms(golden_dir):
    t, lam = 0.7, 1.3
    ct, st, e = np.cos(t), np.sin(t), np.exp(1j * lam)
    closed = {
        (0, 0): 1 / np.sqrt(4 * np.pi),
        (1, 0): np.sqrt(3 / (4 * np.pi)) * ct,
        (1, 1): -np.sqrt(3 / (8 * np.pi)) * st * e,
        (2, 0): np.sqrt(5 / (16 * np.pi)) * (3 * ct ** 2 - 1),
        (2, 1): -np.sqrt(15 / (8 * np.pi)) * st * ct * e,
        (2, 2): np.sqrt(15 / (32 * np.pi)) * st ** 2 * e ** 2,
        (3, 3): -np.sqrt(35 / (64 * np.pi)) * st ** 3 * e ** 3,
    }
    rows = np.loadtxt(os.path.join(golden_dir, "ylm_textbook.txt"), dtype=str)
    for l, m, _ in rows:
        l, m = int(l), int(m)
        assert ylm(l, m, lam, t) == pytest.approx(closed[(l, m)], abs=1e-15)
        # negative order: Y_l^{-m} = (-1)^m conj(Y_l^m)
        assert ylm(l, -m, lam, t) == pytest.approx((-1) ** m * np.conj(closed[(l, m)]), abs=1e-15)


def test_ylm_matches_scipy():
    rng = np.random.default_rng(3)
    th = rng.uniform(0.0, np.pi, 40)
    lam = rng.uniform(0.0, TWO_PI, 40)
    for l in [0, 1, 5, 17, 40, 64]:
        for m in sorted({0, min(1, l), l // 3, l // 2, l}):
            for s in (1, -1):
                np.testing.assert_allclose(ylm(l, s * m, lam, th), sph_harm_y(l, s * m, th, lam),
                                           atol=5e-13, rtol=0)


@pytest.mark.parametrize("lmax", [64, 700])
def test_pbar_orthonormal(lmax):
    """P1: int_{-1}^{1} Pbar_l^m Pbar_l'^m dx = delta_ll' (Gauss-Legendre, exact)."""
    x, w = np.polynomial.legendre.leggauss(lmax + 2)
    for m in sorted({0, 1, 2, lmax // 3, lmax - 1, lmax}):
        P = pbar_table(m, lmax, x)
        G = (P * w) @ P.T
        # rounding grows about linearly with the recurrence length
        np.testing.assert_allclose(G, np.eye(P.shape[0]), atol=3e-14 * lmax)


def test_pbar_large_order_near_pole_scaling():
    """Values far below the float64 range at the start of the recurrence must
    come out right once they grow: compare with the log-space closed form of the
    sectoral Pbar_m^m and the l = m+1 relation Pbar_{m+1}^m = sqrt(2m+3) x Pbar_m^m."""
    m = 1500
    x = np.cos(np.array([0.3, 0.6]))
    P = pbar_table(m, m + 1, x)
    from math import lgamma, log
    # |Pbar_m^m| = sqrt((2m+1)/2 * (2m)!/(2^(2m) (m!)^2)) sin^m
    lg = 0.5 * (log((2 * m + 1) / 2.0) + lgamma(2 * m + 1) - 2 * m * log(2.0) - 2 * lgamma(m + 1))
    ref = np.exp(lg + m * np.log(np.sin(np.arccos(x))))
    np.testing.assert_allclose(np.abs(P[0]), ref, rtol=1e-11)
    np.testing.assert_allclose(P[1], np.sqrt(2 * m + 3) * x * P[0], rtol=1e-13)
    # a deep-underflow start still reaches the right values at higher degree:
    # orthonormality at m = 1500 over l up to 2000 uses those scaled starts
    xg, wg = np.polynomial.legendre.leggauss(2002)
    Pg = pbar_table(m, 2000, xg)
    G = (Pg * wg) @ Pg.T
    np.testing.assert_allclose(G, np.eye(Pg.shape[0]), atol=5e-11)


# ----------------------------------------------------------------- step 1
def test_ring_step_recovers_trig_polynomial():
    """A ring sampled from sum_n c_n e^{i n lambda} (|n| < nphi/2, real) gives back
    exactly the c_n after the half-pixel shift, zero padded beyond."""
    ns = 8
    p = 2 * ns
    rng = np.random.default_rng(11)
    rings = geometry.ring_table(ns)
    th, lam = geometry.pixel_angles(ns)
    f = np.zeros(th.size)
    truth = {}
    for i, r in enumerate(rings):
        half = r["nphi"] // 2
        c = rng.standard_normal(half) + 1j * rng.standard_normal(half)
        c[0] = c[0].real
        truth[i] = c
        ll = lam[r["start"]:r["start"] + r["nphi"]]
        vals = c[0].real + 2 * np.real(np.sum(c[1:, None] * np.exp(1j * np.arange(1, half)[:, None] * ll[None]), axis=0))
        f[r["start"]:r["start"] + r["nphi"]] = vals
    rc = hp2sph.ring_coefficients(f, ns)[0]       # (rings, 2p), k = -p..p-1
    for i, r in enumerate(rings):
        half = r["nphi"] // 2
        c = truth[i]
        for k in range(-p, p):
            want = c[k] if 0 <= k < half else (np.conj(c[-k]) if -half < k < 0 else 0.0)
            assert abs(rc[i, k + p] - want) < 1e-12


def test_ring_step_nyquist_reading():
    """Nyquist term (reading of Eq. trig_expansion vs Eq. interp_cond): data
    cos(nphi/2 (lambda - phi0)) on a ring become 1/2 e^{-+i (nphi/2) phi0} at
    +-nphi/2; on a shifted equatorial ring the two cancel on the upsampled grid."""
    ns = 4
    p = 2 * ns
    rings = geometry.ring_table(ns)
    th, lam = geometry.pixel_angles(ns)
    for i in [1, ns, ns - 1 + 1]:      # polar ring j=2, equatorial shifted/unshifted
        r = rings[i]
        f = np.zeros(th.size)
        ll = lam[r["start"]:r["start"] + r["nphi"]]
        half = r["nphi"] // 2
        f[r["start"]:r["start"] + r["nphi"]] = np.cos(half * (ll - r["phi0"]))
        rc = hp2sph.ring_coefficients(f, ns)[0, i]
        if half < p:
            assert rc[half + p] == pytest.approx(0.5 * np.exp(-1j * half * r["phi0"]), abs=1e-13)
            assert rc[-half + p] == pytest.approx(0.5 * np.exp(1j * half * r["phi0"]), abs=1e-13)
        else:
            assert rc[0] == pytest.approx(np.cos(half * r["phi0"]), abs=1e-13)
        others = np.delete(rc, [half + p, -half + p] if half < p else [0])
        assert np.max(np.abs(others)) < 1e-13


def test_ring_step_interpolates_data():
    """The padded coefficients evaluated at a ring's own pixel longitudes give the
    data back (Eq. interp_cond), for a random map."""
    ns = 4
    p = 2 * ns
    rng = np.random.default_rng(5)
    f = rng.standard_normal(12 * ns * ns)
    rc = hp2sph.ring_coefficients(f, ns)[0]
    th, lam = geometry.pixel_angles(ns)
    k = np.arange(-p, p)
    for i, r in enumerate(geometry.ring_table(ns)):
        ll = lam[r["start"]:r["start"] + r["nphi"]]
        vals = (np.exp(1j * np.outer(ll, k)) @ rc[i])
        if r["nphi"] == 4 * ns:   # +-p share one column: add the missing +p term
            vals = vals  # c_{-p} + c_{p} at -p, and e^{-ip l} != e^{ip l} off the grid
        if r["nphi"] < 4 * ns or r["phi0"] == 0.0:
            np.testing.assert_allclose(vals.real, f[r["start"]:r["start"] + r["nphi"]], atol=1e-12)


# ----------------------------------------------------------------- poles
def test_pole_fit_exact_for_quadratics():
    ns = 8
    th, lam = geometry.pixel_angles(ns)
    x = np.sin(th) * np.cos(lam)
    y = np.sin(th) * np.sin(lam)
    f = 1.7 - 0.3 * x + 0.9 * y + 2.2 * x * x - 1.1 * x * y + 0.4 * y * y
    pv = hp2sph.pole_values(f, ns)[0]
    assert pv[0] == pytest.approx(1.7, abs=1e-13)
    assert pv[1] == pytest.approx(1.7, abs=1e-13)


def test_pole_fit_exact_for_y20_and_m1():
    ns = 8
    th, lam = geometry.pixel_angles(ns)
    f = np.real(ylm(2, 0, lam, th)) + 2 * np.real((0.3 - 0.7j) * ylm(5, 1, lam, th))
    pv = hp2sph.pole_values(f, ns)[0]
    y20_north = np.sqrt(5 / (16 * np.pi)) * 2.0
    assert pv[0] == pytest.approx(y20_north, abs=1e-13)
    assert pv[1] == pytest.approx(y20_north, abs=1e-13)


# ----------------------------------------------------------------- step 2
def test_latitude_ls_parity_equals_full():
    ns = 8
    rng = np.random.default_rng(2)
    f = rng.standard_normal((2, 12 * ns * ns))
    p = 2 * ns
    ks = np.arange(-p, p)
    col = hp2sph.latitude_columns(f, ns, ks)
    a = hp2sph.dfs_ls_full(col, ns, ks)
    b = hp2sph.dfs_ls_parity(col, ns, ks)
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_latitude_ls_normal_equations():
    """The LS solution satisfies V^H (V C - y) = 0 over the DFS nodes."""
    ns = 8
    p = 2 * ns
    rng = np.random.default_rng(4)
    f = rng.standard_normal(12 * ns * ns)
    ks = np.array([-p, -3, 0, 1, 6])
    col = hp2sph.latitude_columns(f, ns, ks)
    C = hp2sph.dfs_ls_parity(col, ns, ks)[0]
    nodes, src, mirrored = hp2sph.dfs_nodes(ns)
    V = np.exp(1j * np.outer(nodes, np.arange(-p, p + 1)))
    for c, k in enumerate(ks):
        y = col[0, src, c] * np.where(mirrored, (-1.0) ** abs(k), 1.0)
        g = V.conj().T @ (V @ C[:, c] - y)
        assert np.max(np.abs(g)) < 1e-11 * max(1.0, np.max(np.abs(y)))


def test_latitude_ls_reproduces_trig_polynomials():
    """Data sampled from a DFS-consistent trigonometric polynomial of degree p
    in theta are reproduced exactly."""
    ns = 8
    p = 2 * ns
    t = geometry.latitude_nodes(ns)
    rng = np.random.default_rng(9)
    ks = np.array([0, 1, 4, 7])
    col = np.zeros((1, t.size, ks.size), dtype=complex)
    want = np.zeros((2 * p + 1, ks.size), dtype=complex)
    for c, k in enumerate(ks):
        if k % 2 == 0:
            g = rng.standard_normal(p + 1) + 1j * rng.standard_normal(p + 1)
            col[0, :, c] = np.cos(np.outer(t, np.arange(p + 1))) @ g
            want[p, c] = g[0]
            want[p + 1:, c] = g[1:] / 2
            want[:p, c] = g[1:][::-1] / 2
        else:
            s = rng.standard_normal(p) + 1j * rng.standard_normal(p)
            col[0, :, c] = np.sin(np.outer(t, np.arange(1, p + 1))) @ s
            want[p + 1:, c] = s / 2j
            want[:p, c] = -s[::-1] / 2j
    np.testing.assert_allclose(hp2sph.dfs_ls_parity(col, ns, ks)[0], want, atol=1e-12)
    np.testing.assert_allclose(hp2sph.dfs_ls_full(col, ns, ks)[0], want, atol=1e-12)


# ----------------------------------------------------------------- step 3
def test_step3_matches_bruteforce_quadrature():
    """P7: the Fourier-to-SH step equals the inner product <f~, Y_l^m> of
    Eq. (sphip) computed by brute force: the DFS bivariate series evaluated on a
    fine grid, 4p-point Gauss-Legendre in cos(theta) times a 4p-point trapezoid
    in lambda, against scipy's Y_l^m."""
    ns = 4
    p = 2 * ns
    rng = np.random.default_rng(7)
    f = rng.standard_normal(12 * ns * ns)
    ks = np.arange(-p, p)
    col = hp2sph.latitude_columns(f, ns, ks)
    C = hp2sph.dfs_ls_parity(col, ns, ks)[0]
    X = np.zeros((2 * p + 1, 2 * p + 1), dtype=complex)     # k = -p..p
    X[:, 1:2 * p] = C[:, 1:]
    X[:, 0] = 0.5 * C[:, 0]
    X[:, 2 * p] = 0.5 * C[:, 0]
    x, w = np.polynomial.legendre.leggauss(4 * p)
    th = np.arccos(x)
    nl = 4 * p
    lam = TWO_PI * np.arange(nl) / nl
    Ej = np.exp(1j * np.outer(th, np.arange(-p, p + 1)))
    Ek = np.exp(1j * np.outer(np.arange(-p, p + 1), lam))
    F = Ej @ X @ Ek                                           # f~(theta_g, lambda_t)
    got = hp2sph.fourier_to_sh(C[None], ns, p, ks, range(-p, p + 1))
    TH, LA = np.meshgrid(th, lam, indexing="ij")
    for l in range(p + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, m, TH, LA)
            ref = np.sum(w[:, None] * F * np.conj(Y)) * TWO_PI / nl
            assert abs(got[m][0, l - abs(m)] - ref) < 1e-12, (l, m)


# ----------------------------------------------------------------- end to end
def _real_map(nside, coeffs):
    th, lam = geometry.pixel_angles(nside)
    f = np.zeros(th.size)
    for (l, m), c in coeffs.items():
        y = ylm(l, m, lam, th)
        f += np.real(c * y) if m == 0 else 2 * np.real(c * y)
    return f


@pytest.mark.parametrize("nside", [4, 16])
def test_exact_subspace(nside):
    """P3: maps in span{Y_0^0, Y_2^0, Y_l^{+-1}} are analysed exactly: order +-1 is
    resolved on every ring, the pole fit is exact for them (quadratic in the
    tangent plane / zero), and their latitude profiles lie in the LS span."""
    p = 2 * nside
    rng = np.random.default_rng(21)
    coeffs = {(0, 0): 0.8, (2, 0): -1.3}
    for l in range(1, p + 1):
        coeffs[(l, 1)] = rng.standard_normal() + 1j * rng.standard_normal()
    a = hp2sph.analyze(_real_map(nside, coeffs), nside)
    want = np.zeros_like(a)
    for (l, m), c in coeffs.items():
        want[hp2sph.alm_index(l, m, p)] = c
    np.testing.assert_allclose(a, want, atol=1e-12)


def test_not_exact_outside_subspace():
    """Y_1^0 is not reproduced exactly (the quadratic pole fit of cos(theta) is
    not exact), so the subspace test above is not vacuous."""
    ns = 8
    a = hp2sph.analyze(_real_map(ns, {(1, 0): 1.0}), ns)
    err = abs(a[hp2sph.alm_index(1, 0, 2 * ns)] - 1.0)
    assert 1e-10 < err < 1e-2


def test_symmetries_quarter_turn_mirror_real():
    """P5: lambda -> lambda + pi/2 maps a_l^m to e^{-i m pi/2} a_l^m exactly (each
    ring has 4j points, a shift by j pixels); the north-south mirror maps a_l^m to
    (-1)^{l+m} a_l^m; real data give a_l^{-m} = (-1)^m conj(a_l^m)."""
    ns = 8
    p = 2 * ns
    rng = np.random.default_rng(13)
    f = rng.standard_normal(12 * ns * ns)
    rings = geometry.ring_table(ns)
    g = np.empty_like(f)
    for r in rings:
        seg = f[r["start"]:r["start"] + r["nphi"]]
        g[r["start"]:r["start"] + r["nphi"]] = np.roll(seg, r["nphi"] // 4)
    h = np.empty_like(f)
    for i, r in enumerate(rings):
        s = rings[len(rings) - 1 - i]
        h[r["start"]:r["start"] + r["nphi"]] = f[s["start"]:s["start"] + s["nphi"]]
    full_f = hp2sph.analyze_columns(f, ns, p, range(-p, p + 1))
    full_g = hp2sph.analyze_columns(g, ns, p, range(0, p + 1))
    full_h = hp2sph.analyze_columns(h, ns, p, range(0, p + 1))
    for m in range(0, p + 1):
        l = np.arange(m, p + 1)
        # rolling data right by nphi/4 pixels evaluates f at lambda - pi/2
        np.testing.assert_allclose(full_g[m], full_f[m] * np.exp(-1j * m * np.pi / 2), atol=1e-12)
        np.testing.assert_allclose(full_h[m], full_f[m] * (-1.0) ** (l + m), atol=1e-12)
        np.testing.assert_allclose(full_f[-m], (-1.0) ** m * np.conj(full_f[m]), atol=1e-12)


def test_linearity():
    ns = 4
    rng = np.random.default_rng(8)
    f, g = rng.standard_normal((2, 12 * ns * ns))
    np.testing.assert_allclose(hp2sph.analyze(2.5 * f - g, ns),
                               2.5 * hp2sph.analyze(f, ns) - hp2sph.analyze(g, ns), atol=1e-12)


def _spline_map_and_exact(nside, golden_dir, lmax):
    rows = np.loadtxt(os.path.join(golden_dir, "potential_spline.txt"))
    th, lam = geometry.pixel_angles(nside)
    X = np.stack([np.sin(th) * np.cos(lam), np.sin(th) * np.sin(lam), np.cos(th)], axis=1)
    f = np.zeros(th.size)
    exact = np.zeros(hp2sph.n_alm(lmax), dtype=complex)
    for c, lc, tc in rows:
        xc = np.array([np.sin(tc) * np.cos(lc), np.sin(tc) * np.sin(lc), np.cos(tc)])
        f += c * np.maximum(2.0 - 2.0 * X @ xc, 0.0) ** 1.5
        for l in range(lmax + 1):
            fac = 18 * np.pi / ((l + 2.5) * (l + 1.5) * (l + 0.5) * (l - 0.5) * (l - 1.5))
            for m in range(l + 1):
                exact[hp2sph.alm_index(l, m, lmax)] += c * fac * np.conj(sph_harm_y(l, m, tc, lc))
    return f, exact


def test_potential_spline_converges(golden_dir):
    """P4 (Sec. 4.1, Fig. 5): the max error against the exact coefficients of
    Eq. (alm) falls steadily as Nside = 2^t grows (the figure gives the trend,
    not the values).  Compared over l <= 8, present at every resolution."""
    errs = []
    for t in [2, 3, 4, 5]:
        ns = 2 ** t
        f, exact = _spline_map_and_exact(ns, golden_dir, 2 * ns)
        a = hp2sph.analyze(f, ns)
        idx = [hp2sph.alm_index(l, m, 2 * ns) for l in range(9) for m in range(l + 1)]
        errs.append(np.max(np.abs(a[idx] - exact[idx])))
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-4, errs


# ----------------------------------------------------------------- C_l, A^T
def test_cl_definition_and_appended_harmonics():
    """Eq. (APS); a real combination (Y_l^m + (-1)^m Y_l^{-m})/sqrt(2) raises C_l by
    exactly 1/(2l+1) (Sec. 4.2)."""
    lmax = 12
    rng = np.random.default_rng(1)
    a = rng.standard_normal(hp2sph.n_alm(lmax)) + 1j * rng.standard_normal(hp2sph.n_alm(lmax))
    for l in range(lmax + 1):
        a[hp2sph.alm_index(l, 0, lmax)] = a[hp2sph.alm_index(l, 0, lmax)].real
    c0 = hp2sph.cl(a, lmax)
    for l in range(lmax + 1):
        s = sum(abs(a[hp2sph.alm_index(l, m, lmax)]) ** 2 * (1 if m == 0 else 2) for m in range(l + 1))
        assert c0[l] == pytest.approx(s / (2 * l + 1), rel=1e-14)
    b = a.copy()
    b[hp2sph.alm_index(9, 4, lmax)] += 1 / np.sqrt(2)        # |a_9^{+-4}|^2 each += 1/2
    # cross term vanishes when the added part is orthogonal: use a fresh zero slot
    z = np.zeros_like(a)
    z[hp2sph.alm_index(9, 4, lmax)] = 1 / np.sqrt(2)
    assert (hp2sph.cl(z, lmax)[9]) == pytest.approx(1.0 / 19.0, rel=1e-15)


def test_dense_transpose_dot():
    """P8 for the oracle: <A f, a> = <f, A^T a> with the stated inner products."""
    ns = 2
    lmax = 4
    A = dense.analysis_matrix(ns, lmax)
    rng = np.random.default_rng(6)
    f = rng.standard_normal(12 * ns * ns)
    a = rng.standard_normal(hp2sph.n_alm(lmax)) + 1j * rng.standard_normal(hp2sph.n_alm(lmax))
    lhs = dense.alm_dot(hp2sph.analyze(f, ns, lmax), a, lmax)
    rhs = float(np.dot(f, dense.transpose_apply(A, a, lmax)[0]))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_synthesis_matches_scipy_brute_force():
    """Oracle SH synthesis = brute-force sum of scipy's Y_l^m at every pixel
    centre (negative orders from a_l^{-m} = (-1)^m conj(a_l^m))."""
    rng = np.random.default_rng(11)
    ns, L = 4, 8
    a = rng.standard_normal(hp2sph.n_alm(L)) + 1j * rng.standard_normal(hp2sph.n_alm(L))
    for l in range(L + 1):
        a[hp2sph.alm_index(l, 0, L)] = a[hp2sph.alm_index(l, 0, L)].real
    f = hp2sph.synthesize(a, ns, L)
    th, ph = geometry.pixel_angles(ns)
    g = np.zeros(len(th), dtype=complex)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            am = a[hp2sph.alm_index(l, abs(m), L)]
            if m < 0:
                am = (-1) ** m * np.conj(am)
            g += am * sph_harm_y(l, m, th, ph)
    assert np.max(np.abs(g.imag)) < 1e-13
    np.testing.assert_allclose(f, g.real, atol=1e-13)


def test_synthesis_then_analysis_exact_subspace():
    """Analysis inverts synthesis exactly on span{Y_0^0, Y_2^0, Y_l^{+-1}}."""
    rng = np.random.default_rng(12)
    ns = 8
    L = 2 * ns
    a = np.zeros(hp2sph.n_alm(L), dtype=complex)
    a[hp2sph.alm_index(0, 0, L)] = 0.7
    a[hp2sph.alm_index(2, 0, L)] = -1.3
    for l in range(1, L + 1):
        a[hp2sph.alm_index(l, 1, L)] = rng.standard_normal() + 1j * rng.standard_normal()
    back = hp2sph.analyze(hp2sph.synthesize(a, ns, L), ns, L)
    np.testing.assert_allclose(back, a, atol=1e-12)


# ---------------------------------------------------------------- Sec. 2.2 (HEALPix software analysis)
def test_equal_weight_matches_brute_force_scipy():
    """Eq. (healsph): (4 pi / N) sum_i conj(Y_l^m(x_i)) f_i, against scipy's Y_l^m at every
    pixel of Nside 2 (a plain double loop)."""
    from scipy.special import sph_harm_y
    from oracle import healpix
    ns, L = 2, 4
    rng = np.random.default_rng(1)
    f = rng.standard_normal(geometry.npix(ns))
    a = healpix.equal_weight(f, ns, L)
    th, ph = geometry.pixel_angles(ns)
    for m in range(L + 1):
        for l in range(m, L + 1):
            ref = 4 * np.pi / f.size * np.sum(np.conj(sph_harm_y(l, m, th, ph)) * f)
            assert abs(a[hp2sph.alm_index(l, m, L)] - ref) < 1e-14


def test_equal_weight_is_scaled_adjoint_of_synthesis():
    """A = (4 pi / N) S^*: <S a, f> = (N / 4 pi) <a, A f> with the real-map coefficient
    inner product (weight 2 for m > 0), S being the pinned synthesis of Eq. (synthesis)."""
    from oracle import healpix
    ns, L = 8, 16
    rng = np.random.default_rng(2)
    f = rng.standard_normal(geometry.npix(ns))
    a = rng.standard_normal(hp2sph.n_alm(L)) + 1j * rng.standard_normal(hp2sph.n_alm(L))
    lhs = float(np.dot(f, hp2sph.synthesize(a, ns, L)))
    rhs = dense.alm_dot(a, healpix.equal_weight(f, ns, L) * geometry.npix(ns) / (4 * np.pi), L)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_jacobi_converges_to_band_limited_coefficients():
    """Eq. (richardson) is Richardson iteration on the normal equations: for a map
    synthesised from coefficients of degree <= Nside (S of full column rank) it converges
    to those coefficients, the error shrinking by more than 10x per iteration here."""
    from oracle import healpix
    ns, L = 8, 8
    rng = np.random.default_rng(3)
    at = rng.standard_normal(hp2sph.n_alm(L)) + 1j * rng.standard_normal(hp2sph.n_alm(L))
    for l in range(L + 1):
        at[hp2sph.alm_index(l, 0, L)] = at[hp2sph.alm_index(l, 0, L)].real
    f = hp2sph.synthesize(at, ns, L)
    errs = [np.abs(healpix.jacobi(f, ns, L, k) - at).max() for k in (0, 1, 2, 3)]
    assert all(errs[k + 1] < 0.1 * errs[k] for k in range(3)), errs
    assert np.abs(healpix.jacobi(f, ns, L, 12) - at).max() < 1e-12
