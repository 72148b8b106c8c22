"""Algorithm 1 (HP2SPH) of Sec. 3, step by step, in float64 (test infrastructure;
see package doc for the readings taken where the paper is silent).

Conventions shared by every function here:

* ``f`` is a real map, shape (N,) or (B, N), RING order, N = 12 Nside^2.
* p = 2 Nside; longitude wavenumbers k run over -p .. p-1 (Eq. bivariateFourier),
  latitude wavenumbers j over -p .. p (m = 4 Nside + 1 modes, Sec. 3.2.2).
* the 4 Nside + 1 latitude nodes on [0, pi] are the north pole (r = 0), the
  4 Nside - 1 rings (r = 1 .. 4 Nside - 1) and the south pole (r = 4 Nside).
* output a_l^m, m >= 0, is packed m-major: idx(l, m) = m (2 lmax + 1 - m) / 2 + l.
"""

import numpy as np

from . import geometry
from .legendre import pbar_table


def alm_index(l, m, lmax):
    return m * (2 * lmax + 1 - m) // 2 + l


def n_alm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def _as_batch(f):
    f = np.asarray(f, dtype=np.float64)
    return (f[None, :], True) if f.ndim == 1 else (f, False)


# --------------------------------------------------------------------------
# Step 1: per-ring trigonometric interpolation, shift and zero padding
# (Sec. 3.1, Eq. trig_expansion and Eq. interp_cond)
# --------------------------------------------------------------------------

def ring_dft(fr, nphi, ns):
    """c~_n = (1/nphi) sum_k f_k exp(-2 pi i n k / nphi) for the wavenumbers ``ns``
    (the solution of the interpolation conditions Eq. interp_cond), as a direct
    sum with the angle reduced exactly: n k mod nphi.  ``fr`` is (B, nphi)."""
    ns = np.asarray(ns, dtype=np.int64)
    k = np.arange(nphi, dtype=np.int64)
    ang = 2.0 * np.pi * (np.mod(ns[:, None] * k[None, :], nphi)) / nphi
    return (fr @ np.exp(-1j * ang).T) / nphi               # (B, len(ns))


def ring_coefficients(f, nside, ks=None):
    """Step 1 for every ring: coefficients of the ring's trigonometric
    interpolant at the un-shifted longitudes of Eq. (upsamp), zero padded to the
    4 Nside wavenumbers k = -p .. p-1.

    For a ring with nphi points and first longitude phi0:
      c_n = c~_n exp(-i n phi0)                        |n| < nphi/2
      c_{+-nphi/2} = 1/2 c~_{-nphi/2} exp(-+i (nphi/2) phi0)   (real-symmetric split)
      c_n = 0                                          |n| > nphi/2 (padding)
    On the 4 Nside-point upsampled grid the wavenumbers +-p coincide, so the
    k = -p entry of an equatorial ring holds c_{-p} + c_{p}.

    Returns (B, 4 Nside - 1, len(ks)) complex for the requested k (default: all).
    """
    f, single = _as_batch(f)
    ns_ = int(nside)
    p = 2 * ns_
    ks = np.arange(-p, p) if ks is None else np.asarray(ks, dtype=np.int64)
    rings = geometry.ring_table(ns_)
    out = np.zeros((f.shape[0], len(rings), ks.size), dtype=np.complex128)
    for i, r in enumerate(rings):
        nphi, phi0 = r["nphi"], r["phi0"]
        half = nphi // 2
        fr = f[:, r["start"]:r["start"] + nphi]
        need = sorted(set(int(k) for k in ks if abs(k) < half) | {-half})
        ct = dict(zip(need, ring_dft(fr, nphi, need).T))
        for c, k in enumerate(ks):
            k = int(k)
            if abs(k) < half:
                out[:, i, c] = ct[k] * np.exp(-1j * k * phi0)
            elif abs(k) == half:
                if half < p:
                    out[:, i, c] = 0.5 * ct[-half] * np.exp(-1j * k * phi0)
                else:   # k == -p on an equatorial ring: c_{-p} + c_{p}
                    out[:, i, c] = 0.5 * ct[-half] * (np.exp(1j * half * phi0)
                                                      + np.exp(-1j * half * phi0))
    return out


def pole_values(f, nside):
    """Values at the north and south poles (Sec. 3.2.1): least squares fit of
    c0 + c1 x + c2 y + c3 x^2 + c4 x y + c5 y^2, (x, y) = (sin t cos l, sin t sin l),
    with unit weights over the pixels of the three rings nearest the pole; the
    pole value is c0.  Returns (B, 2)."""
    f, single = _as_batch(f)
    rings = geometry.ring_table(nside)
    th, lam = geometry.pixel_angles(nside)
    out = np.zeros((f.shape[0], 2))
    for side, idx in enumerate([(0, 1, 2), (len(rings) - 1, len(rings) - 2, len(rings) - 3)]):
        pix = np.concatenate([np.arange(rings[i]["start"], rings[i]["start"] + rings[i]["nphi"])
                              for i in idx])
        x = np.sin(th[pix]) * np.cos(lam[pix])
        y = np.sin(th[pix]) * np.sin(lam[pix])
        V = np.stack([np.ones_like(x), x, y, x * x, x * y, y * y], axis=1)
        coef, *_ = np.linalg.lstsq(V, f[:, pix].T, rcond=None)
        out[:, side] = coef[0]
    return out


def latitude_columns(f, nside, ks=None):
    """Step 1 output with the pole rows added: (B, 4 Nside + 1, len(ks)).
    Row 0 / row 4 Nside hold the pole value at k = 0 and zero elsewhere (a
    function on the sphere is constant in longitude at a pole)."""
    f, single = _as_batch(f)
    p = 2 * int(nside)
    ks = np.arange(-p, p) if ks is None else np.asarray(ks, dtype=np.int64)
    rc = ring_coefficients(f, nside, ks)
    pv = pole_values(f, nside)
    B, R, K = rc.shape
    col = np.zeros((B, R + 2, K), dtype=np.complex128)
    col[:, 1:R + 1, :] = rc
    zero = np.nonzero(ks == 0)[0]
    if zero.size:
        col[:, 0, zero[0]] = pv[:, 0]
        col[:, R + 1, zero[0]] = pv[:, 1]
    return col


# --------------------------------------------------------------------------
# Step 2: DFS doubling and least-squares inverse NUFFT-II in latitude
# (Sec. 3.2.1 Eq. DFS and its remark, Sec. 3.2.2)
# --------------------------------------------------------------------------

def dfs_nodes(nside):
    """The 8 Nside DFS latitude nodes on [0, 2 pi): theta_r (r = 0 .. 4 Nside) and
    2 pi - theta_r (r = 1 .. 4 Nside - 1); second output maps each node to r and a
    flag telling whether it is a mirrored copy."""
    t = geometry.latitude_nodes(nside)
    Q = t.size
    nodes = np.concatenate([t, 2.0 * np.pi - t[1:Q - 1]])
    src = np.concatenate([np.arange(Q), np.arange(1, Q - 1)])
    mirrored = np.concatenate([np.zeros(Q, bool), np.ones(Q - 2, bool)])
    return nodes, src, mirrored


def dfs_ls_full(col, nside, ks):
    """Plain complex least squares per longitude wavenumber k:
    minimise over C_j (j = -p..p)  sum_nodes |sum_j C_j e^{i j theta} - y|^2,
    where the DFS data are y at theta_r and (-1)^k y at 2 pi - theta_r (the remark
    of Sec. 3.2.1: the flipped copy with odd wavenumbers negated).
    ``col`` is (B, 4 Nside + 1, len(ks)); returns C of shape (B, 2p+1, len(ks))."""
    p = 2 * int(nside)
    ks = np.asarray(ks, dtype=np.int64)
    nodes, src, mirrored = dfs_nodes(nside)
    j = np.arange(-p, p + 1)
    V = np.exp(1j * np.outer(nodes, j))
    sign = np.where(mirrored[:, None], ((-1.0) ** np.abs(ks))[None, :], 1.0)   # (nodes, K)
    B = col.shape[0]
    Y = col[:, src, :] * sign[None]                                          # (B, nodes, K)
    Yf = np.transpose(Y, (1, 0, 2)).reshape(nodes.size, -1)
    C, *_ = np.linalg.lstsq(V, Yf, rcond=None)
    return np.transpose(C.reshape(2 * p + 1, B, ks.size), (1, 0, 2))


def dfs_ls_parity(col, nside, ks):
    """The same least squares split by the DFS parity of k (exactly equal, since
    the node set and the data are symmetric under theta -> 2 pi - theta and the
    solution is unique, so C_{-j} = (-1)^k C_j):
      k even: f(theta) = sum_{j=0}^{p} g_j cos(j theta), weights 1 at the poles and
              2 at the rings (each ring appears twice among the DFS nodes);
      k odd:  f(theta) = sum_{j=1}^{p} s_j sin(j theta) over the rings (the pole
              equations read 0 = 0).
    Returns C of shape (B, 2p+1, len(ks))."""
    p = 2 * int(nside)
    ks = np.asarray(ks, dtype=np.int64)
    t = geometry.latitude_nodes(nside)
    Q = t.size
    B = col.shape[0]
    C = np.zeros((B, 2 * p + 1, ks.size), dtype=np.complex128)
    w = np.full(Q, 2.0)
    w[0] = w[-1] = 1.0
    sw = np.sqrt(w)
    jc = np.arange(p + 1)
    Vc = np.cos(np.outer(t, jc)) * sw[:, None]
    js = np.arange(1, p + 1)
    Vs = np.sin(np.outer(t[1:Q - 1], js))
    ev = np.nonzero(ks % 2 == 0)[0]
    od = np.nonzero(ks % 2 != 0)[0]
    if ev.size:
        Y = np.transpose(col[:, :, ev], (1, 0, 2)).reshape(Q, -1) * sw[:, None]
        g, *_ = np.linalg.lstsq(Vc, Y, rcond=None)
        g = np.transpose(g.reshape(p + 1, B, ev.size), (1, 0, 2))
        C[:, p, ev] = g[:, 0]
        C[:, p + 1:, ev] = 0.5 * g[:, 1:]
        C[:, p - 1::-1, ev] = 0.5 * g[:, 1:]
    if od.size:
        Y = np.transpose(col[:, 1:Q - 1, od], (1, 0, 2)).reshape(Q - 2, -1)
        s, *_ = np.linalg.lstsq(Vs, Y, rcond=None)
        s = np.transpose(s.reshape(p, B, od.size), (1, 0, 2))
        C[:, p + 1:, od] = s / 2j
        C[:, p - 1::-1, od] = -s / 2j
    return C


# --------------------------------------------------------------------------
# Step 3: Fourier to spherical harmonic coefficients (Sec. 3.3)
# --------------------------------------------------------------------------

def fourier_to_sh(C, nside, lmax, ks, ms):
    """a_l^m = <f~, Y_l^m> = sqrt(2 pi) int_0^pi F_m(t) Pbar_l^|m|(cos t) sin t dt
    (times (-1)^m for m < 0), where F_m(t) = sum_j X_{j,m} e^{i j t} and X is the
    expanded array of Sec. 3.3 (X_{., +-p} = C_{., -p} / 2).  Gauss-Legendre
    quadrature with p + 2 nodes is exact for these polynomial integrands.

    ``C`` is (B, 2p+1, len(ks)); returns {m: (B, lmax - |m| + 1)} for m in ``ms``."""
    p = 2 * int(nside)
    assert lmax <= p
    ks = [int(k) for k in ks]
    x, w = np.polynomial.legendre.leggauss(p + 2)
    th = np.arccos(x)
    E = np.exp(1j * np.outer(th, np.arange(-p, p + 1)))        # (G, 2p+1)
    out = {}
    for m in ms:
        m = int(m)
        if abs(m) < p:
            Xm = C[:, :, ks.index(m)]
        else:
            Xm = 0.5 * C[:, :, ks.index(-p)]
        F = Xm @ E.T                                            # (B, G)
        P = pbar_table(abs(m), lmax, x)                         # (L, G)
        a = np.sqrt(2.0 * np.pi) * (F * w[None, :]) @ P.T
        if m < 0:
            a = a * (-1.0) ** abs(m)
        out[m] = a
    return out


# --------------------------------------------------------------------------
# Algorithm 1 end to end, and Eq. (APS)
# --------------------------------------------------------------------------

def analyze_columns(f, nside, lmax, ms, ls="parity"):
    """a_l^m for the requested orders ``ms`` (any sign), {m: (B, lmax-|m|+1)}.
    Only the longitude wavenumbers those orders need are computed, by the same
    definitions as the full transform."""
    p = 2 * int(nside)
    ks = sorted(set((int(m) if abs(int(m)) < p else -p) for m in ms))
    col = latitude_columns(f, nside, ks)
    C = (dfs_ls_parity if ls == "parity" else dfs_ls_full)(col, nside, ks)
    return fourier_to_sh(C, nside, lmax, ks, ms)


def analyze(f, nside, lmax=None, ls="parity"):
    """HP2SPH analysis of real map(s): packed a_l^m, m >= 0, (B, n_alm) or (n_alm,)."""
    f, single = _as_batch(f)
    p = 2 * int(nside)
    lmax = p if lmax is None else int(lmax)
    cols = analyze_columns(f, nside, lmax, range(lmax + 1), ls=ls)
    out = np.zeros((f.shape[0], n_alm(lmax)), dtype=np.complex128)
    for m in range(lmax + 1):
        i0 = alm_index(m, m, lmax)
        out[:, i0:i0 + lmax - m + 1] = cols[m]
    return out[0] if single else out


def neumaier_sum(values):
    s = 0.0
    c = 0.0
    for v in values:
        v = float(v)
        t = s + v
        if abs(s) >= abs(v):
            c += (s - t) + v
        else:
            c += (v - t) + s
        s = t
    return s + c


def cl(alm, lmax):
    """Eq. (APS) for a real map from m >= 0 coefficients:
    C_l = (|a_l^0|^2 + 2 sum_{m>0} |a_l^m|^2) / (2l + 1), Neumaier-summed."""
    alm = np.asarray(alm)
    single = alm.ndim == 1
    alm = alm[None] if single else alm
    out = np.zeros((alm.shape[0], lmax + 1))
    for b in range(alm.shape[0]):
        for l in range(lmax + 1):
            terms = [abs(alm[b, alm_index(l, 0, lmax)]) ** 2]
            terms += [2.0 * abs(alm[b, alm_index(l, m, lmax)]) ** 2 for m in range(1, l + 1)]
            out[b, l] = neumaier_sum(terms) / (2 * l + 1)
    return out[0] if single else out


def synthesize(alm, nside, lmax):
    """Spherical-harmonic synthesis at the pixel centres (Appendix A conventions):
    f(theta, phi) = sum_{l <= lmax, |m| <= l} a_l^m Y_l^m(theta, phi) for a real map,
    i.e. a_l^{-m} = (-1)^m conj(a_l^m), with Re(a_l0) used for m = 0.  Plain sums:
    F_m(theta) = (1/sqrt(2 pi)) sum_l a_l^m Pbar_l^m(cos theta) per ring, then
    f = Re F_0 + 2 Re sum_{m >= 1} F_m e^{i m phi} at every pixel of the ring.
    ``alm`` (n_alm,) or (B, n_alm); returns (N,) or (B, N) float64."""
    a = np.asarray(alm, dtype=np.complex128)
    single = a.ndim == 1
    a = a[None] if single else a
    B = a.shape[0]
    rings = geometry.ring_table(nside)
    th = np.array([r["theta"] for r in rings])
    x, st = np.cos(th), np.sin(th)
    F = np.zeros((B, lmax + 1, len(rings)), dtype=np.complex128)
    for m in range(lmax + 1):
        tab = pbar_table(m, lmax, x, st)                      # (lmax - m + 1, rings)
        i0 = alm_index(m, m, lmax)
        am = a[:, i0:i0 + lmax - m + 1]                       # (B, lmax - m + 1)
        F[:, m, :] = am @ tab / np.sqrt(2.0 * np.pi)
    F[:, 0, :] = F[:, 0, :].real
    out = np.zeros((B, geometry.npix(nside)))
    m = np.arange(lmax + 1)
    wm = np.where(m == 0, 1.0, 2.0)
    for i, r in enumerate(rings):
        phi = r["phi0"] + 2.0 * np.pi * np.arange(r["nphi"]) / r["nphi"]
        E = np.exp(1j * np.outer(m, phi))                     # (lmax + 1, nphi)
        out[:, r["start"]:r["start"] + r["nphi"]] = ((F[:, :, i] * wm) @ E).real
    return out[0] if single else out

