"""The HEALPix software's analysis as Sec. 2.2 describes it (test infrastructure;
see package doc): equal-weight quadrature, Eq. (healsph), and its Jacobi
(Richardson) refinement, Eqs. (uzawa) / (richardson).

* ``equal_weight(f, nside, lmax)``: a_l^m = (4 pi / N) sum_i conj(Y_l^m(x_i)) f(x_i)
  for m >= 0 (packed m-major like the rest of the oracle), as a plain double
  sum: per ring the longitude sum sum_k f_k e^{-i m lambda_k} with the angle
  reduced exactly (m k mod nphi), then the latitude sum over the rings with
  Pbar_l^m(cos theta) / sqrt(2 pi) (Appendix A: Y_l^m = Pbar_l^m e^{i m lambda} /
  sqrt(2 pi)).
* ``jacobi(f, nside, lmax, niter)``: a^(0) = A f, then niter times
  r = f - S a, a <- a + A r, with S the synthesis of Eq. (synthesis)
  (``hp2sph.synthesize``) and A = (4 pi / N) S^* the operator above.
"""

import numpy as np

from . import geometry, hp2sph
from .legendre import pbar_table


def equal_weight(f, nside, lmax):
    """Eq. (healsph) for a real map (N,) or maps (B, N): packed a_l^m, m >= 0."""
    f = np.asarray(f, dtype=np.float64)
    single = f.ndim == 1
    f = f[None] if single else f
    B = f.shape[0]
    rings = geometry.ring_table(nside)
    N = geometry.npix(nside)
    m = np.arange(lmax + 1, dtype=np.int64)
    F = np.zeros((B, len(rings), lmax + 1), dtype=np.complex128)   # sum_k f_k e^{-i m lambda_k}
    for i, r in enumerate(rings):
        nphi = r["nphi"]
        k = np.arange(nphi, dtype=np.int64)
        ang = 2.0 * np.pi * np.mod(np.outer(m, k), nphi) / nphi          # m * 2 pi k / nphi, exact reduction
        E = np.exp(-1j * ang) * np.exp(-1j * m * r["phi0"])[:, None]     # e^{-i m (phi0 + 2 pi k / nphi)}
        F[:, i, :] = f[:, r["start"]:r["start"] + nphi] @ E.T
    th = np.array([r["theta"] for r in rings])
    x, st = np.cos(th), np.sin(th)
    out = np.zeros((B, hp2sph.n_alm(lmax)), dtype=np.complex128)
    for mm in range(lmax + 1):
        tab = pbar_table(mm, lmax, x, st)                                # (lmax - mm + 1, rings)
        i0 = hp2sph.alm_index(mm, mm, lmax)
        out[:, i0:i0 + lmax - mm + 1] = (F[:, :, mm] @ tab.T) / np.sqrt(2.0 * np.pi)
    out *= 4.0 * np.pi / N
    return out[0] if single else out


def jacobi(f, nside, lmax, niter=3):
    """Eqs. (uzawa): a^(0) = A f; r^(k+1) = f - S a^(k); a^(k+1) = a^(k) + A r^(k+1)."""
    f = np.asarray(f, dtype=np.float64)
    a = equal_weight(f, nside, lmax)
    for _ in range(int(niter)):
        r = f - hp2sph.synthesize(a, nside, lmax)
        a = a + equal_weight(r, nside, lmax)
    return a
