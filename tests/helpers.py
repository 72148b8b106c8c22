"""Shared test helpers: the per-degree error measure used by every parity test.

e_l = ||a_l - a^o_l||_2 / ||a^o_l||_2 over m >= 0 with weight 2 for m > 0 (the
l2 norm over all m = -l..l for a real map).  Degrees l < 2, which carry no
input power in the seeded skies (C_0 = C_1 = 0), and any degree whose reference
norm is below `floor` times the largest one, are measured in absolute terms
against the total reference norm instead."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def alm_index(l, m, lmax):
    return m * (2 * lmax + 1 - m) // 2 + l


def per_l_norms(a, lmax):
    a = np.asarray(a)
    out = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        i0 = alm_index(m, m, lmax)
        seg = np.abs(a[i0:i0 + lmax - m + 1]) ** 2 * (1.0 if m == 0 else 2.0)
        out[m:] += seg
    return np.sqrt(out)


def per_l_error(a, ref, lmax, floor=1e-6):
    """e_l for one map (vectors of packed m >= 0 coefficients)."""
    d = per_l_norms(np.asarray(a) - np.asarray(ref), lmax)
    r = per_l_norms(ref, lmax)
    tot = np.sqrt(np.sum(r ** 2))
    small = (r < floor * r.max()) | (np.arange(lmax + 1) < 2)
    e = np.where(small, d / tot, d / np.where(small, 1.0, r))
    return e


def sampled_per_l_errors(cols_gpu, cols_ref, ref_norm_l, lmax):
    """Estimate of e_l from a sample of orders: cols_* = {m: (lmax-m+1,)},
    ref_norm_l = ||a_l|| of the input sky (from the seeded generator).
    Returns sqrt(mean_m |da_lm|^2 * (2l+1)) / ref_norm_l per degree (0 where no
    sampled order reaches l or the sky has no power there)."""
    out = np.zeros(lmax + 1)
    for l in range(lmax + 1):
        if ref_norm_l[l] <= 0:
            continue
        ds = [abs(cols_gpu[m][l - m] - cols_ref[m][l - m]) ** 2 for m in cols_ref if m <= l]
        if not ds:
            continue
        out[l] = np.sqrt(np.mean(ds) * (2 * l + 1)) / ref_norm_l[l]
    return out


def sampled_per_l_error(cols_gpu, cols_ref, ref_norm_l, lmax):
    """The largest per-degree estimate of sampled_per_l_errors."""
    return float(sampled_per_l_errors(cols_gpu, cols_ref, ref_norm_l, lmax).max())


def ring_perm(nside, quarter):
    """Pixel permutation of a quarter turn (lambda -> lambda + pi/2: every ring
    shifts by nphi/4 pixels) or of the north-south mirror."""
    from oracle import geometry
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
