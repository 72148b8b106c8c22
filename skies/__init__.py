"""Seeded synthetic HEALPix skies: the only module that both the CUDA path's tests
and the oracle consume.  It holds none of the analysis method's arithmetic.

Skies are Gaussian random fields with a chosen angular power spectrum C_l:
a_l0 ~ N(0, C_l) (real), and for m > 0 Re a_lm, Im a_lm ~ N(0, C_l / 2), drawn
from numpy's PCG64 with the seed 1000 * workload + map index.  Maps are the
spherical-harmonic synthesis f_i = sum_lm a_lm Y_l^m(x_i) (Eq. synthesis) at the
HEALPix pixel centres in RING order, evaluated in float64 by a small C helper
(``synth.c``) plus numpy FFTs along each ring.  The C helper is compiled with
gcc on first use (or by ``build()``).

Workloads (stand-ins for the paper's CMB maps, whose data are not available):
  1  Nside 16, lmax 32, 1 map, C_l = 1/(l(l+1)) for l >= 2
  2  Nside 256, lmax 512, 1 map, C_l = l^-2 exp(-(l/400)^2) for l >= 2
  3  Nside 512, lmax 1024, 64 maps, C_l = l^-alpha (alpha ~ U[1.5, 2.5] per map),
     plus N(0, 1e-3) white pixel noise
  4  200 maps, Nside drawn from {64,128,256,512,1024} w.p. .40/.30/.15/.10/.05,
     lmax = 2 Nside, the generator of workload 3
  5  Nside 2048, lmax 4096, 8 maps, the generator of workload 3
  bench  Nside 1024, lmax 2048, 32 maps, the generator of workload 3
C_0 = C_1 = 0 everywhere.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_skies.so")
_SRC = os.path.join(_HERE, "synth.c")
_lock = threading.Lock()
_lib = None


def build():
    """Compile the synthesis helper (gcc, OpenMP)."""
    cmd = ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-o", _SO, _SRC, "-lm"]
    subprocess.run(cmd, check=True)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
                build()
            lib = ctypes.CDLL(_SO)
            lib.skies_profiles.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
            lib.skies_profiles.restype = None
            _lib = lib
    return _lib


def n_alm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(l, m, lmax):
    return m * (2 * lmax + 1 - m) // 2 + l


# ----------------------------------------------------------------- geometry
def _rings(nside):
    """(theta, nphi, phi0, start) per ring, north to south (HEALPix RING order)."""
    ns = int(nside)
    out = []
    start = 0
    for j in range(1, 4 * ns):
        if j < ns:
            th = 2.0 * np.arcsin(j / (np.sqrt(6.0) * ns)); nphi = 4 * j; sh = True
        elif j <= 3 * ns:
            th = np.arccos(2.0 * (2 * ns - j) / (3.0 * ns)); nphi = 4 * ns; sh = (j % 2) == 0
        else:
            jj = 4 * ns - j
            th = np.pi - 2.0 * np.arcsin(jj / (np.sqrt(6.0) * ns)); nphi = 4 * jj; sh = True
        out.append((th, nphi, (np.pi / nphi) if sh else 0.0, start))
        start += nphi
    return out


# ------------------------------------------------------------------ spectra
def power_law(lmax, alpha):
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    cl[2:] = l ** (-float(alpha))
    return cl


def cl_workload1(lmax):
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    cl[2:] = 1.0 / (l * (l + 1.0))
    return cl


def cl_workload2(lmax):
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    cl[2:] = l ** -2.0 * np.exp(-(l / 400.0) ** 2)
    return cl


def gaussian_alm(cl, lmax, rng):
    """Packed complex a_lm (m >= 0) with <|a_lm|^2> = C_l and real a_l0."""
    a = np.zeros(n_alm(lmax), dtype=np.complex128)
    sd = np.sqrt(cl[:lmax + 1])
    for m in range(lmax + 1):
        i0 = alm_index(m, m, lmax)
        s = sd[m:]
        if m == 0:
            a[i0:i0 + lmax + 1] = s * rng.standard_normal(lmax + 1)
        else:
            n = lmax - m + 1
            a[i0:i0 + n] = s * np.sqrt(0.5) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    return a


# ---------------------------------------------------------------- synthesis
def synthesize(alm, nside, lmax):
    """Real map(s) f = sum a_lm Y_l^m at the pixel centres, float64, RING order.
    ``alm`` is (n_alm,) or (B, n_alm) packed m >= 0."""
    alm = np.asarray(alm, dtype=np.complex128)
    single = alm.ndim == 1
    alm = alm[None] if single else alm
    B = alm.shape[0]
    ns = int(nside)
    rings = _rings(ns)
    R = len(rings)
    half = 2 * ns                               # north rings incl. the equator
    x = np.ascontiguousarray([np.cos(rings[i][0]) for i in range(half)], dtype=np.float64)
    x[-1] = 0.0
    a_t = np.ascontiguousarray(np.stack([alm.real.T, alm.imag.T], axis=-1))   # (n_alm, B, 2)
    fn = np.zeros((B, half, lmax + 1, 2))
    fs = np.zeros((B, half, lmax + 1, 2))
    _load().skies_profiles(int(lmax), half, x.ctypes.data, B, a_t.ctypes.data,
                           fn.ctypes.data, fs.ctypes.data)
    Fn = fn[..., 0] + 1j * fn[..., 1]
    Fs = fs[..., 0] + 1j * fs[..., 1]
    out = np.zeros((B, 12 * ns * ns))
    m = np.arange(lmax + 1)
    wm = np.where(m == 0, 1.0, 2.0)
    for i, (th, nphi, phi0, start) in enumerate(rings):
        F = Fn[:, i] if i < half else Fs[:, R - 1 - i]
        g = np.zeros((B, nphi), dtype=np.complex128)
        np.add.at(g, (slice(None), m % nphi), F * (wm * np.exp(1j * m * phi0))[None, :])
        out[:, start:start + nphi] = np.real(np.fft.ifft(g, axis=1)) * nphi
    return out[0] if single else out


# ---------------------------------------------------------------- workloads
def workload_maps(workload, nmaps=None, dtype=np.float64, return_alm=False, first=0):
    """Seeded maps of a named workload (see module doc).  Returns maps (B, N)
    [and their a_lm].  ``first``/``nmaps`` select a contiguous subset of maps."""
    spec = WORKLOADS[workload]
    ns, lmax = spec["nside"], spec["lmax"]
    n = spec["nmaps"] if nmaps is None else int(nmaps)
    alms = []
    noise = []
    for b in range(first, first + n):
        rng = np.random.Generator(np.random.PCG64(1000 * spec["id"] + b))
        if spec["spectrum"] == "w1":
            cl = cl_workload1(lmax)
        elif spec["spectrum"] == "w2":
            cl = cl_workload2(lmax)
        else:
            cl = power_law(lmax, rng.uniform(1.5, 2.5))
        alms.append(gaussian_alm(cl, lmax, rng))
        noise.append(spec["noise"] * rng.standard_normal(12 * ns * ns) if spec["noise"] else None)
    alms = np.stack(alms)
    maps = synthesize(alms, ns, lmax)
    for b in range(n):
        if noise[b] is not None:
            maps[b] += noise[b]
    maps = maps.astype(dtype)
    return (maps, alms) if return_alm else maps


def uneven_nsides(count=200, seed=4000):
    """Nside of each map of workload 4, drawn with the stated probabilities."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice([64, 128, 256, 512, 1024], size=count, p=[0.40, 0.30, 0.15, 0.10, 0.05])


WORKLOADS = {
    "w1_nside16": dict(id=1, nside=16, lmax=32, nmaps=1, spectrum="w1", noise=0.0),
    "w2_nside256": dict(id=2, nside=256, lmax=512, nmaps=1, spectrum="w2", noise=0.0),
    "w3_nside512x64": dict(id=3, nside=512, lmax=1024, nmaps=64, spectrum="powerlaw", noise=1e-3),
    "w5_nside2048x8": dict(id=5, nside=2048, lmax=4096, nmaps=8, spectrum="powerlaw", noise=1e-3),
    "bench_nside1024x32": dict(id=6, nside=1024, lmax=2048, nmaps=32, spectrum="powerlaw", noise=1e-3),
}


def small_powerlaw_maps(nside, nmaps, seed, alpha=2.0, noise=0.0, lmax=None):
    """Power-law skies at any Nside for parity tests (seed given explicitly)."""
    lmax = 2 * nside if lmax is None else lmax
    rng = np.random.Generator(np.random.PCG64(seed))
    alms = np.stack([gaussian_alm(power_law(lmax, alpha), lmax, rng) for _ in range(nmaps)])
    maps = synthesize(alms, nside, lmax)
    if noise:
        maps = maps + noise * rng.standard_normal(maps.shape)
    return maps, alms
