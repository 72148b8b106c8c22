"""GB300 (sm_103a) HP2SPH: spherical-harmonic analysis of real HEALPix maps.

A thin ctypes binding over the C ABI of ``libhpx.so`` (declared in
include/hpx.h).  The functions keep the C names; they only marshal arguments
(device pointers of torch tensors, the current CUDA stream).  Every step of the
method runs in the library's CUDA kernels; there is no fallback: if the library
is missing, importing the binding's functions raises.

    import torch, paper_1904_10514_gb300 as hp
    plan = hp.Plan(nside=1024, batch=32)                 # FP32, lmax = 2 nside
    alm = plan.analyze(maps)                             # (32, n_alm) complex64
    cl = plan.cl(alm)                                    # (32, lmax+1) float64
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpx.so")

HPX_OK = 0
HPX_ERR_ARG = -1
HPX_ERR_NSIDE = -2
HPX_ERR_LMAX = -3
HPX_ERR_CUDA = -4
HPX_ERR_OOM = -5
HPX_ERR_TIMEOUT = -6
HPX_ERR_STATE = -7
HPX_FP32 = 0
HPX_FP64 = 1

EXPORTS = ["hpx_plan", "hpx_plan_ex", "hpx_set_stream", "hpx_analyze", "hpx_synthesize", "hpx_cl",
           "hpx_sync", "hpx_destroy", "hpx_npix", "hpx_nalm", "hpx_plan_lmax", "hpx_plan_bytes",
           "hpx_last_error", "hpx_strerror", "hpx_set_profiling", "hpx_stage_times",
           "hpx_analyze_noalloc", "hpx_plan_flags", "hpx_selftest_timeout", "hpx_sh_synthesis", "hpx_plan_launches",
           "hpx_analyze_vjp", "hpx_cl_vjp", "hpx_sh_synthesis_adjoint", "hpx_healpix_analysis", "hpx_plan_tuning",
           "hpx_plan_set_tuning"]
HPX_FLAG_SWEEPS = 1
HPX_FLAG_GRAPH = 2
HPX_FLAG_SIMT = 4
HPX_FLAG_CHECKED = 8
HPX_FLAG_AUTOTUNE = 16
HPX_FLAG_SYNTHESIS = 32
HPX_FLAG_CG = 64
HPX_FLAG_JACOBI = 128
HPX_ERR_NONFINITE = -8
HPX_NOALLOC_MAX_NSIDE = 128
HPX_NSTAGES = 6
def stage_names(flags):
    """Names of the HPX_NSTAGES profiled stages of hpx_analyze for a plan's flags."""
    sweeps = bool(flags & HPX_FLAG_SWEEPS)
    return ["ring_fft", "poles", "spread", "lat_fft",
            "lat_solve" if sweeps else "fused_fsht", "rot_sweep" if sweeps else "unused"]


STAGES = stage_names(HPX_FLAG_SWEEPS)   # HPX_FLAG_SWEEPS plans
STAGES_FUSED = stage_names(0)          # per-order operators
STAGES_SYNTH = ["synth_fsht", "synth_nufft", "synth_rings", "unused", "unused", "unused"]   # hpx_sh_synthesis


class hpx_plan_desc(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int), ("lmax", ctypes.c_int), ("batch", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint),
                ("nsides", ctypes.POINTER(ctypes.c_int)), ("lmaxs", ctypes.POINTER(ctypes.c_int))]


class HpxError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))


_lib = None


def build():
    """Compile libhpx.so in-tree for sm_103a."""
    from . import nvcc_build as _b
    return _b.build()


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhpx.so is not built (run paper_1904_10514_gb300.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "hpx_plan": (vp, [i32, i32, i32]),
            "hpx_plan_ex": (vp, [ctypes.POINTER(hpx_plan_desc)]),
            "hpx_set_stream": (i32, [vp, vp]),
            "hpx_analyze": (i32, [vp, vp, vp]),
            "hpx_synthesize": (i32, [vp, vp, vp]),
            "hpx_cl": (i32, [vp, vp, vp]),
            "hpx_sync": (i32, [vp]),
            "hpx_destroy": (None, [vp]),
            "hpx_npix": (i64, [vp]),
            "hpx_nalm": (i64, [vp]),
            "hpx_plan_lmax": (i32, [vp]),
            "hpx_plan_bytes": (i64, [vp]),
            "hpx_plan_flags": (i32, [vp]),
            "hpx_last_error": (i32, []),
            "hpx_strerror": (ctypes.c_char_p, [i32]),
            "hpx_set_profiling": (i32, [vp, i32]),
            "hpx_analyze_noalloc": (i32, [i32, i32, vp, vp, vp]),
            "hpx_selftest_timeout": (i32, [vp, i32]),
            "hpx_sh_synthesis": (i32, [vp, vp, vp]),
            "hpx_plan_launches": (i32, [vp]),
            "hpx_analyze_vjp": (i32, [vp, vp, vp]),
            "hpx_sh_synthesis_adjoint": (i32, [vp, vp, vp]),
            "hpx_healpix_analysis": (i32, [vp, vp, vp, i32]),
            "hpx_plan_tuning": (i32, [vp] + [ctypes.POINTER(ctypes.c_int)] * 5),
            "hpx_plan_set_tuning": (i32, [vp, i32, i32, i32, i32, i32]),
            "hpx_cl_vjp": (i32, [vp, vp, vp, vp]),
            "hpx_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(ctypes.c_int)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().hpx_strerror(int(code)).decode()


# ------------------------------------------------------------ C names
def hpx_plan(nside, lmax, batch):
    return lib().hpx_plan(int(nside), int(lmax), int(batch))


def hpx_plan_ex(nside, lmax=-1, batch=1, precision=HPX_FP32, flags=0, nsides=None, lmaxs=None):
    def arr(v):
        return (ctypes.c_int * len(v))(*[int(x) for x in v]) if v is not None else None
    ns_arr, l_arr = arr(nsides), arr(lmaxs)
    if nsides is not None:
        batch = len(nsides)
    elif lmaxs is not None:
        batch = len(lmaxs)
    ptr = ctypes.POINTER(ctypes.c_int)
    d = hpx_plan_desc(int(nside), int(lmax), int(batch), int(precision), int(flags),
                      ctypes.cast(ns_arr, ptr) if ns_arr is not None else None,
                      ctypes.cast(l_arr, ptr) if l_arr is not None else None)
    return lib().hpx_plan_ex(ctypes.byref(d))


def hpx_selftest_timeout(plan, spins):
    return lib().hpx_selftest_timeout(plan, int(spins))


def hpx_set_stream(plan, stream):
    return lib().hpx_set_stream(plan, stream)


def hpx_analyze(plan, maps_ptr, alm_ptr):
    return lib().hpx_analyze(plan, maps_ptr, alm_ptr)


def hpx_synthesize(plan, alm_ptr, maps_ptr):
    return lib().hpx_synthesize(plan, alm_ptr, maps_ptr)


def hpx_cl(plan, alm_ptr, cl_ptr):
    return lib().hpx_cl(plan, alm_ptr, cl_ptr)


def hpx_sync(plan):
    return lib().hpx_sync(plan)


def hpx_analyze_vjp(plan, galm_ptr, gmaps_ptr):
    return lib().hpx_analyze_vjp(plan, galm_ptr, gmaps_ptr)


def hpx_cl_vjp(plan, alm_ptr, gcl_ptr, galm_ptr):
    return lib().hpx_cl_vjp(plan, alm_ptr, gcl_ptr, galm_ptr)


def hpx_destroy(plan):
    lib().hpx_destroy(plan)


def hpx_analyze_noalloc(nside, lmax, maps_ptr, alm_ptr, stream):
    """Allocation-free one-map FP32 analysis (see include/hpx.h)."""
    return lib().hpx_analyze_noalloc(int(nside), int(lmax), maps_ptr, alm_ptr, stream)


def hpx_set_profiling(plan, enable):
    return lib().hpx_set_profiling(plan, int(enable))


def hpx_stage_times(plan):
    """(summed ms per stage, number of calls) since the last read."""
    ms = (ctypes.c_float * HPX_NSTAGES)()
    nc = ctypes.c_int(0)
    rc = lib().hpx_stage_times(plan, ms, HPX_NSTAGES, ctypes.byref(nc))
    if rc != HPX_OK:
        raise HpxError(rc, "hpx_stage_times")
    return [float(v) for v in ms], nc.value


def hpx_last_error():
    return lib().hpx_last_error()


def n_alm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


# ------------------------------------------------------------ torch wrapper
class Plan:
    """Owns one C plan; tensors must live on the plan's CUDA device."""

    def __init__(self, nside=None, lmax=-1, batch=1, precision="fp32", sweeps=False, graph=False, nsides=None,
                 simt=False, lmaxs=None, checked=False, autotune=False, synthesis=False, cg=False, jacobi=False):
        """Uniform batch (nside, batch), or uneven batch (nsides = nside of every map
        and/or lmaxs = lmax of every map; maps, alm and C_l are then 1-D tensors
        holding the maps concatenated)."""
        import torch
        self.torch = torch
        self.nsides = None if nsides is None else [int(v) for v in nsides]
        self.lmaxs = None if lmaxs is None else [int(v) for v in lmaxs]
        self.nside = int(nside) if nside is not None else 0
        if self.nsides is not None:
            self.batch = len(self.nsides)
        elif self.lmaxs is not None:
            self.batch = len(self.lmaxs)
        else:
            self.batch = int(batch)
        self.concat = self.nsides is not None or self.lmaxs is not None
        self.precision = HPX_FP64 if precision in ("fp64", "float64", HPX_FP64) else HPX_FP32
        self.device = torch.device("cuda", torch.cuda.current_device())
        flags = ((HPX_FLAG_SWEEPS if sweeps else 0) | (HPX_FLAG_GRAPH if graph else 0) |
                 (HPX_FLAG_SIMT if simt else 0) | (HPX_FLAG_CHECKED if checked else 0) |
                 (HPX_FLAG_AUTOTUNE if autotune else 0) | (HPX_FLAG_SYNTHESIS if synthesis else 0) |
                 (HPX_FLAG_CG if cg else 0) | (HPX_FLAG_JACOBI if jacobi else 0))
        h = hpx_plan_ex(self.nside, lmax, self.batch, self.precision, flags, self.nsides, self.lmaxs)
        if not h:
            raise HpxError(hpx_last_error(), "hpx_plan_ex")
        self.handle = h
        self._lmax_arg = int(lmax)
        self.lmax = lib().hpx_plan_lmax(h)
        self.flags = lib().hpx_plan_flags(h)
        self.stages = stage_names(self.flags)
        self.npix = lib().hpx_npix(h)
        self.nalm = lib().hpx_nalm(h)
        self.rdtype = torch.float64 if self.precision == HPX_FP64 else torch.float32
        self.cdtype = torch.complex128 if self.precision == HPX_FP64 else torch.complex64

    @property
    def tuning(self):
        """(ring-FFT elements per thread, grid-FFT elements per thread, sweep form,
        separate packing pass of b, Bluestein ring form) in effect (HPX_FLAG_AUTOTUNE)."""
        v = [ctypes.c_int(0) for _ in range(5)]
        self._check(lib().hpx_plan_tuning(self.handle, *[ctypes.byref(x) for x in v]), "hpx_plan_tuning")
        return tuple(x.value for x in v)

    @tuning.setter
    def tuning(self, shapes):
        self._check(lib().hpx_plan_set_tuning(self.handle, *[int(x) for x in shapes]), "hpx_plan_set_tuning")

    @property
    def nbytes(self):
        return lib().hpx_plan_bytes(self.handle)

    def _stream(self):
        hpx_set_stream(self.handle, self.torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, rc, what):
        if rc != HPX_OK:
            raise HpxError(rc, what)

    def _shape(self, n):
        return (n,) if self.concat else (self.batch, n)

    def _maps(self, maps):
        shape = self._shape(self.npix)
        if maps.dtype != self.rdtype or maps.device.type != "cuda" or tuple(maps.shape) != shape:
            raise ValueError("maps must be a CUDA %s tensor of shape %s" % (self.rdtype, shape))
        return maps.contiguous()

    def map_lmax(self, i):
        """lmax of map i."""
        ns = self.nsides[i] if self.nsides is not None else self.nside
        lm = self.lmaxs[i] if self.lmaxs is not None else self._lmax_arg
        return 2 * ns if lm < 0 else lm

    @property
    def ncl(self):
        if not self.concat:
            return self.lmax + 1
        return sum(self.map_lmax(i) + 1 for i in range(self.batch))

    def analyze(self, maps, out=None):
        """maps (batch, npix) -> alm (batch, n_alm) complex, m-major packing."""
        maps = self._maps(maps)
        if out is None:
            out = self.torch.empty(self._shape(self.nalm), dtype=self.cdtype, device=maps.device)
        self._stream()
        self._check(hpx_analyze(self.handle, maps.data_ptr(), out.data_ptr()), "hpx_analyze")
        return out

    def synthesize(self, alm, out=None):
        """Exact adjoint of analyze: alm (batch, n_alm) complex -> maps (batch, npix)."""
        alm = alm.contiguous()
        if out is None:
            out = self.torch.empty(self._shape(self.npix), dtype=self.rdtype, device=alm.device)
        self._stream()
        self._check(hpx_synthesize(self.handle, alm.data_ptr(), out.data_ptr()), "hpx_synthesize")
        return out

    def analyze_vjp(self, galm, out=None):
        """dL/dmaps from galm = dL/dRe(alm) + i dL/dIm(alm) (hpx_analyze_vjp)."""
        galm = galm.contiguous()
        if out is None:
            out = self.torch.empty(self._shape(self.npix), dtype=self.rdtype, device=galm.device)
        self._stream()
        self._check(hpx_analyze_vjp(self.handle, galm.data_ptr(), out.data_ptr()), "hpx_analyze_vjp")
        return out

    def cl_vjp(self, alm, gcl, out=None):
        """dL/dalm from gcl = dL/dC_l and the coefficients (hpx_cl_vjp)."""
        alm = alm.contiguous()
        gcl = gcl.to(self.torch.float64).contiguous()
        if out is None:
            out = self.torch.empty_like(alm)
        self._stream()
        self._check(hpx_cl_vjp(self.handle, alm.data_ptr(), gcl.data_ptr(), out.data_ptr()), "hpx_cl_vjp")
        return out

    def sh_synthesis(self, alm, out=None):
        """Spherical-harmonic synthesis f = sum a_lm Y_lm at the pixel centres
        (plan made with synthesis=True): alm (batch, n_alm) -> maps (batch, npix)."""
        alm = alm.contiguous()
        if out is None:
            out = self.torch.empty(self._shape(self.npix), dtype=self.rdtype, device=alm.device)
        self._stream()
        self._check(lib().hpx_sh_synthesis(self.handle, alm.data_ptr(), out.data_ptr()), "hpx_sh_synthesis")
        return out

    def sh_synthesis_adjoint(self, maps, out=None):
        """sum_i conj(Y_lm(x_i)) f_i (the transpose of sh_synthesis; plan made with synthesis=True):
        maps (batch, npix) -> alm (batch, n_alm)."""
        maps = self._maps(maps)
        if out is None:
            out = self.torch.empty(self._shape(self.nalm), dtype=self.cdtype, device=maps.device)
        self._stream()
        self._check(lib().hpx_sh_synthesis_adjoint(self.handle, maps.data_ptr(), out.data_ptr()),
                    "hpx_sh_synthesis_adjoint")
        return out

    def healpix_analysis(self, maps, niter=3, out=None):
        """The HEALPix software's analysis (equal weights + niter Jacobi steps; plan made with
        jacobi=True): maps (batch, npix) -> alm (batch, n_alm)."""
        maps = self._maps(maps)
        if out is None:
            out = self.torch.empty(self._shape(self.nalm), dtype=self.cdtype, device=maps.device)
        self._stream()
        self._check(lib().hpx_healpix_analysis(self.handle, maps.data_ptr(), out.data_ptr(), int(niter)),
                    "hpx_healpix_analysis")
        return out

    def cl(self, alm, out=None):
        """C_l (batch, lmax+1) float64 of Eq. (APS)."""
        alm = alm.contiguous()
        if out is None:
            out = self.torch.empty((self.ncl,) if self.concat else (self.batch, self.lmax + 1),
                                   dtype=self.torch.float64, device=alm.device)
        self._stream()
        self._check(hpx_cl(self.handle, alm.data_ptr(), out.data_ptr()), "hpx_cl")
        return out

    def sync(self):
        self._check(hpx_sync(self.handle), "hpx_sync")

    def close(self):
        if getattr(self, "handle", None):
            hpx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ autograd
def _torch_functions():
    import torch

    class AnalyzeFn(torch.autograd.Function):
        """alm = A maps; the backward pass is the library's vector-Jacobian
        product of the analysis (hpx_analyze_vjp)."""

        @staticmethod
        def forward(ctx, maps, plan):
            ctx.plan = plan
            return plan.analyze(maps)

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.analyze_vjp(g), None

    class ClFn(torch.autograd.Function):
        """C_l of Eq. (APS) (hpx_cl); the backward pass is hpx_cl_vjp."""

        @staticmethod
        def forward(ctx, alm, plan):
            ctx.plan = plan
            ctx.save_for_backward(alm)
            return plan.cl(alm)

        @staticmethod
        def backward(ctx, gcl):
            (alm,) = ctx.saved_tensors
            return ctx.plan.cl_vjp(alm, gcl), None

    return AnalyzeFn, ClFn


_FNS = None


def _fns():
    global _FNS
    if _FNS is None:
        _FNS = _torch_functions()
    return _FNS


def analyze(maps, plan):
    """Differentiable analysis (torch.autograd) through the C ABI."""
    return _fns()[0].apply(maps, plan)


def cl(alm, plan):
    """Differentiable C_l (torch.autograd) through the C ABI."""
    return _fns()[1].apply(alm, plan)
