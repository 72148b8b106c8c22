"""The allocation-free entry point hpx_analyze_noalloc, called through the C ABI,
against the plan-based hpx_analyze.

It exists for callers that may not call cudaMalloc (inside someone else's
stream capture, in a process whose device memory belongs to a host pool, in
real-time code that must not allocate after start-up): all its tables and
buffers live in one fixed array inside the library.  This file runs last so that
a failure here leaves every other test already run; it passes alone in a fresh
process and after the other tests."""

import ctypes
import os

import numpy as np
import pytest

import skies
from helpers import per_l_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def hp():
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    assert torch.cuda.is_available()
    return hp


def _reference(hp, maps, nside, lmax):
    plan = hp.Plan(nside, lmax, 1, "fp32")
    out = plan.analyze(torch.as_tensor(maps[None], device="cuda"))
    plan.sync()
    plan.close()
    return out[0].cpu().numpy()


def _noalloc(hp, maps, nside, lmax):
    L = 2 * nside if lmax < 0 else lmax
    x = torch.as_tensor(maps, device="cuda")
    alm = torch.zeros((L + 1) * (L + 2) // 2, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = hp.hpx_analyze_noalloc(nside, lmax, x.data_ptr(), alm.data_ptr(), stream)
    assert rc == hp.HPX_OK, hp.strerror(rc)
    torch.cuda.synchronize()
    return alm.cpu().numpy()


def test_noalloc_matches_plan_two_calls_in_a_row(hp):
    # pairs of consecutive calls of one size, up to the largest size the array takes
    calls = [(16, -1, 1), (16, -1, 2), (64, 100, 3), (64, 100, 4), (128, -1, 5), (128, -1, 6),
             (128, 200, 7), (128, 200, 8)]
    for nside, lmax, seed in calls:
        maps, _ = skies.small_powerlaw_maps(nside, 1, seed=seed, alpha=2.0, noise=1e-3)
        m32 = maps[0].astype(np.float32)
        L = 2 * nside if lmax < 0 else lmax
        got = _noalloc(hp, m32, nside, lmax)
        ref = _reference(hp, m32, nside, lmax)
        e = per_l_error(got, ref, L)
        assert e.max() < TOL_FP32, (nside, lmax, e.max())


def test_noalloc_rejects_sizes_beyond_its_array(hp):
    x = torch.zeros(12 * 256 * 256, dtype=torch.float32, device="cuda")
    a = torch.zeros(10, dtype=torch.complex64, device="cuda")
    rc = hp.hpx_analyze_noalloc(256, -1, x.data_ptr(), a.data_ptr(), None)
    assert rc == hp.HPX_ERR_NSIDE
    rc = hp.hpx_analyze_noalloc(16, 40, x.data_ptr(), a.data_ptr(), None)
    assert rc == hp.HPX_ERR_LMAX
