"""The failure path without a GPU fault: a device-side wait that nothing
completes gives up after a bounded number of polls, records HPX_ERR_TIMEOUT in
the plan's status word, and hpx_sync reports it once; the context stays usable."""

import numpy as np
import pytest

import skies
from oracle import hp2sph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HPX_ERR_TIMEOUT = -6


@pytest.fixture(scope="module")
def hp():
    import os
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    assert torch.cuda.is_available()
    return hp


@pytest.mark.parametrize("uneven", [False, True], ids=["uniform", "group"])
def test_timeout_is_reported_and_cleared(hp, uneven):
    plan = hp.Plan(nsides=[8, 16, 8]) if uneven else hp.Plan(16, -1, 2, "fp32")
    L = hp.lib()
    assert L.hpx_sync(plan.handle) == 0
    assert hp.hpx_selftest_timeout(plan.handle, 1000) == 0
    assert L.hpx_sync(plan.handle) == HPX_ERR_TIMEOUT
    assert L.hpx_last_error() == HPX_ERR_TIMEOUT
    assert L.hpx_sync(plan.handle) == 0                 # reported once, then cleared
    # the context and the plan still work
    if not uneven:
        maps, _ = skies.small_powerlaw_maps(16, 2, seed=3)
        a = plan.analyze(torch.as_tensor(maps.astype(np.float32), device="cuda"))
        plan.sync()
        ref = hp2sph.analyze(maps.astype(np.float32).astype(np.float64), 16, 32)
        assert np.max(np.abs(a.cpu().numpy() - ref)) < 1e-4 * np.max(np.abs(ref))


def test_selftest_rejects_bad_arguments(hp):
    plan = hp.Plan(8, -1, 1, "fp32")
    assert hp.hpx_selftest_timeout(plan.handle, 0) == -1
    assert hp.hpx_selftest_timeout(plan.handle, (1 << 20) + 1) == -1
    assert hp.hpx_selftest_timeout(None, 10) == -1
