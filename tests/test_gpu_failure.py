"""Failure detection without a GPU fault: a bounded mbarrier wait that nothing
completes gives up after its limit and reports SGB_ERR_TIMEOUT through the
device error word; the context stays usable."""
import time

import numpy as np
import pytest
import torch

from paper_2009_04619_gb300 import seisgb
from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _one_step():
    g = seisgb.make_grid(40, 36, 30, 6, 10.0, 10.0, 10.0, 1e-3, 3000.0)
    rng = np.random.default_rng(5)
    L = seisgb.layout(g)
    f = [torch.from_numpy(rng.standard_normal(int(L.elems)).astype(np.float32)).cuda() for _ in range(2)]
    m = torch.full((int(L.elems),), 0.1, device="cuda")
    phi = torch.zeros(int(L.elems), device="cuda")
    seisgb.stencil_step(g, f[0], f[1], m, phi, 0)
    seisgb.device_status()
    return f[1].cpu().numpy()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    before = _one_step()
    torch.cuda.synchronize()
    t = time.perf_counter()
    status = seisgb.selftest_wait_timeout(50_000)  # 50 ms
    waited = time.perf_counter() - t
    assert status == seisgb.ERR_TIMEOUT
    assert waited >= 0.045
    seisgb.device_status()  # the error word was read and cleared
    after = _one_step()  # same step, same result, after the timeout
    assert np.array_equal(before, after) and np.isfinite(after).all()
