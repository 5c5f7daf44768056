"""GPU: the failure path of the tensor-core kernels' bounded waits -- a wait
that nothing completes gives up after its iteration limit, the context's
error flag reports FVN_ERR_TIMEOUT on the host, and the context keeps
working (no fault, no hang: the wait is bounded and the kernel returns)."""
import time

import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def test_bounded_wait_gives_up_and_the_context_stays_usable(fvn):
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        c.device_status()                                  # nothing recorded yet
        t0 = time.perf_counter()
        c.selftest_wait_timeout(1000)
        with pytest.raises(fvn.FvnError, match="FVN_ERR_TIMEOUT"):
            c.device_status()
        assert time.perf_counter() - t0 < 10.0             # the wait gave up, bounded
        c.device_status()                                  # the flag was cleared
        with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
            c.selftest_wait_timeout(0)
        # the same context still reconstructs correctly
        rng = np.random.default_rng(3)
        sp = np.zeros((5, 48, 64), np.float32)
        m = rng.uniform(size=(48, 64)) < 0.3
        sp[0:4] = rng.uniform(0.1, 0.9, (4, 48, 64)) * m
        sp[4] = m
        y = torch.empty(3, 48, 64, device="cuda")
        c.reconstruct(torch.from_numpy(sp).cuda(), 64, 48, y)
        c.device_status()
        ref = onet.forward(onet.unpack(wl.net_weights(3)), sp)
        assert np.abs(y.cpu().numpy() - ref).max() < 2e-2
    finally:
        c.close()
