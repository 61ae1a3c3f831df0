"""A bounded device wait that expires (a flag that nothing sets): the kernel records the timeout
and returns, the host reads AFQMC_ERR_TIMEOUT, and the process keeps using the GPU.  No trap and
no fault is involved.  This file sorts last so that the rest of the GPU suite has run before it."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")
torch = pytest.importorskip("torch")

AFQMC_ERR_TIMEOUT = -5


def test_an_expired_wait_reports_timeout_and_the_context_stays_usable():
    u0 = afqmc.afqmc_debug_uniforms(7, 0, 1, 64)
    t0 = time.perf_counter()
    rc = afqmc.afqmc_debug_wait_timeout(50_000_000, torch.cuda.current_stream())  # 50 ms
    dt = time.perf_counter() - t0
    assert rc == AFQMC_ERR_TIMEOUT
    assert 0.045 <= dt < 2.0
    # the same device generator output, and plain torch work, after the expired wait
    np.testing.assert_array_equal(afqmc.afqmc_debug_uniforms(7, 0, 1, 64), u0)
    x = torch.arange(1024, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 1023 * 1024 / 2
