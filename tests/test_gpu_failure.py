"""Failure detection on the GPU without a fault: a bounded device wait that
runs out is reported through the status word and the context stays usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_11617_gb300 import simplex as sx

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_is_reported():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    assert sx.simplex_device_status() == 0
    sx.simplex_selftest_wait_timeout(2_000_000)      # 2 ms; nothing completes the barrier
    torch.cuda.synchronize()
    st = sx.simplex_device_status()
    assert st != 0
    assert "bounded wait" in sx.simplex_last_error()
    assert sx.simplex_device_status() == 0           # read-and-clear
    # the context is still usable
    mp = sx.simplex_map_create(2, 63, 2, 2, 16)
    out = torch.zeros(mp.numel, dtype=torch.int32, device="cuda")
    sx.simplex_write(mp, out, 5)
    np.testing.assert_array_equal(out.view(mp.shape).cpu().numpy().view(np.uint32), oracle.write(2, 63, 5))


def test_selftest_rejects_out_of_range_limits():
    with pytest.raises(sx.SimplexError):
        sx.simplex_selftest_wait_timeout(10)
    with pytest.raises(sx.SimplexError):
        sx.simplex_selftest_wait_timeout(10 ** 12)
