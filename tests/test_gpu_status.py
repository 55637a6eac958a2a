"""Device-side error reporting without faulting the GPU.

A test hook makes one tile of the first partition pass skip publishing its
look-back counts; its successors wait for it with a short time limit (1 ms),
give up, record BINAR_ERR_DEVICE_TIMEOUT in the workspace status word and
finish.  The status is read on the host, and the next call on the same
stream and workspace succeeds.
"""
import numpy as np
import pytest

from gpu_util import expect_pairs, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def test_lookback_timeout_is_reported_and_recoverable():
    n = 8192 * 40
    keys = inputs.uniform_keys(n, np.uint32, np.random.Generator(np.random.PCG64(9)))
    vals = inputs.index_payload(n)
    tk, tv = to_dev(keys), to_dev(vals)
    ws = binding.workspace(n, 4, 4)
    cfg = {"debug_skip_publish_tile": 3, "lookback_timeout_ns": 1_000_000}
    binding.sort_pairs(tk, tv, ws=ws, config=cfg)
    assert binding.workspace_status(ws) == binding.ERR_DEVICE_TIMEOUT
    # the same workspace and stream work again
    tk.copy_(to_dev(keys))
    tv.copy_(to_dev(vals))
    binding.sort_pairs(tk, tv, ws=ws)
    assert binding.workspace_status(ws) == binding.OK
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)


def test_status_is_clear_after_a_good_call():
    n = 50_000
    keys = to_dev(inputs.uniform_keys(n, np.uint64, np.random.Generator(np.random.PCG64(1))))
    ws = binding.workspace(n, 8, 0)
    binding.sort_keys(keys, ws=ws)
    assert binding.workspace_status(ws) == binding.OK
