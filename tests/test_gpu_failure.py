"""Failure detection without a GPU fault: a bounded device wait that runs out (an
mbarrier that nothing arrives at, waited on through the tensor-core kernels' own
bounded wait) records its code in the device error word; the host reads it as
DEVICE_TIMEOUT, the read clears it, and the context keeps running work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_stays_usable():
    lib = L.get()
    L.device_error(0)  # start from a clear error word
    assert lib.delimit_selftest_wait_timeout(None) == L.OK
    st, code = L.device_error(0)
    assert st == L.ERR_DEVICE_TIMEOUT and code == 0x7F00
    assert b"timed out" in lib.delimit_last_error()
    st, code = L.device_error(0)  # cleared by the read
    assert st == L.OK and code == 0
    # the same context still runs library work
    dirs, bvals = synth.multishell_table([40], [1000], seed=3)
    basis = L.SHBasis(dirs, bvals, 4, 0.006)
    x = layers.empty_act(40, 256, torch.float32)
    x.copy_(torch.from_numpy(synth.gaussian((40, 256), 1.0, seed=4)).float())
    y = layers.transform("signal2sh", basis, x, 1)
    torch.cuda.synchronize()
    assert y.shape[0] == 15 and np.isfinite(y.float().cpu().numpy()).all()
    st, code = L.device_error(0)
    assert st == L.OK and code == 0
