"""GPU: the bounded-wait path of the kernels.  A kernel waits on an mbarrier that nothing
arrives on; it must give up after its limit and report QS_ETIMEOUT, and the CUDA context must
stay usable (a following circuit still matches the oracle)."""
import time

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
from paper_2010_09746_gb300 import _lib  # noqa: E402


def test_wait_expires_and_context_survives():
    for limit_us in (1000, 20000):
        t0 = time.perf_counter()
        status = qs.selftest_bounded_wait(limit_us)
        dt = time.perf_counter() - t0
        assert status == _lib.QS_ETIMEOUT
        assert dt < 2.0
    n = 12
    circ = wc.rzrx_cz_circuit(n, 4, seed=1)
    st = qs.State(n, "c128")
    st.run(circ)
    assert np.max(np.abs(st.amplitudes() - sv.simulate(n, circ))) <= 1e-12


def test_selftest_rejects_bad_limits():
    with pytest.raises(qs.QSError):
        qs.selftest_bounded_wait(0)
