"""GPU: batches of independent circuits (one persistent launch per wave of tile passes,
replayed from a captured CUDA graph) give each circuit bitwise the amplitudes of a solo
qs_execute with the same options, and match the FP64 oracle within the stated tolerance."""
import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
torch = pytest.importorskip("torch")

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_matches_solo_and_oracle(dtype):
    work = wc.batched_workload(24, seed=7, nmin=6, nmax=15, dmin=2, dmax=12)
    stream = torch.cuda.Stream()
    b = qs.Batch(work, dtype=dtype, stream=stream)
    st = b.stats()
    assert st["n_circuits"] == 24 and st["n_waves"] >= 1
    for run in range(3):      # eager, capture, replay
        b.run()
        b.sync()
        norms = b.norms()
        assert np.all(np.abs(norms - 1.0) < (1e-12 if dtype == "c128" else 1e-5))
        for i, (n, circ) in enumerate(work):
            got = b.amplitudes(i)
            solo = qs.State(n, dtype)
            solo.execute(qs.compile(n, circ, mode="tile", dtype=dtype))
            ref = solo.amplitudes(order=qs.QS_ORDER_STORAGE)
            assert got.tobytes() == ref.tobytes(), f"circuit {i} (n={n}) differs from its solo run"
            if run == 0:
                err = np.abs(got.astype(np.complex128) - sv.simulate(n, circ)).max()
                assert err <= TOL[dtype]


def test_batch_config4_shapes():
    """The batched workload's shapes (n in 10..20, depth 10..60), fewer circuits."""
    work = wc.batched_workload(64, seed=0)
    b = qs.Batch(work, dtype="c64", stream=torch.cuda.Stream())
    b.run()
    b.sync()
    assert np.all(np.abs(b.norms() - 1.0) < 1e-5)
    for i in (0, 17, 63):
        n, circ = work[i]
        if n <= 18:
            err = np.abs(b.amplitudes(i).astype(np.complex128) - sv.simulate(n, circ)).max()
            assert err <= TOL["c64"]


def test_batch_rejects_bad_input():
    with pytest.raises(qs.QSError):
        qs.Batch([(31, [])], dtype="c64")
    with pytest.raises(qs.QSError):
        qs.Batch([(4, [wc.Gate("H", (5,))])], dtype="c64")
