"""GPU: the continuous-batching request loop.  Requests admitted while others are on the
device overlap there; each result equals the same request run alone (bitwise: same plan,
same kernels) and the FP64 oracle within the stated tolerance; admission never exceeds
the memory budget."""
import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
pytest.importorskip("torch")
from paper_2010_09746_gb300 import serve  # noqa: E402

TOL = {"c128": 1e-12, "c64": 1e-5}


def make_requests(count, seed):
    reqs = wc.serving_workload(count, rate_hz=2000.0, seed=seed, nmin=8, nmax=15, dmin=3, dmax=12)
    return reqs


def test_mix_equals_alone_and_oracle():
    reqs = make_requests(24, seed=5)
    budget = 6 * (1 << 15) * 16          # room for a few of the largest states only
    srv = serve.Server(slots=6, mem_budget=budget, readout=1 << 15)
    res = srv.run(reqs, realtime=True, timeout_s=120)
    assert len(res) == len(reqs)
    assert srv.peak_in_flight > 1, "no overlap happened"
    assert srv.peak_mem <= budget
    # all at once through two slots: compiled requests queue up and the small ones share slots
    srv2 = serve.Server(slots=2, mem_budget=budget, readout=1 << 15)
    res2 = srv2.run(reqs, realtime=False, timeout_s=120)
    assert srv2.batched_requests > 0, "no small requests were batched"
    for rid in range(len(reqs)):
        assert res2[rid].amplitudes.tobytes() == res[rid].amplitudes.tobytes(), f"request {rid} depends on the mix"
    for rid, r in enumerate(reqs):
        got = res[rid]
        alone = serve.Server(slots=1, readout=1 << 15).run([r], realtime=False)[0]
        assert got.amplitudes.tobytes() == alone.amplitudes.tobytes(), f"request {rid} depends on the mix"
        # a batched request's norm comes from the batch's per-state reduction, whose
        # summation order differs from the solo reduction's: equal up to FP64 rounding
        assert abs(got.norm - alone.norm) <= 1e-15
        ref = sv.simulate(r.n, r.circuit)
        err = np.abs(got.amplitudes.astype(np.complex128) - ref[: got.amplitudes.size]).max()
        assert err <= TOL[r.dtype]
        assert abs(got.norm - 1.0) <= TOL[r.dtype]
    summ = serve.latency_summary(res)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_unbatched_server_gives_the_same_bits():
    reqs = make_requests(12, seed=6)
    a = serve.Server(slots=4, readout=1 << 15).run(reqs, realtime=False)
    b = serve.Server(slots=4, readout=1 << 15, batch_max=1).run(reqs, realtime=False)
    for rid in range(len(reqs)):
        assert a[rid].amplitudes.tobytes() == b[rid].amplitudes.tobytes()


def test_oversized_request_rejected():
    srv = serve.Server(slots=2, mem_budget=1 << 20)
    r = wc.Request(0.0, 20, "c128", [])
    with pytest.raises(ValueError):
        srv.submit(0, r)


def test_sjf_order_same_results():
    """Shortest-work-first admission changes when requests run, not what they compute."""
    reqs = make_requests(16, seed=7)
    a = serve.Server(slots=2, readout=1 << 15, order="fifo").run(reqs, realtime=False)
    b = serve.Server(slots=2, readout=1 << 15, order="sjf").run(reqs, realtime=False)
    for rid in range(len(reqs)):
        assert a[rid].amplitudes.tobytes() == b[rid].amplitudes.tobytes()


def test_server_c_calls_failure_and_take_semantics():
    """Through the C calls directly: a request whose circuit does not compile comes back with
    its status and message (the others are unaffected); a result is taken once; poll with
    max = 0 reports nothing and keeps results for later."""
    import ctypes
    from paper_2010_09746_gb300 import _lib
    L = _lib.load()
    o = _lib.qs_server_opts()
    o.slots = 2
    o.readout = 8
    h = ctypes.c_void_p()
    _lib.check(L.qs_server_create(ctypes.byref(o), ctypes.byref(h)))
    try:
        good = wc.rzrx_cz_circuit(10, 3, seed=1)
        bad = [wc.Gate("H", (0,))]
        ids = []
        for n, circ in ((10, good), (4, bad), (10, good)):
            ops, nops, mats = qs.marshal(circ)
            if circ is bad:
                ops[0].q[0] = 7   # qubit 7 of a 4-qubit circuit: rejected by the compiler
            sid = ctypes.c_int64()
            _lib.check(L.qs_server_submit(h, n, _lib.QS_C128, ops, nops,
                                          mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                          ctypes.byref(sid)))
            ids.append(sid.value)
        cnt = ctypes.c_int()
        _lib.check(L.qs_server_poll(h, None, 0, ctypes.byref(cnt), 0))
        assert cnt.value == 0
        got = {}
        buf = (_lib.qs_server_result * 4)()
        for _ in range(200):
            _lib.check(L.qs_server_poll(h, buf, 4, ctypes.byref(cnt), 50))
            for i in range(cnt.value):
                got[buf[i].id] = (buf[i].status, buf[i].error, buf[i].amplitudes)
            if len(got) == 3:
                break
        assert len(got) == 3
        assert got[ids[1]][0] == _lib.QS_EINVAL and len(got[ids[1]][1]) > 0
        ref = sv.simulate(10, good)
        for k in (0, 2):
            st, _, count = got[ids[k]]
            assert st == _lib.QS_OK and count == 8
            amps = np.empty(8, dtype=np.complex128)
            _lib.check(L.qs_server_take(h, ids[k], amps.ctypes.data_as(ctypes.c_void_p), 8))
            assert np.max(np.abs(amps - ref[:8])) <= 1e-12
            assert L.qs_server_take(h, ids[k], amps.ctypes.data_as(ctypes.c_void_p), 8) == _lib.QS_EINVAL
    finally:
        L.qs_server_destroy(h)


def test_cancel_before_start():
    """Requests withdrawn while they wait behind a long one finish as QS_ECANCELED; the rest
    run and match the oracle."""
    from paper_2010_09746_gb300 import _lib
    srv = serve.Server(slots=1, readout=16, batch_small_n=-1)
    long_req = wc.Request(0.0, 24, "c128", wc.rzrx_cz_circuit(24, 12, seed=3))
    short = [wc.Request(0.0, 10, "c64", wc.rzrx_cz_circuit(10, 4, seed=s)) for s in range(6)]
    sids = [srv.submit(0, long_req)] + [srv.submit(k + 1, r) for k, r in enumerate(short)]
    cancelled = [srv.cancel(sid) for sid in sids[4:]]
    assert all(cancelled)
    while len(srv.results) < len(sids):
        srv.poll(1.0)
    for k in range(1, 4):
        r = srv.results[k]
        assert r.status == _lib.QS_OK
        ref = sv.simulate(10, short[k - 1].circuit)[:16]
        assert np.max(np.abs(r.amplitudes.astype(np.complex128) - ref)) <= 1e-5
    for k in range(4, 7):
        assert srv.results[k].status == _lib.QS_ECANCELED
    assert not srv.cancel(sids[0])   # already ran
    srv.close()
