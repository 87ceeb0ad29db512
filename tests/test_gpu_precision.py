"""GPU: the FP64 inner product between states of either storage type, renormalisation and
periodic renormalisation inside plans, checked against the FP64 oracle and against host
FP64 sums over the read-back amplitudes."""
import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")


def rand_state(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v) * scale


@pytest.mark.parametrize("da,db", [("c128", "c128"), ("c64", "c128"), ("c128", "c64"), ("c64", "c64")])
def test_inner_matches_host_sum(da, db):
    n = 15   # 2^15 amplitudes: more than the 1216 x 256 threads of the reduction
    a, b = qs.State(n, da), qs.State(n, db)
    a.set_amplitudes(rand_state(n, 1))
    b.set_amplitudes(rand_state(n, 2))
    ha = a.amplitudes().astype(np.complex128)
    hb = b.amplitudes().astype(np.complex128)
    got = a.inner(b)
    ref = np.vdot(ha, hb)
    assert abs(got - ref) <= 1e-13
    assert abs(a.inner(a) - a.norm()) <= 1e-14   # the imaginary part is FMA rounding only


def test_inner_rejects_mismatch():
    a, b, c = qs.State(6, "c128"), qs.State(7, "c128"), qs.State(6, "c64")
    with pytest.raises(qs.QSError):
        a.inner(b)
    c.permute([1, 0, 2, 3, 4, 5])
    with pytest.raises(qs.QSError):
        a.inner(c)


def test_inner_small_and_tiny():
    for n in (1, 2, 9):
        a = qs.State(n, "c64")
        b = qs.State(n, "c128")
        a.set_amplitudes(rand_state(n, 3))
        b.set_amplitudes(rand_state(n, 4))
        assert abs(a.inner(b) - np.vdot(a.amplitudes().astype(np.complex128), b.amplitudes())) <= 1e-14


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-15), ("c64", 2e-7)])
def test_renormalize(dtype, tol):
    for n in (1, 5, 13, 18):
        v = rand_state(n, n, scale=2.0)
        st = qs.State(n, dtype)
        st.set_amplitudes(v)
        before = st.amplitudes().astype(np.complex128)
        nrm = st.renormalize()
        assert nrm == pytest.approx(np.vdot(before, before).real, rel=1e-13)
        after = st.amplitudes().astype(np.complex128)
        assert np.max(np.abs(after - before / np.sqrt(nrm))) <= tol * np.max(np.abs(before))
        assert abs(st.norm() - 1.0) <= 4 * tol * max(1, n)


def test_renormalize_zero_state_unchanged():
    st = qs.State(8, "c64")
    st.set_amplitudes(np.zeros(256, dtype=np.complex64))
    assert st.renormalize() == 0.0
    assert np.all(st.amplitudes() == 0)


@pytest.mark.parametrize("mode", ["pergate", "tile"])
def test_periodic_renormalisation_in_plans(mode):
    n = 16
    circ = wc.rzrx_cz_circuit(n, 10, seed=7)
    ref = sv.simulate(n, circ)
    for R in (1, 3):
        st = qs.State(n, "c64")
        st.execute(qs.compile(n, circ, mode=mode, dtype="c64", renorm_every=R))
        got = st.amplitudes().astype(np.complex128)
        assert abs(st.norm() - 1.0) <= 2e-6
        assert sv.fidelity_loss(got, ref) <= 1e-5
        st = qs.State(n, "c128")
        st.execute(qs.compile(n, circ, mode=mode, dtype="c128", renorm_every=R))
        assert np.max(np.abs(st.amplitudes() - ref)) <= 1e-12


def test_precision_study_per_circuit():
    """complex64 against complex128 of the same circuit: the kernel's FP64 fidelity equals
    the host's over the read-back amplitudes, and both meet the complex64 bound against the
    oracle."""
    n = 18
    for seed in range(3):
        circ = wc.rzrx_cz_circuit(n, 12, seed=seed)
        ref = sv.simulate(n, circ)
        s64, s128 = qs.State(n, "c64"), qs.State(n, "c128")
        s64.run(circ)
        s128.run(circ)
        f_dev = 1.0 - s64.fidelity(s128)
        a64 = s64.amplitudes().astype(np.complex128)
        a128 = s128.amplitudes()
        f_host = 1.0 - abs(np.vdot(a64, a128)) ** 2 / (np.vdot(a64, a64).real * np.vdot(a128, a128).real)
        assert abs(f_dev - f_host) <= 1e-12
        assert sv.fidelity_loss(a64, ref) <= 1e-5
