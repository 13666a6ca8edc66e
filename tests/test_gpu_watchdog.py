"""Device watchdog: a bounded wait that nothing satisfies expires, the kernel
records TE_ETIMEOUT in the handle's error word and returns; te_sync reports
it once and the context keeps working (no fault, no hang)."""
import time

import pytest

import tegen
from oracle import t_energy as O
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    return need_gpu()


def test_wait_expires_and_is_reported(te):
    from paper_2412_18553_gb300._lib import TE_ETIMEOUT
    h = te.Handle(0)
    t0 = time.perf_counter()
    h.watchdog_selftest(20_000_000)
    with pytest.raises(te.TEnergyError) as ei:
        h.sync()
    dt = time.perf_counter() - t0
    assert ei.value.status == TE_ETIMEOUT
    assert "site 99" in str(ei.value)
    assert 0.015 <= dt < 5.0
    h.sync()  # the word was cleared
    cl = tegen.make_cluster(3, 17, 80, 4)
    ref = float(O.t_energy(O.inputs(**cl.arrays())))
    for prec in ("fp64", "ozaki"):
        e = float(te.t_energy(cl, prec, handle=h))
        h.sync()
        assert abs(e - ref) <= 1e-9, (prec, e, ref)


def test_limit_is_validated(te):
    h = te.Handle(0)
    for bad in (0, 999_999, 10_000_000_001):
        with pytest.raises(te.TEnergyError):
            h.watchdog_selftest(bad)
    h.sync()
