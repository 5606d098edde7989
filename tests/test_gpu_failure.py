"""Failure detection without a GPU fault: the bounded device waits give up
and report instead of hanging (and the context stays usable), and the guard
bytes around every device allocation catch a write outside an array (the
write is made from the host through the allocator, no kernel misbehaves)."""
import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_2211_05647_gb300 import FdtdError, Solver, selftest_wait_timeout
    assert selftest_wait_timeout(1000) is True
    with pytest.raises(FdtdError):
        selftest_wait_timeout(0)
    s = Solver.from_spec(spec_2d_cylinder(n=96, ny=80, R=16, center=(55, 40), src=(30, 40), steps=20, seed=3))
    s.step(20)
    d = s.diagnostics()
    assert d["finite"] and d["energy"] > 0


def test_timed_wait_gives_up_after_its_limit():
    """The wall-clock-bounded wait of the TMA stencils: a barrier that nothing
    arrives at is given up on after the limit (2 ms here), not sooner and not
    never; the context stays usable."""
    import time
    from paper_2211_05647_gb300 import FdtdError, selftest_timed_wait
    selftest_timed_wait(10)                       # load and warm the module
    t0 = time.perf_counter()
    assert selftest_timed_wait(2000) is True
    dt = time.perf_counter() - t0
    print(f"timed wait of 2 ms gave up after {dt * 1e3:.2f} ms (host clock)")
    assert 2e-3 <= dt < 1.0
    for bad in (0, 10 ** 7):
        with pytest.raises(FdtdError):
            selftest_timed_wait(bad)


def test_canaries_clean_after_a_run_and_catch_a_stray_byte(monkeypatch):
    monkeypatch.setenv("FDTD_PLASMA_CANARIES", "1")
    from paper_2211_05647_gb300 import FdtdError, Solver
    spec = spec_2d_cylinder(n=120, ny=96, R=20, center=(70, 48), src=(30, 48), steps=80, seed=4)
    s = Solver.from_spec(spec)
    s.set_ports([[48 * 120 + 100]], np.linspace(5e9, 15e9, 8))
    s.step(80)
    s.diagnostics()
    assert s.check_canaries() == 0
    # change one guard byte of one allocation (the byte just before its user range)
    blocks = s._alloc.live
    assert blocks
    ptr, t = next(iter(blocks.items()))
    off = ptr - t.data_ptr() + 255           # allocator block = [256 guard | user | 256 guard]
    old = int(t[off].item())
    t[off] = (old + 1) % 256
    assert s.check_canaries() == 1
    t[off] = old
    assert s.check_canaries() == 0
    monkeypatch.delenv("FDTD_PLASMA_CANARIES")
    plain = Solver.from_spec(spec)
    with pytest.raises(FdtdError):
        plain.check_canaries()
