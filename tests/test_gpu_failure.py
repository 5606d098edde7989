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
