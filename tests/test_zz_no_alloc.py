"""heat_energy_noalloc (the energy / flux reduction with its scratch in a fixed
device array, no allocation) against heat_energy, through the C ABI.

Collected last on purpose: it must also pass after every other test has run
in the same process, when the fixed array already holds other contexts'
partial sums."""
import ctypes

import numpy as np
import pytest

from workloads import heat as H

pytestmark = pytest.mark.gpu

# Same FP64 terms grouped per row instead of per block: rounding-level differences only.
REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _close(a, b, scale):
    return abs(a - b) <= REL * max(abs(b), scale)


def _check_pair(s):
    E, F, Q = s.energy()
    first = s.energy_noalloc()
    second = s.energy_noalloc()
    assert first == second  # same decomposition, deterministic reduction
    En, Fn, Qn = first
    assert Qn == Q
    assert _close(En, E, 0.0), (En, E)
    assert _close(Fn, F, 1e-6 * abs(Q)), (Fn, F)
    return first


def test_matches_heat_energy_on_two_calls_in_a_row():
    from paper_1912_03744_gb300 import HeatSolver
    # A larger grid first (Nz = 1024 rows of partials), then smaller ones whose
    # calls must not see the first one's leftover partial sums.
    cases = [(H.config2(256, 1024), "fp64"), (H.config1(), "fp32"), (H.config2(96, 200), "fp32_refined")]
    for p, prec in cases:
        probe = HeatSolver(p, 1.0, precision="fp64")
        tau = 20.0 * probe.tau_exp
        probe.close()
        s = HeatSolver(p, tau, precision=prec)
        s.set_field(H.random_field(p, seed=p.Nz, amp=25.0))
        _check_pair(s)
        s.step(3)
        _check_pair(s)
        s.close()


def test_row_limit():
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300.heat import HeatError
    kw = dict(R=1.0, Z=2.0, k=3.0, C=1.0e6, bc=(0, 0, 0, 1), T_bc=(0, 0, 0, 280.0), T_init=300.0, q=1e4)
    p = H.homogeneous_cylinder(3, 8192, **kw)
    s = HeatSolver(p, 1.0, precision="fp64")
    s.step(1)
    _check_pair(s)
    s.close()
    p = H.homogeneous_cylinder(3, 8193, **kw)
    s = HeatSolver(p, 1.0, precision="fp64")
    with pytest.raises(HeatError) as ei:
        s.energy_noalloc()
    assert ei.value.status == -6
    E, _, _ = s.energy()  # the context is still usable
    assert np.isfinite(E)
    s.close()


def test_null_context_rejected():
    from paper_1912_03744_gb300 import heat as hb
    L = hb.load()
    d = ctypes.c_double()
    assert L.heat_energy_noalloc(None, ctypes.byref(d), None, None) == -1
    assert hb.load().heat_strerror(-6) == b"size beyond a fixed capacity"
