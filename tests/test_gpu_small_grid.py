"""The persistent whole-step kernel of small FP64 instances (both line
lengths up to 256 cells): one cooperative launch runs every step of a
heat_step call, warps solving whole lines, grid barriers between the half
steps.  Checked against the FP64 oracle (relative max-norm 1e-12) on the
64 x 128 cell of config 1, on ragged single-layer shapes (lines of 1 to 256
cells, one or several cells per lane), and against the regular sweep
kernels (heat_set_rsweep with a non-zero kind keeps the regular path)."""
import numpy as np
import pytest

from workloads import heat as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _pair(p, steps, T0=None, chunks=1):
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    s = HeatSolver(p, tau, precision="fp64")
    assert s.launches_per_step() == 1
    if T0 is not None:
        s.set_field(T0)
        o.set_field(T0)
    per = steps // chunks
    for _ in range(chunks):
        s.step(per)
    s.sync()
    o.step(tau, per * chunks)
    Tg = s.field()
    s.close()
    return Tg, o.field()


def test_config1_200_steps():
    """Config 1 as specified (64 x 128, five regions, 200 steps), in one call
    and in 8 calls of 25 steps."""
    p = H.config1()
    for chunks in (1, 8):
        Tg, To = _pair(p, 200, chunks=chunks)
        assert _rel(Tg, To) <= 1e-12, chunks


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (3, 5), (31, 33), (33, 31), (64, 65), (100, 256), (256, 3),
                                   (256, 256), (129, 200)])
def test_ragged_small_grids(shape):
    Nr, Nz = shape
    p = H.homogeneous_cylinder(Nr, Nz, R=2.0, Z=3.0, k=5.0, C=2.0e6,
                               bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
    T0 = H.random_field(p, seed=Nr * 5 + Nz, amp=20.0)
    Tg, To = _pair(p, 7, T0=T0)
    assert _rel(Tg, To) <= 1e-12


def test_matches_the_regular_sweeps_and_larger_grids_keep_them():
    from paper_1912_03744_gb300 import HeatSolver
    p = H.config2(96, 200)
    probe = HeatSolver(p, 1.0, precision="fp64")
    tau = H.DT_FACTOR * probe.tau_exp
    probe.close()
    T0 = H.random_field(p, seed=9, amp=30.0)
    out = []
    for kind in (0, 1):
        s = HeatSolver(p, tau, precision="fp64")
        if kind:
            s.set_rsweep(kind)
        assert s.launches_per_step() == (1 if kind == 0 else 4)
        s.set_field(T0)
        s.step(10)
        out.append(s.field())
        s.close()
    assert _rel(out[0], out[1]) <= 1e-13
    big = H.config2(257, 64)
    s = HeatSolver(big, 1.0, precision="fp64")
    assert s.launches_per_step() == 4
    s.close()
