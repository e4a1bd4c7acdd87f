"""Parity of the cluster r-sweep (heat_set_rsweep kind 5) against the oracle.

An r-line longer than one block holds (2048 cells) is held by a thread-block
cluster of ceil(Nr / 2048) blocks whose warps join their scan maps through
distributed shared memory; the refined FP32 path solves each line twice with
an extended-precision residual in between, exchanging delta0 across block
edges.  The cases cover clusters of 2 to 8 blocks, lines that fill their
blocks exactly or leave the last block partly (or almost) empty, rows that
are not a multiple of 4 cells (4-byte copies), row-class changes inside a
band (the layered cell's z layers), and the 1e4 conductivity contrast.
"""
import numpy as np
import pytest

from workloads import heat as H

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run(p, steps, precision, kind=5, T0=None):
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    s = HeatSolver(p, tau, precision=precision)
    try:
        if kind is not None:
            s.set_rsweep(kind)
        used = s.rsweep()
        if T0 is not None:
            s.set_field(T0)
            o.set_field(T0)
        s.step(steps)
        o.step(tau, steps)
        return s.field(), o.field(), used
    finally:
        s.close()


# (Nr, Nz): blocks per line 2 (one cell in the second block), 2 (exact),
# 3 (ragged, rows not a multiple of 4), 3 (ragged), 4 (exact), 8 (exact)
LONG = [(2049, 64), (4096, 300), (5001, 100), (6000, 200), (8192, 512), (16384, 130)]


@pytest.mark.parametrize("precision", ["fp32", "fp32_refined"])
@pytest.mark.parametrize("shape", LONG)
def test_long_lines_of_the_layered_cell(precision, shape):
    """The five-region cell (config 2's seeded problem) on long r-lines."""
    p = H.config2(*shape)
    Tg, To, used = _run(p, 6, precision)
    assert used == 5
    assert _rel(Tg, To) <= TOL


@pytest.mark.parametrize("precision", ["fp32", "fp32_refined"])
@pytest.mark.parametrize("shape", [(4097, 33), (8192, 40)])
def test_long_lines_random_field(precision, shape):
    """A random initial field (amplitude 20 K) on a single-layer cylinder with
    Dirichlet walls: increments change sign along the line and across block
    edges."""
    Nr, Nz = shape
    p = H.homogeneous_cylinder(Nr, Nz, R=2.0, Z=3.0, k=5.0, C=2.0e6,
                               bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
    T0 = H.random_field(p, seed=Nr + 3 * Nz, amp=20.0)
    Tg, To, used = _run(p, 4, precision, T0=T0)
    assert used == 5
    assert _rel(Tg, To) <= TOL


def test_high_contrast_long_lines_refined():
    """The 1e4 contrast cell (config 4's materials) on 8192-cell lines, 20
    refined steps: the contract norm and the rise-relative norm."""
    p = H.config4(8192, 96)
    Tg, To, used = _run(p, 20, "fp32_refined")
    assert used == 5
    rel = _rel(Tg, To)
    rise = float(np.max(np.abs(Tg - To)) / np.max(np.abs(To - p.T_init)))
    print(f"config4 8192x96 refined: rel {rel:.3e}, rise-relative {rise:.3e}")
    assert rel <= TOL
    assert rise <= TOL


@pytest.mark.parametrize("precision", ["fp32", "fp32_refined"])
def test_one_block_cluster(precision):
    """Kind 5 on lines one block holds (a cluster of one block)."""
    p = H.config2(1024, 130)
    Tg, To, used = _run(p, 6, precision, kind=5)
    assert used == 5
    assert _rel(Tg, To) <= TOL


def test_cluster_lines_match_block_lines():
    """The same refined steps through the cluster r-sweep and through the
    block-line r-sweep (kind 8) agree to FP32 rounding."""
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    p = H.config2(6000, 64)
    tau = H.DT_FACTOR * Oracle(p).tau_exp()
    out = []
    for kind in (5, 8):
        s = HeatSolver(p, tau, precision="fp32_refined")
        s.set_rsweep(kind)
        assert s.rsweep() == kind
        s.step(5)
        out.append(s.field())
        s.close()
    assert _rel(out[0], out[1]) <= 1e-6


def test_fp64_declines_cluster_lines():
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300.heat import HeatError
    p = H.config2(4096, 32)
    s = HeatSolver(p, 1.0, precision="fp64")
    with pytest.raises(HeatError):
        s.set_rsweep(5)
    assert s.rsweep() != 5
    s.close()


def test_longest_cluster_line_and_one_past():
    """The default rule of the plain FP32 form: lines of 2049 to 16384 cells
    (2 to 8 blocks) take the cluster r-sweep, 2048 and 16385 do not."""
    from paper_1912_03744_gb300 import HeatSolver
    for Nr, want in ((2048, False), (2049, True), (16384, True), (16385, False)):
        p = H.homogeneous_cylinder(Nr, 4, R=2.0, Z=3.0, k=5.0, C=2.0e6,
                                   bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
        s = HeatSolver(p, 1.0, precision="fp32")
        assert (s.rsweep() == 5) == want, (Nr, s.rsweep())
        s.close()


def test_block_lines_decline_lines_over_one_block():
    """Block lines of 8 cells per thread hold at most 8192 cells (1024
    threads): a longer line is refused by heat_set_rsweep, not launched."""
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300.heat import HeatError
    p = H.config2(16384, 16)
    s = HeatSolver(p, 1.0, precision="fp32")
    with pytest.raises(HeatError):
        s.set_rsweep(8)
    s.step(1)
    s.sync()
    s.close()
