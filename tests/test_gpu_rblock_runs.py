"""Parity of the register-resident r-sweep (heat_set_rsweep kind 2) when a
single instance's bands are split at row-class boundaries.

Rows of one row class (the same r-line matrix) form runs; with lines of
whole warps (Nr > 128) every run is split into its own bands of rows, so no
line slot changes class inside its band.  The cases stack z slabs of
different materials: runs of one row, of odd and even lengths, 16 runs (the
most the arguments keep) and 17 (uniform bands over the whole height
instead), lines of one warp (several slots per block), of 2 and 8 warps, and
rows that are not a multiple of 4 cells.  Each is compared with the oracle
element by element after a few steps.
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


def stacked_slabs(Nr, z_cells, seed):
    """A cylinder of radius 0.1 m made of len(z_cells) axial slabs, each its
    own material (k log-uniform in [0.1, 100], C uniform in [1e6, 4e6], a
    source in every third slab), Dirichlet on the outer wall and the top."""
    rng = np.random.default_rng(seed)
    n = len(z_cells)
    th = rng.uniform(0.5, 1.5, size=n) * 1e-2
    zf = np.concatenate([[0.0], np.cumsum(th)])
    R = 0.1
    boxes = np.array([[0.0, R, zf[m], zf[m + 1]] for m in range(n)])
    k = np.exp(rng.uniform(np.log(0.1), np.log(100.0), size=n))
    C = rng.uniform(1e6, 4e6, size=n)
    q = np.where(np.arange(n) % 3 == 0, rng.uniform(1e5, 1e7, size=n), 0.0)
    return H.Problem(name=f"slabs_{Nr}x{sum(z_cells)}", r_faces=np.array([0.0, R]),
                     r_cells=np.array([Nr], dtype=np.int32), z_faces=zf,
                     z_cells=np.asarray(z_cells, dtype=np.int32), boxes=boxes,
                     box_region=np.arange(n, dtype=np.int32),
                     bc=np.array([H.BC_NEUMANN, H.BC_DIRICHLET, H.BC_NEUMANN, H.BC_DIRICHLET], dtype=np.int32),
                     T_bc=np.array([0.0, 290.0, 0.0, 330.0]), k=k, C=C, q=q, T_init=300.0)


def _run(p, steps=4, seed=0):
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    s = HeatSolver(p, tau, precision="fp32")
    try:
        used = s.rsweep()
        T0 = H.random_field(p, seed=seed, amp=15.0)
        s.set_field(T0)
        o.set_field(T0)
        s.step(steps)
        o.step(tau, steps)
        return s.field(), o.field(), used
    finally:
        s.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


CASES = [
    # (Nr, slab cells): warps per line, run lengths
    (2048, [401, 7, 1, 190]),                       # 8 warps; runs of 1 and 7 rows
    (2048, [1] * 8 + [33] * 8),                     # exactly 16 runs, eight of one row
    (2048, [3] * 17),                               # 17 runs: uniform bands
    (512, [64, 65, 1, 2, 130]),                     # 2 warps per line, 2 slots per block
    (256, [10, 301, 5]),                            # one warp per line, 8 slots per block
    (1000, [97, 1, 1, 200]),                        # rows not a multiple of 4 cells
    (1531, [250, 251]),                             # odd line, two runs
]


@pytest.mark.parametrize("Nr,z_cells", CASES)
def test_run_bands_match_the_oracle(Nr, z_cells):
    p = stacked_slabs(Nr, z_cells, seed=Nr + len(z_cells))
    Tg, To, used = _run(p, seed=len(z_cells))
    assert used == 2
    assert _rel(Tg, To) <= TOL


def test_run_bands_on_the_layered_cell():
    """The five-region cell at 2048 x 4096 (three row-class runs): 3 steps."""
    p = H.config2(2048, 4096)
    Tg, To, used = _run(p, steps=3, seed=1)
    assert used == 2
    assert _rel(Tg, To) <= TOL


def test_run_bands_with_a_requested_band():
    """A batch of one member with the register-resident r-sweep and a band
    set through the tuning call: the bands still split at run boundaries."""
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatBatch
    p = stacked_slabs(1024, [37, 3, 60, 1], seed=9)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    T0 = H.random_field(p, seed=4, amp=15.0)
    o.set_field(T0)
    o.step(tau, 3)
    for band in (0, 5, 64):
        b = HeatBatch([p], [tau], precision="fp32")
        try:
            b.set_tuning(2, band, 0)
            assert b.tuning()[0] == 2
            b.members[0].set_field(T0)
            b.step(3)
            assert _rel(b.members[0].field(), o.field()) <= TOL, band
        finally:
            b.close()
