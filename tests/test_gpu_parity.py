"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bar: relative max-norm ||T_gpu - T_oracle||_inf / ||T_oracle||_inf over all
cells <= 1e-12 for the FP64 path and <= 1e-5 for the FP32 path (the
tolerances the workload specifies), on the same seeded inputs.
"""
import numpy as np
import pytest

from oracle import Oracle
from workloads import heat as H

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_refined": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _solver(p, tau, precision):
    from paper_1912_03744_gb300 import HeatSolver
    return HeatSolver(p, tau, precision=precision)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run_pair(p, steps, precision, T0=None, factor=H.DT_FACTOR):
    o = Oracle(p)
    tau = factor * o.tau_exp()
    s = _solver(p, tau, precision)
    if T0 is not None:
        o.set_field(T0)
        s.set_field(T0)
    o.step(tau, steps)
    s.step(steps)
    out = s.field(), o.field()
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
def test_config1_full_run(precision):
    """64x128 five-region cell, 200 steps at dt = 50 tau_exp."""
    p = H.config1()
    Tg, To = _run_pair(p, H.STEPS["config1"], precision)
    assert _rel(Tg, To) <= TOL[precision]


def test_grid_and_limit_parity():
    from paper_1912_03744_gb300 import HeatSolver
    for p in (H.config1(), H.config_paper_grid(), H.config3_members(3)[2]):
        o = Oracle(p)
        s = HeatSolver(p, 1.0, precision="fp64")
        rc, zc = s.centres()
        g = o.grid()
        np.testing.assert_allclose(rc, g["rc"], rtol=1e-15)
        np.testing.assert_allclose(zc, g["zc"], rtol=1e-15)
        assert abs(s.tau_exp - o.tau_exp()) <= 1e-13 * o.tau_exp()
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
def test_half_step_parity(precision):
    """The half layer Tbar (eq. scheme_eq_1) and the full step separately."""
    p = H.config2(96, 200)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    T0 = H.random_field(p, seed=21, amp=40.0)
    s = _solver(p, tau, precision)
    o.set_field(T0)
    s.set_field(T0)
    o.step(tau)
    s.sweep(0)
    assert _rel(s.field(), o.half_field()) <= TOL[precision]
    s.sweep(1)
    assert _rel(s.field(), o.field()) <= TOL[precision]
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
@pytest.mark.parametrize("shape", [(256, 512), (333, 517), (1000, 130), (64, 3000)])
def test_config2_reduced_grids(precision, shape):
    """Config 2's seeded problem on reduced (and ragged) grids, 60 steps."""
    p = H.config2(*shape)
    Tg, To = _run_pair(p, 60, precision)
    assert _rel(Tg, To) <= TOL[precision]


ODD = [(1, 1), (1, 7), (2, 2), (3, 5), (31, 33), (33, 31), (32, 64), (257, 3), (1025, 9), (4097, 5),
       (8192, 2), (9000, 2), (16384, 1), (17000, 2), (5, 1100), (3, 4097), (2, 9000)]


@pytest.mark.parametrize("shape", ODD)
def test_ragged_and_long_lines_fp64(shape):
    """Single-layer cylinders of ragged sizes: lines of 1 cell up to 17000
    cells in r, and long z-lines; random initial fields; Dirichlet top."""
    Nr, Nz = shape
    p = H.homogeneous_cylinder(Nr, Nz, R=2.0, Z=3.0, k=5.0, C=2.0e6,
                               bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
    T0 = H.random_field(p, seed=Nr * 7 + Nz, amp=20.0)
    Tg, To = _run_pair(p, 3, "fp64", T0=T0)
    assert _rel(Tg, To) <= 1e-12


# FP32 shapes around the kernel choices: lines that fill their threads
# exactly (2048, 64) or not (2047, 100), one past the register-resident
# r-sweep (2049), ragged and partial z chunks (Nz 33, 40, 65; 8200 gives
# 36-row chunks, not a multiple of the fetch groups)
@pytest.mark.parametrize("shape", [(31, 33), (4097, 5), (9000, 2), (3, 4097), (2048, 40), (2047, 33),
                                   (2049, 9), (64, 65), (100, 40), (8, 8200)])
def test_ragged_fp32(shape):
    Nr, Nz = shape
    p = H.homogeneous_cylinder(Nr, Nz, R=2.0, Z=3.0, k=5.0, C=2.0e6,
                               bc=(0, 1, 0, 1), T_bc=(0, 250.0, 0, 310.0), T_init=300.0, q=1e5)
    T0 = H.random_field(p, seed=Nr + Nz, amp=20.0)
    Tg, To = _run_pair(p, 3, "fp32", T0=T0)
    assert _rel(Tg, To) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_grid_and_annulus(precision):
    """The paper's graded 1210x100 grid (Sec. 5) and a Dirichlet-walled layered annulus."""
    p = H.config_paper_grid()
    Tg, To = _run_pair(p, 20, precision)
    assert _rel(Tg, To) <= TOL[precision]
    p = H.layered_annulus([1.0, 1.3, 1.7, 2.0], [40, 50, 30], [1.0, 20.0, 0.3], 100.0, 0.0, Nz=17)
    T0 = H.random_field(p, seed=2)
    Tg, To = _run_pair(p, 10, precision, T0=T0, factor=5.0)
    assert _rel(Tg, To) <= TOL[precision]


def test_column_tiles_with_thin_layers():
    """FP32 z-sweep on column tiles of one class each, with layers of 3 and 2
    columns: 4096 columns in layers of 2001, 3, 2 and 2090 give 35 tiles of at
    most 128 columns (32 plain warps of 128 would straddle the interfaces), so
    tiles start inside a lane's 16-byte segment, one lane reads three classes
    and tiles of 3 and 2 columns store only their own columns."""
    p = H.layered_annulus([1.0, 2.0, 2.003, 2.005, 4.0], [2001, 3, 2, 2090], [1.0, 20.0, 0.3, 5.0],
                          100.0, 0.0, Nz=24)
    T0 = H.random_field(p, seed=3)
    Tg, To = _run_pair(p, 10, "fp32", T0=T0, factor=5.0)
    assert _rel(Tg, To) <= TOL["fp32"]


@pytest.mark.parametrize("face_mean", [H.FACE_ARITH])
def test_arithmetic_face_mean(face_mean):
    p = H.config1().copy(face_mean=face_mean)
    Tg, To = _run_pair(p, 50, "fp64")
    assert _rel(Tg, To) <= 1e-12


def test_heat_balance_gpu_fp64():
    """E(next) - E(now) = tau Q + (tau/2)(Phi(now) + Phi(next)) on the GPU's own reductions."""
    p = H.config2(512, 1024)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    s = _solver(p, tau, "fp64")
    T0 = H.random_field(p, seed=4, amp=30.0)
    s.set_field(T0)
    E0, F0, Q = s.energy()
    o.set_field(T0)
    Eo, Fo, Qo = o.energy()
    assert abs(E0 - Eo) <= 1e-12 * abs(Eo) and abs(Q - Qo) <= 1e-12 * abs(Qo)
    assert abs(F0 - Fo) <= 1e-9 * max(abs(Fo), 1.0)
    s.step(1)
    E1, F1, _ = s.energy()
    assert abs((E1 - E0) - (tau * Q + 0.5 * tau * (F0 + F1))) <= 1e-12 * abs(E0)
    s.close()


def test_resume_and_determinism():
    """n steps == k steps, save, restore into a fresh context, n-k steps (bitwise);
    two runs are bitwise identical."""
    p = H.config2(300, 700)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    a = _solver(p, tau, "fp64")
    a.step(12)
    Ta = a.field()
    b = _solver(p, tau, "fp64")
    b.step(5)
    mid = b.field()
    c = _solver(p, tau, "fp64")
    c.set_field(mid)
    c.step(7)
    np.testing.assert_array_equal(c.field(), Ta)
    d = _solver(p, tau, "fp64")
    d.step(12)
    np.testing.assert_array_equal(d.field(), Ta)
    for s in (a, b, c, d):
        s.close()


def test_device_field_roundtrip():
    import torch
    p = H.config1()
    s = _solver(p, 10.0, "fp32")
    T0 = H.random_field(p, seed=8)
    t = torch.tensor(T0, dtype=torch.float64, device="cuda").reshape(-1)
    s.set_field(t)
    out = torch.empty_like(t)
    s.field(out)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy().reshape(T0.shape), T0) <= 1e-7
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
def test_full_size_config2_few_steps(precision):
    """Config 2 at its full 2048 x 4096 size, in the launch configuration the
    benchmark times, 3 steps against the oracle on the whole field."""
    p = H.config2()
    Tg, To = _run_pair(p, 3, precision)
    assert _rel(Tg, To) <= TOL[precision]


def test_refined_path_reduces_the_solve_error_at_high_contrast():
    """Config 4's 1e4 conductivity contrast on a 512 x 1024 grid: one half-step
    from T = T_init (increment = the implicit solve of the source term).  The
    plain FP32 factorization leaves an error ~ kappa * eps in the increment;
    one FP64-residual correction brings it to ~ eps (storage rounding).
    After 50 full steps both FP32 paths stay within the FP32 bar."""
    p = H.config4(512, 1024)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    o.step(tau)
    inc_o = o.half_field() - p.T_init
    errs = {}
    for prec in ("fp32", "fp32_refined"):
        s = _solver(p, tau, prec)
        s.sweep(0)
        errs[prec] = _rel(s.field() - p.T_init, inc_o)
        s.sweep(1)
        s.step(49)
        s.close()
    assert errs["fp32_refined"] <= 0.5 * errs["fp32"], errs
    o2 = Oracle(p)
    o2.step(tau, 50)
    for prec in ("fp32", "fp32_refined"):
        s = _solver(p, tau, prec)
        s.step(50)
        assert _rel(s.field(), o2.field()) <= 1e-5
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp32_refined"])
def test_config4_subsample_against_the_oracle(precision):
    """Config 4 as its accuracy is specified: the 1e4 conductivity contrast
    (0.04 against 400) on the 1024 x 2048 subsample grid, 200 steps, against
    the FP64 oracle.  Bars: relative max-norm 1e-5 over the field; the same
    1e-5 against the largest temperature rise |T - T_init| (stricter: the FP32
    fields store T - T_init, so their rounding scales with the rise); the FP64
    energy change E(T) - E(T_init) within 1e-5 of the oracle's."""
    p = H.config4(1024, 2048)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    E_init = o.energy()[0]
    o.step(tau, 200)
    To = o.field()
    Eo = o.energy()[0]
    s = _solver(p, tau, precision)
    s.step(200)
    Tg = s.field()
    E, _, _ = s.energy()
    s.close()
    rel = _rel(Tg, To)
    rise = float(np.max(np.abs(Tg - To)) / np.max(np.abs(To - p.T_init)))
    derr = abs((E - E_init) - (Eo - E_init)) / abs(Eo - E_init)
    print(f"config4 1024x2048 {precision}: rel max {rel:.3e}, rise-relative {rise:.3e}, energy change {derr:.3e}")
    assert rel <= 1e-5, rel
    assert rise <= 1e-5, rise
    assert derr <= 1e-5, derr


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 8, 16, 32])
@pytest.mark.parametrize("shape", [(512, 300), (1024, 130), (2048, 37), (300, 70)])
def test_every_rsweep_kernel_of_a_single_instance(kind, shape):
    """Each r-sweep kernel heat_set_rsweep can pick (line teams, register-
    resident lines, walked lines, block lines), on lines of 300 to 2048 cells
    (300: not a multiple of 4, the walked lines decline), FP32, 6 steps."""
    from paper_1912_03744_gb300.heat import HeatError
    p = H.config2(*shape)
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    s = _solver(p, tau, "fp32")
    try:
        s.set_rsweep(kind)
    except HeatError:
        assert kind == 3 and shape[0] % 4 != 0 or kind == 2 and shape[0] > 2048 or kind in (4,) and shape[0] > 4096
        s.close()
        return
    assert s.rsweep() == kind
    T0 = H.random_field(p, seed=kind + shape[0], amp=20.0)
    s.set_field(T0)
    o.set_field(T0)
    s.step(6)
    o.step(tau, 6)
    assert _rel(s.field(), o.field()) <= TOL["fp32"]
    s.close()
