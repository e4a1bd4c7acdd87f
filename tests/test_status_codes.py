"""Failure detection at the C ABI: bad arguments and non-finite fields are
reported as status codes, never as a crash or a silent result.

The argument checks of ``heat_create`` run on the host before any CUDA call,
so they are exercised here without a GPU.  ``HEAT_ERR_NONFINITE`` needs a live
context: a NaN written into the field through ``heat_set_field`` must make
``heat_energy`` (and its no-allocation twin) return the status, and the
context must stay usable afterwards.  No GPU fault is provoked: the NaN is an
ordinary value in an ordinary buffer.
"""
import ctypes

import numpy as np
import pytest

from workloads import heat as H

HEAT_OK, HEAT_ERR_ARG, HEAT_ERR_NONFINITE = 0, -1, -3


def _create(p, dt=1.0, precision=0, face_mean=0):
    from paper_1912_03744_gb300 import build
    from paper_1912_03744_gb300 import heat as hb
    build.build()
    L = hb.load()
    keep = []
    geo, mat = hb._marshal(p, keep)
    opt = hb._Options(precision, face_mean)
    h = ctypes.c_void_p(12345)
    st = L.heat_create(ctypes.byref(geo), ctypes.byref(mat), ctypes.byref(opt), float(dt), None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("case", ["unordered_r_faces", "unordered_z_faces", "zero_r_cells", "dt_zero",
                                  "dt_negative", "dt_nan", "k_zero", "C_negative", "box_region_out_of_range",
                                  "bad_precision", "bad_face_mean", "bad_bc_kind", "nonfinite_T_init"])
def test_create_rejects_bad_arguments_without_touching_the_gpu(case):
    p = H.config1()
    dt, prec, fm = 1.0, 0, 0
    if case == "unordered_r_faces":
        rf = p.r_faces.copy()
        rf[2], rf[3] = rf[3], rf[2]
        p = p.copy(r_faces=rf)
    elif case == "unordered_z_faces":
        p = p.copy(z_faces=p.z_faces[::-1].copy())
    elif case == "zero_r_cells":
        rc = p.r_cells.copy()
        rc[1] = 0
        p = p.copy(r_cells=rc)
    elif case == "dt_zero":
        dt = 0.0
    elif case == "dt_negative":
        dt = -1.0
    elif case == "dt_nan":
        dt = float("nan")
    elif case == "k_zero":
        k = p.k.copy()
        k[2] = 0.0
        p = p.copy(k=k)
    elif case == "C_negative":
        C = p.C.copy()
        C[0] = -1.0
        p = p.copy(C=C)
    elif case == "box_region_out_of_range":
        br = p.box_region.copy()
        br[0] = len(p.k)
        p = p.copy(box_region=br)
    elif case == "bad_precision":
        prec = 7
    elif case == "bad_face_mean":
        fm = 2
    elif case == "bad_bc_kind":
        bc = p.bc.copy()
        bc[3] = 5
        p = p.copy(bc=bc)
    elif case == "nonfinite_T_init":
        p = p.copy(T_init=float("inf"))
    st, h = _create(p, dt, prec, fm)
    assert st == HEAT_ERR_ARG, (case, st)
    assert h.value is None, "on error *out must be NULL"


def test_null_arguments_rejected_without_gpu():
    from paper_1912_03744_gb300 import heat as hb
    L = hb.load()
    h = ctypes.c_void_p()
    assert L.heat_create(None, None, None, 1.0, None, ctypes.byref(h)) == HEAT_ERR_ARG
    assert L.heat_create(None, None, None, 1.0, None, None) == HEAT_ERR_ARG
    for fn in ("heat_step", "heat_sweep", "heat_set_dt"):
        assert getattr(L, fn)(None, 1) == HEAT_ERR_ARG, fn
    assert L.heat_energy(None, None, None, None) == HEAT_ERR_ARG
    assert L.heat_field(None, None, 0, 0) == HEAT_ERR_ARG
    assert L.heat_set_field(None, None, 0, 0) == HEAT_ERR_ARG
    assert L.heat_sync(None) == HEAT_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refined"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_nonfinite_field_is_reported_and_the_context_recovers(precision, value):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300.heat import HeatError
    p = H.config1()
    s = HeatSolver(p, 1.0, precision="fp64")
    tau = 20.0 * s.tau_exp
    s.close()
    s = HeatSolver(p, tau, precision=precision)
    T = s.field()
    E0, _, _ = s.energy()
    bad = T.copy()
    bad[5, 7] = value  # cell (i=7, j=5): cooler, active
    s.set_field(bad)
    for fn in (s.energy, s.energy_noalloc):
        with pytest.raises(HeatError) as ei:
            fn()
        assert ei.value.status == HEAT_ERR_NONFINITE
    # the context stays usable: a finite field gives a finite balance again
    s.set_field(T)
    E1, _, _ = s.energy()
    assert np.isfinite(E1) and E1 == E0
    s.step(2)
    assert np.isfinite(s.field()).all()
    s.close()


@pytest.mark.gpu
def test_bounded_wait_reports_a_timeout_and_the_context_recovers():
    """The FP32 r-sweep that stages rows by bulk copies waits on mbarriers with
    a time limit.  The test hook makes its first wait run out (a barrier
    nothing completes, no copy issued): heat_sync must return
    HEAT_ERR_TIMEOUT, and with the hook off the next steps must match the
    oracle again."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300 import heat as hb
    p = H.config2(256, 64)
    o = Oracle(p)
    tau = 20.0 * o.tau_exp()
    s = HeatSolver(p, tau, precision="fp32")
    s.set_rsweep(3)  # the r-sweep that stages rows by bulk copies on mbarriers
    L = hb.load()
    assert L.heat_test_stall(s._h, 1) == HEAT_OK
    s.step(1)
    assert L.heat_sync(s._h) == -4  # HEAT_ERR_TIMEOUT
    assert L.heat_sync(s._h) == HEAT_OK  # reported once
    assert L.heat_test_stall(s._h, 0) == HEAT_OK
    T0 = H.random_field(p, seed=5, amp=10.0)
    s.set_field(T0)
    o.set_field(T0)
    s.step(3)
    o.step(tau, 3)
    assert L.heat_sync(s._h) == HEAT_OK
    assert float(np.max(np.abs(s.field() - o.field())) / np.max(np.abs(o.field()))) <= 1e-5
    s.close()


@pytest.mark.gpu
def test_grid_barrier_time_out_is_reported_and_the_context_recovers():
    """The persistent step kernel of a small FP64 instance separates its half
    steps by a grid barrier with a 1 s limit.  The test hook makes the first
    barrier wait for one block more than the launch has: heat_sync must
    return HEAT_ERR_TIMEOUT, and with the hook off the next steps must match
    the oracle again."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from oracle import Oracle
    from paper_1912_03744_gb300 import HeatSolver
    from paper_1912_03744_gb300 import heat as hb
    p = H.config1()
    o = Oracle(p)
    tau = 20.0 * o.tau_exp()
    s = HeatSolver(p, tau, precision="fp64")
    assert s.launches_per_step() == 1  # the persistent kernel
    L = hb.load()
    assert L.heat_test_stall(s._h, 1) == HEAT_OK
    s.step(3)
    assert L.heat_sync(s._h) == -4  # HEAT_ERR_TIMEOUT
    assert L.heat_sync(s._h) == HEAT_OK
    assert L.heat_test_stall(s._h, 0) == HEAT_OK
    T0 = H.random_field(p, seed=6, amp=10.0)
    s.set_field(T0)
    o.set_field(T0)
    s.step(4)
    o.step(tau, 4)
    assert L.heat_sync(s._h) == HEAT_OK
    assert float(np.max(np.abs(s.field() - o.field())) / np.max(np.abs(o.field()))) <= 1e-12
    s.close()
