"""The full method on the GPU (heat_nl_*, FP64) against the oracle's full
method: temperature-dependent k, C and resistivity, the simple iteration,
tau halving, the evolution loop and the pulsed source.

Bar: relative max-norm 1e-12 (FP64), and the integer decisions -- the
iterations each half-step takes, the halvings, the number of steps -- equal.
Those decisions compare max |T^{s+1} - T^s| with eps; the cases keep that
quantity far from eps at every decision (the iterates converge by orders of
magnitude per iteration), so both sides take them in the same FP64.
"""
import ctypes

import numpy as np
import pytest

from oracle import Oracle
from workloads import heat as H

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _pair(p, m, **kw):
    from paper_1912_03744_gb300 import HeatNl
    o = Oracle(p)
    o.nl_setup(m)
    return HeatNl(p, m, **kw), o


def _cell_laws(p, **pulse):
    """The five-region cell with synthetic laws: k ~ T, C ~ T^1.5 around the
    seeded constants, the heater's resistivity ~ T, over 250..900 K."""
    return H.nl_power_laws(p, 250.0, 900.0, 14, a_k=[1.0, 0.5, 1.2, 0.8, 1.0], a_C=[1.5, 1.0, 1.5, 1.0, 1.5],
                           a_chi=1.0, T_ref=300.0, j2=1.0, **pulse)


@pytest.mark.gpu
@pytest.mark.parametrize("face_mean", [H.FACE_HARMONIC, H.FACE_ARITH])
def test_constant_tables_match_the_linear_path(gpu, face_mean):
    """Temperature-independent tables: the full method is the linear step (two
    iterations per half-step), on the GPU as in the oracle."""
    from paper_1912_03744_gb300 import HeatSolver
    p = H.config1().copy(face_mean=face_mean)
    s, o = _pair(p, H.nl_constant(p))
    tau = H.DT_FACTOR * Oracle(p).tau_exp()
    lin = HeatSolver(p, tau, precision="fp64")
    for k in range(5):
        it = s.step(tau)
        ok, i1, i2 = o.nl_step(k * tau, tau, 1e-9, 20)
        assert ok and it == (i1, i2) == (2, 2)
    lin.step(5)
    assert _rel(s.field(), o.field()) <= TOL
    assert _rel(s.field(), lin.field()) <= TOL
    s.close()
    lin.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(64, 128), (37, 53), (130, 70)])
def test_temperature_dependent_steps_match_the_oracle(gpu, shape):
    """The five-region cell heating up under its synthetic laws: each step's
    iterations and field, and the half layer of the last step."""
    p = H.cell_problem(*shape, H.config1().k, H.config1().C, 2e5, name="nl_cell")
    m = _cell_laws(p)
    s, o = _pair(p, m, eps=1e-8, s_max=30)
    tau = 20.0 * Oracle(p).tau_exp()
    its = []
    for k in range(8):
        it = s.step(tau)
        ok, i1, i2 = o.nl_step(k * tau, tau, 1e-8, 30)
        assert ok
        its.append(it)
        assert it == (i1, i2), (k, it, (i1, i2))
    assert max(max(x) for x in its) >= 3, its  # the laws really need iterating
    assert _rel(s.half_field(), o.half_field()) <= TOL
    assert _rel(s.field(), o.field()) <= TOL
    assert np.max(s.field()) > p.T_init + 1.0
    s.close()


@pytest.mark.gpu
def test_halving_matches_the_oracle(gpu):
    """A steep conductivity law (k ~ T^3) at a large tau: ten steps of the
    evolution loop, each halving tau about nine times.  Every halving is a
    decision on max |T^{s+1} - T^s| < eps at iteration s_max, and FP64
    rounding moves that quantity by ~1e-4 of eps here (differences of
    temperatures ~10 K near eps = 1e-10 K), so the test first checks that the
    oracle takes the same decisions at eps (1 -+ 1e-2): none of them lies
    within rounding of the threshold.  (Over hundreds of steps some would.)"""
    p = H.homogeneous_cylinder(12, 16, R=1.0, Z=2.0, k=1.0, C=1.0, bc=(0, 0, 0, 1), T_bc=(0, 0, 0, 1.0),
                               T_init=1.0, q=40.0)
    m = H.nl_power_laws(p, 0.5, 10.0, 40, a_k=[3.0], a_C=[0.0], a_chi=0.0, T_ref=1.0, j2=1.0, heater=0)
    eps, steps = 1e-10, 10
    decisions = set()
    for f in (1 - 1e-2, 1 + 1e-2):
        o = Oracle(p)
        o.nl_setup(m)
        decisions.add(tuple(o.nl_advance(0.0, 100.0, 0.5, 0.5, eps * f, 6, 1e-9, max_steps=steps)[2][:4]))
    s, o = _pair(p, m, eps=eps, s_max=6, tau_base=0.5, tau_trs=0.5, tau_min=1e-9)
    st = s.advance(100.0, max_steps=steps)
    rc, t, so = o.nl_advance(0.0, 100.0, 0.5, 0.5, eps, 6, 1e-9, max_steps=steps)
    assert rc == -2 and decisions == {tuple(so[:4])}, decisions
    assert s.time == t
    assert (st["steps"], st["halvings"], st["iters1"], st["iters2"]) == tuple(int(x) for x in so[:4]), (st, so)
    assert st["halvings"] > steps and st["tau_smallest"] == so[4]
    assert _rel(s.field(), o.field()) <= TOL
    s.close()


@pytest.mark.gpu
def test_pulsed_source_evolution_on_the_paper_grid(gpu):
    """The paper's example shape: the graded 1210 x 100 grid without terminal
    cap, T0 = 4.2 K, the erf-smoothed pulse (t_per 0.1 s, t_src 0.01 s, t_trs
    1e-4 s), the per-step estimates t_trs/1000 and t_src/100, synthetic laws.
    A window from just before the first switch-off through its transition:
    every step count, iteration sum and the field agree."""
    p, m = H.paper_example_nl()
    m.j2 = m.j2 * 4e3  # a heater source that heats the coating by kelvins per pulse
    kw = dict(eps=1e-9, s_max=20, tau_base=m.t_src / 100, tau_trs=m.t_trs / 1000, tau_min=1e-12)
    s, o = _pair(p, m, **kw)
    t0 = m.t_src - 3e-4
    s.set_time(t0)
    t_end = m.t_src + 1.5 * m.t_trs
    st = s.advance(t_end)
    rc, t, so = o.nl_advance(t0, t_end, kw["tau_base"], kw["tau_trs"], kw["eps"], kw["s_max"], kw["tau_min"])
    assert rc == 0 and s.time == t == t_end
    assert (st["steps"], st["halvings"], st["iters1"], st["iters2"]) == tuple(int(x) for x in so[:4]), (st, so)
    assert st["steps"] > 1000  # the transition ran at t_trs/1000
    Tg, To = s.field(), o.field()
    assert _rel(Tg, To) <= TOL
    assert np.max(To) > p.T_init + 1e-3
    s.close()


@pytest.mark.gpu
def test_nonconvergence_is_reported(gpu):
    """tau_min above what the iteration needs: heat_nl_advance returns
    HEAT_ERR_NOCONV and keeps the last completed step; heat_nl_step at a too
    large tau returns it too and leaves the field and time unchanged."""
    from paper_1912_03744_gb300.heat import HeatError
    p = H.homogeneous_cylinder(12, 16, R=1.0, Z=2.0, k=1.0, C=1.0, bc=(0, 0, 0, 1), T_bc=(0, 0, 0, 1.0),
                               T_init=1.0, q=40.0)
    m = H.nl_power_laws(p, 0.5, 10.0, 40, a_k=[3.0], a_C=[0.0], a_chi=0.0, T_ref=1.0, j2=1.0, heater=0)
    s, _ = _pair(p, m, eps=1e-10, s_max=6, tau_base=0.5, tau_trs=0.5, tau_min=0.3)
    T0 = s.field()
    with pytest.raises(HeatError) as ei:
        s.step(0.5)
    assert ei.value.status == -7
    np.testing.assert_array_equal(s.field(), T0)
    assert s.time == 0.0
    with pytest.raises(HeatError) as ei:
        s.advance(3.0)
    assert ei.value.status == -7
    s.close()


def test_full_method_arguments_rejected_without_gpu():
    """heat_nl_create checks its tables and options on the host before any
    CUDA call."""
    from paper_1912_03744_gb300 import build
    from paper_1912_03744_gb300 import heat as hb
    build.build()
    L = hb.load()
    p = H.config1()
    good = H.nl_constant(p)

    def create(m, **kw):
        keep = []
        args = dict(eps=1e-9, s_max=10, tau_base=1.0, tau_trs=1.0, tau_min=1e-9)
        args.update(kw)
        geo, mat, pulse, opt = hb._marshal_nl(p, m, keep=keep, **args)
        h = ctypes.c_void_p(7)
        st = L.heat_nl_create(ctypes.byref(geo), ctypes.byref(mat), ctypes.byref(pulse), ctypes.byref(opt), None,
                              ctypes.byref(h))
        return st, h

    bad_k = H.nl_constant(p)
    bad_k.k = bad_k.k * 0.0
    knots = H.nl_power_laws(p, 250.0, 900.0, 4, [1.0] * 5, [1.0] * 5, 1.0, 300.0, 1.0)
    knots.T_knots = knots.T_knots[:, ::-1].copy()
    pulse = H.nl_constant(p)
    pulse.model, pulse.t_per, pulse.t_src = H.PULSE_ERF, 0.1, 0.2  # heating longer than the period
    for m, kw in ((bad_k, {}), (knots, {}), (pulse, {}), (good, {"eps": 0.0}), (good, {"s_max": 0}),
                  (good, {"tau_base": -1.0})):
        st, h = create(m, **kw)
        assert st == -1 and h.value is None, (kw, st)
    assert L.heat_nl_step(None, 1.0, None, None) == -1
    assert L.heat_nl_advance(None, 1.0, 1, None) == -1


@pytest.mark.gpu
def test_paper_grid_is_stored_without_void_padding(gpu):
    """Sec. 3, eq. "grid": the paper's example has N_j = 1210 cells in the 80
    rows below z0 = 4 and 800 (the core) in the 20 rows above, M_i = 100 in
    the 800 core columns and 80 in the others.  The full method stores
    exactly those 112,800 cells (not 1210 x 100 = 121,000), and its packed
    field is the rectangular field's stored cells, row by row."""
    from paper_1912_03744_gb300 import HeatNl
    p, m = H.paper_example_nl()
    s = HeatNl(p, m, eps=1e-9, s_max=20, tau_base=m.t_src / 100, tau_trs=m.t_trs / 1000)
    Nj, Mi, n = s.layout()
    assert (Nj[:80] == 1210).all() and (Nj[80:] == 800).all()
    assert (Mi[:800] == 100).all() and (Mi[800:] == 80).all()
    assert n == 80 * 1210 + 20 * 800 == 112800
    s.advance(3 * m.t_trs / 1000)
    T, Tp = s.field(), s.field_packed()
    np.testing.assert_array_equal(Tp, np.concatenate([T[j, :Nj[j]] for j in range(p.Nz)]))
    assert (T[80:, 800:] == p.T_init).all()  # not stored: reported as T_init
    s.close()


@pytest.mark.gpu
def test_layout_with_void_inside_lines(gpu):
    """The five-region cell with its terminal cap: the columns past the core
    have void cells between z = 8 and the cap (kept as identity rows inside
    the column), the rows between z = 8 and 10 end at the core.  Parity with
    the oracle on a ragged grid and the stored count."""
    p = H.cell_problem(45, 61, H.config1().k, H.config1().C, 2e5, name="nl_cell")
    m = _cell_laws(p)
    s, o = _pair(p, m, eps=1e-8, s_max=30)
    reg = o.grid()["region"]
    Nj, Mi, n = s.layout()
    want_Nj = np.array([np.max(np.nonzero(reg[j] >= 0)[0]) + 1 for j in range(p.Nz)])
    want_Mi = np.array([np.max(np.nonzero(reg[:, i] >= 0)[0]) + 1 for i in range(p.Nr)])
    np.testing.assert_array_equal(Nj, want_Nj)
    np.testing.assert_array_equal(Mi, want_Mi)
    assert n == want_Nj.sum() < p.Nr * p.Nz
    tau = 20.0 * Oracle(p).tau_exp()
    for k in range(4):
        it = s.step(tau)
        ok, i1, i2 = o.nl_step(k * tau, tau, 1e-8, 30)
        assert ok and it == (i1, i2)
    assert _rel(s.field(), o.field()) <= TOL
    s.close()
