"""Pins of the oracle's full method: temperature-dependent coefficients with
the simple iteration (Sec. 3, eqs. "iter_scheme_eq_1", "iter_scheme_eq_2",
"iter_cond"), adaptive tau (Sec. 3 and 4) and the pulsed source (Sec. 2,
eqs. "unit_model", "trans_model").

None compares the oracle with itself alone: the linear special case is the
already pinned linear oracle; the steady profile under a linear conductivity
law is the Kirchhoff-transform closed form; a manufactured solution with
temperature-dependent k and C checks the order of accuracy; the pulse
functions are checked at values the definitions fix (half height at the
transition midpoint, the rectangular limit, periodicity); tau halving is
checked against a plain step of the halved length.
"""
import numpy as np
import pytest

from oracle import Oracle, pulse
from workloads import heat as H


# ------------------------------------------------- the linear special case
@pytest.mark.parametrize("face_mean", [H.FACE_HARMONIC, H.FACE_ARITH])
def test_constant_tables_reproduce_the_linear_step(face_mean):
    """With temperature-independent tables the iteration is exact after one
    solve: the second iterate equals the first (2 iterations per half-step)
    and the field is the linear step's, bit for bit."""
    p = H.config1().copy(face_mean=face_mean)
    a, b = Oracle(p), Oracle(p)
    a.nl_setup(H.nl_constant(p))
    T0 = H.random_field(p, seed=4, amp=30.0)
    reg = a.grid()["region"]
    T0[reg < 0] = p.T_init
    a.set_field(T0)
    b.set_field(T0)
    tau = H.DT_FACTOR * b.tau_exp()
    for s in range(4):
        ok, i1, i2 = a.nl_step(s * tau, tau, 1e-9, 10)
        b.step(tau)
        assert ok and (i1, i2) == (2, 2)
        np.testing.assert_array_equal(a.field(), b.field())


# --------------------------------------------- Kirchhoff steady closed form
def _kirchhoff_error(n, k0=2.0, beta=0.02, Ta=10.0, Tb=50.0):
    """Steady radial conduction through an annulus 1 <= r <= 2 with
    k(T) = k0 (1 + beta T), T = Ta at r = 1 and Tb at r = 2.  The Kirchhoff
    variable U = k0 (T + beta T^2 / 2) solves the linear problem, so
    U = Ua + (Ub - Ua) ln r / ln 2 and T = (sqrt(1 + 2 beta U / k0) - 1) / beta."""
    p = H.layered_annulus([1.0, 2.0], [n], [k0], T_a=Ta, T_b=Tb, Nz=1)
    o = Oracle(p)
    o.nl_setup(H.nl_linear_laws(p, beta, 0.0, 0.0, 100.0))
    mu_max = 4.0 * k0 * (1 + beta * Tb) * n * n
    taus = 2.0 / np.geomspace(1e-2, mu_max, 24)
    t = 0.0
    for _ in range(40):
        for tau in taus:
            ok, _, _ = o.nl_step(t, tau, 1e-11, 60)
            assert ok
            t += tau
    rc = o.grid()["rc"]
    U = lambda T: k0 * (T + 0.5 * beta * T * T)  # noqa: E731
    Ur = U(Ta) + (U(Tb) - U(Ta)) * np.log(rc) / np.log(2.0)
    exact = (np.sqrt(1.0 + 2.0 * beta * Ur / k0) - 1.0) / beta
    return np.max(np.abs(o.field()[0] - exact))


def test_kirchhoff_steady_profile_second_order():
    """Steady state of the full method against the Kirchhoff closed form: the
    error falls towards order 2 (1.79 and 1.90 over 20 -> 40 -> 80 cells; the
    conductivity at a Dirichlet face is the cell's, an O(h) error over half a
    cell, which keeps the coarse grids pre-asymptotic)."""
    errs = [_kirchhoff_error(n) for n in (20, 40, 80)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3, errs
    assert np.all(orders > 1.7) and orders[-1] > 1.85, (errs, orders)


def test_kirchhoff_profile_differs_from_the_constant_law():
    """The same annulus with beta = 0 has the plain log profile; the two
    steady states must differ by far more than the discretisation error, so
    the previous test sees the conductivity law and not only the geometry."""
    assert _kirchhoff_error(20, beta=0.02) < 0.05 * abs(
        _kirchhoff_error(20, beta=0.02) - _kirchhoff_error_vs_linear(20))


def _kirchhoff_error_vs_linear(n, k0=2.0, beta=0.02, Ta=10.0, Tb=50.0):
    """Distance of the nonlinear steady state from the constant-k closed form."""
    p = H.layered_annulus([1.0, 2.0], [n], [k0], T_a=Ta, T_b=Tb, Nz=1)
    o = Oracle(p)
    o.nl_setup(H.nl_linear_laws(p, beta, 0.0, 0.0, 100.0))
    mu_max = 4.0 * k0 * (1 + beta * Tb) * n * n
    taus = 2.0 / np.geomspace(1e-2, mu_max, 24)
    t = 0.0
    for _ in range(40):
        for tau in taus:
            o.nl_step(t, tau, 1e-11, 60)
            t += tau
    rc = o.grid()["rc"]
    lin = Ta + (Tb - Ta) * np.log(rc) / np.log(2.0)
    return np.max(np.abs(o.field()[0] - lin))


# ------------------------------------------ manufactured solution, k(T), C(T)
def _mms_nl_error(N, R=1.0, Z=1.0, k0=1.3, C0=0.8, beta=0.3, gamma=0.2, T0=2.0, t_end=0.2):
    """T* = T0 + e^-t cos(pi r/R) cos(pi z/2Z) with k = k0 (1 + beta T) and
    C = C0 (1 + gamma T): the source is
    X = C(T*) dT*/dt - k(T*) (T*_rr + T*_r / r + T*_zz) - k0 beta (T*_r^2 + T*_z^2),
    evaluated at t_k + tau/2 and passed in per cell."""
    p = H.homogeneous_cylinder(N, N, R=R, Z=Z, k=k0, C=C0, T_bc=(0, 0, 0, T0), T_init=T0)
    o = Oracle(p)
    o.nl_setup(H.nl_linear_laws(p, beta, gamma, 0.0, 5.0))
    g = o.grid()
    r, z = np.meshgrid(g["rc"], g["zc"])
    a, b = np.pi / R, np.pi / (2 * Z)

    def exact(t):
        return T0 + np.exp(-t) * np.cos(a * r) * np.cos(b * z)

    def source(t):
        A = np.exp(-t)
        T = exact(t)
        Tt = -A * np.cos(a * r) * np.cos(b * z)
        Tr = -A * a * np.sin(a * r) * np.cos(b * z)
        Trr = -A * a * a * np.cos(a * r) * np.cos(b * z)
        Tz = -A * b * np.cos(a * r) * np.sin(b * z)
        Tzz = -A * b * b * np.cos(a * r) * np.cos(b * z)
        k = k0 * (1 + beta * T)
        C = C0 * (1 + gamma * T)
        return C * Tt - k * (Trr + Tr / r + Tzz) - k0 * beta * (Tr * Tr + Tz * Tz)

    o.set_field(exact(0.0))
    steps = N
    tau = t_end / steps
    for s in range(steps):
        ok, _, _ = o.nl_step(s * tau, tau, 1e-13, 60, X=source(s * tau + 0.5 * tau))
        assert ok
    return np.max(np.abs(o.field() - exact(t_end)))


def test_manufactured_solution_with_temperature_dependent_k_and_C_second_order():
    errs = [_mms_nl_error(N) for N in (8, 16, 32)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)


# ------------------------------------------------------------ pulse p(t)
T_PER, T_SRC, T_TRS = 0.1, 0.01, 1e-4


def test_rectangular_pulse_values():
    """u(t) = sum_n [theta(t - n t_per) - theta(t - n t_per - t_src)]: 1 inside
    each pulse (including its first instant, theta(0) = 1), 0 between."""
    on = [0.0, 0.5 * T_SRC, T_PER, T_PER + 0.999 * T_SRC, 7 * T_PER + 0.3 * T_SRC]
    off = [T_SRC, 0.5 * T_PER, T_PER - 1e-9, 2 * T_PER + T_SRC, 7 * T_PER + 0.7 * T_PER]
    for t in on:
        assert pulse(H.PULSE_RECT, t, T_PER, T_SRC, T_TRS) == 1.0, t
    for t in off:
        assert pulse(H.PULSE_RECT, t, T_PER, T_SRC, T_TRS) == 0.0, t
    assert pulse(H.PULSE_CONST, 0.37, T_PER, T_SRC, T_TRS) == 1.0


def test_smoothed_pulse_values():
    """v(t): half height where each erf argument crosses zero (t_trs/zeta after
    a switch), 1 inside a pulse and 0 between pulses to rounding, periodic in
    t_per, and between 0 and 1."""
    xi, zeta = 4.0, 2.0
    v = lambda t: pulse(H.PULSE_ERF, t, T_PER, T_SRC, T_TRS, xi, zeta)  # noqa: E731
    # the erf argument xi (zeta (t - t0)/t_trs - 1) carries the rounding of t
    # magnified by xi zeta t / t_trs (up to 4e4 here), so "half height" holds
    # to ~1e-16 x 4e4 x erf'(0) ~ 5e-12
    for n in (0, 1, 5):
        t0 = n * T_PER
        assert abs(v(t0 + T_TRS / zeta) - 0.5) < 5e-12
        assert abs(v(t0 + T_SRC + T_TRS / zeta) - 0.5) < 5e-12
        assert abs(v(t0 + 0.5 * T_SRC) - 1.0) < 1e-15
        assert abs(v(t0 + 0.5 * (T_SRC + T_PER))) < 1e-15
    ts = np.linspace(0.0, 3 * T_PER, 3001)
    vs = np.array([v(t) for t in ts])
    assert vs.min() >= -1e-15 and vs.max() <= 1.0 + 1e-15
    for t in ts[::37]:
        assert abs(v(t + T_PER) - v(t)) < 1e-14


def test_smoothed_pulse_tends_to_the_shifted_rectangle():
    """As xi grows the transitions sharpen: v(t) -> u(t - t_trs/zeta) away from
    the switch instants."""
    zeta = 2.0
    sh = T_TRS / zeta
    for t in np.linspace(0.0, 2 * T_PER, 401):
        if min(abs((t - sh) % T_PER), abs((t - sh - T_SRC) % T_PER), abs((t - sh) % T_PER - T_PER)) < 1e-6:
            continue
        want = pulse(H.PULSE_RECT, t - sh, T_PER, T_SRC, T_TRS) if t >= sh else 0.0
        assert abs(pulse(H.PULSE_ERF, t, T_PER, T_SRC, T_TRS, 1e7, zeta) - want) < 1e-12, t


def test_source_is_taken_at_the_half_layer():
    """With constant tables and the rectangular pulse, a step of the full
    method equals the linear step whose source is q p(t_k + tau/2): the step
    that ends past the switch-off with its midpoint still inside the pulse
    keeps the full source, the next one (midpoint outside) has none."""
    p = H.config1()
    # (start, length, p at the midpoint): the first step ends past the
    # switch-off with its midpoint inside the pulse; the second starts inside
    # the pulse with its midpoint past the switch-off
    for t, tau, p_mid in ((0.0, 1.2 * T_SRC, 1.0), (0.8 * T_SRC, 0.6 * T_SRC, 0.0)):
        a, b = Oracle(p), Oracle(p.copy(q=p.q * p_mid))
        m = H.nl_constant(p)
        m.model, m.t_per, m.t_src, m.t_trs = H.PULSE_RECT, T_PER, T_SRC, T_TRS
        a.nl_setup(m)
        ok, _, _ = a.nl_step(t, tau, 1e-9, 10)
        b.step(tau)
        assert ok
        np.testing.assert_array_equal(a.field(), b.field())


# ---------------------------------------------------------- adaptive tau
def _stiff_problem():
    """A cylinder whose conductivity rises steeply with T (k ~ T^3): the
    simple iteration converges slowly at large tau."""
    p = H.homogeneous_cylinder(12, 16, R=1.0, Z=2.0, k=1.0, C=1.0, bc=(0, 0, 0, 1), T_bc=(0, 0, 0, 1.0),
                               T_init=1.0, q=40.0)
    m = H.nl_power_laws(p, 0.5, 10.0, 40, a_k=[3.0], a_C=[0.0], a_chi=0.0, T_ref=1.0, j2=1.0, heater=0)
    return p, m


def test_tau_is_halved_until_the_iteration_converges():
    """Sec. 3/4: when s_max iterations do not meet the criterion, tau is
    halved and the step restarts from the old layer.  One step from a tau
    that needs more than s_max iterations must equal one plain step of the
    halved tau it reports (the failed attempts leave no trace)."""
    p, m = _stiff_problem()
    eps, s_max = 1e-10, 6
    a = Oracle(p)
    a.nl_setup(m)
    tau0 = 0.5
    rc, t, st = a.nl_advance(0.0, 10.0, tau0, tau0, eps, s_max, 1e-9, max_steps=1)
    assert rc == -2 and st[0] == 1 and st[1] >= 1, (rc, st)
    tau_used = st[4]
    assert tau_used == tau0 / 2 ** int(st[1]) and t == tau_used
    b = Oracle(p)
    b.nl_setup(m)
    ok, i1, i2 = b.nl_step(0.0, tau_used, eps, s_max)
    assert ok and i1 + i2 == st[2] + st[3]
    np.testing.assert_array_equal(a.field(), b.field())
    c = Oracle(p)
    c.nl_setup(m)
    ok, _, _ = c.nl_step(0.0, 2 * tau_used, eps, s_max)
    assert not ok  # the previous length really fails


def test_evolution_lands_on_the_end_time_and_reports_steps():
    """The loop of Sec. 4: tau restarts from the estimate at every step
    (t_trs/1000 in a transition of the pulse, t_src/100 elsewhere) and the
    last step is shortened to end at t_end exactly."""
    p = H.config1()
    m = H.nl_constant(p)
    m.model, m.t_per, m.t_src, m.t_trs = H.PULSE_ERF, T_PER, T_SRC, T_TRS
    o = Oracle(p)
    o.nl_setup(m)
    t_end = 0.5 * T_SRC + 3.3e-5
    rc, t, st = o.nl_advance(0.0, t_end, T_SRC / 100, T_TRS / 1000, 1e-9, 10, 1e-12)
    assert rc == 0 and t == t_end
    # [0, t_trs): 1000 steps of t_trs/1000; then (t_end - t_trs) / (t_src/100) steps, the last shortened
    n_trs = 1000
    n_base = int(np.ceil((t_end - T_TRS) / (T_SRC / 100) - 1e-9))
    assert abs(st[0] - (n_trs + n_base)) <= 1, st
    # constant tables: one solve is exact, so each half-step stops after two
    # iterations, or after one where the step changes the field by less than eps
    assert st[1] == 0 and st[0] <= st[2] <= 2 * st[0] and st[0] <= st[3] <= 2 * st[0], st


# ------------------------------------------ time levels, exact special cases
def test_uniform_cell_is_the_implicit_midpoint_rule():
    """A uniform, insulated cylinder of one material with C = C0 (1 + g T) and
    X = chi0 (1 + a T) j^2: every difference vanishes, so eq. "iter_scheme_eq_1"
    converges to Tbar = T + (tau/2) X(Tbar) / C(Tbar) (capacity and source at
    the iterate) and eq. "iter_scheme_eq_2" gives That = Tbar + (tau/2)
    X(Tbar) / C(Tbar) (both at Tbar, not iterated): the implicit midpoint rule
    of C dT/dt = X.  Tbar is found here with scipy's brentq."""
    import scipy.optimize
    C0, g, chi0, a, j2, T0, tau = 2.0, 0.05, 3.0, 0.02, 4.0, 10.0, 0.7
    p = H.homogeneous_cylinder(3, 4, R=1.0, Z=1.0, k=1.5, C=C0, bc=(0, 0, 0, 0), T_init=T0, q=0.0)
    m = H.NlMaterials(T_knots=np.array([[0.0, 100.0]]), k=np.array([[1.5, 1.5]]),
                      C=np.array([[C0, C0 * (1 + g * 100.0)]]), chi=np.array([[chi0, chi0 * (1 + a * 100.0)]]),
                      j2=np.array([j2]))
    o = Oracle(p)
    o.nl_setup(m)
    ok, _, _ = o.nl_step(0.0, tau, 1e-13, 60)
    assert ok

    def f(T):
        return chi0 * (1 + a * T) * j2 / (C0 * (1 + g * T))

    Tbar = scipy.optimize.brentq(lambda T: T - T0 - 0.5 * tau * f(T), T0, T0 + 10.0, xtol=1e-15, rtol=1e-15)
    That = Tbar + 0.5 * tau * f(Tbar)
    np.testing.assert_allclose(o.half_field(), Tbar, rtol=1e-14)
    np.testing.assert_allclose(o.field(), That, rtol=1e-14)


def test_one_column_half_step_is_explicit_in_z_at_the_old_layer():
    """One radial cell (no r-couplings): half-step 1 is the explicit Euler
    half-step T + (tau/2) Lambda_z[T] / C with the face conductivities of
    Lambda_z taken at the old layer T, k(T) = k0 (1 + b T), harmonic face means
    of equal half widths 2 ka kb / (ka + kb), insulated ends; written out here
    for the uniform column."""
    N, Z, k0, b, C, tau = 9, 3.0, 2.0, 0.04, 1.7, 0.01
    p = H.homogeneous_cylinder(1, N, R=1.0, Z=Z, k=k0, C=C, bc=(0, 0, 0, 0), T_init=0.0, q=0.0)
    o = Oracle(p)
    o.nl_setup(H.nl_linear_laws(p, b, 0.0, 0.0, 200.0))
    T = np.linspace(20.0, 80.0, N) + 7.0 * np.sin(np.arange(N))
    o.set_field(T.reshape(N, 1))
    ok, _, _ = o.nl_step(0.0, tau, 1e-13, 60)
    assert ok
    dz = Z / N
    k = k0 * (1 + b * T)
    kf = 2 * k[1:] * k[:-1] / (k[1:] + k[:-1])
    flux = np.zeros(N + 1)
    flux[1:-1] = kf * (T[1:] - T[:-1]) / dz
    Tbar = T + 0.5 * tau * (flux[1:] - flux[:-1]) / dz / C
    np.testing.assert_allclose(o.half_field()[:, 0], Tbar, rtol=1e-13)


def test_no_step_passes_over_a_transition():
    """A base step that would cross the switch-off ends at it, and the
    transition then runs at t_trs/1000: from 2.5 base steps before the switch,
    two full steps and a half one reach it, 1000 transition steps follow, then
    base steps to t_end."""
    p = H.config1()
    m = H.nl_constant(p)
    m.model, m.t_per, m.t_src, m.t_trs = H.PULSE_ERF, T_PER, T_SRC, T_TRS
    o = Oracle(p)
    o.nl_setup(m)
    base = T_SRC / 100
    t0 = T_SRC - 2.5 * base
    t_end = T_SRC + T_TRS + 3 * base
    rc, t, st = o.nl_advance(t0, t_end, base, T_TRS / 1000, 1e-9, 10, 1e-12)
    assert rc == 0 and t == t_end
    assert abs(st[0] - (3 + 1000 + 3)) <= 1, st
    assert st[4] < 0.6 * base and st[4] >= T_TRS / 1000 * (1 - 1e-9)
