"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: they use a library banded
solver, closed-form solutions of the PDE (layered logarithmic profile, Bessel
J0 mode decay), a manufactured solution's convergence order, the exact
discrete heat balance under which the scheme telescopes, dense direct solves
of the assembled 2D systems, and a 2x1 grid worked by hand.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.special

from oracle import Oracle, thomas
from workloads import heat as H


# ------------------------------------------------------------------ I5a
def test_thomas_matches_banded_solver():
    """Textbook Thomas (Sec. 3, the line solver) equals scipy's banded LU."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 17, 200):
        a = -rng.uniform(0, 1, n)
        c = -rng.uniform(0, 1, n)
        b = rng.uniform(0.1, 1, n) - a - c  # diagonally dominant like the ADI systems
        d = rng.standard_normal(n)
        x = thomas(a, b, c, d)
        ab = np.zeros((3, n))
        ab[0, 1:] = c[:-1]
        ab[1] = b
        ab[2, :-1] = a[1:]
        ref = scipy.linalg.solve_banded((1, 1), ab, d)
        np.testing.assert_allclose(x, ref, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------------- I6
def _two_cell_problem():
    # Two radial layers of one cell each, one axial cell: r in [0,1] region 0,
    # r in [1,3] region 1, z in [0,2]; Dirichlet T=10 on the top face z=2.
    return H.Problem(
        name="hand2x1", r_faces=np.array([0.0, 1.0, 3.0]), r_cells=np.array([1, 1], np.int32),
        z_faces=np.array([0.0, 2.0]), z_cells=np.array([1], np.int32),
        boxes=np.array([[0.0, 1.0, 0.0, 2.0], [1.0, 3.0, 0.0, 2.0]]),
        box_region=np.array([0, 1], np.int32),
        bc=np.array([0, 0, 0, 1], np.int32), T_bc=np.array([0.0, 0.0, 0.0, 10.0]),
        k=np.array([2.0, 5.0]), C=np.array([1.0, 3.0]), q=np.array([4.0, 0.0]), T_init=0.0)


def test_two_cell_step_by_hand():
    """One PR step on a 2x1 grid, every number worked by hand from Sec. 3.

    Centres r0 = 0.5, r1 = 2; h0 = 2*0.5 = 1 (mirror ghost), h1 = 1.5, h2 = 2*(3-2) = 2;
    hbar0 = 1.25, hbar1 = 1.75; r_{1/2} = 1.25.  Interface conductivity
    (harmonic, half widths 0.5 and 1): 1.5 / (0.5/2 + 1/5) = 10/3.
    Arp(0) = 1.25*(10/3) / (0.5*1.25*1.5) = 40/9;  Arm(1) = 1.25*(10/3) / (2*1.75*1.5) = 50/63.
    z: one cell of height 2, eta0 = eta1 = 2, etabar = 2; Dirichlet coefficient
    2 k / (etabar * eta1) = k/2: 1 for cell 0, 5/2 for cell 1.
    tau = 0.5 -> w = C/(tau/2) = 4 and 12.  T = (1, 2) initially.
    """
    p = _two_cell_problem()
    o = Oracle(p)
    T = np.array([[1.0, 2.0]])
    o.set_field(T)
    tau = 0.5
    o.step(tau)
    Arp0, Arm1 = 40.0 / 9.0, 50.0 / 63.0
    D0, D1 = 1.0, 2.5
    w0, w1 = 4.0, 12.0
    q0, q1 = 4.0, 0.0
    # half-step 1: implicit in r, explicit z (the Dirichlet term), source q
    A1 = np.array([[w0 + Arp0, -Arp0], [-Arm1, w1 + Arm1]])
    rhs1 = np.array([w0 * 1.0 + D0 * (10.0 - 1.0) + q0, w1 * 2.0 + D1 * (10.0 - 2.0) + q1])
    Tbar = np.linalg.solve(A1, rhs1)
    np.testing.assert_allclose(o.half_field()[0], Tbar, rtol=1e-14)
    # half-step 2: explicit r at Tbar, implicit z (Dirichlet on the diagonal)
    Lr = np.array([Arp0 * (Tbar[1] - Tbar[0]), Arm1 * (Tbar[0] - Tbar[1])])
    That = (np.array([w0, w1]) * Tbar + Lr + np.array([q0, q1]) + np.array([D0, D1]) * 10.0) / \
        (np.array([w0, w1]) + np.array([D0, D1]))
    np.testing.assert_allclose(o.field()[0], That, rtol=1e-14)
    # and the grid numbers themselves
    g = o.grid()
    np.testing.assert_allclose(g["rc"], [0.5, 2.0])
    np.testing.assert_allclose(g["hbar"], [1.25, 1.75])
    np.testing.assert_allclose(g["etabar"], [2.0])
    c = o.coeffs()
    np.testing.assert_allclose([c["Arp"][0, 0], c["Arm"][0, 1], c["Dzh"][0, 0], c["Dzh"][0, 1]],
                               [Arp0, Arm1, D0, D1], rtol=1e-14)


# ------------------------------------------------------------- C8 limit
def test_explicit_limit_by_hand():
    """tau_exp = min over active cells of C / (sum of the cell's couplings),
    the forward-Euler positivity limit of the assembled operator (reading of
    the workload's "50x the explicit stability limit"), worked by hand.

    2x1 grid of ``_two_cell_problem``: cell 0 has Arp = 40/9 and the Dirichlet
    coefficient 1, C = 1 -> 9/49; cell 1 has Arm = 50/63 and 5/2, C = 3 ->
    378/415.  The limit is 9/49, set by the Dirichlet-coupled cell 0.
    """
    o = Oracle(_two_cell_problem())
    assert abs(o.tau_exp() - 9.0 / 49.0) <= 1e-15


def _void_corner_problem():
    # 2x2 grid: r faces 0, 1, 3 (one cell each), z faces 0, 2, 4 (one cell
    # each).  Region 0 (k 2, C 1) at the bottom left, region 2 (k 20, C 1)
    # above it, region 1 (k 5, C 3) at the bottom right; the top right cell is
    # in no box (void).  Dirichlet T = 10 on the top face z = 4.
    return H.Problem(
        name="hand2x2", r_faces=np.array([0.0, 1.0, 3.0]), r_cells=np.array([1, 1], np.int32),
        z_faces=np.array([0.0, 2.0, 4.0]), z_cells=np.array([1, 1], np.int32),
        boxes=np.array([[0.0, 1.0, 0.0, 2.0], [1.0, 3.0, 0.0, 2.0], [0.0, 1.0, 2.0, 4.0]]),
        box_region=np.array([0, 1, 2], np.int32),
        bc=np.array([0, 0, 0, 1], np.int32), T_bc=np.array([0.0, 0.0, 0.0, 10.0]),
        k=np.array([2.0, 5.0, 20.0]), C=np.array([1.0, 3.0, 1.0]), q=np.zeros(3), T_init=0.0)


def test_explicit_limit_with_void_and_dirichlet_by_hand():
    """The limit on a grid with a void cell and a Dirichlet face, by hand.

    z: centres 1, 3; eta = 2 everywhere (mirror ghosts), etabar = 2.
    r: as the 2x1 case (Arp(0) = 40/9, Arm(1) = 50/63).
    Bottom-left (k 2) to top-left (k 20) face: harmonic mean with half widths
    1 and 1, 2 / (1/2 + 1/20) = 40/11; Azp = Azm = (40/11) / (2 * 2) = 10/11.
    Cells (sum of couplings, C / sum):
      (0,0): 40/9 + 10/11 = 530/99            -> 99/530 ~ 0.1868
      (1,0): 50/63 (the void neighbour above adds nothing) -> 3 * 63/50 = 3.78
      (0,1): Azm 10/11 + Dirichlet 2*20/(2*2) = 10 (the void neighbour to the
             right adds nothing) = 120/11    -> 11/120 ~ 0.0917
    The void cell is excluded.  Limit: 11/120, set by the Dirichlet face.
    """
    o = Oracle(_void_corner_problem())
    assert (o.grid()["region"] == np.array([[0, 1], [2, -1]])).all()
    c = o.coeffs()
    np.testing.assert_allclose([c["Azp"][0, 0], c["Azm"][1, 0], c["Dzh"][1, 0], c["Arp"][1, 0]],
                               [10.0 / 11.0, 10.0 / 11.0, 10.0, 0.0], rtol=1e-14)
    assert abs(o.tau_exp() - 11.0 / 120.0) <= 1e-15


@pytest.mark.parametrize("top", [H.BC_NEUMANN, H.BC_DIRICHLET])
def test_explicit_limit_of_a_uniform_column_is_textbook(top):
    """One radial cell, N uniform axial cells of height dz, conductivity k,
    capacity C: the interior cells give the textbook explicit limit of the 1D
    heat equation, C dz^2 / (2k); a Dirichlet face at half a cell from the
    last centre adds 2k/dz^2 there, giving C dz^2 / (3k)."""
    k, C, Z, N = 3.0, 5.0, 2.0, 8
    p = H.homogeneous_cylinder(1, N, R=1.0, Z=Z, k=k, C=C, bc=(0, 0, 0, top),
                               T_bc=(0.0, 0.0, 0.0, 1.0), T_init=0.0, q=0.0)
    dz = Z / N
    want = C * dz * dz / ((3.0 if top == H.BC_DIRICHLET else 2.0) * k)
    assert abs(Oracle(p).tau_exp() - want) <= 1e-14 * want


# ------------------------------------------------------------------- I0
def _assemble(o, T, tau, implicit):
    """Dense 2D system of one half-step from the oracle's per-cell couplings."""
    c = o.coeffs()
    g = o.grid()
    Nr, Nz = o.Nr, o.Nz
    n = Nr * Nz
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    Tb = o.problem.T_bc
    act = g["region"] >= 0
    for j in range(Nz):
        for i in range(Nr):
            r = j * Nr + i
            if not act[j, i]:
                A[r, r] = 1.0
                rhs[r] = T[j, i]
                continue
            w = c["C"][j, i] / (0.5 * tau)
            nb_r = [(-1, 0, c["Arm"][j, i]), (1, 0, c["Arp"][j, i])]
            nb_z = [(0, -1, c["Azm"][j, i]), (0, 1, c["Azp"][j, i])]
            Dr = [(c["Drl"][j, i], Tb[0]), (c["Drh"][j, i], Tb[1])]
            Dz = [(c["Dzl"][j, i], Tb[2]), (c["Dzh"][j, i], Tb[3])]
            imp, exp_ = (nb_r, nb_z) if implicit == "r" else (nb_z, nb_r)
            Dimp, Dexp = (Dr, Dz) if implicit == "r" else (Dz, Dr)
            A[r, r] = w
            rhs[r] = w * T[j, i] + c["q"][j, i]
            for di, dj, a in imp:
                if a != 0.0:
                    A[r, r] += a
                    A[r, (j + dj) * Nr + (i + di)] -= a
            for D, v in Dimp:
                A[r, r] += D
                rhs[r] += D * v
            for di, dj, a in exp_:
                if a != 0.0:
                    rhs[r] += a * (T[j + dj, i + di] - T[j, i])
            for D, v in Dexp:
                rhs[r] += D * (v - T[j, i])
    return A, rhs


# radial faces and cells per layer for each tiny case; z cells over (8, 2, 0.2)
_TINY = {
    (3, 4): ((0.0, 2.0, 3.0, 4.2), (1, 1, 1), (2, 1, 1)),
    (5, 6): ((0.0, 2.0, 3.0, 4.0, 4.2), (2, 1, 1, 1), (3, 2, 1)),
    (8, 12): ((0.0, 2.0, 3.0, 4.0, 4.2), (3, 2, 2, 1), (7, 3, 2)),
}


@pytest.mark.parametrize("shape", sorted(_TINY))
def test_line_solves_equal_dense_direct_solve(shape):
    """Both half-steps equal a dense LU solve of the assembled 2D system (I0),
    on the five-region cell (void, interfaces, Dirichlet top)."""
    Nr, Nz = shape
    rf, rcells, zcells = _TINY[shape]
    rng = np.random.default_rng(Nr * 100 + Nz)
    k, C = rng.uniform(0.5, 5, 5), rng.uniform(1, 3, 5)
    p = H.cell_problem(8, 6, k, C, 2.0)
    p = p.copy(r_faces=np.array(rf), r_cells=np.array(rcells, np.int32),
               z_cells=np.array(zcells, np.int32))
    o = Oracle(p)
    assert (o.Nr, o.Nz) == (Nr, Nz)
    T0 = H.random_field(p, seed=7)
    reg = o.grid()["region"]
    T0[reg < 0] = p.T_init
    o.set_field(T0)
    tau = 3.0 * o.tau_exp()
    o.step(tau)
    A1, b1 = _assemble(o, T0, tau, "r")
    Tbar = np.linalg.solve(A1, b1).reshape(Nz, Nr)
    np.testing.assert_allclose(o.half_field(), Tbar, rtol=1e-13, atol=1e-12)
    A2, b2 = _assemble(o, Tbar, tau, "z")
    That = np.linalg.solve(A2, b2).reshape(Nz, Nr)
    np.testing.assert_allclose(o.field(), That, rtol=1e-13, atol=1e-12)
    assert (reg < 0).any(), "the case must contain void cells"


# ------------------------------------------------------------------- I3
@pytest.mark.parametrize("face_mean", [H.FACE_HARMONIC, H.FACE_ARITH])
def test_exact_heat_balance(face_mean):
    """E(That) - E(T) = tau Q + (tau/2)(Phi(T) + Phi(That)) to roundoff: the
    scheme telescopes under the weights r_i hbar_i etabar_j (Sec. 3)."""
    p = H.config1().copy(face_mean=face_mean)
    o = Oracle(p)
    reg = o.grid()["region"]
    T = H.random_field(p, seed=3, amp=50.0)
    T[reg < 0] = p.T_init
    o.set_field(T)
    for tau in (0.3 * o.tau_exp(), 50 * o.tau_exp()):
        E0, F0, Q = o.energy()
        o.step(tau)
        E1, F1, _ = o.energy()
        lhs = E1 - E0
        rhs = tau * Q + 0.5 * tau * (F0 + F1)
        assert abs(lhs - rhs) <= 1e-12 * abs(E0), (lhs, rhs)
        assert abs(F0) > 0 and abs(lhs) > 1e-6 * abs(E0)


def test_insulated_heat_balance_is_source_only():
    p = H.config1()
    p = p.copy(bc=np.zeros(4, np.int32))
    o = Oracle(p)
    reg = o.grid()["region"]
    T = H.random_field(p, seed=5, amp=20.0)
    T[reg < 0] = p.T_init
    o.set_field(T)
    tau = 20 * o.tau_exp()
    E0, F0, Q = o.energy()
    o.step(tau, 3)
    E1, F1, _ = o.energy()
    assert F0 == 0.0 and F1 == 0.0
    assert abs((E1 - E0) - 3 * tau * Q) <= 1e-12 * abs(E0)


# ------------------------------------------------------------------- I1
def _annulus_steady(n, k, face_mean=H.FACE_HARMONIC):
    radii = np.array([1.0, 1.3, 1.7, 2.0])
    p = H.layered_annulus(radii, [n, n, n], k, T_a=100.0, T_b=0.0, Nz=1)
    p = p.copy(face_mean=face_mean)
    o = Oracle(p)
    c = o.coeffs()
    mu_max = float(np.max(c["Arm"] + c["Arp"] + c["Drl"] + c["Drh"]))
    mu_min = 1e-2
    taus = 2.0 / np.geomspace(mu_min, mu_max, 24)
    for _ in range(60):
        for t in taus:
            o.step(t)
    T = o.field()[0]
    # closed form: T = T(rho_m) - F ln(r/rho_m)/k_m, F = (T_a - T_b) / sum ln(rho_{m+1}/rho_m)/k_m
    R = np.log(radii[1:] / radii[:-1]) / np.asarray(k)
    F = 100.0 / R.sum()
    Tface = 100.0 - F * np.concatenate([[0.0], np.cumsum(R)])
    rc = o.grid()["rc"]
    m = np.searchsorted(radii, rc) - 1
    exact = Tface[m] - F * np.log(rc / radii[m]) / np.asarray(k)[m]
    return np.max(np.abs(T - exact))


def test_layered_log_profile_second_order():
    """Steady conduction through concentric layers (flux continuity at each
    interface) converges to the exact T = a_m + b_m ln r at O(h^2) (I1)."""
    k = [1.0, 20.0, 0.3]
    errs = [_annulus_steady(n, k) for n in (8, 16, 32)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3, errs
    assert np.all(orders > 1.8), (errs, orders)


def test_arithmetic_face_mean_is_worse_at_contrast():
    """The literal arithmetic face mean is not flux-consistent at a material
    jump: at contrast 400 its error is far above the harmonic one."""
    k = [1.0, 400.0, 1.0]
    e_h = _annulus_steady(16, k, H.FACE_HARMONIC)
    e_a = _annulus_steady(16, k, H.FACE_ARITH)
    assert e_a > 10 * e_h, (e_h, e_a)


# ------------------------------------------------------------------- I2
J1P = scipy.special.jnp_zeros(0, 1)[0]  # first zero of J0' = -J1


def _bessel_error(N, steps, t_end=0.05):
    p = H.homogeneous_cylinder(N, 2, R=1.0, Z=1.0, k=1.0, C=1.0,
                               bc=(0, 0, 0, 0), T_init=0.0)
    o = Oracle(p)
    rc = o.grid()["rc"]
    eps = 1.0
    T0 = np.tile(eps * scipy.special.j0(J1P * rc), (2, 1))
    o.set_field(T0)
    o.step(t_end / steps, steps)
    exact = eps * np.exp(-J1P ** 2 * t_end) * scipy.special.j0(J1P * rc)
    return np.max(np.abs(o.field()[0] - exact))


def test_bessel_mode_decay_second_order():
    """A homogeneous insulated cylinder started at J0(j'_1 r/R) decays as
    exp(-kappa (j'_1/R)^2 t); the error falls at O(h^2 + tau^2) (I2)."""
    errs = [_bessel_error(N, N) for N in (16, 32, 64)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)
    assert errs[-1] < 1e-3


def test_pr_step_is_exact_cayley_map_for_z_uniform_fields():
    """For a z-uniform field the PR step is (I + tau/2 M)(I - tau/2 M)^-1 with M
    the radial operator; its eigenvectors are multiplied by
    (1 - tau mu/2)/(1 + tau mu/2) (I2, exact discrete form)."""
    N = 12
    p = H.homogeneous_cylinder(N, 3, R=1.0, Z=1.0, k=2.0, C=1.5, bc=(0, 0, 0, 0))
    o = Oracle(p)
    c = o.coeffs()
    Arm, Arp, Cc = c["Arm"][0], c["Arp"][0], c["C"][0]
    M = np.diag(-(Arm + Arp)) + np.diag(Arm[1:], -1) + np.diag(Arp[:-1], 1)
    M = M / Cc[:, None]
    lam, V = np.linalg.eig(M)
    tau = 0.37
    for m in (1, 4, N - 1):
        v = np.real(V[:, m])
        o.set_field(np.tile(v, (3, 1)))
        o.step(tau)
        mu = -np.real(lam[m])
        g = (1 - tau * mu / 2) / (1 + tau * mu / 2)
        np.testing.assert_allclose(o.field()[1], g * v, rtol=1e-12, atol=1e-13)
    assert np.min(-np.real(lam)) > -1e-12  # non-negative spectrum


# ------------------------------------------------------------------- I4
def _mms_error(N, R=1.0, Z=1.0, k=1.3, C=0.8, T0=2.0, t_end=0.2):
    p = H.homogeneous_cylinder(N, N, R=R, Z=Z, k=k, C=C, T_bc=(0, 0, 0, T0), T_init=T0)
    o = Oracle(p)
    g = o.grid()
    r, z = np.meshgrid(g["rc"], g["zc"])

    def exact(t):
        return T0 + np.exp(-t) * np.cos(np.pi * r / R) * np.cos(np.pi * z / (2 * Z))

    def source(t):
        A = np.exp(-t)
        gr, hz = np.cos(np.pi * r / R), np.cos(np.pi * z / (2 * Z))
        lap_r = -(np.pi / R) * (np.sin(np.pi * r / R) / r + (np.pi / R) * gr)
        lap_z = -(np.pi / (2 * Z)) ** 2 * gr
        return A * hz * (-C * gr - k * lap_r) - A * hz * k * lap_z

    o.set_field(exact(0.0))
    steps = N
    tau = t_end / steps
    for s in range(steps):
        o.step_src(tau, source(s * tau + 0.5 * tau))
    return np.max(np.abs(o.field() - exact(t_end)))


def test_manufactured_solution_second_order():
    """T* = T0 + e^-t cos(pi r/R) cos(pi z/2Z) with its analytic source (finite
    at r = 0): Neumann at r=0, R and z=0, Dirichlet at z=Z.  Refining h and tau
    together the error falls at order 2 (I4)."""
    errs = [_mms_error(N) for N in (8, 16, 32)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)


# ------------------------------------------------------------------- I5
def test_uniform_state_is_fixed_point():
    p = H.config1()
    p = p.copy(q=np.zeros(5))
    o = Oracle(p)
    o.step(50 * o.tau_exp(), 5)
    # exact up to the rounding of the Thomas divisions
    assert np.max(np.abs(o.field() - p.T_init)) <= 1e-13 * p.T_init


def test_z_uniform_stays_z_uniform():
    p = H.homogeneous_cylinder(10, 7, R=2.0, Z=3.0, k=3.0, C=2.0, bc=(0, 0, 0, 0))
    o = Oracle(p)
    rng = np.random.default_rng(1)
    o.set_field(np.tile(rng.standard_normal(10), (7, 1)))
    o.step(0.7, 4)
    T = o.field()
    assert np.max(np.abs(T - T[0])) < 1e-13


def test_void_cells_keep_their_value():
    p = H.config1()
    o = Oracle(p)
    reg = o.grid()["region"]
    T = H.random_field(p, seed=9)
    o.set_field(T)
    o.step(50 * o.tau_exp(), 3)
    np.testing.assert_array_equal(o.field()[reg < 0], T[reg < 0])
    assert (reg < 0).sum() == 33 * 25  # r in (2, 4.2) x z in (8, 10): 33 x 25 cells
