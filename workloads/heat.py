"""Seeded synthetic inputs for the layered axisymmetric heat problem.

This module is shared by the CPU oracle tests, the CUDA-path tests and
``bench.py``.  It holds *no arithmetic of the method*: only the geometry tables
(layer faces, per-layer cell counts, region boxes), boundary-condition flags,
material draws and initial values.  Grid centres, spacings, face
conductivities, the time-step limit, the ADI step itself and every derived
quantity are computed independently by the oracle and by the CUDA library.

Geometry of the pulse cryogenic cell (paper, Fig. "object" and its TikZ
macros): cooler core 0 <= r < 2 over 0 <= z <= 10, insulator 2-3, heater
3-4.0 and outer insulator (coating) 4.0-4.2 over 0 <= z <= 8, terminal cap
10 <= z <= 10.2 over 0 <= r <= 4.2.  Units are read as metres.  The paper's
own numerical example (Sec. 5) uses a graded 1210x100 grid with radii
0.24/0.245/0.25/0.2501 and z0=4, zmax=5; ``config_paper_grid`` reproduces
that grid shape with seeded (synthetic) coefficients, because the paper's
temperature-dependent material laws are not given.

Per-layer cell counts: the paper (Sec. 5) prescribes the number of cells in
each layer, and cells are uniform inside a layer (Sec. 3, eq. "grid").  When a
config only fixes the total Nr or Nz, ``apportion`` splits it over the layers
by largest remainder of the thickness quotas (at least 2 cells per layer, ties
to the lower index); the counts are then inputs like the paper's.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

# Boundary-condition kinds, faces ordered (r_lo, r_hi, z_lo, z_hi).
BC_NEUMANN = 0
BC_DIRICHLET = 1

# Face-conductivity readings of the garbled lambda_{i+-1/2} definition (Sec. 3).
FACE_HARMONIC = 0
FACE_ARITH = 1

# Region ids of the five-region cell (Fig. "object", labels 0..4).
COOLER, INSULATOR, HEATER, COATING, TERMINAL = 0, 1, 2, 3, 4
N_REGIONS = 5

# Geometry numbers from the figure macros (\ri=2, \rii=3, \riii=4.0, \riv=4.2,
# \zi=8, \zii=10; the terminal rectangle is drawn from \zii to \zii+0.2).
R_FACES_CELL = (0.0, 2.0, 3.0, 4.0, 4.2)
Z_FACES_CELL = (0.0, 8.0, 10.0, 10.2)


@dataclasses.dataclass
class Problem:
    """One heat-problem instance, as plain arrays.

    r_faces[n_rl+1], r_cells[n_rl]: radial layer faces and cells per layer.
    z_faces[n_zl+1], z_cells[n_zl]: axial segment faces and cells per segment.
    boxes[n_box, 4] = (r0, r1, z0, z1); box_region[n_box]: a cell belongs to
    the first box containing its centre, else it is void.
    bc[4], T_bc[4]: boundary kind and value on faces (r_lo, r_hi, z_lo, z_hi).
    k, C, q [n_regions]: conductivity W/(m K), volumetric heat capacity
    J/(m^3 K), volumetric source W/m^3.
    """

    name: str
    r_faces: np.ndarray
    r_cells: np.ndarray
    z_faces: np.ndarray
    z_cells: np.ndarray
    boxes: np.ndarray
    box_region: np.ndarray
    bc: np.ndarray
    T_bc: np.ndarray
    k: np.ndarray
    C: np.ndarray
    q: np.ndarray
    T_init: float
    face_mean: int = FACE_HARMONIC

    @property
    def Nr(self) -> int:
        return int(np.sum(self.r_cells))

    @property
    def Nz(self) -> int:
        return int(np.sum(self.z_cells))

    def copy(self, **changes) -> "Problem":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
        d.update(changes)
        return Problem(**d)


def apportion(total: int, thicknesses: Sequence[float], min_cells: int = 2) -> np.ndarray:
    """Split ``total`` cells over layers by largest remainder of thickness quotas.

    Every layer gets at least ``min_cells``; ties in the remainder go to the
    lower layer index.  Deterministic and exact in integers.
    """
    th = np.asarray(thicknesses, dtype=np.float64)
    n = len(th)
    if total < min_cells * n:
        raise ValueError(f"total={total} too small for {n} layers of >= {min_cells} cells")
    quota = total * th / th.sum()
    cells = np.maximum(np.floor(quota).astype(np.int64), min_cells)
    # remove surplus created by the minimum, from the layers with most cells
    while cells.sum() > total:
        order = sorted(range(n), key=lambda i: (-(cells[i] - quota[i]), i))
        for i in order:
            if cells[i] > min_cells:
                cells[i] -= 1
                break
    rem = quota - np.floor(quota)
    order = sorted(range(n), key=lambda i: (-rem[i], i))
    idx = 0
    while cells.sum() < total:
        cells[order[idx % n]] += 1
        idx += 1
    return cells.astype(np.int32)


def cell_boxes(r_faces: Sequence[float] = R_FACES_CELL, z_faces: Sequence[float] = Z_FACES_CELL,
               cap: bool = True):
    """Region boxes of the five-region cell for the given layer/segment faces.

    r_faces = (0, r0*, r1*, r2*, rmax), z_faces = (0, z0, zmax[, zmax+cap]).
    """
    r0, r1, r2, r3, r4 = r_faces
    if cap:
        z0, z1, z2, z3 = z_faces
        boxes = [
            (r0, r1, z0, z2, COOLER),
            (r1, r2, z0, z1, INSULATOR),
            (r2, r3, z0, z1, HEATER),
            (r3, r4, z0, z1, COATING),
            (r0, r4, z2, z3, TERMINAL),
        ]
    else:
        z0, z1, z2 = z_faces
        boxes = [
            (r0, r1, z0, z2, COOLER),
            (r1, r2, z0, z1, INSULATOR),
            (r2, r3, z0, z1, HEATER),
            (r3, r4, z0, z1, COATING),
        ]
    b = np.array([x[:4] for x in boxes], dtype=np.float64)
    reg = np.array([x[4] for x in boxes], dtype=np.int32)
    return b, reg


def _paper_bc(T_top: float):
    # insulated everywhere except T = T0 on the top face z = zmax (eq. "boundcond");
    # the r_lo face is the symmetry axis r = 0.
    bc = np.array([BC_NEUMANN, BC_NEUMANN, BC_NEUMANN, BC_DIRICHLET], dtype=np.int32)
    T_bc = np.array([0.0, 0.0, 0.0, T_top], dtype=np.float64)
    return bc, T_bc


def _draw_kC(rng: np.random.Generator, n: int = N_REGIONS):
    k = np.exp(rng.uniform(np.log(0.1), np.log(400.0), size=n))
    C = rng.uniform(1e6, 4e6, size=n)
    return k, C


def cell_problem(Nr: int, Nz: int, k, C, q_heater: float, T0: float = 300.0,
                 T_init: float | None = None, name: str = "cell",
                 r_faces=R_FACES_CELL, z_faces=Z_FACES_CELL, face_mean=FACE_HARMONIC) -> Problem:
    r_faces = np.asarray(r_faces, dtype=np.float64)
    z_faces = np.asarray(z_faces, dtype=np.float64)
    r_cells = apportion(Nr, np.diff(r_faces))
    z_cells = apportion(Nz, np.diff(z_faces))
    boxes, reg = cell_boxes(r_faces, z_faces, cap=True)
    bc, T_bc = _paper_bc(T0)
    q = np.zeros(N_REGIONS)
    q[HEATER] = q_heater
    return Problem(name=name, r_faces=r_faces, r_cells=r_cells, z_faces=z_faces, z_cells=z_cells,
                   boxes=boxes, box_region=reg, bc=bc, T_bc=T_bc,
                   k=np.asarray(k, dtype=np.float64), C=np.asarray(C, dtype=np.float64), q=q,
                   T_init=float(T0 if T_init is None else T_init), face_mean=face_mean)


# ---------------------------------------------------------------- configs
# Step counts of each workload (the number of implicit steps the workload runs).
STEPS = {"config1": 200, "config2": 1000, "config3": 500, "config4": 200, "config5": 2000}
# dt of every workload is this multiple of the method's explicit stability limit.
DT_FACTOR = 50.0


def config1() -> Problem:
    """Plain method, FP64, one instance: 64(r) x 128(z), seed 0, q = 1e6 W/m^3."""
    rng = np.random.default_rng(0)
    k, C = _draw_kC(rng)
    return cell_problem(64, 128, k, C, 1e6, name="config1_64x128")


def config2(Nr: int = 2048, Nz: int = 4096, seed: int = 2) -> Problem:
    """Plain method at scale: 2048 x 4096; log-uniform k, uniform C, q ~ U[1e5, 1e7].

    The same seeded coefficients are used at any (Nr, Nz), so reduced grids of
    this config are the same physical problem, coarser.
    """
    rng = np.random.default_rng(seed)
    k, C = _draw_kC(rng)
    q = rng.uniform(1e5, 1e7)
    return cell_problem(Nr, Nz, k, C, q, name=f"config2_{Nr}x{Nz}")


def config3_members(n: int = 512, seed: int = 3) -> List[Problem]:
    """Batched ensemble: n instances on uneven grids with jittered layer thicknesses.

    Nr ~ U{64..512}, Nz ~ U{128..1024}; each layer/segment thickness scaled by
    U(0.9, 1.1) (thicknesses, not radii, so the ordering is kept); k log-uniform,
    C uniform, q ~ U[1e5, 1e7].  Draw order per member: Nr, Nz, 4 r-thickness
    factors, 3 z-thickness factors, 5 k, 5 C, q.
    """
    rng = np.random.default_rng(seed)
    out = []
    th_r = np.diff(np.asarray(R_FACES_CELL))
    th_z = np.diff(np.asarray(Z_FACES_CELL))
    for m in range(n):
        Nr = int(rng.integers(64, 513))
        Nz = int(rng.integers(128, 1025))
        fr = rng.uniform(0.9, 1.1, size=len(th_r))
        fz = rng.uniform(0.9, 1.1, size=len(th_z))
        k, C = _draw_kC(rng)
        q = rng.uniform(1e5, 1e7)
        r_faces = np.concatenate([[0.0], np.cumsum(th_r * fr)])
        z_faces = np.concatenate([[0.0], np.cumsum(th_z * fz)])
        out.append(cell_problem(Nr, Nz, k, C, q, name=f"config3_m{m}_{Nr}x{Nz}",
                                r_faces=r_faces, z_faces=z_faces))
    return out


def config4(Nr: int = 8192, Nz: int = 16384, seed: int = 4) -> Problem:
    """Precision stress: conductivity contrast 1e4 (0.04 in both insulators, 400 elsewhere)."""
    rng = np.random.default_rng(seed)
    k = np.array([400.0, 0.04, 400.0, 0.04, 400.0])
    C = rng.uniform(1e6, 4e6, size=N_REGIONS)
    q = rng.uniform(1e5, 1e7)
    return cell_problem(Nr, Nz, k, C, q, name=f"config4_{Nr}x{Nz}")


def config5_params(n: int, seed: int = 5) -> np.ndarray:
    """Surrogate inputs [n, 7]: 5 log-uniform k, q ~ U[1e5, 1e7], T_top ~ U[250, 350] K."""
    rng = np.random.default_rng(seed)
    k = np.exp(rng.uniform(np.log(0.1), np.log(400.0), size=(n, 5)))
    q = rng.uniform(1e5, 1e7, size=(n, 1))
    Tt = rng.uniform(250.0, 350.0, size=(n, 1))
    return np.concatenate([k, q, Tt], axis=1)


def config5_problem(params: Sequence[float], Nr: int = 128, Nz: int = 256) -> Problem:
    """One surrogate instance: C fixed to config 1's seed-0 draws, T_init = 300 K."""
    p = np.asarray(params, dtype=np.float64)
    C = config1().C
    return cell_problem(Nr, Nz, p[:5], C, float(p[5]), T0=float(p[6]), T_init=300.0,
                        name="config5")


def config5_reference_problem(Nr: int = 128, Nz: int = 256) -> Problem:
    """Homogeneous k = 400, C = 1e6 instance whose stability limit fixes config 5's dt."""
    return cell_problem(Nr, Nz, np.full(5, 400.0), np.full(5, 1e6), 0.0, name="config5_dt")


def config_paper_grid(seed: int = 6) -> Problem:
    """The paper's own grid shape (Sec. 5): 1210 x 100, graded, no terminal cap.

    Radii 0.24/0.245/0.25/0.2501 with 800/200/200/10 cells; z0 = 4, zmax = 5;
    100 axial cells in the core (80 over 0..4 and 20 over 4..5) and 80 in the
    other layers; Dirichlet only on the core top z = zmax.  Coefficients are
    seeded stand-ins for the missing material laws.
    """
    rng = np.random.default_rng(seed)
    k, C = _draw_kC(rng)
    r_faces = np.array([0.0, 0.24, 0.245, 0.25, 0.2501])
    z_faces = np.array([0.0, 4.0, 5.0])
    boxes, reg = cell_boxes(r_faces, z_faces, cap=False)
    bc, T_bc = _paper_bc(4.2)
    q = np.zeros(N_REGIONS)
    q[HEATER] = 1e6
    return Problem(name="paper_grid_1210x100", r_faces=r_faces,
                   r_cells=np.array([800, 200, 200, 10], dtype=np.int32),
                   z_faces=z_faces, z_cells=np.array([80, 20], dtype=np.int32),
                   boxes=boxes, box_region=reg, bc=bc, T_bc=T_bc, k=k, C=C, q=q, T_init=4.2)


# ---------------------------------------------------------- pin problems
def homogeneous_cylinder(Nr: int, Nz: int, R: float, Z: float, k: float, C: float,
                         bc=(BC_NEUMANN, BC_NEUMANN, BC_NEUMANN, BC_DIRICHLET),
                         T_bc=(0.0, 0.0, 0.0, 0.0), T_init: float = 0.0, q: float = 0.0) -> Problem:
    """Solid cylinder 0 <= r <= R, 0 <= z <= Z of one material, uniform cells."""
    return Problem(name=f"cyl_{Nr}x{Nz}", r_faces=np.array([0.0, R]),
                   r_cells=np.array([Nr], dtype=np.int32), z_faces=np.array([0.0, Z]),
                   z_cells=np.array([Nz], dtype=np.int32),
                   boxes=np.array([[0.0, R, 0.0, Z]]), box_region=np.array([0], dtype=np.int32),
                   bc=np.asarray(bc, dtype=np.int32), T_bc=np.asarray(T_bc, dtype=np.float64),
                   k=np.array([k]), C=np.array([C]), q=np.array([q]), T_init=T_init)


def layered_annulus(radii: Sequence[float], cells: Sequence[int], k: Sequence[float],
                    T_a: float, T_b: float, Nz: int = 2, Z: float = 1.0,
                    C: float = 1.0) -> Problem:
    """Annulus radii[0] <= r <= radii[-1] of concentric layers, Dirichlet T_a / T_b on
    the inner / outer wall, insulated z ends (z-uniform)."""
    radii = np.asarray(radii, dtype=np.float64)
    n = len(radii) - 1
    boxes = np.array([[radii[m], radii[m + 1], 0.0, Z] for m in range(n)])
    return Problem(name="annulus", r_faces=radii, r_cells=np.asarray(cells, dtype=np.int32),
                   z_faces=np.array([0.0, Z]), z_cells=np.array([Nz], dtype=np.int32),
                   boxes=boxes, box_region=np.arange(n, dtype=np.int32),
                   bc=np.array([BC_DIRICHLET, BC_DIRICHLET, BC_NEUMANN, BC_NEUMANN], dtype=np.int32),
                   T_bc=np.array([T_a, T_b, 0.0, 0.0]), k=np.asarray(k, dtype=np.float64),
                   C=np.full(n, C), q=np.zeros(n), T_init=0.5 * (T_a + T_b))


def random_field(p: Problem, seed: int, amp: float = 10.0) -> np.ndarray:
    """A seeded perturbed initial field [Nz, Nr] around T_init (void cells are
    overwritten by the solvers' own rule, so their value here is irrelevant)."""
    rng = np.random.default_rng(seed)
    return p.T_init + amp * rng.standard_normal((p.Nz, p.Nr))


# ------------------------------------------- temperature-dependent materials
# The paper's k(T), c_V(T) and chi(T) are cited, not printed, so the
# temperature-dependent runs use synthetic laws with the qualitative shapes of
# cryogenic materials (conductivity and heat capacity rising with T, the
# heater's resistivity rising with T), tabulated at knots; the method reads
# them by linear interpolation (flat beyond the end knots).
PULSE_CONST, PULSE_RECT, PULSE_ERF = 0, 1, 2


@dataclasses.dataclass
class NlMaterials:
    """Per-region material tables and the source model of the full method.

    T_knots, k, C, chi: [n_regions, K] -- temperature knots (strictly
    increasing per region), conductivity W/(m K), volumetric heat capacity
    rho c_V J/(m^3 K), resistivity Ohm m at the knots.
    j2: [n_regions] squared current density (I / S_C)^2 in A^2/m^4 (zero
    outside the heater); the source is X = chi(T) j2 p(t).
    model, t_per, t_src, t_trs, xi, zeta: the source's time law p(t)
    (PULSE_CONST: p = 1; PULSE_RECT: the rectangular train; PULSE_ERF: the
    erf-smoothed train with transition time t_trs).
    """

    T_knots: np.ndarray
    k: np.ndarray
    C: np.ndarray
    chi: np.ndarray
    j2: np.ndarray
    model: int = PULSE_CONST
    t_per: float = 1.0
    t_src: float = 1.0
    t_trs: float = 1.0
    xi: float = 4.0
    zeta: float = 2.0


def nl_constant(p: Problem) -> NlMaterials:
    """Temperature-independent tables equal to a problem's constants (one knot;
    chi = q with j2 = 1), a constant source: the linear method as a special case."""
    R = len(p.k)
    return NlMaterials(T_knots=np.zeros((R, 1)), k=np.asarray(p.k, np.float64).reshape(R, 1),
                       C=np.asarray(p.C, np.float64).reshape(R, 1), chi=np.asarray(p.q, np.float64).reshape(R, 1),
                       j2=np.ones(R))


def nl_power_laws(p: Problem, T_lo: float, T_hi: float, n_knots: int, a_k, a_C, a_chi, T_ref: float,
                  j2: float, heater: int = 2, **pulse) -> NlMaterials:
    """Synthetic laws k_m (T/T_ref)^a_k[m], C_m (T/T_ref)^a_C[m], and for the
    heater chi(T) = chi_0 (T/T_ref)^a_chi with chi_0 j2 = q_heater, sampled at
    n_knots temperatures spread evenly over [T_lo, T_hi]."""
    R = len(p.k)
    Tk = np.linspace(T_lo, T_hi, n_knots)
    u = Tk / T_ref
    k = np.array([p.k[m] * u ** a_k[m] for m in range(R)])
    C = np.array([p.C[m] * u ** a_C[m] for m in range(R)])
    chi = np.zeros((R, n_knots))
    jj = np.zeros(R)
    chi[heater] = p.q[heater] / j2 * u ** a_chi
    jj[heater] = j2
    return NlMaterials(T_knots=np.tile(Tk, (R, 1)), k=k, C=C, chi=chi, j2=jj, **pulse)


def nl_linear_laws(p: Problem, beta_k: float, beta_C: float, T_lo: float, T_hi: float) -> NlMaterials:
    """k_m (1 + beta_k T), C_m (1 + beta_C T) as two-knot tables over [T_lo, T_hi]
    (linear interpolation reproduces a linear law exactly inside the range);
    the source is the problem's q, constant."""
    R = len(p.k)
    Tk = np.array([T_lo, T_hi])
    k = np.array([[p.k[m] * (1.0 + beta_k * T) for T in Tk] for m in range(R)])
    C = np.array([[p.C[m] * (1.0 + beta_C * T) for T in Tk] for m in range(R)])
    chi = np.array([[p.q[m], p.q[m]] for m in range(R)])
    return NlMaterials(T_knots=np.tile(Tk, (R, 1)), k=k, C=C, chi=chi, j2=np.ones(R))


def paper_example_nl(Nr_cells=(800, 200, 200, 10), Nz_cells=(80, 20)) -> tuple:
    """The paper's own example (Sec. 5) as far as it is given: the graded
    1210 x 100 grid without terminal cap, T0 = 4.2 K, the pulsed source with
    t_per = 0.1 s, t_src = 0.01 s, t_trs = 1e-4 s, xi = 4, zeta = 2.  The
    material laws are synthetic (see nl_power_laws): k and C rising with T
    (exponents 1 and 3, the low-temperature shapes of metals' conductivity and
    Debye heat capacity) around seeded magnitudes, the heater's resistivity
    rising linearly.  Returns (problem, materials)."""
    p = config_paper_grid()
    p = p.copy(r_cells=np.array(Nr_cells, np.int32), z_cells=np.array(Nz_cells, np.int32))
    m = nl_power_laws(p, 4.2, 60.0, 9, a_k=[1.0] * N_REGIONS, a_C=[3.0] * N_REGIONS, a_chi=1.0, T_ref=4.2,
                      j2=1.0, model=PULSE_ERF, t_per=0.1, t_src=0.01, t_trs=1e-4, xi=4.0, zeta=2.0)
    return p, m
