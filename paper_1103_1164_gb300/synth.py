"""Seeded synthetic inputs for the DC-FSPB dose engine.

This module is the only code shared by the CUDA path's callers and the FP64
oracle.  It holds none of the dose method's arithmetic: it draws densities,
beam set-ups, fluences and the commissioned parameter tables, all of which the
method (Section 2.1, eqs. 1-4) consumes as given inputs.

The paper's clinical CT, plans and MC-commissioned parameters (Table 1,
Section 2.3) are not available, so every input here is synthetic:

* phantoms with the geometry of the paper's workloads (128x128x72-103 grids at
  millimetre voxels, water with lung, bone and air inhomogeneities);
* beams with SAD 100 cm, square fields and uniformly sized beamlets;
* commissioning tables drawn from closed forms with the qualitative shape of a
  6 MV beam (build-up then attenuation for A(t_eq, theta); a steep primary and
  a shallow scatter penumbra for u_1^w, u_2^w; a slowly growing scatter weight
  omega_2^w; power-law widening factors f(rho) with f(1) = 1; and a linear
  b(rho) with b(1) = 0).  The closed forms are only used to fill the tables:
  both the oracle and the GPU path look the tables up (Algorithm A1 steps 9-10).

Units: cm, radians, g/cm^3.  Volumes are float32 ``[nz][ny][nx]`` with x
fastest; voxel (i, j, k) has its centre at ``origin + (i*dx, j*dy, k*dz)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Seeds used by the standard workloads (phantom seed is 1000 + config number).
COEFF_SEED = 42
FLUENCE_SEED = 7


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    ox: float
    oy: float
    oz: float

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def centres(self):
        """Voxel-centre coordinate vectors (x, y, z), float64."""
        x = self.ox + self.dx * np.arange(self.nx)
        y = self.oy + self.dy * np.arange(self.ny)
        z = self.oz + self.dz * np.arange(self.nz)
        return x, y, z


def centred_grid(nx, ny, nz, dx, dy=None, dz=None) -> Grid:
    """A grid whose centre is the origin of the patient frame."""
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    return Grid(nx, ny, nz, dx, dy, dz,
                -0.5 * (nx - 1) * dx, -0.5 * (ny - 1) * dy, -0.5 * (nz - 1) * dz)


@dataclasses.dataclass
class Beam:
    gantry_deg: float
    sad: float = 100.0
    iso: Sequence[float] = (0.0, 0.0, 0.0)
    field_x: float = 10.0
    field_y: float = 10.0
    couch_deg: float = 0.0
    coll_deg: float = 0.0


@dataclasses.dataclass
class Commissioning:
    """Tabulated beam model (the inputs of Algorithm A1 steps 9-11).

    A[l, j]   depth dose at theta = l*a_dtheta, t_eq = j*a_dt   (n_theta, n_t)
    water[q, j] q = 0..3: u_1^w, u_2^w, omega_1^w, omega_2^w at t = j*w_dt
    dens[q, j]  q = 0..5: f_u1, f_u2, f_omega1, f_omega2, b_1, b_2 at
                rho = f_rho0 + j*f_drho
    """
    A: np.ndarray
    a_dt: float
    a_dtheta: float
    water: np.ndarray
    w_dt: float
    dens: np.ndarray
    f_rho0: float
    f_drho: float
    roi_radius: float = 5.0
    smooth_sigma: float = 0.5
    rho_surface: float = 0.02
    density_correction: int = 1


@dataclasses.dataclass
class Plan:
    name: str
    grid: Grid
    rho: np.ndarray           # float32 [nz, ny, nx]
    beams: List[Beam]
    beamlet_x: float
    beamlet_y: float
    comm: Commissioning
    fluence: np.ndarray       # float32 [n_beamlets]

    @property
    def beamlets_per_beam(self):
        return [int(round(b.field_x / self.beamlet_x)) * int(round(b.field_y / self.beamlet_y))
                for b in self.beams]

    @property
    def n_beamlets(self) -> int:
        return int(sum(self.beamlets_per_beam))


# ---------------------------------------------------------------------------
# Commissioning tables
# ---------------------------------------------------------------------------

# Parameters of the synthetic beam model's lateral and density-correction
# tables (the quantities Section 2.1 fits to reference doses), in the order
# they are drawn.
MODEL_PARAMS = ("u10", "k1", "u20", "k2", "w20", "w21", "tau", "a1", "a2", "gam", "beta1", "beta2")


def model_params(seed: int = COEFF_SEED) -> dict:
    """The seeded synthetic model: depth-dose shape (beta, mu, horn) and the
    twelve MODEL_PARAMS."""
    rng = np.random.default_rng(seed)
    u = lambda lo, hi: float(rng.uniform(lo, hi))
    names = ("beta", "mu", "horn") + MODEL_PARAMS
    ranges = ((2.0, 4.0), (0.04, 0.06), (2.0, 6.0), (3.0, 8.0), (0.0, 0.02), (0.3, 1.0), (0.0, 0.02),
              (0.03, 0.10), (0.0, 0.08), (2.0, 8.0), (0.5, 1.0), (0.5, 1.0), (0.3, 1.0), (0.0, 0.005),
              (0.002, 0.01))
    return {n: u(*r) for n, r in zip(names, ranges)}


def model_tables(prm: dict, w_dt: float, w_n: int, f_rho0: float, f_drho: float, f_n: int):
    """(water [4, w_n], dens [6, f_n]) in float64 from the model's closed forms:
    u_1^w = u10 / (1 + k1 t), u_2^w = u20 / (1 + k2 t), omega_2^w = w20 +
    w21 (1 - exp(-t / tau)), omega_1^w = 1 - omega_2^w; f_u1 = rho^a1, f_u2 =
    rho^a2, f_omega1 = 1, f_omega2 = rho^gam, b_1 = beta1 (1 - rho), b_2 =
    beta2 (rho - 1)."""
    tw = w_dt * np.arange(w_n)
    w2 = prm["w20"] + prm["w21"] * (1.0 - np.exp(-tw / prm["tau"]))
    water = np.stack([prm["u10"] / (1.0 + prm["k1"] * tw), prm["u20"] / (1.0 + prm["k2"] * tw), 1.0 - w2, w2])
    r = f_rho0 + f_drho * np.arange(f_n)
    dens = np.stack([r ** prm["a1"], r ** prm["a2"], np.ones_like(r), r ** prm["gam"],
                     prm["beta1"] * (1.0 - r), prm["beta2"] * (r - 1.0)])
    return water, dens


def make_commissioning(seed: int = COEFF_SEED, *, roi_radius=5.0, smooth_sigma=0.5,
                       rho_surface=0.02, density_correction=1,
                       a_dt=0.125, a_tmax=80.0, a_dtheta=0.025, a_thmax=0.2,
                       w_dt=0.125, w_tmax=80.0, f_rho0=0.1, f_rho1=2.0,
                       f_drho=0.01) -> Commissioning:
    prm = model_params(seed)
    beta, mu, horn = prm["beta"], prm["mu"], prm["horn"]

    nt = int(round(a_tmax / a_dt)) + 1
    nth = int(round(a_thmax / a_dtheta)) + 1
    t = a_dt * np.arange(nt)
    th = a_dtheta * np.arange(nth)
    depth = (1.0 - np.exp(-beta * t)) * np.exp(-mu * t)
    A = depth[None, :] * (1.0 + horn * th[:, None] ** 2)
    A = A / depth.max()

    nw = int(round(w_tmax / w_dt)) + 1
    nf = int(round((f_rho1 - f_rho0) / f_drho)) + 1
    water, dens = model_tables(prm, w_dt, nw, f_rho0, f_drho, nf)
    return Commissioning(A.astype(np.float32), a_dt, a_dtheta, water.astype(np.float32),
                         w_dt, dens.astype(np.float32), f_rho0, f_drho, roi_radius,
                         smooth_sigma, rho_surface, density_correction)


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

def _mesh(g: Grid):
    x, y, z = g.centres()
    return np.meshgrid(x, y, z, indexing="ij")  # arrays indexed [i, j, k]


def _to_zyx(a_ijk):
    return np.ascontiguousarray(np.transpose(a_ijk, (2, 1, 0))).astype(np.float32)


def slab_phantom(g: Grid, slab_depths=(5.0, 10.0), slab_rho=0.25) -> np.ndarray:
    """Water with a slab of density slab_rho at y-depths [d0, d1) from the y_min face."""
    _, Y, _ = _mesh(g)
    depth = Y - (g.oy - 0.5 * g.dy)
    rho = np.ones_like(Y)
    rho[(depth >= slab_depths[0]) & (depth < slab_depths[1])] = slab_rho
    return _to_zyx(rho)


def thorax_phantom(g: Grid, seed: int) -> np.ndarray:
    """Water ellipse (14 x 10 cm semi-axes) in air with two lungs, a spine and noise."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _mesh(g)
    rho = np.full_like(X, 0.001)
    body = (X / 14.0) ** 2 + (Y / 10.0) ** 2 <= 1.0
    rho[body] = 1.0
    for sx in (-1.0, 1.0):
        lung = ((X - 6.5 * sx) / 4.5) ** 2 + ((Y + 0.5) / 6.0) ** 2 + (Z / 10.0) ** 2 <= 1.0
        rho[lung] = rng.uniform(0.20, 0.35)
    spine = (X ** 2 + (Y - 6.5) ** 2) <= 1.5 ** 2
    rho[spine] = rng.uniform(1.5, 1.8)
    noise = rng.normal(0.0, 0.02, size=X.shape)
    rho[body] += noise[body]
    np.maximum(rho, 0.001, out=rho)
    return _to_zyx(rho)


def head_neck_phantom(g: Grid, seed: int, radius: float = None) -> np.ndarray:
    """Water cylinder with air cavities, bone and a lung base (head-and-neck-like).

    The cylinder's radius is ``radius`` cm, else 0.42 of the grid's smaller
    transverse extent."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _mesh(g)
    ext = np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    rad = 0.42 * min(ext[0], ext[1]) if radius is None else float(radius)
    rho = np.full_like(X, 0.001)
    body = X ** 2 + Y ** 2 <= rad ** 2
    rho[body] = 1.0
    zlo = g.oz - 0.5 * g.dz
    lung = body & (Z < zlo + 0.25 * ext[2])
    rho[lung] = rng.uniform(0.20, 0.35)
    for _ in range(int(rng.integers(2, 5))):
        c = rng.uniform(-0.5, 0.5, size=3) * np.array([rad, rad, 0.5 * ext[2]])
        r = rng.uniform(0.8, 2.0)
        rho[(X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r] = 0.001
    bone_r = rng.uniform(1.0, 2.0)
    bx, by = rng.uniform(-0.3, 0.3) * rad, 0.6 * rad
    rho[((X - bx) ** 2 + (Y - by) ** 2 <= bone_r ** 2) & body] = rng.uniform(1.6, 1.9)
    ring = body & (X ** 2 + Y ** 2 >= (rad - 0.6) ** 2)
    rho[ring & (Z > zlo + 0.25 * ext[2])] = rng.uniform(1.6, 1.9)
    return _to_zyx(rho)


def random_slab_sphere_phantom(g: Grid, rng: np.random.Generator) -> np.ndarray:
    """Water with 1-4 slabs and/or spheres of density U[0.05, 2.0]."""
    X, Y, Z = _mesh(g)
    rho = np.ones_like(X)
    ext = np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    for _ in range(int(rng.integers(1, 5))):
        val = rng.uniform(0.05, 2.0)
        if rng.uniform() < 0.5:
            axis = int(rng.integers(0, 3))
            coord = (X, Y, Z)[axis]
            lo = rng.uniform(-0.4, 0.3) * ext[axis]
            hi = lo + rng.uniform(0.5, 0.3 * ext[axis])
            rho[(coord >= lo) & (coord < hi)] = val
        else:
            c = rng.uniform(-0.35, 0.35, size=3) * ext
            r = rng.uniform(0.5, 0.3 * ext.min())
            rho[(X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r] = val
    return _to_zyx(rho)


# ---------------------------------------------------------------------------
# Standard workloads
# ---------------------------------------------------------------------------

def uniform_fluence(n: int, seed: int = FLUENCE_SEED) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n).astype(np.float32)


def config1(n=64) -> Plan:
    """One 6 MV-like beam on a 64^3 water phantom with a lung slab at 5-10 cm depth."""
    g = centred_grid(n, n, n, 0.25)
    comm = make_commissioning(COEFF_SEED, roi_radius=3.0)
    beams = [Beam(0.0, 100.0, (0.0, 0.0, 0.0), 10.0, 10.0)]
    p = Plan("slab64", g, slab_phantom(g), beams, 0.5, 0.5, comm, np.zeros(0, np.float32))
    p.fluence = np.ones(p.n_beamlets, np.float32)
    return p


def config2(scale: float = 1.0) -> Plan:
    """9-field coplanar plan on a 128x128x96 thorax phantom (0.25 cm voxels).

    ``scale`` < 1 shrinks the grid (voxel count) for quick parity runs while
    keeping the voxel size, field sizes and beam set.
    """
    nx, ny, nz = (int(round(128 * scale)), int(round(128 * scale)), int(round(96 * scale)))
    g = centred_grid(nx, ny, nz, 0.25)
    rng = np.random.default_rng(1002)
    fields = rng.integers(16, 31, size=9) * 0.5      # 8.0 .. 15.0 cm in 0.5 cm steps
    beams = [Beam(40.0 * b, 100.0, (0.0, 0.0, 0.0), float(f), float(f)) for b, f in enumerate(fields)]
    comm = make_commissioning(COEFF_SEED, roi_radius=5.0)
    p = Plan("thorax9", g, thorax_phantom(g, 1002), beams, 0.5, 0.5, comm, np.zeros(0, np.float32))
    p.fluence = uniform_fluence(p.n_beamlets)
    return p


def config5_plans(n_plans: int = 16, seed: int = 1005, max_dim: int = 256) -> List[Plan]:
    """Uneven batch of head-and-neck-like plans (5-9 beams, 0.25 cm beamlets)."""
    rng = np.random.default_rng(seed)
    comm = make_commissioning(COEFF_SEED, roi_radius=5.0)
    plans = []
    for p_i in range(n_plans):
        if p_i == 0:
            nx = ny = max_dim
            nz = int(max_dim * 0.75)
        else:
            nx = ny = int(rng.integers(96, max_dim + 1) // 8 * 8)
            nz = int(rng.integers(64, int(max_dim * 0.75) + 1) // 8 * 8)
        vox = float(np.round(rng.uniform(0.2, 0.3), 3))
        g = centred_grid(nx, ny, nz, vox)
        nb = int(rng.integers(5, 10))
        gantries = np.sort(rng.uniform(0, 360, size=nb))
        size = float(np.round(rng.uniform(8.0, 16.5) / 0.25) * 0.25)
        beams = [Beam(float(a), 100.0, (0.0, 0.0, 0.0), size, size) for a in gantries]
        p = Plan(f"hn{p_i}", g, head_neck_phantom(g, seed * 100 + p_i), beams, 0.25, 0.25,
                 comm, np.zeros(0, np.float32))
        p.fluence = uniform_fluence(p.n_beamlets, FLUENCE_SEED + p_i)
        plans.append(p)
    return plans


def small_plan(seed: int, n=(12, 10, 8), vox=0.5, n_beams=2, field=2.0, beamlet=0.5,
               roi=1.5, phantom="random", density_correction=1,
               beamlet_y=None, couch=False) -> Plan:
    """Tiny randomised plans for brute-force comparisons."""
    rng = np.random.default_rng(seed)
    g = centred_grid(n[0], n[1], n[2], vox)
    if phantom == "water":
        rho = np.ones(g.shape, np.float32)
    elif phantom == "slab":
        rho = slab_phantom(g, (1.0, 2.5), 0.3)
    else:
        rho = random_slab_sphere_phantom(g, rng)
    by = beamlet if beamlet_y is None else beamlet_y
    beams = []
    for b in range(n_beams):
        iso = tuple(float(v) for v in rng.uniform(-0.3, 0.3, size=3))
        beams.append(Beam(float(rng.uniform(0, 360)), float(rng.uniform(60, 110)), iso,
                          field, field if beamlet_y is None else 2 * by,
                          float(rng.uniform(-30, 30)) if couch else 0.0,
                          float(rng.uniform(-30, 30)) if couch else 0.0))
    comm = make_commissioning(COEFF_SEED, roi_radius=roi, smooth_sigma=0.6,
                              density_correction=density_correction)
    p = Plan(f"small{seed}", g, rho, beams, beamlet, by, comm, np.zeros(0, np.float32))
    p.fluence = uniform_fluence(p.n_beamlets, seed + 1)
    return p


# ---------------------------------------------------------------------------
# The ten evaluation cases of Table 1, synthetic
# ---------------------------------------------------------------------------

# Table 1 (Section 2.3): case, site, number of beams, non-coplanar, number of
# beamlets, number of voxels (all 128 x 128 in x, y).  The tumour position
# (x, y, z in cm, patient frame) is this module's choice, placed by the site
# the table names; lung tumours are water-density spheres inside a lung.
TABLE1 = (
    ("H1", "parotid", 8, True, 7264, 72, (4.0, -1.0, 0.0)),
    ("H2", "hypopharynx", 7, True, 4429, 72, (0.0, 1.0, -2.0)),
    ("H3", "nasal cavity", 8, True, 3381, 72, (0.0, -4.0, 3.0)),
    ("H4", "parotid", 5, False, 4179, 72, (-4.0, -1.0, 0.0)),
    ("H5", "larynx", 7, True, 10369, 72, (0.0, -2.0, -1.0)),
    ("L1", "left lung, lower lobe, near the pleura", 6, False, 637, 80, (9.0, 0.0, -4.0)),
    ("L2", "right lung, lower lobe, paravertebral", 6, False, 1720, 103, (-3.5, 4.0, -4.0)),
    ("L3", "left lung, upper lobe, near the pleura", 5, False, 921, 80, (9.0, -1.0, 4.0)),
    ("L4", "right lung, upper lobe, near the heart", 7, False, 841, 80, (-3.0, -1.0, 3.0)),
    ("L5", "left lung, middle", 5, False, 686, 80, (6.5, 0.0, 0.0)),
)
TABLE1_VOXEL = (0.4, 0.4, 0.25)       # cm, the CT resolution of Section 2.3
TABLE1_BEAMLET = (0.2, 0.5)           # cm, 0.2 cm along the leaf motion (x)


def _table1_fields(rng, n_beamlets, n_beams, bx, by):
    """Per-beam (field_x, field_y) whose beamlet counts sum to about n_beamlets:
    near-square fields, per-beam targets jittered by +-20 %, the last beam's
    shape (aspect 0.7-1.4) chosen to close the gap best."""
    share = rng.uniform(0.8, 1.2, size=n_beams)
    share *= n_beamlets / share.sum()
    fields, done = [], 0
    for b in range(n_beams):
        t = share[b] if b < n_beams - 1 else max(n_beamlets - done, 1)
        ny0 = max(1, int(round(math.sqrt(t * bx / by))))
        shapes = [(max(1, int(round(t / ny))), ny) for ny in
                  (range(max(1, ny0 - 3), ny0 + 4) if b == n_beams - 1 else (ny0,))]
        square = [s for s in shapes if 0.7 <= (s[0] * bx) / (s[1] * by) <= 1.4] or shapes
        nx, ny = min(square, key=lambda s: abs(s[0] * s[1] - t))
        fields.append((nx * bx, ny * by))
        done += nx * ny
    return fields


def table1_case(name: str) -> Plan:
    """A synthetic stand-in for one of the ten clinical cases of Table 1.

    Grid 128 x 128 x nz at 0.4 x 0.4 x 0.25 cm; head-and-neck cases use a
    9 cm-radius neck phantom, lung cases the thorax phantom with a 1.5 cm
    water-density tumour at the case's site.  Beams: SAD 100 cm, isocentre at
    the tumour, gantry angles evenly spread from a random start (coplanar) or,
    for the non-coplanar cases, every other beam with a couch rotation of
    15-45 degrees and a collimator rotation within +-15 degrees.  Beamlets are
    0.2 x 0.5 cm and the rectangular fields give about the case's beamlet
    count; fluence U[0, 1] per beamlet.  Commissioning as for the other
    workloads (ROI radius 5 cm, density correction on).
    """
    idx = [c[0] for c in TABLE1].index(name)
    case, _, nb, noncop, n_bl, nz, tumour = TABLE1[idx]
    seed = 1100 + idx
    rng = np.random.default_rng(seed)
    g = centred_grid(128, 128, nz, *TABLE1_VOXEL)
    if case.startswith("H"):
        rho = head_neck_phantom(g, seed, radius=9.0)
    else:
        rho = thorax_phantom(g, seed)
        X, Y, Z = _mesh(g)
        ball = (X - tumour[0]) ** 2 + (Y - tumour[1]) ** 2 + (Z - tumour[2]) ** 2 <= 1.5 ** 2
        rho[_to_zyx(ball.astype(np.float32)) > 0.5] = 1.0
    bx, by = TABLE1_BEAMLET
    fields = _table1_fields(rng, n_bl, nb, bx, by)
    start = float(rng.uniform(0.0, 360.0 / nb))
    beams = []
    for b in range(nb):
        gantry = (start + 360.0 * b / nb + float(rng.uniform(-10.0, 10.0))) % 360.0
        couch = coll = 0.0
        if noncop and b % 2 == 1:
            couch = float(rng.choice([-1.0, 1.0]) * rng.uniform(15.0, 45.0))
            coll = float(rng.uniform(-15.0, 15.0))
        beams.append(Beam(gantry, 100.0, tumour, fields[b][0], fields[b][1], couch, coll))
    comm = make_commissioning(COEFF_SEED, roi_radius=5.0)
    p = Plan(case, g, rho, beams, bx, by, comm, np.zeros(0, np.float32))
    p.fluence = uniform_fluence(p.n_beamlets, FLUENCE_SEED + seed)
    return p


def table1_plans() -> List[Plan]:
    """All ten synthetic Table 1 cases, H1-H5 then L1-L5."""
    return [table1_case(c[0]) for c in TABLE1]


# ---------------------------------------------------------------------------
# MLC leaf sequences (the input from which Section 2.3 makes the fluence maps)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class LeafSequence:
    """One beam's leaf sequence in the collimator frame of the isocentre plane.

    edges [n_leaves + 1]       leaf-pair boundaries along y (cm, increasing)
    mu    [n_cp]               cumulative meterset at each control point
    left, right [n_cp][n_leaves]  leaf tip positions along x (cm), left <= right;
                               tips move linearly in meterset between control
                               points (a step-and-shoot segment is two control
                               points with the same positions, the moves between
                               segments happen at a repeated meterset)
    jaws  (x1, x2, y1, y2)     collimator jaws (cm)
    transmission               fraction of the fluence through closed leaves
    """
    edges: np.ndarray
    mu: np.ndarray
    left: np.ndarray
    right: np.ndarray
    jaws: tuple
    transmission: float = 0.0

    @property
    def n_leaves(self) -> int:
        return int(len(self.edges) - 1)

    @property
    def n_cp(self) -> int:
        return int(len(self.mu))


def leaf_edges(field_y: float, width: float = 0.5, extra: int = 2, offset: float = 0.0) -> np.ndarray:
    """Leaf-pair boundaries of equal width covering [-field_y/2, field_y/2] plus
    ``extra`` leaves on each side, shifted by ``offset`` cm."""
    n = int(math.ceil(field_y / width)) + 2 * extra
    return (offset - 0.5 * n * width + width * np.arange(n + 1)).astype(np.float32)


def sliding_window(rng, field_x, field_y, n_cp=64, mu_total=100.0, width=0.5, min_gap=0.1,
                   offset=0.0, transmission=0.0, jaw_margin=0.0) -> LeafSequence:
    """Unidirectional sliding-window sequence: each leaf pair starts closed at
    the field's -x side and ends closed past its +x side; between control
    points (equal meterset steps) each tip advances by a random non-negative
    amount, the right tip first, with the gap kept >= min_gap."""
    edges = leaf_edges(field_y, width, offset=offset)
    nl = len(edges) - 1
    x0, x1 = -0.5 * field_x - 0.5, 0.5 * field_x + 0.5
    inc_r = rng.gamma(0.7, 1.0, size=(n_cp - 1, nl))
    inc_l = rng.gamma(0.7, 1.0, size=(n_cp - 1, nl))
    r = np.vstack([np.zeros((1, nl)), np.cumsum(inc_r, 0)])
    l = np.vstack([np.zeros((1, nl)), np.cumsum(inc_l, 0)])
    r = x0 + min_gap + (x1 - x0 - min_gap) * r / r[-1]
    l = x0 + (x1 - x0 - min_gap) * l / l[-1]
    l = np.minimum(l, r - min_gap)
    mu = np.linspace(0.0, mu_total, n_cp)
    jaws = (-0.5 * field_x - jaw_margin, 0.5 * field_x + jaw_margin,
            -0.5 * field_y - jaw_margin, 0.5 * field_y + jaw_margin)
    return LeafSequence(edges, mu.astype(np.float32), l.astype(np.float32), r.astype(np.float32),
                        tuple(float(v) for v in jaws), float(transmission))


def step_and_shoot(rng, field_x, field_y, n_seg=5, mu_total=100.0, width=0.5, offset=0.0,
                   transmission=0.0, jaw_margin=0.0) -> LeafSequence:
    """Step-and-shoot sequence: n_seg random apertures (per leaf pair a random
    open interval inside the field, some pairs closed), each delivered with a
    random share of the meterset; leaves move between segments at a repeated
    meterset value."""
    edges = leaf_edges(field_y, width, offset=offset)
    nl = len(edges) - 1
    w = rng.uniform(0.2, 1.0, size=n_seg)
    cum = np.concatenate([[0.0], np.cumsum(w / w.sum() * mu_total)])
    mu, L, R = [], [], []
    for s in range(n_seg):
        a = rng.uniform(-0.6, 0.5, size=nl) * field_x
        b = a + rng.uniform(0.0, 0.8, size=nl) * field_x
        closed = rng.uniform(size=nl) < 0.2
        b[closed] = a[closed]
        for k in (0, 1):
            mu.append(cum[s + k])
            L.append(a)
            R.append(b)
    jaws = (-0.5 * field_x - jaw_margin, 0.5 * field_x + jaw_margin,
            -0.5 * field_y - jaw_margin, 0.5 * field_y + jaw_margin)
    return LeafSequence(edges, np.asarray(mu, np.float32), np.asarray(L, np.float32),
                        np.asarray(R, np.float32), tuple(float(v) for v in jaws), float(transmission))


def plan_sequences(plan: Plan, seed: int, kind: str = "sliding", **kw) -> List[LeafSequence]:
    """One sequence per beam of the plan (sliding window or step and shoot)."""
    rng = np.random.default_rng(seed)
    make = sliding_window if kind == "sliding" else step_and_shoot
    return [make(rng, b.field_x, b.field_y, **kw) for b in plan.beams]
