"""Seeded synthetic dam-break particle sets (inputs only).

This module builds the initial particle layouts and the case constants that
both the CUDA library and the CPU oracle consume.  It holds none of the SPH
arithmetic: no kernel, no density, no pressure, no force, no integration.
Everything here is geometry (lattices, boundary layers, domain box), seeded
random numbers (position jitter, initial velocities, target perturbations,
per-case viscosity) and the configuration constants that define a case.

Layout of a dam break (Example 1a, Section 5.1.1 of the paper, with the
readings of the paper where it is silent):

* fluid particles on a lattice of spacing dx with centres at
  ((i+1/2)dx, (j+1/2)dx[, (k+1/2)dx]) measured from the tank corner, the
  block sitting in the corner of the tank;
* three layers of fixed boundary particles on the same lattice outside the
  floor and the side walls (open top);
* gravity along the last axis;
* the domain box (Section 3.2.1) is the tank plus the three wall layers plus
  a margin of one support radius (2h) on every side, and twice the tank
  height vertically; its uniform cell grid has edge cs = 2h (the kernel
  support radius, the paper's cell size) or, with cells_per_radius = 2,
  cs = h (the search then visits the 5^D cells around a particle's own).

Particles are ordered fluid first (ids 0..n_fluid-1) then boundary.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

FLUID = 0
BOUNDARY = 1

G_EARTH = 9.81

# Cells per support radius of the dam-break workloads: 1 gives cells of edge
# 2h (the 3^D stencil), 2 cells of edge h (the 5^D stencil, fewer candidates).
CELLS_PER_RADIUS = 2


@dataclass
class Case:
    """One SPH case: constants plus the initial particle state (host arrays)."""

    name: str
    dim: int
    dx: float
    h: float
    cs: float
    mass: float
    rho0: float
    c0: float
    gamma: float
    alpha: float
    visc_eps: float
    dt: float
    g: Tuple[float, float, float]
    dom_min: Tuple[float, float, float]
    ncell: Tuple[int, int, int]
    r: np.ndarray            # (N, dim) float64
    v: np.ndarray            # (N, dim) float64
    kind: np.ndarray         # (N,) uint8, FLUID / BOUNDARY
    id: np.ndarray           # (N,) uint32, persistent particle id
    n_fluid: int
    steps: int = 1
    block: Tuple[int, ...] = ()
    tank: Tuple[float, ...] = ()
    target: Optional[np.ndarray] = None   # (n_fluid, dim) float64, diff case only
    extra: dict = field(default_factory=dict)
    model: int = 0                        # 0: WCSPH (summation, Tait); 1: Example 1a form
    bc: Tuple[int, int, int] = (0, 0, 0)  # per axis: 0 cut-off, 1 symmetric, 2 periodic
    rho: Optional[np.ndarray] = None      # (N,) initial density (Example 1a form)

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    @property
    def n_boundary(self) -> int:
        return self.n - self.n_fluid

    @property
    def n_cells(self) -> int:
        nc = self.ncell
        return int(nc[0]) * int(nc[1]) * (int(nc[2]) if self.dim == 3 else 1)

    def copy(self) -> "Case":
        return replace(self, r=self.r.copy(), v=self.v.copy(), kind=self.kind.copy(),
                       id=self.id.copy(),
                       target=None if self.target is None else self.target.copy(),
                       rho=None if self.rho is None else self.rho.copy(),
                       extra={k: (v.copy() if isinstance(v, np.ndarray) else v)
                              for k, v in self.extra.items()})


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.SeedSequence):
        return np.random.default_rng(seed)
    return np.random.default_rng(np.random.SeedSequence(seed))


def _lattice(lo: Sequence[int], hi: Sequence[int]) -> np.ndarray:
    """Integer lattice points lo <= k < hi (x fastest), shape (M, D)."""
    axes = [np.arange(a, b, dtype=np.int64) for a, b in zip(lo, hi)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    pts = np.stack([m.reshape(-1) for m in mesh[::-1]], axis=1)
    return pts


def _boundary_lattice(nt: Sequence[int], layers: int) -> np.ndarray:
    """Lattice indices of `layers` wall layers outside floor and side walls.

    nt = tank size in lattice cells per axis (last axis vertical).  The walls
    cover the tank height; the floor spans the full width including the wall
    layers; the top is open.  Order: lattice order (x fastest, last axis
    slowest), built one horizontal layer at a time.
    """
    dim = len(nt)
    lo = [-layers] * (dim - 1)
    hi = [n + layers for n in nt[:-1]]
    plane = _lattice(lo, hi)  # one horizontal layer, (M, dim-1)
    inside = np.ones(plane.shape[0], dtype=bool)
    for k in range(dim - 1):
        inside &= (plane[:, k] >= 0) & (plane[:, k] < nt[k])
    ring = plane[~inside]
    out = []
    for z in range(-layers, nt[-1]):
        pts = plane if z < 0 else ring
        col = np.full((pts.shape[0], 1), z, dtype=np.int64)
        out.append(np.concatenate([pts, col], axis=1))
    return np.concatenate(out, axis=0)


def dam_break(dim: int, block: Sequence[int], dx: float, tank: Sequence[float], *,
              seed, alpha: float = 0.02, layers: int = 3, jitter: float = 1e-3,
              h_factor: float = 1.3, rho0: float = 1000.0, gamma: float = 7.0,
              visc_eps: float = 0.01, steps: int = 1, name: str = "",
              c0: Optional[float] = None, dom_height_factor: float = 2.0,
              cells_per_radius: Optional[int] = None) -> Case:
    """A dam-break particle set.

    block: fluid lattice counts per axis; tank: tank extent (m) per axis.
    The speed of sound is c0 = 10 sqrt(2 g H) with H the block height, and
    the step is dt = 0.2 h / c0 (configuration constants of the workloads).
    cells_per_radius: 1 for cells of edge 2h, 2 for cells of edge h (default
    CELLS_PER_RADIUS).
    """
    assert dim in (2, 3) and len(block) == dim and len(tank) == dim
    k = CELLS_PER_RADIUS if cells_per_radius is None else int(cells_per_radius)
    assert k in (1, 2)
    h = h_factor * dx
    cs = 2.0 * h / k
    nt = [int(round(t / dx)) for t in tank]
    for k in range(dim):
        if block[k] > nt[k]:
            raise ValueError("fluid block larger than the tank")
    fl = _lattice([0] * dim, list(block))
    bd = _boundary_lattice(nt, layers)
    rng = _rng(seed)
    r_f = (fl.astype(np.float64) + 0.5) * dx
    if jitter:
        r_f = r_f + rng.uniform(-jitter * dx, jitter * dx, size=r_f.shape)
    r_b = (bd.astype(np.float64) + 0.5) * dx
    r = np.concatenate([r_f, r_b], axis=0)
    n_f = r_f.shape[0]
    kind = np.concatenate([np.full(n_f, FLUID, np.uint8),
                           np.full(r_b.shape[0], BOUNDARY, np.uint8)])
    H = block[-1] * dx
    if c0 is None:
        c0 = 10.0 * math.sqrt(2.0 * G_EARTH * H)
    dt = 0.2 * h / c0
    g = [0.0, 0.0, 0.0]
    g[dim - 1] = -G_EARTH
    dom_min = [0.0, 0.0, 0.0]
    ncell = [1, 1, 1]
    for ax in range(dim):
        lo = -layers * dx - 2.0 * h
        if ax < dim - 1:
            hi = nt[ax] * dx + layers * dx + 2.0 * h
        else:
            hi = dom_height_factor * nt[ax] * dx
        dom_min[ax] = lo
        ncell[ax] = int(math.ceil((hi - lo) / cs))
    return Case(name=name or f"dam_break_{dim}d", dim=dim, dx=dx, h=h, cs=cs,
                mass=rho0 * dx ** dim, rho0=rho0, c0=c0, gamma=gamma, alpha=alpha,
                visc_eps=visc_eps, dt=dt, g=tuple(g), dom_min=tuple(dom_min),
                ncell=tuple(ncell), r=r, v=np.zeros_like(r), kind=kind,
                id=np.arange(r.shape[0], dtype=np.uint32), n_fluid=n_f,
                steps=steps, block=tuple(block), tank=tuple(tank))


# --- the named workloads --------------------------------------------------

def dam_break_2d(seed=1, cells_per_radius=None) -> Case:
    """2D FP64 dam break: 64x64 fluid, dx = 0.01 m, 1.6 x 0.8 m tank, 100 steps."""
    return dam_break(2, (64, 64), 0.01, (1.6, 0.8), seed=seed, steps=100,
                     name="dam_break_2d_64x64", cells_per_radius=cells_per_radius)


def dam_break_3d(n: int = 100, seed=2, dx: Optional[float] = None,
                 tank: Sequence[float] = (1.6, 0.6, 0.6), steps: int = 1000, cells_per_radius=None) -> Case:
    """3D dam break: n^3 fluid, dx = 0.005 m (n = 100), 1.6 x 0.6 x 0.6 m tank."""
    if dx is None:
        dx = 0.5 / n
    return dam_break(3, (n, n, n), dx, tank, seed=seed, steps=steps,
                     name=f"dam_break_3d_{n}^3", cells_per_radius=cells_per_radius)


def dam_break_3d_large(seed=6, cells_per_radius=None) -> Case:
    """Large 3D dam break: 256^3 fluid, dx = 0.002 m, 1.6 x 0.6 x 0.6 m tank."""
    return dam_break(3, (256, 256, 256), 0.002, (1.6, 0.6, 0.6), seed=seed, steps=200,
                     name="dam_break_3d_256^3", cells_per_radius=cells_per_radius)


def compressed_swirl(case: Case, strain: float = 5e-3, speed: float = 1.0, seed=21) -> Case:
    """The dam-break set moved away from rest (an input for one-step checks
    whose relative errors must be well conditioned).

    The fluid block (floor at 0, top at H = block height) is compressed along
    the vertical axis by a local strain that grows linearly with depth, from
    0 at the top to `strain` at the floor: z -> z - strain (H z - z^2/2) / H.
    Its particles then sit closer together the deeper they are, as in a
    column that has settled under gravity (5e-3 at the floor is the
    compression of the workloads' weakly compressible fluid under its own
    weight, since their c0^2 = 200 g H).  Fluid velocities are the
    divergence-free swirl v = U (sin(pi x/W) cos(pi z/H), [sin(pi y/W)
    cos(pi z/H),] -(H/W) (cos(pi x/W) [+ cos(pi y/W)]) sin(pi z/H)) with
    U = `speed` and W the block width, plus seeded N(0, (0.01 U)^2) noise per
    component.  Boundary particles are unchanged (at rest).
    """
    c = case.copy()
    D = c.dim
    fl = c.kind == FLUID
    H = c.block[-1] * c.dx
    W = c.block[0] * c.dx
    z = c.r[fl, D - 1]
    c.r[fl, D - 1] = z - strain * (H * z - 0.5 * z * z) / H
    x = c.r[fl, 0]
    zz = c.r[fl, D - 1]
    U = speed
    v = np.zeros((int(fl.sum()), D))
    cz = np.cos(math.pi * zz / H)
    sz = np.sin(math.pi * zz / H)
    v[:, 0] = U * np.sin(math.pi * x / W) * cz
    horiz = np.cos(math.pi * x / W)
    if D == 3:
        y = c.r[fl, 1]
        v[:, 1] = U * np.sin(math.pi * y / W) * cz
        horiz = horiz + np.cos(math.pi * y / W)
    v[:, D - 1] = -U * (H / W) * horiz * sz
    v += _rng(seed).normal(0.0, 0.01 * U, size=v.shape)
    c.v[fl] = v
    c.name = case.name + "_compressed_swirl"
    return c


def diff_case(seed=4, target_seed=5, n: int = 128, steps: int = 200, cells_per_radius=None) -> Case:
    """Differentiable 2D case: n x n fluid at dx = 0.01 m, v0 ~ N(0, 0.01) m/s.

    The tank is 2.5 x 1.25 times the block; the loss target is the initial
    fluid position plus N(0, (0.5 dx)^2) per coordinate (seeded separately).
    """
    dx = 0.01
    W = n * dx
    c = dam_break(2, (n, n), dx, (2.5 * W, 1.25 * W), seed=seed, steps=steps,
                  name=f"diff_2d_{n}x{n}", cells_per_radius=cells_per_radius)
    rng = _rng(np.random.SeedSequence([seed, 1]))
    v = np.zeros_like(c.r)
    v[: c.n_fluid] = rng.normal(0.0, 0.01, size=(c.n_fluid, 2))
    c.v = v
    trng = _rng(target_seed)
    c.target = c.r[: c.n_fluid] + trng.normal(0.0, 0.5 * dx, size=(c.n_fluid, 2))
    return c


def batched_cases(seed=3, ncases: int = 256, lo: int = 1024, hi: int = 65536,
                  dx: float = 0.01, steps: int = 500, cells_per_radius=None) -> List[Case]:
    """Independent 2D dam breaks with log-uniform fluid counts in [lo, hi].

    Per case: count N = round(exp(U[ln lo, ln hi])), block nx = round(sqrt N),
    ny = round(N / nx), tank = (2.5 nx dx, 1.25 ny dx), alpha ~ U[0.01, 0.05],
    and its own jitter stream; each case's seeds are spawned from `seed`.
    """
    root = np.random.SeedSequence(seed)
    children = root.spawn(ncases)
    out = []
    for i, ss in enumerate(children):
        rng = np.random.default_rng(ss)
        cnt = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        nx = max(1, int(round(math.sqrt(cnt))))
        ny = max(1, int(round(cnt / nx)))
        alpha = float(rng.uniform(0.01, 0.05))
        jit = ss.spawn(1)[0]
        c = dam_break(2, (nx, ny), dx, (2.5 * nx * dx, 1.25 * ny * dx), seed=jit,
                      alpha=alpha, steps=steps, name=f"batch_{i}", cells_per_radius=cells_per_radius)
        out.append(c)
    return out


def small_dam_break(dim: int, n: int, seed=11, dx: float = 0.01, alpha: float = 0.02,
                    tank_factor: Tuple[float, float] = (2.5, 1.25), steps: int = 1,
                    cells_per_radius=None) -> Case:
    """A small dam break for parity tests: n^D fluid in a tank 2.5 n dx wide and
    1.25 n dx high (same proportions as the batched cases)."""
    W = n * dx
    tank = [tank_factor[0] * W] * (dim - 1) + [tank_factor[1] * W]
    if dim == 3:
        tank[1] = 1.5 * W
    return dam_break(dim, (n,) * dim, dx, tank, seed=seed, alpha=alpha, steps=steps,
                     name=f"small_{dim}d_{n}", cells_per_radius=cells_per_radius)


def random_cloud(dim: int, n: int, seed, h: float = 0.013, box: float = 0.1,
                 fluid_frac: float = 0.7, cells_per_radius: int = 1) -> Case:
    """Uniform random particles in a box (for neighbour-search tests); cells
    of edge 2h / cells_per_radius, a margin of 2h around the box."""
    rng = _rng(seed)
    r = rng.uniform(0.0, box, size=(n, dim))
    cs = 2.0 * h / int(cells_per_radius)
    dom_min = [0.0, 0.0, 0.0]
    ncell = [1, 1, 1]
    for k in range(dim):
        dom_min[k] = -2.0 * h
        ncell[k] = int(math.ceil((box + 4.0 * h) / cs))
    nf = int(round(fluid_frac * n))
    kind = np.concatenate([np.zeros(nf, np.uint8), np.ones(n - nf, np.uint8)])
    perm = rng.permutation(n).astype(np.uint32)
    g = [0.0, 0.0, 0.0]
    g[dim - 1] = -G_EARTH
    dx = h / 1.3
    return Case(name=f"cloud_{dim}d_{n}", dim=dim, dx=dx, h=h, cs=cs,
                mass=1000.0 * dx ** dim, rho0=1000.0, c0=20.0, gamma=7.0, alpha=0.02,
                visc_eps=0.01, dt=0.2 * h / 20.0, g=tuple(g), dom_min=tuple(dom_min),
                ncell=tuple(ncell), r=r, v=rng.normal(0, 0.1, size=(n, dim)), kind=kind,
                id=perm, n_fluid=nf)


# --- the paper's own forms: Example 1a and the sampling benchmark -----------
#
# Boundary treatment codes of a domain axis (Section 3.2.1).
BC_CUTOFF = 0
BC_SYMMETRIC = 1
BC_PERIODIC = 2

MODEL_WCSPH = 0
MODEL_EXAMPLE_1A = 1
MODEL_DEM = 2


def example_1a(scale: int = 1) -> Case:
    """The dam break of Example 1a (Section 5.1.1, Appendix A) at `scale`
    times its resolution.

    Appendix A: rho0 = 1000, h = 0.25 m, dx = h/1.1, c = 50 m/s, m = dx^2
    rho0, g = (0, -9.81), dt = 1e-3 s, cells of edge 2h, the domain
    [0, 7/h cells] x [0, 10/h cells] (14 m x 20 m) with symmetric faces, and
    a water block of 7 m x 4 m at the origin filled on the dx grid.  At
    scale s the lengths h, dx and the step dt shrink by s and the cell
    counts grow by s (same 14 m x 20 m domain, same CFL number).  The block
    holds floor(7/dx) x floor(4/dx) particles at ((i+1/2)dx, (j+1/2)dx),
    at rest with rho = rho0.
    """
    s = int(scale)
    h = 0.25 / s
    dx = h / 1.1
    cs = 2.0 * h
    nx = int(math.floor(7.0 / dx + 1e-9))
    ny = int(math.floor(4.0 / dx + 1e-9))
    pts = _lattice([0, 0], [nx, ny])
    r = (pts.astype(np.float64) + 0.5) * dx
    n = r.shape[0]
    rho0 = 1000.0
    return Case(name=f"example_1a_x{s}", dim=2, dx=dx, h=h, cs=cs, mass=rho0 * dx * dx, rho0=rho0,
                c0=50.0, gamma=1.0, alpha=0.1, visc_eps=0.0, dt=1e-3 / s, g=(0.0, -G_EARTH, 0.0),
                dom_min=(0.0, 0.0, 0.0), ncell=(28 * s, 40 * s, 1), r=r, v=np.zeros_like(r),
                kind=np.zeros(n, np.uint8), id=np.arange(n, dtype=np.uint32), n_fluid=n,
                block=(nx, ny), tank=(14.0, 20.0), model=MODEL_EXAMPLE_1A,
                bc=(BC_SYMMETRIC, BC_SYMMETRIC, BC_CUTOFF), rho=np.full(n, rho0))


def paper_box(dim: int, block: Sequence[int], ncell: Sequence[int], bc: Sequence[int], *, seed,
              dx: float = 0.01, h_factor: float = 1.1, cs_factor: float = 1.0, v_sigma: float = 0.0,
              rho_sigma: float = 0.0, jitter: float = 0.0, offset: Sequence[float] = (),
              c: float = 20.0, visc: float = 0.1, g: Optional[Sequence[float]] = None,
              shuffle_ids: bool = True) -> Case:
    """A small Example 1a-form case for tests: a lattice block of fluid
    (`block` particles per axis, spacing dx, starting `offset` lattice
    cells from dom_min = 0) in a grid of `ncell` cells of edge cs_factor * 2h
    with boundary treatment `bc` per axis; seeded velocities N(0, v_sigma),
    densities rho0 (1 + N(0, rho_sigma)) and jitter U(+-jitter dx)."""
    rng = _rng(seed)
    h = h_factor * dx
    cs = cs_factor * 2.0 * h
    off = list(offset) + [0.0] * (dim - len(offset))
    pts = _lattice([0] * dim, list(block)).astype(np.float64)
    r = (pts + 0.5 + np.asarray(off[:dim])) * dx
    if jitter:
        r = r + rng.uniform(-jitter * dx, jitter * dx, size=r.shape)
    n = r.shape[0]
    rho0 = 1000.0
    v = rng.normal(0.0, v_sigma, size=r.shape) if v_sigma else np.zeros_like(r)
    rho = rho0 * (1.0 + rng.normal(0.0, rho_sigma, size=n)) if rho_sigma else np.full(n, rho0)
    ids = rng.permutation(n).astype(np.uint32) if shuffle_ids else np.arange(n, dtype=np.uint32)
    gg = [0.0, 0.0, 0.0]
    if g is None:
        gg[dim - 1] = -G_EARTH
    else:
        gg[: len(g)] = list(g)
    nc = list(ncell) + [1] * (3 - len(ncell))
    bb = list(bc) + [BC_CUTOFF] * (3 - len(bc))
    return Case(name=f"paper_box_{dim}d_{n}", dim=dim, dx=dx, h=h, cs=cs, mass=rho0 * dx ** dim,
                rho0=rho0, c0=c, gamma=1.0, alpha=visc, visc_eps=0.0, dt=0.1 * h / c, g=tuple(gg),
                dom_min=(0.0, 0.0, 0.0), ncell=tuple(nc), r=r, v=v, kind=np.zeros(n, np.uint8), id=ids,
                n_fluid=n, model=MODEL_EXAMPLE_1A, bc=tuple(bb), rho=rho)


def periodic_cube(n_side: int, *, seed=7, dx: float = 0.01, h_factor: float = 1.1,
                  rho_sigma: float = 0.0, jitter: float = 0.0, shuffle_ids: bool = True) -> Case:
    """The workload of the performance benchmark of Section 6: n_side^3
    particles on a uniform rectilinear grid filling a cube with periodic
    faces, and a scalar field A to sample.

    The cube has edge L = n_side dx (particles at (i+1/2) dx); the cell grid
    has nc = floor(L / 2h) cells of edge L / nc >= 2h per axis (n_side >= 3
    at h = 1.1 dx).  Fields: A ~ U(0, 1), m = rho0 dx^3, rho = rho0 (1 +
    N(0, rho_sigma)); seeded.  extra holds "A" and "m"; case.rho the
    density.
    """
    rng = _rng(seed)
    h = h_factor * dx
    L = n_side * dx
    nc = int(math.floor(L / (2.0 * h)))
    while nc > 1 and L / nc < 2.0 * h:     # rounding: keep the cell edge >= 2h
        nc -= 1
    if nc < 1 or L / nc < 2.0 * h:
        raise ValueError("periodic cube smaller than the kernel support (n_side too small)")
    cs = L / nc
    pts = _lattice([0, 0, 0], [n_side] * 3).astype(np.float64)
    r = (pts + 0.5) * dx
    if jitter:
        r = r + rng.uniform(-jitter * dx, jitter * dx, size=r.shape)
    n = r.shape[0]
    rho0 = 1000.0
    A = rng.uniform(0.0, 1.0, size=n)
    m = np.full(n, rho0 * dx ** 3)
    rho = rho0 * (1.0 + rng.normal(0.0, rho_sigma, size=n)) if rho_sigma else np.full(n, rho0)
    ids = rng.permutation(n).astype(np.uint32) if shuffle_ids else np.arange(n, dtype=np.uint32)
    return Case(name=f"periodic_cube_{n_side}^3", dim=3, dx=dx, h=h, cs=cs, mass=rho0 * dx ** 3,
                rho0=rho0, c0=1.0, gamma=1.0, alpha=0.0, visc_eps=0.0, dt=0.0, g=(0.0, 0.0, 0.0),
                dom_min=(0.0, 0.0, 0.0), ncell=(nc, nc, nc), r=r, v=np.zeros_like(r),
                kind=np.zeros(n, np.uint8), id=ids, n_fluid=n, model=MODEL_EXAMPLE_1A,
                bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC), rho=rho, extra={"A": A, "m": m})


def dem_damper(nx: int = 9, ny: int = 9, nz: int = 7, *, R: float = 0.004, spacing: Optional[float] = None,
               L: Optional[Sequence[float]] = None, rho: float = 7850.0, E: float = 2.06e6, nu: float = 0.33,
               cf: float = 0.3, dt: float = 5e-5, tank_M: Optional[float] = None, S: float = 78956.8,
               z0: float = -0.05, seed=8, v_sigma: float = 0.0, jitter: float = 0.0,
               radius_spread: float = 0.0) -> Case:
    """The particle damper of Example 2 (Section 5.2, table of parameters):
    spheres of radius R = 4 mm, density 7850 kg/m^3, E = 2.06 MPa, nu = 0.33
    in a cubic tank of edge L = 0.1 m (the domain, symmetric faces), tank
    mass M = 20 kg on a spring S = 78956.8 kg/s^2, released at rest from
    Z = -0.05 m; 567 = 9 x 9 x 7 spheres.

    Layout (the paper does not give one): a simple cubic lattice of spacing
    L / nx from the floor, ((i+1/2) s, (j+1/2) s, (k+1/2) s), at rest.  The
    Coulomb coefficient c_f (not given) is 0.3, the step dt = 5e-5 s (about
    1/50 of the Hertz contact time at 1 m/s).  Larger damper workloads keep
    R, the spacing and the material and scale the tank edge with the
    lattice and the tank mass with the particle count (tank_M = 20 kg x
    N / 567 unless given).  radius_spread draws radii uniformly in
    R (1 +- spread); v_sigma, jitter perturb the start (tests).
    The cell grid has cells of edge >= 2 max(R) (the contact distance).
    extra: E, nu, cf, tank_M, tank_S, z0; case.rho holds the radii and
    extra["m"] the masses.
    """
    rng = _rng(seed)
    s = (0.1 / 9.0) if spacing is None else spacing
    if L is None:
        L = (nx * s, ny * s, max(nz * s, 0.1 * max(nx, ny) / 9.0))
    pts = _lattice([0, 0, 0], [nx, ny, nz]).astype(np.float64)
    r = (pts + 0.5) * s
    n = r.shape[0]
    if jitter:
        r = r + rng.uniform(-jitter * s, jitter * s, size=r.shape)
    radii = np.full(n, R) if not radius_spread else R * (1.0 + rng.uniform(-radius_spread, radius_spread, n))
    mass = rho * 4.0 / 3.0 * math.pi * radii ** 3
    v = rng.normal(0.0, v_sigma, size=r.shape) if v_sigma else np.zeros_like(r)
    h = float(radii.max())
    # one cell edge: the largest whole fraction of the x edge that is >= 2h;
    # the other edges round up to whole cells (the tank is never smaller than
    # the lattice it holds)
    ncx = max(1, int(math.floor(L[0] / (2.0 * h))))
    while ncx > 1 and L[0] / ncx < 2.0 * h:
        ncx -= 1
    cs = L[0] / ncx
    if cs < 2.0 * h:
        raise ValueError("tank narrower than one sphere")
    nc = [ncx] + [max(1, int(math.ceil(L[k] / cs - 1e-9))) for k in (1, 2)]
    L = tuple(nc[k] * cs for k in range(3))
    M = tank_M if tank_M is not None else 20.0 * n / 567.0
    return Case(name=f"dem_damper_{n}", dim=3, dx=s, h=h, cs=cs, mass=float(mass.mean()), rho0=rho,
                c0=1.0, gamma=1.0, alpha=0.0, visc_eps=0.0, dt=dt, g=(0.0, 0.0, -G_EARTH),
                dom_min=(0.0, 0.0, 0.0), ncell=tuple(nc), r=r, v=v, kind=np.zeros(n, np.uint8),
                id=rng.permutation(n).astype(np.uint32), n_fluid=n, model=MODEL_DEM,
                bc=(BC_SYMMETRIC, BC_SYMMETRIC, BC_SYMMETRIC), rho=radii,
                extra={"E": E, "nu": nu, "cf": cf, "tank_M": M, "tank_S": S * (M / 20.0), "z0": z0,
                       "m": mass, "L": tuple(L)})


def social_force_crowd(n: int = 120, seed=12, h: float = 0.6, aspect: float = 2.4):
    """People walking along a corridor (x periodic, side walls y symmetric)
    for the social force model of Section 6 (Eq. social_force_model):
    masses m ~ U[50, 100] kg and radii R = 0.002 m + 0.15 (the paper's law),
    desired directions e0 at N(0, 0.2) rad from +x, initial speed 0.3 m/s,
    placed on a grid with U[-0.05, 0.05] m jitter.  The corridor keeps about
    1.4 people per m^2: cells of edge 2h, ncell = (aspect k, k) with k chosen
    from n.  Constants: v0 = 1.3 m/s, tau = 0.5 s, A = 2000 N, B = 0.08 m,
    k = 1.2e5 kg/s^2, no attraction (cA = 0), dt = 5 ms (Helbing's values;
    the paper lists none).  Returns (case, fields, constants)."""
    rng = _rng(seed)
    cs = 2.0 * h
    area = n / 1.4
    ky = max(2, int(round(math.sqrt(area / aspect) / cs)))
    nc = (max(3, int(round(aspect * ky))), ky)
    Lx, Ly = nc[0] * cs, nc[1] * cs
    c = paper_box(2, (1, 1), nc, (BC_PERIODIC, BC_SYMMETRIC), seed=seed, dx=h / 1.1)
    side = int(math.ceil(math.sqrt(n * Lx / Ly)))
    rows = int(math.ceil(n / side))
    gx = (np.arange(n) % side + 0.5) * (Lx / side)
    gy = (np.arange(n) // side + 0.5) * (Ly / rows)
    r = np.stack([gx + rng.uniform(-0.05, 0.05, n), gy + rng.uniform(-0.05, 0.05, n)], axis=1)
    r[:, 1] = np.clip(r[:, 1], 0.01, Ly - 0.01)
    r[:, 0] = np.mod(r[:, 0], Lx)
    m = rng.uniform(50.0, 100.0, n)
    R = 0.002 * m + 0.15
    ang = rng.normal(0.0, 0.2, n)
    e0 = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    v = 0.3 * e0
    c.r, c.v = r, v
    c.kind = np.zeros(n, np.uint8)
    c.id = rng.permutation(n).astype(np.uint32)
    c.n_fluid = n
    c.name = f"social_force_{n}"
    fields = {"v": ("vector", v), "vdot": ("vector", np.zeros((n, 2))), "e0": ("vector", e0),
              "R": ("scalar", R), "m": ("scalar", m)}
    consts = {"v0": 1.3, "tau": 0.5, "A": 2000.0, "B": 0.08, "k": 1.2e5, "cA": 0.0, "dt": 0.005}
    return c, fields, consts
