"""Seeded synthetic workloads shared by the oracle side and the CUDA side.

This module holds the problem recipes only: domain, mesh, kinetic speed,
time step, subdomain tiling and the initial data sampled at the cell nodes.
It contains none of the scheme's arithmetic (no transport, no Maxwellian, no
relaxation) and imports neither the oracle nor the CUDA library.

Storage order of a macroscopic field ``W``: ``[v][cz][cy][cx][nz][ny][nx]``
(cells row-major with x fastest, then the tensor Gauss-Lobatto nodes of the
cell with the x node fastest).  The node positions inside a cell are the
Gauss-Lobatto points of degree p on [0, 1], written here from their closed
forms (p <= 3) so that this module depends on nothing else.

Workloads (the paper's experiments use Maxwell on tetrahedral meshes that are
not available; these periodic Cartesian problems stand in for them):

* ``advection1d``  scalar u_t + a u_x = 0 on [0,1], D1Q2, p = 1, 256 cells,
  lambda = 2, dt = 4h/lambda, omega = 2, u0 = A sin(2 pi x) + B with
  A, B ~ U(0.5, 1.5) from the seed; FP64.
* ``vortex2d``     Euler (gamma = 1.4) on [0,10]^2, D2Q4, p = 2, 256^2 cells,
  isentropic vortex (centre ~ U(box), strength ~ U(3, 5), free stream
  rho = p = 1, u = (1, 1)), dt = 5 x the explicit DG limit, 8x8 subdomains.
* ``densitywave3d`` Euler on the periodic unit cube, D3Q6, p = 1, 128^3 cells,
  rho = 1 + 0.2 sin(2 pi (x + y + z) + phi), phi ~ U(0, 2 pi), u = (1,1,1),
  p = 1, dt = 5 x the explicit DG limit, 16^3 subdomains.
* ``densitywave2d`` the 2D analogue on [0,1]^2 (used by the batched mix).
* ``maxwell3d``    Maxwell's equations on the periodic unit cube, D3Q6, three
  superposed plane waves, optional uniform conductivity sigma.

Kinetic speed: lambda = 1.1 d max_nodes max_a (|u_a| + c), which keeps the
2d-velocity equilibria W/(2d) +- Q^a/(2 lambda) monotone.  Explicit DG limit
on Cartesian Q_p cells: dt_exp = h / ((2p + 1) d a_max).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Callable, Optional

import numpy as np

ADVECTION = 0
EULER = 1
MAXWELL = 2     # 3D only, W = (E, H)

# Gauss-Lobatto points on [0, 1] (closed forms; Abramowitz & Stegun 25.4.32).
_GLL = {
    1: (0.0, 1.0),
    2: (0.0, 0.5, 1.0),
    3: (0.0, 0.5 - 0.5 / math.sqrt(5.0), 0.5 + 0.5 / math.sqrt(5.0), 1.0),
}


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    degree: int
    system: int
    lam: float
    dt: float
    omega: float
    gamma: float
    adv: tuple
    tiles: tuple
    iters: int
    steps: int
    precision: str            # "f64" or "f32"
    W0: np.ndarray = field(repr=False)
    exact: Optional[Callable] = field(default=None, repr=False)  # exact(t) -> W
    velset: int = 0           # 0: 2d velocities +-lambda e_a; 1: d + 1 velocities (D2Q3, D3Q4)
    sigma: float = 0.0        # conductivity (Maxwell only)
    inflow: tuple = (0, 0, 0)  # 1: axis a has inflow boundaries instead of being periodic
    Wb: object = field(default=None, repr=False)   # boundary states (3 axes, 2 faces, m)

    @property
    def m(self) -> int:
        return {ADVECTION: 1, EULER: self.dim + 2, MAXWELL: 6}[self.system]

    @property
    def nvel(self) -> int:
        return self.dim + 1 if (self.velset == 1 and self.dim > 1) else 2 * self.dim

    @property
    def npop(self) -> int:
        return self.nvel * self.m

    @property
    def nodes(self) -> int:
        return int(np.prod(self.n)) * (self.degree + 1) ** self.dim

    @property
    def kinetic_dofs(self) -> int:
        return self.npop * self.nodes

    def oracle_kwargs(self) -> dict:
        return dict(dim=self.dim, n=self.n, lo=self.lo, hi=self.hi, degree=self.degree,
                    system=self.system, lam=self.lam, dt=self.dt, omega=self.omega,
                    gamma=self.gamma, adv=self.adv, tiles=self.tiles, iters=self.iters,
                    velset=self.velset, sigma=self.sigma, inflow=self.inflow, Wb=self.Wb)


def node_coords(dim, n, lo, hi, degree) -> np.ndarray:
    """Node positions (nodes, dim) in storage order."""
    xi = np.asarray(_GLL[degree])
    axes = []
    for a in range(dim):
        h = (hi[a] - lo[a]) / n[a]
        axes.append(lo[a] + (np.arange(n[a])[:, None] + xi[None, :]) * h)  # (n_a, np)
    npn = degree + 1
    if dim == 1:
        return axes[0].reshape(-1, 1)
    if dim == 2:
        X = np.broadcast_to(axes[0][None, :, None, :], (n[1], n[0], npn, npn))
        Y = np.broadcast_to(axes[1][:, None, :, None], (n[1], n[0], npn, npn))
        return np.stack([X.reshape(-1), Y.reshape(-1)], axis=1)
    X = np.broadcast_to(axes[0][None, None, :, None, None, :], (n[2], n[1], n[0], npn, npn, npn))
    Y = np.broadcast_to(axes[1][None, :, None, None, :, None], (n[2], n[1], n[0], npn, npn, npn))
    Z = np.broadcast_to(axes[2][:, None, None, :, None, None], (n[2], n[1], n[0], npn, npn, npn))
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)


def _tiles(tiles, dim):
    return tuple(tiles) if isinstance(tiles, (tuple, list)) else (int(tiles),) * dim


def _euler_conserved(rho, vel, pr, gamma):
    d = len(vel)
    E = pr / (gamma - 1.0) + 0.5 * rho * sum(u * u for u in vel)
    return np.stack([rho] + [rho * u for u in vel] + [E], axis=0)


def _max_speed(rho, vel, pr, gamma):
    c = np.sqrt(gamma * pr / rho)
    return float(max(np.max(np.abs(u) + c) for u in vel))


def advection1d(seed: int = 0, n: int = 256, tiles: int = 1, iters: int = 3,
                lam: float = 2.0, a: float = 1.0, dt: Optional[float] = None,
                omega: float = 2.0, steps: int = 100, degree: int = 1,
                precision: str = "f64") -> Workload:
    rng = np.random.default_rng(seed)
    A, B = rng.uniform(0.5, 1.5, size=2)
    h = 1.0 / n
    if dt is None:
        dt = 4.0 * h / lam
    x = node_coords(1, (n,), (0.0,), (1.0,), degree)[:, 0]

    def u0(xx):
        return A * np.sin(2 * np.pi * xx) + B

    def exact(t):
        return u0((x - a * t) % 1.0)[None, :]

    return Workload("advection1d", 1, (n,), (0.0,), (1.0,), degree, ADVECTION, lam, dt, omega, 1.4,
                    (a, 0.0, 0.0), _tiles(tiles, 1), iters, steps, precision,
                    u0(x)[None, :].copy(), exact)


def _vortex_fields(X, Y, xc, yc, eps, gamma, box, uinf, vinf):
    dx = X - xc
    dy = Y - yc
    dx -= box * np.round(dx / box)     # minimum image on the periodic box
    dy -= box * np.round(dy / box)
    r2 = dx * dx + dy * dy
    e = np.exp(0.5 * (1.0 - r2))
    u = uinf - eps / (2 * np.pi) * e * dy
    v = vinf + eps / (2 * np.pi) * e * dx
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi * np.pi) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    pr = rho ** gamma
    return rho, (u, v), pr


def vortex2d(seed: int = 0, n: int = 256, degree: int = 2, tiles: int = 8, iters: int = 3,
             dt_mult: float = 5.0, omega: float = 2.0, steps: int = 200,
             precision: str = "f32", box: float = 10.0, velset: int = 0) -> Workload:
    rng = np.random.default_rng(seed)
    xc, yc = rng.uniform(0.0, box, size=2)
    eps = rng.uniform(3.0, 5.0)
    gamma = 1.4
    uinf, vinf = 1.0, 1.0
    xyz = node_coords(2, (n, n), (0.0, 0.0), (box, box), degree)
    X, Y = xyz[:, 0], xyz[:, 1]
    rho, vel, pr = _vortex_fields(X, Y, xc, yc, eps, gamma, box, uinf, vinf)
    amax = _max_speed(rho, vel, pr, gamma)
    lam = (SIMPLEX_LAMBDA[2] if velset == 1 else 1.1 * 2) * amax
    h = box / n
    dt = dt_mult * h / ((2 * degree + 1) * 2 * amax)

    def exact(t):
        r, vv, p = _vortex_fields(X, Y, xc + uinf * t, yc + vinf * t, eps, gamma, box, uinf, vinf)
        return _euler_conserved(r, vv, p, gamma)

    W0 = _euler_conserved(rho, vel, pr, gamma)
    return Workload("vortex2d", 2, (n, n), (0.0, 0.0), (box, box), degree, EULER, lam, dt, omega,
                    gamma, (0.0, 0.0, 0.0), _tiles(tiles, 2), iters, steps, precision, W0, exact,
                    velset)


# Kinetic speed factor for the d + 1 velocity sets (lambda = factor * a_max):
# D2Q3 (|V_k| = lambda) and D3Q4 (components +-lambda); chosen with margin
# above the stability limits observed with the FP64 oracle at omega = 2: the
# vortex with D2Q3 at factor 2.0 blows up near step 80 (64^2) or 100 (256^2),
# at 2.5 it runs 400 steps (64^2) and 200 steps (256^2) stably.
SIMPLEX_LAMBDA = {2: 2.5, 3: 1.5}


def _densitywave(dim, seed, n, degree, tiles, iters, dt_mult, omega, steps, precision, amp=0.2,
                 velset=0):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2 * np.pi)
    gamma = 1.4
    vel0 = (1.0,) * dim
    lo, hi = (0.0,) * dim, (1.0,) * dim
    xyz = node_coords(dim, (n,) * dim, lo, hi, degree)
    s = xyz.sum(axis=1)

    def fields(t):
        rho = 1.0 + amp * np.sin(2 * np.pi * (s - dim * t) + phi)
        vel = tuple(np.full_like(rho, u) for u in vel0)
        pr = np.ones_like(rho)
        return rho, vel, pr

    rho, vel, pr = fields(0.0)
    amax = _max_speed(rho, vel, pr, gamma)
    lam = (SIMPLEX_LAMBDA[dim] if velset == 1 else 1.1 * dim) * amax
    h = 1.0 / n
    dt = dt_mult * h / ((2 * degree + 1) * dim * amax)

    def exact(t):
        r, vv, p = fields(t)
        return _euler_conserved(r, vv, p, gamma)

    return Workload(f"densitywave{dim}d", dim, (n,) * dim, lo, hi, degree, EULER, lam, dt, omega,
                    gamma, (0.0, 0.0, 0.0), _tiles(tiles, dim), iters, steps, precision,
                    _euler_conserved(rho, vel, pr, gamma), exact, velset)


def densitywave3d(seed: int = 0, n: int = 128, degree: int = 1, tiles: int = 16, iters: int = 3,
                  dt_mult: float = 5.0, omega: float = 2.0, steps: int = 200,
                  precision: str = "f32", velset: int = 0) -> Workload:
    return _densitywave(3, seed, n, degree, tiles, iters, dt_mult, omega, steps, precision,
                        velset=velset)


def densitywave2d(seed: int = 0, n: int = 64, degree: int = 1, tiles: int = 2, iters: int = 3,
                  dt_mult: float = 5.0, omega: float = 2.0, steps: int = 100,
                  precision: str = "f32", velset: int = 0) -> Workload:
    return _densitywave(2, seed, n, degree, tiles, iters, dt_mult, omega, steps, precision,
                        velset=velset)


def maxwell3d(seed: int = 0, n: int = 64, degree: int = 1, tiles: int = 16, iters: int = 3,
              dt_mult: float = 5.0, omega: float = 2.0, sigma: float = 0.0, steps: int = 100,
              precision: str = "f32") -> Workload:
    """Maxwell (light speed 1) on the periodic unit cube, D3Q6: three plane
    waves, along x (E_y = H_z), along y (E_z = H_x) and along z (E_x = H_y),
    each cos(2 pi (s - t) + phi_k) with phases phi_k ~ U(0, 2 pi) and
    amplitudes ~ U(0.5, 1.5) from the seed; lambda = 3.3 (1.1 d x the light
    speed); dt = dt_mult x h / ((2p + 1) d).  With sigma = 0 the exact
    solution is the translated waves; with sigma > 0 there is no closed form
    here (exact = None)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2 * np.pi, size=3)
    amp = rng.uniform(0.5, 1.5, size=3)
    lo, hi = (0.0,) * 3, (1.0,) * 3
    xyz = node_coords(3, (n,) * 3, lo, hi, degree)

    def fields(t):
        W = np.zeros((6, xyz.shape[0]))
        # (propagation axis a, E component, H component): E x H points along +e_a
        for k, (a, e, h) in enumerate(((0, 1, 2), (1, 2, 0), (2, 0, 1))):
            c = amp[k] * np.cos(2 * np.pi * (xyz[:, a] - t) + phi[k])
            W[e] += c
            W[3 + h] += c
        return W

    h = 1.0 / n
    dt = dt_mult * h / ((2 * degree + 1) * 3)
    exact = fields if sigma == 0.0 else None
    return Workload("maxwell3d", 3, (n,) * 3, lo, hi, degree, MAXWELL, 3.3, dt, omega, 1.4,
                    (0.0, 0.0, 0.0), _tiles(tiles, 3), iters, steps, precision, fields(0.0), exact,
                    0, sigma)


def with_(w: Workload, **kw) -> Workload:
    """Copy of a workload with some recipe fields replaced (initial data kept)."""
    return replace(w, **kw)


def batched_mix(seed: int = 0, count: int = 64, sizes=(64, 128, 256, 512), degrees=(1, 2, 3),
                dt_range=(2.0, 8.0), steps: int = 100):
    """Uneven 2D Euler/D2Q4 instances: n ~ sizes, p ~ degrees, vortex or density
    wave 50/50, dt multiple ~ U(dt_range); subdomains of 32 cells per side."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        p = int(rng.choice(degrees))
        mult = float(rng.uniform(*dt_range))
        sub_seed = int(rng.integers(0, 2 ** 31 - 1))
        tiles = max(1, n // 32)
        if rng.uniform() < 0.5:
            w = vortex2d(seed=sub_seed, n=n, degree=p, tiles=tiles, dt_mult=mult, steps=steps)
        else:
            w = densitywave2d(seed=sub_seed, n=n, degree=p, tiles=tiles, dt_mult=mult, steps=steps)
        out.append(w)
    return out


@dataclass
class Request:
    """One simulation request of a serving stream."""
    rid: int
    arrival: float        # seconds after the start of the stream
    kind: str             # "vortex" or "densitywave"
    n: int
    degree: int
    steps: int
    seed: int


def serving_stream(seed: int = 0, count: int = 64, rate: float = 200.0, sizes=(64, 128, 256, 512, 1024),
                   degrees=(1, 2, 3), steps=(50, 500), size_range=None, size_step: int = 32):
    """Poisson arrivals (mean 'rate' per second) of 2D Euler / D2Q4 requests:
    DG degree uniform in 'degrees', step count uniform in [steps[0],
    steps[1]], vortex or density wave 50/50.  Mesh n x n: with size_range =
    (lo, hi), n is log-uniform on [lo, hi] rounded to a multiple of size_step
    (the 32-cell subdomain extent) -- the serving configuration's
    64^2..1024^2; otherwise n is uniform over the list 'sizes'."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = "vortex" if rng.uniform() < 0.5 else "densitywave"
        if size_range is not None:
            lo, hi = size_range
            n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
            n = int(min(hi, max(lo, size_step * round(n / size_step))))
        else:
            n = int(rng.choice(sizes))
        out.append(Request(i, t, kind, n, int(rng.choice(degrees)),
                           int(rng.integers(steps[0], steps[1] + 1)), int(rng.integers(0, 8))))
    return out


_request_cache = {}


def request_workload(r: Request, cache: bool = True) -> Workload:
    """The problem of a request (dt = 5 x the explicit DG limit, 32-cell
    subdomains, FP32).  Initial data of equal (kind, n, degree, seed) are
    generated once and shared."""
    key = (r.kind, r.n, r.degree, r.seed)
    if cache and key in _request_cache:
        w = _request_cache[key]
    else:
        tiles = max(1, r.n // 32)
        if r.kind == "vortex":
            w = vortex2d(seed=r.seed, n=r.n, degree=r.degree, tiles=tiles)
        else:
            w = densitywave2d(seed=r.seed, n=r.n, degree=r.degree, tiles=tiles)
        if cache:
            _request_cache[key] = w
    return replace(w, steps=r.steps)


# ---------------------------------------------------------------------------
# tetrahedral meshes (the paper's setting: unstructured tetrahedral cells)
# ---------------------------------------------------------------------------

@dataclass
class TetMesh:
    """A conforming tetrahedral mesh of a periodic box: every cube of an
    n x n x n grid split into six tetrahedra along its main diagonal.
    Cell c has local vertices a = 0..3; its face a is the one opposite vertex
    a.  Arrays: xyz (cells, 4, 3) vertex coordinates, unwrapped so that each
    cell is a geometric tetrahedron; vid (cells, 4) global vertex ids
    (periodic); nbr (cells, 4) the cell across face a; wrap (cells, 4) 1
    where face a crosses the periodic boundary of the box (the two cells'
    copies of the face lie one period apart); cube (cells, 3) the parent
    cube.  Connectivity only: no geometry of the method is computed here."""
    n: int
    lo: tuple
    hi: tuple
    xyz: np.ndarray = field(repr=False)
    vid: np.ndarray = field(repr=False)
    nbr: np.ndarray = field(repr=False)
    cube: np.ndarray = field(repr=False)
    wrap: np.ndarray = field(default=None, repr=False)

    @property
    def cells(self) -> int:
        return self.vid.shape[0]

    def subdomains(self, tiles: int) -> np.ndarray:
        """Subdomain id per cell: the parent cubes cut into tiles^3 boxes."""
        L = self.n // tiles
        t = self.cube // L
        return (t[:, 2] * tiles + t[:, 1]) * tiles + t[:, 0]

    def node_coords(self) -> np.ndarray:
        """(cells * 4, 3): the P1 nodes (the vertices of every cell), cell-major."""
        return self.xyz.reshape(-1, 3)


_KUHN = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def tet_box(n: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> TetMesh:
    """Periodic box [lo, hi]^3 of n^3 cubes (n >= 2), six tetrahedra per cube:
    vertex 0 at the cube's lower corner, then one step along each axis in the
    order of a permutation of (x, y, z), ending at the upper corner."""
    if n < 2:
        raise ValueError("n must be at least 2 (periodic vertex ids must separate the faces)")
    lo = np.asarray(lo, float)
    h = (np.asarray(hi, float) - lo) / n
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for perm in _KUHN:
                    p = np.array([i, j, k])
                    pts = [p.copy()]
                    for a in perm:
                        p = p.copy()
                        p[a] += 1
                        pts.append(p)
                    cells.append(pts)
    ijk = np.array(cells)                                      # (cells, 4, 3) integer lattice points
    xyz = lo + ijk * h
    w = ijk % n
    vid = (w[..., 2] * n + w[..., 1]) * n + w[..., 0]
    cube = ijk[:, 0, :]
    # faces: the three vertex ids other than a, shared by exactly two cells
    owner = {}
    nbr = -np.ones((len(cells), 4), dtype=np.int64)
    for c in range(len(cells)):
        for a in range(4):
            key = tuple(sorted(int(vid[c, b]) for b in range(4) if b != a))
            if key in owner:
                c2, a2 = owner.pop(key)
                nbr[c, a] = c2
                nbr[c2, a2] = c
            else:
                owner[key] = (c, a)
    if owner or (nbr < 0).any():
        raise ValueError("tet_box: the mesh is not closed")
    # a face wraps when the lattice points of its vertices differ between the
    # two cells (they agree modulo n)
    wrap = np.zeros((len(cells), 4), dtype=np.int32)
    for c in range(len(cells)):
        for a in range(4):
            R = nbr[c, a]
            for b in range(4):
                if b == a:
                    continue
                j = int(np.nonzero(vid[R] == vid[c, b])[0][0])
                if (ijk[R, j] != ijk[c, b]).any():
                    wrap[c, a] = 1
                    break
    return TetMesh(n, tuple(lo), tuple(hi), xyz, vid.astype(np.int64), nbr, cube.astype(np.int64), wrap)


@dataclass
class TetWorkload:
    """A kinetic DG problem on a tetrahedral mesh (P1 nodal basis, the four
    vertices of each cell): the recipe and the initial data at the nodes,
    W0 (m, cells * 4)."""
    name: str
    mesh: TetMesh
    system: int
    velset: int               # 0: D3Q6 (+-lambda e_a), 1: D3Q4 (cube diagonals, Sec. 6.1.3)
    lam: float
    dt: float
    omega: float
    gamma: float
    adv: tuple
    tiles: int
    iters: int
    precision: str
    W0: np.ndarray = field(repr=False)
    exact: Optional[Callable] = field(default=None, repr=False)
    sigma: float = 0.0

    @property
    def m(self) -> int:
        return {ADVECTION: 1, EULER: 5, MAXWELL: 6}[self.system]

    @property
    def nvel(self) -> int:
        return 4 if self.velset == 1 else 6

    @property
    def npop(self) -> int:
        return self.nvel * self.m

    @property
    def nodes(self) -> int:
        return 4 * self.mesh.cells

    @property
    def kinetic_dofs(self) -> int:
        return self.npop * self.nodes

    def subdomains(self) -> np.ndarray:
        return self.mesh.subdomains(self.tiles)


def tet_h_min(mesh: TetMesh) -> float:
    """h_min = volume / surface of the Kuhn tetrahedra (all congruent), the
    length in the paper's CFL-number definition that the recipes' time steps
    use: for a cube of side h a cell has volume h^3/6 and two faces of area
    h^2/2 and two of area h^2 sqrt(2)/2."""
    h = (mesh.hi[0] - mesh.lo[0]) / mesh.n
    vol = h ** 3 / 6.0
    surf = 2 * (h * h / 2.0) + 2 * (h * h * math.sqrt(2.0) / 2.0)
    return vol / surf


def tet_densitywave(seed: int = 0, n: int = 16, tiles: int = 2, velset: int = 1, dt_mult: float = 5.0,
                    iters: int = 3, omega: float = 2.0, precision: str = "f32", amp: float = 0.2) -> TetWorkload:
    """3D Euler density wave rho = 1 + amp sin(2 pi (x + y + z) + phi),
    u = (1, 1, 1), p = 1 (phi ~ U(0, 2 pi) from the seed) on the periodic
    unit cube meshed by tet_box(n); subdomains of (n / tiles)^3 cubes.
    Kinetic speed: D3Q4 lambda = 1.5 a_max, D3Q6 lambda = 3.3 a_max.  Time
    step: dt = dt_mult x h_min / |V|_max with h_min = vol / surf (the paper's
    CFL-number definition; dt_mult = 1 is the explicit DG limit)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2 * np.pi)
    gamma = 1.4
    mesh = tet_box(n)
    xyz = mesh.node_coords()
    s = xyz.sum(axis=1)

    def fields(t):
        rho = 1.0 + amp * np.sin(2 * np.pi * (s - 3 * t) + phi)
        vel = tuple(np.ones_like(rho) for _ in range(3))
        return rho, vel, np.ones_like(rho)

    rho, vel, pr = fields(0.0)
    amax = _max_speed(rho, vel, pr, gamma)
    lam = (SIMPLEX_LAMBDA[3] if velset == 1 else 1.1 * 3) * amax
    vmax = lam * math.sqrt(3.0) if velset == 1 else lam
    dt = dt_mult * tet_h_min(mesh) / vmax

    def exact(t):
        r, vv, p = fields(t)
        return _euler_conserved(r, vv, p, gamma)

    return TetWorkload("tet-densitywave", mesh, EULER, velset, lam, dt, omega, gamma, (0.0, 0.0, 0.0), tiles,
                       iters, precision, _euler_conserved(rho, vel, pr, gamma), exact)


def tet_advection(seed: int = 0, n: int = 8, tiles: int = 1, velset: int = 1, dt_mult: float = 5.0,
                  iters: int = 3, omega: float = 2.0, adv=(1.0, 0.5, 0.25), lam: float = 2.0,
                  precision: str = "f64") -> TetWorkload:
    """Scalar advection u_t + a . grad u = 0 on the periodic unit cube meshed
    by tet_box(n): u0 = A sin(2 pi (x + 2y - z) + phi) + B with A, B ~
    U(0.5, 1.5), phi ~ U(0, 2 pi) from the seed."""
    rng = np.random.default_rng(seed)
    A, B = rng.uniform(0.5, 1.5, size=2)
    phi = rng.uniform(0.0, 2 * np.pi)
    mesh = tet_box(n)
    xyz = mesh.node_coords()
    kvec = np.array([1.0, 2.0, -1.0])
    a = np.asarray(adv, float)

    def exact(t):
        return (A * np.sin(2 * np.pi * ((xyz - a * t) @ kvec) + phi) + B)[None, :]

    vmax = lam * math.sqrt(3.0) if velset == 1 else lam
    dt = dt_mult * tet_h_min(mesh) / vmax
    return TetWorkload("tet-advection", mesh, ADVECTION, velset, lam, dt, omega, 1.4, tuple(adv), tiles, iters,
                       precision, exact(0.0), exact)


def tet_maxwell(seed: int = 0, n: int = 8, tiles: int = 2, velset: int = 0, dt_mult: float = 5.0,
                iters: int = 3, omega: float = 2.0, sigma: float = 0.0, precision: str = "f64") -> TetWorkload:
    """Maxwell's equations (light speed 1) on the periodic unit cube meshed by
    tet_box(n): the three plane waves of maxwell3d sampled at the P1 nodes.
    Kinetic speed: D3Q6 lambda = 3.3, D3Q4 lambda = 1.5 (|V_k| = 1.5 sqrt 3)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2 * np.pi, size=3)
    amp = rng.uniform(0.5, 1.5, size=3)
    mesh = tet_box(n)
    xyz = mesh.node_coords()

    def fields(t):
        W = np.zeros((6, xyz.shape[0]))
        for k, (a, e, h) in enumerate(((0, 1, 2), (1, 2, 0), (2, 0, 1))):
            c = amp[k] * np.cos(2 * np.pi * (xyz[:, a] - t) + phi[k])
            W[e] += c
            W[3 + h] += c
        return W

    lam = 1.5 if velset == 1 else 3.3
    vmax = lam * math.sqrt(3.0) if velset == 1 else lam
    dt = dt_mult * tet_h_min(mesh) / vmax
    return TetWorkload("tet-maxwell", mesh, MAXWELL, velset, lam, dt, omega, 1.4, (0.0, 0.0, 0.0), tiles, iters,
                       precision, fields(0.0), fields if sigma == 0.0 else None, sigma)
