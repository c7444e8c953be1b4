"""Plain FP64 CPU oracle of the kinetic DG step (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it; the C source (``kin_oracle.c``) follows the paper's
Sec. 2.2 (kinetic algorithm), Sec. 3 (implicit upwind DG, eq. dg_imp, with
Crank-Nicolson in time, downwind solve) and Sec. 5.1 (subdomain iteration,
eq. ibvp), in FP64.

Arrays use the storage order of ``kin_oracle.h``:
``W[v][cz][cy][cx][nz][ny][nx]`` and ``f[pop][...]`` with ``pop = k*m + v``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kin_oracle.c")
_SRC_TET = os.path.join(_HERE, "kin_oracle_tet.c")
_HDR = os.path.join(_HERE, "kin_oracle.h")
_LIB = os.path.join(_HERE, "libkin_oracle.so")

ADVECTION = 0
EULER = 1
MAXWELL = 2     # 3D, W = (E, H)
AXIS = 0        # 2d velocities +-lambda e_a (D1Q2, D2Q4, D3Q6)
SIMPLEX = 1     # d + 1 velocities (D1Q2, D2Q3, D3Q4)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable: x86_64 and aarch64),
    with OpenMP when the compiler has it (the parallel loops run over the
    subdomains of one iteration and over nodes; results do not depend on the
    thread count).

    ``KIN_ORACLE_LIB`` names a prebuilt oracle library to load instead (used
    by the planted-mistake test, which builds altered copies of the source)."""
    override = os.environ.get("KIN_ORACLE_LIB")
    if override:
        return override
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _SRC_TET, _HDR))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, _SRC_TET, "-o", tmp, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)          # no OpenMP runtime: one thread
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("degree", ctypes.c_int),
        ("system", ctypes.c_int),
        ("lam", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("adv", ctypes.c_double * 3),
        ("omega", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("tiles", ctypes.c_int * 3),
        ("iters", ctypes.c_int),
        ("velset", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("inflow", ctypes.c_int * 3),
        ("Wb", ctypes.c_double * (3 * 2 * 6)),
    ]


class _TetMesh(ctypes.Structure):
    _fields_ = [
        ("ncells", ctypes.c_int),
        ("xyz", ctypes.POINTER(ctypes.c_double)),
        ("vid", ctypes.POINTER(ctypes.c_longlong)),
        ("nbr", ctypes.POINTER(ctypes.c_longlong)),
        ("sub", ctypes.POINTER(ctypes.c_int)),
        ("nsub", ctypes.c_int),
        ("wrap", ctypes.POINTER(ctypes.c_int)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        ip = ctypes.POINTER(ctypes.c_int)
        tp = ctypes.POINTER(_TetMesh)
        sig = {
            "ko_num_vars": ([pp], ctypes.c_int),
            "ko_num_vel": ([pp], ctypes.c_int),
            "ko_num_nodes": ([pp], ctypes.c_size_t),
            "ko_velocity": ([pp, ctypes.c_int, dp], ctypes.c_int),
            "ko_gll": ([ctypes.c_int, dp, dp], ctypes.c_int),
            "ko_diff_matrix": ([ctypes.c_int, dp], ctypes.c_int),
            "ko_node_coords": ([pp, dp], ctypes.c_int),
            "ko_flux": ([pp, dp, ctypes.c_int, dp], ctypes.c_int),
            "ko_maxwellian": ([pp, dp, dp], ctypes.c_int),
            "ko_cell_matrix": ([pp, ctypes.c_int, dp], ctypes.c_int),
            "ko_init": ([pp, dp, dp], ctypes.c_int),
            "ko_moments": ([pp, dp, dp], ctypes.c_int),
            "ko_transport": ([pp, dp, dp, ip], ctypes.c_int),
            "ko_relax": ([pp, dp], ctypes.c_int),
            "ko_step": ([pp, dp, ctypes.c_int], ctypes.c_int),
            "ko_mass": ([pp, dp, dp], ctypes.c_int),
            "ko_set_threads": ([ctypes.c_int], ctypes.c_int),
            "ko_init_n": ([pp, dp, dp, ctypes.c_size_t], ctypes.c_int),
            "ko_moments_n": ([pp, dp, dp, ctypes.c_size_t], ctypes.c_int),
            "ko_relax_n": ([pp, dp, ctypes.c_size_t], ctypes.c_int),
            "ko_tet_cell_matrix": ([pp, tp, ctypes.c_int, ctypes.c_int, dp, dp, dp], ctypes.c_int),
            "ko_tet_transport": ([pp, tp, dp, dp, ip], ctypes.c_int),
            "ko_tet_step": ([pp, tp, dp, ctypes.c_int], ctypes.c_int),
            "ko_tet_mass": ([pp, tp, dp, dp], ctypes.c_int),
            "ko_tet_order": ([pp, tp, ctypes.c_int, ctypes.c_int, ip, ip], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = res
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


@dataclass
class Problem:
    """A periodic Cartesian kinetic DG problem (mirrors ``ko_problem``)."""
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    degree: int
    system: int
    lam: float
    dt: float
    omega: float = 2.0
    gamma: float = 1.4
    adv: tuple = (1.0, 0.0, 0.0)
    tiles: tuple = (1, 1, 1)
    iters: int = 3
    velset: int = AXIS
    sigma: float = 0.0
    inflow: tuple = (0, 0, 0)      # 1: axis a has inflow boundaries instead of being periodic
    Wb: object = None              # boundary states, array (3 axes, 2 faces, m) (lower, upper face)
    _c: _Problem = field(default=None, repr=False, compare=False)

    def c(self) -> _Problem:
        def pad(t, fill):
            t = tuple(t)
            return t + (fill,) * (3 - len(t))
        p = _Problem()
        p.dim = self.dim
        p.n = (ctypes.c_int * 3)(*pad(self.n, 1))
        p.lo = (ctypes.c_double * 3)(*pad(self.lo, 0.0))
        p.hi = (ctypes.c_double * 3)(*pad(self.hi, 1.0))
        p.degree = self.degree
        p.system = self.system
        p.lam = self.lam
        p.gamma = self.gamma
        p.adv = (ctypes.c_double * 3)(*pad(self.adv, 0.0))
        p.omega = self.omega
        p.dt = self.dt
        p.tiles = (ctypes.c_int * 3)(*pad(self.tiles, 1))
        p.iters = self.iters
        p.velset = self.velset
        p.sigma = self.sigma
        p.inflow = (ctypes.c_int * 3)(*pad(self.inflow, 0))
        wb = np.zeros((3, 2, 6))
        if self.Wb is not None:
            a = np.asarray(self.Wb, dtype=float)
            wb[:a.shape[0], :, :a.shape[2]] = a
        p.Wb = (ctypes.c_double * 36)(*wb.reshape(-1))
        self._c = p
        return p

    @property
    def m(self) -> int:
        return lib().ko_num_vars(ctypes.byref(self.c()))

    @property
    def nvel(self) -> int:
        return lib().ko_num_vel(ctypes.byref(self.c()))

    @property
    def npop(self) -> int:
        return self.nvel * self.m

    @property
    def nodes(self) -> int:
        return int(lib().ko_num_nodes(ctypes.byref(self.c())))


def velocity(P: Problem, k: int) -> np.ndarray:
    V = np.zeros(3)
    _check(lib().ko_velocity(ctypes.byref(P.c()), k, _dp(V)), "velocity")
    return V[:P.dim]


def gll(p: int):
    xi = np.zeros(p + 1)
    w = np.zeros(p + 1)
    _check(lib().ko_gll(p, _dp(xi), _dp(w)), "gll")
    return xi, w


def diff_matrix(p: int) -> np.ndarray:
    D = np.zeros((p + 1) * (p + 1))
    _check(lib().ko_diff_matrix(p, _dp(D)), "diff_matrix")
    return D.reshape(p + 1, p + 1)


def node_coords(P: Problem) -> np.ndarray:
    xyz = np.zeros(3 * P.nodes)
    _check(lib().ko_node_coords(ctypes.byref(P.c()), _dp(xyz)), "node_coords")
    return xyz.reshape(-1, 3)


def flux(P: Problem, W, axis: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    Q = np.zeros(P.m)
    _check(lib().ko_flux(ctypes.byref(P.c()), _dp(W), axis, _dp(Q)), "flux")
    return Q


def maxwellian(P: Problem, W) -> np.ndarray:
    """M_k(W) at one point, shape (nvel, m)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    M = np.zeros(P.npop)
    _check(lib().ko_maxwellian(ctypes.byref(P.c()), _dp(W), _dp(M)), "maxwellian")
    return M.reshape(P.nvel, P.m)


def cell_matrix(P: Problem, k: int) -> np.ndarray:
    nn = (P.degree + 1) ** P.dim
    A = np.zeros(nn * nn)
    _check(lib().ko_cell_matrix(ctypes.byref(P.c()), k, _dp(A)), "cell_matrix")
    return A.reshape(nn, nn)


def init(P: Problem, W0: np.ndarray) -> np.ndarray:
    W0 = np.ascontiguousarray(W0, dtype=np.float64).reshape(-1)
    assert W0.size == P.m * P.nodes
    f = np.zeros(P.npop * P.nodes)
    _check(lib().ko_init(ctypes.byref(P.c()), _dp(W0), _dp(f)), "init")
    return f


def moments(P: Problem, f: np.ndarray) -> np.ndarray:
    W = np.zeros(P.m * P.nodes)
    _check(lib().ko_moments(ctypes.byref(P.c()), _dp(f), _dp(W)), "moments")
    return W


def transport(P: Problem, f: np.ndarray):
    """In-place CN transport; returns (per-variable interface mass defect, iterations)."""
    defect = np.zeros(P.m)
    it = ctypes.c_int(0)
    _check(lib().ko_transport(ctypes.byref(P.c()), _dp(f), _dp(defect), ctypes.byref(it)),
           "transport")
    return defect, it.value


def relax(P: Problem, f: np.ndarray) -> None:
    _check(lib().ko_relax(ctypes.byref(P.c()), _dp(f)), "relax")


def step(P: Problem, f: np.ndarray, nsteps: int = 1) -> None:
    _check(lib().ko_step(ctypes.byref(P.c()), _dp(f), nsteps), "step")


def mass(P: Problem, W: np.ndarray) -> np.ndarray:
    out = np.zeros(P.m)
    _check(lib().ko_mass(ctypes.byref(P.c()), _dp(np.ascontiguousarray(W)), _dp(out)), "mass")
    return out


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (n <= 0: unchanged); returns
    the count in use (1 when built without OpenMP)."""
    return int(lib().ko_set_threads(int(n)))


# ---------------------------------------------------------------------------
# tetrahedral meshes
# ---------------------------------------------------------------------------

class TetMesh:
    """ko_tetmesh over numpy arrays (kept alive here): xyz (cells, 4, 3),
    vid (cells, 4), nbr (cells, 4), sub (cells,) subdomain ids, wrap
    (cells, 4) periodic-boundary faces."""

    def __init__(self, xyz, vid, nbr, sub, wrap):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.vid = np.ascontiguousarray(vid, dtype=np.int64)
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int64)
        self.sub = np.ascontiguousarray(sub, dtype=np.int32)
        self.wrap = np.ascontiguousarray(wrap, dtype=np.int32)
        self.ncells = self.vid.shape[0]
        self.nsub = int(self.sub.max()) + 1
        self._c = _TetMesh(self.ncells, self.xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           self.vid.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                           self.nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                           self.sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.nsub,
                           self.wrap.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))

    @classmethod
    def from_workload(cls, w):
        return cls(w.mesh.xyz, w.mesh.vid, w.mesh.nbr, w.subdomains(), w.mesh.wrap)

    @property
    def nodes(self) -> int:
        return 4 * self.ncells


def tet_problem(w) -> Problem:
    """The ko_problem of a tetrahedral workload (its kinetic model, dt, K)."""
    return Problem(dim=3, n=(1, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1), degree=1, system=w.system, lam=w.lam,
                   dt=w.dt, omega=w.omega, gamma=w.gamma, adv=w.adv, tiles=(1, 1, 1), iters=w.iters,
                   velset=w.velset, sigma=w.sigma)


def tet_init(P: Problem, T: TetMesh, W0) -> np.ndarray:
    W0 = np.ascontiguousarray(W0, dtype=np.float64).reshape(-1)
    assert W0.size == P.m * T.nodes
    f = np.zeros(P.npop * T.nodes)
    _check(lib().ko_init_n(ctypes.byref(P.c()), _dp(W0), _dp(f), T.nodes), "tet init")
    return f


def tet_moments(P: Problem, T: TetMesh, f: np.ndarray) -> np.ndarray:
    W = np.zeros(P.m * T.nodes)
    _check(lib().ko_moments_n(ctypes.byref(P.c()), _dp(f), _dp(W), T.nodes), "tet moments")
    return W


def tet_relax(P: Problem, T: TetMesh, f: np.ndarray) -> None:
    _check(lib().ko_relax_n(ctypes.byref(P.c()), _dp(f), T.nodes), "tet relax")


def tet_transport(P: Problem, T: TetMesh, f: np.ndarray):
    defect = np.zeros(P.m)
    it = ctypes.c_int(0)
    _check(lib().ko_tet_transport(ctypes.byref(P.c()), ctypes.byref(T._c), _dp(f), _dp(defect),
                                  ctypes.byref(it)), "tet transport")
    return defect, it.value


def tet_step(P: Problem, T: TetMesh, f: np.ndarray, nsteps: int = 1) -> None:
    _check(lib().ko_tet_step(ctypes.byref(P.c()), ctypes.byref(T._c), _dp(f), nsteps), "tet step")


def tet_mass(P: Problem, T: TetMesh, W: np.ndarray) -> np.ndarray:
    out = np.zeros(P.m)
    _check(lib().ko_tet_mass(ctypes.byref(P.c()), ctypes.byref(T._c), _dp(np.ascontiguousarray(W)),
                             _dp(out)), "tet mass")
    return out


def tet_cell_matrix(P: Problem, T: TetMesh, c: int, k: int):
    """(A, M, V.N_a |F_a| per face) of cell c and velocity k."""
    A = np.zeros(16)
    M = np.zeros(16)
    vna = np.zeros(4)
    _check(lib().ko_tet_cell_matrix(ctypes.byref(P.c()), ctypes.byref(T._c), c, k, _dp(A), _dp(M), _dp(vna)),
           "tet cell matrix")
    return A.reshape(4, 4), M.reshape(4, 4), vna


def tet_order(P: Problem, T: TetMesh, k: int, s: int):
    """(cells in breadth-first topological order, their levels) of subdomain s."""
    order = np.zeros(T.ncells, dtype=np.int32)
    level = np.zeros(T.ncells, dtype=np.int32)
    n = lib().ko_tet_order(ctypes.byref(P.c()), ctypes.byref(T._c), k, s,
                           order.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           level.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if n < 0:
        raise ValueError(f"oracle tet order failed with code {n}")
    return order[:n].copy(), level[:n].copy()
