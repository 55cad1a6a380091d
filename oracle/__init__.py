"""FP64 CPU oracle (test infrastructure only).

Plain serial C (``oracle.c``) behind ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package; the product path never does.
It shares no code with ``paper_2212_08836_gb300`` (no headers, constants or
helpers): both sides are written from the paper (arXiv:2212.08836, Sec. 2.1,
Eqs. 2-4) and the same readings of its discretisation.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or independent library routines; see the docstrings for which.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# CODATA 2018 (defined here independently of the GPU package)
QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
M_AR = 39.948 * AMU
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no fused multiply-add).
    OpenMP, where the compiler has it, only serves the timing form of the
    push (set_threads > 1); every test runs the serial form."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads of the oracle's push (1: serial, the form every test uses;
    more: the timing form of the CPU baseline, particles split over threads
    with per-thread crossed-charge arrays summed at the end)."""
    lib().oracle_set_threads(int(n))


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_P = C.c_void_p
_I = C.c_int
_L = C.c_int64
_D = C.c_double
_U = C.c_uint64


class Species(C.Structure):
    _fields_ = [("cell", _P), ("a", _P), ("b", _P), ("vr", _P), ("vt", _P), ("vz", _P),
                ("w", _P), ("id", _P), ("n", _L), ("cap", _L), ("next_id", C.c_uint32),
                ("q", _D), ("m", _D)]


class Cfg(C.Structure):
    _fields_ = [("nr", _I), ("nz", _I), ("dr", _D), ("dz", _D), ("R", _D), ("L", _D),
                ("dt", _D), ("freq", _D), ("volt", _D), ("eps", _D), ("mu", _D), ("bz", _D),
                ("tol", _D), ("kmax", _I), ("mcc_on", _I), ("ng", _D), ("tg", _D),
                ("numax_e", _D), ("pnull_e", _D), ("pnull_i", _D), ("gmax", _D),
                ("seed", _U), ("cblock", _D), ("xa", _I), ("wave", _I), ("nd", _I),
                ("erd", _D)]


class Stats(C.Structure):
    _fields_ = [("picard_iters", _I), ("converged", _I), ("last_res", _D),
                ("src_energy", _D), ("ke_lost", _D), ("de_coll", _D),
                ("counters", _L * 4), ("mcc", _L * 8)]


def _declare(L):
    L.oracle_philox4x64.argtypes = [_P, _P, _P]
    L.oracle_load.argtypes = ([_I, _I, _D, _D, _I, _I, _D, _D, _D, _D, _L, _D, _D, _D, _D, _U]
                              + [_P] * 11)
    L.oracle_set_threads.argtypes = [_I]
    L.oracle_set_threads.restype = None
    L.oracle_push.argtypes = ([_I, _I, _D, _D, _I, _I, _D, _D, _D, _D, _D, _L] + [_P] * 11 + [_I]
                              + [_P] * 5)
    L.oracle_node_charge.argtypes = [_I, _I, _D, _L, _P, _P, _P, _P, _P]
    L.oracle_field_create.argtypes = [_I, _I, _D, _D, _I, _I, _D, _D, _D, _D, _D, _I]
    L.oracle_field_create.restype = _P
    L.oracle_field_destroy.argtypes = [_P]
    L.oracle_field_solve.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _D, _P, _P, _P, _P]
    L.oracle_port_create.argtypes = [_I, _I, _D, _D, _I, _I, _I, _D, _D, _D, _D, _D]
    L.oracle_port_create.restype = _P
    L.oracle_port_create_graded.argtypes = [_I, _I, _D, _D, _I, _I, _I, _P, _D, _D, _D, _D]
    L.oracle_port_create_graded.restype = _P
    L.oracle_port_destroy.argtypes = [_P]
    L.oracle_port_solve.argtypes = [_P] + [_P] * 8 + [_D, _D] + [_P] * 7
    L.oracle_port_energy.argtypes = [_P] * 7
    L.oracle_port_energy.restype = _D
    L.oracle_conduction_charge.argtypes = [_P, _P, _P, _P, _P, _P]
    L.oracle_conduction_charge.restype = _D
    L.oracle_field_energy.argtypes = [_I, _I, _D, _D, _I, _I, _D, _D, _D, _P, _P, _P]
    L.oracle_field_energy.restype = _D
    L.oracle_gauss_residual.argtypes = [_I, _I, _D, _D, _I, _I, _D, _D, _P, _P, _P, _P]
    L.oracle_kinetic_energy.argtypes = [_D, _L, _P, _P, _P, _P, _P]
    L.oracle_kinetic_energy.restype = _D
    for f in ("oracle_sigma_el", "oracle_sigma_ex", "oracle_sigma_iz"):
        getattr(L, f).argtypes = [_D]
        getattr(L, f).restype = _D
    L.oracle_numax_e.argtypes = [_D, _D]
    L.oracle_numax_e.restype = _D
    L.oracle_mcc.argtypes = ([_U, _U, _D, _D, _D, _D, _D, _D, _D, _D]
                             + [_P, _L] + [_P] * 9 + [_P, _L] + [_P] * 9 + [_P, _P])
    L.oracle_mcc.restype = _I
    L.oracle_sort.argtypes = [_I, _L] + [_P] * 8
    L.oracle_sort.restype = _L
    L.oracle_step.argtypes = [C.POINTER(Cfg), _P, _U, C.POINTER(Species), _I, _P, _P, _P, _P,
                              _P, _P, C.POINTER(Stats), _P]
    L.oracle_step.restype = _I
    L.oracle_step_port.argtypes = [C.POINTER(Cfg), _P, _U, C.POINTER(Species), _I] + [_P] * 9 + \
        [C.POINTER(Stats), _P]
    L.oracle_step_port.restype = _I


def _p(x):
    if x is None:
        return None
    assert x.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return x.ctypes.data


# ------------------------------------------------------------------ RNG
def philox4x64(ctr, key):
    """Philox4x64-10 block (Salmon et al., SC'11).  Pinned against numpy."""
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().oracle_philox4x64(_p(c), _p(k), _p(o))
    return o


# ---------------------------------------------------------------- layout
class Grid:
    """r-z mesh, uniform in the logical coordinates (Sec. 2.1).  xa > 0 maps
    the radius: r = 2 dr sqrt(xa xi) for xi <= xa, dr (xi + xa) beyond (the
    mapped mesh with r proportional to sqrt(xi) near the axis), linear in xi
    within each cell; xa = 0 is the uniform mesh r = xi dr."""

    def __init__(self, nr, nz, R, L, xa=0, nd=0, erd=1.0, sgd=0.0):
        """nd > 0: the outer nd cells are a ring of relative permittivity erd
        and conductivity sgd [S/m]; particles move inside it and stick at its
        face.  A large sgd models a metal (electromagnetic model only)."""
        self.nr, self.nz, self.R, self.L = int(nr), int(nz), float(R), float(L)
        self.xa = int(xa)
        self.nd, self.erd, self.sgd = int(nd), float(erd), float(sgd)
        self.dr = self.R / (self.nr + self.xa)
        self.dz = self.L / self.nz

    def r_nodes(self):
        """Node radii r_0..r_nr."""
        i = np.arange(self.nr + 1, dtype=np.float64)
        return np.where(i < self.xa, 2.0 * self.dr * np.sqrt(self.xa * i), (i + self.xa) * self.dr)

    @property
    def n_er(self):
        return self.nr * (self.nz + 1)

    @property
    def n_ez(self):
        return (self.nr + 1) * self.nz

    @property
    def n_h(self):
        return self.nr * self.nz

    @property
    def n_node(self):
        return (self.nr + 1) * (self.nz + 1)

    def zeros_fields(self):
        return (np.zeros(self.n_er), np.zeros(self.n_ez), np.zeros(self.n_h))


FIELDS = ("cell", "a", "b", "vr", "vt", "vz", "w", "id")
DTYPES = {"cell": np.int32, "id": np.uint32}


def empty_species(cap):
    return {k: np.zeros(cap, dtype=DTYPES.get(k, np.float64)) for k in FIELDS}


def load(grid: Grid, n, n0, te_ev, ti_ev, seed, me=ME, mi=M_AR):
    """Pair loading (a1): returns (electrons, ions) dicts of numpy arrays."""
    e = empty_species(n)
    i = empty_species(n)
    lib().oracle_load(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, grid.nd, grid.erd, grid.R,
                      grid.L, n0, n, te_ev, ti_ev,
                      me, mi, seed, _p(e["cell"]), _p(e["a"]), _p(e["b"]), _p(e["vr"]),
                      _p(e["vt"]), _p(e["vz"]), _p(i["vr"]), _p(i["vt"]), _p(i["vz"]),
                      _p(e["w"]), _p(e["id"]))
    for k in ("cell", "a", "b", "w", "id"):
        i[k][:] = e[k]
    return e, i


def push(grid: Grid, dt, q, m, sp, er_half, ez_half, write=False, bz=0.0, ir=None, iz=None,
         walls=None):
    """Push + deposit of one species (rows a2/a3; a6 when write).

    Returns (ir, iz, counters, ke_lost).  ``sp`` arrays are updated in place
    only when ``write``.  ``walls`` = (wall_z0[nr+1], wall_zl[nr+1], wall_r[nz+1]).
    """
    if ir is None:
        ir = np.zeros(grid.n_er)
    if iz is None:
        iz = np.zeros(grid.n_ez)
    cnt = np.zeros(4, dtype=np.int64)
    kel = np.zeros(1)
    wz0, wzl, wr = walls if walls is not None else (None, None, None)
    n = len(sp["cell"])
    lib().oracle_push(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, grid.nd, grid.erd, dt, q, m,
                      bz, n,
                      _p(sp["cell"]),
                      _p(sp["a"]), _p(sp["b"]), _p(sp["vr"]), _p(sp["vt"]), _p(sp["vz"]),
                      _p(sp["w"]), _p(np.ascontiguousarray(er_half, dtype=np.float64)),
                      _p(np.ascontiguousarray(ez_half, dtype=np.float64)), _p(ir), _p(iz),
                      1 if write else 0, _p(wz0), _p(wzl), _p(wr), _p(cnt), _p(kel))
    return ir, iz, cnt, float(kel[0])


def node_charge(grid: Grid, q, sp, Q=None):
    if Q is None:
        Q = np.zeros(grid.n_node)
    lib().oracle_node_charge(grid.nr, grid.nz, q, len(sp["cell"]), _p(sp["cell"]), _p(sp["a"]),
                             _p(sp["b"]), _p(sp["w"]), _p(Q))
    return Q


def kinetic_energy(m, sp):
    return lib().oracle_kinetic_energy(m, len(sp["cell"]), _p(sp["cell"]), _p(sp["vr"]),
                                       _p(sp["vt"]), _p(sp["vz"]), _p(sp["w"]))


def field_energy(grid: Grid, er, ez, h, eps=EPS0, mu=MU0):
    return lib().oracle_field_energy(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, grid.nd,
                                     grid.erd, eps, mu, _p(er),
                                     _p(ez), _p(h))


def gauss_residual(grid: Grid, er, ez, Q, eps=EPS0):
    G = np.zeros(grid.n_node)
    lib().oracle_gauss_residual(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, grid.nd, grid.erd,
                                eps, _p(er), _p(ez),
                                _p(Q), _p(G))
    return G


class FieldSolver:
    """Implicit CN Maxwell solve (row a4) by banded Cholesky of the H system."""

    def __init__(self, grid: Grid, dt, eps=EPS0, mu=MU0, wave=False):
        """wave: the r = R boundary is the matched wave port (incoming wave
        E_in = V/(2L)) instead of the prescribed gap field V/L."""
        self.grid, self.dt, self.eps, self.mu = grid, dt, eps, mu
        self._h = lib().oracle_field_create(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, grid.nd,
                                            grid.erd, grid.sgd, dt, eps, mu, 1 if wave else 0)
        if not self._h:
            raise RuntimeError("oracle field matrix not positive definite")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_field_destroy(self._h)
            self._h = None

    def solve(self, er0, ez0, h0, ir, iz, v0=0.0, v1=0.0):
        g = self.grid
        er1, ez1, h1 = g.zeros_fields()
        src = np.zeros(1)
        lib().oracle_field_solve(self._h, _p(er0), _p(ez0), _p(h0), _p(ir), _p(iz), v0, v1, g.L,
                                 _p(er1), _p(ez1), _p(h1), _p(src))
        return er1, ez1, h1, float(src[0])

    def conduction(self, er0, ez0, er1, ez1, qc):
        """Subtract from the node array qc the charge the ring's conduction
        current carries over the step from (er0, ez0) to (er1, ez1); returns
        the Ohmic energy of the step."""
        return lib().oracle_conduction_charge(self._h, _p(er0), _p(ez0), _p(er1), _p(ez1),
                                              _p(qc))


def port_heights(nzp, port_len, grade=1.0):
    """Row heights of the axial port, q = 0 at its end to nzp - 1 at the
    junction with the reactor: a geometric progression of ratio grade from the
    junction down (grade 1: uniform) that sums to port_len."""
    if grade == 1.0:
        return np.full(nzp, port_len / nzp)
    top = port_len * (grade - 1.0) / (grade ** nzp - 1.0)
    return np.array([top * grade ** (nzp - 1 - q) for q in range(nzp)])


class PortSolver:
    """Implicit CN Maxwell solve with the axial dielectric port below the
    powered electrode (Sec. 2.2, Eqs. 5 and 7), by banded Cholesky of the
    H system of reactor and port together.  ip: the port's inner radius is
    r(ip) (the electrode's); nzp cells of height dzp, or of the row heights
    `heights` (q = 0 at the port's end; see port_heights); erq: its relative
    permittivity."""

    def __init__(self, grid: Grid, dt, ip, nzp, dzp, erq, eps=EPS0, mu=MU0, heights=None):
        self.grid, self.dt, self.eps, self.mu = grid, dt, eps, mu
        self.ip, self.nzp, self.dzp, self.erq = ip, nzp, dzp, erq
        if heights is None:
            self.heights = np.full(nzp, float(dzp))
            self._h = lib().oracle_port_create(grid.nr, grid.nz, grid.dr, grid.dz, grid.xa, ip,
                                               nzp, dzp, erq, dt, eps, mu)
        else:
            self.heights = np.ascontiguousarray(heights, dtype=np.float64)
            assert self.heights.shape == (nzp,)
            self._h = lib().oracle_port_create_graded(grid.nr, grid.nz, grid.dr, grid.dz,
                                                      grid.xa, ip, nzp, _p(self.heights), erq,
                                                      dt, eps, mu)
        if not self._h:
            raise RuntimeError("oracle port matrix not positive definite")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_port_destroy(self._h)
            self._h = None

    def zeros_port(self):
        """(erp, ezp, hp): port E_r edges and H cells (nr - ip) x nzp, E_z edges
        (nr - ip + 1) x nzp."""
        m = self.grid.nr - self.ip
        return (np.zeros(m * self.nzp), np.zeros((m + 1) * self.nzp), np.zeros(m * self.nzp))

    def solve(self, er0, ez0, h0, erp0, ezp0, hp0, ir, iz, phi0, phi1):
        g = self.grid
        er1, ez1, h1 = g.zeros_fields()
        erp1, ezp1, hp1 = self.zeros_port()
        src = np.zeros(1)
        lib().oracle_port_solve(self._h, _p(er0), _p(ez0), _p(h0), _p(erp0), _p(ezp0), _p(hp0),
                                _p(ir), _p(iz), phi0, phi1, _p(er1), _p(ez1), _p(h1), _p(erp1),
                                _p(ezp1), _p(hp1), _p(src))
        return er1, ez1, h1, erp1, ezp1, hp1, float(src[0])

    def energy(self, er, ez, h, erp, ezp, hp):
        return lib().oracle_port_energy(self._h, _p(er), _p(ez), _p(h), _p(erp), _p(ezp), _p(hp))


def sigma_el(eps):
    return lib().oracle_sigma_el(eps)


def sigma_ex(eps):
    return lib().oracle_sigma_ex(eps)


def sigma_iz(eps):
    return lib().oracle_sigma_iz(eps)


def numax_e(ng, me=ME):
    return lib().oracle_numax_e(ng, me)


def mcc(seed, step, ng, tg, numax, pnull_e, pnull_i, gmax, e, ne, ni, i, next_ids,
        me=ME, mi=M_AR):
    """Null-collision MCC (row a7) on capacity-sized species dicts.

    Returns (rc, ne, ni, next_ids, counts[8], dE)."""
    ne_ = C.c_int64(ne)
    ni_ = C.c_int64(ni)
    nid_e = C.c_uint32(next_ids[0])
    nid_i = C.c_uint32(next_ids[1])
    counts = np.zeros(8, dtype=np.int64)
    de = np.zeros(1)
    rc = lib().oracle_mcc(seed, step, ng, tg, me, mi, numax, pnull_e, pnull_i, gmax,
                          C.addressof(ne_), len(e["cell"]), _p(e["cell"]), _p(e["a"]),
                          _p(e["b"]), _p(e["vr"]), _p(e["vt"]), _p(e["vz"]), _p(e["w"]),
                          _p(e["id"]), C.addressof(nid_e),
                          C.addressof(ni_), len(i["cell"]), _p(i["cell"]), _p(i["a"]),
                          _p(i["b"]), _p(i["vr"]), _p(i["vt"]), _p(i["vz"]), _p(i["w"]),
                          _p(i["id"]), C.addressof(nid_i), _p(counts), _p(de))
    return rc, ne_.value, ni_.value, (nid_e.value, nid_i.value), counts, float(de[0])


def sort(grid: Grid, sp, n):
    """Stable counting sort by cell; drops absorbed (cell < 0).  Returns new n."""
    return lib().oracle_sort(grid.nr * grid.nz, n, _p(sp["cell"]), _p(sp["a"]), _p(sp["b"]),
                             _p(sp["vr"]), _p(sp["vt"]), _p(sp["vz"]), _p(sp["w"]),
                             _p(sp["id"]))


class Sim:
    """Whole-step oracle (rows a2-a8) holding its own state in numpy arrays."""

    def __init__(self, grid: Grid, dt, *, freq=0.0, volt=0.0, tol=1e-8, kmax=50, bz=0.0,
                 mcc_on=False, ng=0.0, tg=300.0, seed=0, eps=EPS0, mu=MU0, numax=None,
                 gmax=None, cap=None, species=None, charges=(-QE, QE), masses=(ME, M_AR),
                 cblock=0.0, wave=False, port=None):
        """cblock: blocking capacitor [F] in series with the generator (Eq. 6),
        0 = the electrode follows V(t); its state is self.circ = [q^n, phi^n].
        port: (ip, nzp, port_len, erq[, grade]) for the axial dielectric port (rows
        graded by port_heights; the reactor's
        side wall then a conductor; the electrode at V(t) or, with cblock, Eq. 6's
        circuit); its fields are self.hp, self.erp, self.ezp."""
        self.grid = grid
        self.cfg = Cfg()
        c = self.cfg
        c.nr, c.nz, c.dr, c.dz, c.R, c.L = grid.nr, grid.nz, grid.dr, grid.dz, grid.R, grid.L
        c.dt, c.freq, c.volt, c.eps, c.mu, c.bz = dt, freq, volt, eps, mu, bz
        c.tol, c.kmax, c.mcc_on, c.ng, c.tg, c.seed = tol, kmax, 1 if mcc_on else 0, ng, tg, seed
        c.cblock = cblock
        c.xa = grid.xa
        c.wave = 1 if wave else 0
        c.nd, c.erd = grid.nd, grid.erd
        self.circ = np.zeros(2)
        if mcc_on:
            me, mi = masses
            nu_e = numax_e(ng, me) if numax is None else numax
            vthg = np.sqrt(KB * tg / mi)
            g_max = (np.sqrt(2.0 * QE * 1000.0 / mi) + 5.0 * vthg) if gmax is None else gmax
            nu_i = ng * 5e-19 * g_max
            c.numax_e, c.gmax = nu_e, g_max
            c.pnull_e = -np.expm1(-nu_e * dt)
            c.pnull_i = -np.expm1(-nu_i * dt)
        self.port = None
        if port is not None:
            ip, nzp, lp, erq = port[:4]
            grade = port[4] if len(port) > 4 else 1.0
            self.port = PortSolver(grid, dt, ip, nzp, lp / nzp, erq, eps, mu,
                                   heights=port_heights(nzp, lp, grade) if grade != 1.0 else None)
            self.erp, self.ezp, self.hp = self.port.zeros_port()
        else:
            self.field = FieldSolver(grid, dt, eps, mu, wave)
        self.er, self.ez, self.h = grid.zeros_fields()
        self.wall_z0 = np.zeros(2 * (grid.nr + 1))
        self.wall_zl = np.zeros(2 * (grid.nr + 1))
        self.wall_r = np.zeros(2 * (grid.nz + 1))
        self.qcond = np.zeros(grid.n_node)  # charge moved by the ring's conduction current
        self.ohmic = 0.0                     # Ohmic energy dissipated in the ring
        self.step_index = 0
        self.sp = []
        species = species or []
        for s, arrs in enumerate(species):
            n = len(arrs["cell"])
            capn = cap if cap is not None else max(1, int(n * 1.5) + 16)
            d = empty_species(capn)
            for k in FIELDS:
                d[k][:n] = arrs[k]
            self.sp.append({"arr": d, "n": n, "next_id": int(arrs["id"].max()) + 1 if n else 0,
                            "q": charges[s], "m": masses[s]})

    def _species_table(self):
        T = (Species * max(1, len(self.sp)))()
        for s, d in enumerate(self.sp):
            a = d["arr"]
            T[s] = Species(_p(a["cell"]), _p(a["a"]), _p(a["b"]), _p(a["vr"]), _p(a["vt"]),
                           _p(a["vz"]), _p(a["w"]), _p(a["id"]), d["n"], len(a["cell"]),
                           d["next_id"], d["q"], d["m"])
        return T

    def state(self, s):
        d = self.sp[s]
        return {k: d["arr"][k][: d["n"]].copy() for k in FIELDS}

    def step(self):
        T = self._species_table()
        st = Stats()
        if self.grid.sgd > 0.0:
            er0, ez0 = self.er.copy(), self.ez.copy()
        if self.port is not None:
            rc = lib().oracle_step_port(C.byref(self.cfg), self.port._h, self.step_index, T,
                                        len(self.sp), _p(self.er), _p(self.ez), _p(self.h),
                                        _p(self.hp), _p(self.erp), _p(self.ezp), _p(self.wall_z0),
                                        _p(self.wall_zl), _p(self.wall_r), C.byref(st),
                                        _p(self.circ))
        else:
            rc = lib().oracle_step(C.byref(self.cfg), self.field._h, self.step_index, T,
                                   len(self.sp), _p(self.er), _p(self.ez), _p(self.h),
                                   _p(self.wall_z0), _p(self.wall_zl), _p(self.wall_r),
                                   C.byref(st), _p(self.circ))
        for s, d in enumerate(self.sp):
            d["n"] = T[s].n
            d["next_id"] = T[s].next_id
        if rc in (0, -4, -5):
            self.step_index += 1
            if self.grid.sgd > 0.0:
                self.ohmic += self.field.conduction(er0, ez0, self.er, self.ez, self.qcond)
        return rc, st
