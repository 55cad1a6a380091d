"""FP64 CPU oracle of the electrostatic field model (Eq. 8 of Sec. 2.2),
test infrastructure only.

On the uniform r-z mesh, with the same integral form as the electromagnetic
scheme: the potential lives on the nodes (i, j), E_r = -(phi_{i+1,j} -
phi_{i,j}) / dr on the radial edges and E_z = -(phi_{i,j+1} - phi_{i,j}) / dz
on the axial edges, and Gauss's law is imposed on every interior node
(i < nr, 0 < j < nz) in the flux form

    eps [A_r(i) E_r(i+1/2, j) - A_r(i-1) E_r(i-1/2, j)
         + A_z(i) (E_z(i, j+1/2) - E_z(i, j-1/2))] = Q_ij,

A_r(i) = 2 pi r_{i+1/2} dz, A_z(i) = 2 pi r_i dr (pi (dr/2)^2 on the axis).
Boundary values: phi = phi0 on the powered plate z = 0, 0 on the grounded
plate z = L, and phi0 (1 - z/L) across the drive gap at r = R (the potential
of the lumped gap source, E_z = phi0 / L there).  With the axial port (port =
ip, Sec. 2.2's electrostatic model): the powered electrode is the disc r <=
r_p = r(ip) of z = 0, the port's opening r_p < r < R carries the potential of
the coaxial line's TEM field, phi0 ln(r / R) / ln(r_p / R), and the side wall
r = R is grounded.  The linear system is solved directly with scipy's sparse
LU.
"""
from __future__ import annotations

import numpy as np

EPS0 = 8.8541878128e-12


def radii(nr, dr, xa=0):
    """Node radii r_i, cell centres r_{i+1/2} and cell widths of the mesh:
    uniform (xa = 0), or mapped with r = 2 dr sqrt(xa xi) for xi <= xa and
    dr (xi + xa) beyond, linear within each cell (Sec. 2.1)."""
    i = np.arange(nr + 1, dtype=np.float64)
    rn = np.where(i < xa, 2.0 * dr * np.sqrt(xa * i), (i + xa) * dr)
    rc = 0.5 * (rn[:-1] + rn[1:])
    return rn, rc, np.diff(rn)


def _areas(nr, nz, dr, dz, xa=0, nd=0, erd=1.0):
    """Dual-face areas weighted by the relative permittivity of the cells they
    cross (the outer nd cells form a dielectric ring of permittivity erd)."""
    rn, rc, _ = radii(nr, dr, xa)
    f = np.where(np.arange(nr) >= nr - nd, erd, 1.0)              # per cell
    ar = 2.0 * np.pi * rc * dz * f                                # faces (i+1/2), i < nr
    az = np.empty(nr + 1)
    az[0] = np.pi * rc[0] ** 2 * f[0]                             # axis disc
    inner = np.pi * (rn[1:nr] ** 2 - rc[:-1] ** 2) * f[:-1]       # half ring in cell i-1
    outer = np.pi * (rc[1:] ** 2 - rn[1:nr] ** 2) * f[1:]         # half ring in cell i
    az[1:nr] = inner + outer
    az[nr] = np.pi * (rn[nr] ** 2 - rc[nr - 1] ** 2) * f[nr - 1]
    return ar, az


def boundary_phi(nr, nz, phi0, port=None, rn=None):
    """Node potentials with the Dirichlet values set (interior zero); port:
    the node index ip of the electrode's rim (rn: the node radii)."""
    phi = np.zeros((nr + 1, nz + 1))
    if port is None:
        phi[:, 0] = phi0
        phi[nr, :] = phi0 * (1.0 - np.arange(nz + 1) / nz)
    else:
        ip = int(port)
        phi[: ip + 1, 0] = phi0
        phi[ip + 1:, 0] = phi0 * np.log(rn[ip + 1:] / rn[nr]) / np.log(rn[ip] / rn[nr])
    return phi


def fields(phi, dr, dz, xa=0):
    """Yee-layout E_r (nr x (nz+1)) and E_z ((nr+1) x nz) of node potentials."""
    _, _, w = radii(phi.shape[0] - 1, dr, xa)
    er = -(phi[1:, :] - phi[:-1, :]) / w[:, None]
    ez = -(phi[:, 1:] - phi[:, :-1]) / dz
    return er.ravel(), ez.ravel()


def solve(nr, nz, dr, dz, Q, phi0, eps=EPS0, xa=0, nd=0, erd=1.0, port=None):
    """Potential and fields for node charges Q ((nr+1) x (nz+1), only interior
    nodes used) and powered-plate potential phi0 (port: see boundary_phi)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ar, az = _areas(nr, nz, dr, dz, xa, nd, erd)
    wr = radii(nr, dr, xa)[2]
    Q = np.asarray(Q, dtype=np.float64).reshape(nr + 1, nz + 1)
    phi = boundary_phi(nr, nz, phi0, port, radii(nr, dr, xa)[0])
    M = nz - 1
    idx = lambda i, j: i * M + (j - 1)
    rows, cols, vals = [], [], []
    rhs = np.zeros(nr * M)
    for i in range(nr):
        for j in range(1, nz):
            k = idx(i, j)
            # eps * sum of outward fluxes of -grad phi = Q  ->  coefficients of phi
            terms = [(i + 1, j, eps * ar[i] / wr[i])]
            if i >= 1:
                terms.append((i - 1, j, eps * ar[i - 1] / wr[i - 1]))
            terms.append((i, j + 1, eps * az[i] / dz))
            terms.append((i, j - 1, eps * az[i] / dz))
            diag = 0.0
            for (ii, jj, c) in terms:
                diag += c
                if ii < nr and 1 <= jj <= nz - 1:
                    rows.append(k)
                    cols.append(idx(ii, jj))
                    vals.append(-c)
                else:
                    rhs[k] += c * phi[ii, jj]
            rows.append(k)
            cols.append(k)
            vals.append(diag)
            rhs[k] += Q[i, j]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(nr * M, nr * M))
    x = spla.spsolve(A.tocsc(), rhs)
    phi[:nr, 1:nz] = x.reshape(nr, M)
    er, ez = fields(phi, dr, dz, xa)
    return phi, er, ez


def electrode_charge_flow(nr, nz, dr, dz, ez_new, ez_old, iz, eps=EPS0, xa=0, nd=0, erd=1.0,
                          port=None):
    """dt times the reactor-side current of Eq. 6: the displacement current
    plus the crossed charge through the dual faces of the first row of E_z
    edges above the powered plate (i < nr, j = 1/2; with the port i < ip, the
    electrode disc), i.e. the integral over the electrode in Eq. 6 on the
    integral-form mesh."""
    _, az = _areas(nr, nz, dr, dz, xa, nd, erd)
    s = 0.0
    for i in range(nr if port is None else int(port)):
        s += eps * az[i] * (ez_new[i * nz] - (ez_old[i * nz] if ez_old is not None else 0.0))
        if iz is not None:
            s += iz[i * nz]
    return s


def circuit_potential(nr, nz, dr, dz, Q, ez_old, iz, v1, qn, cblock, eps=EPS0, xa=0, nd=0,
                      erd=1.0, port=None):
    """Electrode potential phi^{n+1} of Eq. 6 with a blocking capacitor cblock
    between the generator V^{n+1} = v1 and the electrode: the reactor-side
    charge flow must equal C (V^{n+1} - phi^{n+1}) - q^n.  The field is affine
    in phi^{n+1}; a solve at v1 and the unit-potential solve fix it."""
    _, _, eza = solve(nr, nz, dr, dz, Q, v1, eps, xa, nd, erd, port)
    _, _, ezu = solve(nr, nz, dr, dz, np.zeros((nr + 1) * (nz + 1)), 1.0, eps, xa, nd, erd, port)
    dq = electrode_charge_flow(nr, nz, dr, dz, eza, ez_old, iz, eps, xa, nd, erd, port)
    gu = electrode_charge_flow(nr, nz, dr, dz, ezu, None, None, eps, xa, nd, erd, port)
    return v1 - (qn + dq) / (cblock + gu)


def divergence_out(nr, nz, ir, iz):
    """Charge leaving each interior node (i < nr, 0 < j < nz) through the dual
    faces of its edges during the step, (nr+1) x (nz+1) (zero elsewhere)."""
    ir = np.asarray(ir).reshape(nr, nz + 1)
    iz = np.asarray(iz).reshape(nr + 1, nz)
    out = np.zeros((nr + 1, nz + 1))
    for i in range(nr):
        for j in range(1, nz):
            o = ir[i, j] + iz[i, j] - iz[i, j - 1]
            if i >= 1:
                o -= ir[i - 1, j]
            out[i, j] = o
    return out.ravel()


class Sim:
    """Whole-step oracle of the electrostatic model without collisions: the
    Picard iteration of the push + deposit (Eqs. 3-4, the oracle's mover)
    and the Eq. 8 solve for the node charge Q^{n+1,k} = Q^n - div I^k
    (continuity, Q^n from the particles), the commit push with the half field
    of the last iteration, and the sort.  With cblock > 0 the electrode
    potential of every iteration solves Eq. 6 (state self.circ = [q^n, phi^n]);
    otherwise it is V(t) = volt sin(2 pi freq t)."""

    def __init__(self, grid, dt, *, freq=0.0, volt=0.0, tol=1e-8, kmax=50, eps=EPS0,
                 cblock=0.0, species=(), charges=None, masses=None, cap=None, drive=None,
                 fixed=(), port=None):
        """drive: optional V(t) replacing volt sin(2 pi freq t); fixed: indices of
        species that stay in place (not pushed, deposited or sorted); port: the
        node index ip of the axial port's inner radius (see boundary_phi)."""
        import oracle as O
        if getattr(grid, "sgd", 0.0) > 0.0:
            # Sec. 2.1: electrostatic runs model metals by a large permittivity
            raise ValueError("a conducting ring needs the electromagnetic model")
        self.O = O
        self.drive, self.fixed, self.port = drive, tuple(fixed), port
        self.g, self.dt, self.freq, self.volt = grid, dt, freq, volt
        self.tol, self.kmax, self.eps, self.cblock = tol, kmax, eps, cblock
        charges = charges or (-O.QE, O.QE)
        masses = masses or (O.ME, O.M_AR)
        self.er, self.ez, _ = grid.zeros_fields()
        self.circ = np.zeros(2)
        self.step_index = 0
        self.wall = [np.zeros(2 * (grid.nr + 1)), np.zeros(2 * (grid.nr + 1)),
                     np.zeros(2 * (grid.nz + 1))]
        self.sp = []
        for s, arrs in enumerate(species):
            n = len(arrs["cell"])
            capn = cap if cap is not None else max(1, int(n * 1.5) + 16)
            d = O.empty_species(capn)
            for k in O.FIELDS:
                d[k][:n] = arrs[k]
            self.sp.append({"arr": d, "n": n, "q": charges[s], "m": masses[s]})

    def _view(self, d):
        return {k: d["arr"][k][: d["n"]] for k in self.O.FIELDS}

    def state(self, s):
        return {k: v.copy() for k, v in self._view(self.sp[s]).items()}

    def volt_at(self, step):
        if self.drive is not None:
            return self.drive(step * self.dt)
        return self.volt * np.sin(2.0 * np.pi * self.freq * step * self.dt)

    def step(self):
        """Returns (rc, stats dict); rc = -3 when the iteration does not converge."""
        O, g = self.O, self.g
        nr, nz = g.nr, g.nz
        v1 = self.volt_at(self.step_index + 1)
        Qn = np.zeros(g.n_node)
        for d in self.sp:
            O.node_charge(g, d["q"], self._view(d), Qn)
        if g.nd > 0:
            # the charge stuck on the dielectric ring's face stays in Gauss's law
            wr = self.wall[2]
            Qn.reshape(nr + 1, nz + 1)[nr - g.nd, :] += wr[: nz + 1] + wr[nz + 1:]
        er1, ez1 = self.er.copy(), self.ez.copy()
        if not self.cblock > 0.0 and self.port is None:
            ez1[nr * nz:] = v1 / g.L
        phi1 = v1
        conv, res, k = False, 0.0, 0
        for k in range(self.kmax):
            erh, ezh = 0.5 * (self.er + er1), 0.5 * (self.ez + ez1)
            ir, iz = np.zeros(g.n_er), np.zeros(g.n_ez)
            for s, d in enumerate(self.sp):
                if s not in self.fixed:
                    O.push(g, self.dt, d["q"], d["m"], self._view(d), erh, ezh, ir=ir, iz=iz)
            Q1 = Qn - divergence_out(nr, nz, ir, iz)
            if self.cblock > 0.0:
                phi1 = circuit_potential(nr, nz, g.dr, g.dz, Q1, self.ez, iz, v1, self.circ[0],
                                         self.cblock, self.eps, g.xa, g.nd, g.erd, self.port)
            _, ern, ezn = solve(nr, nz, g.dr, g.dz, Q1, phi1, self.eps, g.xa, g.nd, g.erd,
                                self.port)
            mr = np.ones((nr, nz + 1), bool)
            mr[:, 0] = mr[:, nz] = False
            dr_ = (ern - er1)[mr.ravel()]
            dz_ = (ezn - ez1)[: nr * nz]
            num = np.sqrt(np.sum(dr_ * dr_) + np.sum(dz_ * dz_))
            den = np.sqrt(np.sum(ern[mr.ravel()] ** 2) + np.sum(ezn[: nr * nz] ** 2))
            res = num / max(den, 1e-30)
            er1, ez1 = ern, ezn
            if res < self.tol:
                conv = True
                break
        st = {"picard_iters": k + 1 if conv else k, "last_res": res, "converged": conv,
              "absorbed": 0, "ke_lost": 0.0, "phi": phi1, "ir": ir, "iz": iz}
        if not conv:
            return -3, st
        for s, d in enumerate(self.sp):
            if s in self.fixed:
                continue
            walls = tuple(w[s * (len(w) // 2):(s + 1) * (len(w) // 2)] for w in self.wall)
            _, _, cnt, kel = O.push(g, self.dt, d["q"], d["m"], self._view(d), erh, ezh,
                                    write=True, walls=walls)
            st["absorbed"] += int(cnt[1])
            st["ke_lost"] += kel
        for s, d in enumerate(self.sp):
            if s not in self.fixed:
                d["n"] = O.sort(g, d["arr"], d["n"])
        self.er, self.ez = er1, ez1
        if self.cblock > 0.0:
            self.circ[:] = (self.cblock * (v1 - phi1), phi1)
        self.step_index += 1
        return 0, st
