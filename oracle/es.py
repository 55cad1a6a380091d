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
of the lumped gap source, E_z = phi0 / L there).  The linear system is solved
directly with scipy's sparse LU.
"""
from __future__ import annotations

import numpy as np

EPS0 = 8.8541878128e-12


def _areas(nr, nz, dr, dz):
    ar = 2.0 * np.pi * (np.arange(nr) + 0.5) * dr * dz           # faces (i+1/2), i < nr
    az = 2.0 * np.pi * np.arange(nr + 1) * dr * dr                # node rings
    az[0] = np.pi * (0.5 * dr) ** 2
    return ar, az


def boundary_phi(nr, nz, phi0):
    """Node potentials with the Dirichlet values set (interior zero)."""
    phi = np.zeros((nr + 1, nz + 1))
    phi[:, 0] = phi0
    phi[nr, :] = phi0 * (1.0 - np.arange(nz + 1) / nz)
    return phi


def fields(phi, dr, dz):
    """Yee-layout E_r (nr x (nz+1)) and E_z ((nr+1) x nz) of node potentials."""
    er = -(phi[1:, :] - phi[:-1, :]) / dr
    ez = -(phi[:, 1:] - phi[:, :-1]) / dz
    return er.ravel(), ez.ravel()


def solve(nr, nz, dr, dz, Q, phi0, eps=EPS0):
    """Potential and fields for node charges Q ((nr+1) x (nz+1), only interior
    nodes used) and powered-plate potential phi0."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ar, az = _areas(nr, nz, dr, dz)
    Q = np.asarray(Q, dtype=np.float64).reshape(nr + 1, nz + 1)
    phi = boundary_phi(nr, nz, phi0)
    M = nz - 1
    idx = lambda i, j: i * M + (j - 1)
    rows, cols, vals = [], [], []
    rhs = np.zeros(nr * M)
    for i in range(nr):
        for j in range(1, nz):
            k = idx(i, j)
            # eps * sum of outward fluxes of -grad phi = Q  ->  coefficients of phi
            terms = [(i + 1, j, eps * ar[i] / dr)]
            if i >= 1:
                terms.append((i - 1, j, eps * ar[i - 1] / dr))
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
    er, ez = fields(phi, dr, dz)
    return phi, er, ez
