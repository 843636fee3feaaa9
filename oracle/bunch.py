"""Self-consistent initial fields of an externally injected relativistic electron bunch
(Sec. 3: the field initialisation of Vay 2008 / Massimo 2019 carried over to cylindrical
symmetry), in FP64 with numpy and a sparse direct solve.

TEST INFRASTRUCTURE ONLY: used by the test-suite; it shares nothing with the CUDA library.

A bunch moving along x at beta = v/c, gamma = 1/sqrt(1 - beta^2), carries the fields of a
charge in uniform motion: E = -(d phi/dx / gamma^2, d phi/dr), B_theta = beta E_r, where
    (1/gamma^2) d^2 phi/dx^2 + (1/r) d/dr (r d phi/dr) = -rho.
Discretely this is the Gauss law of the Yee grid in flux form, node by node,
    A_j (Ex(i+1/2, j) - Ex(i-1/2, j)) + 2 pi dx (r_{j+1/2} Er(i, j+1/2) - r_{j-1/2} Er(i, j-1/2))
        = Q_ij,
with Q_ij = sum q w S_x S_r the charge deposited on node (i, j) (linear weights), A_j = V_j/dx
the ring area of the charge volumes (V_0 = pi (dr/2)^2 dx on the axis, where r_{-1/2} = 0),
Ex(i+1/2) = -(phi_{i+1} - phi_i)/(gamma^2 dx), Er(j+1/2) = -(phi_{j+1} - phi_j)/dr, no x flux
through the window's ends (Ex(-1/2) = Ex(Nx+1/2) = 0) and phi = 0 on the wall r = r_max.
B_theta(i+1/2, j+1/2) at t = -dt/2 is beta E_r of the field moved back by beta dt/2: E_r
interpolated linearly in x at x_{i+1/2} + beta dt/2.  Er on the two x ends is set to zero
afterwards (the perfect conductor of the Maxwell solver).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def node_charge(x, y, z, w, nx, nr, dx, dr, q=-1.0):
    """Q_ij = sum q w S_x S_r on the primal nodes (window-relative x)."""
    Q = np.zeros((nx + 1, nr + 1))
    xn, rn = x / dx, np.sqrt(y * y + z * z) / dr
    i0, j0 = np.floor(xn).astype(int), np.floor(rn).astype(int)
    fx, fr = xn - i0, rn - j0
    for di, wx in ((0, 1 - fx), (1, fx)):
        for dj, wr in ((0, 1 - fr), (1, fr)):
            np.add.at(Q, (i0 + di, j0 + dj), q * w * wx * wr)
    return Q


def ring_area(nr, dx, dr):
    a = 2 * np.pi * np.arange(nr + 1) * dr * dr
    a[0] = np.pi * dr * dr / 4
    return a


def solve_potential(Q, nx, nr, dx, dr, gamma):
    """phi on the nodes (i, j), j < Nr (phi = 0 at j = Nr), from the flux-form Gauss law."""
    n = (nx + 1) * nr
    idx = lambda i, j: i * nr + j  # noqa: E731
    area = ring_area(nr, dx, dr)
    cx = area / (gamma * gamma * dx)                  # x coupling of row j
    rh = (np.arange(nr) + 0.5) * dr
    cr = 2 * np.pi * dx * rh / dr                     # r coupling through face j + 1/2
    rows, cols, vals = [], [], []
    for i in range(nx + 1):
        for j in range(nr):
            k = idx(i, j)
            diag = 0.0
            for ii in (i - 1, i + 1):
                if 0 <= ii <= nx:
                    rows.append(k); cols.append(idx(ii, j)); vals.append(-cx[j])
                    diag += cx[j]
            # face j + 1/2 (to j + 1, which is the wall phi = 0 when j + 1 = Nr)
            diag += cr[j]
            if j + 1 < nr:
                rows.append(k); cols.append(idx(i, j + 1)); vals.append(-cr[j])
            if j > 0:
                diag += cr[j - 1]
                rows.append(k); cols.append(idx(i, j - 1)); vals.append(-cr[j - 1])
            rows.append(k); cols.append(k); vals.append(diag)
    K = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    phi = spla.spsolve(K.tocsc(), Q[:, :nr].reshape(-1))
    out = np.zeros((nx + 1, nr + 1))
    out[:, :nr] = phi.reshape(nx + 1, nr)
    return out


def bunch_fields(x, y, z, w, nx, nr, dx, dr, dt, gamma, q=-1.0):
    """(Ex, Er, Bt) of the bunch: Ex, Er at t = 0, Bt at t = -dt/2, in the oracle's layouts."""
    Q = node_charge(x, y, z, w, nx, nr, dx, dr, q)
    phi = solve_potential(Q, nx, nr, dx, dr, gamma)
    beta = np.sqrt(1.0 - 1.0 / (gamma * gamma))
    ex = -(phi[1:, :] - phi[:-1, :]) / (gamma * gamma * dx)          # (nx, nr+1)
    er = -(phi[:, 1:] - phi[:, :-1]) / dr                              # (nx+1, nr)
    f = 0.5 + beta * dt / (2 * dx)
    bt = beta * ((1 - f) * er[:-1, :] + f * er[1:, :])                # (nx, nr)
    er[0, :] = 0.0
    er[nx, :] = 0.0
    return ex, er, bt
