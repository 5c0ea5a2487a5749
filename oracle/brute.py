"""Dense-matrix brute force of the SE substep on tiny meshes (numpy, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is an independent construction of the same discrete operators the C oracle
uses, built the finite-element way instead of edge by edge:

* gradient G (2E x V): the constant gradients of the linear (P1) basis functions,
  grad(phi_a) = rot90(p_c - p_b) / (2 A_e) for a counter-clockwise triangle (a, b, c);
* divergence D (V x 2E): the negative adjoint of G in the area-weighted inner products
  (lumped vertex areas A_v = sum of A_e/3), D = -diag(1/A_v) G^T diag(A_e);
* one substep of Eq. (4.10) as a single block linear system in the unknowns
  (U^{m+1}, eta^{m+1}), solved with numpy.linalg.solve:
      (I + a J) U^{m+1}                          = (I - a J) U^m - dt g H G eta^m + dt R
      dt (1+theta) D U^{m+1} + eta^{m+1}         = eta^m + dt theta D U^m
  with J the rotation e_z x, a = f dt / 2 per element and H per element.
"""
from __future__ import annotations

import numpy as np


def p1_operators(mesh):
    """Return (G, D, A_e, A_v) as dense arrays."""
    xy = np.asarray(mesh.xy, dtype=np.float64)
    tri = np.asarray(mesh.tri)
    E, V = tri.shape[0], mesh.nv
    p0, p1, p2 = xy[:, 0], xy[:, 1], xy[:, 2]
    A = 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))
    G = np.zeros((2 * E, V))
    for k in range(3):
        pb = xy[:, (k + 1) % 3]
        pc = xy[:, (k + 2) % 3]
        d = pc - pb
        gx = -d[:, 1] / (2.0 * A)
        gy = d[:, 0] / (2.0 * A)
        for e in range(E):
            G[2 * e, tri[e, k]] += gx[e]
            G[2 * e + 1, tri[e, k]] += gy[e]
    Av = np.zeros(V)
    for k in range(3):
        np.add.at(Av, tri[:, k], A / 3.0)
    Ae2 = np.repeat(A, 2)
    D = -(G.T * Ae2[None, :]) / Av[:, None]
    return G, D, A, Av


def substep_system(mesh, params, H_e):
    """Block matrices (Lhs, Rhs_U, Rhs_eta) of one substep for a given element depth."""
    G, D, A, Av = p1_operators(mesh)
    E, V = mesh.ne, mesh.nv
    dt = params.tau / params.M
    a = 0.5 * dt * np.asarray(mesh.coriolis)
    J = np.array([[0.0, -1.0], [1.0, 0.0]])
    Ip = np.zeros((2 * E, 2 * E))
    Im = np.zeros((2 * E, 2 * E))
    for e in range(E):
        Ip[2 * e:2 * e + 2, 2 * e:2 * e + 2] = np.eye(2) + a[e] * J
        Im[2 * e:2 * e + 2, 2 * e:2 * e + 2] = np.eye(2) - a[e] * J
    Hrep = np.repeat(H_e, 2)
    n = 2 * E + V
    Lhs = np.zeros((n, n))
    Lhs[:2 * E, :2 * E] = Ip
    Lhs[2 * E:, :2 * E] = dt * (1.0 + params.theta) * D
    Lhs[2 * E:, 2 * E:] = np.eye(V)
    Rhs = np.zeros((n, n))
    Rhs[:2 * E, :2 * E] = Im
    Rhs[:2 * E, 2 * E:] = -dt * params.g * Hrep[:, None] * G
    Rhs[2 * E:, :2 * E] = dt * params.theta * D
    Rhs[2 * E:, 2 * E:] = np.eye(V)
    return Lhs, Rhs, dt, G, D, A, Av


def advance(mesh, R, params, nsteps, eta, U):
    """Brute-force run; returns (eta, U, Umean) after nsteps baroclinic steps."""
    E, V = mesh.ne, mesh.nv
    H0e = np.asarray(mesh.depth)[np.asarray(mesh.tri)].mean(axis=1)
    eta = np.array(eta, dtype=np.float64)
    U = np.array(U, dtype=np.float64).reshape(E, 2)
    Rv = np.asarray(R, dtype=np.float64).reshape(-1)
    Umean = np.zeros((E, 2))
    lin = None
    for _ in range(nsteps):
        U0 = U.copy()
        S = np.zeros((E, 2))
        for _m in range(params.M):
            if params.nonlinear_h:
                H = H0e + eta[np.asarray(mesh.tri)].mean(axis=1)
                Lhs, Rhs, dt, *_ = substep_system(mesh, params, H)
            else:
                if lin is None:
                    lin = substep_system(mesh, params, H0e)
                Lhs, Rhs, dt, *_ = lin
            x = np.concatenate([U.reshape(-1), eta])
            b = Rhs @ x
            b[:2 * E] += dt * Rv
            y = np.linalg.solve(Lhs, b)
            U = y[:2 * E].reshape(E, 2)
            eta = y[2 * E:]
            S += U
        Umean = S / params.M + params.theta / params.M * (U - U0)
    return eta, U, Umean


def advance_sesm(mesh, R, params, coef, nsteps, eta, U):
    """SESM steps (Eqs. 4.7-4.8) with the dense finite-element operators; levels before the start of a
    subcycle equal level 0. Returns (eta, U, Umean)."""
    beta, delta, gamma, zeta = coef
    G, D, A, Av = p1_operators(mesh)
    E, V = mesh.ne, mesh.nv
    tri = np.asarray(mesh.tri)
    H0e = np.asarray(mesh.depth)[tri].mean(axis=1)
    f = np.asarray(mesh.coriolis)
    dt = params.tau / params.M
    eta = np.array(eta, dtype=np.float64)
    U = np.array(U, dtype=np.float64).reshape(E, 2)
    Rv = np.asarray(R, dtype=np.float64).reshape(E, 2)
    Umean = np.zeros((E, 2))
    for _ in range(nsteps):
        Uh = [U.copy(), U.copy(), U.copy()]            # U^m, U^{m-1}, U^{m-2}
        Eh = [eta.copy(), eta.copy(), eta.copy()]      # eta^m, eta^{m-1}, eta^{m-2}
        S = np.zeros((E, 2))
        for _m in range(params.M):
            UAB = (1.5 + beta) * Uh[0] - (0.5 + 2 * beta) * Uh[1] + beta * Uh[2]
            S += UAB
            enew = Eh[0] - dt * (D @ UAB.reshape(-1))
            eAM = delta * enew + (1 - delta - gamma - zeta) * Eh[0] + gamma * Eh[1] + zeta * Eh[2]
            H = H0e + (eAM[tri].mean(axis=1) if params.nonlinear_h else 0.0)
            grad = (G @ eAM).reshape(E, 2)
            cor = np.stack([f * UAB[:, 1], -f * UAB[:, 0]], axis=1)
            Unew = Uh[0] + dt * (cor - params.g * H[:, None] * grad + Rv)
            Uh = [Unew, Uh[0], Uh[1]]
            Eh = [enew, Eh[0], Eh[1]]
        U, eta = Uh[0], Eh[0]
        Umean = S / params.M
    return eta, U, Umean
