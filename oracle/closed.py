"""Closed forms from Sect. 3 of the paper, for the pins of the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``se_matrix(c, theta)``  the characteristic matrix of the SE scheme, Eq. (3.7),
  in the Fourier variables of the 1-D prototype Eq. (3.1): (eta, u) -> next substep.
* ``se_poly(c, theta)``    coefficients of P_SE(lambda), Eq. (dp_1), highest power first.
* ``lattice_recurrence``   the same scheme applied to one eigenmode of the discrete
  operator -D(gH G) with eigenvalue kappa^2: a real 2x2 recurrence for the mode
  amplitudes (u, e) of U = u G(phi), eta = e phi.
* ``kappa2_square``        eigenvalue of the 5-point Laplacian for Fourier mode (kx, ky)
  on an n x n periodic grid of spacing dx; on a right-triangle mesh with consistent
  diagonals the lumped-area P1 operator -D G equals this stencil (cot 90 deg = 0).
"""
from __future__ import annotations

import math

import numpy as np


def se_matrix(c, theta):
    return np.array([[1.0 - c * c * (1.0 + theta), -1j * c], [-1j * c, 1.0]], dtype=complex)


def se_poly(c, theta):
    return np.array([1.0, c * c * theta + c * c - 2.0, 1.0 - c * c * theta])


def kappa2_square(n, dx, kx, ky):
    return 4.0 / dx ** 2 * (math.sin(math.pi * kx / n) ** 2 + math.sin(math.pi * ky / n) ** 2)


def lattice_recurrence(kappa2, gH, dt, theta):
    """Matrix A with (u, e)_{m+1} = A (u, e)_m for one substep on an eigenmode."""
    # u' = u - dt gH e ;  e' = e + dt kappa2 ((1+theta) u' - theta u)
    #                        = e + dt kappa2 u - dt^2 kappa2 gH (1+theta) e
    return np.array([[1.0, -dt * gH],
                     [dt * kappa2, 1.0 - dt * dt * kappa2 * gH * (1.0 + theta)]])


def mode_amplitude(kappa2, gH, dt, theta, nsub, e0=1.0, u0=0.0):
    A = lattice_recurrence(kappa2, gH, dt, theta)
    return np.linalg.matrix_power(A, nsub) @ np.array([u0, e0])


def stability_limit(theta):
    """Largest substep Courant number c = sqrt(gH kappa2) dt with |lambda| <= 1 for P_SE."""
    return 2.0 / math.sqrt(1.0 + 2.0 * theta)


def inertial_rotation(f, dt):
    """Angle (clockwise for f > 0) by which a Crank-Nicolson Coriolis substep turns U."""
    return 2.0 * math.atan(0.5 * f * dt)


# ---------------------------------------------------------------- SESM (AB3-AM4, Eqs. 4.7-4.8)

def sesm_params(chi, beta=0.281105):
    """(beta, delta, gamma, zeta) for dissipation chi, Eq. (dp_6) second row with Eq. (dp_4):
    zeta = 0.010 - 0.135 chi, gamma = 0.083 - 0.514 chi, 2 chi = delta - gamma - 2 zeta - 1/2."""
    zeta = 0.010 - 0.135 * chi
    gamma = 0.083 - 0.514 * chi
    delta = 2.0 * chi + gamma + 2.0 * zeta + 0.5
    return beta, delta, gamma, zeta


def sesm_matrix(c, beta, delta, gamma, zeta):
    """Characteristic matrix of Eq. (3.5): (eta^{n+1}, eta^n, eta^{n-1}, u^{n+1}, u^n, u^{n-1}) from the
    state one level earlier."""
    i = 1j
    return np.array([
        [1, 0, 0, -i * c * (1.5 + beta), i * c * (0.5 + 2 * beta), -i * c * beta],
        [1, 0, 0, 0, 0, 0],
        [0, 1, 0, 0, 0, 0],
        [-i * c * (1 - gamma - zeta), -i * c * gamma, -i * c * zeta,
         1 - c * c * delta * (1.5 + beta), c * c * delta * (0.5 + 2 * beta), -c * c * delta * beta],
        [0, 0, 0, 1, 0, 0],
        [0, 0, 0, 0, 1, 0]], dtype=complex)


def sesm_poly(c, beta, delta, gamma, zeta):
    """P_SESM(lambda) of Eq. (dp_1), coefficients from lambda^6 down to lambda^0."""
    c2 = c * c
    b, d, g, z = beta, delta, gamma, zeta
    return np.array([
        1.0,
        -2.0 + c2 * d / 2.0 * (2 * b + 3),
        1.0 + c2 / 2.0 * (b * (-6 * d - 2 * g - 2 * z + 2) - 4 * d - 3 * g - 3 * z + 3),
        c2 / 2.0 * (b * (6 * d + 6 * g + 4 * z - 4) + d + 4 * g + z - 1),
        -c2 * ((d + 3 * g - 1) * b + g / 2.0 - 3 * z / 2.0),
        c2 * (b * (g - 2 * z) - z / 2.0),
        b * z * c2])


def sesm_small_c(beta, delta, gamma, zeta):
    """(chi, n, q) of Eqs. (dp_4)-(dp_5), SESM rows."""
    b, d, g, z = beta, delta, gamma, zeta
    chi = (d - g - 2 * z - 0.5) / 2.0
    n = -0.5 * (0.5 + d - g - 2 * z)
    q = -1j / 8.0 * (0.25 * (z * (16 * g - 16 * d + 24) + g * (-8 * d + 4) - 7) + 4 * z * z + g * g + d * d
                     + 3 * d + 4 * b)
    return chi, n, q


def sesm_lattice_matrix(kappa2, gH, dt, beta, delta, gamma, zeta):
    """One SESM substep on an eigenmode: state (e^m, e^{m-1}, e^{m-2}, u^m, u^{m-1}, u^{m-2}) with
    eta = e phi, U = u G(phi), -D G phi = kappa2 phi:
        u_AB = a0 u^m + a1 u^{m-1} + a2 u^{m-2};   e^{m+1} = e^m + dt kappa2 u_AB
        e_AM = delta e^{m+1} + (1-delta-gamma-zeta) e^m + gamma e^{m-1} + zeta e^{m-2}
        u^{m+1} = u^m - dt gH e_AM."""
    a0, a1, a2 = 1.5 + beta, -(0.5 + 2 * beta), beta
    k = dt * kappa2
    w = dt * gH
    A = np.zeros((6, 6))
    A[0] = [1, 0, 0, k * a0, k * a1, k * a2]
    A[1] = [1, 0, 0, 0, 0, 0]
    A[2] = [0, 1, 0, 0, 0, 0]
    A[3] = [-w * (1 - gamma - zeta), -w * gamma, -w * zeta, 1 - w * delta * k * a0, -w * delta * k * a1,
            -w * delta * k * a2]
    A[4] = [0, 0, 0, 1, 0, 0]
    A[5] = [0, 0, 0, 0, 1, 0]
    return A


def sesm_mode_amplitude(kappa2, gH, dt, coef, M, nsteps, e0=1.0, u0=0.0):
    """Mode amplitudes after nsteps baroclinic steps of M SESM substeps, each step starting with the
    history levels equal to level 0."""
    A = sesm_lattice_matrix(kappa2, gH, dt, *coef)
    P = np.linalg.matrix_power(A, M)
    e, u = e0, u0
    for _ in range(nsteps):
        x = P @ np.array([e, e, e, u, u, u])
        e, u = x[0], x[3]
    return u, e
