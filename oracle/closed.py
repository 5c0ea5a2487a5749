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
