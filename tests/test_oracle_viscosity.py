"""Pins of the oracle's two optional terms of the barotropic system: the viscous regularisation
R_hV = div(H A grad(U/H)) of Eq. (viscosity_BT) and the freshwater flux W of Eq. (4.5).

The paper gives neither a discretisation of R_hV nor the form of A beyond "a background value plus
a part proportional to the velocity differences across cell edges" (Sect. 2.2). The oracle's
reading is a two-point flux between neighbouring triangles:

    flux into e1 across edge (L, d) = H_edge A_edge (u2' - u1) L / d,   u = U / H,
    H_edge = (H1 + H2) / 2,   A_edge = A_bg + C_v |u2' - u1| L,

with u2' the neighbour's velocity in e1's frame and d the centroid distance in the plane unfolded
across the edge; coasts carry no flux. These tests pin it with what geometry and the continuous
operator fix: a Bloch eigenvalue worked out by hand on the right-triangle lattice, convergence to
div(H A grad u) on the equilateral lattice, conservation, dissipation, frame covariance, and the
step-level rules (the term's start-of-step value is subtracted; W drains volume at the rate
sum A_v W and enters Eq. 4.11).
"""
import math

import numpy as np
import pytest

from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I


def _centroids(mesh):
    return np.asarray(mesh.xy).mean(axis=1)


def _rot(v, phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.stack([c * v[..., 0] - s * v[..., 1], s * v[..., 0] + c * v[..., 1]], axis=-1)


def _H_e(mesh, eta=None, nonlinear=False):
    H = np.asarray(mesh.depth)[mesh.tri].mean(axis=1)
    if nonlinear:
        H = H + np.asarray(eta)[mesh.tri].mean(axis=1)
    return H


# ---------------------------------------------------------------- the operator


def pin_right_lattice_bloch(L=None):
    """On the doubly periodic right-triangle lattice (cell h x h cut by the rising diagonal) the
    operator with constant H and C_v = 0 maps a Bloch wave to A/A_e times one of the eigenvalues
    -D +- |c| of [[-D, c], [conj c, -D]], with D = 3 + 6/sqrt5 and
    c = 3 e^{i k.(-h/3, h/3)} + (3/sqrt5) (e^{i k.(-h/3, -2h/3)} + e^{i k.(2h/3, h/3)}):
    across the diagonal L = h sqrt2, d = h sqrt2/3; across each leg L = h, d = h sqrt5/3."""
    n, h, A = 12, 5e3, 700.0
    mesh = I.periodic_square_mesh(n, h, H=2500.0)
    om = orc.OracleMesh(mesh, L)
    cen = _centroids(mesh)
    ae = h * h / 2
    D = 3.0 + 6.0 / math.sqrt(5.0)
    for kx, ky in ((1, 0), (2, 3), (5, 1)):
        kv = 2 * math.pi * np.array([kx, ky]) / (n * h)
        ph = lambda dx, dy: np.exp(1j * (kv[0] * dx + kv[1] * dy))
        c = 3.0 * ph(-h / 3, h / 3) + (3.0 / math.sqrt(5.0)) * (ph(-h / 3, -2 * h / 3) + ph(2 * h / 3, h / 3))
        for sign in (1.0, -1.0):
            lam = -D + sign * abs(c)
            amp = np.where(np.arange(mesh.ne) % 2 == 0, c, sign * abs(c))
            wave = amp * np.exp(1j * (cen @ kv))
            U = np.stack([np.real(wave), 0.4 * np.imag(wave)], axis=1)
            V = om.viscosity(U, np.zeros(mesh.nv), 0, A, 0.0)
            want = (A / ae) * lam * U
            assert np.max(np.abs(V - want)) <= 1e-9 * np.max(np.abs(want)), (kx, ky, sign)


def _equilateral_channel(nx, ny, h, depth_fn):
    P, tri = I.staggered_lattice(nx, ny, h, periodic_x=True)
    xy = I._unwrapped_corners(P, tri, period_x=nx * h)
    pos = np.concatenate([P, np.zeros((P.shape[0], 1))], axis=1)
    return I._contig(I.Mesh("equilateral", tri, xy, pos, depth_fn(P[:, 0], P[:, 1]), np.zeros(tri.shape[0])))


def pin_equilateral_convergence(L=None):
    """On equilateral triangles the line between neighbouring centroids is normal to the shared edge,
    and the two-point flux converges to the continuous div(H A grad u) (smooth H and u, C_v = 0).
    Checked away from the coasts of an x-periodic channel on two resolutions."""
    Lx, Ly, A = 600e3, 520e3, 900.0
    errs = []
    for nx in (24, 48):
        h = Lx / nx
        ny = int(round(Ly / (h * math.sqrt(3.0) / 2.0))) + 1
        kx = 2 * math.pi / Lx
        depth = lambda x, y: 3000.0 + 800.0 * np.sin(kx * x) * np.cos(math.pi * y / Ly)
        mesh = _equilateral_channel(nx, ny, h, depth)
        om = orc.OracleMesh(mesh, L)
        cen = _centroids(mesh)
        x = np.mod(cen[:, 0], Lx)
        y = cen[:, 1]
        ay = math.pi / Ly
        u = np.stack([0.1 * np.sin(kx * x) * np.sin(ay * y), 0.05 * np.cos(2 * kx * x) * np.cos(ay * y)], axis=1)
        He = _H_e(mesh)
        V = om.viscosity(u * He[:, None], np.zeros(mesh.nv), 0, A, 0.0)
        # continuous A (grad H . grad u + H lap u) at the centroids, with H from the corner mean of H0
        Hc = 3000.0 + 800.0 * np.sin(kx * x) * np.cos(ay * y)
        Hx = 800.0 * kx * np.cos(kx * x) * np.cos(ay * y)
        Hy = -800.0 * ay * np.sin(kx * x) * np.sin(ay * y)
        ux_x = 0.1 * kx * np.cos(kx * x) * np.sin(ay * y)
        ux_y = 0.1 * ay * np.sin(kx * x) * np.cos(ay * y)
        ux_l = -0.1 * (kx * kx + ay * ay) * np.sin(kx * x) * np.sin(ay * y)
        uy_x = -0.05 * 2 * kx * np.sin(2 * kx * x) * np.cos(ay * y)
        uy_y = -0.05 * ay * np.cos(2 * kx * x) * np.sin(ay * y)
        uy_l = -0.05 * (4 * kx * kx + ay * ay) * np.cos(2 * kx * x) * np.cos(ay * y)
        want = A * np.stack([Hx * ux_x + Hy * ux_y + Hc * ux_l, Hx * uy_x + Hy * uy_y + Hc * uy_l], axis=1)
        inner = (y > 3 * h) & (y < y.max() - 3 * h)
        errs.append(np.max(np.abs(V[inner] - want[inner])) / np.max(np.abs(want[inner])))
    assert errs[1] < 0.6 * errs[0], errs
    assert errs[1] < 0.05, errs


def pin_uniform_velocity_is_free(L=None):
    """A uniform velocity u (U = H u) feels no viscosity, with varying depth, nonlinear H and the
    flow-dependent coefficient on."""
    case = I.tiny_jittered_case(nx=9, ny=7, seed=21)
    m = case.mesh
    om = orc.OracleMesh(m, L)
    eta = 0.5 * np.random.default_rng(3).standard_normal(m.nv)
    He = _H_e(m, eta, nonlinear=True)
    U = He[:, None] * np.array([0.3, -0.2])[None, :]
    V = om.viscosity(U, eta, 1, 800.0, 2.0)
    scale = 800.0 * 0.3 * np.max(He) / np.min(om.areas()[1])
    assert np.max(np.abs(V)) <= 1e-12 * scale


def pin_conserves_momentum_on_the_plane(L=None):
    """Every edge flux enters one neighbour and leaves the other: sum_e A_e R_hV_e = 0 on a plane."""
    case = I.tiny_jittered_case(nx=9, ny=7, seed=22)
    om = orc.OracleMesh(case.mesh, L)
    _, ae = om.areas()
    rng = np.random.default_rng(4)
    V = om.viscosity(case.U0, 0.4 * rng.standard_normal(case.mesh.nv), 1, 500.0, 3.0)
    tot = (ae[:, None] * V).sum(axis=0)
    assert np.max(np.abs(tot)) <= 1e-11 * np.sum(ae[:, None] * np.abs(V))


def pin_dissipates(L=None):
    """sum_e A_e u_e . R_hV_e = -sum_edges H A (L/d) |u2' - u1|^2 <= 0: the term removes kinetic
    energy, on the plane and on the sphere (where u2' is rotated between element frames)."""
    for case in (I.tiny_jittered_case(nx=9, ny=7, seed=23), I.sphere_case(level=2, nsteps=1)):
        m = case.mesh
        om = orc.OracleMesh(m, L)
        _, ae = om.areas()
        rng = np.random.default_rng(5)
        U = rng.standard_normal((m.ne, 2)) * _H_e(m)[:, None]
        for Abg, Cv in ((1000.0, 0.0), (0.0, 5.0), (300.0, 2.0)):
            V = om.viscosity(U, np.zeros(m.nv), 0, Abg, Cv)
            u = U / _H_e(m)[:, None]
            work = float(np.sum(ae[:, None] * u * V))
            assert work < 0.0, (case.name, Abg, Cv, work)


def pin_flow_dependent_part(L=None):
    """C_v alone: the flux is C_v |du| L^2/d H du, so the operator is homogeneous of degree 2 in U;
    on the right-triangle lattice with u = (a, 0) on one triangle family and (b, 0) on the other,
    R_hV = (H C_v |b - a| (b - a) / A_e) sum L^2/d = H C_v |b - a| (b - a) (3 sqrt2 + 6/sqrt5) h / A_e
    on the first family (and the opposite on the second)."""
    n, h, H, Cv = 8, 4e3, 3000.0, 1.7
    mesh = I.periodic_square_mesh(n, h, H=H)
    om = orc.OracleMesh(mesh, L)
    a, b = 0.2, -0.15
    first = np.arange(mesh.ne) % 2 == 0
    U = np.zeros((mesh.ne, 2))
    U[:, 0] = np.where(first, a, b) * H
    V = om.viscosity(U, np.zeros(mesh.nv), 0, 0.0, Cv)
    mag = H * Cv * abs(b - a) * (b - a) * (3.0 * math.sqrt(2.0) + 6.0 / math.sqrt(5.0)) * h / (h * h / 2)
    want = np.where(first, mag, -mag)
    assert np.max(np.abs(V[:, 0] - want)) <= 1e-10 * abs(mag)
    assert np.max(np.abs(V[:, 1])) <= 1e-10 * abs(mag)
    case = I.sphere_case(level=2, nsteps=1)
    om = orc.OracleMesh(case.mesh, L)
    U = np.random.default_rng(6).standard_normal((case.mesh.ne, 2)) * 100.0
    V1 = om.viscosity(U, np.zeros(case.mesh.nv), 0, 0.0, Cv)
    V2 = om.viscosity(2.0 * U, np.zeros(case.mesh.nv), 0, 0.0, Cv)
    assert np.max(np.abs(V2 - 4.0 * V1)) <= 1e-12 * np.max(np.abs(V2))


def pin_frame_covariance(L=None):
    """Turning one element's frame (its corner coordinates and its U) by phi turns its R_hV by phi
    and leaves every other element's R_hV unchanged: the neighbour rotation is taken from the frames."""
    for case in (I.tiny_jittered_case(nx=9, ny=7, seed=24), I.sphere_case(level=2, nsteps=1)):
        m = case.mesh
        rng = np.random.default_rng(7)
        U = rng.standard_normal((m.ne, 2)) * 50.0
        eta = 0.3 * rng.standard_normal(m.nv)
        V = orc.OracleMesh(m, L).viscosity(U, eta, 1, 600.0, 4.0)
        for j, phi in ((0, 0.7), (m.ne // 2, -2.1), (m.ne - 1, 3.0)):
            xy = np.array(m.xy, copy=True)
            xy[j] = _rot(xy[j], phi) + np.array([1234.0, -567.0])
            m2 = I._contig(I.Mesh(m.name, m.tri, xy, m.pos, m.depth, m.coriolis))
            U2 = U.copy()
            U2[j] = _rot(U[j], phi)
            V2 = orc.OracleMesh(m2, L).viscosity(U2, eta, 1, 600.0, 4.0)
            want = V.copy()
            want[j] = _rot(V[j], phi)
            assert np.max(np.abs(V2 - want)) <= 1e-9 * np.max(np.abs(V)), (case.name, j)


# ---------------------------------------------------------------- the step


def pin_zero_coefficients_and_M1_are_the_plain_step(L=None):
    """With A_bg = C_v = 0 and W = 0 the step is Eq. (4.10); with M = 1 the subtracted start-of-step
    value cancels the term exactly, so the step is again the plain one."""
    case = I.tiny_jittered_case(nx=8, ny=6, seed=25, M=5, tau=50.0)
    om = orc.OracleMesh(case.mesh, L)
    ref = om.advance(case.R, case.params, 3, case.eta0, case.U0)[:3]
    got = om.advance_ext(case.R, case.params, 3, case.eta0, case.U0, W=np.zeros(case.mesh.nv), visc=(0.0, 0.0))
    for a, b in zip(ref, got):
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(a)))
    p1 = I.Params(g=case.params.g, theta=case.params.theta, tau=10.0, M=1, nonlinear_h=1)
    ref = om.advance(case.R, p1, 4, case.eta0, case.U0)[:3]
    got = om.advance_ext(case.R, p1, 4, case.eta0, case.U0, visc=(5000.0, 10.0))
    for a, b in zip(ref, got):
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(a)))


def pin_start_value_is_subtracted(L=None):
    """Without gravity, Coriolis and forcing the momentum equation of a substep reduces to
    U^{m+1} = U^m + dt (R_hV(U^m) - R_hV(U^0)): starting from U^1 = U^0 the transport never moves,
    and eta^{n} = eta^0 - n tau div(U^0) (linear H)."""
    case = I.tiny_jittered_case(nx=8, ny=6, seed=26, M=6, tau=60.0, nonlinear_h=0)
    m = case.mesh
    p = I.Params(g=0.0, theta=0.14, tau=60.0, M=6, nonlinear_h=0)
    mesh0 = I._contig(I.Mesh(m.name, m.tri, m.xy, m.pos, m.depth, np.zeros(m.ne)))
    om = orc.OracleMesh(mesh0, L)
    eta, U, Um = om.advance_ext(np.zeros((m.ne, 2)), p, 3, case.eta0, case.U0, visc=(2000.0, 5.0))
    assert np.max(np.abs(U - case.U0)) <= 1e-13 * np.max(np.abs(case.U0))
    assert np.max(np.abs(Um - case.U0)) <= 1e-13 * np.max(np.abs(case.U0))
    want = case.eta0 - 3 * p.tau * om.divergence(case.U0)
    assert np.max(np.abs(eta - want)) <= 1e-12 * np.max(np.abs(want))


def pin_uniform_freshwater_closed_form(L=None):
    """From rest and a flat surface, a uniform W only lowers the surface: eta = -n tau W everywhere
    and U stays zero (the gradient of a uniform eta vanishes), with Coriolis and nonlinear H on."""
    case = I.tiny_jittered_case(nx=8, ny=6, seed=27, M=7, tau=70.0)
    m = case.mesh
    om = orc.OracleMesh(m, L)
    W = np.full(m.nv, 2.5e-5)
    eta, U, Um = om.advance_ext(np.zeros((m.ne, 2)), case.params, 4, np.zeros(m.nv), np.zeros((m.ne, 2)), W=W)
    assert np.max(np.abs(eta + 4 * 70.0 * 2.5e-5)) <= 1e-15
    # (the contour-sum gradient of a uniform field is zero up to the rounding of the edge normals)
    assert np.max(np.abs(U)) <= 1e-12 and np.max(np.abs(Um)) <= 1e-12


def pin_freshwater_volume_and_eq_4_11(L=None):
    """On a closed basin the divergence integrates to zero, so each step changes the volume by
    -tau sum A_v W exactly; and eta^{n+1} - eta^n = -tau (div <<U>> + W) (Eq. 4.11 with W), with the
    viscous term on as well."""
    case = I.tiny_jittered_case(nx=9, ny=7, seed=28, M=8, tau=80.0)
    m = case.mesh
    om = orc.OracleMesh(m, L)
    av, _ = om.areas()
    W = 1e-5 * np.random.default_rng(8).standard_normal(m.nv)
    eta, U = case.eta0, case.U0
    for _ in range(3):
        e1, U1, Um = om.advance_ext(case.R, case.params, 1, eta, U, W=W, visc=(400.0, 1.5))
        dv = float(np.sum(av * (e1 - eta)))
        assert abs(dv + case.params.tau * float(np.sum(av * W))) <= 1e-12 * float(np.sum(av * np.abs(eta)))
        r = (e1 - eta) + case.params.tau * (om.divergence(Um) + W)
        assert np.max(np.abs(r)) <= 1e-12 * max(1.0, np.max(np.abs(eta)))
        eta, U = e1, U1


def pin_sesm_freshwater(L=None):
    """The SESM continuity update carries W as Eq. (4.8) prints it: a uniform W from rest lowers a
    flat surface by exactly tau W per step, and with a random state and W the volume falls by
    tau sum A_v W per step while eta^{n+1} - eta^n = -tau (div <<U>> + W)."""
    from oracle import closed
    coef = closed.sesm_params(0.07)
    case = I.tiny_jittered_case(nx=8, ny=6, seed=29, M=7, tau=70.0)
    m = case.mesh
    om = orc.OracleMesh(m, L)
    eta, U, Um = om.advance_sesm(np.zeros((m.ne, 2)), case.params, coef, 3, np.zeros(m.nv), np.zeros((m.ne, 2)),
                                 W=np.full(m.nv, 4e-5))
    assert np.max(np.abs(eta + 3 * 70.0 * 4e-5)) <= 1e-15
    assert np.max(np.abs(U)) <= 1e-12
    av, _ = om.areas()
    W = 1e-5 * np.random.default_rng(9).standard_normal(m.nv)
    e0 = case.eta0
    e1, U1, Um = om.advance_sesm(case.R, case.params, coef, 1, e0, case.U0, W=W)
    assert abs(float(np.sum(av * (e1 - e0))) + 70.0 * float(np.sum(av * W))) <= 1e-12 * float(np.sum(av * np.abs(e0)))
    r = (e1 - e0) + 70.0 * (om.divergence(Um) + W)
    assert np.max(np.abs(r)) <= 1e-12 * max(1.0, np.max(np.abs(e0)))
    ref = om.advance_sesm(case.R, case.params, coef, 2, e0, case.U0)
    got = om.advance_sesm(case.R, case.params, coef, 2, e0, case.U0, W=np.zeros(m.nv))
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


PINS = [pin_right_lattice_bloch, pin_equilateral_convergence, pin_uniform_velocity_is_free,
        pin_conserves_momentum_on_the_plane, pin_dissipates, pin_flow_dependent_part, pin_frame_covariance,
        pin_zero_coefficients_and_M1_are_the_plain_step, pin_start_value_is_subtracted,
        pin_uniform_freshwater_closed_form, pin_freshwater_volume_and_eq_4_11, pin_sesm_freshwater]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ---------------------------------------------------------------- the pins catch planted mistakes

PLANTS = {
    "rotation_sign": ("const double rot = geo[0][0] - geo[1][0];", "const double rot = geo[1][0] - geo[0][0];"),
    "normal_distance_only": ("sqrt((geo[0][1] - geo[1][1]) * (geo[0][1] - geo[1][1]) +",
                             "sqrt(0.0 * (geo[0][1] - geo[1][1]) +"),
    "edge_depth_one_side": ("const real k = (H1 + H2) / 2 * A * (real)(L / d);", "const real k = H1 * A * (real)(L / d);"),
    "length_not_over_distance": ("const real k = (H1 + H2) / 2 * A * (real)(L / d);",
                                 "const real k = (H1 + H2) / 2 * A * (real)(L);"),
    "flow_part_without_length": ("const real A = Abg + Cv * (real)sqrt((double)(dx * dx + dy * dy)) * (real)L;",
                                 "const real A = Abg + Cv * (real)sqrt((double)(dx * dx + dy * dy));"),
    "e2_not_rotated_back": ("out[2 * e2] += (-(cr * fx + sr * fy)) / m->area_e[e2];",
                            "out[2 * e2] += (-fx) / m->area_e[e2];"),
    "velocity_not_transport": ("const real u1x = U[2 * e1] / H1, u1y = U[2 * e1 + 1] / H1;",
                               "const real u1x = U[2 * e1], u1y = U[2 * e1 + 1];"),
    "start_value_not_subtracted": ("rx += Vm[2 * e] - V0[2 * e]; ry += Vm[2 * e + 1] - V0[2 * e + 1];",
                                   "rx += Vm[2 * e]; ry += Vm[2 * e + 1];"),
    "freshwater_sign": ("for (int v = 0; v < nv; v++) eta[v] -= dt * (div[v] + W[v]);",
                        "for (int v = 0; v < nv; v++) eta[v] -= dt * (div[v] - W[v]);"),
    "sesm_freshwater_sign": ("for (int v = 0; v < nv; v++) enew[v] = E[0][v] - dt * (div[v] + W[v]);",
                             "for (int v = 0; v < nv; v++) enew[v] = E[0][v] - dt * (div[v] - W[v]);"),
    "viscosity_at_start_depth": ("if (xy) viscosity(m, U, eta, nonlinear_h, (real)Abg, (real)Cv, xy, Vm);",
                                 "if (xy) viscosity(m, U, eta, 0, (real)Abg, (real)Cv, xy, Vm);"),
}


def _pins_failing(L):
    failed = []
    for pin in PINS:
        try:
            pin(L)
        except (AssertionError, RuntimeError, FloatingPointError):
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_pins_catch_planted_mistake(plant):
    old, new = PLANTS[plant]
    src = orc.source_text()
    assert old in src, plant
    L = orc.build_variant(src.replace(old, new), "visc_" + plant)
    failed = _pins_failing(L)
    print(plant, "caught by", failed)
    assert failed, f"planted mistake {plant} went unnoticed"
