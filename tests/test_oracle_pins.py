"""Pins of the FP64 oracle to what the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself: the paper's printed
characteristic matrix and polynomial (Sect. 3), exact invariants of Eqs. (4.10)-(4.12),
closed-form solutions of special cases and a dense brute force built the
finite-element way.
"""
import math

import numpy as np
import pytest

from oracle import brute, closed
from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I


# ---------------------------------------------------------------- Sect. 3 closed forms

def _same_roots(a, b, atol):
    a = list(a)
    for r in b:
        i = int(np.argmin([abs(r - x) for x in a]))
        if abs(r - a[i]) > atol:
            return False
        a.pop(i)
    return True


def _physical_root(c, theta):
    lam = np.linalg.eigvals(closed.se_matrix(c, theta))
    return lam[np.argmin(np.abs(lam - np.exp(1j * c)))]


def test_se_matrix_roots_are_roots_of_printed_polynomial(golden_se):
    th = golden_se["theta"]
    for c in (0.01, 0.3, 1.0, 1.5):
        ev = np.linalg.eigvals(closed.se_matrix(c, th))
        rt = np.roots(closed.se_poly(c, th))
        assert _same_roots(ev, rt, 1e-12)


def test_small_courant_expansion_matches_printed_coefficients(golden_se):
    """Eqs. (dp_2)-(dp_5): lambda = 1 + i c + n c^2 + q c^3 + O(c^4), |lambda| = 1 - chi c^2 + O(c^4)."""
    th = golden_se["theta"]
    assert golden_se["chi_fig1"] == pytest.approx(th / 2.0)          # 2 chi = theta
    n, q = golden_se["n_se"], 1j * golden_se["q_se_imag"]
    res = []
    for c in (2e-2, 1e-2, 5e-3):
        lam = _physical_root(c, th)
        res.append(abs(lam - (1 + 1j * c + n * c * c + q * c ** 3)))
        assert abs(abs(lam) - (1 - golden_se["chi_fig1"] * c * c)) < 2 * c ** 4
    # the remainder is O(c^4) (for this scheme even O(c^5)): halving c divides it by >= ~16,
    # while a wrong n or q would leave an O(c^2) or O(c^3) remainder (ratio 4 or 8)
    assert res[0] / res[1] > 14 and res[1] / res[2] > 14


def test_lattice_recurrence_has_the_printed_spectrum(golden_se):
    """The per-mode recurrence of the mesh scheme has the eigenvalues of Eq. (3.7) with c^2 = gH kappa^2 dt^2."""
    th = golden_se["theta"]
    for kappa2, gH, dt in ((1e-9, 4e4, 20.0), (3e-8, 3e4, 12.0), (8e-8, 5e4, 5.0)):
        c = math.sqrt(gH * kappa2) * dt
        a = np.linalg.eigvals(closed.lattice_recurrence(kappa2, gH, dt, th))
        b = np.linalg.eigvals(closed.se_matrix(c, th))
        assert _same_roots(a, b, 1e-12)


def test_phase_speed_tends_to_sqrt_gH():
    """Long waves: arg(lambda) / (k dt) -> sqrt(gH) and damping per substep -> 1 as k dx -> 0."""
    gH = 9.81 * 4000.0
    th = 0.14
    errs = []
    for n in (32, 64, 128, 256):
        dx = 1e6 / n
        dt = 0.4 * dx / math.sqrt(gH)
        k2 = closed.kappa2_square(n, dx, 1, 0)
        lam = np.linalg.eigvals(closed.lattice_recurrence(k2, gH, dt, th))
        lam = lam[np.argmax(lam.imag)]
        k = 2 * math.pi / 1e6
        errs.append(abs(np.angle(lam) / (k * dt) - math.sqrt(gH)) / math.sqrt(gH))
    assert errs[-1] < 1e-3
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(len(errs) - 1))  # second order


# ---------------------------------------------------------------- oracle vs closed forms

@pytest.mark.parametrize("kx,ky,theta", [(1, 0, 0.14), (3, 2, 0.14), (5, 7, 0.0), (2, 1, 0.5)])
def test_oracle_periodic_wave_matches_closed_form(kx, ky, theta):
    """P1: a cosine mode on the periodic right-triangle mesh evolves by the 2x2 recurrence exactly."""
    case = I.periodic_wave_case(n=16, kx=kx, ky=ky, theta=theta, nsteps=3)
    p = case.params
    eta, U, Umean, _ = orc.run_case(case)
    dt = p.tau / p.M
    gH = p.g * 4000.0
    k2 = closed.kappa2_square(16, 10e3, kx, ky)
    u_e = closed.mode_amplitude(k2, gH, dt, p.theta, case.nsteps * p.M)
    assert np.max(np.abs(eta - u_e[1] * case.eta0)) < 1e-11
    assert abs(u_e[1]) < 1.0          # dissipative for theta > 0, neutral for theta = 0
    if theta == 0.0:
        assert abs(abs(u_e[1]) - 1.0) < 1.0 and np.max(np.abs(eta)) > 0.1


def test_oracle_stability_boundary():
    """P8: c = 2/sqrt(1+2 theta) separates bounded from growing runs (checkerboard mode)."""
    n, dx, H, th = 8, 10e3, 4000.0, 0.14
    gH = 9.81 * H
    kappa_max = math.sqrt(closed.kappa2_square(n, dx, n // 2, n // 2))
    out = {}
    for frac in (0.97, 1.03):
        dt = frac * closed.stability_limit(th) / (kappa_max * math.sqrt(gH))
        case = I.periodic_wave_case(n=n, kx=n // 2, ky=n // 2, theta=th, M=40, tau=40 * dt, nsteps=5)
        eta, *_ = orc.run_case(case)
        out[frac] = np.max(np.abs(eta))
    assert out[0.97] <= 1.0
    assert out[1.03] > 10.0


def test_oracle_inertial_oscillation():
    """P4: uniform U on a periodic mesh turns clockwise by 2 atan(f dt/2) per substep, eta stays 0."""
    mesh = I.periodic_square_mesh(8, 10e3, f=1e-4)
    p = I.Params(tau=600.0, M=30, nonlinear_h=1)
    U0 = np.tile([1.3, -0.4], (mesh.ne, 1))
    eta, U, Umean, _ = orc.OracleMesh(mesh).advance(np.zeros((mesh.ne, 2)), p, 4, np.zeros(mesh.nv), U0)
    dt = p.tau / p.M
    phi = closed.inertial_rotation(1e-4, dt)

    def rot(m):
        c, s = math.cos(m * phi), math.sin(m * phi)
        return np.array([c * 1.3 + s * -0.4, -s * 1.3 + c * -0.4])

    assert np.max(np.abs(eta)) < 1e-12
    assert np.max(np.abs(U - rot(4 * p.M))) < 1e-12
    # time mean of the last step from the analytic sequence (Eq. 4.12)
    m0 = 3 * p.M
    want = sum(rot(m0 + m) for m in range(1, p.M + 1)) / p.M + p.theta / p.M * (rot(4 * p.M) - rot(m0))
    assert np.max(np.abs(Umean - want)) < 1e-12


def test_oracle_uniform_forcing_closed_form():
    """P5: uniform R, f != 0: U^m = U* + Rot^m (U^0 - U*), with f e_z x U* = R."""
    f = 1.2e-4
    mesh = I.periodic_square_mesh(6, 10e3, f=f)
    p = I.Params(tau=480.0, M=40, nonlinear_h=0)
    R = np.tile([2e-4, -1e-4], (mesh.ne, 1))
    eta, U, Umean, _ = orc.OracleMesh(mesh).advance(R, p, 3, np.zeros(mesh.nv), np.zeros((mesh.ne, 2)))
    Ustar = np.array([R[0, 1] / f, -R[0, 0] / f])
    phi = closed.inertial_rotation(f, p.tau / p.M)
    m = 3 * p.M
    d = -Ustar
    c, s = math.cos(m * phi), math.sin(m * phi)
    want = Ustar + np.array([c * d[0] + s * d[1], -s * d[0] + c * d[1]])
    assert np.max(np.abs(U - want)) < 1e-10
    assert np.max(np.abs(eta)) < 1e-12


# ---------------------------------------------------------------- invariants

def test_oracle_volume_conservation_basin():
    """P3: sum A_v eta_v is constant on the closed basin (20 steps, nonlinear H)."""
    case = I.basin_case()
    om = orc.OracleMesh(case.mesh)
    av, ae = om.areas()
    v0 = float(np.sum(av * case.eta0))
    eta, U, Umean, diag = om.advance(case.R, case.params, case.nsteps, case.eta0, case.U0, want_diag=True)
    scale = float(np.sum(av * np.abs(case.eta0)))
    assert np.max(np.abs(diag[:, 0] - v0)) <= 1e-12 * scale
    assert np.max(np.abs(eta - case.eta0)) > 1e-2       # the bump did move


@pytest.mark.parametrize("nonlinear_h", [0, 1])
def test_oracle_summation_identity(nonlinear_h):
    """P2, Eqs. (4.11)-(4.12): eta^M - eta^0 = -tau D <<U>> at every vertex, to roundoff."""
    case = I.tiny_jittered_case(nx=9, ny=7, seed=3, nonlinear_h=nonlinear_h, M=7, tau=70.0)
    om = orc.OracleMesh(case.mesh)
    eta1, U1, Um, _ = om.advance(case.R, case.params, 1, case.eta0, case.U0)
    lhs = eta1 - case.eta0
    rhs = -case.params.tau * om.divergence(Um)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1.0, np.max(np.abs(lhs)))
    # a second step starts from the carried U^M
    eta2, U2, Um2, _ = om.advance(case.R, case.params, 1, eta1, U1)
    assert np.max(np.abs((eta2 - eta1) + case.params.tau * om.divergence(Um2))) < 1e-12


def test_oracle_point_symmetry_basin():
    """P7: the basin mesh and the centred bump are symmetric under a 180-degree turn."""
    case = I.basin_case(nsteps=5)
    eta, U, Umean, _ = orc.run_case(case)
    nx, ny = 101, 51
    e2 = eta.reshape(ny, nx)
    assert np.max(np.abs(e2 - e2[::-1, ::-1])) < 1e-12 * np.max(np.abs(eta))


def test_oracle_geometry_invariants():
    """Median-dual cells tile the mesh; Green-Gauss is exact for linear fields; closed cells leak nothing."""
    case = I.tiny_jittered_case(nx=10, ny=8, seed=5)
    om = orc.OracleMesh(case.mesh)
    av, ae = om.areas()
    assert abs(av.sum() - ae.sum()) < 1e-9 * ae.sum()
    P = case.mesh.pos[:, :2]
    g = om.gradient(3e-6 * P[:, 0] - 7e-6 * P[:, 1] + 0.25)
    assert np.max(np.abs(g - np.array([3e-6, -7e-6]))) < 1e-18
    rng = np.random.default_rng(0)
    F = rng.standard_normal((case.mesh.ne, 2))
    assert abs(np.sum(av * om.divergence(F))) < 1e-9 * np.sum(av * np.abs(om.divergence(F)))
    # a uniform field has zero divergence on a periodic mesh (every cell is closed)
    pm = I.periodic_square_mesh(5, 1e3)
    pom = orc.OracleMesh(pm)
    assert np.max(np.abs(pom.divergence(np.tile([0.7, -0.2], (pm.ne, 1))))) < 1e-15
    pav, _ = pom.areas()
    assert np.allclose(pav, 1e3 ** 2, rtol=1e-13)


def test_oracle_rejects_bad_meshes():
    case = I.tiny_jittered_case()
    m = case.mesh
    bad = I.Mesh(m.name, m.tri.copy(), m.xy.copy(), m.pos, m.depth, m.coriolis)
    bad.tri[0, 0] = m.nv
    with pytest.raises(ValueError, match="-1"):
        orc.OracleMesh(bad)
    bad = I.Mesh(m.name, m.tri.copy(), m.xy.copy(), m.pos, m.depth, m.coriolis)
    bad.xy[0, [1, 2]] = bad.xy[0, [2, 1]]
    with pytest.raises(ValueError, match="-2"):
        orc.OracleMesh(bad)
    # an edge shared by three triangles
    tri = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    xy = np.array([[[0, 0], [1, 0], [0, 1]], [[1, 0], [0, 0], [0, -1]], [[0, 0], [1, 0], [1, 1]]], float)
    nm = I.Mesh("t", tri, xy, np.zeros((5, 3)), np.ones(5), np.zeros(3))
    with pytest.raises(ValueError, match="-3"):
        orc.OracleMesh(nm)


# ---------------------------------------------------------------- brute force

def _brute_meshes():
    yield "jittered-nonlinear", I.tiny_jittered_case(nx=6, ny=5, seed=11, nonlinear_h=1)
    yield "jittered-linear", I.tiny_jittered_case(nx=7, ny=5, seed=12, nonlinear_h=0)
    X, F = I.icosphere(1)
    xy, lat = I.sphere_element_frames(X * 6.371e6, F)
    rng = np.random.default_rng(4)
    sm = I.Mesh("sphere1", F, xy, X, 3000.0 + 1000.0 * rng.random(X.shape[0]), 2 * 7.292e-5 * np.sin(lat))
    p = I.Params(tau=3000.0, M=6, nonlinear_h=1)
    yield "sphere-level1", I.Case("s", sm, p, 1e-2 * rng.standard_normal((F.shape[0], 2)),
                                  0.2 * rng.standard_normal(X.shape[0]),
                                  20.0 * rng.standard_normal((F.shape[0], 2)), 2)


@pytest.mark.parametrize("name,case", list(_brute_meshes()), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_matches_brute_force(name, case):
    """P6: the edge-form oracle equals the finite-element dense construction on tiny meshes."""
    om = orc.OracleMesh(case.mesh)
    e1, U1, M1, _ = om.advance(case.R, case.params, case.nsteps, case.eta0, case.U0)
    e2, U2, M2 = brute.advance(case.mesh, case.R, case.params, case.nsteps, case.eta0, case.U0)
    se = max(1.0, np.max(np.abs(e2)))
    su = max(1.0, np.max(np.abs(U2)))
    assert np.max(np.abs(e1 - e2)) < 1e-11 * se
    assert np.max(np.abs(U1 - U2)) < 1e-11 * su
    assert np.max(np.abs(M1 - M2)) < 1e-11 * su


def test_oracle_operators_match_finite_element_adjoint():
    """The edge-form divergence is minus the area-weighted adjoint of the P1 gradient."""
    case = I.tiny_jittered_case(nx=8, ny=6, seed=21)
    om = orc.OracleMesh(case.mesh)
    G, D, Ae, Av = brute.p1_operators(case.mesh)
    rng = np.random.default_rng(1)
    eta = rng.standard_normal(case.mesh.nv)
    F = rng.standard_normal((case.mesh.ne, 2))
    assert np.allclose(om.gradient(eta).reshape(-1), G @ eta, rtol=1e-12, atol=1e-18)
    assert np.allclose(om.divergence(F), D @ F.reshape(-1), rtol=1e-11, atol=1e-16)
    av, ae = om.areas()
    assert np.allclose(av, Av, rtol=1e-13) and np.allclose(ae, Ae, rtol=1e-13)


# ---------------------------------------------------------------- the pins catch planted mistakes

PLANTS = {
    # dropped theta weighting in the continuity flux
    "drop_theta": ("F[2 * e] = (1 + theta) * nx - theta * ux;", "F[2 * e] = nx;"),
    # wrong sign of the pressure gradient (the sign printed in the Eq. 4.10 bracket)
    "pressure_sign": ("real bx = ux + a * uy + dt * (-g * H * gx + R[2 * e]);",
                      "real bx = ux + a * uy + dt * (g * H * gx + R[2 * e]);"),
    # Coriolis turned the wrong way
    "coriolis_sign": ("real A11 = 1, A12 = -a, A21 = a, A22 = 1;",
                      "real A11 = 1, A12 = a, A21 = -a, A22 = 1;"),
    # mean without the theta correction of Eq. (4.12)
    "mean_no_theta": ("+ theta / (real)M * (U[2 * e + c] - U0[2 * e + c]))", ")"),
    # divergence counted into the wrong cell
    "flux_side": ("s += (m->edge_v[2 * q] == v) ? edgeflux[q] : -edgeflux[q];",
                  "s += (m->edge_v[2 * q] == v) ? -edgeflux[q] : edgeflux[q];"),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_pins_catch_planted_mistake(plant):
    old, new = PLANTS[plant]
    src = orc.source_text()
    assert old in src
    L = orc.build_variant(src.replace(old, new), plant)
    case = I.tiny_jittered_case(nx=6, ny=5, seed=11, nonlinear_h=1)
    om = orc.OracleMesh(case.mesh, L)
    e1, U1, M1, _ = om.advance(case.R, case.params, case.nsteps, case.eta0, case.U0)
    e2, U2, M2 = brute.advance(case.mesh, case.R, case.params, case.nsteps, case.eta0, case.U0)
    err = max(np.max(np.abs(e1 - e2)), np.max(np.abs(U1 - U2)) / max(1.0, np.max(np.abs(U2))),
              np.max(np.abs(M1 - M2)) / max(1.0, np.max(np.abs(M2))))
    assert err > 1e-6, f"planted mistake {plant} went unnoticed"


# ---------------------------------------------------------------- SESM (Eqs. 4.7-4.8, Sect. 3)

def _sesm_coef(golden_se):
    chi = golden_se["chi_fig1"]
    b = golden_se["beta_sesm"]
    z = golden_se["zeta_c0"] + golden_se["zeta_c1"] * chi
    g = golden_se["gamma_c0"] + golden_se["gamma_c1"] * chi
    d = 2 * chi + g + 2 * z + 0.5
    return b, d, g, z


def test_sesm_parameters_follow_printed_rules(golden_se):
    b, d, g, z = _sesm_coef(golden_se)
    assert (b, d, g, z) == pytest.approx(closed.sesm_params(golden_se["chi_fig1"]))
    chi, n, q = closed.sesm_small_c(b, d, g, z)
    assert chi == pytest.approx(golden_se["chi_fig1"])


def test_sesm_matrix_roots_are_roots_of_printed_polynomial(golden_se):
    coef = _sesm_coef(golden_se)
    for c in (0.05, 0.3, 0.9, 1.3):
        ev = np.linalg.eigvals(closed.sesm_matrix(c, *coef))
        rt = np.roots(closed.sesm_poly(c, *coef))
        assert _same_roots(ev, rt, 1e-9)


def test_sesm_small_courant_expansion(golden_se):
    """The physical root of Eq. (3.5) follows lambda = 1 + i c + n c^2 + q c^3 + O(c^4) with the printed
    SESM n and q (Eq. dp_5), and |lambda| = 1 - chi c^2 + O(c^4) (Eq. dp_3)."""
    coef = _sesm_coef(golden_se)
    chi, n, q = closed.sesm_small_c(*coef)
    res = []
    for c in (2e-2, 1e-2, 5e-3):
        lam = np.linalg.eigvals(closed.sesm_matrix(c, *coef))
        lam = lam[np.argmin(np.abs(lam - np.exp(1j * c)))]
        res.append(abs(lam - (1 + 1j * c + n * c * c + q * c ** 3)))
        assert abs(abs(lam) - (1 - chi * c * c)) < 5 * c ** 4
    assert res[0] / res[1] > 12 and res[1] / res[2] > 12


def test_sesm_lattice_recurrence_has_the_printed_spectrum(golden_se):
    coef = _sesm_coef(golden_se)
    for kappa2, gH, dt in ((1e-9, 4e4, 20.0), (3e-8, 3e4, 12.0), (6e-8, 5e4, 5.0)):
        c = math.sqrt(gH * kappa2) * dt
        a = np.linalg.eigvals(closed.sesm_lattice_matrix(kappa2, gH, dt, *coef))
        b = np.linalg.eigvals(closed.sesm_matrix(c, *coef))
        assert _same_roots(a, b, 1e-9)


@pytest.mark.parametrize("kx,ky", [(1, 0), (3, 2), (5, 7)])
def test_oracle_sesm_periodic_wave_matches_closed_form(golden_se, kx, ky):
    coef = _sesm_coef(golden_se)
    case = I.periodic_wave_case(n=16, kx=kx, ky=ky, nsteps=3, M=30, tau=450.0)
    p = case.params
    om = orc.OracleMesh(case.mesh)
    eta, U, Um = om.advance_sesm(case.R, p, coef, case.nsteps, case.eta0, case.U0)
    k2 = closed.kappa2_square(16, 10e3, kx, ky)
    u, e = closed.sesm_mode_amplitude(k2, p.g * 4000.0, p.tau / p.M, coef, p.M, case.nsteps)
    assert np.max(np.abs(eta - e * case.eta0)) < 1e-11
    assert abs(e) < 1.0


@pytest.mark.parametrize("nonlinear_h", [0, 1])
def test_oracle_sesm_summation_identity_and_volume(golden_se, nonlinear_h):
    coef = _sesm_coef(golden_se)
    case = I.tiny_jittered_case(nx=9, ny=7, seed=3, nonlinear_h=nonlinear_h, M=7, tau=70.0)
    om = orc.OracleMesh(case.mesh)
    eta1, U1, Um = om.advance_sesm(case.R, case.params, coef, 1, case.eta0, case.U0)
    assert np.max(np.abs((eta1 - case.eta0) + case.params.tau * om.divergence(Um))) < 1e-12
    av, _ = om.areas()
    eta3, _, _ = om.advance_sesm(case.R, case.params, coef, 3, case.eta0, case.U0)
    assert abs(np.sum(av * eta3) - np.sum(av * case.eta0)) < 1e-12 * np.sum(av * np.abs(case.eta0))


def test_oracle_sesm_matches_brute_force(golden_se):
    coef = _sesm_coef(golden_se)
    for nl in (0, 1):
        case = I.tiny_jittered_case(nx=6, ny=5, seed=13, nonlinear_h=nl)
        om = orc.OracleMesh(case.mesh)
        e1, U1, M1 = om.advance_sesm(case.R, case.params, coef, case.nsteps, case.eta0, case.U0)
        e2, U2, M2 = brute.advance_sesm(case.mesh, case.R, case.params, coef, case.nsteps, case.eta0, case.U0)
        assert np.max(np.abs(e1 - e2)) < 1e-11 * max(1.0, np.max(np.abs(e2)))
        assert np.max(np.abs(U1 - U2)) < 1e-11 * max(1.0, np.max(np.abs(U2)))
        assert np.max(np.abs(M1 - M2)) < 1e-11 * max(1.0, np.max(np.abs(M2)))


SESM_PLANTS = {
    "ab3_weights": ("const real ab0 = (real)1.5 + beta, ab1 = -((real)0.5 + 2 * beta), ab2 = beta;",
                    "const real ab0 = (real)1.5, ab1 = -((real)0.5), ab2 = 0;"),
    "am4_order": ("eAM[v] = am0 * enew[v] + am1 * E[0][v] + am2 * E[1][v] + am3 * E[2][v];",
                  "eAM[v] = am1 * enew[v] + am0 * E[0][v] + am2 * E[1][v] + am3 * E[2][v];"),
    "coriolis_sign": ("unew[2 * e] = U[0][2 * e] + dt * (m->f_e[e] * uy - g * H * gx + R[2 * e]);",
                      "unew[2 * e] = U[0][2 * e] + dt * (-m->f_e[e] * uy - g * H * gx + R[2 * e]);"),
}


@pytest.mark.parametrize("plant", sorted(SESM_PLANTS))
def test_sesm_pins_catch_planted_mistake(golden_se, plant):
    old, new = SESM_PLANTS[plant]
    src = orc.source_text()
    assert old in src
    L = orc.build_variant(src.replace(old, new), "sesm_" + plant)
    coef = _sesm_coef(golden_se)
    case = I.tiny_jittered_case(nx=6, ny=5, seed=13, nonlinear_h=1)
    om = orc.OracleMesh(case.mesh, L)
    e1, U1, M1 = om.advance_sesm(case.R, case.params, coef, case.nsteps, case.eta0, case.U0)
    e2, U2, M2 = brute.advance_sesm(case.mesh, case.R, case.params, coef, case.nsteps, case.eta0, case.U0)
    err = max(np.max(np.abs(e1 - e2)), np.max(np.abs(U1 - U2)) / max(1.0, np.max(np.abs(U2))))
    assert err > 1e-6, f"planted mistake {plant} went unnoticed"


def test_oracle_summed_momentum_identity():
    """Summing Eq. 4.10 over a step (linear H): U^M - U^0 + tau [f e_z x S' + g H0 grad(eta_bar) - R] = 0,
    S' = <<U>> - (theta/M)(U^M - U^0) + (U^0 - U^M)/(2M), eta_bar = (1/M) sum_{m<M} eta^m."""
    case = I.tiny_jittered_case(nx=9, ny=7, seed=8, nonlinear_h=0, M=9, tau=90.0)
    om = orc.OracleMesh(case.mesh)
    p = case.params
    eta1, U1, Um, _, eb = om.advance(case.R, p, 1, case.eta0, case.U0, want_eta_mean=True)
    M, th, tau = p.M, p.theta, p.tau
    Sp = Um - th / M * (U1 - case.U0) + (case.U0 - U1) / (2 * M)
    f = case.mesh.coriolis[:, None]
    cor = np.stack([-Sp[:, 1], Sp[:, 0]], axis=1) * f
    H0e = case.mesh.depth[case.mesh.tri].mean(axis=1)[:, None]
    resid = U1 - case.U0 + tau * (cor + p.g * H0e * om.gradient(eb) - case.R)
    assert np.max(np.abs(resid)) < 1e-10 * np.max(np.abs(U1 - case.U0))
    assert np.max(np.abs(U1 - case.U0)) > 1.0


# ---------------------------------------------------------------- surrogate reference network

def test_mpnn_reference_gradient_matches_finite_differences():
    """The numpy FP64 backward of the surrogate equals central differences of its forward."""
    from oracle import mpnn

    case = I.tiny_jittered_case(nx=6, ny=5, seed=2)
    G = mpnn.Graph(case.mesh)
    rng = np.random.default_rng(0)
    s = dict(eta=0.3, H=3000.0, U=5.0, R=1e-3, f=1e-4, L=1e4, out_U=1.0, out_eta=0.1)
    xv, xe = mpnn.features(G, case.eta0, case.U0, case.R, s)
    te = rng.standard_normal((G.ne, 4))
    tv = rng.standard_normal((G.nv, 1))
    w = 0.3 * rng.standard_normal(mpnn.nparams())
    L0, g = mpnn.loss_and_grad(G, w, xv, xe, te, tv, s)
    idx = rng.choice(len(w), 40, replace=False)
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mpnn.loss(*mpnn.forward(G, wp, xv, xe, s), te, tv) - mpnn.loss(*mpnn.forward(G, wm, xv, xe, s), te, tv)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mpnn_bf16_rounding():
    from oracle import mpnn

    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 1e-3], dtype=np.float32)
    r = mpnn.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125      # ties to even, then round up
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert abs(r[4] - 1e-3) < 4e-6


# ---------------------------------------------------------------- volume and energy diagnostics

ETA_OFFSET = 1.0    # a uniform elevation on top of the mode (m)


def _mode_energy(case, k2, steps):
    """Closed-form (volume, energy) after each baroclinic step of a cosine mode plus a uniform
    offset c on the periodic right-triangle mesh (linear H, f = 0, R = 0). A uniform elevation has
    no gradient and stays put, so eta = c + e phi and U = u G(phi), with (u, e) from the mode
    recurrence and the lumped operator -D G phi = kappa^2 phi (the 5-point stencil):
      volume                  = c A_v n^2                                  (sum_v phi_v = 0)
      sum_v A_v g eta^2 / 2   = g A_v (c^2 n^2 + e^2 sum_v phi_v^2) / 2
      sum_e A_e |U|^2 / (2 H0) = u^2 kappa^2 A_v sum_v phi_v^2 / (2 H0)
    because sum_e A_e |G phi|^2 = phi^T (A_v (-D G)) phi; and sum_v phi_v^2 = n^2 / 2 for a cosine
    mode whose doubled wavenumber is not a multiple of n. A_v = dx^2."""
    p = case.params
    n = int(round(math.sqrt(case.mesh.nv)))
    dx = 10e3
    H0 = 4000.0
    c = ETA_OFFSET
    sum_phi2 = n * n / 2.0
    out = []
    for s in range(1, steps + 1):
        u, e = closed.mode_amplitude(k2, p.g * H0, p.tau / p.M, p.theta, s * p.M)
        pe = p.g * dx * dx * (c * c * n * n + e * e * sum_phi2) / 2.0
        ke = u * u * k2 * dx * dx * sum_phi2 / (2.0 * H0)
        out.append((c * dx * dx * n * n, pe + ke, ke))
    return np.array(out)


def _energy_error(L=None, kx=3, ky=2):
    case = I.periodic_wave_case(n=16, kx=kx, ky=ky, theta=0.14, nsteps=3)
    case.eta0 = case.eta0 + ETA_OFFSET
    _, _, _, diag = orc.run_case(case, want_diag=True, L=L)
    want = _mode_energy(case, closed.kappa2_square(16, 10e3, kx, ky), case.nsteps)
    rel_e = np.max(np.abs(diag[:, 1] - want[:, 1]) / want[:, 1])
    rel_v = np.max(np.abs(diag[:, 0] - want[:, 0])) / want[0, 0]
    return rel_e, rel_v, want


@pytest.mark.parametrize("kx,ky", [(1, 0), (3, 2), (5, 7)])
def test_oracle_energy_matches_mode_closed_form(kx, ky):
    """Volume and energy of oracle_diagnostics along a cosine-mode trajectory (Eq. 4.10, linear H)
    equal the closed form of the 2x2 mode recurrence after every step."""
    rel, vol, want = _energy_error(kx=kx, ky=ky)
    assert rel < 1e-12
    assert vol < 1e-13
    # the kinetic part is a real share of the total at some step (the wave exchanges the two)
    assert np.max(want[:, 2] / want[:, 1]) > 1e-3


def test_oracle_diagnostics_by_hand_two_triangles():
    """oracle_diagnostics on a two-triangle mesh, every number worked out by hand.

    Triangles (0,1,2) with corners (0,0),(2,0),(0,2) (area 2) and (1,3,2) with (2,0),(4,4),(0,2)
    (area 6). Median-dual areas A_v = sum A_e / 3: (2/3, 8/3, 8/3, 2). Depth (100, 200, 300, 400),
    eta (1, -2, 3, 0.5), U = (3, 4) and (-1, 2), g = 10.
      volume = 2/3*1 + 8/3*(-2) + 8/3*3 + 2*0.5 = 2/3 + 8/3 + 1 = 13/3
      PE     = 5 * (2/3*1 + 8/3*4 + 8/3*9 + 2*0.25) = 5 * (2/3 + 104/3 + 1/2) = 5 * 106/3 + 5/2
      KE (H = H0)      = 2*25/(2*200) + 6*5/(2*300) = 1/8 + 1/20
      KE (H = H0+eta)  = 2*25/(2*(200+2/3)) + 6*5/(2*(300+1/2)) = 50/(400+4/3) + 30/601"""
    tri = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    P = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0], [4.0, 4.0]])
    xy = P[tri]
    mesh = I.Mesh("two", tri, xy, np.concatenate([P, np.zeros((4, 1))], axis=1),
                  np.array([100.0, 200.0, 300.0, 400.0]), np.zeros(2))
    om = orc.OracleMesh(mesh)
    eta = np.array([1.0, -2.0, 3.0, 0.5])
    U = np.array([[3.0, 4.0], [-1.0, 2.0]])
    pe = 5.0 * 106.0 / 3.0 + 2.5
    vol, en = om.diagnostics(eta, U, 10.0, 0)
    assert vol == pytest.approx(13.0 / 3.0, rel=1e-14)
    assert en == pytest.approx(pe + 1.0 / 8.0 + 1.0 / 20.0, rel=1e-14)
    vol, en = om.diagnostics(eta, U, 10.0, 1)
    assert en == pytest.approx(pe + 50.0 / (400.0 + 4.0 / 3.0) + 30.0 / 601.0, rel=1e-14)


ENERGY_PLANTS = {
    # potential energy without the 1/2
    "pe_half": ("en += (double)m->area_v[v] * 0.5 * g * eta[v] * eta[v];",
                "en += (double)m->area_v[v] * g * eta[v] * eta[v];"),
    # potential energy without g
    "pe_g": ("en += (double)m->area_v[v] * 0.5 * g * eta[v] * eta[v];",
             "en += (double)m->area_v[v] * 0.5 * eta[v] * eta[v];"),
    # kinetic energy without the 1/2
    "ke_half": ("(U[2 * e] * U[2 * e] + U[2 * e + 1] * U[2 * e + 1]) / (2.0 * H);",
                "(U[2 * e] * U[2 * e] + U[2 * e + 1] * U[2 * e + 1]) / H;"),
    # H = H0 + eta even when the linear form is asked for
    "ke_depth": ("if (nonlinear_h) H += (eta[t[0]] + eta[t[1]] + eta[t[2]]) / 3.0;",
                 "H += (eta[t[0]] + eta[t[1]] + eta[t[2]]) / 3.0;"),
    # the element area in place of the vertex (median-dual) area
    "pe_area": ("en += (double)m->area_v[v] * 0.5 * g * eta[v] * eta[v];",
                "en += (double)m->area_e[v] * 0.5 * g * eta[v] * eta[v];"),
}


@pytest.mark.parametrize("plant", sorted(ENERGY_PLANTS))
def test_energy_pins_catch_planted_mistake(plant):
    old, new = ENERGY_PLANTS[plant]
    src = orc.source_text()
    assert old in src
    L = orc.build_variant(src.replace(old, new), "energy_" + plant)
    rel, _, _ = _energy_error(L=L)
    assert rel > 1e-9, f"planted mistake {plant} went unnoticed by the closed form"


# ---------------------------------------------------------------- surrogate reference: forward pins

def _mpnn_setup(seed=0):
    from oracle import mpnn

    case = I.tiny_jittered_case(nx=7, ny=6, seed=17)
    rng = np.random.default_rng(seed)
    s = dict(eta=0.3, H=3000.0, U=5.0, R=1e-3, f=1e-4, L=1e4, out_U=1.0, out_eta=0.1)
    w = 0.3 * rng.standard_normal(mpnn.nparams())
    return mpnn, case, s, w


def _relabel(mesh, vp, ep, rot):
    """The same mesh with vertices renumbered (new index of old vertex v is vp[v]), triangles in the
    order ep (new triangle i is old triangle ep[i]) and each triangle's corners turned by rot[i]
    (a cyclic turn keeps the counter-clockwise orientation)."""
    inv_v = np.argsort(vp)
    tri = np.empty_like(mesh.tri)
    xy = np.empty_like(mesh.xy)
    for i, e in enumerate(ep):
        order = [(k + rot[i]) % 3 for k in range(3)]
        tri[i] = vp[mesh.tri[e, order]]
        xy[i] = mesh.xy[e, order]
    return I.Mesh("relabelled", tri, xy, mesh.pos[inv_v], mesh.depth[inv_v], mesh.coriolis[ep])


@pytest.mark.parametrize("bf16", [False, True])
def test_mpnn_forward_is_permutation_equivariant(bf16):
    """Renumbering vertices and triangles and turning each triangle's corner list permutes the
    network's outputs the same way: no aggregation depends on a label or a corner position."""
    mpnn, case, s, w = _mpnn_setup()
    mesh = case.mesh
    rng = np.random.default_rng(5)
    vp = rng.permutation(mesh.nv)
    ep = rng.permutation(mesh.ne)
    rot = rng.integers(0, 3, mesh.ne)
    G1 = mpnn.Graph(mesh)
    xv, xe = mpnn.features(G1, case.eta0, case.U0, case.R, s)
    oe1, ov1 = mpnn.forward(G1, w, xv, xe, s, bf16_msgs=bf16)
    m2 = _relabel(mesh, vp, ep, rot)
    G2 = mpnn.Graph(m2)
    eta2 = np.empty_like(case.eta0)
    eta2[vp] = case.eta0
    xv2, xe2 = mpnn.features(G2, eta2, case.U0[ep], case.R[ep], s)
    oe2, ov2 = mpnn.forward(G2, w, xv2, xe2, s, bf16_msgs=bf16)
    tol = 1e-2 if bf16 else 1e-12     # bf16 rounding may flip at different summation orders
    assert np.max(np.abs(oe2 - oe1[ep])) <= tol * max(1.0, np.max(np.abs(oe1)))
    assert np.max(np.abs(ov2 - ov1[np.argsort(vp)])) <= tol * max(1.0, np.max(np.abs(ov1)))
    assert np.max(np.abs(oe1)) > 1e-3 and np.max(np.abs(ov1)) > 1e-3


def _two_triangle_net():
    """Two triangles, weights zero except a few ones; the forward pass is written out by hand in
    test_mpnn_forward_by_hand."""
    from oracle import mpnn

    tri = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    P = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0], [4.0, 4.0]])
    mesh = I.Mesh("two", tri, P[tri], np.concatenate([P, np.zeros((4, 1))], axis=1),
                  np.array([100.0, 200.0, 300.0, 400.0]), np.array([1e-4, 2e-4]))
    p = {name: np.zeros(shp) for name, shp in mpnn.param_shapes()}
    C = mpnn.C
    p["Wv0"][0, 0] = 1.0        # h_v[0] = tanh(eta / s_eta)
    p["We0"][0, 1] = 1.0        # h_e[1] = tanh(U_x / s_U)
    p["We0"][5, 5] = 1.0        # h_e[5] = tanh(H0_e / s_H)
    p["We1"][C + 0, 2] = 1.0    # layer 1: h_e[2] += tanh(L d/dx h_v[0])
    p["We1"][2 * C + 0, 3] = 1.0  # layer 1: h_e[3] += tanh(L d/dy h_v[0])
    p["Wv1"][C + 1, 3] = 1.0    # layer 1: h_v[3] += tanh(area-weighted mean of h_e[1])
    p["Wv1"][0, 4] = 2.0        # layer 1: h_v[4] += tanh(2 h_v[0])
    p["We2"][2, 6] = 1.0        # layer 2: h_e[6] += tanh(h_e[2])  (after layer 1)
    p["Weo"][2, 0] = 1.0        # o_e[0] = h_e[2]
    p["Weo"][6, 1] = 1.0        # o_e[1] = h_e[6]
    p["Weo"][3, 2] = 1.0        # o_e[2] = h_e[3]
    p["Weo"][5, 3] = -1.0       # o_e[3] = -h_e[5]
    p["Wvo"][3, 0] = 1.0        # o_v = h_v[3] + 0.5 h_v[4]
    p["Wvo"][4, 0] = 0.5
    w = np.concatenate([p[n].reshape(-1) for n, _ in mpnn.param_shapes()])
    s = dict(eta=0.5, H=1000.0, U=4.0, R=1.0, f=1e-4, L=0.25, out_U=1.0, out_eta=1.0)
    eta = np.array([0.5, -0.25, 1.0, 0.0])
    U = np.array([[2.0, 1.0], [-4.0, 3.0]])
    return mpnn, mesh, w, s, eta, U


def _mpnn_by_hand():
    """The forward pass of _two_triangle_net, every step written out for this mesh.

    P1 gradients (d/dx, d/dy of each corner's basis function):
      triangle 0, corners (0,0),(2,0),(0,2): (-1/2,-1/2), (1/2,0), (0,1/2)
      triangle 1, corners (2,0),(4,4),(0,2), area 6: rot90(p_c - p_b)/(2A) gives
        corner (2,0): p_b=(4,4), p_c=(0,2): (-(2-4), (0-4))/12 = (1/6, -1/3)
        corner (4,4): p_b=(0,2), p_c=(2,0): (-(0-2), (2-0))/12 = (1/6, 1/6)
        corner (0,2): p_b=(2,0), p_c=(4,4): (-(4-0), (4-2))/12 = (-1/3, 1/6)
    Areas 2 and 6; vertex 0 touches triangle 0, vertex 3 triangle 1, vertices 1 and 2 both."""
    t = math.tanh
    hv0 = [t(0.5 / 0.5), t(-0.25 / 0.5), t(1.0 / 0.5), t(0.0)]
    L = 0.25
    dx0 = L * (-0.5 * hv0[0] + 0.5 * hv0[1] + 0.0 * hv0[2])
    dy0 = L * (-0.5 * hv0[0] + 0.0 * hv0[1] + 0.5 * hv0[2])
    dx1 = L * (hv0[1] / 6 + hv0[3] / 6 - hv0[2] / 3)
    dy1 = L * (-hv0[1] / 3 + hv0[3] / 6 + hv0[2] / 6)
    he1 = [t(2.0 / 4.0), t(-4.0 / 4.0)]             # channel 1, unchanged by the layers
    he5 = [t(200.0 / 1000.0), t(300.0 / 1000.0)]    # H0_e = corner mean of depth
    he2 = [t(dx0), t(dx1)]                          # 0 + tanh(...) after layer 1
    he3 = [t(dy0), t(dy1)]
    he6 = [t(he2[0]), t(he2[1])]                    # layer 2
    mean1 = [he1[0], (2 * he1[0] + 6 * he1[1]) / 8, (2 * he1[0] + 6 * he1[1]) / 8, he1[1]]
    hv3 = [t(m) for m in mean1]
    hv4 = [t(2 * h) for h in hv0]
    oe = np.array([[he2[e], he6[e], he3[e], -he5[e]] for e in range(2)])
    ov = np.array([[hv3[v] + 0.5 * hv4[v]] for v in range(4)])
    return oe, ov


def test_mpnn_forward_by_hand():
    """The reference network's forward pass equals a hand evaluation on two triangles: P1 gradient
    messages with their signs and the length scale, the area-weighted vertex mean, residual tanh
    updates across layers, input scaling and output wiring."""
    mpnn, mesh, w, s, eta, U = _two_triangle_net()
    G = mpnn.Graph(mesh)
    xv, xe = mpnn.features(G, eta, U, np.zeros((2, 2)), s)
    oe, ov = mpnn.forward(G, w, xv, xe, s)
    want_e, want_v = _mpnn_by_hand()
    assert np.max(np.abs(oe - want_e)) < 1e-14
    assert np.max(np.abs(ov - want_v)) < 1e-14


class _PlainMeanGraph:
    """Planted mistake: the vertex message is the unweighted mean of the incident triangles."""

    @staticmethod
    def make(mpnn, mesh):
        G = mpnn.Graph(mesh)
        cnt = np.zeros(G.nv)
        for k in range(3):
            np.add.at(cnt, G.tri[:, k], 1.0)

        def mean_msg(he):
            m = np.zeros((G.nv, he.shape[1]))
            for k in range(3):
                np.add.at(m, G.tri[:, k], he)
            return m / cnt[:, None]

        G.mean_msg = mean_msg
        return G


def _shifted_corner_graph(mpnn, mesh):
    """Planted mistake: each gradient weight paired with the next corner's features."""
    G = mpnn.Graph(mesh)

    def grad_msg(hv, L):
        gx = np.zeros((G.ne, hv.shape[1]))
        gy = np.zeros((G.ne, hv.shape[1]))
        for k in range(3):
            gx += G.grad[:, k, 0:1] * hv[G.tri[:, (k + 1) % 3]]
            gy += G.grad[:, k, 1:2] * hv[G.tri[:, (k + 1) % 3]]
        return L * gx, L * gy

    G.grad_msg = grad_msg
    return G


def _flipped_gradient_graph(mpnn, mesh):
    """Planted mistake: the x and y gradient messages swapped."""
    G = mpnn.Graph(mesh)
    orig = G.grad_msg
    G.grad_msg = lambda hv, L: orig(hv, L)[::-1]
    return G


def _label_dependent_graph(mpnn, mesh):
    """Planted mistake: the vertex mean divides by the area sum of the vertex with the next label."""
    G = mpnn.Graph(mesh)
    orig = G.mean_msg

    def mean_msg(he):
        m = orig(he) * G.asum[:, None]
        return m / np.roll(G.asum, 1)[:, None]

    G.mean_msg = mean_msg
    return G


@pytest.mark.parametrize("plant", ["plain_mean", "shifted_corner", "flipped_gradient", "label_dependent"])
def test_mpnn_pins_catch_planted_mistake(plant):
    """Each planted mistake in the reference network's message operators fails the hand evaluation
    or the permutation test."""
    from oracle import mpnn

    make = {"plain_mean": lambda m: _PlainMeanGraph.make(mpnn, m),
            "shifted_corner": lambda m: _shifted_corner_graph(mpnn, m),
            "flipped_gradient": lambda m: _flipped_gradient_graph(mpnn, m),
            "label_dependent": lambda m: _label_dependent_graph(mpnn, m)}[plant]
    _, mesh, w, s, eta, U = _two_triangle_net()
    G = make(mesh)
    xv, xe = mpnn.features(G, eta, U, np.zeros((2, 2)), s)
    oe, ov = mpnn.forward(G, w, xv, xe, s)
    want_e, want_v = _mpnn_by_hand()
    hand_err = max(np.max(np.abs(oe - want_e)), np.max(np.abs(ov - want_v)))
    # permutation test on the jittered mesh with the planted operator
    _, case, s2, w2 = _mpnn_setup()
    m1 = case.mesh
    rng = np.random.default_rng(5)
    vp, ep, rot = rng.permutation(m1.nv), rng.permutation(m1.ne), rng.integers(0, 3, m1.ne)
    G1 = make(m1)
    xv1, xe1 = mpnn.features(G1, case.eta0, case.U0, case.R, s2)
    oe1, ov1 = mpnn.forward(G1, w2, xv1, xe1, s2)
    m2 = _relabel(m1, vp, ep, rot)
    G2 = make(m2)
    eta2 = np.empty_like(case.eta0)
    eta2[vp] = case.eta0
    xv2, xe2 = mpnn.features(G2, eta2, case.U0[ep], case.R[ep], s2)
    oe2, ov2 = mpnn.forward(G2, w2, xv2, xe2, s2)
    perm_err = max(np.max(np.abs(oe2 - oe1[ep])), np.max(np.abs(ov2 - ov1[np.argsort(vp)])))
    assert max(hand_err, perm_err) > 1e-6, f"planted mistake {plant} went unnoticed"
