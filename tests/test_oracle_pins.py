"""Pins of the FP64 oracle to the paper and to mathematics (no GPU).

Each test checks the oracle against something other than itself: the covariant
definition of T^{mu nu} (Eq. 1), a generic root solve, flux-Jacobian
eigenvalues, exact polynomial reconstruction, the integral definition of the
WENO smoothness indicators (sympy), invariants of the discrete scheme, the
exact p = e/3 shock tube, Simpson's rule for the source (Eq. 3 integrated
along the light-speed path), an independent ODE solution for the time
integrator's order and the run parameters printed in the paper.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import physics_ref as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- pointwise physics

def _random_prims(rng, n, vmax_gamma=50.0):
    e = 10 ** rng.uniform(-3, 2, n)
    # four-velocity with random direction and gamma up to vmax_gamma
    g = 1.0 + (vmax_gamma - 1.0) * rng.uniform(0, 1, n) ** 3
    umag = np.sqrt(g * g - 1.0)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = umag * d
    nn = rng.uniform(0, 1, n)
    return np.stack([e, u[0], u[1], u[2], nn])


def test_prim_to_cons_matches_tensor_definition(orc):
    rng = np.random.default_rng(1)
    prim = _random_prims(rng, 200)
    cons = orc.prim_to_cons(prim)
    for s in range(prim.shape[1]):
        want = ref.conserved(prim[0, s], prim[1:4, s], prim[4, s])
        np.testing.assert_allclose(cons[:, s], want, rtol=1e-13, atol=0)


def test_cons_to_prim_round_trip_up_to_gamma_7000(orc):
    rng = np.random.default_rng(2)
    n = 200000
    e = 10 ** rng.uniform(-3, 2, n)
    v = 1.0 - 10 ** rng.uniform(-8, 0, n)          # |v| up to 1 - 1e-8
    v[: n // 10] = rng.uniform(0, 0.9, n // 10)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    gamma = 1.0 / np.sqrt((1.0 - v) * (1.0 + v))
    u = gamma * v * d
    nn = rng.uniform(0.01, 1, n)
    cons = orc.prim_to_cons(np.stack([e, u[0], u[1], u[2], nn]))
    prim, hits = orc.cons_to_prim(cons, e_floor=1e-30)
    assert hits == 0
    g2 = gamma * gamma
    # the closed form loses digits like the conserved variables themselves (E ~ |M| as gamma grows)
    assert np.max(np.abs(prim[0] / e - 1.0) / g2) < 1e-14
    vrec = np.sqrt(prim[1] ** 2 + prim[2] ** 2 + prim[3] ** 2)
    assert np.max(np.abs(vrec - v) / g2) < 1e-15
    np.testing.assert_allclose(prim[1:4] * vrec / np.where(vrec > 0, vrec, 1), v * d, atol=1e-12)
    np.testing.assert_allclose(prim[4], e / 3.0, rtol=1e-13 * np.max(g2))
    assert np.max(np.abs(prim[5] / nn - 1.0) / g2) < 1e-14


def test_cons_to_prim_matches_generic_root_solve(orc):
    rng = np.random.default_rng(3)
    prim = _random_prims(rng, 40, vmax_gamma=5.0)
    cons = orc.prim_to_cons(prim)
    out, _ = orc.cons_to_prim(cons, e_floor=1e-30)
    for s in range(prim.shape[1]):
        e, u3, n = ref.primitives_by_solve(cons[:, s])
        g = math.sqrt(1.0 + u3 @ u3)
        np.testing.assert_allclose(out[0, s], e, rtol=1e-9)
        np.testing.assert_allclose(out[1:4, s], u3 / g, atol=1e-9)
        np.testing.assert_allclose(out[5, s], n, rtol=1e-9)


def test_cons_to_prim_floors_and_rest_frame(orc):
    cons = np.array([[2.0, 1e-40, 5.0], [0.0, 0.0, 5.0 + 1e-6], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0],
                     [0.3, 0.0, 0.0]])
    prim, hits = orc.cons_to_prim(cons, e_floor=1e-20)
    # rest frame: e = E, v = 0, n = R
    assert prim[0, 0] == 2.0 and prim[1, 0] == 0.0 and prim[5, 0] == 0.3
    assert hits == 2        # E below the floor, and |M| > E
    assert prim[0, 1] == 1e-20
    assert 0.0 < prim[0, 2] and prim[1, 2] < 1.0


def test_characteristic_speeds_special_cases(orc):
    c = 1.0 / math.sqrt(3.0)
    lm, lp = orc.char_speeds([0.0, 0.0, 0.0], 0)
    assert abs(lp - c) < 1e-15 and abs(lm + c) < 1e-15
    for v in (0.3, -0.7, 0.99):
        for d in range(3):
            vec = [0.0, 0.0, 0.0]
            vec[d] = v
            lm, lp = orc.char_speeds(vec, d)
            assert abs(lp - (v + c) / (1 + v * c)) < 1e-14     # relativistic velocity addition
            assert abs(lm - (v - c) / (1 - v * c)) < 1e-14


def test_characteristic_speeds_are_flux_jacobian_eigenvalues(orc):
    rng = np.random.default_rng(4)
    for _ in range(6):
        e = rng.uniform(0.5, 20)
        u3 = rng.normal(size=3) * 0.6
        g = math.sqrt(1 + u3 @ u3)
        for d in range(3):
            ev = ref.jacobian_eigenvalues(e, u3, 0.4, d)
            lm, lp = orc.char_speeds(u3 / g, d)
            assert abs(ev[0] - lm) < 2e-6 and abs(ev[-1] - lp) < 2e-6


# --------------------------------------------------------------- WENO

def _cell_averages(coeffs, cells):
    P = np.polynomial.Polynomial(coeffs)
    Q = P.integ()
    return np.array([Q(j + 0.5) - Q(j - 0.5) for j in cells]), P


def test_weno7_reconstructs_degree6_polynomials_exactly_with_linear_weights(orc):
    rng = np.random.default_rng(5)
    for deg in range(7):
        coeffs = rng.normal(size=deg + 1)
        f, P = _cell_averages(coeffs, range(-3, 4))
        val, q, _, w = orc.weno7(f, eps=1e30)
        np.testing.assert_allclose(w, np.array([1, 12, 18, 4]) / 35.0, rtol=1e-15)
        assert abs(val - P(0.5)) < 1e-12 * max(1.0, np.abs(coeffs).sum())
    # degree 7 is not reproduced: the composite stencil is exactly 7th order
    f, P = _cell_averages([0, 0, 0, 0, 0, 0, 0, 1.0], range(-3, 4))
    val, _, _, _ = orc.weno7(f, eps=1e30)
    assert abs(val - P(0.5)) > 1e-3


def test_weno7_candidates_exact_for_cubics(orc):
    rng = np.random.default_rng(6)
    coeffs = rng.normal(size=4)
    f, P = _cell_averages(coeffs, range(-3, 4))
    _, q, _, _ = orc.weno7(f)
    np.testing.assert_allclose(q, P(0.5), rtol=1e-13)


def _beta_integral_sympy(vals, cells):
    """Sum_{l>=1} int_{-1/2}^{1/2} (d^l p / dx^l)^2 dx for the polynomial p whose
    cell averages on `cells` equal `vals` (exact rationals)."""
    import sympy as sp
    x = sp.symbols("x")
    n = len(cells)
    c = sp.symbols("c0:%d" % n)
    P = sum(c[k] * x**k for k in range(n))
    eqs = [sp.integrate(P, (x, j - sp.Rational(1, 2), j + sp.Rational(1, 2))) - sp.Rational(v) for j, v in
           zip(cells, vals)]
    P = P.subs(sp.solve(eqs, c))
    return sum(sp.integrate(sp.diff(P, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
               for l in range(1, n))


def test_weno7_smoothness_indicators_match_integral_definition(orc):
    rng = np.random.default_rng(7)
    for _ in range(3):
        vals = [Fraction(int(v), 8) for v in rng.integers(-40, 40, 7)]
        _, _, beta, _ = orc.weno7(np.array([float(v) for v in vals]))
        for k in range(4):
            exact = _beta_integral_sympy(vals[k:k + 4], list(range(k - 3, k + 1)))
            assert abs(beta[k] - float(exact)) <= 1e-12 * max(1.0, abs(float(exact)))


def test_weno7_eno_property_on_a_step(orc):
    f = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    val, q, beta, w = orc.weno7(f)
    assert beta[0] == 0.0 and w[0] > 1 - 1e-9     # only the stencil left of the jump is smooth
    assert abs(val) < 1e-9
    np.testing.assert_allclose(w.sum(), 1.0, rtol=1e-15)


def test_weno5_polynomial_exactness_and_indicators(orc):
    rng = np.random.default_rng(8)
    for deg in range(5):
        f, P = _cell_averages(rng.normal(size=deg + 1), range(-2, 3))
        val, _, _, w = orc.weno5(f, eps=1e30)
        np.testing.assert_allclose(w, [0.1, 0.6, 0.3], rtol=1e-15)
        assert abs(val - P(0.5)) < 1e-12
    f, P = _cell_averages(rng.normal(size=3), range(-2, 3))
    _, q, _, _ = orc.weno5(f)
    np.testing.assert_allclose(q, P(0.5), rtol=1e-13)
    vals = [Fraction(int(v), 4) for v in rng.integers(-20, 20, 5)]
    _, _, beta, _ = orc.weno5(np.array([float(v) for v in vals]))
    for k in range(3):
        exact = _beta_integral_sympy(vals[k:k + 3], list(range(k - 2, k + 1)))
        assert abs(beta[k] - float(exact)) <= 1e-12 * max(1.0, abs(float(exact)))


# --------------------------------------------------------------- source terms (Eqs. 2-3)

def test_paper_parameters_golden():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        g = json.load(fh)
    from paper_1511_02137_b300 import workloads
    import oracle
    c = oracle.Config(8, 8, 8)
    assert (c.k_rad, c.k_coll, c.cr_over_cf) == (g["k_rad"]["value"], g["k_coll"]["value"], g["cr_over_cf"]["value"])
    w = workloads.ELLIPSOIDAL_256
    assert w.n == tuple(g["grid"]["value"])
    assert w.dx == g["dx_fm"]["value"] and w.dt == g["dt_fm_per_c"]["value"] and w.t0 == g["t0_fm_per_c"]["value"]
    assert abs(w.t0 + w.steps * w.dt - g["t_end_fm_per_c"]["value"]) < 1e-12


def test_temperature_inverts_the_eos(orc):
    c = orc.Config(8, 8, 8)
    for e in (1e-3, 0.03, 1.0, 30.0, 1e4):
        T = orc.temperature(c, e)
        back = math.pi ** 2 / 30.0 * 47.5 * T ** 4 / 0.1973 ** 3
        assert abs(back / e - 1.0) < 1e-14
    assert abs(orc.temperature(c, 30.0) - 0.3485) < 5e-5


def test_energy_loss_law_scaling(orc):
    """Eq. 3: radiative part ~ T^3 x, collisional part ~ T^2, both ~ C_R/C_F."""
    rad = orc.Config(8, 8, 8, k_coll=0.0)
    col = orc.Config(8, 8, 8, k_rad=0.0)
    T, ell = 0.31, 1.7
    assert abs(orc.jet_dEdx(rad, 2 * T, ell) / orc.jet_dEdx(rad, T, ell) - 8.0) < 1e-13
    assert abs(orc.jet_dEdx(rad, T, 3 * ell) / orc.jet_dEdx(rad, T, ell) - 3.0) < 1e-13
    assert abs(orc.jet_dEdx(col, 2 * T, ell) / orc.jet_dEdx(col, T, ell) - 4.0) < 1e-13
    assert orc.jet_dEdx(col, T, 0.0) == orc.jet_dEdx(col, T, 5.0)
    assert orc.jet_dEdx(rad, T, 0.0) == 0.0
    both = orc.Config(8, 8, 8, cr_over_cf=2.25)
    ref1 = orc.Config(8, 8, 8)
    assert abs(orc.jet_dEdx(both, T, ell) / orc.jet_dEdx(ref1, T, ell) - 2.25) < 1e-13


def test_jet_cell_index(orc):
    c = orc.Config(16, 16, 16, dx=0.1, t0=1.0)
    j = orc.Jet((-0.8, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0)
    inside, ijk, ell = orc.jet_cell(c, j, 1.0)
    assert inside and ijk == (0, 8, 8) and ell == 0.0   # y = z = 0 lies on a face: upper cell
    inside, ijk, _ = orc.jet_cell(c, j, 1.0 + 0.85)
    assert ijk[0] == 8
    inside, ijk, _ = orc.jet_cell(c, j, 1.0 + 1.61)     # x = 0.81 > 0.8: left the grid
    assert not inside and ijk == (-1, -1, -1)
    inside, _, _ = orc.jet_cell(c, j, 0.9)               # before t_start
    assert not inside


def _uniform_U(orc, shape, e, u3, n):
    prim = np.empty((5,) + shape)
    prim[0], prim[1], prim[2], prim[3], prim[4] = e, u3[0], u3[1], u3[2], n
    return orc.prim_to_cons(prim)


def test_source_only_deposit_equals_closed_form_integral(orc):
    """Fluid off, constant T: RK3 stage times (t, t+dt, t+dt/2) with weights
    (1, 1, 4)/6 are Simpson's rule, exact for the linear-in-path law, so the
    deposited energy is k_rad T^3 L^2/(2 hc^2) + k_coll T^2 L/hc and the
    momentum is n times that."""
    scale = 1e-13  # keeps the deposit negligible against e, so T stays constant
    c = orc.Config(24, 8, 8, dx=0.1, dt=0.02, t0=1.0, fluid=False, k_rad=4.0 * scale, k_coll=2.5 * scale)
    e = 30.0
    U = _uniform_U(orc, (8, 8, 24), e, (0.0, 0.0, 0.0), 0.0)
    d = np.array([1.0, 0.2, -0.1])
    jet = orc.Jet((-1.0, 0.0, 0.0), tuple(d), 1.0)
    nsteps = 40
    _, diag = orc.run(c, U, nsteps, [jet])
    T = orc.temperature(c, e)
    L = nsteps * c.dt
    hc = 0.1973
    want = 4.0 * scale * T ** 3 * L ** 2 / (2 * hc ** 2) + 2.5 * scale * T ** 2 * L / hc
    assert abs(diag.dep_E / want - 1.0) < 1e-10
    n = d / np.linalg.norm(d)
    np.testing.assert_allclose(diag.dep_M, n * diag.dep_E, rtol=1e-14)


def test_source_only_state_change_matches_reported_deposit(orc):
    c = orc.Config(24, 8, 8, fluid=False)
    U0 = _uniform_U(orc, (8, 8, 24), 30.0, (0.0, 0.0, 0.0), 0.1)
    jet = orc.Jet((-1.0, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0)
    U1, diag = orc.run(c, U0, 20, [jet])
    dU = (U1 - U0).reshape(5, -1)
    changed = np.nonzero(np.any(dU != 0, axis=0))[0]
    assert len(changed) <= 5                       # the jet crossed at most 0.4 fm = 4-5 cells
    vol = c.dx ** 3
    assert abs(dU[0].sum() * vol / diag.dep_E - 1.0) < 1e-12
    assert abs(dU[1].sum() * vol / diag.dep_E - 1.0) < 1e-12
    assert np.all(dU[2:] == 0)


def test_rk3_is_third_order_in_time_on_the_jet_source_ode(orc):
    """Fluid off, so that the jet's cell obeys the ODE dE/dt = dM^x/dt = S^0 of
    Eq. 2-3, with T taken from the cell's state (the deposit heats and moves it:
    the ODE is nonlinear, unlike the constant-T case where any rule exact for
    linear integrands would pass).  The oracle's RK3 steps converge to an
    independent solution of the same ODE (scipy DOP853, primitives by a generic
    root solve, T from the EOS e = (pi^2/30) dof T^4/(hbar c)^3) at third order in
    dt: a second-order combination or wrong stage times give order 2 or less."""
    from scipy.integrate import solve_ivp
    hc, dof, kr, kc = 0.1973, 47.5, 4.0, 2.5
    dx, t0, span, e0, n0 = 1.0, 1.0, 0.4, 1.0, 0.1

    def rhs(t, y):
        e, _, _ = ref.primitives_by_solve(np.array([y[0], y[1], 0.0, 0.0, 0.0]))
        T = (e * hc ** 3 / (math.pi ** 2 / 30.0 * dof)) ** 0.25
        S0 = (kr * T ** 3 * (t - t0) / hc ** 2 + kc * T ** 2 / hc) / dx ** 3
        return [S0, S0]

    U0 = ref.conserved(e0, np.zeros(3), n0)
    sol = solve_ivp(rhs, (t0, t0 + span), [U0[0], U0[1]], method="DOP853", rtol=1e-13, atol=1e-15)
    want = sol.y[:, -1]
    assert want[0] > 1.1 * U0[0]                 # the deposit is not a perturbation
    U = _uniform_U(orc, (4, 4, 4), e0, (0.0, 0.0, 0.0), n0)
    jet = orc.Jet((0.3, 0.5, 0.5), (1.0, 0.0, 0.0), t0)   # stays in cell (2, 2, 2): x in [0.3, 0.7]
    errs = []
    for nsteps in (4, 8, 16, 32):
        c = orc.Config(4, 4, 4, dx=dx, dt=span / nsteps, t0=t0, fluid=False, k_rad=kr, k_coll=kc)
        U1, diag = orc.run(c, U, nsteps, [jet])
        assert diag.jet_cells[0] == (2, 2, 2)
        got = np.array([U1[0, 2, 2, 2], U1[1, 2, 2, 2]])
        errs.append(np.max(np.abs(got - want) / np.abs(want)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(2.85 < q < 3.15 for q in orders), (errs, orders)   # measured 3.01, 3.01, 3.00
    assert errs[-1] < 2e-8, errs


# --------------------------------------------------------------- whole operator

@pytest.mark.parametrize("boundary", ["outflow", "periodic"])
@pytest.mark.parametrize("u3", [(0.0, 0.0, 0.0), (0.3, -0.5, 0.2)])
def test_uniform_state_has_zero_rhs_bitwise(orc, boundary, u3):
    c = orc.Config(9, 6, 5, boundary=boundary)
    U = _uniform_U(orc, (5, 6, 9), 7.0, u3, 0.2)
    L, hits, vmax = orc.rhs(c, U, 1.0)
    assert hits == 0
    assert np.all(L == 0.0)
    U1, _ = orc.run(c, U, 2)
    # the RK3 combination itself rounds (e.g. 3/4 u + 1/4 u), but every cell rounds alike
    for q in range(5):
        assert np.all(U1[q] == U1[q].flat[0])
    np.testing.assert_allclose(U1, U, rtol=1e-15, atol=0)


@pytest.mark.parametrize("boundary,pad_mode", [("outflow", "edge"), ("periodic", "wrap")])
def test_boundaries_equal_explicit_ghost_layers(orc, boundary, pad_mode):
    """The ghost fill by definition: outflow copies the edge cell into every
    ghost layer (zero gradient), periodic wraps.  L of a grid with that boundary
    equals, bit for bit, L on the interior of the same grid padded by 4 explicit
    layers (numpy's 'edge' / 'wrap' padding; 4 = the reach of the interface
    stencils) and stepped with outflow boundaries, whose own ghosts the interior
    never reaches."""
    rng = np.random.default_rng(11)
    shape = (8, 9, 10)   # (nz, ny, nx)
    prim = np.empty((5,) + shape)
    prim[0] = 10 ** rng.uniform(-1, 1, shape)
    prim[1:4] = rng.uniform(-0.8, 0.8, (3,) + shape)
    prim[4] = rng.uniform(0.05, 0.2, shape)
    U = orc.prim_to_cons(prim)
    Up = np.pad(U, ((0, 0), (4, 4), (4, 4), (4, 4)), mode=pad_mode)
    L, _, _ = orc.rhs(orc.Config(10, 9, 8, boundary=boundary), U, 1.0)
    Lp, _, _ = orc.rhs(orc.Config(18, 17, 16, boundary="outflow"), Up, 1.0)
    assert np.array_equal(L, Lp[:, 4:-4, 4:-4, 4:-4])
    assert np.any(L != 0.0)
    if boundary == "outflow":   # not what a mirror (reflecting) fill would give
        Um = np.pad(U, ((0, 0), (4, 4), (4, 4), (4, 4)), mode="symmetric")
        Lm, _, _ = orc.rhs(orc.Config(18, 17, 16, boundary="outflow"), Um, 1.0)
        assert not np.array_equal(L, Lm[:, 4:-4, 4:-4, 4:-4])


def test_conservation_with_periodic_boundaries(orc):
    """Periodic box: sum(E) and sum(M) change only by the RK3-weighted jet deposit."""
    rng = np.random.default_rng(9)
    c = orc.Config(16, 12, 10, boundary="periodic")
    z, y, x = np.meshgrid(np.arange(10), np.arange(12), np.arange(16), indexing="ij")
    prim = np.stack([5 + 2 * np.sin(2 * np.pi * x / 16) * np.cos(2 * np.pi * y / 12),
                     0.2 * np.sin(2 * np.pi * z / 10), 0.1 * np.cos(2 * np.pi * x / 16), 0.05 + 0 * x,
                     0.3 + 0.1 * np.sin(2 * np.pi * y / 12)])
    U = orc.prim_to_cons(prim)
    jets = [orc.Jet((-0.5, 0.1, 0.0), (1.0, 0.3, 0.1), 1.0), orc.Jet((0.2, -0.3, 0.1), (-0.2, 1.0, 0.4), 1.02)]
    U1, diag = orc.run(c, U, 6, jets)
    vol = c.dx ** 3
    dE = (U1[0].sum() - U[0].sum()) * vol
    assert diag.dep_E > 0
    assert abs(dE - diag.dep_E) <= 1e-13 * U[0].sum() * vol
    for a in range(3):
        dM = (U1[1 + a].sum() - U[1 + a].sum()) * vol
        assert abs(dM - diag.dep_M[a]) <= 1e-13 * U[0].sum() * vol
    assert abs(U1[4].sum() - U[4].sum()) <= 1e-13 * U[4].sum()


def _tube(orc, N, axis, eL=10.0, eR=1.0, length=10.0, t_end=2.0):
    dx = length / N
    shape = [1, 1, 1]
    shape[axis] = N
    c = orc.Config(shape[0], shape[1], shape[2], dx=dx, dt=0.2 * dx, t0=0.0)
    xc = (np.arange(N) + 0.5 - N / 2) * dx
    e = np.where(xc < 0, eL, eR)
    prim = np.zeros((5, N))
    prim[0] = e
    prim[4] = 0.1
    U = orc.prim_to_cons(prim).reshape((5, shape[2], shape[1], shape[0]))
    steps = int(round(t_end / c.dt))
    U1, diag = orc.run(c, U, steps)
    return U1.reshape(5, N), xc, steps * c.dt, diag


def test_shock_tube_against_exact_riemann_solution(orc):
    errs = []
    for N in (50, 100, 200):
        U, xc, t, diag = _tube(orc, N, 0)
        assert diag.floor_hits == 0
        prim, _ = orc.cons_to_prim(U)
        exact, es, vs, vshock = ref.riemann_profile(10.0, 1.0, xc / t)
        errs.append(np.abs(prim[0] - exact).mean())
        # shock position: right-most crossing of the mid level between e* and e_R
        mid = 0.5 * (es + 1.0)
        i = np.nonzero(prim[0] > mid)[0].max()
        assert abs(xc[i] + 0.5 * (xc[1] - xc[0]) - vshock * t) < 2 * (xc[1] - xc[0])
    # first order overall (discontinuities): each halving of dx at least 1.6x smaller L1 error
    assert errs[1] < errs[0] / 1.6 and errs[2] < errs[1] / 1.6
    assert errs[2] < 0.05


def test_shock_tube_axis_permutation_is_bitwise(orc):
    Ux, _, _, _ = _tube(orc, 60, 0, t_end=0.6)
    Uy, _, _, _ = _tube(orc, 60, 1, t_end=0.6)
    Uz, _, _, _ = _tube(orc, 60, 2, t_end=0.6)
    assert np.array_equal(Ux[0], Uy[0]) and np.array_equal(Ux[0], Uz[0])
    assert np.array_equal(Ux[1], Uy[2]) and np.array_equal(Ux[1], Uz[3])
    assert np.array_equal(Ux[4], Uy[4]) and np.array_equal(Ux[4], Uz[4])
    assert np.all(Ux[2:4] == 0) and np.all(Uy[1] == 0) and np.all(Uz[1] == 0)


def _smooth_wave_L_error(orc, N, eps, axis=0):
    Lbox = 6.4
    dx = Lbox / N
    k = 2 * np.pi / Lbox
    xc = (np.arange(N) + 0.5 - N / 2) * dx
    shape = [1, 1, 1]
    shape[axis] = N
    c = orc.Config(shape[0], shape[1], shape[2], dx=dx, boundary="periodic", weno_eps=eps)

    def prim_at(x):
        e = 1.0 + 0.3 * np.sin(k * x)
        u = [0.0 * x, 0.0 * x, 0.0 * x]
        u[axis] = 0.2 * np.cos(k * x)
        u[(axis + 1) % 3] = 0.1 * np.sin(k * x)
        n = 0.5 + 0.1 * np.sin(k * x)
        return e, u, n

    e, u, n = prim_at(xc)
    prim = np.stack([e, u[0], u[1], u[2], n])
    U = orc.prim_to_cons(prim).reshape((5, shape[2], shape[1], shape[0]))
    L, _, _ = orc.rhs(c, U, 0.0)
    L = L.reshape(5, N)
    # exact -dF/dx by complex-step differentiation of the covariant flux
    h = 1e-30
    exact = np.empty((5, N))
    for i, x in enumerate(xc):
        ee, uu, nn = prim_at(np.array(x + 1j * h))
        F = ref.flux(ee, np.array([uu[0], uu[1], uu[2]], dtype=complex), nn, axis)
        exact[:, i] = -F.imag / h
    return np.abs(L - exact).max()


@pytest.mark.parametrize("axis", [0, 2])
def test_spatial_operator_is_seventh_order_with_linear_weights(orc, axis):
    errs = [_smooth_wave_L_error(orc, N, 1e30, axis) for N in (16, 32, 64)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 6.8, (errs, orders)


def test_spatial_operator_converges_with_js_weights(orc):
    """With the Jiang-Shu weights (eps = 1e-6) the nonlinear weights approach
    the linear ones as the grid is refined, so the spatial operator reaches 7th
    order on the finest pair (measured 6.57 for 64 -> 128)."""
    errs = [_smooth_wave_L_error(orc, N, 1e-6) for N in (32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] >= 6.5, (errs, orders)


def test_passive_charge_wave_is_exact_solution(orc):
    """Uniform e and v with a charge wave: E and M stay uniform bitwise and R
    follows n(x - v t) gamma."""
    N = 64
    Lbox = 6.4
    dx = Lbox / N
    k = 2 * np.pi / Lbox
    c = orc.Config(N, 1, 1, dx=dx, dt=0.1 * dx, boundary="periodic", t0=0.0)
    xc = (np.arange(N) + 0.5 - N / 2) * dx
    ux = 0.5
    gamma = math.sqrt(1 + ux * ux)
    v = ux / gamma
    prim = np.stack([2.0 + 0 * xc, ux + 0 * xc, 0 * xc, 0 * xc, 0.5 + 0.2 * np.sin(k * xc)])
    U = orc.prim_to_cons(prim).reshape(5, 1, 1, N)
    steps = 40
    U1, _ = orc.run(c, U, steps)
    for q in range(4):
        assert np.all(U1[q] == U1[q].flat[0])
    np.testing.assert_allclose(U1[:4], U[:4], rtol=1e-14, atol=1e-300)
    t = steps * c.dt
    exact = (0.5 + 0.2 * np.sin(k * (xc - v * t))) * gamma
    assert np.abs(U1[4].ravel() - exact).max() < 1e-8


def test_jet_raises_energy_along_its_path(orc):
    """Sec. 2: the region the jet crossed holds more energy than the same run
    without the jet, and the excess grows with time."""
    from paper_1511_02137_b300 import workloads
    w = workloads.scaled(workloads.ELLIPSOIDAL_32, 16, steps=6)
    w = workloads.replace(w, sigma=(0.8, 1.0, 1.2))
    c = orc.Config(16, 16, 16)
    U = orc.prim_to_cons(workloads.ellipsoidal_primitives(w))
    jet = orc.Jet((-0.6, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0)
    excess = []
    Uj, Un = U, U
    for s in range(3):
        Uj, _ = orc.run(c, Uj, 2, [jet], step0=2 * s)
        Un, _ = orc.run(c, Un, 2, [], step0=2 * s)
        excess.append((Uj[0] - Un[0]).sum())
    assert excess[0] > 0 and excess[1] > excess[0] and excess[2] > excess[1]
