"""Independent test-side physics used to pin the oracle.

Nothing here calls the oracle or the CUDA library.  The stress tensor is built
from its covariant definition (Eq. 1) with numpy, primitives are recovered by
a generic nonlinear solve instead of the closed form, and the shock tube is
solved exactly from the Riemann invariant of the rarefaction and the Taub
jump conditions of the shock for p = e/3 (textbook relativistic gas dynamics).
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import optimize

G_INV = np.diag([1.0, -1.0, -1.0, -1.0])   # g^{mu nu}, signature (+,-,-,-)
C_S = 1.0 / math.sqrt(3.0)                   # sound speed for p = e/3


def stress_tensor(e, u3, n=0.0):
    """T^{mu nu} = (e+p) u^mu u^nu - p g^{mu nu} and N^mu = n u^mu, p = e/3."""
    u3 = np.asarray(u3, dtype=np.result_type(float, np.asarray(u3).dtype, np.asarray(e).dtype))
    gamma = np.sqrt(1.0 + np.dot(u3, u3))
    u = np.concatenate([[gamma], u3])
    p = e / 3.0
    T = (e + p) * np.outer(u, u) - p * G_INV
    N = n * u
    return T, N


def conserved(e, u3, n=0.0):
    T, N = stress_tensor(e, u3, n)
    return np.array([T[0, 0], T[0, 1], T[0, 2], T[0, 3], N[0]])


def flux(e, u3, n, d):
    """Flux along spatial axis d (0, 1, 2): (T^{d0}, T^{dx}, T^{dy}, T^{dz}, N^d)."""
    T, N = stress_tensor(e, u3, n)
    a = d + 1
    return np.array([T[a, 0], T[a, 1], T[a, 2], T[a, 3], N[a]])


def primitives_by_solve(U):
    """(e, u^x, u^y, u^z, n) from conserved U by a generic root solve of the
    tensor definition (no closed form)."""
    U = np.asarray(U, dtype=float)

    def resid(x):
        e, ux, uy, uz = x
        return conserved(e, np.array([ux, uy, uz]))[:4] - U[:4]

    guess = np.array([U[0], 0.0, 0.0, 0.0])
    with warnings.catch_warnings():
        # at xtol = 1e-14 fsolve reports that it cannot improve further once the
        # residual is at rounding level: that is the converged answer here
        warnings.simplefilter("ignore", RuntimeWarning)
        sol = optimize.fsolve(resid, guess, xtol=1e-14, maxfev=10000)
    gamma = math.sqrt(1.0 + sol[1:] @ sol[1:])
    return sol[0], sol[1:], U[4] / gamma


def flux_from_conserved(U, d):
    e, u3, n = primitives_by_solve(U)
    return flux(e, u3, n, d)


def jacobian_eigenvalues(e, u3, n, d, h=1e-6):
    """Eigenvalues of dF_d/dU by central differences in U."""
    U0 = conserved(e, np.asarray(u3, float), n)
    J = np.empty((5, 5))
    for k in range(5):
        s = h * max(1.0, abs(U0[k]))
        Up = U0.copy()
        Um = U0.copy()
        Up[k] += s
        Um[k] -= s
        J[:, k] = (flux_from_conserved(Up, d) - flux_from_conserved(Um, d)) / (2 * s)
    return np.sort(np.linalg.eigvals(J).real)


# ---------------------------------------------------------------- shock tube

def riemann_star(eL, eR):
    """Star state (e*, v*) of the p = e/3 Riemann problem with both sides at
    rest, eL > eR: left rarefaction, right shock."""
    pR = eR / 3.0

    def v_raref(es):   # Riemann invariant artanh(v) + (sqrt(3)/4) ln e conserved across the fan
        return math.tanh(math.sqrt(3.0) / 4.0 * math.log(eL / es))

    def v_shock(es):   # relative velocity across the shock from the Taub adiabat
        ps = es / 3.0
        return math.sqrt((ps - pR) * (es - eR) / ((eR + ps) * (es + pR)))

    es = optimize.brentq(lambda x: v_raref(x) - v_shock(x), eR * (1 + 1e-12), eL * (1 - 1e-12), xtol=1e-15,
                         rtol=1e-15)
    return es, v_raref(es)


def riemann_profile(eL, eR, xi):
    """Exact e at similarity coordinate xi = x/t."""
    es, vs = riemann_star(eL, eR)
    gs2 = 1.0 / (1.0 - vs * vs)
    Es = 4.0 / 3.0 * es * gs2 - es / 3.0
    Ms = 4.0 / 3.0 * es * gs2 * vs
    vshock = Ms / (Es - eR)          # from the jump of E and M
    xi_head = -C_S
    xi_tail = (vs - C_S) / (1.0 - vs * C_S)
    out = np.empty_like(xi)
    for i, s in enumerate(xi):
        if s <= xi_head:
            out[i] = eL
        elif s <= xi_tail:
            v = (s + C_S) / (1.0 + s * C_S)
            out[i] = eL * math.exp(-4.0 / math.sqrt(3.0) * math.atanh(v))
        elif s <= vshock:
            out[i] = es
        else:
            out[i] = eR
    return out, es, vs, vshock
