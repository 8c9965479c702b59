"""Constant-G ground-state energy from Richardson's equations (test infrastructure).

For the standard pairing Hamiltonian (all V_ij = G) written as
H = sum_i x_i n_i + G sum_{i,j} P_i^+ P_j with pair energies x_i = 2 e_i,
the pair energies E_alpha of an N-pair eigenstate obey Richardson's equations
    1 + G sum_i 1/(x_i - E_alpha) - 2 G sum_{beta != alpha} 1/(E_beta - E_alpha) = 0,
and E = sum_alpha E_alpha.  The paper compares its Lanczos results with a
Richardson solver (Sec. 5.2, Table 3) without printing the equations.

This module solves them in the eigenvalue-based variables
Lambda_i = sum_alpha 1/(x_i - E_alpha), which avoid the singular points of the
pair energies.  Eliminating E_alpha with partial fractions gives, for every i,
    Lambda_i^2 = sum_{j != i} (Lambda_j - Lambda_i)/(x_j - x_i) - Lambda_i / G,
and the energy follows as E = G [ N (Omega - N + 1) - sum_i x_i Lambda_i ].
With u_i = G Lambda_i the system reads
    F_i(u; G) = u_i^2 + u_i - G sum_{j != i} (u_j - u_i)/(x_j - x_i) = 0,
whose G -> 0 solutions are u_i = -n_i for an occupation pattern n.  The ground
state is continued from the pattern that fills the N lowest x_i, in small steps
of G with a secant predictor and Newton's method as corrector.

Requires distinct x_i (non-degenerate levels).
"""
from __future__ import annotations

import numpy as np


def _residual(u, x, G):
    dx = x[None, :] - x[:, None]          # dx[i, j] = x_j - x_i
    np.fill_diagonal(dx, np.inf)
    du = u[None, :] - u[:, None]          # du[i, j] = u_j - u_i
    return u * u + u - G * np.sum(du / dx, axis=1)


def _jacobian(u, x, G):
    dx = x[None, :] - x[:, None]
    np.fill_diagonal(dx, np.inf)
    J = -G / dx
    np.fill_diagonal(J, 2.0 * u + 1.0 + G * np.sum(1.0 / dx, axis=1))
    return J


def ground_energy(e, G: float, n_pairs: int, steps: int = 400) -> float:
    """Ground-state energy of H = sum_i (2 e_i) n_i + G sum_{ij} P_i^+ P_j with N pairs."""
    x = 2.0 * np.asarray(e, dtype=np.float64)
    omega = len(x)
    if len(np.unique(x)) != omega:
        raise ValueError("Richardson solver needs distinct single-particle energies")
    if n_pairs == 0:
        return 0.0
    order = np.argsort(x)
    u = np.zeros(omega)
    u[order[:n_pairs]] = -1.0
    prev_u, prev_g = None, None
    g_path = np.linspace(0.0, G, steps + 1)[1:]
    g_last = 0.0
    for g in g_path:
        if prev_u is not None:                       # secant predictor
            guess = u + (u - prev_u) * (g - g_last) / (g_last - prev_g)
        else:
            guess = u.copy()
        v = guess
        for _ in range(60):
            F = _residual(v, x, g)
            # stop once the residual is at rounding level for the size of u
            if np.max(np.abs(F)) <= 8e-16 * (1.0 + np.max(np.abs(v))) ** 2:
                break
            v = v + np.linalg.solve(_jacobian(v, x, g), -F)
        else:
            raise RuntimeError("Newton did not converge at G=%g" % g)
        prev_u, prev_g = u, g_last
        u, g_last = v, g
    return float(G * n_pairs * (omega - n_pairs + 1) - np.dot(x, u))
