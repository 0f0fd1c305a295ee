"""HMC trajectory oracle (TEST INFRASTRUCTURE): the steps either side of the
MD force step of Alg. 2 -- momenta, link update, leapfrog -- written plainly
in numpy on top of the FP64 oracle's forces and actions.

Only ``tests/`` may import this module.  It shares no code with the CUDA
library.  Readings (the paper gives the HMC algorithm of Sec. 2 by name and
fixes none of these):

* momenta P_mu(x) = sum_a P^a T^a, T^a = lambda^a / 2, on the dynamic links
  (U_0(x) for x0 = 0..T-1, U_k(x) for x0 = 1..T-1); the spatial boundary links
  at x0 = 0, T are fixed and carry no momentum;
* H = sum (P^a)^2 / 2 + S_g + S_f, S_f = sum_i |Dhat^-1 phi_i|^2 (Eq. 2);
* equations of motion dU/dt = i P U, dP^a/dt = -F^a with F^a = dS/d omega^a
  for U -> exp(i omega^a T^a) U (the force of Eq. 3 plus the gauge force);
* leapfrog: P -= dt/2 F; n times {U <- exp(i dt P) U; P -= dt F}, the last
  kick dt/2;
* the second-order minimum-norm integrator of Omelyan, Mryglod and Folk
  (2003): per step P -= lam dt F; U <- exp(i dt/2 P) U; P -= (1 - 2 lam) dt F;
  U <- exp(i dt/2 P) U; P -= lam dt F, lam = 0.1931833275037836 (the value
  that minimises the norm of its leading error terms); the closing kick of a
  step and the opening kick of the next add up to one kick of 2 lam dt;
* two time scales (Sexton and Weingarten 1992): the fermion force kicks with
  the leapfrog's step dt, and each step's drift is split into m gauge-force
  leapfrog steps of dt / m:  P -= dt/2 F_f;  n times {m times {P -= dt/(2m) F_g;
  U <- exp(i dt/m P) U; P -= dt/(2m) F_g};  P -= dt/2 F_f}, neighbouring
  half kicks merged.
"""
from __future__ import annotations

import numpy as np

from . import force, gauge_force, plaquette_action, solve_pair

# Gell-Mann matrices, written out here
_GM = np.zeros((8, 3, 3), np.complex128)
_GM[0][0, 1] = _GM[0][1, 0] = 1
_GM[1][0, 1], _GM[1][1, 0] = -1j, 1j
_GM[2][0, 0], _GM[2][1, 1] = 1, -1
_GM[3][0, 2] = _GM[3][2, 0] = 1
_GM[4][0, 2], _GM[4][2, 0] = -1j, 1j
_GM[5][1, 2] = _GM[5][2, 1] = 1
_GM[6][1, 2], _GM[6][2, 1] = -1j, 1j
_GM[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)


def gell_mann() -> np.ndarray:
    return _GM.copy()


def dynamic_mask(L: int, T: int) -> np.ndarray:
    """[(T+1) L^3, 4] bool: the links the MD moves."""
    x0 = np.repeat(np.arange(T + 1), L ** 3)
    m = np.zeros(((T + 1) * L ** 3, 4), bool)
    m[:, 0] = x0 <= T - 1
    m[:, 1:] = ((x0 >= 1) & (x0 <= T - 1))[:, None]
    return m


def algebra(P: np.ndarray) -> np.ndarray:
    """sum_a P^a lambda^a / 2 for P [..., 8] -> Hermitian [..., 3, 3]."""
    return np.einsum("...a,abc->...bc", P, _GM) / 2.0


def expi(H: np.ndarray, dt: float) -> np.ndarray:
    """exp(i dt H) of Hermitian H [..., 3, 3] by its eigen-decomposition."""
    w, V = np.linalg.eigh(H)
    return np.einsum("...ab,...b,...cb->...ac", V, np.exp(1j * dt * w), V.conj())


def update_links(U: np.ndarray, P: np.ndarray, dt: float, L: int, T: int) -> np.ndarray:
    """U <- exp(i dt P) U on the dynamic links."""
    out = U.copy()
    m = dynamic_mask(L, T)
    E = expi(algebra(P[m]), dt)
    out[m] = np.einsum("nab,nbc->nac", E, U[m])
    return out


def kinetic(P: np.ndarray, L: int, T: int) -> float:
    return 0.5 * float(np.sum(P[dynamic_mask(L, T)] ** 2))


def fermion_action_and_force(U, phi, L, T, theta, kappa, tol=1e-13):
    """(S_f, F_f) at U: X = Dhat^-1 phi, Y = Dhat^-dag X by the oracle solver."""
    X, Y, _ = solve_pair(U, phi, L, T, theta, kappa, tol=tol)
    return float(np.sum(np.abs(X) ** 2)), force(U, X, Y, L, T, theta, kappa)


def leapfrog(U, P, phi, L, T, theta, kappa, beta, nsteps, dt, tol=1e-13):
    """One leapfrog trajectory.  Returns (U, P, H parts at start, at end)."""
    m = dynamic_mask(L, T)
    P = P.copy()
    P[~m] = 0.0
    K0, G0 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    S0, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
    P -= 0.5 * dt * (gauge_force(U, L, T, beta) + Ff)
    S1 = S0
    for k in range(nsteps):
        U = update_links(U, P, dt, L, T)
        S1, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
        e = 0.5 * dt if k == nsteps - 1 else dt
        P -= e * (gauge_force(U, L, T, beta) + Ff)
    K1, G1 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    return U, P, (K0, G0, S0), (K1, G1, S1)


# the minimum-norm parameter of the second-order integrator (Omelyan, Mryglod, Folk 2003)
OMELYAN_LAMBDA = 0.1931833275037836


def omelyan(U, P, phi, L, T, theta, kappa, beta, nsteps, dt, lam=OMELYAN_LAMBDA, tol=1e-13):
    """One trajectory of the second-order minimum-norm integrator, two force
    evaluations per step.  lam = 1/2 is the leapfrog of step dt (its middle
    kick vanishes and its two half drifts make one).  Returns (U, P, H parts
    at start, at end)."""
    m = dynamic_mask(L, T)
    P = P.copy()
    P[~m] = 0.0
    K0, G0 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    S0, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
    P -= lam * dt * (gauge_force(U, L, T, beta) + Ff)
    S1 = S0
    for k in range(nsteps):
        U = update_links(U, P, 0.5 * dt, L, T)
        _, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
        P -= (1.0 - 2.0 * lam) * dt * (gauge_force(U, L, T, beta) + Ff)
        U = update_links(U, P, 0.5 * dt, L, T)
        S1, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
        e = lam * dt if k == nsteps - 1 else 2.0 * lam * dt
        P -= e * (gauge_force(U, L, T, beta) + Ff)
    K1, G1 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    return U, P, (K0, G0, S0), (K1, G1, S1)


def leapfrog_two_scales(U, P, phi, L, T, theta, kappa, beta, nsteps, dt, m, tol=1e-13):
    """Nested leapfrog: the fermion force on steps of dt, the gauge force on
    m substeps of dt / m per step (m = 1 is the leapfrog).  Returns (U, P, H
    parts at start, at end)."""
    mk = dynamic_mask(L, T)
    P = P.copy()
    P[~mk] = 0.0
    K0, G0 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    S0, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
    h = dt / m
    P -= 0.5 * h * gauge_force(U, L, T, beta)
    P -= 0.5 * dt * Ff
    S1 = S0
    for k in range(nsteps):
        for j in range(m):
            U = update_links(U, P, h, L, T)
            e = 0.5 * h if (k == nsteps - 1 and j == m - 1) else h
            P -= e * gauge_force(U, L, T, beta)
        S1, Ff = fermion_action_and_force(U, phi, L, T, theta, kappa, tol)
        P -= (0.5 * dt if k == nsteps - 1 else dt) * Ff
    K1, G1 = kinetic(P, L, T), plaquette_action(U, L, T, beta)
    return U, P, (K0, G0, S0), (K1, G1, S1)
