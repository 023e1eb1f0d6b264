"""Eigenvalue-weighted CP-ALS of the RR projectors (Eqs. 15-16, App. I).

Test infrastructure only (see the package docstring).

Minimises  f = sum_P eps_P^2 sum_ia (U_ia^P - sum_W y_i^W y_a^W tau^PW)^2
over the occupied factor y_o (o x W), the virtual factor y_v (v x W) and
tau (N x W) by alternating least squares, in the order y_o, y_v, tau:
  y_o:  S = (y_v^T y_v) o (tau^T E tau),  R_i^X = sum_aP E_P U_ia^P y_a^X tau^PX
        (Eq. 16; E = diag(eps^2)),  y_o = R S^-1;
  y_v:  the same with the roles of i and a exchanged;
  tau:  S = (y_o^T y_o) o (y_v^T y_v),  R_P^X = sum_ia U_ia^P y_i^X y_a^X,
        tau = R S^-1 (the weight of row P cancels in its own normal equations).
App. I solves S X = R by diagonally preconditioned CG; here a dense solve.
U is stored as (o*v) x N with row (i, a) = i*v + a.
"""
from __future__ import annotations

import numpy as np


def objective(U, eps, yo, yv, tau):
    o, v = yo.shape[0], yv.shape[0]
    rec = (yo[:, None, :] * yv[None, :, :]).reshape(o * v, -1) @ tau.T
    return float(np.sum((eps[None, :] * (U - rec)) ** 2))


def update_yo(U, eps, yo, yv, tau):
    o, v = yo.shape[0], yv.shape[0]
    E = eps ** 2
    S = (yv.T @ yv) * (tau.T @ (E[:, None] * tau))
    M = (U * E[None, :]) @ tau                          # (ov) x W
    R = np.einsum('iaX,aX->iX', M.reshape(o, v, -1), yv)
    return np.linalg.solve(S, R.T).T


def update_yv(U, eps, yo, yv, tau):
    o, v = yo.shape[0], yv.shape[0]
    E = eps ** 2
    S = (yo.T @ yo) * (tau.T @ (E[:, None] * tau))
    M = (U * E[None, :]) @ tau
    R = np.einsum('iaX,iX->aX', M.reshape(o, v, -1), yo)
    return np.linalg.solve(S, R.T).T


def update_tau(U, yo, yv):
    o, v = yo.shape[0], yv.shape[0]
    S = (yo.T @ yo) * (yv.T @ yv)
    KR = (yo[:, None, :] * yv[None, :, :]).reshape(o * v, -1)
    R = U.T @ KR
    return np.linalg.solve(S, R.T).T


def als(U, eps, yo, yv, tau, iters):
    """`iters` sweeps from (yo, yv, tau); returns the factors and the
    objective after every sweep."""
    hist = []
    for _ in range(iters):
        yo = update_yo(U, eps, yo, yv, tau)
        yv = update_yv(U, eps, yo, yv, tau)
        tau = update_tau(U, yo, yv)
        hist.append(objective(U, eps, yo, yv, tau))
    return yo, yv, tau, hist
