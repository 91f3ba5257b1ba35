"""Characteristic outflow boundary (Sec. 4, Eqs. 17-28), in float64.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

At the east column x = L of a lattice, for every fluid node (L, y), one time
step t -> t+1 does, in the paper's order:

1. macroscopic state at t (rho, u, v; p = c_s^2 rho) at columns L, L-1, L-2
   from the post-collision populations f*(t) (collision conserves rho and
   rho u, so these are the moments of the state at t);
2. derivatives: d/dx second-order one-sided backward over L, L-1, L-2,
   (3 q_L - 4 q_{L-1} + q_{L-2}) / 2; d/dy central with periodic wrap, first
   order one-sided where a neighbouring row of column L is solid (0 if both);
3. wave amplitudes L5 = (u + c_s)(p_x + rho c_s u_x), L3 = u v_x (Eqs. 20-22,
   with d rho / dx read as dp/dx in the pressure units of Eqs. 17-18);
   transverse terms T1, T3, T5 (Eqs. 23-25, as printed);
4. incoming amplitude L1 = kappa1 (p - p_inf) - kappa2 (T1 - T1_exact) + T1
   (Eq. 26), kappa1 = sigma (1 - M^2) c_s / length (Eq. 27), T1_exact = 0,
   p_inf = c_s^2 rho_out;
5. time derivatives of Eqs. 17-19 and one explicit Euler step (dt = 1) give
   the prescribed (rho, u, v) at t+1;
6. Zou & He reconstruction of the unknowns 3, 6, 7 with that prescribed
   state (f_i = f_i^eq + f_ibar^neq form, the same as the pressure outflow),
   then the correction of f_0 (Eq. 28) g_0 = f_0 + rho - (rho_0 + 2 rho_+)/(1 + u);
   ``exact_mass`` instead adds rho (1 + u) - (rho_0 + 2 rho_+), which makes
   the node's density exactly rho.

The tuner (Sec. 4.2) maps the six spatial derivatives (p_x, u_x, v_x, p_y,
u_y, v_y) of a node through an MLP to one or two outputs s; sigma = sigma_max
sigmoid(s_0) and, with a second output, kappa2 = kappa2_max sigmoid(s_1)
(else kappa2 is the given constant).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import lbm as _lbm

CS2 = _lbm.CS2
CS = math.sqrt(CS2)


@dataclass
class CBCOutflow:
    sigma: float = 0.0          # sigma of Eq. 27 (sigma_max with a tuner)
    kappa2: float = 0.0         # kappa2 of Eq. 26 (kappa2_max with a two-output tuner)
    mach: float = 0.0           # M of Eq. 27
    length: Optional[float] = None   # characteristic length of Eq. 27; None -> nx
    tuner: Optional[object] = None   # oracle.mlp.MLP, 6 inputs, 1 or 2 outputs
    exact_mass: bool = False
    tuner_bf16: bool = False    # evaluate the tuner with BF16 operands (MLP.predict_bf16)


def d_dx_backward(q, L):
    """Second-order one-sided derivative at column L over L, L-1, L-2; q (ny, nx)."""
    return 0.5 * (3.0 * q[:, L] - 4.0 * q[:, L - 1] + q[:, L - 2])


def d_dy(q, L, solid_col):
    """d/dy at column L: central with periodic wrap; where one neighbouring
    row is solid, the first-order difference towards the fluid one; 0 where
    both are.  solid_col: (ny,) bool of column L."""
    ny = q.shape[0]
    col = q[:, L]
    up = np.roll(col, -1)          # q(y+1)
    dn = np.roll(col, 1)           # q(y-1)
    s_up = np.roll(solid_col, -1)
    s_dn = np.roll(solid_col, 1)
    out = 0.5 * (up - dn)
    only_up = ~s_up & s_dn
    only_dn = s_up & ~s_dn
    out = np.where(only_up, up - col, out)
    out = np.where(only_dn, col - dn, out)
    out = np.where(s_up & s_dn, 0.0, out)
    assert out.shape == (ny,)
    return out


def sigmoid(s):
    return 1.0 / (1.0 + np.exp(-s))


def tuner_features(px, ux, vx, py, uy, vy):
    """Tuner inputs of Sec. 4.2 (spatial derivatives only), shape (ny, 6)."""
    return np.stack([px, ux, vx, py, uy, vy], axis=1)


def boundary_update(rho, u, v, px, ux, vx, py, uy, vy, sigma, kappa2, mach, length, rho_inf):
    """Steps 3-5: the prescribed (rho, u, v) at t+1 from the state and its
    derivatives at t (all arrays over the boundary rows)."""
    p = CS2 * rho
    L5 = (u + CS) * (px + rho * CS * ux)                          # Eq. 22
    L3 = u * vx                                                   # Eq. 21
    T1 = -(v * py + p * vy - rho * CS * v * vy)                   # Eq. 23
    T3 = -(v * vy + py / rho)                                     # Eq. 24
    T5 = -(v * py + p * vy + rho * CS * v * vy)                   # Eq. 25
    kappa1 = sigma * (1.0 - mach * mach) * CS / length            # Eq. 27
    L1 = kappa1 * (p - CS2 * rho_inf) - kappa2 * (T1 - 0.0) + T1  # Eq. 26
    drho = -(L5 + L1) / (2.0 * CS2) + (T5 + T1) / (2.0 * CS2)     # Eq. 17
    du = -(L5 - L1) / (2.0 * rho * CS) + (T5 - T1) / (2.0 * rho * CS)   # Eq. 18
    dv = -L3 + T3                                                 # Eq. 19
    return rho + drho, u + du, v + dv


def reconstruct(gcol, rho, u, v, exact_mass=False):
    """Step 6 on post-stream columns gcol (9, ny): Zou & He unknowns with the
    prescribed state, then the f_0 correction of Eq. 28."""
    rho0 = gcol[0] + gcol[2] + gcol[4]
    rhop = gcol[1] + gcol[5] + gcol[8]
    out = _lbm._zouhe_east_unknowns(gcol, rho, u, v)
    if exact_mass:
        out[0] = gcol[0] + rho * (1.0 + u) - (rho0 + 2.0 * rhop)
    else:
        out[0] = gcol[0] + rho - (rho0 + 2.0 * rhop) / (1.0 + u)
    return out


def cbc_east(solver, f, g):
    """East column of the step: f = post-collision f*(t) (9, ny, nx),
    g = post-stream populations at t+1.  Returns (rebuilt column (9, ny),
    per-row (sigma, kappa2) used)."""
    cfg = solver.cfg
    cb = cfg.cbc
    nx = cfg.nx
    L = nx - 1
    rho, ux, uy = _lbm.moments(f)
    p = CS2 * rho
    solid_col = solver.kind[:, L] != _lbm.FLUID
    px, uxx, vxx = d_dx_backward(p, L), d_dx_backward(ux, L), d_dx_backward(uy, L)
    py, uyy, vyy = d_dy(p, L, solid_col), d_dy(ux, L, solid_col), d_dy(uy, L, solid_col)
    ny = cfg.ny
    sigma = np.full(ny, float(cb.sigma))
    kappa2 = np.full(ny, float(cb.kappa2))
    if cb.tuner is not None:
        feats = tuner_features(px, uxx, vxx, py, uyy, vyy)
        s = np.asarray(cb.tuner.predict_bf16(feats) if cb.tuner_bf16 else cb.tuner.predict(feats))
        sigma = cb.sigma * sigmoid(s[:, 0])
        if s.shape[1] > 1:
            kappa2 = cb.kappa2 * sigmoid(s[:, 1])
    length = float(nx if cb.length is None else cb.length)
    rn, un, vn = boundary_update(rho[:, L], ux[:, L], uy[:, L], px, uxx, vxx, py, uyy, vyy,
                                 sigma, kappa2, float(cb.mach), length, float(cfg.rho_out))
    col = reconstruct(g[:, :, L], rn, un, vn, cb.exact_mass)
    return col, (sigma, kappa2)
