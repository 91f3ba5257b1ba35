"""D2Q9 lattice Boltzmann solver in float64: the oracle of the hot path.

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Nothing here is
blocked, fused or reordered: each function applies one definition from the
paper to whole arrays, and ``Solver.step`` calls them in the order of the
paper's Fig. 1 (collision, streaming, reconstruction of the unknown outflow
populations), written from the post-collision state f*(t):

  1. pull streaming                      f_i(x, t+1) = f*_i(x - c_i, t)   (Eq. 1)
  2. momentum exchange at solid links                                    (Eqs. 13-14)
  3. full-way bounce-back at solid nodes                                 (Eq. 11)
  4. inlet, Zou & He velocity (Sec. 2.2, "by symmetry")
  5. outflow: Zou & He (Eqs. 5-10), NN direct (Eq. 15) or CBC (Eqs. 17-28)
  6. collision at every fluid node, boundary nodes included (Eqs. 2-4 / MRT)

Array layout: populations are ``f[i, y, x]`` (9, ny, nx); the lateral (y)
direction is periodic (Fig. 2) and walls, where a workload wants them, are rows
of solid nodes.  x is periodic only when both open boundaries are switched off.

Lattice (D2Q9; the numbering follows the right-boundary unknowns 3, 6, 7 and
rho+ = f1 + f5 + f8, rho0 = f0 + f2 + f4 of Sec. 2.2):
  c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1)
  c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1)
  w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36, c_s^2 = 1/3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import mlp as _mlp
from . import rng as _rng

C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)
CS2 = 1.0 / 3.0
CS = math.sqrt(CS2)

FLUID, SOLID, WALL = 0, 1, 2   # cell kinds; SOLID is counted in the force, WALL is not


# --------------------------------------------------------------------------- #
# Sec. 2.1: equilibrium (Eq. 3), moments (Eq. 4), BGK (Eq. 2)
# --------------------------------------------------------------------------- #
def equilibrium(rho, ux, uy):
    """Second-order equilibrium of Eq. 3 for every direction; shape (9,) + rho.shape."""
    rho = np.asarray(rho, dtype=np.float64)
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    usq = ux * ux + uy * uy
    out = np.empty((9,) + np.broadcast(rho, ux, uy).shape)
    for i in range(9):
        cu = C[i, 0] * ux + C[i, 1] * uy
        out[i] = W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2)
                               - usq / (2.0 * CS2))
    return out


def moments(f):
    """rho = sum_i f_i and u = sum_i c_i f_i / rho (Eq. 4)."""
    rho = f.sum(axis=0)
    jx = np.tensordot(C[:, 0].astype(np.float64), f, axes=(0, 0))
    jy = np.tensordot(C[:, 1].astype(np.float64), f, axes=(0, 0))
    return rho, jx / rho, jy / rho


def collide_bgk(f, tau):
    """f* = f - (f - f^eq) / tau (Eqs. 1-2); nu = c_s^2 (tau - 1/2)."""
    rho, ux, uy = moments(f)
    return f - (f - equilibrium(rho, ux, uy)) / tau


# --------------------------------------------------------------------------- #
# MRT (named in Sec. 3.2 only): Lallemand & Luo's orthogonal D2Q9 moment basis
# --------------------------------------------------------------------------- #
def mrt_matrix():
    """Rows: rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy, from their definitions
    in terms of |c|^2 (Lallemand & Luo, Phys. Rev. E 61, 2000)."""
    cx = C[:, 0].astype(np.float64)
    cy = C[:, 1].astype(np.float64)
    c2 = cx * cx + cy * cy
    return np.array([
        np.ones(9),
        3.0 * c2 - 4.0,
        (9.0 * c2 * c2 - 21.0 * c2) / 2.0 + 4.0,
        cx,
        (3.0 * c2 - 5.0) * cx,
        cy,
        (3.0 * c2 - 5.0) * cy,
        cx * cx - cy * cy,
        cx * cy,
    ])


def mrt_default_rates(tau, s_e=1.0, s_eps=1.0, s_q=1.0):
    """Rates for the moments in ``mrt_matrix`` order.  The stress moments relax
    with 1/tau, so the shear viscosity is that of BGK with the same tau; the
    conserved moments (rho, j) get rate 0, which leaves them untouched."""
    s_nu = 1.0 / tau
    return np.array([0.0, s_e, s_eps, 0.0, s_q, 0.0, s_q, s_nu, s_nu])


def collide_mrt(f, rates):
    """m = M f; m* = m - S (m - m^eq); f* = M^-1 m*, with m^eq = M f^eq."""
    M = mrt_matrix()
    Minv = np.linalg.inv(M)
    rho, ux, uy = moments(f)
    m = np.tensordot(M, f, axes=(1, 0))
    meq = np.tensordot(M, equilibrium(rho, ux, uy), axes=(1, 0))
    S = np.asarray(rates, dtype=np.float64).reshape((9,) + (1,) * (f.ndim - 1))
    return np.tensordot(Minv, m - S * (m - meq), axes=(1, 0))


# --------------------------------------------------------------------------- #
# Eq. 1 streaming (pull form) and Eq. 11 full-way bounce-back
# --------------------------------------------------------------------------- #
def stream_pull(f):
    """g_i(x) = f_i(x - c_i) with periodic wrap in both directions.  Values
    pulled across a non-periodic x edge are the unknowns that the open
    boundaries overwrite afterwards."""
    g = np.empty_like(f)
    for i in range(9):
        g[i] = np.roll(f[i], shift=(C[i, 1], C[i, 0]), axis=(0, 1))
    return g


def momentum_exchange(f_prev, g, kind, x_periodic):
    """Force on the counted solid nodes over one step (Eqs. 13-14, dx = dt = 1).

    A link joins a counted solid node s and a fluid node s - c_i.  Across it,
    during this step, the population f_i arrives at s (``g[i, s]``, momentum
    c_i f_i into the body) and the population that full-way bounce-back stored
    at s in slot i-bar one step earlier leaves s towards the fluid
    (``f_prev[OPP[i], s]``, momentum c_ibar f = -c_i f out of the body).  Eq. 13
    sums incoming minus reflected momentum, so
        F = sum_links c_i (g_i(s) + f_prev_ibar(s)).
    This is exactly the momentum the fluid loses in the step.
    """
    ny, nx = kind.shape
    xs = np.arange(nx)
    F = np.zeros(2)
    for i in range(1, 9):
        src_kind = np.roll(kind, shift=(C[i, 1], C[i, 0]), axis=(0, 1))
        links = (kind == SOLID) & (src_kind == FLUID)
        if not x_periodic:
            src_x = xs - C[i, 0]
            links &= ((src_x >= 0) & (src_x < nx))[None, :]
        s = g[i][links].sum() + f_prev[OPP[i]][links].sum()
        F += C[i].astype(np.float64) * s
    return F


def bounce_back(g, kind):
    """Full-way bounce-back (Eq. 11): every solid node reverses what arrived."""
    solid = kind != FLUID
    out = g.copy()
    out[:, solid] = g[OPP][:, solid]
    return out


# --------------------------------------------------------------------------- #
# Sec. 2.2: Zou & He
# --------------------------------------------------------------------------- #
def zouhe_pressure_east(g, rho_out):
    """Right boundary with prescribed density (Eqs. 5-10) for columns of
    post-stream populations ``g`` (9, n).  The unknowns are 3, 6, 7.

    rho = rho_out; u follows from Eq. 7, u = (rho0 + 2 rho+) / rho - 1; the
    tangential velocity is zero.  f^neq of the known populations is taken
    against f^eq(rho_out, u, 0) of the boundary node itself."""
    rho0 = g[0] + g[2] + g[4]
    rhop = g[1] + g[5] + g[8]
    rho = np.full_like(rho0, rho_out)
    u = (rho0 + 2.0 * rhop) / rho - 1.0
    v = np.zeros_like(u)
    return _zouhe_east_unknowns(g, rho, u, v), (rho, u, v)


def _zouhe_east_unknowns(g, rho, u, v):
    """g3, g6, g7 of Eqs. 8-10 given the boundary state (rho, u, v)."""
    feq = equilibrium(rho, u, v)
    neq = g - feq
    out = g.copy()
    out[3] = feq[3] + neq[1]
    out[6] = feq[6] + neq[8] + 0.5 * (neq[4] - neq[2])
    out[7] = feq[7] + neq[5] - 0.5 * (neq[4] - neq[2])
    return out


def zouhe_velocity_west(g, u, v):
    """Left boundary with prescribed velocity: the mirror image (x -> -x,
    1<->3, 5<->6, 8<->7) of Eqs. 5-10.  Known: 0, 2, 3, 4, 6, 7; unknown 1, 5, 8.
    rho (1 - u) = rho0 + 2 rho-, rho- = f3 + f6 + f7."""
    rho0 = g[0] + g[2] + g[4]
    rhom = g[3] + g[6] + g[7]
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho0.shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho0.shape)
    rho = (rho0 + 2.0 * rhom) / (1.0 - u)
    feq = equilibrium(rho, u, v)
    neq = g - feq
    out = g.copy()
    out[1] = feq[1] + neq[3]
    out[5] = feq[5] + neq[7] + 0.5 * (neq[4] - neq[2])
    out[8] = feq[8] + neq[6] - 0.5 * (neq[4] - neq[2])
    return out


# --------------------------------------------------------------------------- #
# Sec. 3.1: NN direct reconstruction (Eq. 15)
# --------------------------------------------------------------------------- #
NN_POPS = (3, 6, 7)


def nn_features(g, x_b):
    """81 inputs for every row of boundary column ``x_b``: the nine post-stream
    populations of columns x_b-1, x_b-2, x_b-3 at rows y-1, y, y+1 (periodic).
    Index = k * 27 + j * 9 + i for column x_b-1-k, row y-1+j, population i."""
    ny = g.shape[1]
    feats = np.empty((ny, 81))
    ys = np.arange(ny)
    for k in range(3):
        for j in range(3):
            rows = (ys + j - 1) % ny
            for i in range(9):
                feats[:, k * 27 + j * 9 + i] = g[i, rows, x_b - 1 - k]
    return feats


def nn_base_index(i):
    """Feature index of f_i at (x_b - 1, y): the base of the residual in Eq. 15."""
    return 9 + i


@dataclass
class NNOutflow:
    net: "_mlp.MLP"
    fallback_drho: float = 0.05


def nn_reconstruct_east(g_col, feats, net, rho_out, fallback_drho):
    """Eq. 15 at the right boundary: g_i(L) = f_i(L-1) + s_i for i = 3, 6, 7,
    s = net(feats).  A node falls back to Zou & He (rho_out) if an output is
    non-finite, a rebuilt population is negative, or its density leaves
    rho_out by more than ``fallback_drho``.  Returns (columns, fallback mask)."""
    s = net.predict(feats)                       # (ny, 3), already scaled
    out = g_col.copy()
    for n, i in enumerate(NN_POPS):
        out[i] = feats[:, nn_base_index(i)] + s[:, n]
    rho = out.sum(axis=0)
    bad = ~np.all(np.isfinite(s), axis=1)
    bad |= (out[3] < 0) | (out[6] < 0) | (out[7] < 0)
    bad |= ~(np.abs(rho - rho_out) <= fallback_drho)
    zh, _ = zouhe_pressure_east(g_col, rho_out)
    out[:, bad] = zh[:, bad]
    return out, bad


# --------------------------------------------------------------------------- #
# Whole-domain solver
# --------------------------------------------------------------------------- #
@dataclass
class Config:
    nx: int
    ny: int
    tau: float
    collision: str = "bgk"                 # "bgk" | "mrt"
    mrt_rates: Optional[np.ndarray] = None  # None -> mrt_default_rates(tau)
    x_periodic: bool = False               # True: no open boundaries at all
    u_in: float = 0.0                      # inlet velocity (Zou & He, west)
    u_ramp_steps: int = 0                  # > 0: inlet velocity u_in min(1, (t+1)/ramp)
    v_pert_amp: float = 0.0                # amplitude of the seeded inlet v
    seed: int = 0
    rho_out: float = 1.0
    outflow: str = "zouhe"                 # "zouhe" | "nn" | "cbc"
    nn: Optional[NNOutflow] = None
    cbc: Optional[object] = None           # oracle.cbc.CBCOutflow


class Solver:
    """Whole-domain FP64 solver.  ``f`` holds the post-collision populations
    f*(t) (solid nodes hold what bounce-back stored there)."""

    def __init__(self, cfg: Config, kind: np.ndarray):
        self.cfg = cfg
        self.kind = np.asarray(kind, dtype=np.uint8)
        assert self.kind.shape == (cfg.ny, cfg.nx)
        self.f = equilibrium(np.ones((cfg.ny, cfg.nx)), np.zeros((cfg.ny, cfg.nx)),
                             np.zeros((cfg.ny, cfg.nx)))
        self.t = 0
        self.forces = []          # (Fx, Fy) per step
        self.nn_fallbacks = 0
        self.cbc_state = None
        self.capture = None       # (x_t, every) of the data-set capture, or None
        self.captured = []        # captured blocks of rows, (ny, 84) each

    def capture_plane(self, x_t, every):
        """Record training rows of Sec. 3.1 at column ``x_t``: during every step
        t -> t+1 with (t+1) % every == 0, after streaming, bounce-back and the
        open boundaries and before collision, one row per lattice row y (in
        order): the 81 inputs of Eq. 15 taken as if x_t were the outflow
        column (``nn_features(g, x_t)``) followed by the post-stream
        f_3, f_6, f_7 at (x_t, y), the values the network learns to rebuild."""
        self.capture = (int(x_t), int(every))
        self.captured = []

    def snapshot_rows(self, x_begin, x_end):
        """Training rows of Sec. 3.1 from the current state alone (one
        converged snapshot, each column a batch): for every column x in
        [x_begin, x_end) the ny rows that ``capture_plane(x, ...)`` records
        during the next step -- the pull of the stored post-collision state
        with bounce-back at solid nodes (columns 4..nx-2 never touch the open
        boundaries) -- stacked column by column, float64 (n, 84)."""
        g = bounce_back(stream_pull(self.f), self.kind)
        out = [np.hstack([nn_features(g, x), g[list(NN_POPS), :, x].T])
               for x in range(x_begin, x_end)]
        return np.vstack(out)

    def dataset(self):
        """All captured rows, float64 (n, 84), in capture order."""
        if not self.captured:
            return np.zeros((0, 84))
        return np.vstack(self.captured)

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        shape = (self.cfg.ny, self.cfg.nx)
        rho = np.ones(shape) if rho is None else np.asarray(rho, dtype=np.float64)
        ux = np.zeros(shape) if ux is None else np.asarray(ux, dtype=np.float64)
        uy = np.zeros(shape) if uy is None else np.asarray(uy, dtype=np.float64)
        self.f = equilibrium(rho, ux, uy)
        self.t = 0
        self.forces = []
        self.cbc_state = None

    # the collision operator configured for this run
    def collide(self, g):
        if self.cfg.collision == "bgk":
            return collide_bgk(g, self.cfg.tau)
        rates = self.cfg.mrt_rates
        if rates is None:
            rates = mrt_default_rates(self.cfg.tau)
        return collide_mrt(g, rates)

    def step(self, n=1):
        for _ in range(n):
            self._step()

    def _step(self):
        cfg, kind = self.cfg, self.kind
        f = self.f
        fluid = kind == FLUID
        g = stream_pull(f)                                            # Eq. 1
        F = momentum_exchange(f, g, kind, cfg.x_periodic)            # Eqs. 13-14
        g = bounce_back(g, kind)                                      # Eq. 11
        if not cfg.x_periodic:
            # inlet (column 0): Zou & He velocity with the seeded perturbation
            v = np.asarray(_rng.inlet_perturbation(cfg.seed, self.t, cfg.ny,
                                                   cfg.v_pert_amp))
            u = cfg.u_in
            if cfg.u_ramp_steps > 0:
                u = cfg.u_in * min(1.0, (self.t + 1) / cfg.u_ramp_steps)
            col = zouhe_velocity_west(g[:, :, 0], u, v)
            m = fluid[:, 0]
            g[:, m, 0] = col[:, m]
            # outflow (column nx-1)
            xb = cfg.nx - 1
            m = fluid[:, xb]
            if cfg.outflow == "zouhe":
                col, _ = zouhe_pressure_east(g[:, :, xb], cfg.rho_out)
            elif cfg.outflow == "nn":
                feats = nn_features(g, xb)
                col, bad = nn_reconstruct_east(g[:, :, xb], feats, cfg.nn.net,
                                               cfg.rho_out, cfg.nn.fallback_drho)
                self.nn_fallbacks += int(np.count_nonzero(bad & m))
            elif cfg.outflow == "cbc":
                from . import cbc as _cbc
                col, self.cbc_state = _cbc.cbc_east(self, f, g)
            else:
                raise ValueError(cfg.outflow)
            g[:, m, xb] = col[:, m]
        if self.capture is not None and (self.t + 1) % self.capture[1] == 0:
            x_t = self.capture[0]
            self.captured.append(np.hstack([nn_features(g, x_t), g[list(NN_POPS), :, x_t].T]))
        post = self.collide(g)                                        # Eq. 2 / MRT
        g[:, fluid] = post[:, fluid]
        self.f = g
        self.t += 1
        self.forces.append(F)

    # diagnostics
    def fields(self):
        return moments(self.f)

    def mass(self):
        """Sum of every population on every node (fluid and solid)."""
        return float(self.f.sum())

    def fluid_momentum(self):
        fl = self.kind == FLUID
        jx = np.tensordot(C[:, 0].astype(np.float64), self.f, axes=(0, 0))
        jy = np.tensordot(C[:, 1].astype(np.float64), self.f, axes=(0, 0))
        return np.array([jx[fl].sum(), jy[fl].sum()])

    def force_series(self):
        return np.array(self.forces).reshape(-1, 2)


def tau_from_re(u, length, re):
    """tau from Re = u L / nu and nu = c_s^2 (tau - 1/2)."""
    nu = u * length / re
    return nu / CS2 + 0.5
