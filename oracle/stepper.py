"""Explicit Boussinesq natural-convection step, FP64.  Test infrastructure only.

Section 3: Eqs. 2-4 (continuity, momentum with the Boussinesq buoyancy term
-Ra Pr g T_delta, heat transfer) in dimensionless form, explicit Euler in time,
velocity updated first with the previous-step temperature, pressure-velocity
coupling by Chorin's projection, and dt = 0.1 h^2 / 2.

One step, in the order the paper states it (rho = 1):
  1. v* = v + dt [ -(v . grad) v + Pr lap v + Ra Pr (T - T_ref) e_up ]
     on interior nodes; v* = 0 on boundary nodes (no-slip).
  2. Pressure: lap p = (1/dt) div v* on interior rows, n . grad p = 0 on
     boundary rows, and the constant null space fixed by the bordered system
         [ L  1 ] [ p ]   [ rhs ]
         [ 1' 0 ] [ c ] = [  0  ].
  3. v_new = v* - dt grad p on interior nodes, 0 on boundary nodes.
  4. T_new = T + dt [ -v_new . grad T + lap T ] on interior nodes (the new
     velocity advects the temperature).
  5. Temperature boundary conditions: Dirichlet nodes take T_bc; insulated
     (Neumann) nodes solve their own n . grad T = 0 row for the centre value,
     T_b = -sum_{i != b} wn_i T_i / wn_b, with every other node's value taken
     after step 4 (Neumann neighbours keep their previous value).

Readings where the paper is silent: gravity g = -e_up with e_up the last axis
(y in 2D, z in 3D), so the buoyancy term is +Ra Pr (T - T_ref) e_up; plain
central (un-upwinded) derivative weights for advection; Neumann pressure on all
walls; the bordered system above for the pressure null space (solved here by a
sparse LU factored once, which gives the exact discrete solution).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import apply as oapply

BC_INTERIOR = 0
BC_T_DIRICHLET = 1
BC_T_NEUMANN = 2


class Stepper:
    def __init__(self, coords, bc, T_bc, normals, T_ref, st, W, Ra, Pr, dt):
        self.dim, self.N = coords.shape
        dim, N = self.dim, self.N
        self.ops = ["dx", "dy", "dz"][:dim]
        self.D = [oapply.to_csr(N, st, W, op) for op in self.ops]
        self.L = oapply.to_csr(N, st, W, "lap")
        self.bc = np.asarray(bc)
        self.inner = self.bc == BC_INTERIOR
        self.bnd = ~self.inner
        self.dir = self.bc == BC_T_DIRICHLET
        self.neu = self.bc == BC_T_NEUMANN
        self.T_bc = np.asarray(T_bc, dtype=np.float64)
        self.T_ref = float(T_ref)
        self.Ra, self.Pr, self.dt = float(Ra), float(Pr), float(dt)
        # normal-derivative operator rows of boundary nodes
        Dn = sp.csr_matrix((N, N))
        for k in range(dim):
            Dn = Dn + sp.diags(normals[k]) @ self.D[k]
        self.Dn = Dn.tocsr()
        # pressure operator: Laplacian rows inside, normal-derivative rows on the boundary
        Lp = sp.diags(self.inner.astype(float)) @ self.L + sp.diags(self.bnd.astype(float)) @ self.Dn
        ones = np.ones((N, 1))
        Bm = sp.bmat([[Lp, sp.csr_matrix(ones)], [sp.csr_matrix(ones.T), None]], format="csc")
        self.lu = spla.splu(Bm)
        self.Lp = Lp.tocsr()
        # Neumann temperature rows: diagonal entry and off-diagonal part
        self.neu_ids = np.flatnonzero(self.neu)
        Dn_neu = self.Dn[self.neu_ids]
        self.wn_diag = np.asarray(Dn_neu[np.arange(len(self.neu_ids)), self.neu_ids]).ravel()
        off = Dn_neu.tolil()
        off[np.arange(len(self.neu_ids)), self.neu_ids] = 0.0
        self.Dn_off = off.tocsr()
        self.last_c = 0.0

    def pressure_rhs(self, vstar):
        div = np.zeros(self.N)
        for k in range(self.dim):
            div = div + self.D[k] @ vstar[k]
        return np.where(self.inner, div / self.dt, 0.0)

    def solve_pressure(self, rhs):
        sol = self.lu.solve(np.r_[rhs, 0.0])
        self.last_c = sol[-1]
        return sol[:-1]

    def predictor(self, v, T):
        """Step 1: v* (boundary rows zero)."""
        dim, dt = self.dim, self.dt
        vstar = np.zeros_like(v)
        for k in range(dim):
            adv = np.zeros(self.N)
            for j in range(dim):
                adv = adv + v[j] * (self.D[j] @ v[k])
            force = -adv + self.Pr * (self.L @ v[k])
            if k == dim - 1:
                force = force + self.Ra * self.Pr * (T - self.T_ref)
            vstar[k] = np.where(self.inner, v[k] + dt * force, 0.0)
        return vstar

    def correct(self, vstar, p):
        """Step 3: v_new = v* - dt grad p inside, 0 on the boundary."""
        vnew = np.zeros_like(vstar)
        for k in range(self.dim):
            vnew[k] = np.where(self.inner, vstar[k] - self.dt * (self.D[k] @ p), 0.0)
        return vnew

    def temperature(self, vnew, T):
        """Steps 4 and 5."""
        adv = np.zeros(self.N)
        for k in range(self.dim):
            adv = adv + vnew[k] * (self.D[k] @ T)
        Tn = np.where(self.inner, T + self.dt * (-adv + self.L @ T), T)
        Tn = np.where(self.dir, self.T_bc, Tn)
        if len(self.neu_ids):
            Tn[self.neu_ids] = -(self.Dn_off @ Tn) / self.wn_diag
        return Tn

    def step(self, v, T):
        """One step. v [dim, N], T [N] -> (v_new, T_new, p)."""
        vstar = self.predictor(v, T)
        p = self.solve_pressure(self.pressure_rhs(vstar))
        vnew = self.correct(vstar, p)
        return vnew, self.temperature(vnew, T), p

    def run(self, v, T, n_steps):
        p = np.zeros(self.N)
        for _ in range(n_steps):
            v, T, p = self.step(v, T)
        return v, T, p


def initial_state(dim, N, bc, T_bc, T_init=0.0):
    """v = 0, T = T_init inside with Dirichlet values applied (Section 4)."""
    v = np.zeros((dim, N))
    T = np.full(N, float(T_init))
    T = np.where(np.asarray(bc) == BC_T_DIRICHLET, T_bc, T)
    return v, T


def dt_rule(h):
    """dt = 0.1 h^2 / 2 (Section 3)."""
    return 0.1 * h * h / 2.0
