"""Pins for the oracle's explicit Boussinesq step (Section 3, Eqs. 2-4)."""
import json
import os

import numpy as np

from oracle import stencils as ost
from oracle import weights as ow
from oracle import stepper as ostep
from paper_2303_01760_gb300 import nodesets

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_values.json")))


def _setup(ns, Ra, Pr, dt=None, m=2):
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, ow.stencil_size(ns.dim, m),
                            normals=ns.normals)
    W = ow.all_weights(ns.coords, st, m)
    dt = ostep.dt_rule(ns.h) if dt is None else dt
    return ostep.Stepper(ns.coords, ns.bc, ns.T_bc, ns.normals, ns.T_ref, st, W, Ra, Pr, dt)


def test_dt_rule_matches_paper_3d_value():
    g = PAPER["dt_3d"]
    assert abs(ostep.dt_rule(g["h"]) - g["value"]) <= 1e-18


def test_linear_conduction_is_a_fixed_point():
    """Ra = 0, v = 0, T = x - 0.5: satisfies the dVD walls (Section 4.1) and has
    zero Laplacian, and both bases reproduce linear fields exactly."""
    ns = nodesets.square_wall_band(n=20)
    S = _setup(ns, Ra=0.0, Pr=0.71)
    v = np.zeros((2, ns.N))
    T = ns.coords[0] - 0.5
    v2, T2, _ = S.run(v, T.copy(), 30)
    assert np.abs(T2 - T).max() <= 1e-12
    assert np.abs(v2).max() <= 1e-12


def test_heat_equation_decay_with_insulated_walls():
    """Ra = 0 and v = 0 reduce Eq. 4 to dT/dt = lap T; with all walls insulated
    T = exp(-pi^2 t) cos(pi x) is exact, and explicit Euler with dt = 0.1 h^2/2
    must follow it to discretisation accuracy."""
    ns = nodesets.square_wall_band(n=40)
    ns.bc[:] = np.where(ns.is_boundary == 1, nodesets.BC_T_NEUMANN, nodesets.BC_INTERIOR)
    S = _setup(ns, Ra=0.0, Pr=0.71)
    T0 = np.cos(np.pi * ns.coords[0])
    steps = 400
    _, T, _ = S.run(np.zeros((2, ns.N)), T0.copy(), steps)
    exact = np.exp(-np.pi ** 2 * steps * S.dt) * T0
    assert np.abs(T - exact).max() <= 3e-3
    # and it did decay by the expected factor (a wrong sign grows instead)
    assert abs(T[np.argmax(T0)] / T0.max() - np.exp(-np.pi ** 2 * steps * S.dt)) < 3e-3


def test_predictor_terms_against_analytic_fields():
    """Step 1 of the projection: (v* - v)/dt = -(v.grad)v + Pr lap v +
    Ra Pr (T - T_ref) e_y, checked at interior nodes with closed-form
    derivatives of smooth fields (discretisation error O(h^2))."""
    ns = nodesets.square_wall_band(n=80, wall_band=0.0)
    S = _setup(ns, Ra=100.0, Pr=0.71)
    x, y = ns.coords
    pi = np.pi
    v = np.stack([np.sin(pi * x) * np.sin(pi * y), np.cos(pi * x) * np.sin(2 * pi * y)])
    T = x * y
    vs = S.predictor(v, T)
    # analytic right-hand side
    u, w = v
    ux, uy = pi * np.cos(pi * x) * np.sin(pi * y), pi * np.sin(pi * x) * np.cos(pi * y)
    wx, wy = -pi * np.sin(pi * x) * np.sin(2 * pi * y), 2 * pi * np.cos(pi * x) * np.cos(2 * pi * y)
    lap_u = -2 * pi ** 2 * u
    lap_w = -5 * pi ** 2 * w
    rhs_u = -(u * ux + w * uy) + 0.71 * lap_u
    rhs_w = -(u * wx + w * wy) + 0.71 * lap_w + 100.0 * 0.71 * (T - ns.T_ref)
    inner = ns.bc == 0
    got_u = (vs[0] - u) / S.dt
    got_w = (vs[1] - w) / S.dt
    sel = inner & (np.minimum(ns.coords, 1 - ns.coords).min(0) > 0.05)
    assert np.abs(got_u[sel] - rhs_u[sel]).max() <= 2e-2 * np.abs(rhs_u).max()
    assert np.abs(got_w[sel] - rhs_w[sel]).max() <= 2e-2 * np.abs(rhs_w).max()
    assert np.all(vs[:, ~inner] == 0.0)


def test_pressure_solve_recovers_neumann_compatible_field():
    """Step 2: with rhs = lap p_true inside and 0 on the walls, where
    p_true = cos(pi x) cos(pi y) has zero normal derivative on the box, the
    bordered solve returns p_true up to its mean, with error falling as h^2."""
    errs = []
    for n in (20, 40):
        ns = nodesets.square_wall_band(n=n)
        S = _setup(ns, Ra=0.0, Pr=0.71)
        x, y = ns.coords
        pt = np.cos(np.pi * x) * np.cos(np.pi * y)
        rhs = np.where(ns.bc == 0, -2 * np.pi ** 2 * pt, 0.0)
        p = S.solve_pressure(rhs)
        assert abs(p.sum()) <= 1e-9 * np.abs(p).sum()
        errs.append(np.abs((p - p.mean()) - (pt - pt.mean())).max())
    assert errs[1] < errs[0] / 2.5, errs
    assert errs[1] < 2e-2


def test_temperature_update_against_analytic_fields():
    """Steps 4-5: (T_new - T)/dt = -v_new . grad T + lap T inside; Dirichlet
    nodes take T_bc; insulated nodes satisfy their own n.grad T row."""
    ns = nodesets.square_wall_band(n=60)
    S = _setup(ns, Ra=0.0, Pr=0.71)
    x, y = ns.coords
    pi = np.pi
    v = np.stack([np.sin(pi * x) * np.sin(pi * y), 0.5 * np.sin(pi * x) ** 2 * np.sin(2 * pi * y)])
    T = np.sin(pi * x) * np.cos(pi * y) + x
    Tn = S.temperature(v, T.copy())
    Tx = pi * np.cos(pi * x) * np.cos(pi * y) + 1.0
    Ty = -pi * np.sin(pi * x) * np.sin(pi * y)
    lapT = -2 * pi ** 2 * np.sin(pi * x) * np.cos(pi * y)
    ref = -(v[0] * Tx + v[1] * Ty) + lapT
    inner = ns.bc == 0
    depth = np.minimum(ns.coords, 1 - ns.coords).min(0)
    got = (Tn - T) / S.dt
    # regular (MON) region: second-order accurate
    sel = inner & (depth > 0.12)
    assert np.abs(got[sel] - ref[sel]).max() <= 2e-2 * np.abs(ref).max()
    # scattered band (RBF-FD, m = 2: first-order Laplacian)
    sel = inner & (depth <= 0.12) & (depth > 0.04)
    assert np.abs(got[sel] - ref[sel]).max() <= 1.5e-1 * np.abs(ref).max()
    assert np.all(Tn[ns.bc == 1] == ns.T_bc[ns.bc == 1])
    neu = np.flatnonzero(ns.bc == 2)
    # boundary stencils hold only the node and interior nodes, so every
    # insulated row n.grad T = 0 holds exactly after the update
    resid = S.Dn[neu] @ Tn
    scale = np.abs(S.Dn[neu]).sum(1).A1 * np.abs(Tn).max()
    assert np.all(np.abs(resid) <= 1e-12 * scale)


def test_buoyancy_drives_flow_up_the_hot_wall():
    """de Vahl Davis set-up (Section 4.1): hot right wall, cold left wall; the
    Boussinesq term must make the fluid rise along the hot wall and sink along
    the cold one."""
    ns = nodesets.square_wall_band(n=20)
    S = _setup(ns, Ra=1e5, Pr=0.71)
    v, T = ostep.initial_state(2, ns.N, ns.bc, ns.T_bc)
    v, T, _ = S.run(v, T, 300)
    x, y = ns.coords
    mid = (y > 0.3) & (y < 0.7)
    assert v[1, mid & (x > 0.8)].mean() > 0
    assert v[1, mid & (x < 0.2)].mean() < 0
    # heat has entered from the hot wall and left through the cold one
    assert T[(x > 0.85) & (ns.bc == 0)].mean() > 0.0
    assert T[(x < 0.15) & (ns.bc == 0)].mean() < 0.0


def test_projection_removes_divergence():
    """Steps 2-3 (Chorin): the corrected velocity v* - dt grad p is close to
    divergence free; with a wrong scale on the pressure right-hand side the
    divergence of v* survives."""
    ns = nodesets.square_wall_band(n=60, wall_band=0.0)
    S = _setup(ns, Ra=0.0, Pr=0.71)
    x, y = ns.coords
    pi = np.pi
    vstar = np.stack([np.sin(pi * x) ** 2 * np.sin(pi * y), np.sin(pi * x) * np.sin(pi * y) ** 2])
    vstar[:, ns.bc != 0] = 0.0
    p = S.solve_pressure(S.pressure_rhs(vstar))
    v1 = S.correct(vstar, p)
    div0 = S.D[0] @ vstar[0] + S.D[1] @ vstar[1]
    div1 = S.D[0] @ v1[0] + S.D[1] @ v1[1]
    sel = (ns.bc == 0) & (np.minimum(ns.coords, 1 - ns.coords).min(0) > 0.1)
    assert np.abs(div1[sel]).max() <= 0.05 * np.abs(div0[sel]).max()
