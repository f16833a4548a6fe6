"""Oracle pins of the wall-flux reduction (the average Nusselt number of
Section 4.1): closed forms that the first-derivative weights reproduce
exactly (monomials of degree <= m)."""
import numpy as np

from oracle import apply as oap
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets


def _setup(layout="hybrid", n=24):
    ns = nodesets.square_quarters(n=n, layout=layout)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    cold = np.flatnonzero((ns.is_boundary == 1) & (ns.coords[0] == 0.0))
    return ns, st, W, cold


def test_conduction_profile_gives_nusselt_one():
    """T = x - 1/2 (pure conduction between T_C = -1/2 and T_H = 1/2): the
    normal derivative on the cold wall is -1 everywhere, so Nu = 1."""
    for layout in ("hybrid", "scattered", "regular"):
        ns, st, W, cold = _setup(layout)
        assert len(cold) > 10
        T = ns.coords[0] - 0.5
        nu = oap.wall_flux_mean(ns.N, st, W, T, cold, ns.normals, scale=1.0)
        assert abs(nu - 1.0) <= 1e-11


def test_quadratic_field_and_scale():
    """T = (x - 1/2)^2 + 3y: on x = 0 the gradient is (-1, 3) and the outward
    normal (-1, 0), so |n . grad T| = 1; the scale L/(T_H - T_C) multiplies."""
    ns, st, W, cold = _setup()
    x, y = ns.coords
    T = (x - 0.5) ** 2 + 3.0 * y
    assert abs(oap.wall_flux_mean(ns.N, st, W, T, cold, ns.normals, scale=2.5) - 2.5) <= 1e-10


def test_flux_is_absolute_and_uses_the_normal():
    """T = 2 - x: n . grad T = +1 on the cold wall; a field varying only along
    the wall (T = y) has no normal flux."""
    ns, st, W, cold = _setup()
    x, y = ns.coords
    assert abs(oap.wall_flux_mean(ns.N, st, W, 2.0 - x, cold, ns.normals) - 1.0) <= 1e-11
    assert abs(oap.wall_flux_mean(ns.N, st, W, y, cold, ns.normals)) <= 1e-11


def test_quarters_layout():
    """Hybrid quarters: bottom-left and top-right scattered, the other two
    regular; the regular-only set has every interior node on the lattice."""
    ns = nodesets.square_quarters(n=40, layout="hybrid")
    x, y = ns.coords
    interior = ns.is_boundary == 0
    reg = ns.is_regular == 1
    # regular nodes only in the top-left and bottom-right quarters (up to the
    # lattice nodes kept on the quarter lines)
    assert np.all(~reg | ((x <= 0.5) & (y >= 0.5)) | ((x >= 0.5) & (y <= 0.5)))
    assert np.any(interior & ~reg & (x < 0.5) & (y < 0.5))
    assert np.any(interior & ~reg & (x > 0.5) & (y > 0.5))
    r = nodesets.square_quarters(n=40, layout="regular")
    assert np.all(r.is_regular[r.is_boundary == 0] == 1)
    assert r.N == 41 * 41 - 4
