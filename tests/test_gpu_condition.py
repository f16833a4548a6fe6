"""Per-stencil condition numbers (Section 2.1) through the C ABI against the
oracle."""
import numpy as np
import pytest

from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import make_plan

pytestmark = pytest.mark.gpu


def _check(ns, m):
    n = ow.stencil_size(ns.dim, m)
    plan, code, _ = make_plan(ns, m=m)
    kap = plan.condition().cpu().numpy()
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, n, normals=ns.normals)
    ref = ow.condition_numbers(ns.coords, st, m)
    for grp in ("mon", "rbf"):
        nodes = st[grp + "_nodes"]
        if len(nodes):
            # systems singular to working precision have no meaningful kappa:
            # both sides must only agree that it is huge
            ok = ref[grp] < 1e12
            rel = np.abs(kap[nodes][ok] / ref[grp][ok] - 1.0)
            assert rel.max() <= 1e-8, (grp, rel.max())
            assert np.all(kap[nodes][~ok] > 1e12)
    plan.close()
    return kap, st


def test_condition_2d_and_3d():
    kap, st = _check(nodesets.square_wall_band(n=30), 2)
    # RBF-FD systems are worse conditioned than MON ones (Section 2.1)
    assert np.median(kap[st["rbf_nodes"]]) > 10 * np.median(kap[st["mon_nodes"]])
    _check(nodesets.cube_spheres(n=14, n_holes=2, r_range=(0.1, 0.15), band=0.12, seed=nodesets.SEED_BASE + 21), 2)
    # a coarser 3D set with one system singular to working precision
    _check(nodesets.cube_spheres(n=10, n_holes=1, r_range=(0.1, 0.15), band=0.12, seed=7), 2)


def test_lattice_mon_closed_form():
    ns = nodesets.square_quarters(n=20, layout="regular")
    kap, st = _check(ns, 2)
    assert np.allclose(kap[st["mon_nodes"]], (7 + np.sqrt(41)) / (2 * np.sqrt(2)), rtol=1e-12)
