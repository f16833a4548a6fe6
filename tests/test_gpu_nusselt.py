"""Wall-flux reduction (average Nusselt number, Section 4.1) through the C
ABI against the oracle, on the de Vahl Davis quarter layouts."""
import numpy as np
import pytest

from oracle import apply as oap
from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets

from gpu_helpers import make_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", ["hybrid", "scattered", "regular"])
def test_wall_flux_matches_the_oracle(layout):
    import torch

    ns = nodesets.square_quarters(n=40, layout=layout)
    plan, code, _ = make_plan(ns, m=2)
    assert code == 0
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    cold = np.flatnonzero((ns.is_boundary == 1) & (ns.coords[0] == 0.0))
    rng = np.random.default_rng(4)
    x, y = ns.coords
    fields = [x - 0.5, np.sin(3 * x) * np.cos(2 * y) + rng.uniform(-1e-3, 1e-3, ns.N)]
    nrm = plan._dev["normals"]
    nodes = torch.from_numpy(cold.astype(np.int32)).cuda()
    for T in fields:
        Td = torch.from_numpy(T).cuda()
        got = float(plan.wall_flux_mean(Td, nodes, nrm, scale=1.0).item())
        ref = oap.wall_flux_mean(ns.N, st, W, T, cold, ns.normals, scale=1.0)
        assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref))
        # fixed summation order: the same bits every call
        again = float(plan.wall_flux_mean(Td, nodes, nrm, scale=1.0).item())
        assert again == got
    plan.close()


def test_wall_flux_rejects_node_ids_out_of_range():
    """Node ids outside [0, N), forged on the host, are not followed: the
    result is NaN, and the same call with the valid ids alone is unchanged."""
    import torch

    ns = nodesets.square_quarters(n=40, layout="hybrid")
    plan, code, _ = make_plan(ns, m=2)
    assert code == 0
    cold = np.flatnonzero((ns.is_boundary == 1) & (ns.coords[0] == 0.0)).astype(np.int32)
    Td = torch.from_numpy(ns.coords[0] - 0.5).cuda()
    nrm = plan._dev["normals"]
    good = float(plan.wall_flux_mean(Td, torch.from_numpy(cold).cuda(), nrm, scale=1.0).item())
    assert np.isfinite(good)
    for bad_id in (-1, ns.N, np.iinfo(np.int32).max, np.iinfo(np.int32).min):
        forged = cold.copy()
        forged[len(forged) // 2] = bad_id
        got = float(plan.wall_flux_mean(Td, torch.from_numpy(forged).cuda(), nrm, scale=1.0).item())
        assert np.isnan(got), bad_id
    again = float(plan.wall_flux_mean(Td, torch.from_numpy(cold).cuda(), nrm, scale=1.0).item())
    assert again == good
    plan.close()
