"""Stencil validation and check mode (a debugging aid; the paper has no
counterpart).  A bad stencil index is forged from the host with the
library's test hook, which turns check mode on before it writes, so no
kernel ever gathers through the bad index: the validation scan reads only
the index tables themselves."""
import numpy as np
import pytest

from paper_2303_01760_gb300 import nodesets

from gpu_helpers import make_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("arrange", [0, 2])
def test_validation_and_check_mode_on_a_forged_index(arrange):
    """arrange 2: the weights are solved inside the build; a forgery after the
    build must still be caught by the weights call's gate."""
    import torch
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.square_holes(n=100)
    plan, code, _ = make_plan(ns, m=2)
    assert code == 0
    if arrange:
        plan.set_tuning(knn_qt=1, rbf_lanes=8, rbf_lanes32=8, apply_threads=256, arrange=arrange, chunks=1)
        plan.build_stencils()
        assert plan.compute_weights(hsm.HSM_PREC_FP64) == 0
    assert plan.validate() == hsm.HSM_OK
    u = torch.from_numpy(nodesets.field_sincos(ns.coords)[0]).cuda()
    ref = plan.apply(u).clone()
    # check mode on valid tables changes nothing
    plan.set_checks(True)
    assert torch.equal(plan.apply(u), ref)

    plan.inject_stencil_fault()
    assert plan.validate() == hsm.HSM_EBOUNDS
    assert "RBF-FD stencil indices" in hsm.last_error(plan.h)
    out = torch.full_like(ref, 7.0)
    with pytest.raises(hsm.HsmError) as e:
        plan.apply(u, out=out)
    assert e.value.code == hsm.HSM_EBOUNDS
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))  # refused before any gather: out untouched
    for call in (lambda: plan.compute_weights(hsm.HSM_PREC_FP64), lambda: plan.condition()):
        with pytest.raises(hsm.HsmError) as e:
            call()
        assert e.value.code == hsm.HSM_EBOUNDS

    # a rebuild gives valid tables, and the same operator values as before
    plan.build_stencils()
    assert plan.validate() == hsm.HSM_OK
    plan.compute_weights(hsm.HSM_PREC_FP64)
    assert torch.equal(plan.apply(u), ref)
    plan.set_checks(False)
    assert torch.equal(plan.apply(u), ref)
    plan.close()


def test_inject_needs_built_stencils():
    import torch
    from paper_2303_01760_gb300 import hsm

    ns = nodesets.square_wall_band(n=20)
    d = torch.device("cuda:0")
    c = torch.from_numpy(np.ascontiguousarray(ns.coords)).to(d)
    r = torch.from_numpy(np.ascontiguousarray(ns.is_regular)).to(d)
    b = torch.from_numpy(np.ascontiguousarray(ns.is_boundary)).to(d)
    plan = hsm.Plan(c, r, b, ns.h, m=2)
    with pytest.raises(hsm.HsmError) as e:
        plan.inject_stencil_fault()
    assert e.value.code == hsm.HSM_ESTATE
    assert plan.validate() == hsm.HSM_ESTATE
    assert hsm.lib.hsm_plan_set_checks(plan.h, 2) == hsm.HSM_EINVAL
    plan.close()
