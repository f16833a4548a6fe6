"""Plans are independent: two host threads, each driving its own plan on its
own stream (the way a caller streams node sets), get the same stencils,
weights and operator values as one thread driving the plans in turn."""
import threading

import numpy as np
import pytest

from paper_2303_01760_gb300 import nodesets

pytestmark = pytest.mark.gpu


def _sets():
    return [nodesets.square_holes(n=200), nodesets.cube_spheres(n=24)]


def _cycle(hsm, plan, u, out, reps):
    """Build, weigh and apply `reps` times; the outputs of every pass."""
    import torch

    got = []
    for _ in range(reps):
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64)
        plan.apply(u, out=out)
        got.append(out.clone())
    torch.cuda.current_stream().synchronize()
    return got


def test_two_threads_two_plans_match_one_thread():
    import torch
    from paper_2303_01760_gb300 import hsm

    d = torch.device("cuda:0")
    sets = _sets()
    streams = [torch.cuda.Stream(d) for _ in sets]
    plans, us, outs = [], [], []
    for ns, s in zip(sets, streams):
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(d)
             for k in ("coords", "is_regular", "is_boundary", "normals")}
        plans.append(hsm.Plan(t["coords"], t["is_regular"], t["is_boundary"], ns.h, m=2, normals=t["normals"],
                              stream=s))
        plans[-1]._t = t
        us.append(torch.from_numpy(nodesets.field_sincos(ns.coords)[0]).to(d))
        outs.append(torch.empty((ns.dim + 1, ns.N), dtype=torch.float64, device=d))
    torch.cuda.synchronize()

    ref = []
    for i, s in enumerate(streams):
        with torch.cuda.stream(s):
            ref.append(_cycle(hsm, plans[i], us[i], outs[i], 1)[0])

    got, errors = [None, None], []

    def worker(i):
        try:
            torch.cuda.set_device(d)
            with torch.cuda.stream(streams[i]):
                got[i] = _cycle(hsm, plans[i], us[i], outs[i], 6)
        except Exception as exc:
            errors.append(exc)

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for i in range(2):
        for g in got[i]:
            assert torch.equal(g, ref[i])
    for p in plans:
        p.close()
