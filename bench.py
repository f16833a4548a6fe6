"""Benchmark of the hybrid scattered-regular operators on one GB300.

Metric: hybrid operator nodes/s (weights + apply) on the 2D irregular
workload (unit square minus 8 seeded circular holes, lattice h = 0.002,
scattered nodes within 0.05 of a hole, PHS r^3 + monomials m = 2, n = 12,
FP64 weights, operators d/dx, d/dy and the Laplacian).  One step is one pass
of the operator path on that node set: stencil build (lattice + kNN), MON and
RBF-FD weight solves, and one fused application of all operators to
u = sin(pi x) cos(pi y); value = nodes / step time.  The same node set with
every node forced to RBF-FD is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (test infrastructure; plain FP64
numpy/scipy) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid operator nodes/s (weights+apply) vs all-RBF-FD, same GPU, at L-inf tol"
UNIT = "nodes/s"
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2070e6  # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock
L2_FLUSH_BYTES = 512 << 20


def workload_desc(ns):
    return {
        "workload": "2D irregular domain: unit square minus 8 seeded circular holes (r 0.03-0.08), "
                    "lattice h=0.002, scattered within 0.05 of a hole, PHS r^3 + monomials m=2 (n=12), "
                    "FP64 weights, ops dx,dy,lap",
        "nodes": int(ns.N),
        "scattered_fraction": round(ns.n_scattered / ns.N, 4),
        "l2": "flushed (512 MiB write) before every timed step",
        "seed": 20230302,
    }


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def rbf_flops(n, m, nops, dim=2):
    """Algorithmic FP64 flops of one RBF-FD system (n nodes, m monomials, nops
    right-hand sides; dim + 1 operators: the first derivatives and the
    Laplacian), assembly included.
    Assembly: offsets and their scaling (2 n dim), pair values r^3 (dim
    subtractions, dim products, dim - 1 sums, a root and a product per pair),
    monomials of degree >= 2 (one product each per node), the RHS (2 products
    per node for each first derivative, 1 for the Laplacian) and the unscaling
    of the weights (n nops).
    Solve, by the null-space method of the FP64 kernel, r = n - m: LU of P with
    row pivoting, U^T and L1^T triangular solves, [A Z | b], [Z^T A Z | Z^T b],
    the r x r LU with its substitutions, and w = w_t - X y."""

    higher = m - 1 - dim  # monomials of degree >= 2
    asm = (2 * n * dim + n * (n - 1) // 2 * (3 * dim + 1) + n * max(higher, 0)
           + n * (2 * (nops - 1) + 1) + n * nops)
    r = n - m
    lu_p = sum((n - k - 1) * (1 + 2 * (m - k - 1)) for k in range(m))
    tri = nops * m * m + (r + nops) * m * (m - 1)
    bz = 2 * m * n * (r + nops)
    sz = 2 * m * r * (r + nops)
    lu_s = 2.0 / 3.0 * r ** 3 + 2.0 * nops * r ** 2
    out = 2 * m * r * nops
    return asm + lu_p + tri + bz + sz + lu_s + out


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index=0):
        self.dev = dev_index
        self.proc = None
        self.path = os.path.join(ROOT, "build", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is producing samples
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
            if getattr(self, "f", None) is not None:
                self.f.close()
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        import statistics

        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


CPU_SAMPLE_SEED = 7


def cpu_sample_nodes(N, n_sample, seed=CPU_SAMPLE_SEED):
    """``n_sample`` random nodes in ascending order; every node when
    n_sample <= 0 or >= N."""
    import numpy as np

    if n_sample <= 0 or n_sample >= N:
        return np.arange(N)
    return np.sort(np.random.default_rng(seed).choice(N, n_sample, replace=False))


def cpu_sample_run(n_sample, gpu_npz=None, seed=CPU_SAMPLE_SEED):
    """The oracle (as it stands) on a bounded sample of the workload: stencils,
    weights and one application for ``n_sample`` randomly chosen nodes.
    Returns (seconds, nodes, parity).  After the timed part, when ``gpu_npz``
    holds the GPU's stencils, weights and outputs for the same nodes, they are
    compared with the oracle's (weights 1e-10 relative per stencil, apply 1e-9
    of sum |w u|)."""
    import numpy as np

    from oracle import apply as oap
    from oracle import stencils as ost
    from oracle import weights as ow
    from paper_2303_01760_gb300 import nodesets

    ns = nodesets.cached(nodesets.square_holes)
    centers = cpu_sample_nodes(ns.N, n_sample, seed)
    n_sample = len(centers)
    u, _ = nodesets.field_sincos(ns.coords)
    t0 = time.perf_counter()
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, centers=centers,
                            use_kdtree=True, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    ref = {}
    for op in ("dx", "dy", "lap"):
        ref[("mon", op)] = oap.apply_group(st["mon_idx"], W["mon"][op], u)
        ref[("rbf", op)] = oap.apply_group(st["rbf_idx"], W["rbf"][op], u)
    t = time.perf_counter() - t0
    parity = None
    if gpu_npz and seed == CPU_SAMPLE_SEED and os.path.exists(gpu_npz):
        g = np.load(gpu_npz)
        row = {int(c): i for i, c in enumerate(g["nodes"])}
        worst_w, worst_a, ok_idx = 0.0, 0.0, True
        for k, op in enumerate(("dx", "dy", "lap")):
            for grp, width in (("mon", 5), ("rbf", 12)):
                nodes = st[grp + "_nodes"]
                if not len(nodes):
                    continue
                r = np.array([row[int(c)] for c in nodes])
                if not (np.all(g["width"][r] == width) and np.array_equal(g["col"][r, :width], st[grp + "_idx"])):
                    ok_idx = False
                    continue
                wv = g["val"][k][r, :width]
                e = np.abs(wv - W[grp][op]).max(1) / np.abs(W[grp][op]).max(1)
                worst_w = max(worst_w, float(e.max()))
                sc = (np.abs(W[grp][op]) * np.abs(u[st[grp + "_idx"]])).sum(1)
                worst_a = max(worst_a, float((np.abs(g["out"][k][r] - ref[(grp, op)]) / sc).max()))
        parity = {"ok": ok_idx and worst_w <= 1e-10 and worst_a <= 1e-9, "sampled_nodes": int(n_sample),
                  "stencils_identical": ok_idx, "max_rel_weight_err": worst_w, "max_rel_apply_err": worst_a}
    return t, n_sample, parity


def _oracle_share(args):
    """One worker's share of the all-cores oracle run: stencils, weights and
    one application for the nodes ``centers`` (single-threaded)."""
    centers, = args
    import numpy as np

    from oracle import apply as oap
    from oracle import stencils as ost
    from oracle import weights as ow
    from paper_2303_01760_gb300 import nodesets

    ns = nodesets.cached(nodesets.square_holes)
    u, _ = nodesets.field_sincos(ns.coords)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, centers=np.asarray(centers),
                            use_kdtree=True, normals=ns.normals)
    W = ow.all_weights(ns.coords, st, 2)
    for op in ("dx", "dy", "lap"):
        oap.apply_group(st["mon_idx"], W["mon"][op], u)
        oap.apply_group(st["rbf_idx"], W["rbf"][op], u)
    return len(centers)


def cpu_baseline_all_cores():
    """The same oracle work over the whole workload, split into equal shares
    across every host core by a process pool (started with spawn, each worker
    single-threaded); the pool's start-up and the node set's load are outside
    the timed region.  Returns the cpu_baseline-style record."""
    import multiprocessing as mp

    import numpy as np

    from paper_2303_01760_gb300 import nodesets

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    N = nodesets.cached(nodesets.square_holes).N
    shares = [(c.tolist(),) for c in np.array_split(np.arange(N), cores)]
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_share, [(list(range(8)),)] * cores)  # start-up and imports
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_share, shares, chunksize=1))
            t = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": done / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {done} nodes of the workload in {len(shares)} equal shares over a {cores}-process pool "
                      f"(spawn, one thread each): stencils by k-d tree, weights, one application; {t:.2f} s",
            "seconds": t}


def cpu_baseline(n_sample=0, gpu_npz=None):
    """Runs the oracle sample in a fresh single-threaded process (and, after
    its timing, the parity check of the GPU's outputs for the same nodes).
    Returns (cpu_baseline, parity)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "t, n, par = bench.cpu_sample_run(%d, %r); print(json.dumps([t, n, par]))" % (ROOT, n_sample, gpu_npz))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-500:]}, None
    t, n, par = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": n / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} nodes of the workload{' (all of it)' if n_sample <= 0 else ' at random'}: their "
                      f"stencils by k-d tree, MON/RBF-FD weights by numpy batched solve, one application of "
                      f"dx,dy,lap; {t:.1f} s single-threaded",
            "seconds": t}, par


def save_gpu_sample(ns, plan, u, n_sample, path):
    """The timed plan's stencils, weights and operator outputs for the nodes
    of the CPU sample, for the parity check in the cpu_baseline leg."""
    import numpy as np

    nodes = cpu_sample_nodes(ns.N, n_sample)
    out = plan.apply(u).cpu().numpy()[:, nodes]
    col = np.full((len(nodes), 12), -1, dtype=np.int64)
    val = np.zeros((3, len(nodes), 12))
    width = None
    for k, bit in enumerate((1, 2, 8)):
        rp, c, v = [t.cpu().numpy() for t in plan.export_csr(bit)]
        a, b = rp[nodes], rp[nodes + 1]
        width = b - a
        for j in range(12):
            has = j < width
            if k == 0:
                col[has, j] = c[a[has] + j]
            val[k, has, j] = v[a[has] + j]
    np.savez(path, nodes=nodes, width=width, col=col, val=val, out=out)


# ---------------------------------------------------------------------------
# GPU arm
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# k_rbf_fp64<2, 3, 8> on the hybrid workload, from an ncu capture of
# the kernel as it stands.  None whenever that kernel changes until it is
# re-captured.
RBF64_TRAFFIC_BYTES = 2465280 + 0
# the same for k_weights_grouped<2, 3, 8> (both groups in one launch)
GROUPED_TRAFFIC_BYTES = 9752832 + 18688
# the same summed over the chunk launches of k_rbf_fp64_chunk<2, 3, 8> (the
# solve inside the stencil build), per chunk count; absent: not captured
CHUNK_TRAFFIC_BYTES = {1: 2464256 + 0}


def roofline_kernel(tune):
    if tune["arrange"] == 1:
        return ("k_weights_grouped (FP64 weights of both groups in one persistent launch; the RBF-FD null-space "
                "solves bound it; algorithmic flops of the RBF-FD systems only)")
    if tune["arrange"] == 2:
        return (f"k_rbf_fp64_chunk (RBF-FD FP64 null-space solve inside the stencil build, {tune['chunks']} "
                "chunk(s), chunk c beside the kNN search of chunk c + 1; timed over the span of its launches, "
                "which overlaps the kNN search)")
    return ("k_rbf_fp64 (RBF-FD FP64 null-space solve, hybrid set; the MON weights run beside the kNN search "
            "in the stencil build)")


def aggregate_ranks(times, n_nodes, dist, device):
    """Replicas on several ranks: the step times are the maximum over ranks
    (the job is as slow as its slowest replica) and the nodes processed per
    step are summed over ranks (each rank runs its own seeded node set)."""
    import torch

    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(n_nodes)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], float(n[0])


# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    import __graft_entry__

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda", local)
    # every rank runs its own replica of the workload (independent node sets)
    ns = nodesets.cached(nodesets.square_holes) if rank == 0 else \
        nodesets.cached(nodesets.square_holes, seed=nodesets.SEED_BASE + 1 + 100 * rank)
    d = dict(coords=torch.from_numpy(ns.coords).to(dev), reg=torch.from_numpy(ns.is_regular).to(dev),
             bnd=torch.from_numpy(ns.is_boundary).to(dev), nrm=torch.from_numpy(ns.normals).to(dev))
    d["reg0"] = torch.zeros_like(d["reg"])
    u_np, _ = nodesets.field_sincos(ns.coords)
    u = torch.from_numpy(u_np).to(dev)
    out = torch.empty((3, ns.N), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make(reg):
        p = hsm.Plan(d["coords"], reg, d["bnd"], ns.h, m=2, normals=d["nrm"], stream=stream)
        p.set_timing(True)
        return p

    def one_step(plan):
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64)
        plan.apply(u, out=out)

    def timed(plan, K, W):
        for _ in range(W):
            one_step(plan)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        phases = []
        launches0 = plan.profile()[1]
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_step(plan)
            b.record(stream)
            evs.append((a, b))
            phases.append(plan.profile()[0])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        launches = plan.profile()[1] - launches0
        return ms, phases, launches

    hyb = make(d["reg"])
    allr = make(d["reg0"])
    # one-off autotuning of the kernel variants (cached per device and shape)
    cache = os.path.join(ROOT, "build", "hsm_tune.txt")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    for pl in (hyb, allr):
        pl.build_stencils()
        pl.autotune(cache)
    # correctness gate of this exact launch configuration: sampled nodes vs the oracle
    hyb.build_stencils()
    hyb.compute_weights(hsm.HSM_PREC_FP64)
    gpu_npz = os.path.join(ROOT, "build", "gpu_sample.npz")
    if rank == 0:
        save_gpu_sample(ns, hyb, u, args.cpu_sample, gpu_npz)
    with Clocks(local) as clk:
        ms_h, ph_h, launches_h = timed(hyb, args.steps, args.warmup)
        ms_a, ph_a, launches_a = timed(allr, args.steps, args.warmup)
    clocks = clk.summary()
    q_h, q_a = hyb.query(), allr.query()
    tune_h, tune_a = hyb.tuning(), allr.tuning()
    t_h = float(np.mean(ms_h))
    t_a = float(np.mean(ms_a))
    n_total = float(ns.N)
    if world > 1:
        (t_h, t_a), n_total = aggregate_ranks([t_h, t_a], ns.N, dist, dev)

    # roofline of the dominant kernel: the FP64 RBF-FD weight solve
    rbf_ms = float(np.mean([p[2] for p in ph_h]))
    rbf_ms_all = float(np.mean([p[2] for p in ph_a]))
    n_rbf_h = ns.N - q_h["n_mon"]
    n_rbf_a = ns.N - q_a["n_mon"]
    ach_h = rbf_flops(12, 6, 3) * n_rbf_h / (rbf_ms * 1e-3) / 1e9
    ach_a = rbf_flops(12, 6, 3) * n_rbf_a / (rbf_ms_all * 1e-3) / 1e9
    peak_derived = FP64_PEAK_DERIVED / 1e9
    # measured FP64 FMA rate of this GPU (FMA chains, CUDA events), with the
    # SM clock sampled while it runs
    with Clocks(local) as clk_p:
        peak, peak_ms = hsm.probe_fp64_peak(stream)
    peak_clocks = clk_p.summary()
    # combined rate over a simulation of S explicit steps: the weights once,
    # then S applications (S = 2,000, the step count of this workload's
    # configuration); at S = 1 it is the timed step's rate
    S_STEPS = 2000

    def combined(ms, ph, S):
        # T_w: the step's time (CUDA events around the whole step) less its
        # apply phase, whatever the arrangement of the weights (with the
        # weights in the build, the RBF-FD phase lies inside the stencil phase)
        ta = float(np.mean([p[3] for p in ph]))
        tw = float(np.mean(ms)) - ta
        return n_total * S / ((tw + S * ta) * 1e-3), tw, ta

    # end to end through the C ABI from pinned host buffers
    e2e = run_e2e(ns, hsm, dev, stream, args, cache)
    # large-scale apply roofline and the learned-weight comparison
    big = run_big_apply(hsm, nodesets, dev, stream, flush, args) if (rank == 0 and not args.no_extras) else None
    learned = run_learned(hsm, nodesets, dev, stream, flush, args) if (rank == 0 and not args.no_extras) else None
    three_d = run_3d(hsm, nodesets, dev, stream, flush, args) if (rank == 0 and not args.no_extras) else None

    res = None
    if rank == 0:
        value = n_total / (t_h * 1e-3)
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_h, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded node sets; no paper geometry)",
            "parity_ok": None, "parity": None,
            "config": workload_desc(ns),
            "e2e": e2e,
            "gpu_launches": int(launches_h // max(args.steps, 1)) * args.steps,
            "roofline": {"bound": "alu",
                         "kernel": roofline_kernel(tune_h),
                         "achieved": ach_h, "peak": peak, "unit": "GFLOP/s", "frac": ach_h / peak,
                         "traffic": ({0: RBF64_TRAFFIC_BYTES, 1: GROUPED_TRAFFIC_BYTES}.get(tune_h["arrange"])
                                     if tune_h["arrange"] != 2 else CHUNK_TRAFFIC_BYTES.get(tune_h["chunks"])),
                         "peak_source": "measured: FP64 FMA-chain probe (hsm_probe_fp64_peak) in this run, "
                                        f"{peak_ms:.3f} ms, SM clock median {peak_clocks.get('sm_mhz')} MHz",
                         "peak_clocks": peak_clocks,
                         "peak_derived": peak_derived, "frac_of_derived": ach_h / peak_derived,
                         "peak_derived_source": "152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz"},
            "all_rbffd": {"value": n_total / (t_a * 1e-3), "ms_per_step": t_a,
                          "hybrid_over_all_rbffd": t_a / t_h,
                          "roofline_frac_rbf_kernel": ach_a / peak,
                          "rbf_kernel_gflops": ach_a},
            "combined": {
                "definition": "N*S/(T_w + S*T_a): T_a = one fused apply of dx,dy,lap (phase events), T_w = the "
                              "timed step (stencils + weights + apply, L2 flushed before each step) less T_a; "
                              "S = 2000 is the step count of the configuration and the defining figure, S = 1 is "
                              "the timed step (the headline value)",
                "S": S_STEPS,
                "hybrid": combined(ms_h, ph_h, S_STEPS)[0], "all_rbffd": combined(ms_a, ph_a, S_STEPS)[0],
                "hybrid_over_all_rbffd": combined(ms_h, ph_h, S_STEPS)[0] / combined(ms_a, ph_a, S_STEPS)[0],
                "S1_hybrid_over_all_rbffd": combined(ms_h, ph_h, 1)[0] / combined(ms_a, ph_a, 1)[0],
                "T_w_ms": {"hybrid": combined(ms_h, ph_h, 1)[1], "all_rbffd": combined(ms_a, ph_a, 1)[1]},
                "T_a_ms": {"hybrid": combined(ms_h, ph_h, 1)[2], "all_rbffd": combined(ms_a, ph_a, 1)[2]}},
            "phases_ms": {"weights_in_build": {"hybrid": tune_h["arrange"] == 2, "all_rbffd": tune_a["arrange"] == 2},
                          "hybrid": dict(zip(["stencils", "mon_weights", "weights", "apply"],
                                             np.mean(ph_h, 0).round(4).tolist())),
                          "all_rbffd": dict(zip(["stencils", "mon_weights", "weights", "apply"],
                                                np.mean(ph_a, 0).round(4).tolist()))},
            "counts": {"mon": q_h["n_mon"], "rbf": n_rbf_h, "demoted": q_h["n_demoted"]},
            "apply_roofline": big,
            "three_d": three_d,
            "learned": learned,
            "clocks": clocks,
            "tuning": {"note": "kernel variants picked by hsm_plan_autotune before the timed region",
                       "hybrid": tune_h, "all_rbffd": tune_a},
        }
    stepper = run_stepper(hsm, ns, hyb, d, dev, stream, args) if (rank == 0 and not args.no_extras) else None
    cond = run_condition(hsm, ns, hyb, dev) if (rank == 0 and not args.no_extras) else None
    if res is not None:
        res["stepper"] = stepper
        res["condition"] = cond
    hyb.close()
    allr.close()
    if rank == 0:
        if world == 1:
            res["cpu_baseline"], res["parity"] = cpu_baseline(args.cpu_sample, gpu_npz)
            res["parity_ok"] = bool(res["parity"] and res["parity"].get("ok"))
            try:
                res["cpu_baseline_all_cores"] = cpu_baseline_all_cores()
            except Exception as exc:  # reported, never fatal to the GPU line
                res["cpu_baseline_all_cores"] = {"error": repr(exc)[:300]}
        else:
            res["cpu_baseline"] = None
        print(json.dumps(res))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_condition(hsm, ns, plan, dev):
    """Condition numbers kappa_2 of every node's weight system on the timed
    hybrid set (Section 2.1): MON nodes, RBF-FD nodes, and the demoted
    regular nodes, which sit where the lattice meets the scattered band."""
    import numpy as np
    import torch

    plan.build_stencils()
    plan.compute_weights(hsm.HSM_PREC_FP64)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    kap = plan.condition()
    b.record()
    torch.cuda.synchronize()
    k = kap.cpu().numpy()
    # MON nodes are the rows of width 2d+1
    rp = plan.export_csr(hsm.HSM_LAP)[0]
    mon = ((rp[1:] - rp[:-1]).cpu().numpy() == 2 * ns.dim + 1)
    assert int(mon.sum()) == plan.query()["n_mon"]
    demoted = (ns.is_regular == 1) & ~mon

    def stats(v):
        v = v[np.isfinite(v)]
        return {"count": int(v.size), "median": float(np.median(v)) if v.size else None,
                "p99": float(np.quantile(v, 0.99)) if v.size else None, "max": float(v.max()) if v.size else None}

    return {"workload": "the timed 2D irregular node set; kappa_2 of the scaled weight systems",
            "ms": a.elapsed_time(b), "mon": stats(k[mon]), "rbf": stats(k[~mon]),
            "rbf_demoted_regular": stats(k[demoted]), "rbf_scattered": stats(k[~mon & ~demoted]),
            "singular": int((~np.isfinite(k)).sum())}


def run_stepper(hsm, ns, plan, d, dev, stream, args, steps=30):
    """Explicit Boussinesq steps (Section 3) on the timed hybrid plan:
    Ra = 1e6, Pr = 0.71, dt = 0.1 h^2/2, pressure to a relative residual of
    1e-10; node-steps/s over the last steps (warm-started pressure)."""
    import numpy as np
    import torch

    bc = torch.from_numpy(ns.bc).to(dev)
    Tbc = torch.from_numpy(ns.T_bc).to(dev)
    dt = 0.1 * ns.h * ns.h / 2.0
    st = hsm.Stepper(plan, 1e6, 0.71, dt, ns.T_ref, bc, Tbc, d["nrm"], krylov_tol=1e-10, krylov_max_it=4000)
    v = torch.zeros((2, ns.N), dtype=torch.float64, device=dev)
    T = torch.where(bc == 1, Tbc, torch.zeros_like(Tbc)).contiguous()
    p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
    it0, _ = st.step(v, T, p, 5, allow_notconv=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    its, code = st.step(v, T, p, steps, allow_notconv=True)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    info = st.info()
    st.close()
    iters = float(np.mean(its))
    us_it = ms * 1e3 / steps / max(iters, 1e-9)
    wk = krylov_iteration_work(info, ns.N, gmres=True, j_avg=min(iters, 30.0) / 2.0)
    peak_h, src_h = hbm_peak()
    return {"workload": "2D irregular domain (the timed node set), Ra=1e6, Pr=0.71, dt=0.1h^2/2, "
                        "bordered pressure by GMRES(30) to 1e-10, right-preconditioned by an aggregation-multigrid "
                        "V(2,2)-cycle (one cycle per iteration)",
            "steps": steps, "ms_per_step": ms / steps, "node_steps_per_s": ns.N * steps / (ms * 1e-3),
            "krylov_iters_per_step": iters, "first_steps_iters": it0,
            "converged": code == 0, "T_finite": bool(torch.isfinite(T).all()),
            "us_per_iteration": us_it,
            "cycle": {k: info[k] for k in ("mg_levels", "mg_persistent", "mg_tail_level", "mg_fused_level",
                                           "kernels_per_iter", "tail_ms_10_cycles", "fused_ms_10_cycles",
                                           "persistent_ms_10_cycles", "level_rows", "level_entries")},
            "roofline": {"bound": "latency", "unit": "GB/s",
                         "note": "per GMRES iteration (one V(2,2)-cycle, one operator application, the "
                                 "orthogonalisation against the basis so far): algorithmic bytes and FP64 flops "
                                 "from the level sizes, over "
                                 "ms_per_step / krylov_iters_per_step (the step's other kernels included); the "
                                 "working set (%.0f MB) stays in L2, so neither HBM nor the FP64 pipe bounds it"
                                 % (wk["working_set_bytes"] / 1e6),
                         "bytes_per_iteration": wk["bytes"], "flops_per_iteration": wk["flops"],
                         "achieved": wk["bytes"] / (us_it * 1e3), "peak": peak_h, "peak_source": src_h,
                         "frac": wk["bytes"] / (us_it * 1e3) / peak_h,
                         "fp64_gflops": wk["flops"] / (us_it * 1e3)}}


def krylov_iteration_work(info, N, gmres=False, j_avg=0.0):
    """Algorithmic work of one Krylov iteration with the multigrid
    preconditioner, from the rows R and stored matrix entries Z of each
    level (12 bytes per entry: a 4-byte column and an 8-byte value; 8 bytes
    per vector element read or written).  Per non-coarsest level and cycle:
    pre-smoothing 12Z + 24R bytes, 3Z + 3R flops; restriction 12Z + 20R +
    12Rc bytes, 2Z + 2R flops; the two post-smoothing sweeps 12Z + 36R + 8Rc
    and 12Z + 32R bytes, 4Z + 4R and 2Z + 3R flops (Rc: rows of the next
    level).  Coarsest level: the dense m x m solve, 8m^2 + 16m bytes, 2m^2
    flops.  BiCGSTAB: two cycles, two applications of the fine bordered
    operator (12Z0 + 16N bytes, 2Z0 + 2N flops each) and the vector updates
    and dot products (20 vector passes, 160N bytes, 22N flops).  GMRES: one
    cycle, one application, and against a basis of j + 1 vectors (j_avg on
    average) the dot products and the update (each (j + 1) 8N + 16N bytes,
    2 (j + 1) N flops), the scaling (24N bytes, N flops) and the copy of the
    cycle's output into the basis (16N bytes)."""
    R = list(info["level_rows"])
    Z = list(info["level_entries"])
    L = len(R)
    by = fl = 0.0
    for l in range(L - 1):
        Rc = R[l + 1]
        by += 48 * Z[l] + 112 * R[l] + 20 * Rc
        fl += 11 * Z[l] + 12 * R[l]
    if L:
        m = R[-1]
        by += 8 * m * m + 16 * m
        fl += 2 * m * m
    if gmres:
        jb = j_avg + 1.0
        by += (12 * Z[0] + 16 * N) + 2 * (jb * 8 * N + 16 * N) + 24 * N + 16 * N if L else 0
        fl += (2 * Z[0] + 2 * N) + 2 * (2 * jb * N) + N if L else 0
    else:
        by, fl = 2 * by, 2 * fl
        by += 2 * (12 * Z[0] + 16 * N) + 160 * N if L else 0
        fl += 2 * (2 * Z[0] + 2 * N) + 22 * N if L else 0
    ws = sum(12 * z + 48 * r for z, r in zip(Z, R)) + 12 * 8 * N
    return {"bytes": by, "flops": fl, "working_set_bytes": ws}


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def apply_bytes(plan_q, N, n_rbf, n_mon, wm, wr, nops, f32):
    """Algorithmic bytes of one fused application: per node its index stream,
    its weight streams, one read of u and the operator outputs."""
    wb = 4 if f32 else 8
    ub = 4 if f32 else 8
    per = lambda W: 4 * W + wb * W * nops + ub + 8 * nops
    return n_mon * per(wm) + n_rbf * per(wr)


def run_big_apply(hsm, nodesets, dev, stream, flush, args):
    """The 8M-node 2D workload shape (30 % scattered, m = 2): 12 x 12 tiled
    copies of a unit square minus 8 holes (lattice h = 1/250, scattered band
    0.09 around the holes).  Weights (FP64) throughput and the HBM roofline of
    the fused operator application with f64 and f32 storage."""
    import numpy as np
    import torch

    base = nodesets.cached(nodesets.square_holes, n=250, band=0.09)
    ns = nodesets.tiled(base, 12, 12)
    d = dict(c=torch.from_numpy(ns.coords).to(dev), r=torch.from_numpy(ns.is_regular).to(dev),
             b=torch.from_numpy(ns.is_boundary).to(dev), n=torch.from_numpy(ns.normals).to(dev))
    plan = hsm.Plan(d["c"], d["r"], d["b"], ns.h, m=2, normals=d["n"], stream=stream)
    plan.set_timing(True)
    plan.build_stencils()
    plan.autotune(os.path.join(ROOT, "build", "hsm_tune.txt"))
    res = {"workload": f"2D, {ns.N} nodes ({ns.n_scattered / ns.N:.1%} scattered): 12x12 tiled copies of a unit "
                       "square minus 8 holes, lattice h=1/250, band 0.09, m=2 n=12",
           "nodes": int(ns.N)}
    ws = []
    for prec, name in ((hsm.HSM_PREC_FP64, "fp64"), (hsm.HSM_PREC_FP32_REFINE, "fp32_refine")):
        plan.compute_weights(prec)
        ts = []
        for _ in range(2):
            flush.zero_()
            plan.compute_weights(prec)
            ph = plan.profile()[0]
            ts.append(ph[1] + ph[2])
        q = plan.query()
        ws.append((name, float(np.mean(ts)), q["n_fallback"]))
    res["weights_ms"] = {k: round(t, 3) for k, t, _ in ws}
    res["weights_nodes_per_s"] = {k: ns.N / (t * 1e-3) for k, t, _ in ws}
    res["fp32_refine_fallbacks"] = ws[1][2]
    plan.compute_weights(hsm.HSM_PREC_FP64)
    q = plan.query()
    n_mon = q["n_mon"]
    n_rbf = ns.N - n_mon
    u = torch.from_numpy(nodesets.field_sincos(ns.coords)[0]).to(dev)
    out = torch.empty((3, ns.N), dtype=torch.float64, device=dev)
    peak, src = hbm_peak()
    for name, uu, f32 in (("f64", u, False), ("f32", u.float(), True)):
        plan.apply(uu, out=out)
        ts = []
        for _ in range(max(args.steps, 5)):
            flush.zero_()
            plan.apply(uu, out=out)
            ts.append(plan.profile()[0][3])
        t = float(np.median(ts))
        b = apply_bytes(q, ns.N, n_rbf, n_mon, 5, 12, 3, f32)
        gbs = b / (t * 1e-3) / 1e9
        res[name] = {"ms": t, "algorithmic_bytes": int(b), "bytes_per_node": b / ns.N,
                     "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak}
    res["bound"] = "hbm"
    res["peak_source"] = f"{src} (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    plan.close()
    return res


def run_3d(hsm, nodesets, dev, stream, flush, args):
    """The 3D configuration at full size: unit cube minus 20 seeded spheres,
    lattice h = 1/125, scattered within 0.05 of a sphere (about 1.9M nodes;
    the seeded set takes about 1.5 minutes to generate on the host and is
    cached).  For m = 2 (n = 20) and m = 3 (n = 40): FP64 and FP32 +
    FP64-refinement weights (times, fallbacks, nodes that took a lower
    monomial degree, the refinement's largest weight difference from the FP64
    solve) and the fused application of grad and Laplacian with f64 and f32
    storage, against the measured HBM copy bandwidth."""
    import numpy as np
    import torch

    t0 = time.time()
    ns = nodesets.cached(nodesets.cube_spheres, n=125)
    gen_s = time.time() - t0
    d = [torch.from_numpy(a).to(dev) for a in (ns.coords, ns.is_regular, ns.is_boundary, ns.normals)]
    u = torch.from_numpy(nodesets.field_random_smooth(ns.coords)[0]).to(dev)
    res = {"workload": f"3D, {ns.N} nodes ({ns.n_scattered / ns.N:.1%} scattered): unit cube minus 20 spheres, "
                       "lattice h=1/125, band 0.05; ops dx,dy,dz,lap", "nodes": int(ns.N),
           "nodeset_seconds": round(gen_s, 1)}
    peak, _ = hbm_peak()
    for m in (2, 3):
        n = 2 * (10 if m == 2 else 20)
        plan = hsm.Plan(d[0], d[1], d[2], ns.h, m=m, normals=d[3], stream=stream)
        plan.set_timing(True)
        plan.build_stencils()
        plan.autotune(os.path.join(ROOT, "build", "hsm_tune.txt"))
        out = {"n": n}
        status = torch.zeros(ns.N, dtype=torch.uint8, device=dev)
        ref = None
        for prec, name in ((hsm.HSM_PREC_FP64, "fp64"), (hsm.HSM_PREC_FP32_REFINE, "fp32_refine")):
            plan.compute_weights(prec, status, allow_singular=True)
            ts = []
            for _ in range(2):
                flush.zero_()
                plan.compute_weights(prec, status, allow_singular=True)
                ph = plan.profile()[0]
                ts.append(ph[1] + ph[2])
            q = plan.query()
            stat = status.cpu().numpy()
            singular = stat == 255
            vals = [plan.export_csr(1 << k)[2].cpu().numpy() for k in range(4)]
            rp = plan.export_csr(1)[0].cpu().numpy()
            rows = np.flatnonzero((rp[1:] - rp[:-1] == n) & ~singular)
            ix = rp[rows][:, None] + np.arange(n)[None, :]
            entry = {"weights_ms": float(np.mean(ts)), "nodes_per_s": ns.N / (np.mean(ts) * 1e-3),
                     "fallbacks": q["n_fallback"], "singular_nodes": int(singular.sum()),
                     "reduced_degree_nodes": int((stat == hsm.HSM_NODE_REDUCED_DEGREE).sum())}
            if ref is None:
                ref = [v[ix] for v in vals]
            else:
                worst = 0.0
                for k in range(4):
                    e = np.abs(vals[k][ix] - ref[k]).max(1) / np.abs(ref[k]).max(1)
                    worst = max(worst, float(e.max()) if e.size else 0.0)
                entry["max_rel_weight_diff_from_fp64"] = worst
            out[name] = entry
        plan.compute_weights(hsm.HSM_PREC_FP64, allow_singular=True)
        q = plan.query()
        o = torch.empty((4, ns.N), dtype=torch.float64, device=dev)
        for name, uu, f32 in (("apply_f64", u, False), ("apply_f32", u.float(), True)):
            plan.apply(uu, out=o)
            ts = []
            for _ in range(max(args.steps, 5)):
                flush.zero_()
                plan.apply(uu, out=o)
                ts.append(plan.profile()[0][3])
            t = float(np.median(ts))
            b = apply_bytes(q, ns.N, ns.N - q["n_mon"], q["n_mon"], 7, n, 4, f32)
            out[name] = {"ms": t, "achieved_GBs": b / (t * 1e-3) / 1e9, "frac": b / (t * 1e-3) / 1e9 / peak}
        res[f"m{m}"] = out
        plan.close()
    return res


def run_learned(hsm, nodesets, dev, stream, flush, args):
    """Learned + projected weights against the plain FP64 solve (the
    predictor's workload shape): trained on about 3.6M interior stencils of
    64 jittered copies (jitter 0-30 %) of one Poisson-disk set, tested on as
    many stencils from a second set with disjoint seeds."""
    import numpy as np
    import torch

    def plan_of(ns):
        d = dict(c=torch.from_numpy(ns.coords).to(dev), r=torch.from_numpy(ns.is_regular).to(dev),
                 b=torch.from_numpy(ns.is_boundary).to(dev), n=torch.from_numpy(ns.normals).to(dev))
        p = hsm.Plan(d["c"], d["r"], d["b"], ns.h, m=2, normals=d["n"], stream=stream)
        p._d = d
        p.set_timing(True)
        return p

    t0 = time.perf_counter()
    base_tr = nodesets.cached(nodesets.square_all_scattered, n=300, seed=nodesets.SEED_BASE + 700)
    base_te = nodesets.cached(nodesets.square_all_scattered, n=300, seed=nodesets.SEED_BASE + 701)
    tr = nodesets.tiled(base_tr, 8, 8, jitter=lambda k: 0.3 * k / 63, seed=1000)
    te = nodesets.tiled(base_te, 8, 8, jitter=lambda k: 0.3 * ((k * 37) % 64) / 63, seed=2000)
    ptr = plan_of(tr)
    ptr.build_stencils()
    ptr.compute_weights(hsm.HSM_PREC_FP64)
    X, Y = ptr.learned_data()
    ptr.close()
    mlp = hsm.MLP(24, 256, 3, 36, seed=5, stream=stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    schedule = ((1e-3, 6000), (3e-4, 3000), (1e-4, 3000))
    for lr, steps in schedule:
        log = mlp.train(X, Y, steps=steps, batch=4096, lr=lr, seed=int(lr * 1e7))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    n_steps = sum(st for _, st in schedule)
    # GEMM work of one training step with the padded layer widths (din 64,
    # 256, 256, 256; dout 256, 256, 256, 128): forward and dW over every
    # layer, dX over every layer but the first
    wd = [(64, 256), (256, 256), (256, 256), (256, 128)]
    train_flops = 2 * 4096 * (2 * sum(a * b for a, b in wd) + sum(a * b for a, b in wd[1:]))
    del X, Y
    pte = plan_of(te)
    pte.build_stencils()
    pte.attach(mlp)
    times, gate = {}, {}
    # fp64; learned with the batch validation (tolerance 1e-3, 512 samples);
    # learned without it (the predictor's own speed and accuracy)
    for name, prec, samples in (("fp64", hsm.HSM_PREC_FP64, 512), ("learned_validated", hsm.HSM_PREC_LEARNED, 512),
                                ("learned", hsm.HSM_PREC_LEARNED, 0)):
        pte.set_learned_gate(1e-3, samples)
        pte.compute_weights(prec)
        ts = []
        for _ in range(2):
            flush.zero_()
            pte.compute_weights(prec)
            ph = pte.profile()[0]
            ts.append(ph[2])
        times[name] = float(np.mean(ts))
        if name == "learned_validated":
            err, failed, n_acc = pte.learned_gate()
            gate = {"tolerance": 1e-3, "samples": 512, "mean_rel_weight_err": err, "accepted_samples": n_acc,
                    "batch_took_direct_solve": failed}
    # reference weights: this plan's FP64 solve (checked against the oracle by the tests)
    pte.set_learned_gate(1e-3, 0)
    pte.compute_weights(hsm.HSM_PREC_FP64)
    rp, col, val_d = [t.cpu().numpy() for t in pte.export_csr(8)]
    st = torch.zeros(te.N, dtype=torch.uint8, device=dev)
    pte.compute_weights(hsm.HSM_PREC_LEARNED, st)
    q = pte.query()
    n_rbf = te.N - q["n_mon"]
    status = st.cpu().numpy()
    val = pte.export_csr(8)[2].cpu().numpy()
    rng = np.random.default_rng(5)
    inner = np.flatnonzero(te.is_boundary == 0)
    nodes = np.sort(rng.choice(inner, 3000, replace=False))
    ix = rp[nodes][:, None] + np.arange(12)[None, :]
    wl, wd = val[ix], val_d[ix]
    acc = status[nodes] == hsm.HSM_NODE_OK
    rel = np.abs(wl - wd).max(1) / np.abs(wd).max(1)
    local = te.coords[:, nodes] % ((300 + 2) / 300)
    u, der = nodesets.field_sincos(te.coords % ((300 + 2) / 300))
    deep = np.minimum(local, 1 - local).min(0) > 0.15
    el = np.abs((wl * u[col[ix]]).sum(1) - der["lap"][nodes])[deep & acc]
    ed = np.abs((wd * u[col[ix]]).sum(1) - der["lap"][nodes])[deep & acc]
    pte.close()
    mlp.close()
    return {"workload": f"train {tr.N} nodes, test {te.N} nodes (interior scattered stencils, n=12, m=2)",
            "train_s": round(t_train, 2), "final_train_loss": float(np.mean(log[-50:])),
            "train_steps": n_steps, "train_step_ms": t_train * 1e3 / n_steps,
            "train_gemm_tflops": train_flops * n_steps / t_train / 1e12,
            "train_note": "batch 4096 rows; every GEMM of the step is a tcgen05 kernel (host wall clock over all "
                          "steps, the Adam update and packing included)",
            "weights_ms": times, "rbf_weights_per_s": {k: n_rbf / (v * 1e-3) for k, v in times.items()},
            "learned_over_fp64": times["fp64"] / times["learned"],
            "learned_validated_over_fp64": times["fp64"] / times["learned_validated"],
            "batch_validation": gate,
            "accepted_fraction": float(np.mean(status[inner] == hsm.HSM_NODE_OK)),
            "fallbacks": q["n_fallback"],
            "lap_weight_rel_diff_median": float(np.median(rel[acc])) if acc.any() else None,
            "lap_error_on_sincos_max": {"learned": float(el.max()) if el.size else None,
                                        "fp64": float(ed.max()) if ed.size else None},
            "setup_s": round(time.perf_counter() - t0, 1)}


def run_e2e(ns, hsm, dev, stream, args, cache=None):
    """Same metric end to end: every step copies its pinned host inputs in,
    builds the stencils, computes the weights, applies the operators and
    copies the three outputs back.  Steps run the way a caller streaming node
    sets would run them: two host threads, each driving its own plan on its
    own stream with its own device buffers, take the steps in turn, so one
    plan's copies and host round trips overlap the other plan's kernels.  The
    timed region runs from an event both streams wait on to the event after
    both streams' last download (CUDA events)."""
    import threading

    import torch

    h = dict(coords=torch.from_numpy(ns.coords).pin_memory(), reg=torch.from_numpy(ns.is_regular).pin_memory(),
             bnd=torch.from_numpy(ns.is_boundary).pin_memory(), nrm=torch.from_numpy(ns.normals).pin_memory(),
             u=torch.from_numpy(nodesets_u(ns)).pin_memory())
    out_h = [torch.empty((3, ns.N), dtype=torch.float64).pin_memory() for _ in range(2)]
    bufs = [{k: torch.empty_like(v, device=dev) for k, v in h.items()} for _ in range(2)]
    outs = [torch.empty((3, ns.N), dtype=torch.float64, device=dev) for _ in range(2)]
    streams = [torch.cuda.Stream(dev) for _ in range(2)]
    for i in range(2):
        for k in h:
            bufs[i][k].copy_(h[k])
    torch.cuda.synchronize()
    plans = [hsm.Plan(bufs[i]["coords"], bufs[i]["reg"], bufs[i]["bnd"], ns.h, m=2, normals=bufs[i]["nrm"],
                      stream=streams[i]) for i in range(2)]
    for pl in plans:
        pl.build_stencils()
        if cache:
            pl.autotune(cache)  # the variants tuned for this shape (cached)
    h2d = sum(v.numel() * v.element_size() for v in h.values())
    d2h = out_h[0].numel() * 8
    errors = []

    def worker(i, n):
        try:
            torch.cuda.set_device(dev)
            s = streams[i]
            with torch.cuda.stream(s):
                for _ in range(n):
                    for k in h:
                        bufs[i][k].copy_(h[k], non_blocking=True)
                    plans[i].build_stencils()
                    plans[i].compute_weights(hsm.HSM_PREC_FP64)
                    plans[i].apply(bufs[i]["u"], out=outs[i])
                    out_h[i].copy_(outs[i], non_blocking=True)
        except Exception as exc:  # re-raised by the caller
            errors.append(exc)

    def run(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(streams[0])
        streams[1].wait_event(a)
        ts = [threading.Thread(target=worker, args=(i, (n + 1 - i) // 2)) for i in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errors:
            raise errors[0]
        streams[0].wait_stream(streams[1])
        b.record(streams[0])
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    run(max(args.warmup, 2))
    ms = run(args.steps) / args.steps
    for pl in plans:
        pl.close()
    return {"value": ns.N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "pipelining": "two host threads, each driving one plan on its own stream, take the steps in turn; "
                          "every step uploads its inputs, builds, weighs, applies and downloads; tuned variants"}


def nodesets_u(ns):
    from paper_2303_01760_gb300 import nodesets

    return nodesets.field_sincos(ns.coords)[0]


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle runs single-threaded (set before numpy is first imported)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from paper_2303_01760_gb300 import nodesets

    ns = nodesets.cached(nodesets.square_holes)
    # each step processes the whole workload, unless K + W steps of it would
    # take more than a few minutes; then each step takes an equal share
    n_sample = args.ref_sample if args.ref_sample > 0 else \
        (ns.N if args.steps + args.warmup <= 40 else max(5000, ns.N * 40 // (args.steps + args.warmup)))
    n_sample = min(n_sample, ns.N)
    cpu_sample_run(500)  # warm imports / caches
    times = []
    for _ in range(args.warmup):
        cpu_sample_run(n_sample)
    for k in range(args.steps):
        t, n, _ = cpu_sample_run(n_sample, seed=100 + k)
        times.append(t)
    t = sum(times) / len(times)
    value = n_sample / t
    cores = 1
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_desc(ns),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{n_sample} of the workload's {ns.N} nodes per step (stencils, weights, "
                                      f"one application of dx,dy,lap), single-threaded"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def run_kernels(args):
    """Profiling driver: the timed operator path on the hybrid workload, with
    no oracle, no parity gate and no JSON (for ncu captures)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    if args.three_d:
        # the 1.88M-node 3D set with m = args.three_d: FP64 weights, then f64
        # and f32 applies of dx, dy, dz, lap
        ns = nodesets.cached(nodesets.cube_spheres, n=125)
        dd = [torch.from_numpy(a).to(dev) for a in (ns.coords, ns.is_regular, ns.is_boundary, ns.normals)]
        plan = hsm.Plan(dd[0], dd[1], dd[2], ns.h, m=args.three_d, normals=dd[3])
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64, allow_singular=True)
        u = torch.from_numpy(nodesets.field_random_smooth(ns.coords)[0]).to(dev)
        out = torch.empty((4, ns.N), dtype=torch.float64, device=dev)
        for uu in (u, u.float()):
            for _ in range(args.warmup + args.steps):
                plan.apply(uu, out=out)
        torch.cuda.synchronize()
        plan.close()
        print("3d apply ok", ns.N)
        return
    if args.big_apply:
        # the 7.3M-node tiled set: FP64 weights, then f64 applies of dx, dy, lap
        base = nodesets.cached(nodesets.square_holes, n=250, band=0.09)
        ns = nodesets.tiled(base, 12, 12)
    else:
        ns = nodesets.cached(nodesets.square_holes)
    c = torch.from_numpy(ns.coords).to(dev)
    reg = torch.from_numpy(ns.is_regular).to(dev)
    if args.all_rbffd:
        reg = torch.zeros_like(reg)
    bnd = torch.from_numpy(ns.is_boundary).to(dev)
    nrm = torch.from_numpy(ns.normals).to(dev)
    u = torch.from_numpy(nodesets.field_sincos(ns.coords)[0]).to(dev)
    plan = hsm.Plan(c, reg, bnd, ns.h, m=2, normals=nrm)
    if args.knn_qt or args.arrange:
        plan.set_tuning(knn_qt=args.knn_qt or 1, arrange=args.arrange, chunks=args.chunks)
    prec = {"fp64": hsm.HSM_PREC_FP64, "fp32r": hsm.HSM_PREC_FP32_REFINE}[args.prec]
    if args.learned:
        # learned weights on the predictor's workload shape: a short training on
        # one tiled Poisson-disk set, then learned weights of a second set
        def plan_of(nsx):
            dd = [torch.from_numpy(a).to(dev) for a in (nsx.coords, nsx.is_regular, nsx.is_boundary, nsx.normals)]
            px = hsm.Plan(dd[0], dd[1], dd[2], nsx.h, m=2, normals=dd[3])
            px._d = dd
            return px

        base_tr = nodesets.cached(nodesets.square_all_scattered, n=300, seed=nodesets.SEED_BASE + 700)
        base_te = nodesets.cached(nodesets.square_all_scattered, n=300, seed=nodesets.SEED_BASE + 701)
        tr = nodesets.tiled(base_tr, 8, 8, jitter=lambda k: 0.3 * k / 63, seed=1000)
        te = nodesets.tiled(base_te, 8, 8, jitter=lambda k: 0.3 * ((k * 37) % 64) / 63, seed=2000)
        ptr_ = plan_of(tr)
        ptr_.build_stencils()
        ptr_.compute_weights(hsm.HSM_PREC_FP64)
        X, Y = ptr_.learned_data()
        ptr_.close()
        mlp = hsm.MLP(24, 256, 3, 36, seed=5)
        mlp.train(X, Y, steps=args.train_steps, batch=4096, lr=1e-3, seed=3)
        pte = plan_of(te)
        pte.build_stencils()
        pte.attach(mlp)
        for _ in range(args.warmup + args.steps):
            pte.compute_weights(hsm.HSM_PREC_LEARNED)
        torch.cuda.synchronize()
        print("learned ok", te.N, pte.query()["n_fallback"])
        pte.close()
        mlp.close()
        return
    if args.stepper:
        # explicit Boussinesq steps on the hybrid plan (Ra = 1e6, as in the bench's stepper section)
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64)
        bc = torch.from_numpy(ns.bc).to(dev)
        Tbc = torch.from_numpy(ns.T_bc).to(dev)
        st = hsm.Stepper(plan, 1e6, 0.71, 0.1 * ns.h * ns.h / 2.0, ns.T_ref, bc, Tbc, nrm, krylov_tol=1e-10,
                         krylov_max_it=4000, guess_order=args.guess_order, mg_sweeps=args.mg_sweeps,
                         krylov=args.krylov)
        v = torch.zeros((2, ns.N), dtype=torch.float64, device=dev)
        T = torch.where(bc == 1, Tbc, torch.zeros_like(Tbc)).contiguous()
        p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
        st.step(v, T, p, args.warmup, allow_notconv=True)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        its, _ = st.step(v, T, p, args.steps, allow_notconv=True)
        ev[1].record()
        torch.cuda.synchronize()
        print("stepper ok", ns.N, its, "ms/step %.3f" % (ev[0].elapsed_time(ev[1]) / args.steps), st.info())
        st.close()
        plan.close()
        return
    if args.big_apply:
        plan.build_stencils()
        plan.compute_weights(prec)
        out = torch.empty((3, ns.N), dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            plan.apply(u, out=out)
        torch.cuda.synchronize()
        plan.close()
        print("big apply ok", ns.N)
        return
    for _ in range(args.warmup + args.steps):
        plan.build_stencils()
        plan.compute_weights(prec)
        plan.apply(u)
    torch.cuda.synchronize()
    plan.close()
    print("kernels ok", ns.N)


PAPER_NU_DVD = {"hybrid": 8.870, "scattered": 8.867, "regular": 8.852}  # Section 4.1, Table 1


def run_dvd(args):
    """De Vahl Davis natural convection (Section 4.1): Ra = 1e6, Pr = 0.71, from
    rest to t = args.t_end on the quarter layouts, dt = 0.1 h^2 / 2, with the
    average Nusselt number on the cold wall sampled along the way.  Prints one
    JSON line (a validation run, not the benchmark metric)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    ns = nodesets.square_quarters(n=args.dvd, layout=args.layout)
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(dev)
         for k in ("coords", "is_regular", "is_boundary", "normals", "bc", "T_bc")}
    t0 = time.time()
    plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=2, normals=d["normals"])
    plan.build_stencils()
    plan.compute_weights(hsm.HSM_PREC_FP64)
    q = plan.query()
    dt = 0.1 * ns.h * ns.h / 2.0
    st = hsm.Stepper(plan, 1e6, 0.71, dt, ns.T_ref, d["bc"], d["T_bc"], d["normals"], krylov_tol=1e-10,
                     krylov_max_it=4000)
    v = torch.zeros((2, ns.N), dtype=torch.float64, device=dev)
    T = torch.where(d["bc"] == 1, d["T_bc"], torch.zeros_like(d["T_bc"])).contiguous()
    p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
    cold = np.flatnonzero((ns.is_boundary == 1) & (ns.coords[0] == 0.0)).astype(np.int32)
    cold_d = torch.from_numpy(cold).to(dev)
    n_steps = int(round(args.t_end / dt))
    chunk = max(1, n_steps // 150)
    series, iters, done, worst = [], 0, 0, 0
    torch.cuda.synchronize()
    t_run = time.time()
    while done < n_steps:
        k = min(chunk, n_steps - done)
        its, code = st.step(v, T, p, k, allow_notconv=True)
        iters += sum(its)
        worst = max(worst, max(its))
        done += k
        nu = float(plan.wall_flux_mean(T, cold_d, d["normals"], scale=1.0).item())
        series.append([round(done * dt, 6), nu])
    torch.cuda.synchronize()
    wall = time.time() - t_run
    vmax = float(v.abs().max().item())
    ref = PAPER_NU_DVD[args.layout]
    # vertical velocity across the section y = 0.5 (the nodes within h/2 of it,
    # by x), the comparison the paper draws between the three layouts
    sec = np.flatnonzero(np.abs(ns.coords[1] - 0.5) <= 0.5 * ns.h)
    sec = sec[np.argsort(ns.coords[0][sec], kind="stable")]
    vy = v[1].cpu().numpy()
    profile = [[round(float(ns.coords[0][i]), 6), round(float(ns.coords[1][i]), 6), float(vy[i])] for i in sec]
    out = {"dvd": {"layout": args.layout, "n": args.dvd, "h": ns.h, "N": int(ns.N), "n_mon": int(q["n_mon"]),
                   "n_scattered": int(ns.n_scattered), "Ra": 1e6, "Pr": 0.71, "dt": dt, "t_end": args.t_end,
                   "steps": n_steps, "krylov_iters_per_step": iters / n_steps, "krylov_iters_max": worst},
           "nu_final": series[-1][1], "nu_paper": ref, "nu_rel_diff": series[-1][1] / ref - 1.0,
           "nu_last_tenth_spread": float(np.ptp([x[1] for x in series[-max(2, len(series) // 10):]])),
           "max_speed": vmax, "finite": bool(torch.isfinite(T).all() and torch.isfinite(v).all()),
           "run_s": wall, "ms_per_step": 1e3 * wall / n_steps, "setup_s": t_run - t0, "nu_series": series,
           "vy_profile_y05": profile}
    st.close()
    plan.close()
    print(json.dumps(out))


PAPER_2D_REFINED = {"hybrid": {"Nu": 12.36, "minutes": 29.11, "N": 11535},
                    "scattered": {"Nu": 12.32, "minutes": 46.31, "N": 10534}}  # Section 4.2, Table 2
PAPER_3D = {"hybrid": {"Nu": 6.91, "hours": 20.54, "N": 74137},
            "scattered": {"Nu": 7.36, "hours": 48.12, "N": 65526}}  # Section 4.3, Table 3
REFINED_2D = dict(n=100, n_holes=4, r_range=(0.06, 0.12), ratio=3.0, seed=20230351)
REFINED_3D = dict(dim=3, n=40, n_holes=4, r_range=(0.08, 0.16), delta_h=4.0, ratio=2.0, seed=20230341)


def _refined_dev(ns, dev, reg=None):
    import numpy as np
    import torch

    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(dev)
         for k in ("coords", "is_regular", "is_boundary", "normals", "bc", "T_bc", "spacing")}
    if reg is not None:
        d["is_regular"] = reg
    return d


def _time_steps(hsm, plan, ns, d, dev, n_steps, Ra, dt, cold=None, chunks=1):
    """n_steps explicit Boussinesq steps from rest; returns ms/step (CUDA
    events), Krylov iterations per step and, with ``cold``, the final mean
    |dT/dn| on those nodes (and, with chunks > 1, its value after each of
    ``chunks`` equal parts of the run)."""
    import numpy as np
    import torch

    st = hsm.Stepper(plan, Ra, 0.71, dt, ns.T_ref, d["bc"], d["T_bc"], d["normals"], krylov_tol=1e-10,
                     krylov_max_it=4000)
    v = torch.zeros((ns.dim, ns.N), dtype=torch.float64, device=dev)
    T = torch.where(d["bc"] == 1, d["T_bc"], torch.zeros_like(d["T_bc"])).contiguous()
    p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
    st.step(v, T, p, 3, allow_notconv=True)
    torch.cuda.synchronize()
    cd = torch.from_numpy(cold).to(dev) if cold is not None else None
    history = []
    its, gpu_ms, done = [], 0.0, 0
    for c in range(chunks):
        k = (n_steps * (c + 1)) // chunks - done
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        it_c, _ = st.step(v, T, p, k, allow_notconv=True)
        ev[1].record()
        torch.cuda.synchronize()
        gpu_ms += ev[0].elapsed_time(ev[1])
        its += list(it_c)
        done += k
        if cd is not None and chunks > 1:
            history.append([round((done + 3) * dt, 6), float(plan.wall_flux_mean(T, cd, d["normals"]).item())])
    out = {"ms_per_step": gpu_ms / n_steps, "krylov_iters_per_step": float(np.mean(its)),
           "max_speed": float(v.abs().max().item()),
           "finite": bool(torch.isfinite(T).all() and torch.isfinite(v).all())}
    if cold is not None:
        out["nu_cold"] = float(plan.wall_flux_mean(T, cd, d["normals"]).item())
        if history:
            out["nu_cold_history"] = history
    st.close()
    return out


def run_refined(args):
    """h-refinement and the width of the scattered layer (Section 4.2 and its
    delta_h study): unit square minus 4 seeded circular holes (standing in for
    the ducks), h_r = 0.01, spacing falling linearly to h_s = h_r/3 at the
    holes over h_r * delta_h, which is also the layer width; delta_h swept over
    2..32, plus the fully scattered set with the same refinement.  Per set:
    node counts, the operator pass (stencils + FP64 weights + one apply of
    dx, dy, Laplacian) of the set and of the same nodes all RBF-FD, the
    operator error on u = sin(pi x) cos(pi y), and the explicit step
    (Ra = 1e6, dt = 0.1 h_s^2 / 2).  Prints one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    rows = []
    for dh, full in [(2.0, False), (4.0, False), (8.0, False), (16.0, False), (32.0, False), (4.0, True)]:
        ns = nodesets.cached(nodesets.holes_refined, delta_h=dh, all_scattered=full, **REFINED_2D)
        d = _refined_dev(ns, dev)
        u, ex = nodesets.field_sincos(ns.coords)
        ut = torch.from_numpy(u).to(dev)
        inner = ns.is_boundary == 0
        row = {"delta_h": dh, "layout": "scattered" if full else "hybrid", "N": int(ns.N),
               "n_scattered": int(ns.n_scattered), "n_regular": int(ns.N - ns.n_scattered)}
        for name, reg in (("set", None), ("all_rbffd", torch.zeros_like(d["is_regular"]))):
            if full and name == "all_rbffd":
                continue
            dd = dict(d, is_regular=d["is_regular"] if reg is None else reg)
            plan = hsm.Plan(dd["coords"], dd["is_regular"], dd["is_boundary"], ns.h, m=2, normals=dd["normals"],
                            spacing=dd["spacing"])
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            times = []
            for it in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                ev[0].record()
                plan.build_stencils()
                plan.compute_weights(hsm.HSM_PREC_FP64)
                out = plan.apply(ut)
                ev[1].record()
                torch.cuda.synchronize()
                if it >= args.warmup:
                    times.append(ev[0].elapsed_time(ev[1]))
            q = plan.query()
            o = out.cpu().numpy()
            err = {op: float(np.abs(o[k, inner] - ex[op][inner]).max() / np.abs(ex[op][inner]).max())
                   for k, op in enumerate(("dx", "dy", "lap"))}
            row[name] = {"ms": float(np.median(times)), "n_mon": int(q["n_mon"]), "rel_err": err}
            if name == "set":
                cold = np.flatnonzero((ns.is_boundary == 1) & (ns.bc == nodesets.BC_T_DIRICHLET)
                                      & (ns.T_bc == 0.0)).astype(np.int32)
                dt = 0.1 * float(ns.spacing.min()) ** 2 / 2.0
                row["step"] = _time_steps(hsm, plan, ns, dd, dev, args.refined_steps, 1e6, dt, cold)
                row["step"]["dt"] = dt
            plan.close()
        if "all_rbffd" in row:
            row["operator_speedup_vs_all_rbffd"] = row["all_rbffd"]["ms"] / row["set"]["ms"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr)
    h4 = next(r for r in rows if r["delta_h"] == 4.0 and r["layout"] == "hybrid")
    s4 = next(r for r in rows if r["layout"] == "scattered")
    out = {"refined": {"domain": "unit square minus 4 circular holes (r 0.06-0.12), h_r = 0.01, h_s = h_r/3",
                       "Ra": 1e6, "Pr": 0.71, "steps_timed": args.refined_steps, "sets": rows},
           "delta_h_4": {"N_hybrid": h4["N"], "N_scattered": s4["N"],
                         "step_ms_hybrid": h4["step"]["ms_per_step"], "step_ms_scattered": s4["step"]["ms_per_step"],
                         "step_time_ratio_hybrid_over_scattered":
                             h4["step"]["ms_per_step"] / s4["step"]["ms_per_step"],
                         "paper": PAPER_2D_REFINED,
                         "paper_time_ratio": PAPER_2D_REFINED["hybrid"]["minutes"]
                         / PAPER_2D_REFINED["scattered"]["minutes"]}}
    print(json.dumps(out))


def run_spheres3d(args):
    """Natural convection in the unit cube minus 4 seeded spheres (Section 4.3:
    two spheres at T_C = 0, two at T_H = 1, insulated box, Ra = 1e4,
    Pr = 0.71), h_r = 1/n, spacing falling linearly to h_s = h_r/2 at the
    spheres over 4 h_r (delta_h = 4), dt = 0.1 h_s^2 / 2 (7.8125e-6 at
    n = 40, the paper's step).  Hybrid and fully scattered sets, each run from
    rest for ``--t-end`` time units (or ``--spheres3d-steps`` steps), with the
    average Nusselt number on the cold spheres.  The paper's spheres are random
    and unpublished, so its Nu and hours are context.  Prints one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    cfg = dict(REFINED_3D, n=args.spheres3d)
    out = {"spheres3d": {"n": args.spheres3d, "h_r": 1.0 / args.spheres3d, "Ra": 1e4, "Pr": 0.71},
           "paper": PAPER_3D}
    for layout in ("hybrid", "scattered"):
        ns = nodesets.cached(nodesets.holes_refined, all_scattered=layout == "scattered", **cfg)
        d = _refined_dev(ns, dev)
        t0 = time.time()
        plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=2, normals=d["normals"],
                        spacing=d["spacing"])
        plan.build_stencils()
        plan.compute_weights(hsm.HSM_PREC_FP64)
        q = plan.query()
        dt = 0.1 * float(ns.spacing.min()) ** 2 / 2.0
        n_steps = args.spheres3d_steps if args.t_end is None else int(round(args.t_end / dt))
        cold = np.flatnonzero((ns.is_boundary == 1) & (ns.bc == nodesets.BC_T_DIRICHLET)
                              & (ns.T_bc == 0.0)).astype(np.int32)
        setup = time.time() - t0
        r = _time_steps(hsm, plan, ns, d, dev, n_steps, 1e4, dt, cold, chunks=10 if args.t_end else 1)
        plan.close()
        r.update({"N": int(ns.N), "n_mon": int(q["n_mon"]), "n_scattered": int(ns.n_scattered), "dt": dt,
                  "steps": n_steps, "t_reached": n_steps * dt, "setup_s": setup,
                  "hours_per_time_unit": r["ms_per_step"] * (1.0 / dt) / 3.6e6})
        out[layout] = r
    out["time_ratio_hybrid_over_scattered"] = out["hybrid"]["ms_per_step"] / out["scattered"]["ms_per_step"]
    out["paper_time_ratio"] = PAPER_3D["hybrid"]["hours"] / PAPER_3D["scattered"]["hours"]
    print(json.dumps(out))


# band widths of square_holes (h = 0.002, 8 holes) whose scattered fraction is
# within 1 % of 5 / 20 / 50 %, found by bisecting the band on the host
SWEEP_BANDS = {0.05: 0.02344, 0.20: 0.07031, 0.50: 0.12891}


def run_sweep(args):
    """The 2D irregular configuration with the scattered fraction swept over
    about 5 / 13 (the nominal 0.05 band) / 20 / 50 / 100 %, for m = 2 (n = 12)
    and m = 4 (n = 30), FP64 weights.  Per set: the operator pass (stencils +
    weights + one apply of dx, dy, Laplacian; L2 flushed before each rep) and
    the apply alone, nodes/s, the same nodes all RBF-FD, the combined rate
    N S / (T_w + S T_a) for S = 2000 steps, and for m = 2 the explicit step
    (Ra = 1e6).  Prints one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    S = 2000
    sets = [("5%", SWEEP_BANDS[0.05]), ("nominal", 0.05), ("20%", SWEEP_BANDS[0.20]), ("50%", SWEEP_BANDS[0.50]),
            ("100%", None)]
    rows = []
    for label, band in sets:
        ns = nodesets.cached(nodesets.square_holes) if label in ("nominal", "100%") else \
            nodesets.cached(nodesets.square_holes, band=band)
        d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(dev)
             for k in ("coords", "is_regular", "is_boundary", "normals", "bc", "T_bc")}
        if label == "100%":
            d["is_regular"] = torch.zeros_like(d["is_regular"])
        u = torch.from_numpy(nodesets.field_sincos(ns.coords)[0]).to(dev)
        out = torch.empty((3, ns.N), dtype=torch.float64, device=dev)
        row = {"set": label, "band": band, "N": int(ns.N),
               "scattered_fraction": 1.0 if label == "100%" else round(ns.n_scattered / ns.N, 4)}
        for m in (2, 4):
            plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=m, normals=d["normals"])
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            tw, ta = [], []
            for it in range(args.warmup + args.steps):
                flush.fill_(it)
                ev[0].record()
                plan.build_stencils()
                plan.compute_weights(hsm.HSM_PREC_FP64)
                ev[1].record()
                flush.fill_(it + 1)
                ev[2].record()
                plan.apply(u, out=out)
                ev[3].record()
                torch.cuda.synchronize()
                if it >= args.warmup:
                    tw.append(ev[0].elapsed_time(ev[1]))
                    ta.append(ev[2].elapsed_time(ev[3]))
            Tw, Ta = float(np.median(tw)), float(np.median(ta))
            q = plan.query()
            r = {"n": plan.n, "n_mon": int(q["n_mon"]), "weights_ms": Tw, "apply_ms": Ta,
                 "nodes_per_s_weights": ns.N / (Tw * 1e-3), "nodes_per_s_apply": ns.N / (Ta * 1e-3),
                 "nodes_per_s_combined": ns.N * S / ((Tw + S * Ta) * 1e-3)}
            if m == 2:
                dt = 0.1 * ns.h * ns.h / 2.0
                r["step"] = _time_steps(hsm, plan, ns, d, dev, args.sweep_steps, 1e6, dt)
            plan.close()
            row[f"m{m}"] = r
        rows.append(row)
        print(json.dumps(row), file=sys.stderr)
    full = rows[-1]
    for row in rows:
        for m in (2, 4):
            # throughput (nodes/s) relative to the all-RBF-FD set
            row[f"m{m}"]["combined_vs_all_rbffd"] = (row[f"m{m}"]["nodes_per_s_combined"]
                                                     / full[f"m{m}"]["nodes_per_s_combined"])
    print(json.dumps({"sweep": {"workload": "unit square minus 8 holes, lattice h = 0.002, scattered band swept",
                                "S": S, "sets": rows}}))


def oracle_steps(n_steps, out_npz, seed_set="square_holes"):
    """The oracle's stepper on the 2D irregular workload from rest, Ra = 1e6,
    Pr = 0.71, dt = 0.1 h^2/2 (exact pressure solve by sparse LU): the fields
    after ``n_steps`` steps go to ``out_npz``, with the host seconds it took."""
    import numpy as np

    from oracle import stencils as ost
    from oracle import stepper as ostep
    from oracle import weights as ow
    from paper_2303_01760_gb300 import nodesets

    ns = nodesets.cached(getattr(nodesets, seed_set))
    t0 = time.perf_counter()
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals,
                            use_kdtree=True)
    W = ow.all_weights(ns.coords, st, 2)
    S = ostep.Stepper(ns.coords, ns.bc, ns.T_bc, ns.normals, ns.T_ref, st, W, 1e6, 0.71, ostep.dt_rule(ns.h))
    v, T = ostep.initial_state(2, ns.N, ns.bc, ns.T_bc)
    t1 = time.perf_counter()
    v, T, p = S.run(v, T, n_steps)
    t2 = time.perf_counter()
    np.savez(out_npz, v=v, T=T, p=p, setup_s=t1 - t0, steps_s=t2 - t1)


def run_field_linf(args):
    """Field L-inf error of the GPU stepper after a fixed number of steps on
    the full 2D irregular workload (222,555 nodes), against the oracle run for
    the same steps in a separate single-threaded process: T and v, each
    relative to the largest magnitude of the oracle's field."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    S = args.field_linf
    dev = torch.device("cuda:0")
    ns = nodesets.cached(nodesets.square_holes)
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(dev)
         for k in ("coords", "is_regular", "is_boundary", "normals", "bc", "T_bc")}
    plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=2, normals=d["normals"])
    plan.build_stencils()
    plan.compute_weights(hsm.HSM_PREC_FP64)
    dt = 0.1 * ns.h * ns.h / 2.0
    st = hsm.Stepper(plan, 1e6, 0.71, dt, ns.T_ref, d["bc"], d["T_bc"], d["normals"], krylov_tol=args.krylov_tol,
                     krylov_max_it=4000)
    v = torch.zeros((2, ns.N), dtype=torch.float64, device=dev)
    T = torch.where(d["bc"] == 1, d["T_bc"], torch.zeros_like(d["T_bc"])).contiguous()
    p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    its, code = st.step(v, T, p, S, allow_notconv=True)
    ev[1].record()
    torch.cuda.synchronize()
    gpu_ms = ev[0].elapsed_time(ev[1])
    info = st.info()
    g = dict(v=v.cpu().numpy(), T=T.cpu().numpy())
    st.close()
    plan.close()
    out_npz = os.path.join(ROOT, "build", "oracle_field_linf.npz")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code_s = ("import sys; sys.path.insert(0, %r); import bench; bench.oracle_steps(%d, %r)" % (ROOT, S, out_npz))
    r = subprocess.run([sys.executable, "-c", code_s], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        print(json.dumps({"field_linf": {"error": r.stderr[-800:]}}))
        return
    o = np.load(out_npz)
    rel = {k: float(np.abs(g[k] - o[k]).max() / max(np.abs(o[k]).max(), 1e-300)) for k in ("T", "v")}
    print(json.dumps({"field_linf": {
        "workload": "2D irregular domain, 222,555 nodes (h = 0.002, 8 holes), Ra = 1e6, Pr = 0.71, "
                    "dt = 0.1 h^2/2, from rest; FP64 weights and state",
        "steps": S, "krylov_tol": args.krylov_tol, "rel_linf": rel,
        "gpu": {"ms_per_step": gpu_ms / S, "krylov_iters_mean": float(np.mean(its)),
                "krylov_iters_last100": float(np.mean(its[-100:])), "status": int(code), **info},
        "oracle": {"setup_s": float(o["setup_s"]), "steps_s": float(o["steps_s"]), "cores": 1,
                   "pressure": "sparse LU of the bordered system, factored once"},
        "max_abs": {"T": float(np.abs(o["T"]).max()), "v": float(np.abs(o["v"]).max())}}}))


def run_precision_sweep(args):
    """The 8M-node 2D precision sweep on one connected domain: the unit square
    minus the 8 seeded holes of the 222k-node workload, lattice h = 1/2800,
    scattered band 0.094 (about 31 % scattered; the seeded set takes several
    minutes to generate on the host and is cached).  FP64 vs FP32 +
    FP64-refinement weights for m = 2 and m = 4 (time, fallbacks and the
    largest relative weight difference per stencil), and ``S`` explicit
    Boussinesq steps at Ra = 1e6 from rest with FP64 and with FP32 operator
    applications (FP64 state, time accumulation and pressure solve): field
    L-inf of the FP32 run against the FP64 run, each relative to the largest
    magnitude of the FP64 field.  The FP64 stepper matches the oracle to
    ~1e-13 after 2,000 steps on the 222k-node set (``--field-linf``); at this
    size the oracle's sparse LU is out of reach.  (The tiled 7.3M-node set of
    the apply roofline is 144 disconnected squares, whose Neumann pressure
    problem has one null vector per square: not a stepper workload.)"""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2303_01760_gb300 import hsm, nodesets

    dev = torch.device("cuda:0")
    S = args.precision_sweep
    t0 = time.time()
    ns = nodesets.cached(nodesets.square_holes, n=2800, band=0.094)
    gen_s = time.time() - t0
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(ns, k))).to(dev)
         for k in ("coords", "is_regular", "is_boundary", "normals", "bc", "T_bc")}
    out = {"workload": f"2D, {ns.N} nodes ({ns.n_scattered / ns.N:.1%} scattered): unit square minus 8 holes, "
                       "lattice h=1/2800, band 0.094", "nodes": int(ns.N), "nodeset_seconds": round(gen_s, 1),
           "weights": {}}
    for m in (2, 4):
        plan = hsm.Plan(d["coords"], d["is_regular"], d["is_boundary"], ns.h, m=m, normals=d["normals"])
        plan.set_timing(True)
        plan.build_stencils()
        res = {}
        w = {}
        for prec, name in ((hsm.HSM_PREC_FP64, "fp64"), (hsm.HSM_PREC_FP32_REFINE, "fp32_refine")):
            plan.compute_weights(prec)
            torch.cuda.synchronize()
            plan.compute_weights(prec)
            ph = plan.profile()[0]
            w[name] = [plan.export_csr(b)[2] for b in (1, 2, 8)]
            res[name] = {"weights_ms": ph[1] + ph[2], "fallbacks": plan.query()["n_fallback"]}
        rp = plan.export_csr(1)[0]
        rows = torch.repeat_interleave(torch.arange(ns.N, device=dev), (rp[1:] - rp[:-1]))
        worst = 0.0
        for a, b in zip(w["fp64"], w["fp32_refine"]):
            num = torch.zeros(ns.N, dtype=torch.float64, device=dev).scatter_reduce(0, rows, (a - b).abs(), "amax")
            den = torch.zeros(ns.N, dtype=torch.float64, device=dev).scatter_reduce(0, rows, a.abs(), "amax")
            worst = max(worst, float((num / den.clamp_min(1e-300)).max()))
        res["max_rel_weight_diff_fp32_refine_vs_fp64"] = worst
        out["weights"][f"m{m}"] = res
        if m == 2:
            plan.compute_weights(hsm.HSM_PREC_FP64)
            dt = 0.1 * ns.h * ns.h / 2.0
            fields = {}
            for name, f32 in (("fp64_apply", False), ("fp32_apply", True)):
                st = hsm.Stepper(plan, 1e6, 0.71, dt, ns.T_ref, d["bc"], d["T_bc"], d["normals"], krylov_tol=1e-10,
                                 krylov_max_it=4000, apply_f32=f32)
                v = torch.zeros((2, ns.N), dtype=torch.float64, device=dev)
                T = torch.where(d["bc"] == 1, d["T_bc"], torch.zeros_like(d["T_bc"])).contiguous()
                p = torch.zeros(ns.N, dtype=torch.float64, device=dev)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record()
                its, code = st.step(v, T, p, S, allow_notconv=True)
                ev[1].record()
                torch.cuda.synchronize()
                fields[name] = (v, T)
                out[name] = {"ms_per_step": ev[0].elapsed_time(ev[1]) / S, "krylov_iters_mean": float(np.mean(its)),
                             "status": int(code)}
                st.close()
            (v64, T64), (v32, T32) = fields["fp64_apply"], fields["fp32_apply"]
            out["steps"] = S
            out["field_linf_fp32_apply_vs_fp64"] = {
                "T": float((T32 - T64).abs().max() / T64.abs().max()),
                "v": float((v32 - v64).abs().max() / v64.abs().max().clamp_min(1e-300))}
        plan.close()
    print(json.dumps({"precision_sweep": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle nodes in cpu_baseline (0: all)")
    ap.add_argument("--ref-sample", type=int, default=0, help="oracle nodes per --impl reference step (0: all, "
                    "or an equal share of a few minutes when --steps + --warmup > 40)")
    ap.add_argument("--kernels", action="store_true", help="profiling driver only (no JSON line)")
    ap.add_argument("--no-extras", action="store_true", help="skip the 7M-node apply and learned sections")
    ap.add_argument("--all-rbffd", action="store_true", help="with --kernels: force every node to RBF-FD")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32r"], help="with --kernels")
    ap.add_argument("--stepper", action="store_true", help="with --kernels: run --steps Boussinesq steps instead")
    ap.add_argument("--learned", action="store_true", help="with --kernels: learned weights instead")
    ap.add_argument("--big-apply", action="store_true", help="with --kernels: f64 applies on the 7.3M-node set")
    ap.add_argument("--three-d", type=int, default=0, help="with --kernels: m of f64 and f32 applies on the 3D set")
    ap.add_argument("--knn-qt", type=int, default=0, help="with --kernels: fix the kNN threads per query (1, 2, 4)")
    ap.add_argument("--arrange", type=int, default=0, help="with --kernels: FP64 weights arrangement (0 split, "
                    "1 grouped launch, 2 in the stencil build)")
    ap.add_argument("--chunks", type=int, default=1, help="with --kernels --arrange 2: kNN / solve chunks (1, 2, 4)")
    ap.add_argument("--train-steps", type=int, default=3000, help="with --kernels --learned")
    ap.add_argument("--dvd", type=int, default=0, help="de Vahl Davis validation run on a 1/n lattice (no benchmark)")
    ap.add_argument("--layout", default="hybrid", choices=["hybrid", "scattered", "regular"], help="with --dvd")
    ap.add_argument("--t-end", type=float, default=None, help="with --dvd (default 0.15) or --spheres3d (default 1)")
    ap.add_argument("--spheres3d", type=int, default=0, help="3D natural-convection validation run on a 1/n lattice")
    ap.add_argument("--spheres3d-steps", type=int, default=2000, help="with --spheres3d when --t-end is not given")
    ap.add_argument("--refined", action="store_true", help="h-refinement / scattered-layer width sweep (2D)")
    ap.add_argument("--refined-steps", type=int, default=500, help="with --refined")
    ap.add_argument("--sweep", action="store_true", help="scattered-fraction sweep (5..100 %%), m = 2 and 4")
    ap.add_argument("--sweep-steps", type=int, default=100, help="with --sweep: explicit steps timed per set")
    ap.add_argument("--krylov", type=int, default=0, help="with --kernels --stepper: 0 GMRES(30), 1 BiCGSTAB")
    ap.add_argument("--mg-sweeps", type=int, default=0, help="with --kernels --stepper: 1 or 2 Jacobi sweeps "
                    "each way in the multigrid cycle (0: the library default)")
    ap.add_argument("--guess-order", type=int, default=0, help="with --kernels --stepper: pressure initial "
                    "guess (0 quadratic extrapolation, 1 linear, -1 last solution)")
    ap.add_argument("--field-linf", type=int, default=0,
                    help="GPU stepper vs the oracle after this many steps on the 2D irregular workload")
    ap.add_argument("--krylov-tol", type=float, default=1e-12, help="with --field-linf")
    ap.add_argument("--precision-sweep", type=int, default=0,
                    help="the 7.3M-node precision sweep with this many explicit steps")
    args = ap.parse_args()
    if args.precision_sweep:
        run_precision_sweep(args)
        return
    if args.field_linf:
        run_field_linf(args)
        return
    if args.dvd:
        args.t_end = 0.15 if args.t_end is None else args.t_end
        run_dvd(args)
        return
    if args.spheres3d:
        run_spheres3d(args)
        return
    if args.refined:
        run_refined(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.kernels:
        run_kernels(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
