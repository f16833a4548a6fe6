"""The algorithmic work per unit that the benchmark's roofline figures divide
by: FP64 flops of one RBF-FD system and bytes of one fused application."""
import bench


def test_rbf_flops_per_system():
    # 2D, m = 2 (6 monomials), n = 12, dx/dy/lap: assembly 642 + null-space solve 3,239
    assert round(bench.rbf_flops(12, 6, 3)) == 3881
    # the assembly part alone: offsets 48, pairs 66 x 7, higher monomials 36, RHS 60, unscaling 36
    assert 2 * 12 * 2 + 66 * 7 + 12 * 3 + 12 * 5 + 12 * 3 == 642


def test_apply_bytes_per_node():
    """Per node: int32 indices, FP64 weights of 3 operators, one read of u and
    three FP64 outputs: 172 B (MON, 5 nodes), 368 B (RBF-FD, n = 12) and
    872 B (n = 30); FP32 storage halves the weights and u (outputs stay FP64)."""
    per = lambda w, f32=False: bench.apply_bytes(None, 1, 1, 0, 5, w, 3, f32)
    assert bench.apply_bytes(None, 1, 0, 1, 5, 12, 3, False) == 172
    assert per(12) == 368
    assert per(30) == 872
    assert per(12, True) == 48 + 144 + 4 + 24


def test_krylov_iteration_work_counts():
    """A two-level hierarchy counted by hand: level 0 with R = 10 rows and
    Z = 50 stored entries, coarsest level m = 3 rows, N = 10 nodes."""
    info = {"level_rows": [10, 3], "level_entries": [50, 9]}
    w = bench.krylov_iteration_work(info, 10)
    cycle_bytes = 48 * 50 + 112 * 10 + 20 * 3 + 8 * 9 + 16 * 3
    cycle_flops = 11 * 50 + 12 * 10 + 2 * 9
    assert w["bytes"] == 2 * cycle_bytes + 2 * (12 * 50 + 16 * 10) + 160 * 10
    assert w["flops"] == 2 * cycle_flops + 2 * (2 * 50 + 2 * 10) + 22 * 10


def test_krylov_iteration_work_gmres_counts():
    """GMRES: one cycle, one application, orthogonalisation against j + 1 = 3
    basis vectors (j_avg = 2), N = 10."""
    info = {"level_rows": [10, 3], "level_entries": [50, 9]}
    w = bench.krylov_iteration_work(info, 10, gmres=True, j_avg=2.0)
    cycle_bytes = 48 * 50 + 112 * 10 + 20 * 3 + 8 * 9 + 16 * 3
    cycle_flops = 11 * 50 + 12 * 10 + 2 * 9
    assert w["bytes"] == cycle_bytes + (12 * 50 + 16 * 10) + 2 * (3 * 80 + 160) + 240 + 160
    assert w["flops"] == cycle_flops + (2 * 50 + 2 * 10) + 2 * (2 * 3 * 10) + 10
