"""Host-side helpers of bench.py (no GPU): the algorithmic work count used by
the roofline, the whole-job throughput, and the code hash that keys recorded
DRAM traffic to the kernel source it was measured on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flops_per_column_iteration_matches_the_stated_count():
    b = _bench()
    # 2(H-1)^2 + 43H - 19 flops per column and iteration (6 933 at H = 50)
    assert b.flops_per_column_iteration(50) == 6933
    for H in (2, 13, 64, 132):
        assert b.flops_per_column_iteration(H) == 2 * (H - 1) ** 2 + 43 * H - 19


def test_whole_job_throughput_counts_every_rank():
    b = _bench()
    assert b.weak_scaling_value(1, 4096, 10, 10.0) == 4096 * 10 / 0.010
    assert b.weak_scaling_value(4, 4096, 10, 10.0) == 4 * 4096 * 10 / 0.010


def test_code_hash_ignores_comments_and_layout_only():
    b = _bench()
    src = "int f(int a) {\n  return a + 1;  // add one\n}\n/* note */\n"
    assert b.code_hash(src) == b.code_hash("int f(int a) { return a + 1; }")
    assert b.code_hash(src) != b.code_hash("int f(int a) { return a + 2; }")
    assert len(b.kernel_source_hash()) == 16


def test_pipe_rooflines_split_the_work_between_the_pipes():
    b = _bench()
    H = 50
    total = b.flops_per_column_iteration(H)
    kap = b.kapply_flops_per_column_iteration(H)
    assert kap == 2 * 49 ** 2 + 2 * 49 and 0 < kap < total
    r = b.pipe_rooflines(total * 1e9, kap * 1e9, 1.0, 148, {"bf16_tflops": 1800.0})
    assert abs(r["simt"]["achieved"] - (total - kap) * 1e-3) < 1e-9
    assert abs(r["tensor"]["peak"] - 900.0) < 1e-9
    assert abs(r["tensor"]["frac"] - kap * 1e-3 / 900.0) < 1e-12
    assert "ncu" not in r
    assert b.pipe_rooflines(1.0, 0.0, 1.0, 148, {})["tensor"]["frac"] is None
    # the bf16 split K-apply is measured against the bf16 rate itself
    rb = b.pipe_rooflines(total * 1e9, kap * 1e9, 1.0, 148, {"bf16_tflops": 1800.0}, operand="bf16")
    assert abs(rb["tensor"]["peak"] - 1800.0) < 1e-9
