"""bench.py's roofline arithmetic on the CPU: per-entry operation counts of each distance form, and
which pipe binds. Pinned on the bench's own recorded figures and on hand-computed bounds."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_per_entry_operation_counts(bench):
    # difference form, split path: 2D + kernel value + 2 (RBF 0, M52 3, M12 1, M32 2)
    assert bench.per_pair_ops(1, 8, True, 32)[0] == 21
    assert bench.per_pair_ops(0, 4, True, 32)[0] == 10
    # dot form: 1 (r^2 = a_i - d) + kernel value + 4 (Veltkamp split and lo)
    assert bench.per_pair_ops(1, 8, True, 32, dot=True)[0] == 8
    assert bench.per_pair_ops(0, 8, True, 32, dot=True)[0] == 5
    assert bench.per_pair_ops(3, 8, True, 32, dot=True)[0] == 7
    # FP32 SIMT path: 2D + kernel value + t multiply-adds
    assert bench.per_pair_ops(1, 8, False, 1)[0] == 20
    # MUFU: RBF one ex2; the Matern forms a sqrt as well
    assert bench.per_pair_ops(0, 8, True, 32)[1] == {"ex2": 1.0, "sqrt": 0.0}
    assert bench.per_pair_ops(1, 8, True, 32)[1] == {"ex2": 1.0, "sqrt": 1.0}


def _cfg3(bench, ops, mufu, dot, seconds):
    N = 100000
    return bench.binding_pipe(N * (N + 1) / 2, float(N) ** 2, ops, mufu, 32, 8, True, dot, seconds, 152, 1890.0)


def test_dot_form_matern_is_mufu_bound(bench):
    """The bench's line at cfg3 (dot form, Matern-5/2, 3.2312 ms product) reported MUFU, frac 0.4611."""
    r = _cfg3(bench, 8.0, {"ex2": 1.0, "sqrt": 1.0}, True, 3.2312319755554197e-3)
    assert r["binding"] == "mufu"
    assert r["frac"] == pytest.approx(0.46107, rel=1e-4)
    # bound by hand: 5.00005e9 entries x 3 ex2 slots / (152 x 32 x 2.07e9 /s) = 1.4898 ms
    assert r["frac"] * 3.2312319755554197e-3 == pytest.approx(5.00005e9 * 3 / (152 * 32 * 2.07e9), rel=1e-9)
    assert r["pipe_fracs"]["fp32"] < r["frac"] and r["pipe_fracs"]["tensor"] < r["frac"]


def test_difference_form_is_fp32_bound(bench):
    """The earlier bench line (difference form, 5.2642 ms product) reported the FP32 pipe, frac 0.4953."""
    r = _cfg3(bench, 21.0, {"ex2": 1.0, "sqrt": 1.0}, False, 5.264172744750977e-3)
    assert r["binding"] == "fp32"
    assert r["frac"] == pytest.approx(0.49527, rel=1e-4)


def test_dot_form_rbf_is_tensor_bound(bench):
    """RBF has no sqrt and five FP32 operations per entry in the dot form: the contraction's
    N^2 6t flops plus the Gram tile's 64 per entry take the longest at the bf16 burst rate."""
    r = _cfg3(bench, 5.0, {"ex2": 1.0, "sqrt": 0.0}, True, 2.93e-3)
    assert r["binding"] == "tensor"
    assert r["tensor_flops"] == pytest.approx(1e10 * 6 * 32 + 5.00005e9 * 64, rel=1e-12)


def test_low_dimension_gram_tile_counts_its_full_width(bench):
    """The Gram operand rows are 32 values wide at every D (3 x 4 split coordinates and 6 norm and
    unit columns need more than 16 at D <= 4), so the Gram tile costs 64 flops per entry at D = 2 as
    at D = 8. The N = 500000, D = 2, t = 32 RBF product's line (65.5735 ms kernel) reported the tensor
    pipe at 0.4526 of the 1887 TFLOP/s burst."""
    N = 500000
    e = N * (N + 1) / 2
    r = bench.binding_pipe(e, float(N) ** 2, 5.0, {"ex2": 1.0, "sqrt": 0.0}, 32, 2, True, True,
                           65.57327270507812e-3, 152, 1887.0)
    assert r["binding"] == "tensor"
    assert r["tensor_flops"] == pytest.approx(float(N) ** 2 * 6 * 32 + e * 64, rel=1e-12)
    assert r["frac"] == pytest.approx(0.45257, rel=1e-4)
