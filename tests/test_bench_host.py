"""Host-side pieces of bench.py that need no GPU: the algorithmic byte counts
behind the roofline figure, and the committed DRAM-traffic record that the
benchmark's `roofline.traffic` field reads (it is used only while it was
taken on the current Map source, so an edit of that source must come with a
new capture)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_map_bytes_of_the_benchmark_system():
    # A once (m n s_A), the per-row record (b0, Av, 1/||a||^2: 12 bytes; 16 with
    # the FP8 row scale) and x (4 n)
    m, n = 131072, 16384
    assert bench.map_bytes(m, n, "f32") == m * n * 4 + m * 12 + 4 * n == 8591572992
    assert bench.map_bytes(m, n, "bf16") == m * n * 2 + m * 12 + 4 * n
    assert bench.map_bytes(m, n, "fp8") == m * n * 1 + m * 16 + 4 * n


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_traffic_record_matches_the_map_source(storage):
    """Every storage of the default workload has a traffic line for the
    current Map source, and it is within 1 % of the algorithmic bytes (a
    Map that re-read A would show far more)."""
    t = bench.profiled_traffic("dense-131072x16384", storage)
    assert t is not None, "profiles/map_kernel_traffic.txt was taken on another Map source"
    alg = bench.map_bytes(131072, 16384, storage)
    assert abs(t / alg - 1.0) < 0.01


def test_map_source_hash_covers_the_map_kernel():
    """The hashed prefix (up to the long-row section) holds the Map kernel's
    body and its kernels; the long-row kernel lies after it."""
    src = open(os.path.join(ROOT, "paper_2003_09956_gb300", "csrc", "nsli_kernels.cu")).read()
    end = src.find(bench.MAP_SOURCE_END)
    assert end > 0
    assert "map_body(" in src[:end] and "map_kernel(const MapArgs p)" in src[:end]
    assert "map_long_kernel(const MapArgs p)" in src[end:]
    assert len(bench.kernels_sha()) == 12


def test_oracle_max_violation_at_a_final_iterate_matches_the_oracle():
    """The CPU leg's max-violation error of a result: the oracle's own
    maximum over all rows, taken per row block in threads, equals the
    oracle over the whole matrix on each storage type's exact values."""
    import oracle
    from paper_2003_09956_gb300 import workloads

    p = workloads.dense_system(1001, 130, seed=17)
    x = p["x0"] * 0.3
    for st in ("f32", "bf16", "fp8"):
        A = p["A"] if st == "f32" else (oracle.quantize_bf16(p["A"]) if st == "bf16"
                                        else oracle.quantize_e4m3_rows(p["A"])[0])
        n2, _ = oracle.norms2(A)
        ref = oracle.map_reduce(A, oracle.tick_b(p["b0"], p["Av"], 1e-3, 5), n2, x)["maxviol"]
        r = bench.oracle_max_violation(p, (st, x, 5, 1e-3, ref + 1.0), threads=3)
        assert r["oracle_f64"] == ref and r["threads"] == 3
        assert abs(r["abs_diff"] - 1.0) < 1e-9


def test_pool_and_feasibility_workloads_are_defined():
    assert set(bench.POOL) == {"pool-40", "pool-20"}
    for w in bench.FEASIBILITY.values():
        assert w["m"] in (4 * w["n"], 8 * w["n"])
