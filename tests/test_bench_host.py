"""Host logic of bench.py that needs no GPU: the algorithmic byte models
behind the roofline numerators and the launch-list summary.

Bars: the byte models equal the per-unit figures written out by hand
(entries x (value + column bytes) + row pointers + vectors; DCGS2 step j:
10 j n + 46 n), exactly; the launch summary converts units, counts launches
and reports shares that add up.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_apply_bytes_by_hand():
    n, nl, nu = 2097152, 20726144, 20726144  # 128^3 SAIT pair, m_terms = 3, rowrel 1e-3
    # FP64 values + int32 columns, two row-pointer arrays, r in, w out and in, z out
    assert bench.apply_bytes(n, nl, nu, "f64") == (nl + nu) * 12 + 2 * 4 * (n + 1) + 4 * 8 * n == 581313544
    # FP32 values: the intermediate w is FP32 (4 B out + 4 B in)
    assert bench.apply_bytes(n, nl, nu, "f32") == (nl + nu) * 8 + 2 * 4 * (n + 1) + (8 + 4 + 4 + 8) * n
    assert bench.apply_bytes(n, nl, nu, "bf16") == (nl + nu) * 6 + 2 * 4 * (n + 1) + 24 * n
    # *_X64 keep an FP64 intermediate
    assert bench.apply_bytes(n, nl, nu, "f32x64") == (nl + nu) * 8 + 2 * 4 * (n + 1) + 32 * n


def test_spmv_a_bytes_by_hand():
    class A:
        n, nnz = 2097152, 14581760
    assert bench.spmv_a_bytes(A) == 14581760 * 12 + 4 * (2097152 + 1) + 16 * 2097152 == 216924164


def test_ortho_bytes_closed_form():
    n, m = 1000, 50
    step = lambda j: 10 * j * n + 46 * n  # noqa: E731
    # full cycles restart at j = 0
    assert bench.ortho_bytes(n, 2 * m, m) == 2 * sum(step(j) for j in range(m))
    assert bench.ortho_bytes(n, m, m) == 10 * n * m * (m - 1) // 2 + 46 * n * m
    # a partial last cycle
    assert bench.ortho_bytes(n, m + 7, m) == sum(step(j) for j in range(m)) + sum(step(j) for j in range(7))
    # the benchmark's 172 steps at 128^3 (3 cycles of 50 and one of 22): per step
    # (3 (10 * 1225 + 46 * 50) + 10 * 231 + 46 * 22) n / 172
    assert int(bench.ortho_bytes(2097152, 172, 50) / 172) == 46972 * 2097152 // 172 == 572717579


def test_summarize_launches(tmp_path, capsys):
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [
        '"0","void <unnamed>::k_spmv_sell<double>(long)","gpu__time_duration.sum","us","30"\n',
        '"1","<unnamed>::k_dcgs_dot(long)","gpu__time_duration.sum","ns","10,000"\n',
        '"2","void <unnamed>::k_spmv_sell<double>(long)","gpu__time_duration.sum","usecond","20"\n',
        '"3","k_other(int)","gpu__time_duration.sum","ms","0.04"\n',
        '"4","k_other(int)","dram__bytes_read.sum","byte","123"\n',  # other metrics are ignored
    ]
    p = tmp_path / "launches.csv"
    p.write_text("==PROF== Connected\n" + hdr + "".join(rows))
    bench.summarize_launches(str(p))
    out = capsys.readouterr().out.splitlines()
    assert out[0] == "launches 4, total 0.1 ms (serialised, cold cache)"
    table = {line.split(" | ")[0].lstrip("| "): line for line in out[3:]}
    assert "void k_spmv_sell<double>" in table and table["void k_spmv_sell<double>"].endswith("| 2 | 0.05 | 50.0% | 25.0 |")
    assert table["k_other"].endswith("| 1 | 0.04 | 40.0% | 40.0 |")
    assert table["k_dcgs_dot"].endswith("| 1 | 0.01 | 10.0% | 10.0 |")


def test_batched_iteration_bytes_by_hand():
    class A:
        n, nnz = 1000, 4960
    nl = nu = 5000
    # two SAIT applies (FP32 values: 8 B per entry, w FP32), two A products, 22 FP64 vector passes
    one = 2 * ((nl + nu) * 8 + 8 * 1001 + 24 * 1000) + 2 * (4960 * 12 + 4 * 1001 + 16 * 1000) + 22 * 8 * 1000
    assert bench.batched_iter_bytes(A, nl, nu, "f32", 1) == one
    # k columns: the matrices are read once, every vector term scales with k
    k64 = 2 * ((nl + nu) * 8 + 8 * 1001 + 24 * 1000 * 64) + 2 * (4960 * 12 + 4 * 1001 + 16 * 1000 * 64) \
        + 22 * 8 * 1000 * 64
    assert bench.batched_iter_bytes(A, nl, nu, "f32", 64) == k64
    # converged systems skip the vector passes: 600 of the 1000 rows iterate 8 times over 8 replays
    part = one - 22 * 8 * 1000 + 22 * 8 * 600
    assert bench.batched_iter_bytes(A, nl, nu, "f32", 1, row_iters=600 * 8, replays=8) == part


def test_batched_iteration_bound_by_hand(monkeypatch):
    class A:
        n, nnz = 1000, 4960
    nl = nu = 5000
    monkeypatch.setattr(bench, "peaks", lambda: (1000.0, "test"))  # 1000 GB/s = 1e9 bytes per ms
    rate = 2 * 152 * 2070e6 / 1e3                                   # FP64 multiply-adds per ms
    bw = 1e9
    # FP64 storage, 64 columns: each SAIT product does (nl + nu) x 64 FMAs against its bytes
    k = 64
    apply_b, apply_f = (nl + nu) * 12 + 8 * 1001 + 32 * 1000 * k, (nl + nu) * k
    spmv_b, spmv_f = 4960 * 12 + 4 * 1001 + 16 * 1000 * k, 4960 * k
    vec_b, vec_f = 22 * 8 * 1000 * k, 12 * 1000 * k
    want = 2 * max(apply_b / bw, apply_f / rate) + 2 * max(spmv_b / bw, spmv_f / rate) + max(vec_b / bw, vec_f / rate)
    got = bench.batched_iter_bound(A, nl, nu, "f64", k)
    assert abs(got["bound_ms"] - want) < 1e-12 * want
    assert got["fp64_fma"] == 2 * apply_f + 2 * spmv_f + vec_f
    # the FP32 mode multiplies the SAIT products in FP32: no FP64 term there
    got32 = bench.batched_iter_bound(A, nl, nu, "f32", k)
    assert got32["fp64_fma"] == 2 * spmv_f + vec_f
    apply32_b = (nl + nu) * 8 + 8 * 1001 + 24 * 1000 * k
    want32 = 2 * apply32_b / bw + 2 * max(spmv_b / bw, spmv_f / rate) + max(vec_b / bw, vec_f / rate)
    assert abs(got32["bound_ms"] - want32) < 1e-12 * want32
