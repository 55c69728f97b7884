"""Host logic of bench.py (no GPU): the single-system roofline and how the
oracle legs count a verified solve."""
import numpy as np
import pytest

import bench

PEAKS = {"hbm_gbs": 6783.5, "bf16_tflops": 1917.9, "src": "measured"}


def fp64_peak():
    _, dfma, dmma, _ = bench.pipe_peaks()
    return max(dfma, dmma)


def test_fp64_lu_is_alu_bound_at_the_fp64_pipe_rate():
    n, ms = 8192, 444.6
    r = bench.large_case_roofline("general", "fp64", n, 1, ms, PEAKS)
    flops = 2.0 / 3.0 * n ** 3 + 2.0 * n * n
    assert r["bound"] == "alu"
    assert r["flops"] == pytest.approx(flops)
    assert r["floor_ms"] == pytest.approx(flops / fp64_peak() * 1e3)
    assert r["frac"] == pytest.approx(r["floor_ms"] / ms)
    assert r["achieved_tflops"] / r["peak_tflops"] == pytest.approx(r["frac"])


def test_precision_selects_the_peak():
    n, ms = 16384, 50.0  # large enough that every precision is ALU-bound
    mixed = bench.large_case_roofline("spd", "mixed", n, 1, ms, PEAKS)
    bf16 = bench.large_case_roofline("spd", "bf16", n, 1, ms, PEAKS)
    fp16 = bench.large_case_roofline("spd", "fp16", n, 1, ms, PEAKS)
    assert mixed["peak_tflops"] == pytest.approx(1917.9 / 6)   # three TF32 products
    assert bf16["peak_tflops"] == fp16["peak_tflops"] == pytest.approx(1917.9)
    assert mixed["bound"] == bf16["bound"] == "alu"
    assert mixed["floor_ms"] == pytest.approx(6 * bf16["floor_ms"])


def test_triangular_route_peak_follows_its_update_product():
    """The triangular route is FP64 in every mode; its blocked updates (from
    32 right-hand sides) are Ozaki-split tensor products in every mode but
    plain FP64, whose peak is the bf16 rate over the 28 slice products."""
    for prec in ("mixed", "fp64", "bf16", "fp64_oz"):
        r = bench.large_case_roofline("lower", prec, 16384, 256, 285.8, PEAKS)
        want = fp64_peak() / 1e12 if prec == "fp64" else 1917.9 / 28
        assert r["peak_tflops"] == pytest.approx(want)
        assert r["flops"] == pytest.approx(16384.0 ** 2 * 256)
    for prec in ("mixed", "fp64"):  # few right-hand sides: the FP64 wavefront solve
        r = bench.large_case_roofline("lower", prec, 16384, 16, 30.0, PEAKS)
        assert r["peak_tflops"] == pytest.approx(fp64_peak() / 1e12)
    oz = bench.large_case_roofline("general", "fp64_oz", 16384, 1, 1000.0, PEAKS)
    assert oz["peak_tflops"] == pytest.approx(1917.9 / 28)


def test_one_rhs_triangular_solve_is_hbm_bound():
    # n^2 flops against one 8 n^2-byte read of A: far below the ridge point
    n, ms = 16384, 27.7
    r = bench.large_case_roofline("lower", "fp64", n, 1, ms, PEAKS)
    assert r["bound"] == "hbm"
    assert r["floor_ms"] == pytest.approx(8.0 * n * n / 6783.5e9 * 1e3)
    assert 0 < r["frac"] < 1


def test_oracle_verified_counts_like_the_metric(orc):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((40, 40)) + 10 * np.eye(40)
    assert bench.oracle_solve_verified(orc, A, rng.standard_normal((40, 3)))
    # a zero column: LU fails, the SVD route answers (status W_APPROX): not counted
    S = A.copy()
    S[:, 5] = 0.0
    assert not bench.oracle_solve_verified(orc, S, rng.standard_normal((40, 1)))


def test_cpu_baseline_leg_runs_on_a_small_batch(orc):
    pk = bench.make_batch("cpu", bench.SEED, count=48)
    r = bench.oracle_sample(pk, budget_s=0.2, max_threads=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["unit"] == bench.UNIT
    assert r["value"] > 0 and "systems of the same batch" in r["sample"]


@pytest.mark.parametrize("kind,cls,route", [("band5", 1, 1), ("lower", 2, 2), ("sympd", 4, 4),
                                            ("dense", 5, 6)])
def test_replica_batches_take_their_tables_routes(orc, kind, cls, route):
    """Each kind of the paper's Tables 1-4 reaches the solver its table is
    about (banded, triangular, Cholesky, LU) with an answer of status OK;
    offsets are 32-element aligned as the batched API wants."""
    from paper_2007_11208_gb300 import synth
    n, count = 100, 3
    pk = synth.replica_batch(kind, n, count, 11)
    assert all(int(o) % 32 == 0 for o in pk["a_off"]) and all(int(o) % 32 == 0 for o in pk["b_off"])
    for s in range(count):
        o, q = int(pk["a_off"][s]), int(pk["b_off"][s])
        A = pk["A"][o:o + n * n].numpy().reshape(n, n).T
        b = pk["B"][q:q + n].numpy()
        assert 0.0 <= b.min() and b.max() <= 1.0
        X, info = orc.solve(A, b)
        assert (info["cls"], info["route"], info["status"]) == (cls, route, 0)
        if kind == "band5":
            assert info["kl"] == info["ku"] == 2
        if kind == "sympd":
            assert np.array_equal(A, A.T)


def test_launch_floor_never_raises():
    # without a GPU the capture fails and the plain workload reports None
    r = bench.launch_floor_us(reps=5)
    assert r is None or r > 0


def test_oracle_large_baseline_extrapolates_by_the_route_order(orc):
    r = bench.oracle_large_baseline(["general", "lower"], [1024, 2048], n0=256)
    g, t = r["general"], r["lower"]
    assert g["n"] == t["n"] == 256 and g["measured_ms"] > 0 and t["measured_ms"] > 0
    assert g["extrapolated_ms"]["2048"] == pytest.approx(g["measured_ms"] * 8 ** 3)
    assert t["extrapolated_ms"]["1024"] == pytest.approx(t["measured_ms"] * 4 ** 2)


def test_oracle_reproduces_the_papers_band_and_triangular_savings(orc):
    """Tables 1 and 2 of the paper, on the oracle: the adaptive solve of a
    5-diagonal band or a triangular system takes a fraction of the forced
    LU solve's time (the paper reports 68-91% less; the margin here is
    wide so that a loaded host does not decide the test)."""
    r = bench.oracle_replica_tables(sizes=(250, 500), count=3)
    for kind in ("band5", "lower"):
        for row in r[kind]:
            assert row["reduction_pct"] > 50.0, (kind, row)


def test_flops_model_charges_each_pipe():
    """Mixed-route systems: FP32 factor + solves on the FP32 pipe, FP64
    residuals on the FP64 pipe; FP64-route systems: everything FP64."""
    specs = [("general", 100, 2), ("spd", 64, 1), ("ill", 50, 3)]
    infos = [dict(route=6, precision=1, ir_iters=1, detail=0),
             dict(route=4, precision=1, ir_iters=2, detail=0),
             dict(route=6, precision=0, ir_iters=0, detail=1)]
    fm = bench.flops_model(specs, infos)
    e = bench.EST_SOLVES
    lu32 = 2 / 3 * 100 ** 3 + 2 * 100 ** 2 * (2 * 2 + e) + 2 / 3 * 50 ** 3 + 2 * 50 ** 2 * e
    lu64 = 2 * 100 ** 2 * 2 * 2 + 2 / 3 * 50 ** 3 + 2 * 50 ** 2 * (3 + e) + 2 * 50 ** 2 * 3
    assert fm["flops_fp32"]["k_lu_class"] == pytest.approx(lu32)
    assert fm["flops_fp64"]["k_lu_class"] == pytest.approx(lu64)
    assert fm["flops_fp64"]["k_chol_class"] == pytest.approx(2 * 64 ** 2 * 1 * 3)
    p32, p64 = fm["peaks_tflops"]["fp32"] * 1e12, fm["peaks_tflops"]["fp64"] * 1e12
    assert fm["t_min_ms"]["k_lu_class"] == pytest.approx(max(lu32 / p32, lu64 / p64) * 1e3)
