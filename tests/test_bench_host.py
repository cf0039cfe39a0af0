"""Host-side arithmetic of bench.py (no GPU): the roofline object of the dominant kernel
and the parsing of the clock samples that decide whether a run is rejected."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = ({"hbm_gbs": 6698.5, "bf16_tflops": 1938.1}, "measured")


def test_roofline_of_the_solver(bench):
    # 4 launches moving 2 GB each in 1.0 ms each: 2,000 GB/s
    r = bench.roofline(2, 10, 3.0, 1e9, 4, 4.0, 8e9, *PEAKS)  # the solver dominates (4 ms > 3 ms)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(2000.0) and r["frac"] == pytest.approx(2000.0 / 6698.5)
    assert r["traffic"] == pytest.approx(bench.PCG_TRAFFIC_RATIO * 2e9)
    assert bench.roofline(1, 10, 3.0, 1e9, 4, 4.0, 8e9, *PEAKS)["traffic"] is None


def test_roofline_of_the_far_field(bench):
    # DF64: 2 launches of 1e8 entries in 10 ms each
    r = bench.roofline(2, 2, 20.0, 2e8, 1, 1.0, 1e9, *PEAKS)
    assert r["bound"] == "alu" and r["traffic"] is None
    ops = 1e8 * bench.DF_FAR_OPS_PER_ENTRY
    assert r["achieved"] == pytest.approx(ops / 0.010 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_PEAK_TOPS)
    # FP32: 49 reciprocal square roots per entry against the MUFU issue peak
    r32 = bench.roofline(1, 2, 20.0, 2e8, 1, 1.0, 1e9, *PEAKS)
    assert r32["achieved"] == pytest.approx(1e8 * 49 / 0.010 / 1e12)
    assert r32["peak"] == pytest.approx(152 * 16 * 2.07e9 / 1e12)


def test_percentile(bench):
    xs = [5.0, 1.0, 4.0, 2.0, 3.0]
    assert bench._pct(xs, 0.5) == 3.0 and bench._pct(xs, 0.99) == 5.0 and bench._pct(xs, 0.0) == 1.0


def test_clock_samples_and_throttle_reasons(bench, tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 400.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 650.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.p = _Done()
    c.f = open(os.devnull, "w")
    out = c.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["power_w_max"] == 1390.0


def test_oracle_baseline_threads(bench):
    """The cpu_baseline leg on a tiny case: all cores and one thread run the same oracle
    (the oracle's reductions are sequential, so the Cap does not depend on threads)."""
    import oracle

    b = bench.oracle_baseline(max_n=700, max_n_1t=700)
    assert b["kind"] == "oracle" and b["cores"] >= 1 and b["value"] > 0
    assert b["threads"]["one_thread_runs_per_s"] > 0 and b["threads"]["all_cores_runs_per_s"] > 0
    assert oracle.num_threads() == b["cores"]  # restored
    oracle.set_num_threads(1)
    try:
        h1 = oracle.adaptive_run(*[getattr(bench_inputs(), k) for k in ("verts", "tris")], max_N=700)
    finally:
        oracle.set_num_threads(0)
    hn = oracle.adaptive_run(*[getattr(bench_inputs(), k) for k in ("verts", "tris")], max_N=700)
    assert [h["cap"] for h in h1] == [h["cap"] for h in hn]


def bench_inputs():
    from paper_1901_08393_gb300 import inputs

    return inputs.workload_polycube_adaptive()
