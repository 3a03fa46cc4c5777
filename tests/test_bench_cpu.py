"""Host logic of bench.py on CPU: the kernel-class breakdown, the roofline
object built from the library's event profiler, and the clock sampler's
parsing (fed a fake nvidia-smi process)."""
import math

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def prof_entry(launches=0, ms=0.0, bytes_=0.0, flops=0.0):
    return {"launches": launches, "ms": ms, "bytes": bytes_, "flops": flops}


def empty_prof(bench):
    return {c: prof_entry() for c in bench.CLASS_KERNELS}


def test_breakdown_shares(bench):
    prof = empty_prof(bench)
    prof["hpsi_sparse"] = prof_entry(26, 5.0)
    prof["features"] = prof_entry(4, 2.0)
    out = bench.breakdown(prof, 10.0)
    assert set(out) == {"hpsi_sparse", "features"}      # classes that never ran are left out
    assert out["hpsi_sparse"] == {"launches": 26, "ms": 5.0, "share_of_step": 0.5}
    assert out["features"]["share_of_step"] == 0.2


def test_roofline_picks_the_longest_class_with_known_work(bench):
    peaks = {"hbm_gbs": 6712.6}
    prof = empty_prof(bench)
    # the longest class has no known work: it is named as dominant only
    prof["sparse_excite"] = prof_entry(51, 9.0)
    prof["features"] = prof_entry(4, 2.0, bytes_=4 * 1.0e9)
    prof["reduce"] = prof_entry(26, 1.0, bytes_=26 * 1.0e6)
    r = bench.step_roofline(prof, peaks, "measured", 80.5)
    assert r["kernel_class"] == "features" and r["dominant_class"] == "sparse_excite"
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    gbs = 4.0e9 / (2.0e-3) / 1e9
    assert math.isclose(r["achieved"], round(gbs, 1))
    assert math.isclose(r["frac"], round(gbs / 6712.6, 4))
    assert r["bytes_per_launch"] == 1.0e9
    assert r["traffic"] is None


def test_timed_region_records_the_roofline_class_only(bench):
    """The class the timed region records is the one the roofline reports
    from a fully recorded warm-up job, and the roofline built from a
    one-class record names the warm-up's dominant class."""
    peaks = {"hbm_gbs": 6696.8}
    warm = empty_prof(bench)
    warm["sparse_excite"] = prof_entry(210, 9.0)          # longest, no known work
    warm["hpsi_sparse"] = prof_entry(105, 5.0, bytes_=105 * 49.0e6)
    warm["screen_sparse"] = prof_entry(10, 2.8)
    warm["reduce"] = prof_entry(1, 0.01, bytes_=1.0e6)
    assert bench.roofline_class(warm) == "hpsi_sparse"
    assert bench.roofline_class(empty_prof(bench)) is None
    timed = empty_prof(bench)
    timed["hpsi_sparse"] = prof_entry(525, 26.0, bytes_=525 * 49.0e6)
    r = bench.step_roofline(timed, peaks, "measured", 80.5, dominant="sparse_excite")
    assert r["kernel_class"] == "hpsi_sparse" and r["dominant_class"] == "sparse_excite"
    assert math.isclose(r["achieved"], round(525 * 49.0e6 / 26.0e-3 / 1e9, 1))


def test_roofline_alu_class_uses_flops(bench):
    prof = empty_prof(bench)
    prof["hpsi"] = prof_entry(2, 400.0, bytes_=2 * 1.3e9, flops=2 * 20.0e12)
    r = bench.step_roofline(prof, {"hbm_gbs": 6712.6}, "measured", 80.5)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    tf = 40.0e12 / 0.4 / 1e12
    assert math.isclose(r["achieved"], round(tf, 3))
    assert math.isclose(r["frac"], round(tf / 80.5, 4))


def test_traffic_record_follows_the_kernel_sources(bench, tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu record of the class and
    turns None once the class's kernel sources differ from the hashed ones."""
    import json
    f = tmp_path / "traffic.json"
    good = bench.source_hash(bench.CLASS_SOURCES["hmat"])
    f.write_text(json.dumps({
        "hmat": {"dram_bytes_per_launch": 1.5e9, "workload": "w", "source_sha": good},
        "features": {"dram_bytes_per_launch": 2.0e6, "workload": "w", "source_sha": "stale"}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_for("hmat") == (1.5e9, "w")
    assert bench.traffic_for("features") == (None, "w")
    assert bench.traffic_for("reduce") == (None, None)
    prof = empty_prof(bench)
    prof["features"] = prof_entry(4, 2.0, bytes_=4 * 1.0e9)
    assert bench.step_roofline(prof, {"hbm_gbs": 6712.6}, "measured", 80.5)["traffic"] is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.traffic_for("hmat") == (None, None)


def test_screens_used_counts_each_iteration(bench):
    jobs = [([{"screen": 1}, {"screen": 1}, {"screen": 2}], -1.0, 0.1),
            ([{"screen": 3}, {"screen": 0}], -1.0, 0.1)]
    assert bench.screens_used(jobs) == {"exact_sparse": 2, "ranker": 1, "ranker_then_full": 1,
                                        "exact_dense": 1}


def test_roofline_without_known_work(bench):
    prof = empty_prof(bench)
    prof["sparse_excite"] = prof_entry(10, 1.0)
    r = bench.step_roofline(prof, {"hbm_gbs": 6712.6}, "measured", 80.5)
    assert r["achieved"] is None and r["frac"] is None
    assert r["dominant_class"] == "sparse_excite"


class _FakeSmi:
    def __init__(self, text):
        self.text = text
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_sampler_parsing(bench):
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1390.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
    ]
    c = bench.Clocks(0)
    c.proc = _FakeSmi("\n".join(rows) + "\n")
    out = c.stop()
    assert c.proc.terminated
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(bench):
    c = bench.Clocks(0)
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_job_throughput_counts_all_ranks(bench):
    # 4 iterations on each of 2 ranks in 10 ms (max over ranks): 800 iterations/s
    assert math.isclose(bench.job_throughput(2, 4, 10.0), 800.0)


def test_c_tilde(bench):
    # the paper's amortised coefficient: j iterations in T_j seconds -> j / sqrt(T_j)
    recs = [{"t_total": 0.25}, {"t_total": 0.5}, {"t_total": 0.25}]
    c = bench.c_tilde(recs)
    assert c["iterations"] == 3 and math.isclose(c["t_s"], 1.0)
    assert math.isclose(c["value"], 3.0)
    assert bench.c_tilde([])["value"] is None
