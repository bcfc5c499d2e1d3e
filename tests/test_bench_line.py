"""bench.py's last stdout line: one short JSON object (well under 2 KB) with the metric on
the quoted workload, its end-to-end form, the dominant kernel's roofline, the CPU baseline,
the clocks and a one-number summary per section; the full result goes to a file."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _full_result():
    sweep = [{"rate_req_s": r, "offered_inferences_s": 4.5 * r, "inferences_s": 4.4 * r, "requests": 1000,
              "batches": 900, "p50_ms": 2.0, "p99_ms": 6.0} for r in (10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0)]
    mix = [{"rate_req_s": r, "offered_inferences_s": 4.5 * r, "inferences_s": 4.4 * r,
            "per_net": [{"net": n, "inferences_s": 2.0 * r, "requests": 500, "batches": 400,
                         "max_in_flight_ciphertexts": 40, "p50_ms": 2.0, "p99_ms": 9.0} for n in ("small", "large")]}
           for r in (100.0, 300.0, 1000.0)]
    stages = {"stage_%d" % i: 0.1 * i for i in range(12)}
    return {
        "metric": bench.METRIC, "value": 1149.9, "unit": bench.UNIT, "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 0.87, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "p50_ms": 0.86, "p99_ms": 0.89, "gpu_launches": 2100,
        "config": {"workload": "x" * 300,
                   "workload_short": "small: N=2^14, q=60+7x40, p=60 bits, FC 2048->128->x^2->FC 128->2, "
                                     "1 clip(s) in 1 ciphertext(s)",
                   "parallelism": "single", "l2": "no flush",
                   "fc_form": {"fc_n1": 32, "hoist_moddown": True, "hoist_sums": True, "tuned": [{"ms": 1.0}] * 12},
                   "ntt_table": "3" * 32, "ks_table": "1" * 24,
                   "pdl_launches_captured": 500},
        "e2e": {"value": 1062.0, "unit": bench.UNIT, "h2d_bytes_per_step": 2097152, "d2h_bytes_per_step": 1310720},
        "roofline": {"bound": "alu", "kernel": "ntt_fwd", "achieved": 470.1234, "peak": 1500.0,
                     "unit": "G butterflies/s", "frac": 0.3134, "traffic": 9.18e6, "peak_kind": "measured " * 20,
                     "derived_alu_frac": 0.17, "hbm_achieved_gbs": 542.0, "hbm_peak_gbs": 6800.0,
                     "hbm_frac": 0.0797, "algorithmic_bytes_per_call": 1.262e7, "avg_call_us": 23.3},
        "roofline_keyswitch": {"bound": "hbm", "kernel": "k_ks_inner", "achieved": 4480.123, "peak": 6800.0,
                               "unit": "GB/s", "frac": 0.6588, "peak_kind": "fallback",
                               "algorithmic_bytes_per_call": 5.1e7, "calls_per_step": 8.0},
        "ntt": {"achieved_gbs": 300.0}, "stages_ms_per_step": stages,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 30},
        "cpu_baseline": {"value": 1.76, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                         "sample": "18 whole ciphertext evaluation(s) of 1 clip(s) each, 10.2 s"},
        "served": {"workload": "w" * 200, "sweep": sweep},
        "served_c5": {"workload": "w" * 200, "sweep": sweep},
        "served_mix": {"workload": "w" * 200, "sweep": mix},
        "batched": {"value": 1975.0, "vs_plain": 1.72, "stages_ms_per_step": stages},
        "batched_small": {"rows": [{"clips": c, "value": 8000.0 + c, "vs_plain": 7.0} for c in (128, 512, 512)]},
        "min_start_level": {"small": {"value": 1832.0}, "large": {"value": 6403.0}},
        "ragged_mix": {"value": 4132.0},
        "batched_simd": {"rows": [{"value": 257100.0, "vs_plain": 224.0, "roofline": {"frac": 0.737}}] * 3},
        "cnn": {"batches": [{"ms": 8.9}, {"ms": 114.8}]},
        "conv_table1": {"rows": [{"speedup": 1.0 + i} for i in range(8)]},
    }


def test_headline_is_short_and_complete(tmp_path):
    full = _full_result()
    path = bench.write_sections(full, str(tmp_path / "sections.json"))
    assert path and json.load(open(os.path.join(ROOT, path) if not os.path.isabs(path) else path))["served"]
    line = json.dumps(bench.headline(full, path), separators=(",", ":"))
    # realistic field contents (the longest the bench prints) stay well under 2 KB
    assert len(line) < 1900, len(line)
    h = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "cpu_baseline", "clocks", "gpu_launches",
              "p50_ms", "p99_ms"):
        assert k in h, k
    assert h["config"]["workload"].startswith("small")
    assert set(h["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert h["roofline_keyswitch"]["bound"] == "hbm" and h["roofline_keyswitch"]["frac"] == 0.6588
    assert h["e2e"]["h2d_bytes_per_step"] == 2097152
    assert h["summary"]["served_c5"]["rate_req_s"] == 2000.0
    assert h["value"] == full["value"]


def test_keyswitch_roofline_sums_every_form():
    # stages: name -> (launches, ms, algorithmic bytes) over psteps profiled steps
    stages = {"k_ks_inner<8>": (8, 0.5, 2.0e9), "k_ks_inner<16>": (2, 0.5, 1.0e9), "ntt_fwd": (40, 1.0, 1.0e9)}
    r = bench.ks_roofline(stages, 2)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 3.0e9 / 1e-3 / 1e9) < 1e-6          # 3 GB in 1 ms
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["calls_per_step"] == 5.0 and abs(r["stage_share"] - 0.5) < 1e-12
    assert bench.ks_roofline({"ntt_fwd": (1, 1.0, 1.0)}, 1) is None
