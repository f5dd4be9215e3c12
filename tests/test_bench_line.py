"""The benchmark's stdout line: one compact JSON object with the required keys.

Builds the line from fake section data of the same shape the GPU run produces
(no GPU needed) and checks the size bound, that it is valid JSON on one line,
and that every key the benchmark contract names is present.
"""
import json

import bench

REQUIRED = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches",
            "clocks")


def _fake():
    headline = {
        "metric": "dslash_hbm_gbs", "value": 5459.2, "unit": "GB/s", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 0.0922, "dtype": "f32",
        "config": {"workload": "wilson_dslash_full_fp32_recon18_32x32x32x32", "lattice": [32, 32, 32, 32],
                   "l2": "inputs 503 MB per step > 129 MB L2, no flush"},
        "gflops": 15012.0,
        "roofline": {"bound": "hbm", "kernel": "hop_kernel<F32, 18>", "achieved": 5459.2, "peak": 6784.8,
                     "unit": "GB/s", "frac": 0.805, "traffic": 502.7e6, "mean_launch_ms": 0.0922},
        "e2e": {"value": 210.0, "unit": "GB/s", "h2d_bytes_per_step": 100663296, "d2h_bytes_per_step": 100663296,
                "ms_per_step": 2.4, "path": "pinned FP32 canonical H2D -> pack -> dslash -> unpack -> D2H"},
        "gpu_launches": 20,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 40},
        "cpu_baseline": {"value": 2.1, "unit": "GB/s", "cores": 16, "kind": "oracle", "sample": "8^4 x 900 reps",
                         "cpu_model": "Neoverse-V2", "host_threads": 16},
    }
    # detail sections as large as the real ones: a big variants table and a serving sweep
    detail = {
        "variants": {f"32x32x32x32/f32/full/r18/{k}": {"ms": 0.09, "gbs": 5400.0, "tuned": list(range(30))}
                     for k in range(200)},
        "cg": {"runs": {"m0.1/fp64": {"seconds": 0.21, "iters": 1200, "true_rel_resid": 9e-11},
                        "m0.1/fp16": {"seconds": 0.026, "iters": 1300, "true_rel_resid": 9.5e-11},
                        "m0.05/fp64": {"seconds": 0.4, "iters": 2400, "true_rel_resid": 9e-11},
                        "m0.05/fp16": {"seconds": 0.05, "iters": 2500, "true_rel_resid": 9.7e-11}}},
        "cpu_oracle_cg": {"seconds": 9.7, "iters": 1200},
        "multi_rhs": {"eo": {"multi_ms": 0.371, "singles_ms": 0.76, "multi_frac_hbm": 0.6}},
        "serving": {"rate_200": {"p50_ms": 20441.2, "p99_ms": 38679.9, "achieved_per_s": 41.15, "frac_hbm": 0.3},
                    "sweep": [{"offered_per_s": r, "p50_ms": 1.0} for r in range(100)]},
        "batch": {"graph": {"seconds": 0.23}, "persistent": {"seconds": 0.26}, "sequential": {"seconds": 0.3}},
    }
    return headline, detail


def test_headline_compact_and_complete(tmp_path):
    headline, detail = _fake()
    path = bench.write_detail(detail, str(tmp_path / "detail.json"))
    assert path is not None
    line = bench.compose_headline(headline, detail, path)
    text = json.dumps(line, separators=(",", ":"))
    assert "\n" not in text
    assert len(text.encode()) <= bench.HEADLINE_MAX_BYTES, len(text)
    back = json.loads(text)
    for k in REQUIRED:
        assert k in back, k
    assert back["impl"] == "wdirac"
    assert back["value"] > 0
    assert back["config"]["workload"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in back["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in back["cpu_baseline"], k
    assert "cpu_model" not in back["cpu_baseline"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in back["e2e"], k
    sec = back["secondary"]
    assert sec["cg_24x24x24x48_m0.1"]["speedup"] == round(0.21 / 0.026, 2)
    assert sec["serving_200_per_s"]["p99_ms"] == 38679.9
    assert sec["cpu_oracle_cg_24x24x24x48_m0.1_s"] == 9.7
    # the bulky sections stay in the detail file
    assert "variants" not in back and "sweep" not in text
    with open(path) as f:
        assert len(json.load(f)["variants"]) == 200


def test_headline_without_optional_sections():
    headline, _ = _fake()
    del headline["cpu_baseline"]
    line = bench.compose_headline(headline, {}, None)
    assert "secondary" not in line and "cpu_baseline" not in line
    assert line["detail"] is None
    json.loads(json.dumps(line))
