"""The benchmark's headline line (the last line bench.py prints) stays short and carries the
contract's keys; the detailed sections go out on earlier lines. The roofline names the lower of
the two ceilings as the bound."""
import json
import types

import bench


def _plan():
    return types.SimpleNamespace(n_master_sectors=4194304, n_files=20000)


def _args(**kw):
    a = dict(steps=20, warmup=5, config="scale", kernel_config=0, sections_out="", signature=0)
    a.update(kw)
    return types.SimpleNamespace(**a)


INT_PEAK = {"mixed_ops_per_s": 39.2, "alu_ops_per_s": 20.1, "fma_ops_per_s": 20.1}


def _full_line():
    args = _args()
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 40, "power_w_max": 900.0}
    roof = bench.scan_roofline(7.2, 67108864, 160000, clocks, INT_PEAK, args)
    roof.pop("detail")
    e2e = {"value": 200.0, "unit": "GB/s", "h2d_bytes_per_step": 1 << 35, "d2h_bytes_per_step": 16 * 1500000,
           "frac_of_h2d_link": 0.95, "steps": 3, "h2d_link_GBps": 210.0, "streamed_128GiB": {"GBps": 200.0}}
    cpu = {"value": 2.4, "unit": "GB/s", "cores": 16, "kind": "oracle",
           "sample": "24 windows of 2097152 sectors (1 GiB each) at seeded offsets of the image; lookup only, "
                     "signature database of 4194304 master sectors built untimed", "seconds": 10.0,
           "matches_in_sample": 1000, "single_core_GBps": 0.14}
    batched = {"graph_GBps": 4400.0, "speedup_vs_sequential": 4.5, "bit_exact_vs_plant_log": True, "other": "x" * 500}
    served = {"p50_ms": 0.4, "p99_ms": 200.0, "throughput_GBps": 40.0, "bit_exact_vs_plant_log": True,
              "workload": "y" * 500}
    return bench.headline(value=4600.0, world=1, args=args, ms=7.4, nbytes=1 << 35, sectors=67108864, plan=_plan(),
                          kernel_config="default", matches=1500000, exact=True, roof=roof, clocks=clocks, e2e=e2e,
                          cpu=cpu, launches=100, batched=batched, served=served)


def test_headline_is_short_and_complete():
    line = _full_line()
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) <= 2048, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "cpu_baseline", "gpu_launches",
              "p99_served_ms"):
        assert k in line, k
    assert line["metric"] == bench.METRIC
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert "workload" in line["config"]


def test_roofline_names_the_lower_ceiling(monkeypatch):
    args = _args()
    # HBM below the integer ceiling at 2,070 MHz (7.23 TB/s of image): the bound is HBM
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6789.0})
    r = bench.scan_roofline(7.2, 67108864, 0, {"sm_mhz": 2070.0}, INT_PEAK, args)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6789.0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    # achieved counts the image bytes and the per-tile counts of one launch
    alg = 67108864 * 512 + (67108864 // 32) * 12
    assert abs(r["achieved"] - alg / 7.2e-3 / 1e9) < 1e-6
    # at a low clock the integer ceiling is the lower one
    r = bench.scan_roofline(7.2, 67108864, 0, {"sm_mhz": 1000.0}, INT_PEAK, args)
    assert r["bound"] == "alu" and r["unit"] == "Top/s"
    assert abs(r["peak"] - 152 * 128 * 1000e6 / 1e12) < 1e-9


def test_sections_are_separate_lines(capsys, tmp_path):
    out = tmp_path / "s.jsonl"
    args = _args(sections_out=str(out))
    bench.emit_section(args, "tables", {"a": 1})
    bench.emit_section(args, "fragments", {"b": 2})
    lines = capsys.readouterr().out.strip().splitlines()
    assert [json.loads(x)["section"] for x in lines] == ["tables", "fragments"]
    assert out.read_text().strip().splitlines() == lines
