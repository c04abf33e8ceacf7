"""CPU checks of the benchmark line's compact summary: the last key of the
JSON line repeats every block's numbers (so a reader that keeps only the end
of the line still has them) and stays short."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _blocks():
    fmt = lambda m, f, e: {"mlups": m, "frac_of_measured_hbm": f, "rel_l2_u": e}
    formats = {"fp64": dict(fmt(4141.2, 0.0879, 0.0), roofline={"frac": 1.0051}),
               "fp32": fmt(85113.4, 0.9031, 3.84e-05), "fp16": fmt(176993.1, 0.9391, 0.00731),
               "bf16": fmt(179347.0, 0.9513, 0.0155), "fp16_sr": fmt(162715.3, 0.8634, 0.000538),
               "bf16_sr": fmt(166882.9, 0.8851, 0.00431)}
    obstacles = {"formats": {k: fmt(v["mlups"] * 0.8, v["frac_of_measured_hbm"] * 0.8, 0.001)
                             for k, v in formats.items()},
                 "fastest_within_bound": "fp16_sr", "speedup_vs_fp64_at_bound": 31.7}
    batch = {"mlups": 79005.2, "frac_of_measured_hbm": 0.8513, "tuning": [16, 1, 2, 0],
             "mode": {"persistent": 1, "resident": 1, "order": 0}, "speedup_vs_sequential": 2.54,
             "errors": {"e2_median": 0.000378, "order_steady_heights_median": 2.0016}}
    config2 = {"formats": {"fp64": {"mlups": 3878.2, "transpose_residual_u": 7e-15},
                           "fp32": {"mlups": 108056.1, "transpose_residual_u": 3.8e-06, "rel_l2_u": 0.000107}}}
    extras = {"shan_chen_fp32_4096": {"mlups": 50932.3, "frac_of_measured_hbm": 0.8702},
              "forcing_m2_fp32_8192": {"mlups": 84144.0, "frac_of_measured_hbm": 0.8932}}
    return formats, obstacles, batch, config2, extras


def test_summary_repeats_every_block():
    b = _bench()
    s = b.summary(*_blocks())
    assert set(s) >= {"key", "formats_8192", "obstacles_16384x8192", "obstacles_fastest_within_1e-3",
                      "batch_256", "config2_1024_l2_resident", "config2_key", "extras"}
    assert s["formats_8192"]["fp16"] == [176993, 0.939, 0.0073]
    assert s["formats_8192"]["fp64"][1] == 1.01          # FP64 against its ALU roof
    assert s["batch_256"]["mode"] == [16, 1, 2, 0, 1, 1, 0]
    assert s["extras"]["shan_chen_fp32_4096"] == [50932, 0.87]


def test_summary_is_short_and_skips_missing_blocks():
    b = _bench()
    full = json.dumps(b.summary(*_blocks()))
    assert len(full) < 1600
    only = b.summary(None, None, None, None, None)
    assert set(only) == {"key"}
