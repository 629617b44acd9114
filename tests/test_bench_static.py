"""bench.py calls only functions it defines, imports or gets from builtins, and
its argument parser accepts the flags of the benchmark contract (CPU only, nothing is run)."""
import ast
import builtins
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_calls_are_defined():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    defined = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    imported = set()
    for n in ast.walk(tree):
        if isinstance(n, (ast.Import, ast.ImportFrom)):
            imported |= {a.asname or a.name.split(".")[0] for a in n.names}
    missing = sorted(x for x in called if x not in defined | imported and not hasattr(builtins, x))
    assert not missing, missing


def test_bench_accepts_driver_flags(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "1", "--steps", "7", "--warmup", "3"])
    a = bench.parse()
    assert a.gpus == 1 and a.steps == 7 and a.warmup == 3 and a.impl == "ours"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    assert bench.parse().impl == "reference"


def test_roofline_entry_arithmetic():
    # 10 launches of 1 ms with 2e8 candidate and 1e8 composited pairs in total at 2,070 MHz:
    # FP32 work per launch (2e7 x 27 + 1e7 x 78) = 1.32 GFLOP -> 1.32 TFLOP/s of 80.55
    sys.path.insert(0, ROOT)
    import bench
    r = bench.roofline_entry((5e8, 2e8, 1e8), {"splat_fused": [1.0] * 10}, 10,
                             {"sm_max_mhz": 2070.0}, "no-such-source", {"hbm_gbs": 6790.0})
    assert r["kernel"] == "splat_fused" and r["bound"] == "alu"
    assert abs(r["achieved"] - 1.32) < 1e-9 and abs(r["peak"] - 80.55) < 0.01
    assert r["per_launch"]["candidate_pairs"] == 2e7 and r["per_launch"]["composited_pairs"] == 1e7
    # special functions: (2e7 x 3 + 1e7 x 4) per ms = 0.1 Tops/s of 152 x 16 x 2.07 GHz
    assert abs(r["other_roofs"]["mufu"]["achieved"] - 0.1) < 1e-9
    assert abs(r["other_roofs"]["mufu"]["peak"] - 5.034) < 1e-3
    # profile-derived roofs apply only to the source they were measured on
    assert r["traffic"] is None and "issue" not in r["other_roofs"] and "hbm" not in r["other_roofs"]
    for regime in (0, 1000, 2000, 4000):
        cap = bench.CAPTURES["splat_fused"][regime]
        r2 = bench.roofline_entry((5e8, 2e8, 1e8), {"splat_fused": [1.0] * 10}, 10, {"sm_max_mhz": 2070.0},
                                  bench.CAPTURES["src_sha"], {"hbm_gbs": 6790.0}, regime=regime)
        assert r2["traffic"] == cap["dram_bytes"]
        assert abs(r2["other_roofs"]["issue"]["achieved"] - cap["warp_instructions"] / 1e6) < 0.06
        assert abs(r2["other_roofs"]["hbm"]["achieved"] - cap["dram_bytes"] / 1e6) < 0.1
    # a regime without a capture reports no traffic
    r3 = bench.roofline_entry((5e8, 2e8, 1e8), {"splat_fused": [1.0] * 10}, 10, {"sm_max_mhz": 2070.0},
                              bench.CAPTURES["src_sha"], {"hbm_gbs": 6790.0}, regime=8000)
    assert r3["traffic"] is None



def test_common_rooms_are_the_rooms_every_arm_reaches():
    import bench
    arms = {"plain": [(100, 50.0), (200, 80.0), None, (400, 10.0)],
            "batched": [(110, 40.0), (210, 60.0), (300, 90.0), (380, 95.0)],
            "batched_learned": [(50, 20.0), (100, 35.0), (120, 40.0), None]}
    common, out = bench.common_rooms(arms)
    assert common == [0, 1]
    assert out["rooms"] == 2 and out["reached"] == {"plain": 3, "batched": 4, "batched_learned": 3}
    assert out["plain"]["mean_iterations"] == 150.0 and out["batched_learned"]["mean_iterations"] == 75.0
    assert bench.common_rooms({"plain": [None], "batched": [(1, 1.0)]})[1]["rooms"] == 0
