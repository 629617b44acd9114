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
