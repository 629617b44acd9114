"""Every function and method of the repository's Python modules binds every
name it reads (locally, in an enclosing function, at module level, or as a
builtin).  Much of this code runs only on a GPU; this catches a name lost in a
refactor on the CPU, before any run."""
import ast
import builtins
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "paper_2412_03451_gb300", "*.py")) +
               [os.path.join(ROOT, "__graft_entry__.py"), os.path.join(ROOT, "bench.py")] +
               glob.glob(os.path.join(ROOT, "oracle", "*.py")) +
               glob.glob(os.path.join(ROOT, "tests", "*.py")))


def _imported(node):
    return {(a.asname or a.name).split(".")[0] for a in node.names}


def _module_names(tree):
    names = set(dir(builtins)) | {"__file__", "__name__"}
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            names |= _imported(n)
        else:
            # assignments, and names bound inside module-level if / try / for / with blocks
            for x in ast.walk(n):
                if isinstance(x, ast.Name) and isinstance(x.ctx, ast.Store):
                    names.add(x.id)
                elif isinstance(x, (ast.Import, ast.ImportFrom)):
                    names |= _imported(x)
                elif isinstance(x, (ast.FunctionDef, ast.ClassDef)):
                    names.add(x.name)
    return names


def _unbound(func, module):
    bound = set()
    for x in ast.walk(func):
        if isinstance(x, ast.Name) and isinstance(x.ctx, (ast.Store, ast.Del)):
            bound.add(x.id)
        elif isinstance(x, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
            if not isinstance(x, ast.Lambda):
                bound.add(x.name)
            a = x.args
            bound |= {y.arg for y in a.args + a.kwonlyargs + a.posonlyargs}
            bound |= {y.arg for y in (a.vararg, a.kwarg) if y is not None}
        elif isinstance(x, ast.ClassDef):
            bound.add(x.name)
        elif isinstance(x, (ast.Import, ast.ImportFrom)):
            bound |= _imported(x)
        elif isinstance(x, ast.ExceptHandler) and x.name:
            bound.add(x.name)
    loads = {x.id for x in ast.walk(func) if isinstance(x, ast.Name) and isinstance(x.ctx, ast.Load)}
    return sorted(loads - bound - module)


@pytest.mark.parametrize("path", FILES, ids=lambda p: os.path.relpath(p, ROOT))
def test_functions_bind_every_name_they_read(path):
    tree = ast.parse(open(path).read())
    module = _module_names(tree)
    funcs = [n for n in tree.body if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef))]
    for c in (n for n in tree.body if isinstance(n, ast.ClassDef)):
        funcs += [m for m in c.body if isinstance(m, (ast.FunctionDef, ast.AsyncFunctionDef))]
    bad = {f.name: _unbound(f, module) for f in funcs}
    assert not {k: v for k, v in bad.items() if v}
