"""bench.py runs only where a GPU is: a static check here catches a name that a refactor
left undefined in one of its functions (a NameError there would otherwise show only on a
GPU machine)."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _undefined_names(path):
    tree = ast.parse(open(path).read())
    module = set()
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            module.add(n.name)
        elif isinstance(n, ast.Assign):
            module.update(t.id for t in n.targets if isinstance(t, ast.Name))
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            module.update((a.asname or a.name).split(".")[0] for a in n.names)
    bad = []

    def check(fn, outer):
        local = set(outer) | {a.arg for a in fn.args.args + fn.args.kwonlyargs}
        if fn.args.vararg:
            local.add(fn.args.vararg.arg)
        if fn.args.kwarg:
            local.add(fn.args.kwarg.arg)
        for n in ast.walk(fn):
            if isinstance(n, (ast.Import, ast.ImportFrom)):
                local.update((a.asname or a.name).split(".")[0] for a in n.names)
            elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
                local.add(n.id)
            elif isinstance(n, (ast.FunctionDef, ast.Lambda)) and n is not fn:
                if isinstance(n, ast.FunctionDef):
                    local.add(n.name)
                local.update(a.arg for a in n.args.args)
            elif isinstance(n, ast.ExceptHandler) and n.name:
                local.add(n.name)
            elif isinstance(n, ast.arg):
                local.add(n.arg)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load):
                if n.id not in local and n.id not in module and not hasattr(builtins, n.id):
                    bad.append((fn.name, n.id, n.lineno))

    for n in tree.body:
        if isinstance(n, ast.FunctionDef):
            check(n, ())
    return bad


def test_bench_functions_reference_defined_names():
    assert _undefined_names(os.path.join(ROOT, "bench.py")) == []
