"""Every name a function of bench.py, __graft_entry__.py or the Python
package loads is defined somewhere it can see (a parameter, a local, an
import, a module-level name or a builtin).  bench.py's GPU paths only run on
a GPU, so a misplaced name there would otherwise surface only in the
driver's timed run."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2605_25872_gb300")
FILES = [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")] + sorted(
    os.path.join(PKG, f) for f in os.listdir(PKG) if f.endswith(".py"))


def _bound_in(node):
    names = set()
    for n in ast.walk(node):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            names |= {(a.asname or a.name).split(".")[0] for a in n.names}
        elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
            if not isinstance(n, ast.Lambda):
                names.add(n.name)
            a = n.args
            names |= {x.arg for x in a.args + a.kwonlyargs + a.posonlyargs}
            names |= {x.arg for x in (a.vararg, a.kwarg) if x is not None}
        elif isinstance(n, ast.ClassDef):
            names.add(n.name)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            names |= set(n.names)
    return names


def _module_names(tree):
    """Names bound by top-level statements (not inside function bodies), plus
    names that a function declares global."""
    names = set()
    for st in tree.body:
        if isinstance(st, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(st.name)
            continue
        stack = [st]
        while stack:
            n = stack.pop()
            if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda, ast.ClassDef)):
                if not isinstance(n, ast.Lambda):
                    names.add(n.name)
                continue
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store):
                names.add(n.id)
            elif isinstance(n, (ast.Import, ast.ImportFrom)):
                names |= {(a.asname or a.name).split(".")[0] for a in n.names}
            stack.extend(ast.iter_child_nodes(n))
    for n in ast.walk(tree):
        if isinstance(n, ast.Global):
            names |= set(n.names)
    return names


def undefined_names(path):
    tree = ast.parse(open(path).read(), path)
    module = _module_names(tree)
    parent = {c: p for p in ast.walk(tree) for c in ast.iter_child_nodes(p)}
    bad = []
    for fn in (n for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef))):
        visible = _bound_in(fn) | module
        up = parent.get(fn)
        while up is not None:             # closures see their enclosing functions' names
            if isinstance(up, (ast.FunctionDef, ast.AsyncFunctionDef)):
                visible |= _bound_in(up)
            up = parent.get(up)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load):
                if n.id not in visible and not hasattr(builtins, n.id) and n.id != "__file__":
                    bad.append(f"{os.path.basename(path)}:{n.lineno} {fn.name}: {n.id}")
    return bad


@pytest.mark.parametrize("path", FILES, ids=lambda p: os.path.relpath(p, ROOT))
def test_no_undefined_names(path):
    assert undefined_names(path) == []


def test_the_check_catches_a_name_used_out_of_its_scope(tmp_path):
    # a function reading main()'s local `args` (a NameError only when it runs)
    src = open(FILES[0]).read().replace("def micsa_measure(dev, J, seeds, n_emcs=10):",
                                        "def micsa_measure(dev, J, seeds, n_emcs=10):\n    if args.tuned:\n        pass", 1)
    p = tmp_path / "bench.py"
    p.write_text(src)
    assert [b.split()[-1] for b in undefined_names(str(p))] == ["args"]
