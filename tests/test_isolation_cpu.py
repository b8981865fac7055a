"""The oracle is test infrastructure: the product path neither imports nor
links it, and the two implementations share no code. Checked by reading the
sources (no GPU needed)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1407_2737_gb300")


def _oracle_imports(path):
    """(enclosing function or None, line) of every import of the oracle."""
    tree = ast.parse(open(path).read(), filename=path)
    found = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            mods = []
            if isinstance(child, ast.Import):
                mods = [a.name for a in child.names]
            elif isinstance(child, ast.ImportFrom):
                mods = [child.module or ""] + [a.name for a in child.names]
            if any(m == "oracle" or m.startswith("oracle.") for m in mods):
                found.append((fn, child.lineno))
            visit(child, name)

    visit(tree, None)
    return found


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True)
    assert files
    for f in files:
        assert _oracle_imports(f) == [], f


def test_bench_and_entry_use_the_oracle_only_in_their_cpu_legs():
    allowed = {"bench.py": {"cpu_oracle_sample", "run_row", "run_reference"},
               "__graft_entry__.py": {"build", "smoke"}}
    for name, fns in allowed.items():
        uses = _oracle_imports(os.path.join(ROOT, name))
        assert uses, name
        for fn, line in uses:
            assert fn in fns, (name, fn, line)


def test_cuda_path_and_oracle_share_no_code():
    native = [f for f in glob.glob(os.path.join(PKG, "csrc", "**", "*"), recursive=True)
              if os.path.isfile(f)] + glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert native
    for f in native:
        text = open(f).read()
        assert "kmc_oracle" not in text and not re.search(r'#include\s*[<"][^>"]*oracle', text), f
    ours = {os.path.basename(f) for f in native}
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read()):
            assert os.path.basename(inc) not in ours, (f, inc)


def test_nothing_committed_reads_work_files():
    work = "_" + "work" + os.sep  # the git-ignored scratch folder
    for f in glob.glob(os.path.join(ROOT, "**", "*.py"), recursive=True):
        rel = os.path.relpath(f, ROOT)
        if rel.startswith(work) or rel.startswith("baseline" + os.sep):
            continue
        assert work not in open(f).read(), rel
