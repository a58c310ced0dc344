"""bench.py's host-side helpers on CPU: every name it loads is bound (a
missing helper would only show on the GPU, in the middle of a run), and the
traffic tables and writer rooflines keep their shapes."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _unbound_names(path):
    tree = ast.parse(open(path).read())
    bound = set(dir(builtins)) | {"__file__", "__name__"}
    for n in ast.walk(tree):
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            bound.add(n.name)
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            bound.add(n.id)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            bound.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.arg):
            bound.add(n.arg)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            bound.add(n.name)
    loads = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    return sorted(loads - bound)


@pytest.mark.parametrize("rel", ["bench.py", "__graft_entry__.py", "paper_2607_02543_gb300/binding.py",
                                 "paper_2607_02543_gb300/serve.py", "paper_2607_02543_gb300/experiments.py",
                                 "paper_2607_02543_gb300/workloads.py", "paper_2607_02543_gb300/build.py"])
def test_no_unbound_names(rel):
    assert _unbound_names(os.path.join(ROOT, rel)) == []


def test_traffic_tables():
    import bench
    from paper_2607_02543_gb300.binding import WORK_KINDS
    t = bench.writer_traffic("int256-1m-d128")
    assert isinstance(t, dict) and set(t) <= set(WORK_KINDS)
    assert all(v > 0 for v in t.values())
    assert bench.writer_traffic("gauss64-10k-d128") == {}
    s = bench.search_traffic("int256-1m-d128", 1000.0)
    assert s is None or s > 0
    assert bench.search_traffic("gauss64-10k-d128", 1000.0) is None


def test_writer_rooflines():
    import bench
    work = {"prune": (3_000_000, 1_000_000), "compact": (0, 2_000_000), "refine": (0, 0)}
    prof = {"prune": (2.0, 4), "compact": (1.0, 2)}
    out = bench.writer_rooflines(work, prof, 2, 1000.0, "measured", {"prune": 5_000_000})
    assert set(out) == {"prune", "compact"}
    p = out["prune"]
    assert p["alg_bytes_per_step"] == 2_000_000 and p["ms_per_step"] == 1.0 and p["launches_per_step"] == 2
    assert p["achieved"] == pytest.approx(2.0)          # 2 MB in 1 ms = 2 GB/s
    assert p["frac"] == pytest.approx(0.002)
    assert p["traffic_per_step"] == 5_000_000 and out["compact"]["traffic_per_step"] is None
