"""The README's Python API table names only calls that exist, and the
committed profile summaries name only bench workloads that exist."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_api_names_exist():
    import paper_2606_31598_gb300 as mf
    from paper_2606_31598_gb300 import planner_sweep, rowgroup  # noqa: F401
    text = open(os.path.join(ROOT, "README.md")).read()
    table = text[text.index("Python API"):]
    for name in set(re.findall(r"`plan\.([a-z_]+)\(", table)):
        assert hasattr(mf.Plan, name), name
    for name in set(re.findall(r"`Plan\.([a-z_]+)\(", table)):
        assert hasattr(mf.Plan, name), name
    for name in set(re.findall(r"`(mf_[a-z_]+)", table)):
        assert hasattr(mf, name) or name == "mf_options" or name == "mf_plan_create", name
    for name in ("rows_cheb_begin", "rows_cheb_init", "rows_cheb_term", "rows_cheb_final"):
        assert hasattr(mf.Plan, name)
    assert hasattr(mf, "Batch") and hasattr(mf, "MLP") and hasattr(rowgroup, "propagate")


def test_profile_commands_use_existing_workloads():
    import bench  # noqa: F401
    src = open(os.path.join(ROOT, "bench.py")).read()
    choices = re.search(r'choices=\[([^\]]*)\]', src[src.index('"--workload"'):]).group(1)
    workloads = set(re.findall(r'"([a-z]+)"', choices))
    pdir = os.path.join(ROOT, "profiles")
    for fn in os.listdir(pdir):
        for w in re.findall(r"--workload ([a-z]+)", open(os.path.join(pdir, fn)).read()):
            assert w in workloads, (fn, w)
