"""bench.py's command line on CPU: which secondary figures --extras selects."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_all_selects_every_figure_in_order():
    # the co-runner on its own is part of bfs_rmat22 in a full run
    assert bench.selected_extras("all") == tuple(x for x in bench.EXTRAS if x != "corunner")
    assert len(set(bench.EXTRAS)) == len(bench.EXTRAS)
    assert bench.selected_extras("corunner") == ("corunner",)


def test_subset_keeps_the_fixed_order_and_ignores_spaces():
    got = bench.selected_extras(" serving, octree ,topology_driven_sssp")
    assert got == ("topology_driven_sssp", "octree", "serving")
    assert bench.selected_extras("octree,octree") == ("octree",)


def test_unknown_name_is_refused():
    with pytest.raises(SystemExit):
        bench.selected_extras("octree,nonsense")


def test_unknown_name_fails_before_any_work():
    """The command line is checked before torch, the library or a GPU is touched."""
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--extras", "nonsense"],
                         capture_output=True, text=True, timeout=120)
    assert res.returncode != 0
    assert "unknown --extras" in (res.stderr + res.stdout)
