"""The refactorisation schedule of the host symbolic phase, checked on the host.

`rf_schedule_check.cpp` (beside this file) is compiled against the library's
symbolic phase and emulates the refactorisation on the host with random values on
the pattern of A: the level updates with every group forming its bus's pivot
quantities from the raw block, against the library's schedule of pivot jobs (the
leaves' first, then each level's quads after its updates) and its pivot steps by
entry.  The factors must agree bit for bit, every sparse bus must get exactly one
pivot job in a launch before any group reads it, and a quad's lane may hold only
its own block entry.  Runs without a GPU, for several grids and dense-tail bounds.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2201_00241_gb300 import gridgen as gg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("rfcheck")
    exe = str(d / "rf_schedule_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "rf_schedule_check.cpp"),
                    os.path.join(ROOT, "paper_2201_00241_gb300", "csrc", "symbolic.cpp")], check=True)
    return exe, d


def write_grid(g, path):
    with open(path, "wb") as f:
        np.array([g.n_bus, g.n_branch], np.int32).tofile(f)
        np.array([g.order_level_cost], np.int64).tofile(f)
        np.asarray(g.fr, np.int32).tofile(f)
        np.asarray(g.to, np.int32).tofile(f)
        for a in (g.r, g.x, g.b):
            np.asarray(a, np.float64).tofile(f)
        np.asarray(g.bus_type, np.int8).tofile(f)


@pytest.mark.parametrize("case,bounds", [("tiny9", (0, 2)), ("tiny30", (0, 2, 16)), ("case118", (0, 2, 64)),
                                         ("case1354", (0, 2, 128, 256)), ("case2869", (0, 96)),
                                         ("case9241", (0, 64, 256))])
def test_refactorisation_schedule(checker, case, bounds):
    exe, d = checker
    g = gg.make_grid(9, 12, 3, 2) if case == "tiny9" else gg.make_grid(30, 41, 6, 4) if case == "tiny30" \
        else gg.make_case(case)
    path = str(d / f"{case}.bin")
    write_grid(g, path)
    for bound in bounds:
        r = subprocess.run([exe, path, str(bound)], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, (case, bound, r.stdout, r.stderr)
        fields = dict(kv.split("=") for kv in r.stdout.split())
        assert int(fields["diff_updates"]) == 0 and int(fields["missing"]) == 0
