"""bench.py's single-network workloads: the configurations its lines are quoted on
(sector counts, bond dimensions, sector scaling and the names in the line)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name,chi,nsec,scaled", [("chi512", 512, 21, False), ("chi2048", 2048, 41, True),
                                                  ("chi4096", 4096, 81, True), ("dense32", 32, 1, False)])
def test_workload_table(name, chi, nsec, scaled):
    sys.path.insert(0, ROOT)
    import bench
    wl, wname = bench.workload(name)
    assert wl.chi == chi
    assert len(wl.left_sectors) == nsec and sum(d for _, d in wl.left_sectors) == chi
    assert wl.sector_scale == scaled
    assert f"chi{chi}" in wname and ("sectorscaled" in wname) == scaled and wname.endswith("lanczos20")
    assert bench.WORKLOAD_NAMES[name] == wname   # the oracle sample of the CPU baseline finds it by that name
