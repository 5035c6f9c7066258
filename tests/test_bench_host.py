"""Host logic of bench.py (no GPU): the oracle sample lattices, the
algorithmic byte counts behind the roofline, and the workload recipes."""
import math

import pytest

import bench
from paper_2212_12559_gb300 import inputs


@pytest.mark.parametrize("cfg", sorted(inputs.CONFIGS))
def test_sample_dims_keep_level_structure(cfg):
    """The oracle sample lattice keeps every coarsening (each aggregate
    extent divides the level's extent), the workload's aspect ratio and even
    extents of at least 4, and is no larger than the workload."""
    c = inputs.CONFIGS[cfg]
    dims = bench.sample_dims(cfg)
    assert all(d >= 4 and d % 2 == 0 for d in dims)
    assert all(s <= d and d % s == 0 for s, d in zip(dims, c["dims"]))
    ratio = {d // s for s, d in zip(dims, c["dims"])}
    assert len(ratio) == 1                      # the same reduction in every direction
    cd = list(dims)
    for a in c["agg"]:
        assert all(x % y == 0 for x, y in zip(cd, a))
        cd = [x // y for x, y in zip(cd, a)]


def test_sample_dims_of_the_benchmark_workloads():
    assert bench.sample_dims(3) == (8, 8, 8, 8)
    assert bench.sample_dims(4) == (8, 8, 8, 16)


def test_algorithmic_bytes():
    """Coarse apply: 9 N^2 FP16 complex entries, N row scales, input and
    output vectors of every system once; 32^4 coarse level, 12 systems."""
    N, nsys, Vc = 128, 12, 4096
    assert bench.coarse_bytes(N, nsys) == 9 * N * N * 4 + 4 * N + 2 * N * 8 * nsys
    assert bench.coarse_bytes(N, nsys) * Vc == 2518679552
    # naive dslash: four FP16 3x3 links, in and out colour vectors per system
    assert bench.dslash_bytes(False, 1) == 4 * 9 * 4 + 2 * 3 * 8
    assert bench.dslash_bytes(True, 1) == 8 * 9 * 4 + 2 * 3 * 8
    assert bench.kd_bytes(1) == 144 * 4 + 12 + 48


def test_recipes_cover_the_workloads():
    for cfg in (1, 2, 3, 4):
        rec = bench.SOLVER[cfg]
        assert 0 < rec["inner"][0] < 1 and 1 <= rec["inner"][1] <= 16
        assert cfg in bench.REF_OUTER_ITERS and cfg in bench.WORKLOADS
    # the light-mass workloads: tighter level-1 rule, Table 1's rule below it, deflated coarsest level
    for cfg in (3, 4):
        assert bench.SOLVER[cfg]["inner"] == (0.05, 16)
        assert bench.SOLVER[cfg]["coarse_inner"] == (0.25, 8)
        assert bench.SOLVER[cfg]["coarsest_deflate"] == 48
    assert math.isclose(inputs.log_masses(0.001, 0.05, 8)[-1], 0.05)
