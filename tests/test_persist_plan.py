"""Host logic of the persistent coarse-level solver's launch plan (no GPU).

The kernel gives CTA c the rows [c*per, (c+1)*per) of every vector, keeps
partial restrictions per (CTA, touched site) and, in the resident mode,
places the CTA's stencil rows, row scales, prolongator rows and input staging
in shared memory.  For many level shapes and device sizes this checks, by
brute force, what the kernel relies on: every row has exactly one owner, no
CTA touches more sites than its slots, the owners and slots the restriction
assembly derives from a site are the ones that hold its rows, and the
resident layout is aligned, disjoint and within the shared-memory limit.
"""
import pytest

from paper_2212_12559_gb300 import binding


@pytest.fixture(scope="module", autouse=True)
def built_library():
    """The library is built here if needed (nvcc cross-compiles; no GPU call)."""
    from paper_2212_12559_gb300 import build
    return build.build()

SHAPES = [
    # V, N, nsys, nvec of the next level (0: coarsest), storage
    (256, 48, 1, 32, binding.PREC_HALF),    # 16^4 workload, level 2
    (256, 48, 16, 32, binding.PREC_HALF),
    (16, 48, 1, 32, binding.PREC_HALF),     # 8^4 workload, level 2
    (4096, 128, 12, 0, binding.PREC_HALF),  # 32^4 workload, coarsest
    (2592, 48, 16, 32, binding.PREC_HALF),  # 24^3 x 48 workload, level 2
    (81, 48, 3, 32, binding.PREC_SINGLE),
    (72, 8, 2, 3, binding.PREC_HALF),
    (5, 6, 1, 0, binding.PREC_SINGLE),
    (1000, 64, 4, 16, binding.PREC_SINGLE),
]
DEVICES = [(152, 232448), (148, 232448), (132, 101376), (16, 49152)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dev", DEVICES)
def test_plan_invariants(shape, dev):
    V, N, nsys, nv, prec = shape
    sms, cap = dev
    p = binding.persist_plan(V, N, nsys, nv, prec, sms, cap)
    n = V * N
    G, per, nslot = p["grid"], p["per"], p["nslot"]
    assert G == min(sms, V) and per == -(-n // G)
    owner = [None] * n
    covers = {}
    for c in range(G):
        r0 = min(n, c * per)
        r1 = min(n, r0 + per)
        for row in range(r0, r1):
            assert owner[row] is None
            owner[row] = c
        if r1 > r0:
            xs0 = r0 // N
            nts = (r1 - 1) // N - xs0 + 1
            assert nts <= nslot
            for xl in range(nts):
                covers.setdefault(xs0 + xl, []).append((c, xl))
    assert all(o is not None for o in owner)
    for x in range(V):
        c_lo, c_hi = x * N // per, (x * N + N - 1) // per
        derived = [(c, x - c * per // N) for c in range(c_lo, c_hi + 1)]
        assert derived == covers[x]
        assert all(0 <= slot < nslot for _, slot in derived)
    if p["resident"]:
        sb = 4 if prec == binding.PREC_HALF else 8
        assert N % 4 == 0 and nslot <= 8
        assert 1 <= p["sg"] <= nsys
        offs = [p["off_S"], p["off_sc"], p["off_P"], p["off_stg"]]
        assert all(o % 16 == 0 for o in offs) and offs == sorted(offs)
        assert p["off_sc"] - p["off_S"] >= per * 9 * N * sb
        assert p["off_P"] - p["off_sc"] >= per * 4
        assert p["off_stg"] - p["off_P"] >= per * nv * sb
        assert p["smem"] - p["off_stg"] >= p["sg"] * nslot * 9 * N * 8
        assert p["smem"] <= cap
    else:
        assert p["sg"] == 0


def test_resident_for_the_16x4_workload():
    p = binding.persist_plan(256, 48, 1, 32, binding.PREC_HALF, 152, 232448)
    assert p["resident"] == 1 and p["grid"] == 152 and p["per"] == 81 and p["nslot"] == 3


def test_bad_shapes_are_refused():
    with pytest.raises(binding.SmgError):
        binding.persist_plan(0, 48, 1, 0, binding.PREC_HALF, 152, 232448)
    with pytest.raises(binding.SmgError):
        binding.persist_plan(16, 48, 1, 0, binding.PREC_DOUBLE, 152, 232448)
