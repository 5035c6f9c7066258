"""Host logic of the launch-shape autotuner (no GPU): which coarse-apply
kernels serve which shapes, and the table's text round trip."""
import pytest


@pytest.fixture(scope="module")
def binding():
    from paper_2212_12559_gb300 import build
    build.build()
    from paper_2212_12559_gb300 import binding as b
    b.load()
    return b


def test_coarse_candidates_by_shape(binding):
    b = binding
    tc = [b.COARSE_TC_2x4, b.COARSE_TC_1x4, b.COARSE_TC_1x6]
    cores = [b.COARSE_CORES, b.COARSE_ROWS]
    multi = cores + [b.COARSE_ROWS_MULTI]    # several FP32-vector systems, N % 4 == 0
    # tcgen05 needs N = 128, FP16 storage and several systems; its default comes first
    assert b.coarse_paths(128, 12, b.PREC_HALF) == tc + [b.COARSE_MMA] + multi
    assert b.coarse_paths(128, 2, b.PREC_HALF) == tc + [b.COARSE_MMA] + multi
    # one system: only the two one-system CUDA-core kernels
    assert b.coarse_paths(128, 1, b.PREC_HALF) == cores
    # mma.sync: N % 16 == 0 and N <= 128
    assert b.coarse_paths(48, 12, b.PREC_HALF) == [b.COARSE_MMA] + multi
    assert b.coarse_paths(40, 12, b.PREC_HALF) == multi
    assert b.coarse_paths(144, 12, b.PREC_HALF) == multi
    assert b.coarse_paths(42, 12, b.PREC_HALF) == cores
    # FP32 / FP64 storage: CUDA cores only, while 9N vector entries fit 48 KB of shared memory
    assert b.coarse_paths(128, 12, b.PREC_SINGLE) == multi
    assert b.coarse_paths(256, 4, b.PREC_DOUBLE) == cores
    assert b.coarse_paths(512, 4, b.PREC_DOUBLE) == []
    with pytest.raises(b.SmgError):
        b.coarse_paths(0, 1, b.PREC_HALF)


def test_tune_table_round_trip(binding, tmp_path):
    b = binding
    b.tune_clear()
    assert b.tune_table() == []
    f = tmp_path / "tune.txt"
    f.write_text("# comment\ncoarse_apply V=4096 N=128 nsys=12 vec=f32 store=f16 sub=0\t3\ttcgen05 1 CTA/SM 4 stages\n"
                 "coarse_apply V=2592 N=48 nsys=32 vec=f32 store=f16 sub=1\t2\n")
    b.tune_load(f)
    rows = {r[0]: r[1] for r in b.tune_table()}
    assert rows == {"coarse_apply V=4096 N=128 nsys=12 vec=f32 store=f16 sub=0": 3,
                    "coarse_apply V=2592 N=48 nsys=32 vec=f32 store=f16 sub=1": 2}
    g = tmp_path / "saved.txt"
    b.tune_save(g)
    b.tune_clear()
    b.tune_load(g)
    assert {r[0]: r[1] for r in b.tune_table()} == rows
    bad = tmp_path / "bad.txt"
    bad.write_text("key without id\n")
    with pytest.raises(b.SmgError):
        b.tune_load(bad)
    bad.write_text("key\tnot-a-number\n")
    with pytest.raises(b.SmgError):
        b.tune_load(bad)
    with pytest.raises(b.SmgError):
        b.tune_load(tmp_path / "missing.txt")
    assert {r[0]: r[1] for r in b.tune_table()} == rows   # a refused file changes nothing
    b.tune_mode(0)
    b.tune_mode(1)
    with pytest.raises(b.SmgError):
        b.tune_mode(2)
    b.tune_clear()
