"""The q database across cases (paper Sec. 3.3: a case starts from the
database an earlier case ended with): set, save and load through the C ABI,
with the warm-start snapshots (Sec. 2.4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BASE = dict(n_sections=12, dx=50.0, h0=12.0, Lx=10.0, Lz=10.0, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
            period=1000.0, dt=20.0, T=1.1, md_steps_eq=1000, md_steps_sample=1000, seed=5, sf2=100.0,
            l2=1.0, sn2=0.25)


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


def test_save_and_load_round_trip(native, tmp_path):
    ctx = native.Context(0, native.PREC_FP32)
    a = native.Hybrid(ctx, **dict(BASE, warm_start=1))
    a.step(0.0)
    a.step(0.0)
    X, y, se = a.database()
    assert len(y) == 24
    path = str(tmp_path / "db.bin")
    a.save(path)
    a.close()
    # a new case from the file: the same database bit for bit, and its MD
    # runs start from the loaded snapshots at once
    b = native.Hybrid(ctx, **dict(BASE, warm_start=1))
    b.load(path)
    X2, y2, se2 = b.database()
    np.testing.assert_array_equal(X2, X)
    np.testing.assert_array_equal(y2, y)
    np.testing.assert_array_equal(se2, se)
    st = b.step(0.0)
    assert st["md_runs"] == 12 and st["md_warm"] == 12
    b.close()
    # without snapshots: the database only, cold starts
    c = native.Hybrid(ctx, **dict(BASE, warm_start=1))
    c.load(path)
    c.save(path + ".nosnap", snapshots=False)
    c.close()
    d = native.Hybrid(ctx, **dict(BASE, warm_start=1))
    d.load(path + ".nosnap")
    np.testing.assert_array_equal(d.database()[1], y)
    assert d.step(0.0)["md_warm"] == 0
    d.close()
    ctx.close()


def test_bad_files_leave_the_case_unchanged(native, tmp_path):
    ctx = native.Context(0, native.PREC_FP32)
    a = native.Hybrid(ctx, **BASE)
    a.step(0.0)
    path = str(tmp_path / "db.bin")
    a.save(path)
    X, y, _ = a.database()
    raw = open(path, "rb").read()
    bad = str(tmp_path / "bad.bin")
    for blob in (raw[:40], b"NOTADB!!" + raw[8:], b""):
        open(bad, "wb").write(blob)
        with pytest.raises(native.MdgpError):
            a.load(bad)
        np.testing.assert_array_equal(a.database()[1], y)
    # another input dimension (the paper's (h, n, F) form) cannot take it
    b = native.Hybrid(ctx, **dict(BASE, inputs=1))
    with pytest.raises(native.MdgpError):
        b.load(path)
    assert len(b.database()[1]) == 0
    with pytest.raises(native.MdgpError):
        a.load(str(tmp_path / "missing.bin"))
    b.close()
    a.close()
    ctx.close()


def test_refined_case_reuses_the_coarse_database(native):
    # Sec. 3.3: twice the sections (bisecting the old ones), the coarse
    # case's database as the initial one: the refined case needs fewer MD
    # runs at the same threshold than the same case started empty
    ctx = native.Context(0, native.PREC_FP32)
    coarse = native.Hybrid(ctx, **BASE)
    for _ in range(3):
        coarse.step(0.5)
    X, y, se = coarse.database()
    coarse.close()
    fine = dict(BASE, n_sections=24, dx=25.0)
    runs = {}
    for name, db in (("empty", None), ("reused", (X, y, se))):
        h = native.Hybrid(ctx, **fine)
        if db is not None:
            h.set_database(*db)
            assert len(h.database()[1]) == len(y)
        runs[name] = sum(h.step(0.5)["md_runs"] for _ in range(3))
        h.close()
    print("refined case MD runs:", runs)
    assert runs["reused"] < runs["empty"]
    ctx.close()
