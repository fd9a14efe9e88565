"""Host-side checks of bench.py's roofline bookkeeping (no GPU): every kernel class the bench profiles
has an ncu traffic figure for its workload, and that figure was captured from the sources the library
is built from now (the stored digest equals the digest of the class's source files), so the bench line
never reports a traffic figure of a kernel that has changed since its capture."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_for_tests", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_profiled_class_has_current_traffic():
    b = _bench()
    for workload in ("2d", "3d"):
        for cls in b.PROFILED[workload]:
            value, note = b.traffic_for(workload, cls)
            assert value is not None, (workload, cls, note)
            assert value > 0


def test_traffic_digest_follows_the_sources(tmp_path, monkeypatch):
    # a changed source file makes the stored figure stale: traffic_for then reports None
    b = _bench()
    csrc = tmp_path / "csrc"
    csrc.mkdir()
    for f in set(sum((list(v[3]) for v in b.KERNEL_CLASSES.values()), [])):
        (csrc / f).write_bytes(open(os.path.join(b.CSRC, f), "rb").read())
    monkeypatch.setattr(b, "CSRC", str(csrc))
    assert b.traffic_for("2d", "arnoldi")[0] is not None
    with open(csrc / "control.cu", "ab") as fh:
        fh.write(b"\n// edited\n")
    value, note = b.traffic_for("2d", "arnoldi")
    assert value is None and "stale" in note
    assert b.traffic_for("2d", "fp32_dst")[0] is not None  # other classes' sources are untouched


def test_roofline_peaks_and_units():
    b = _bench()
    hbm, how = b.measured_hbm_gbs()
    assert hbm > 1000.0 and how in ("measured", "fallback")
    # the FP64 issue-rate peak of the Arnoldi class: 152 SMs x 2 FMA/clk x 2 flop at 2.07 GHz
    assert abs(b.FP64_ALU_PEAK_FLOPS - 1.25856e12) < 1e9
    for cls, (kind, bound, _desc, srcs) in b.KERNEL_CLASSES.items():
        assert bound in ("hbm", "alu"), cls
        for f in srcs:
            assert os.path.exists(os.path.join(b.CSRC, f)), (cls, f)
