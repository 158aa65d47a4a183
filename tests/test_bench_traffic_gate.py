"""bench.py reports the dose kernel's captured DRAM traffic only for the build it
was captured on: a changed kernel source or another workload scale gives null."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _copy_sources(bench, dst):
    for rel in bench.DOSE_TRAFFIC_SOURCES:
        os.makedirs(os.path.join(dst, os.path.dirname(rel)), exist_ok=True)
        shutil.copyfile(os.path.join(ROOT, rel), os.path.join(dst, rel))


def test_traffic_follows_the_recorded_sources(tmp_path):
    bench = _bench()
    expected = bench.dose_traffic(1.0)
    assert expected is None or expected == bench.DOSE_TRAFFIC_BYTES
    # a byte-identical copy of the sources gives the repository's answer
    _copy_sources(bench, tmp_path)
    bench.ROOT = str(tmp_path)
    assert bench.dose_traffic(1.0) == expected


def test_changed_source_or_scale_gives_null(tmp_path):
    bench = _bench()
    _copy_sources(bench, tmp_path)
    bench.ROOT = str(tmp_path)
    assert bench.dose_traffic(0.5) is None
    rel = next(iter(bench.DOSE_TRAFFIC_SOURCES))
    with open(os.path.join(tmp_path, rel), "ab") as f:
        f.write(b"\n// changed\n")
    assert bench.dose_traffic(1.0) is None
    os.remove(os.path.join(tmp_path, rel))
    assert bench.dose_traffic(1.0) is None
