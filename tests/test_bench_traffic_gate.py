"""bench.py reports a pair kernel's captured DRAM traffic only for the build it
was captured on: a changed kernel source, another workload scale or a kernel
without a capture gives null."""
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
    for _, sources in bench.KERNEL_TRAFFIC.values():
        for rel in sources:
            os.makedirs(os.path.join(dst, os.path.dirname(rel)), exist_ok=True)
            shutil.copyfile(os.path.join(ROOT, rel), os.path.join(dst, rel))


def test_traffic_follows_the_recorded_sources(tmp_path):
    bench = _bench()
    for kernel, (nbytes, _) in bench.KERNEL_TRAFFIC.items():
        expected = bench.kernel_traffic(kernel, 1.0)
        assert expected is None or expected == nbytes
        # a byte-identical copy of the sources gives the repository's answer
        _copy_sources(bench, tmp_path)
        bench.ROOT = str(tmp_path)
        assert bench.kernel_traffic(kernel, 1.0) == expected
        bench.ROOT = ROOT
    assert bench.kernel_traffic("no such kernel", 1.0) is None


def test_changed_source_or_scale_gives_null(tmp_path):
    bench = _bench()
    _copy_sources(bench, tmp_path)
    bench.ROOT = str(tmp_path)
    for kernel, (_, sources) in bench.KERNEL_TRAFFIC.items():
        assert bench.kernel_traffic(kernel, 0.5) is None
        rel = next(iter(sources))
        with open(os.path.join(tmp_path, rel), "ab") as f:
            f.write(b"\n// changed\n")
        assert bench.kernel_traffic(kernel, 1.0) is None
        os.remove(os.path.join(tmp_path, rel))
        assert bench.kernel_traffic(kernel, 1.0) is None
