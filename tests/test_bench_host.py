"""Host logic of bench.py that needs no GPU: the source items a recorded ncu
capture is tied to, and the record's lookup."""
import hashlib
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


SRC = """#define A(x) (x + 1)
int unrelated() { return 0; }
__device__ float f(int a) {
    if (a) { return 1.f; }
    return 0.f;
}
__global__ void k(float *y) { y[0] = f(A(1)); }
"""


def test_source_items_cut_functions_and_defines():
    b = _bench()
    out = b._source_items(SRC, ["#define A(x)", "__device__ float f(", "void k(float"])
    assert out == ("#define A(x) (x + 1)\n"
                   "__device__ float f(int a) {\n    if (a) { return 1.f; }\n    return 0.f;\n}\n"
                   "__global__ void k(float *y) { y[0] = f(A(1)); }")
    assert b._source_items(SRC, ["missing("]) is None


def test_traffic_record_follows_its_kernel_source():
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        records = json.load(f)
    for r in records:
        assert set(r) >= {"kind", "workload", "kernel", "bytes_per_launch", "algorithmic_bytes_per_launch",
                          "source", "source_items", "source_sha256", "summary"}
        assert os.path.exists(os.path.join(ROOT, r["summary"]))
        with open(os.path.join(ROOT, r["source"])) as f:
            src = b._source_items(f.read(), r["source_items"])
        assert src is not None
        current = hashlib.sha256(src.encode()).hexdigest() == r["source_sha256"]
        # a record applies exactly while its kernel source is unchanged
        assert (b._dram_traffic(r["kind"], r["workload"]) is not None) == current
