"""Host logic of bench.py that needs no GPU: the key under which stored ncu
traffic figures stay attached to a kernel's code."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// a kernel
__global__ void k(float *x) {   /* one
   block */
    x[threadIdx.x] *= 2.f;      // doubled
}
"""


def test_code_hash_ignores_comments_and_blank_space():
    h = bench.code_sha256(SRC)
    edited = SRC.replace("// doubled", "// twice its value").replace("/* one\n   block */", "")
    assert bench.code_sha256(edited) == h
    assert bench.code_sha256(SRC.replace("    x[", "\tx[")) == h


def test_code_hash_changes_with_the_code():
    h = bench.code_sha256(SRC)
    assert bench.code_sha256(SRC.replace("2.f", "3.f")) != h
    assert bench.code_sha256(SRC.replace("threadIdx.x]", "threadIdx.x + 1]")) != h


def test_stored_traffic_needs_a_matching_entry():
    assert bench.stored_traffic("induced_current.cu", "no_such_workload") is None
