"""CPU checks of the C ABI: the library loads, exports every declared entry
point, agrees with the binding's struct layouts, and rejects bad arguments on
the host before any launch (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2212_09807_gb300 import build, sim
    build.build()
    return sim.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for f in ("sim_quench_drift", "sim_pixel_map", "sim_induced_current", "sim_electronics", "sim_event"):
        assert f in names


def test_library_exports_every_declared_symbol(L):
    import subprocess
    from paper_2212_09807_gb300 import sim
    out = subprocess.run(["nm", "-D", "--defined-only", sim.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sim_[a-z_0-9]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(L, f)


def test_struct_sizes_match_binding(L):
    from paper_2212_09807_gb300 import sim
    sizes = (C.c_int64 * 5)()
    L.sim_abi_sizes(sizes)
    assert list(sizes) == [C.sizeof(sim.SimConfig), C.sizeof(sim.SimSegments), C.sizeof(sim.SimResponse),
                           C.sizeof(sim.SimDrifted), C.sizeof(sim.SimHits)]


def test_strerror(L):
    assert L.sim_strerror(0) == b"ok"
    assert b"invalid" in L.sim_strerror(-1)


def test_host_argument_checks_reject_before_launch(L):
    from paper_2212_09807_gb300 import sim
    from synth import params
    cfg = sim.make_config(params.module_config())
    b = C.c_size_t()
    assert L.sim_workspace_size(C.byref(cfg), 0, 100, 1000, 100, C.byref(b)) == 0 and b.value > 0
    assert L.sim_workspace_size(C.byref(cfg), 0, -1, 1000, 100, C.byref(b)) == -1
    assert L.sim_workspace_size(C.byref(cfg), 20000, 1, 1, 1, C.byref(b)) == -1   # > 2^31 virtual pixels
    bad = sim.make_config(params.module_config(n_ticks=0))
    assert L.sim_workspace_size(C.byref(bad), 0, 1, 1, 1, C.byref(b)) == -1
    seg = sim.SimSegments()
    seg.n = 5                                   # null columns
    d = sim.SimDrifted()
    assert L.sim_quench_drift(C.byref(cfg), C.byref(seg), C.byref(d), None) == -1
    r = sim.SimResponse()
    r.nb, r.nt, r.ld, r.bins_per_pitch = 45, 1950, 1950, 30   # ld not a multiple of 4
    h = sim.SimHits()
    assert L.sim_event(C.byref(cfg), C.byref(seg), C.byref(r), 10, 10, C.byref(h), None, 0, None) == -1


def test_workspace_grows_with_capacities(L):
    from paper_2212_09807_gb300 import sim
    from synth import params
    cfg = sim.make_config(params.module_config())
    a = sim.workspace_size(cfg, 1000, 10000, 1000)
    b = sim.workspace_size(cfg, 1000, 10000, 2000)
    assert b - a >= 1000 * 2000 * 4      # the current array [pixels][ticks] is inside


def test_post_hit_entry_points_check_arguments(L):
    from paper_2212_09807_gb300 import sim
    from synth import params
    cfg = sim.make_config(params.module_config())
    seg, d, r, h = sim.SimSegments(), sim.SimDrifted(), sim.SimResponse(), sim.SimHits()
    r.nb, r.nt, r.ld, r.bins_per_pitch = 45, 1950, 1952, 30
    t = sim.SimTruth()
    t.k = 0                                         # k outside 1 .. SIM_TRUTH_MAX_K
    fake = C.c_void_p(16)                           # never dereferenced: the checks fail first
    assert L.sim_hit_truth(C.byref(cfg), C.byref(seg), C.byref(d), C.byref(r), fake, None, None, None, fake, 0,
                           C.byref(h), C.byref(t), 0, fake, 1 << 20, None) == -1
    b = C.c_size_t()
    assert L.sim_hit_truth_workspace_size(1000, 10000, C.byref(b)) == 0 and b.value > 8 * 10000
    assert L.sim_hit_truth_workspace_size(1000, 1 << 31, C.byref(b)) == -1
    assert L.sim_hit_points(C.byref(cfg), C.byref(h), None, None, None, None, None) == -1   # no n_out
    o = (C.c_double * 3)(0, 0, 0)
    assert L.sim_track_dqdx(None, None, None, None, fake, 0, o, o, 0.0, 4, 1.0, fake, fake, None) == -1
    assert L.sim_response_cumulative(C.byref(r), None, None) == -1


def test_tuning_fields_are_checked(L):
    from paper_2212_09807_gb300 import sim
    from synth import params
    b = C.c_size_t()
    for bad in (dict(tc_units_per_sm=17), dict(tc_record_chunk=5000), dict(tc_record_chunk=1 << 21),
                dict(direct_ctas_per_sm=5)):
        cfg = sim.make_config(params.module_config(**bad))
        assert L.sim_workspace_size(C.byref(cfg), 0, 100, 1000, 100, C.byref(b)) == -1, bad
    cfg = sim.make_config(params.module_config(precision=2, tc_units_per_sm=8, tc_record_chunk=1 << 16))
    assert L.sim_workspace_size(C.byref(cfg), 0, 100, 1000, 100, C.byref(b)) == 0
    for bad in (-1, (1 << 30) + 1):                     # the bounded waits' poll limit
        cfg = sim.make_config(params.module_config(wait_spin_limit=bad))
        assert L.sim_workspace_size(C.byref(cfg), 0, 100, 1000, 100, C.byref(b)) == -1, bad
    cfg = sim.make_config(params.module_config(wait_spin_limit=16))
    assert L.sim_workspace_size(C.byref(cfg), 0, 100, 1000, 100, C.byref(b)) == 0


def test_noalloc_map_checks_the_response_like_the_map(L):
    """sim_pixel_map_noalloc rejects on the host every response sim_pixel_map
    rejects (table limits, row stride), before it looks up its scratch."""
    from paper_2212_09807_gb300 import sim
    from synth import params
    cfg = sim.make_config(params.module_config())
    seg, d = sim.SimSegments(), sim.SimDrifted()      # an empty event: no device pointer is needed
    fake = C.c_void_p(16)                             # never dereferenced: the checks fail first
    counts = C.c_void_p(64)
    for nb, nt, ld, bpp in ((45, 1950, 1950, 30), (45, 4000, 4000, 30), (46, 1950, 1952, 30), (45, 1950, 1952, 0)):
        r = sim.SimResponse()
        r.nb, r.nt, r.ld, r.bins_per_pitch = nb, nt, ld, bpp
        for fn in ("sim_pixel_map_noalloc", "sim_pixel_map"):
            args = [C.byref(cfg), C.byref(seg), C.byref(d), C.byref(r), fake, fake, 10, fake, fake, fake, 10]
            rc = (L.sim_pixel_map_noalloc(*args, counts, None) if fn == "sim_pixel_map_noalloc"
                  else L.sim_pixel_map(*args, fake, 1 << 20, None))
            assert rc == -1, (fn, nb, nt, ld, bpp)


def test_autotuner_candidates_are_valid_configurations(L):
    """Every shape the autotuner may pick passes the ABI's checks, and the
    tensor-core workspace grows with the record chunk (two buffers of 32-byte
    records per CTA)."""
    from paper_2212_09807_gb300 import sim, tune
    from synth import params
    b = C.c_size_t()
    sizes = {}
    for prec in (0, 1, 2):
        for cand in tune.candidates(prec):
            cfg = sim.make_config(params.module_config(precision=prec, **cand))
            assert L.sim_workspace_size(C.byref(cfg), 0, 1000, 40000, 4000, C.byref(b)) == 0, (prec, cand)
            if prec == 2 and cand["tc_units_per_sm"] == 1:
                sizes[cand["tc_record_chunk"]] = b.value
    chunks = sorted(sizes)
    assert chunks[-1] == 1 << 20
    for lo, hi in zip(chunks, chunks[1:]):
        assert sizes[hi] - sizes[lo] >= 2 * 32 * (hi - lo)        # at least one CTA's two record buffers


def test_precision_range(L):
    """precision 0..3 are the four forms of the current; 4 and -1 are rejected."""
    from paper_2212_09807_gb300 import sim
    from synth import params
    b = C.c_size_t()
    for prec in (0, 1, 2, 3):
        cfg = sim.make_config(params.module_config(precision=prec))
        assert L.sim_workspace_size(C.byref(cfg), 0, 1000, 40000, 4000, C.byref(b)) == 0, prec
        assert b.value > 0
    for bad in (-1, 4):
        cfg = sim.make_config(params.module_config(precision=bad))
        assert L.sim_workspace_size(C.byref(cfg), 0, 1000, 40000, 4000, C.byref(b)) == -1, bad
