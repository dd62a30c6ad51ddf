"""GPU parity of the induced current for response tables of other shapes than
the default one (45 x 45 bins of 1/30 pitch, 1950 ticks), through the C ABI:

  * the largest table the ABI accepts: nt = 2048 ticks (nt mod 16 = 0);
  * coarse bins and an odd row length: nb = 20 bins of 1/15 pitch, nt = 1001
    (rows padded to 1004; nt mod 16 = 9);
  * short rows: nt = 200 (nt mod 16 = 8).

The FP32 form stages rows by 16-byte chunks at a tick shift of nt mod 16, the
term-by-term form stages quads of rows rounded up to 4, and the tensor-core
form builds phase tables of (nt + 126) / 8 + 18 blocks with node sets over nb
rows: each form is compared on every pixel of a small event with the FP64
oracle at its own tolerances (those of tests/test_gpu_parity.py and
tests/test_gpu_tensor_core.py).
"""
import numpy as np
import pytest

import oracle
from synth import events, params

from gpu_harness import Steps, current_errors, lut_pair, prefix_charge_ok

pytestmark = pytest.mark.gpu

SHAPES = {
    "nt2048": dict(nb=45, nt=2048, bins_per_pitch=30, z0_cm=0.1),
    "nb20_nt1001": dict(nb=20, nt=1001, bins_per_pitch=15, z0_cm=0.1),
    "nt200": dict(nb=45, nt=200, bins_per_pitch=30, z0_cm=0.1),
}
FP32_TOL = {0: (1e-4, 1e-6), 3: (1e-4, 1e-5)}           # per-pixel inf-norm hard cap and median
TC_TOL = dict(l2=5e-4, inf=1e-3, q=5e-4, event=2e-4)   # FP16 operands
Q_MIN = 1.0


def _run(shape, precision):
    lut_par = SHAPES[shape]
    cfg = params.small_config(precision=precision)
    seg = events.scatter_event(cfg, 707 + len(shape), 40, max_len=0.6)
    lut_dev, lut64 = lut_pair(cfg, lut_par)
    st = Steps(cfg, seg, lut_dev, event_id=3, lut_par=lut_par).quench_drift().pixel_map().induced_current()
    m = st.maps_np()
    cur = st.current_np()
    o = oracle.Oracle(cfg, lut_par, lut64)
    d = o.quench_drift(seg)
    ref = np.array([o.pixel_current(seg, d, int(p), m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]], event_id=3)
                    for i, p in enumerate(m["active"].tolist())])
    assert len(ref) > 100
    return cur[: len(ref)], ref


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("precision", [0, 3])
def test_fp32_forms_on_other_table_shapes(shape, precision):
    cur, ref = _run(shape, precision)
    rel, _ = current_errors(cur, ref)
    big = np.abs(ref).max(axis=1) > 0
    q_ok, q_worst = prefix_charge_ok(cur, ref, 1e-5)
    hard, med = FP32_TOL[precision]
    print(f"{shape} precision {precision}: pixels {big.sum()} rel max {rel[big].max():.2e} "
          f"med {np.median(rel[big]):.2e} prefix-charge worst {q_worst:.2e}")
    assert rel[big].max() <= hard and np.median(rel[big]) <= med
    assert q_ok, q_worst


@pytest.mark.parametrize("shape", list(SHAPES))
def test_tensor_core_form_on_other_table_shapes(shape):
    cur, ref = _run(shape, 2)
    d = cur - ref
    sig = np.abs(ref).sum(axis=-1) >= Q_MIN
    l2 = np.linalg.norm(d[sig], axis=-1) / np.linalg.norm(ref[sig], axis=-1)
    inf = np.abs(d[sig]).max(axis=-1) / np.abs(ref[sig]).max(axis=-1)
    q = np.abs(d[sig].sum(-1)) / np.abs(ref[sig]).sum(-1)
    fro = np.linalg.norm(d) / np.linalg.norm(ref)
    mx = np.abs(d).max() / np.abs(ref).max()
    print(f"{shape} FP16: pixels {sig.sum()} l2 max {l2.max():.2e} inf max {inf.max():.2e} q max {q.max():.2e} "
          f"event fro {fro:.2e} max {mx:.2e}")
    assert sig.sum() > 50
    assert l2.max() <= TC_TOL["l2"] and inf.max() <= TC_TOL["inf"] and q.max() <= TC_TOL["q"]
    assert fro <= TC_TOL["event"] and mx <= TC_TOL["event"]
