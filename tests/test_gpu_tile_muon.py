"""The plain-method configuration at full size: one 70x70-pixel anode tile,
one straight muon of 200 x 0.5 cm segments (Moyal dE/dx, MPV 2.1 MeV/cm,
isotropic direction, centred), FP64 oracle vs the GPU path through the C ABI:
every active pixel's current (FP32 and FP16 tensor-core forms) and the
hits end to end (bit-exact up to the oracle's first decision within the
form's band, gpu_harness.BAND; tied pixels at most gpu_harness.tie_cap of the
oracle's own tie probabilities)."""
import numpy as np
import pytest

import oracle
from synth import events, params

from gpu_harness import BAND, Steps, compare_pixel_hits, current_errors, hits_of_pixel, lut_pair, tie_cap

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 2])
def test_tile_muon_every_pixel_and_hits(precision):
    cfg = params.tile_config(precision=precision)
    seg = events.tile_muon(cfg, params.BASE["seed"])
    assert len(seg["x0"]) >= 200
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=2).all()
    m, cur, h = st.maps_np(), st.current_np(), st.hits_np()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    assert (d["anode"] >= 0).sum() > 20          # the part of the track inside the volume
    ref_pix, _, _, _ = o.pixel_map(seg, d)
    assert len(set(m["active"].tolist()) ^ set(ref_pix)) <= 2
    band = BAND[precision]
    refs, n_cmp, n_tied, n_hit_pix, p_ties = [], 0, 0, 0, []
    for i, p in enumerate(m["active"]):
        I = o.pixel_current(seg, d, int(p), m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]], event_id=2)
        refs.append(I)
        ref = o.electronics(int(p), I, event_id=2, band=band)
        g = hits_of_pixel(h, int(p))
        if len(ref["t_cross"]) or len(g["t_cross"]):
            n_hit_pix += 1
            p_ties.append(ref["p_tie"])
        n_tied += ref["tie_tick"] >= 0
        ok, nc = compare_pixel_hits(g, ref, 976.5625)
        assert ok, (p, ref, g)
        n_cmp += nc
    ref = np.array(refs)
    sig = np.abs(ref).sum(-1) >= 1.0
    rel, qrel = current_errors(cur[sig], ref[sig])
    print(f"tile muon, precision {precision}: pixels {sig.sum()} rel max {rel.max():.2e} med {np.median(rel):.2e} "
          f"q max {qrel.max():.2e}; hits compared {n_cmp}, tied pixels {n_tied} of {n_hit_pix}")
    assert rel.max() <= (1e-4 if precision == 0 else 5e-4)
    assert n_cmp > 20 and n_tied <= tie_cap(p_ties)
