"""The bounded device-side waits of the tensor-core current kernel.

Every mbarrier wait of k_induced_current_tc gives up after a bounded number of
polls (sim_config.wait_spin_limit; default 2^22, about two seconds), sets
SIM_STATUS_TIMEOUT in the status word and winds the kernel down, still waiting
for the MMAs and copies it has issued.  Here the limit is lowered to a single
poll so that the waits of a normal small call give up: the call must return
(the stream completes), report the timeout, and leave the context usable: the
next call with the default limit reproduces the currents of an untouched run
bit for bit (the tensor-core form is bitwise reproducible call by call).
"""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import Steps, lut_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [2, 1])
def test_wait_timeout_is_reported_and_the_next_call_is_correct(precision):
    cfg = params.small_config(precision=precision)
    seg = events.scatter_event(cfg, 41, 80, max_len=0.6)
    lut_dev, _ = lut_pair(cfg)
    ref = Steps(cfg, seg, lut_dev, event_id=2).quench_drift().pixel_map().induced_current()
    cur_ref = ref.current_np().copy()
    assert ref.count_values()[3] == 0 and len(cur_ref) > 100

    st = Steps(dict(cfg, wait_spin_limit=1), seg, lut_dev, event_id=2).quench_drift().pixel_map()
    st.induced_current()
    torch.cuda.synchronize()                       # the call returned and its kernels completed
    status = st.count_values()[3]
    assert status & sim.SIM_STATUS_TIMEOUT, status

    # the caller clears the status word and calls again with the default bound
    st.counts[3] = 0
    st.cfg = sim.make_config(cfg)
    st.current.zero_()
    st.induced_current()
    assert st.count_values()[3] == 0
    assert np.array_equal(st.current_np(), cur_ref)

