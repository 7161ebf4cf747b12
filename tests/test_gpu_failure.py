"""Failure handling on the GPU without a GPU fault: every wait of the
tensor-core network is bounded.  The self-test runs the same bounded wait on
a barrier that nothing completes; the wait gives up after 2 ms, raises the
device timeout flag and returns, the call reports NNP_ERR_TIMEOUT, and the
context keeps evaluating (BF16 form, whose network uses those waits)."""
import numpy as np
import pytest

import synth
from common import box9, weights32

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    s = synth.water_box(64, 101)
    w = weights32(2, 128, 102, 103)
    pot = P.NNP(atomic_numbers=(1, 8), precision="bf16")
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    E0, F0 = pot.eval(s.pos, s.Z, box9(s.box))
    with pytest.raises(P.NNPError) as e:
        pot.selftest_wait_timeout()
    assert e.value.code == 6  # NNP_ERR_TIMEOUT
    E1, F1 = pot.eval(s.pos, s.Z, box9(s.box))  # the flag was cleared; nothing else changed
    assert abs(E1 - E0) <= 1e-9 * abs(E0) and np.abs(F1 - F0).max() <= 1e-5
