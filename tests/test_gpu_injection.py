"""FP32 against FP64 on a state with injected electrons (FP32 fields,
momenta, offsets and currents with FP64 reductions; Sec. 3.2, Table 1
reports the injected charge).

The c1/c2 runs carry no charge above gamma 20 in their first 1000 steps (the
window is still in the density up-ramp), which makes a charge gate there
degenerate.  The `inj` recipe is a denser, shorter window in which the wake
traps electrons within a few thousand steps: after 5000 steps the FP64 run
holds a few nC above gamma 20.

Gates, FP32 fields, momenta, offsets and currents (FP64 window accumulator
and reductions) against FP64:
- charge above gamma 20 within 2 % at step 5000, on a state whose FP64
  charge there is above 0.1 nC; the spectrum within 2 % (L1);
- on-axis Ex lineout within 1 % (L2) and field energy within 1 % at step
  1500.  Once electrons are trapped the on-axis lineout follows the trapped
  bunch's microstructure, which is chaotic: two FP64 runs that differ only in
  the order of their atomic sums already differ by 5 % at step 3000 and by
  27 % at step 5000 (lineout L2, measured on a GB300), so the lineout is gated
  before that.
The FP64 path itself is checked against the oracle step by step in
test_gpu_parity.py; this state is too large for the oracle.
"""
import numpy as np
import pytest

from paper_1204_0838_gb300 import pic, workloads as W

from .pairs import make_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

STEPS = 5000
Q_FLOOR = 1e-10  # C: the FP64 state must hold at least this much above gamma 20


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pic.lib()


def test_fp32_injected_charge_and_lineout_against_fp64():
    cfg = W.config("inj")
    g64 = make_gpu(cfg, track_ids=False, precision="fp64")
    g32 = make_gpu(cfg, track_ids=False, precision="fp32")
    early = 1500
    for g in (g64, g32):
        g.step(early)
    l64, l32 = g64.diag("ex_lineout", cfg["nx"]), g32.diag("ex_lineout", cfg["nx"])
    e64, e32 = g64.diag("field_energy")[0], g32.diag("field_energy")[0]
    lo = np.linalg.norm(l32 - l64) / np.linalg.norm(l64)
    print("step %d: lineout L2 %.3e, energy %.3e" % (early, lo, abs(e32 / e64 - 1)))
    assert lo <= 0.01
    assert abs(e32 / e64 - 1) <= 0.01
    for g in (g64, g32):
        for done in range(early, STEPS, 500):
            g.step(min(500, STEPS - done))
    q64, q32 = g64.diag("charge", 1, 20.0)[0], g32.diag("charge", 1, 20.0)[0]
    s64, s32 = g64.diag("spectrum", 100, 0.0, 100.0), g32.diag("spectrum", 100, 0.0, 100.0)
    spec = np.abs(s32 - s64).sum() / s64.sum()
    print("step %d: Q(g>20) FP64 %.4e C, FP32 %.4e C; spectrum L1 %.3e" % (STEPS, q64, q32, spec))
    assert q64 > Q_FLOOR
    assert abs(q32 / q64 - 1) <= 0.02
    assert spec <= 0.02
    g64.close()
    g32.close()
