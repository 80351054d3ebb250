"""Eq. 8: with fbar = 0 the update keeps only the band.  It is the exact
update of a potential whose incompatible pairs are 0.  On the stereo workload
that pruned model drives message entries towards 0 within a few iterations
(1e-24 after two red-black iterations, 1e-195 after three, in FP64), so the
FP32 kernels are compared with the FP64 oracle over the first two iterations,
where every entry still carries weight in FP32."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("iters", [1, 2])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_pruned_update_matches_the_oracle(iters, schedule):
    cfg = wl.CONFIGS["grid384x288_m16"]
    st, g, _ = H.stereo_inputs(cfg)
    tab, _ = wl.pair_table_f32(cfg.alpha, cfg.T)
    H.check_sum_case(g, tab, cfg.T, 0.0, iters, schedule)
