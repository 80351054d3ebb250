"""The paper's pruning experiment (Sec. 6, Fig. 3) on the synthetic
384 x 288 workload, with the FP64 oracle: setting fbar = 0 (Eq. 8) instead of
the truncated potential's fbar = exp(-alpha T) alters the disparity map and
makes it worse.  (The exact model converges to a map within one disparity of
the ground truth almost everywhere; the pruned model does not.)"""
import numpy as np
import pytest

from oracle import grid, stereo
from paper_1010_0012_gb300 import workload as wl


@pytest.mark.slow
def test_pruning_alters_and_worsens_the_map():
    cfg = wl.CONFIGS["grid384x288_m16"]
    st = wl.make_stereo(cfg)
    g = wl.unary_f32(st).astype(np.float64)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    maps = {}
    for name, fb in (("exact", fbar), ("pruned", 0.0)):
        F = stereo.compatibility_matrix(tab.astype(np.float64), cfg.T, fb, cfg.M)
        _, bel = grid.grid_sum_product(g, F, 20, "redblack")
        maps[name] = np.argmax(bel, -1)
    err = {k: float(np.mean(np.abs(v - st.d_gt) > 1)) for k, v in maps.items()}
    changed = float(np.mean(maps["exact"] != maps["pruned"]))
    assert changed > 0.01
    assert err["pruned"] > 10 * err["exact"]
