"""Eq. 8: with fbar = 0 the update keeps only the band.  It is exact for a
potential whose incompatible pairs really are 0, and for the stereo potential
(fbar = exp(-alpha T) > 0) it is an approximation that changes the result
(Sec. 6, the pruned map of Fig. 3).  Sum-product, 384 x 288, M = 16, T = 2,
50 red-black iterations."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def test_pruned_update_is_exact_for_its_own_potential_and_alters_the_map():
    cfg = wl.CONFIGS["grid384x288_m16"]
    st, g, _ = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    # exact model (Eq. 7) and the pruned form (Eq. 8) of the same table
    bel_x, map_x, _ = H.run_gpu_sum(g, tab, cfg.T, fbar, cfg.iters, "redblack")
    bel_p, map_p, _ = H.run_gpu_sum(g, tab, cfg.T, 0.0, cfg.iters, "redblack")
    # the pruned run is the exact BP of the potential that is 0 off the band
    F0 = H.oracle_F_from_table(tab, cfg.T, 0.0, cfg.M)
    _, b64 = grid.grid_sum_product(g.astype(np.float64), F0, cfg.iters, "redblack")
    assert H.node_rel_err(bel_p, b64) <= H.REL_TOL
    # ... and it is not the exact model's answer
    differ = float(np.mean(map_x != map_p))
    assert differ > 0.0
    err_x = float(np.mean(np.abs(map_x - st.d_gt) > 1))
    err_p = float(np.mean(np.abs(map_p - st.d_gt) > 1))
    print(f"pixels where the pruned MAP differs: {differ:.4f}; "
          f"error rate (|d - d_gt| > 1): exact {err_x:.4f}, pruned {err_p:.4f}")
