"""GPU bin-packed selection (Sec. 5.3: one draw per group of listed tuples whose probabilities sum
to at most 1) against the oracle on the oracle's own index: the per-point selections and the
|U|, |S|, |B| totals bit-exact, and the estimates within 1e-4; plus the whole path."""
import os

import numpy as np
import pytest
import torch

from paper_2504_19163_gb300 import scenes as S
from test_gpu_sample import E_REL, B, c1, upload_index  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [3, 777])
def test_binned_selection_on_oracle_index(B, orc, c1, seed):
    sc, rec, off, key, et, gamma = c1
    gamma = gamma / 10.0  # smaller P, so that groups hold several tuples
    ds = B.DeviceScene(sc)
    idx = upload_index(B, off, key, et, sc.grid_res)
    r = B.sample_and_solve(ds, idx, gamma, seed, with_sel_count=True, bins=True)
    torch.cuda.synchronize()
    wp, wk, wP, n_u, n_b = orc.sample(off, key, et, sc.grid_res, sc.su, sc.sv, gamma, seed, bins=True,
                                      with_bins=True)
    cnt = r.counters.cpu().numpy()
    assert cnt[0] == n_u and cnt[1] == wp.shape[0] and cnt[3] == n_b
    assert n_b < 0.8 * n_u  # fewer draws than listed tuples
    assert np.array_equal(r.sel_count.cpu().numpy(), np.bincount(wp, minlength=sc.su.shape[0]))
    contrib, _, _, st = orc.solve(sc, wp, wk, wP, n_threads=os.cpu_count())
    E_o = orc.accumulate(sc.su.shape[0], wp, contrib)
    E_g = r.E.cpu().numpy().astype(np.float64)
    pos = E_o > 0
    assert int(st.sum()) > 50 and cnt[2] == int(st.sum())
    assert (np.abs(E_g[pos] - E_o[pos]) / E_o[pos]).max() <= E_REL
    assert np.all(E_g[~pos] == 0)


def test_binned_whole_path_matches_oracle(B, orc):
    sc = S.config("tiny", n=6, depth=2, points=32)
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, sc.depth)
    idx = B.build_index(cb, sc.grid_res)
    gamma = 50.0
    r = B.sample_and_solve(ds, idx, gamma, 9, bins=True)
    torch.cuda.synchronize()
    out = orc.render(sc, gamma, 9, bins=True)
    E_g = r.E.cpu().numpy().astype(np.float64)
    E_o = out["E"]
    pos = E_o > 0
    assert pos.sum() > 100
    rel = np.abs(E_g[pos] - E_o[pos]) / E_o[pos]
    assert np.mean(rel <= E_REL) >= 0.99, np.sort(rel)[-5:]
