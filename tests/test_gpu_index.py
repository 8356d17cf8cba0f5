"""GPU parity of the index pass (bnb_build_index): bit-exact against the oracle on the
same float32 records, including per-record fallback and oversized grid cells."""
import numpy as np
import pytest
import torch

from paper_2504_19163_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2504_19163_gb300 import build
    build.build()
    from paper_2504_19163_gb300 import bnb
    return bnb


def upload_records(B, rec, capacity=None):
    n = rec["u_lo"].shape[0]
    cb = B.CellBounds(capacity or n, torch.device("cuda"))
    for k in ("u_lo", "u_hi", "v_lo", "v_hi", "e_lo", "e_hi"):
        getattr(cb, k)[:n] = torch.as_tensor(rec[k])
    for k in ("emitter", "tri0", "tri1"):
        getattr(cb, k)[:n] = torch.as_tensor(rec[k])
    cb.cell[:n] = torch.as_tensor(rec["cell"].view(np.int32))
    cb.flags[:n] = torch.as_tensor(rec["flags"].view(np.int32))
    cb.count.fill_(n)
    cb.c.n_base = rec["n_base"]
    cb.c.depth = rec["depth"]
    return cb


def oracle_index(orc, rec, G, m=1.0):
    return orc.index(rec["u_lo"], rec["u_hi"], rec["v_lo"], rec["v_hi"], rec["e_hi"], rec["emitter"], rec["tri0"],
                     rec["tri1"], rec["flags"], G, m)


def assert_same_index(gi, oi):
    go, gk, ge = gi
    oo, ok, oe = oi
    assert np.array_equal(go, oo)
    assert np.array_equal(gk, ok)
    assert np.array_equal(ge.view(np.uint32), oe.view(np.uint32))


@pytest.mark.parametrize("depth,G", [(2, 512), (1, 100), (3, 512)])
def test_index_bit_exact(B, orc, depth, G):
    rec = S.synthetic_cell_records(3000, depth, n_tris=20000, n_emitters=4, n_overflow=777, seed=5 + depth, grid_res=G)
    cb = upload_records(B, rec)
    idx = B.build_index(cb, grid_res=G)
    torch.cuda.synchronize()
    assert int(idx.status.item()) == 0
    assert_same_index(idx.to_numpy(), oracle_index(orc, rec, G))


def test_index_large_footprints_and_crowded_cells(B, orc):
    """Boxes wider than the merge tile and >1024 entries in one grid cell."""
    rec = S.synthetic_cell_records(2500, 1, n_tris=5000, n_emitters=2, n_overflow=100, seed=11, grid_res=64)
    n = rec["u_lo"].shape[0]
    rng = np.random.default_rng(3)
    wide = rng.random(n) < 0.3
    rec["u_lo"][wide] = 0.0
    rec["u_hi"][wide] = np.float32(0.8)
    rec["v_lo"][wide] = np.float32(0.1)
    rec["v_hi"][wide] = np.float32(0.45)
    rec["flags"][wide] = (rec["flags"][wide] & np.uint32(0xFF000000)) | np.uint32(1)
    cb = upload_records(B, rec)
    idx = B.build_index(cb, grid_res=64)
    torch.cuda.synchronize()
    off, key, et = idx.to_numpy()
    assert np.diff(off).max() > 1024
    assert_same_index((off, key, et), oracle_index(orc, rec, 64))


def test_index_multiplier_m(B, orc):
    rec = S.synthetic_cell_records(500, 2, n_tris=1000, n_emitters=1, n_overflow=0, seed=2)
    cb = upload_records(B, rec)
    idx = B.build_index(cb, grid_res=512, m=2.0)
    torch.cuda.synchronize()
    assert_same_index(idx.to_numpy(), oracle_index(orc, rec, 512, m=2.0))


def test_index_capacity_reported_then_exact(B, orc):
    """A too-small output reports BNB_ERR_CAPACITY and the needed size; re-calling with it is exact.
    A too-small pre-merge workspace reports the pre-merge entries it needed."""
    rec = S.synthetic_cell_records(1000, 2, n_tris=5000, n_emitters=2, n_overflow=50, seed=8)
    cb = upload_records(B, rec)
    o = oracle_index(orc, rec, 512)
    small = B.Index(512, 100, torch.device("cuda"))
    idx = B.build_index(cb, grid_res=512, pre_capacity=4 * o[1].shape[0], capacity=100, out=small,
                        sync_check=False)
    torch.cuda.synchronize()
    assert int(idx.status.item()) == B.BNB_ERR_CAPACITY
    need = int(idx.count[0].item())
    assert need == o[1].shape[0]
    idx2 = B.build_index(cb, grid_res=512, capacity=need)
    torch.cuda.synchronize()
    assert int(idx2.status.item()) == 0
    assert_same_index(idx2.to_numpy(), o)
    # pre-merge workspace too small: status and the pre-merge count that is needed
    idx3 = B.build_index(cb, grid_res=512, pre_capacity=64, capacity=need, sync_check=False)
    torch.cuda.synchronize()
    assert int(idx3.status.item()) == B.BNB_ERR_CAPACITY
    pre_need = int(idx3.count[1].item())
    assert pre_need >= need
    idx4 = B.build_index(cb, grid_res=512, pre_capacity=pre_need, capacity=need)
    torch.cuda.synchronize()
    assert_same_index(idx4.to_numpy(), o)


def test_index_of_nothing(B):
    rec = S.synthetic_cell_records(0, 2, n_tris=10, n_emitters=1, n_overflow=0, seed=1)
    cb = upload_records(B, rec, capacity=16)
    idx = B.build_index(cb, grid_res=32)
    torch.cuda.synchronize()
    off, key, et = idx.to_numpy()
    assert off.shape[0] == 32 * 32 + 1 and off.max() == 0 and key.shape[0] == 0


@pytest.mark.parametrize("n_emitters,vary_t1", [(1, False), (4, False), (400, False), (3, True)])
def test_index_direct_mode_crowded(B, orc, n_emitters, vary_t1):
    """No per-record emission (no split children, every footprint within the merge tile), so the
    per-cell ordering writes the CSR directly; grid cells of <= 128 (rank), 129..512 (warp bitonic
    sort), 513..1024 (block sort) and > 1024 entries; keys spanning < 2^32, one second-triangle
    field over < 256 emitters, and neither (400 emitters, or varied second triangles), which
    select the 32- and 64-bit orderings."""
    rec = S.synthetic_cell_records(5000, 1, n_tris=20000, n_emitters=n_emitters, n_overflow=0, seed=21 + n_emitters,
                                   grid_res=64)
    rng = np.random.default_rng(n_emitters)
    if vary_t1:
        rec["tri1"] = np.repeat(rng.integers(-1, 5000, 5000), 4).astype(np.int32)
    group = rng.random(5000)
    for sel, lo, hi in ((group < 0.15, 0.1, 0.3), ((group >= 0.15) & (group < 0.4), 0.5, 0.7),
                        ((group >= 0.4) & (group < 0.46), 0.75, 0.9)):
        r = np.repeat(sel, 4)
        for k in ("u_lo", "v_lo"):
            rec[k][r] = np.float32(lo)
        for k in ("u_hi", "v_hi"):
            rec[k][r] = np.float32(hi)
        rec["flags"][r] = (rec["flags"][r] & np.uint32(0xFF000000)) | np.uint32(1)
    cb = upload_records(B, rec)
    idx = B.build_index(cb, grid_res=64)
    torch.cuda.synchronize()
    assert int(idx.status.item()) == 0
    off, key, et = idx.to_numpy()
    n_per = np.diff(off)
    for lo, hi in ((1, 128), (129, 512), (513, 1024), (1025, 1 << 40)):
        assert np.any((n_per >= lo) & (n_per <= hi)), (lo, hi)
    assert_same_index((off, key, et), oracle_index(orc, rec, 64))
