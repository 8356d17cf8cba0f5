"""bnb_bound_tuples_noalloc: the bound pass for callers that cannot allocate device memory
(a plug-in inside an application that owns the device memory, or a program that forbids
allocation after start-up).  It runs with a fixed scratch array inside the library; its results
must equal those of bnb_bound_tuples with a caller workspace, on two calls in a row (the second
one reuses the array with the first call's contents still in it), for one and for two specular
surfaces, and after a call of the other kind has left its own layout in the array.

The file name makes pytest collect it last, so that if it fails, a run that stops at the first
failure (-x) has already run every other test.  The tests do not depend on that order: they pass
alone in a fresh process (the first call there also looks up the array's address) and after the
other tests."""
import ctypes as C

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
    assert torch.cuda.is_available()
    return bnb


def _sorted_records(cb):
    g = cb.to_numpy()
    order = np.lexsort((g["cell"], g["flags"] >> np.uint32(24), g["tri0"], g["emitter"]))
    return {k: v[order] for k, v in g.items()}


def _noalloc(B, ds, depth, out):
    cfg = B.bnb_bound_cfg(depth, 4, 1, 0)
    out.reset()
    rc = B.bnb_bound_tuples_noalloc(C.byref(ds.s1), ds.s2_ref(), C.byref(ds.rec), C.byref(ds.em), C.byref(cfg),
                                    C.byref(out.c), B._stream(None))
    return rc


def _pair_sorted(cb):
    g = cb.to_numpy()
    order = np.lexsort((g["tri1"], g["cell"], g["tri0"], g["emitter"]))
    return {k: v[order] for k, v in g.items()}


@pytest.mark.parametrize("name,kw", [("mirror32", {}), ("tiny", {"n": 5, "depth": 3})])
def test_noalloc_matches_workspace_entry_point_twice(B, name, kw):
    sc = S.config(name, **kw)
    ds = B.DeviceScene(sc)
    ref = B.bound_tuples(ds, sc.depth)
    torch.cuda.synchronize()
    assert int(ref.status.item()) == 0
    want = _sorted_records(ref)
    for _ in range(2):
        out = B.CellBounds(ref.capacity, ds.device)
        assert _noalloc(B, ds, sc.depth, out) == B.BNB_OK
        torch.cuda.synchronize()
        assert int(out.status.item()) == 0
        assert out.c.n_base == ref.c.n_base
        got = _sorted_records(out)
        assert set(got) == set(want)
        for k in want:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_noalloc_rejects_scratch_beyond_its_maximum(B):
    """A mesh whose workspace exceeds the 8 MiB array is refused before anything is launched."""
    sc = S.config("mirror256")
    ds = B.DeviceScene(sc)
    cfg = B.bnb_bound_cfg(3, 4, 1, 0)
    need = B.bnb_bound_tuples_ws(C.byref(ds.s1), None, C.byref(ds.em), C.byref(cfg))
    assert need > 8 * 1024 * 1024
    out = B.CellBounds(16, ds.device)
    rc = B.bnb_bound_tuples_noalloc(C.byref(ds.s1), None, C.byref(ds.rec), C.byref(ds.em), C.byref(cfg),
                                    C.byref(out.c), B._stream(None))
    assert rc == B.BNB_ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(out.count.item()) == 0


def test_noalloc_two_surfaces_twice_and_after_a_single_surface_call(B):
    """Two specular surfaces (a reduced glass slab) use another layout of the scratch array (both
    packed meshes, the T2 grid, per-cell candidate counts and offsets).  Two calls in a row, then a
    larger single-surface call that overwrites the array, then the slab again: every call's records
    equal those of bnb_bound_tuples with a caller workspace."""
    sc = S.config("slab", n=12, depth=2)
    ds = B.DeviceScene(sc)
    ref = B.bound_tuples(ds, sc.depth)
    torch.cuda.synchronize()
    assert int(ref.status.item()) == 0
    n_ref = ref.n_records()
    assert n_ref > 0
    want = _pair_sorted(ref)

    def check():
        out = B.CellBounds(ref.capacity, ds.device)
        assert _noalloc(B, ds, sc.depth, out) == B.BNB_OK
        torch.cuda.synchronize()
        assert int(out.status.item()) == 0
        assert out.n_records() == n_ref
        got = _pair_sorted(out)
        for k in want:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)

    check()
    check()
    # dirty the array with a single-surface call whose packed mesh and split queues cover the
    # slab's grid and candidate regions, then run the slab again
    big = S.config("mirror32")
    dsb = B.DeviceScene(big)
    outb = B.CellBounds(big.emitters.n * big.s1.n_tris * 4 ** 3 * 2, dsb.device)
    assert _noalloc(B, dsb, 3, outb) == B.BNB_OK
    torch.cuda.synchronize()
    assert int(outb.status.item()) == 0
    check()
