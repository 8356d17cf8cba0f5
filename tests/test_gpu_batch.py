"""GPU tests of the batched rendering pass (bnb_sample_and_solve_batched), its CUDA-graph replay,
the launch-shape autotuner and the serving loop.

The batched pass must give, per job, exactly the result of the single-call rendering pass on the
job's points (same index, gamma and seed), whatever else shares the batch; with an emitter subset
it must select exactly what the oracle selects on the index restricted to those emitters."""
import os

import numpy as np
import pytest
import torch

from paper_2504_19163_gb300 import scenes as S

pytestmark = pytest.mark.gpu

E_REL = 1e-4


@pytest.fixture(scope="module")
def B():
    from paper_2504_19163_gb300 import build
    build.build()
    from paper_2504_19163_gb300 import bnb
    return bnb


@pytest.fixture(scope="module")
def BA(B):
    from paper_2504_19163_gb300 import batch
    return batch


def upload_index(B, off, key, et, G):
    idx = B.Index(G, max(1, key.shape[0]), torch.device("cuda"))
    idx.offsets.copy_(torch.as_tensor(off))
    if key.shape[0]:
        idx.key[: key.shape[0]] = torch.as_tensor(key.view(np.int64))
        idx.etilde[: key.shape[0]] = torch.as_tensor(et)
    idx.count[0] = key.shape[0]
    return idx


def oracle_index(orc, sc):
    rec = orc.bound(sc, n_threads=os.cpu_count())
    f = orc.records_to_f32(rec)
    return orc.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"], f["tri1"],
                     f["flags"], sc.grid_res)


def gamma_of(sc, off, et, target=4.0):
    G = sc.grid_res
    g = np.clip(np.floor(sc.sv * np.float32(G)), 0, G - 1).astype(np.int64) * G + \
        np.clip(np.floor(sc.su * np.float32(G)), 0, G - 1).astype(np.int64)
    mean_sum = float(np.mean([et[off[i]:off[i + 1]][np.isfinite(et[off[i]:off[i + 1]])].sum() for i in g]))
    return target / mean_sum


@pytest.fixture(scope="module")
def scenes2(B, BA, orc):
    """Two resident scenes: the 32^2 mirror with one light, and a 3-light variant of it."""
    out = []
    for name, em in (("one", None), ("three", S.emitter_pool((0.0, 0.0, 2.0), 0.3, 3, seed=9))):
        sc = S.config("mirror32", points=48)
        if em is not None:
            sc = S.Scene(sc.name + "_3", sc.s1, None, sc.receiver, em, sc.depth, sc.su, sc.sv)
        off, key, et = oracle_index(orc, sc)
        ds = B.DeviceScene(sc)
        idx = upload_index(B, off, key, et, sc.grid_res)
        gamma = gamma_of(sc, off, et)
        out.append((sc, ds, idx, (off, key, et), BA.ResidentScene(ds, idx, gamma)))
    torch.cuda.synchronize()
    return out


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    return np.array_equal(np.asarray(a, np.float32).view(np.uint32), np.asarray(b, np.float32).view(np.uint32))


def make_jobs(BA, scenes2):
    """Three jobs: all points of scene one, a ragged slice of them with another seed, and scene three."""
    (sc1, ds1, _, _, rs1), (sc3, ds3, _, _, rs3) = scenes2
    n1 = sc1.su.shape[0]
    jobs = [BA.Job(rs1, dev(sc1.su), dev(sc1.sv), torch.empty(n1, device="cuda"), 5),
            BA.Job(rs1, dev(sc1.su[7:1000]), dev(sc1.sv[7:1000]), torch.empty(993, device="cuda"), 99),
            BA.Job(rs3, dev(sc3.su[:777]), dev(sc3.sv[:777]), torch.empty(777, device="cuda"), 12345)]
    return jobs


def test_batched_job_equals_single_call(B, BA, scenes2):
    jobs = make_jobs(BA, scenes2)
    r = BA.BatchRunner(8, sum(j.n_points for j in jobs), 1 << 20, use_graph=True)
    r.submit(jobs)
    status, cnt = r.result()
    assert status == 0
    tot_u = tot_s = tot_roots = 0
    for j in jobs:
        s = B.sample_and_solve(j.scene.ds, j.scene.index, j.scene.gamma, j.seed, su=j.su, sv=j.sv)
        torch.cuda.synchronize()
        assert same_bits(j.E_out.cpu().numpy(), s.E.cpu().numpy())
        c = s.counters.cpu().numpy()
        tot_u += int(c[0])
        tot_s += int(c[1])
        tot_roots += int(c[2])
    assert cnt == [tot_u, tot_s, tot_roots]
    assert tot_roots > 100


def test_alone_vs_mix_with_graph_replay(B, BA, scenes2):
    """One captured graph, replayed with rewritten job tables: a job's estimate is bit-identical
    alone and in any mix, in any position of the table."""
    jobs = make_jobs(BA, scenes2)
    r = BA.BatchRunner(8, sum(j.n_points for j in jobs) + 64, 1 << 20, use_graph=True)
    alone = []
    for j in jobs:
        r.submit([j])
        assert r.result()[0] == 0
        alone.append(j.E_out.cpu().numpy().copy())
    assert r.graph is not None
    for order in ([2, 0, 1], [1, 2, 0], [0, 1, 2]):
        for j in jobs:
            j.E_out.fill_(-1.0)
        r.submit([jobs[i] for i in order])
        assert r.result()[0] == 0
        for i, j in enumerate(jobs):
            assert same_bits(j.E_out.cpu().numpy(), alone[i]), (order, i)


def test_emitter_subset_against_oracle(B, BA, orc, scenes2):
    """emitter_on = {0, 2} of three lights: selection counts exact and estimates within 1e-4 of the
    oracle run on the index restricted to those lights' tuples."""
    sc, ds, idx, (off, key, et), rs = scenes2[1]
    on = torch.tensor([1, 0, 1], dtype=torch.uint8, device="cuda")
    n = sc.su.shape[0]
    job = BA.Job(rs, dev(sc.su), dev(sc.sv), torch.empty(n, device="cuda"), 77, emitter_on=on)
    r = BA.BatchRunner(2, n, 1 << 20, use_graph=False)
    r.submit([job])
    status, cnt = r.result()
    assert status == 0
    # the oracle index restricted to emitters 0 and 2
    G = sc.grid_res
    em = (key >> np.uint64(48)).astype(np.int64)
    keep = em != 1
    ck = np.concatenate([[0], np.cumsum(keep.astype(np.int64))])
    off2 = ck[off].astype(np.int64)
    key2, et2 = key[keep], et[keep]
    wp, wk, wP, n_u = orc.sample(off2, key2, et2, G, sc.su, sc.sv, rs.gamma, 77)
    contrib, _, _, st = orc.solve(sc, wp, wk, wP, n_threads=os.cpu_count())
    E_o = orc.accumulate(n, wp, contrib)
    assert cnt[0] == n_u and cnt[1] == wp.shape[0] and cnt[2] == int(st.sum())
    E_g = job.E_out.cpu().numpy().astype(np.float64)
    pos = E_o > 0
    assert np.max(np.abs(E_g[pos] - E_o[pos]) / E_o[pos]) <= E_REL
    assert np.all(E_g[~pos] == 0)
    assert int(st.sum()) > 50


@pytest.mark.parametrize("shape", [(128, 2), (512, 16), (64, 1)])
def test_launch_shape_does_not_change_results(B, BA, scenes2, shape):
    jobs = make_jobs(BA, scenes2)
    n = sum(j.n_points for j in jobs)
    ref = BA.BatchRunner(8, n, 1 << 20, use_graph=False)
    ref.submit(jobs)
    assert ref.result()[0] == 0
    want = [j.E_out.cpu().numpy().copy() for j in jobs]
    r = BA.BatchRunner(8, n, 1 << 20, block_threads=shape[0], blocks_per_sm=shape[1], use_graph=True)
    r.submit(jobs)
    assert r.result()[0] == 0
    for j, w in zip(jobs, want):
        assert same_bits(j.E_out.cpu().numpy(), w)


def test_batch_capacities_reported(B, BA, scenes2):
    jobs = make_jobs(BA, scenes2)
    n = sum(j.n_points for j in jobs)
    r = BA.BatchRunner(8, n, 16, use_graph=True)
    r.submit(jobs)
    status, cnt = r.result()
    assert status == B.BNB_ERR_CAPACITY and cnt[1] > 16
    r2 = BA.BatchRunner(8, n, int(cnt[1]), use_graph=True)
    r2.submit(jobs)
    assert r2.result()[0] == 0
    # more points than max_points, written straight into the table: reported on the device
    r3 = BA.BatchRunner(8, n - 1, 1 << 20, use_graph=False)
    for i, j in enumerate(jobs):
        j.scene.fill_job(r3.table[i], j.su, j.sv, j.E_out, j.seed)
    r3.host_n[0] = len(jobs)
    with torch.cuda.stream(r3.stream):
        r3._enqueue()
    r3.done.record(r3.stream)
    assert r3.result()[0] == B.BNB_ERR_CAPACITY
    # an empty batch is valid and touches nothing
    r2.submit([])
    assert r2.result() == (0, [0, 0, 0])


def test_autotune_picks_a_candidate_and_caches(B, BA, scenes2, tmp_path, monkeypatch):
    monkeypatch.setenv("BNB_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    jobs = make_jobs(BA, scenes2)
    cands = [(128, 4), (256, 8)]
    e = BA.autotune(jobs, 1 << 20, reps=2, candidates=cands)
    assert (e["block_threads"], e["blocks_per_sm"]) in cands and e["ms"] > 0
    assert BA.autotune(jobs, 1 << 20, candidates=cands) == e  # served from the cache file
    assert os.path.exists(tmp_path / "tune.json")


def test_serving_results_same_alone_and_in_the_mix(B):
    """Requests served by the continuous-batching loop (several per batch, graphs replayed) give
    bit-identical estimates to the same requests served one at a time."""
    from paper_2504_19163_gb300 import serving as SV
    cache = SV.SceneCache(S.serving_scene, budget_bytes=4 << 30)
    try:
        reqs = SV.make_requests(24, seed=3, scene_names=("serve32",), sides=(64, 128))
        SV.poisson_arrivals(reqs, rate=2000.0, seed=3)
        srv = SV.Server(cache, max_jobs=8, max_points=1 << 16)
        srv.warm_up()
        SV.reset(reqs)
        srv.serve(reqs, timeout_s=120.0)
        assert all(r.E is not None and r.status == 0 for r in reqs)
        assert max(srv.batch_sizes) > 1
        mixed = {r.rid: r.E.copy() for r in reqs}
        SV.reset(reqs)
        SV.plain_cached(reqs, cache, honour_arrivals=False)
        for r in reqs:
            assert same_bits(r.E, mixed[r.rid]), r.rid
        assert sum(float(np.sum(v)) for v in mixed.values()) > 0
        s = SV.summarize(reqs)
        assert s["completed"] == len(reqs)
    finally:
        cache.close()


def bound_cases():
    return [S.config("mirror32"),
            S.config("tiny", n=5, depth=1, lights=[(0.1, -0.05, 2.0), (-0.4, 0.3, 1.7), (0.5, 0.5, 2.5)]),
            S.config("water", n=6, depth=2, steep=0.08, lights=[(0.3, 0.2, 1.2)])]


def test_batched_bound_equals_single_scene(B, BA):
    """Three scenes (two mirrors, one refracting water surface) in one batched bound launch: every
    job's base records are bit-identical to the single-scene pass with no extra split levels."""
    items, singles = [], []
    for sc in bound_cases():
        ds = B.DeviceScene(sc)
        nb = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
        items.append((ds, sc.depth, B.CellBounds(nb, ds.device)))
        singles.append(B.bound_tuples(ds, sc.depth, max_extra_split=0))
    BA.bound_batched(items)
    torch.cuda.synchronize()
    for (ds, depth, out), single in zip(items, singles):
        nb = out.c.n_base
        assert int(out.status.item()) == 0 and int(out.count.item()) == nb == int(single.count.item())
        a, b = out.to_numpy(), single.to_numpy()
        for k in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "e_lo"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
        for k in ("emitter", "tri0", "tri1", "cell", "flags"):
            assert np.array_equal(a[k], b[k]), k
    assert any(np.any(o.to_numpy()["flags"] & 1) for _, _, o in items)


def test_batched_bound_capacity_is_per_job(B, BA):
    sc1, sc2 = bound_cases()[:2]
    ds1, ds2 = B.DeviceScene(sc1), B.DeviceScene(sc2)
    n1 = sc1.emitters.n * sc1.s1.n_tris * 4 ** sc1.depth
    n2 = sc2.emitters.n * sc2.s1.n_tris * 4 ** sc2.depth
    small = B.CellBounds(n1 - 1, ds1.device)
    ok = B.CellBounds(n2, ds2.device)
    BA.bound_batched([(ds1, sc1.depth, small), (ds2, sc2.depth, ok)])
    torch.cuda.synchronize()
    assert int(small.status.item()) == B.BNB_ERR_CAPACITY and int(small.count.item()) == 0
    assert int(ok.status.item()) == 0 and int(ok.count.item()) == n2


def test_serving_prefetch_builds_scenes_in_one_batch(B):
    """The cache builds two catalogue scenes with one batched bound launch; requests on both are
    then served bit-identically in the mix and alone."""
    from paper_2504_19163_gb300 import serving as SV
    cache = SV.SceneCache(S.serving_scene, budget_bytes=8 << 30)
    try:
        es = cache.prefetch(["serve32", "serve256"])
        for e in es:
            assert e.ready.wait(600) and e.error is None and e.resident is not None
        reqs = SV.make_requests(12, seed=4, scene_names=("serve32", "serve256"), sides=(64,))
        SV.poisson_arrivals(reqs, rate=5000.0, seed=4)
        srv = SV.Server(cache, max_jobs=8, max_points=1 << 16)
        srv.warm_up()
        srv.serve(reqs, timeout_s=120.0)
        assert all(r.E is not None and r.status == 0 for r in reqs)
        mixed = {r.rid: r.E.copy() for r in reqs}
        SV.reset(reqs)
        SV.plain_cached(reqs, cache, honour_arrivals=False)
        for r in reqs:
            assert same_bits(r.E, mixed[r.rid]), r.rid
    finally:
        cache.close()


def test_batched_bound_encloses_the_single_pass_split_cells(B, BA):
    """Steep water at depth 2: the single pass splits the cells whose position denominator has no
    certified sign (up to 4 extra levels); the batched pass takes no extra level and bounds such a
    cell at once (reciprocal rule or the receiver box).  Where the single pass did not split, the
    records are bit-identical; where it did, the batched record is live and holds the box and the
    E_hi of every live descendant the single pass produced (looser, still a valid bound)."""
    sc = S.config("water", n=8, depth=2, steep=0.3, lights=[(0.8, 0.2, 0.6)])
    ds = B.DeviceScene(sc)
    nb = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    out = B.CellBounds(nb, ds.device)
    BA.bound_batched([(ds, sc.depth, out)])
    single = B.bound_tuples(ds, sc.depth)
    torch.cuda.synchronize()
    assert int(out.status.item()) == 0 and int(single.status.item()) == 0
    a, s = out.to_numpy(), single.to_numpy()
    assert a["u_lo"].shape[0] == nb and s["u_lo"].shape[0] > nb
    split = (s["flags"][:nb] & 2) != 0
    assert split.sum() > 20
    keep = ~split
    for k in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi"):
        assert np.array_equal(a[k][keep].view(np.uint32), s[k][:nb][keep].view(np.uint32)), k
    for k in ("emitter", "tri0", "cell", "flags"):
        assert np.array_equal(a[k][keep], s[k][:nb][keep]), k
    # descendants of each split base cell: same (emitter, triangle), cell id prefix = the base id
    d = s["flags"][nb:] >> np.uint32(24)
    live = (s["flags"][nb:] & 1) != 0
    anc = s["cell"][nb:].astype(np.int64) >> (2 * (d.astype(np.int64) - sc.depth))
    base_of = {(int(e), int(t), int(c)): i for i, (e, t, c) in
               enumerate(zip(a["emitter"], a["tri0"], a["cell"]))}
    checked = 0
    for j in np.nonzero(live)[0]:
        i = base_of[(int(s["emitter"][nb + j]), int(s["tri0"][nb + j]), int(anc[j]))]
        assert split[i]
        assert a["flags"][i] & 1, i
        assert a["u_lo"][i] <= s["u_lo"][nb + j] and a["u_hi"][i] >= s["u_hi"][nb + j]
        assert a["v_lo"][i] <= s["v_lo"][nb + j] and a["v_hi"][i] >= s["v_hi"][nb + j]
        assert a["e_hi"][i] >= s["e_hi"][nb + j]
        checked += 1
    assert checked > 20
