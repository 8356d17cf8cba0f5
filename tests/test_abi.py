"""The C-ABI library loads on a machine without a GPU, exports every function that
include/*.h declares, and rejects bad arguments on the host (no launch)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bnb():
    from paper_2504_19163_gb300 import build as B
    B.build()
    from paper_2504_19163_gb300 import bnb as M
    return M


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(bnb_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(bnb):
    names = declared_functions()
    assert {"bnb_bound_tuples", "bnb_build_index", "bnb_sample_and_solve"} <= names
    L = C.CDLL(bnb.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(bnb.EXPORTS) == names


def test_status_strings_and_version(bnb):
    assert bnb.bnb_status_string(0) == "ok"
    assert "capacity" in bnb.bnb_status_string(-2)
    assert bnb.lib().bnb_abi_version() == 11


def test_workspace_queries_are_host_only(bnb):
    s = bnb.bnb_surface()
    s.n_tris = 2048
    s.n_verts = 33 * 33
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)  # dummy non-null pointers: the queries never dereference them
    em = bnb.bnb_emitters(1, 4096, 4096, 4096, 4096)
    cfg = bnb.bnb_bound_cfg(2, 4, 1, 0)
    wb = bnb.bnb_bound_tuples_ws(C.byref(s), None, C.byref(em), C.byref(cfg))
    assert wb >= 2048 * 80
    assert bnb.bnb_build_index_ws(None, 512, 1000) > 512 * 512 * 8 * 3
    assert bnb.bnb_build_index_ws(None, 0, 1000) == 0
    assert bnb.bnb_sample_and_solve_ws(C.byref(s), None, 4096, 10000) > 10000 * 24
    s2 = bnb.bnb_surface()
    C.pointer(s2)[0] = s
    s2.n_tris = 4608
    s2.kind = s.kind = bnb.BNB_REFRACT
    wp = bnb.bnb_bound_tuples_ws(C.byref(s), C.byref(s2), C.byref(em), C.byref(cfg))
    assert wp >= (2048 + 4608) * 80 + 2048 * 16 * 16  # both packed meshes, per-cell counts and offsets
    assert (bnb.bnb_sample_and_solve_ws(C.byref(s), C.byref(s2), 4096, 10000) -
            bnb.bnb_sample_and_solve_ws(C.byref(s), None, 4096, 10000)) >= 4608 * 80
    # adaptive subdivision: a caller-sized split queue widens the workspace; bad fields are refused
    ad = bnb.bnb_bound_cfg(2, 4, 1, 0, 6, 1e-4, 2.0, 0, 1 << 20)
    assert bnb.bnb_bound_tuples_ws(C.byref(s), None, C.byref(em), C.byref(ad)) >= 2 * (1 << 20) * 16  # two queues
    assert bnb.bnb_bound_tuples_ws(C.byref(s), None, C.byref(em), C.byref(
        bnb.bnb_bound_cfg(2, 4, 1, 0, 0, 0.0, 0.0, 0, -1))) == 0
    bad = bnb.bnb_bound_cfg(11, 0, 1, 0)
    assert bnb.bnb_bound_tuples_ws(C.byref(s), None, C.byref(em), C.byref(bad)) == 0


def test_invalid_arguments_rejected_before_launch(bnb):
    s = bnb.bnb_surface()
    s.n_tris = 8
    s.n_verts = 9
    rec = bnb.bnb_receiver()
    em = bnb.bnb_emitters(1, None, None, None, None)  # n > 0 with NULL arrays
    cfg = bnb.bnb_bound_cfg(1, 0, 1, 0)
    out = bnb.bnb_cell_bounds()
    rc = bnb.bnb_bound_tuples(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(cfg), C.byref(out), None, 0, None)
    assert rc == bnb.BNB_ERR_INVALID
    # chains: a refracting second vertex with eta' outside (0, 1e6) is unsupported
    em_ok = bnb.bnb_emitters(1, 4096, 4096, 4096, 4096)
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)
    s2 = bnb.bnb_surface()
    C.pointer(s2)[0] = s
    s2.kind, s2.eta = bnb.BNB_REFRACT, 0.0
    rc = bnb.bnb_bound_tuples(C.byref(s), C.byref(s2), C.byref(rec), C.byref(em_ok), C.byref(cfg), C.byref(out),
                              None, 0, None)
    assert rc == bnb.BNB_ERR_UNSUPPORTED
    idx = bnb.bnb_index()
    assert bnb.bnb_build_index(None, 1.0, 0, C.byref(idx), None, 0, None) == bnb.BNB_ERR_INVALID
    cells = bnb.bnb_cell_bounds()
    assert bnb.bnb_build_index(C.byref(cells), 1.0, 0, C.byref(idx), None, 0, None) == bnb.BNB_ERR_INVALID
    scfg = bnb.bnb_sample_cfg(1.0, 0, 100, 2, 1e-5, 0)  # newton_iters > 64
    stats = bnb.bnb_sample_stats()
    rc = bnb.bnb_sample_and_solve(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(idx), None, None, 0,
                                  C.byref(scfg), None, C.byref(stats), None, 0, None)
    assert rc == bnb.BNB_ERR_INVALID


def test_new_configuration_fields_rejected_before_launch(bnb):
    """Adaptive depth beyond the cell-id limit, a negative split capacity, a bins flag other than 0/1
    and a negative stochastic-trial cap are refused by the argument checks (nothing is launched)."""
    s = bnb.bnb_surface()
    s.n_tris, s.n_verts = 8, 9
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)
    em = bnb.bnb_emitters(1, 4096, 4096, 4096, 4096)
    rec = bnb.bnb_receiver()
    out = bnb.bnb_cell_bounds()
    out.capacity = 0
    out.count = out.status = 4096
    for cfg in (bnb.bnb_bound_cfg(1, 4, 1, 0, 16, 0.0, 0.0, 0, 0),   # adapt_depth > 15
                bnb.bnb_bound_cfg(1, 4, 1, 0, 12, 0.0, 0.0, 0, 0),   # adapt_depth + extra splits > 15
                bnb.bnb_bound_cfg(1, 4, 1, 0, 3, -1.0, 0.0, 0, 0),   # sigma < 0
                bnb.bnb_bound_cfg(1, 4, 1, 0, 3, 0.0, float("nan"), 0, 0),
                bnb.bnb_bound_cfg(1, 4, 1, 0, 0, 0.0, 0.0, 0, -5)):  # split capacity < 0
        rc = bnb.bnb_bound_tuples(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(cfg), C.byref(out), None, 0,
                                  None)
        assert rc == bnb.BNB_ERR_INVALID
    idx = bnb.bnb_index()
    idx.grid_res, idx.capacity, idx.count, idx.status, idx.offsets = 512, 0, 4096, 4096, 4096
    stats = bnb.bnb_sample_stats(4096, 4096, None)
    for scfg in (bnb.bnb_sample_cfg(1.0, 0, 16, 1, 1e-5, 0, 2, 0), bnb.bnb_sample_cfg(1.0, 0, 16, 1, 1e-5, 0, 0, -1)):
        rc = bnb.bnb_sample_and_solve(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(idx), None, None, 0,
                                      C.byref(scfg), None, C.byref(stats), None, 0, None)
        assert rc == bnb.BNB_ERR_INVALID
    # stochastic starts for two-vertex chains are not built
    s2 = bnb.bnb_surface()
    C.pointer(s2)[0] = s
    s.kind = s2.kind = bnb.BNB_REFRACT
    s.eta, s2.eta = 0.66, 1.5
    scfg = bnb.bnb_sample_cfg(1.0, 0, 16, 1, 1e-5, 0, 0, 8)
    rc = bnb.bnb_sample_and_solve(C.byref(s), C.byref(s2), C.byref(rec), C.byref(em), C.byref(idx), None, None, 0,
                                  C.byref(scfg), None, C.byref(stats), None, 0, None)
    assert rc == bnb.BNB_ERR_UNSUPPORTED


def test_no_oracle_import_in_library_path():
    """The product path never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2504_19163_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert "import oracle" not in src and "from oracle" not in src and "liboracle" not in src, f


def test_ctypes_structs_match_the_header(bnb, tmp_path):
    """Field offsets and sizes of the Python mirrors equal the C compiler's for every struct."""
    structs = {n: getattr(bnb, n) for n in ("bnb_surface", "bnb_receiver", "bnb_emitters", "bnb_bound_cfg",
                                              "bnb_cell_bounds", "bnb_index", "bnb_sample_cfg", "bnb_sample_stats",
                                              "bnb_job", "bnb_batch_cfg", "bnb_bound_job")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "bnb.h")}"',
             "int main(void) {"]
    for n, cls in structs.items():
        lines.append(f'  printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        n, f, v = ln.split()
        got[(n, f)] = int(v)
    for n, cls in structs.items():
        assert got[(n, "sizeof")] == C.sizeof(cls), n
        for f, _ in cls._fields_:
            assert got[(n, f)] == getattr(cls, f).offset, (n, f)


def test_batched_queries_and_rejections_are_host_only(bnb):
    s = bnb.bnb_surface()
    s.n_tris = 100
    s.n_verts = 121
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)
    assert bnb.bnb_pack_surface_bytes(C.byref(s)) == 100 * 80
    assert bnb.bnb_pack_surface(C.byref(s), 4096, 100, None) == bnb.BNB_ERR_INVALID  # too small
    assert bnb.bnb_pack_surface(C.byref(s), 4100, 8000, None) == bnb.BNB_ERR_INVALID  # misaligned
    cfg = bnb.bnb_batch_cfg(16, 16, 1 << 20, 1 << 22, 2, 1e-5, 0, 0)
    ws = bnb.bnb_sample_and_solve_batched_ws(C.byref(cfg))
    assert ws >= (1 << 20) * 16 + (1 << 22) * 24
    for bad in (bnb.bnb_batch_cfg(0, 16, 1, 1, 2, 1e-5, 0, 0),         # no job slot
                bnb.bnb_batch_cfg(16, 65, 1, 1, 2, 1e-5, 0, 0),        # newton_iters > 64
                bnb.bnb_batch_cfg(16, 16, 1, 1, 2, 0.0, 0, 0),         # tol <= 0
                bnb.bnb_batch_cfg(16, 16, 1, 1, 2, 1e-5, 96 + 1, 0),   # not a multiple of 32
                bnb.bnb_batch_cfg(16, 16, 1, 1, 2, 1e-5, 1024, 0),     # above 512 threads
                bnb.bnb_batch_cfg(16, 16, 1, 1, 2, 1e-5, 0, 65)):      # blocks_per_sm > 64
        assert bnb.bnb_sample_and_solve_batched_ws(C.byref(bad)) == 0
    stats = bnb.bnb_sample_stats(4096, 4096, None)
    assert bnb.bnb_sample_and_solve_batched(4096, 4096, C.byref(cfg), C.byref(stats), 4096, 100, None) == \
        bnb.BNB_ERR_INVALID  # workspace too small
    assert bnb.bnb_sample_and_solve_batched(None, 4096, C.byref(cfg), C.byref(stats), 4096, ws, None) == \
        bnb.BNB_ERR_INVALID
    assert bnb.bnb_sample_and_solve_batched(4100, 4096, C.byref(cfg), C.byref(stats), 4096, ws, None) == \
        bnb.BNB_ERR_INVALID  # job table not 8-byte aligned


def test_implicit_irradiance_arguments(bnb):
    """Argument checks of the implicit-differentiation pass, all before any launch."""
    s = bnb.bnb_surface()
    s.n_tris, s.n_verts = 8, 9
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)
    rec = bnb.bnb_receiver()
    em = bnb.bnb_emitters(1, 4096, 4096, 4096, 4096)
    cells = bnb.bnb_cell_bounds()
    cells.capacity = 16
    s.kind = bnb.BNB_REFLECT
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), 0, 0, None) == \
        bnb.BNB_ERR_UNSUPPORTED
    s.kind, s.eta = bnb.BNB_REFRACT, 0.75
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), 0, 2, None) == \
        bnb.BNB_ERR_INVALID
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), 17, 0, None) == \
        bnb.BNB_ERR_INVALID
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), -1, 0, None) == \
        bnb.BNB_ERR_INVALID  # n = -1 needs the device count
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), 0, 1, None) == \
        bnb.BNB_OK
    assert bnb.bnb_implicit_irradiance(C.byref(s), C.byref(rec), C.byref(em), C.byref(cells), 4, 0, None) == \
        bnb.BNB_ERR_INVALID  # record arrays missing
    # the bound pass: irradiance 2 needs a refracting surface, 3 is not a mode
    out = bnb.bnb_cell_bounds()
    out.capacity = 1 << 20
    out.count = 4096
    out.status = 4096
    for f in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "emitter", "tri0", "tri1", "cell", "flags"):
        setattr(out, f, 4096)
    cfg = bnb.bnb_bound_cfg(1, 0, 3, 0)
    assert bnb.bnb_bound_tuples(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(cfg), C.byref(out), None, 0,
                                None) == bnb.BNB_ERR_INVALID
    s.kind = bnb.BNB_REFLECT
    cfg = bnb.bnb_bound_cfg(1, 0, 2, 0)
    assert bnb.bnb_bound_tuples(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(cfg), C.byref(out), None, 0,
                                None) == bnb.BNB_ERR_UNSUPPORTED


def test_gamma_for_target_arguments(bnb):
    """Argument checks of the gamma <-> E|S| call (Sec. 5.4), all before any launch."""
    assert bnb.bnb_gamma_for_target_ws(512) >= 512 * 512 * 4
    assert bnb.bnb_gamma_for_target_ws(0) == 0
    idx = bnb.bnb_index()
    idx.grid_res, idx.capacity, idx.count, idx.status, idx.offsets, idx.key, idx.etilde = 512, 16, 4096, 4096, 4096, \
        4096, 4096
    ws = bnb.bnb_gamma_for_target_ws(512)
    g = C.c_void_p(4096)
    call = bnb.bnb_gamma_for_target
    assert call(None, None, None, 0, 4.0, g, 4096, ws, None) == bnb.BNB_ERR_INVALID            # no index
    assert call(C.byref(idx), None, None, 0, 4.0, None, 4096, ws, None) == bnb.BNB_ERR_INVALID  # no output
    assert call(C.byref(idx), None, None, 0, float("nan"), g, 4096, ws, None) == bnb.BNB_ERR_INVALID
    assert call(C.byref(idx), None, None, 0, -1.0, g, 4096, ws, None) == bnb.BNB_ERR_INVALID
    assert call(C.byref(idx), 4096, None, 10, 4.0, g, 4096, ws, None) == bnb.BNB_ERR_INVALID    # su without sv
    assert call(C.byref(idx), 4096, 4096, 0, 4.0, g, 4096, ws, None) == bnb.BNB_ERR_INVALID     # no points
    assert call(C.byref(idx), None, None, 0, 4.0, g, 4096, ws - 1, None) == bnb.BNB_ERR_INVALID  # small workspace
    assert call(C.byref(idx), None, None, 0, 4.0, g, 4100, ws, None) == bnb.BNB_ERR_INVALID     # misaligned
    idx.grid_res = 0
    assert call(C.byref(idx), None, None, 0, 4.0, g, 4096, ws, None) == bnb.BNB_ERR_INVALID


def test_ffma_probe_arguments(bnb):
    for args in ((0, 256, 1, 0), (8, 33, 1, 0), (8, 2048, 1, 0), (8, 256, 0, 0), (8, 256, 1, 2)):
        assert bnb.bnb_ffma_probe(*args, 4096, None) == bnb.BNB_ERR_INVALID
    assert bnb.bnb_ffma_probe(8, 256, 1, 0, None, None) == bnb.BNB_ERR_INVALID


def test_bound_block_threads_checked(bnb):
    s = bnb.bnb_surface()
    s.n_tris, s.n_verts = 8, 9
    for f in ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2"):
        setattr(s, f, 4096)
    em = bnb.bnb_emitters(1, 4096, 4096, 4096, 4096)
    rec = bnb.bnb_receiver()
    out = bnb.bnb_cell_bounds()
    out.capacity = 1 << 20
    out.count = out.status = 4096
    for f in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "emitter", "tri0", "tri1", "cell", "flags"):
        setattr(out, f, 4096)  # never dereferenced: the block size is refused before any launch
    cfg = bnb.bnb_bound_cfg(1, 4, 1, 0, 0, 0.0, 0.0, 300, 0)  # not a compiled block size
    assert bnb.bnb_bound_tuples(C.byref(s), None, C.byref(rec), C.byref(em), C.byref(cfg), C.byref(out), None, 0,
                                None) == bnb.BNB_ERR_INVALID
