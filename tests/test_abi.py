"""The C-ABI library builds for sm_103a, loads, exports every function that
include/difftrans.h declares, and the Python binding's struct layouts match
the header's (checked by compiling a probe against the header with gcc).
No GPU is needed and no compute entry point is called."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "difftrans.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_00413_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dt_build_bvh", "dt_render", "dt_render_backward", "dt_refit_bvh", "dt_vertex_normals"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_header():
    import paper_2603_00413_gb300 as dt
    assert set(_declared_functions()) == set(dt._PROTOS)


def test_no_cuda_needed_for_size_queries(lib):
    import paper_2603_00413_gb300 as dt
    dt._lib = None
    L = dt.load_library()
    bb, sb = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.dt_bvh_size(1280, ctypes.byref(bb), ctypes.byref(sb)) == 0
    assert bb.value >= 1279 * 64 + 1280 * 48 and sb.value > 0
    assert L.dt_bvh_size(0, ctypes.byref(bb), ctypes.byref(sb)) == dt.DT_ERR_INVALID_ARG
    assert b"nf" in L.dt_last_error()
    wb = ctypes.c_size_t()
    assert L.dt_render_workspace_size(1000, ctypes.byref(wb)) == 0
    assert wb.value >= 1000 * 72
    assert L.dt_render_workspace_size(0, ctypes.byref(wb)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_render_workspace_size(2 ** 31, ctypes.byref(wb)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_backward_workspace_size(10, 5, ctypes.byref(wb)) == 0
    assert L.dt_version() == b"difftrans-gb300 0.3 (sm_103a)"


def test_host_side_argument_checks_fire_before_any_launch(lib):
    """NULL pointers are rejected on the host, without touching a GPU."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    assert L.dt_render(None, None, None, None, None, 0, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_build_bvh(None, 3, None, 1, None, None, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_vertex_normals(None, 3, None, 1, None, None, None) == dt.DT_ERR_INVALID_ARG
    sc = dt.DtScene()
    assert L.dt_render(ctypes.byref(sc), None, None, None, None, 0, None) == dt.DT_ERR_INVALID_ARG
    assert b"NULL" in L.dt_last_error()


def test_tuning_round_trips_and_is_validated(lib):
    """dt_get_tuning / dt_set_tuning are host-only; a rejected set changes
    nothing."""
    import paper_2603_00413_gb300 as dt
    old = dt.get_tuning()
    assert (old["trace_order"] == 0 or 12 <= old["trace_order"] <= 22) and old["bvh_width"] in (2, 4)
    try:
        dt.set_tuning(trace_order=0)
        assert dt.get_tuning()["trace_order"] == 0
        dt.set_tuning(order_min_rays=0)
        assert dt.get_tuning()["order_min_rays"] == 0
        dt.set_tuning(order_min_rays=old["order_min_rays"])
        for bad in (dict(trace_order=1), dict(trace_order=23), dict(bvh_width=3), dict(trace_steps=0),
                    dict(bvh_builder=-1), dict(order_min_rays=-1)):
            with pytest.raises(dt.DiffTransError):
                dt.set_tuning(**bad)
        assert dt.get_tuning() == dict(old, trace_order=0)
    finally:
        dt.set_tuning(**old)


def test_struct_layouts_match_header():
    import paper_2603_00413_gb300 as dt
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "difftrans.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(dt_scene), sizeof(dt_views), sizeof(dt_params), sizeof(dt_stats));
  printf("%zu %zu %zu %zu\n", offsetof(dt_scene, env_w), offsetof(dt_params, seed), offsetof(dt_params, t_min),
         offsetof(dt_stats, max_level));
  printf("%zu %zu %zu\n", sizeof(dt_batch_entry), offsetof(dt_batch_entry, d_grad_sigma), sizeof(dt_tuning));
  printf("%zu %zu %zu\n", offsetof(dt_params, tape_mode), offsetof(dt_params, level_capacity),
         offsetof(dt_stats, level_needed));
  printf("%zu %zu %zu %zu %zu\n", sizeof(dt_medium), offsetof(dt_medium, lo), offsetof(dt_medium, step),
         offsetof(dt_scene, medium), offsetof(dt_stats, medium_samples));
  printf("%zu\n", offsetof(dt_scene, d_grad_env));
  printf("%zu %zu %zu %d\n", offsetof(dt_medium, levels), offsetof(dt_medium, log2_table), offsetof(dt_medium, res),
         DT_MAX_HASH_LEVELS);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(probe)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:4] == [ctypes.sizeof(dt.DtScene), ctypes.sizeof(dt.DtViews), ctypes.sizeof(dt.DtParams),
                         ctypes.sizeof(dt.DtStats)]
    assert sizes[4:8] == [dt.DtScene.env_w.offset, dt.DtParams.seed.offset, dt.DtParams.t_min.offset,
                          dt.DtStats.max_level.offset]
    assert sizes[8:11] == [ctypes.sizeof(dt.DtBatchEntry), dt.DtBatchEntry.d_grad_sigma.offset,
                           ctypes.sizeof(dt.DtTuning)]
    assert sizes[11:14] == [dt.DtParams.tape_mode.offset, dt.DtParams.level_capacity.offset,
                            dt.DtStats.level_needed.offset]
    assert sizes[14:19] == [ctypes.sizeof(dt.DtMedium), dt.DtMedium.lo.offset, dt.DtMedium.step.offset,
                            dt.DtScene.medium.offset, dt.DtStats.medium_samples.offset]
    assert sizes[19:20] == [dt.DtScene.d_grad_env.offset]
    assert sizes[20:] == [dt.DtMedium.levels.offset, dt.DtMedium.log2_table.offset, dt.DtMedium.res.offset,
                          dt.MAX_HASH_LEVELS]


def test_checkpointed_workspace_is_smaller_and_validated():
    """A checkpointed workspace drops the per-segment hit records (16 of 72
    bytes) for a two-level ring; bad tape modes and ring sizes are refused."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    cap, ring = 10_000_000, 1_000_000
    full = dt.render_workspace_size(cap)
    ck = dt.render_workspace_size(cap, ring)
    assert full - ck == pytest.approx(16 * (cap - 2 * ring), abs=4096)
    b = ctypes.c_size_t()
    assert L.dt_render_workspace_size_ex(cap, 0, 0, ctypes.byref(b)) == dt.DT_OK and b.value == full
    assert L.dt_render_workspace_size_ex(cap, 3, ring, ctypes.byref(b)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_render_workspace_size_ex(cap, -1, 0, ctypes.byref(b)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_render_workspace_size_ex(cap, 1, 0, ctypes.byref(b)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_render_workspace_size_ex(cap, 1, cap + 1, ctypes.byref(b)) == dt.DT_ERR_INVALID_ARG


def test_moments_workspace_adds_96_bytes_per_segment():
    """tape_mode 2 keeps the full tape and 24 floats of medium moments per
    segment; the binding sizes it through the same query and refuses a
    checkpointed tape that would also keep moments."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    cap = 10_000_000
    full = dt.render_workspace_size(cap)
    mom = dt.render_workspace_size(cap, moments=True)
    assert mom - full == pytest.approx(96 * cap, abs=512)
    b = ctypes.c_size_t()
    assert L.dt_render_workspace_size_ex(cap, 2, 0, ctypes.byref(b)) == dt.DT_OK and b.value == mom
    assert L.dt_render_workspace_size_ex(cap, 2, 12345, ctypes.byref(b)) == dt.DT_OK and b.value == mom
    assert dt.Params(4, moments=True).c().tape_mode == 2
    assert dt.Params(4).c().tape_mode == 0 and dt.Params(4, checkpoint=True).c(10).tape_mode == 1
    with pytest.raises(ValueError):
        dt.Params(4, checkpoint=True, moments=True)
    # the parameters and the workspace must agree on the moments
    from types import SimpleNamespace
    plain, with_moments = SimpleNamespace(level_capacity=0, moments=False), SimpleNamespace(level_capacity=0, moments=True)
    assert dt._effective_params(dt.Params(4, moments=True), with_moments).tape_mode == 2
    for p, w in ((dt.Params(4, moments=True), plain), (dt.Params(4), with_moments)):
        with pytest.raises(ValueError):
            dt._effective_params(p, w)


def test_python_calls_fail_loudly_without_the_library(tmp_path):
    import paper_2603_00413_gb300 as dt
    saved = dt._lib
    dt._lib = None
    try:
        with pytest.raises(RuntimeError, match="no fallback"):
            dt.load_library(str(tmp_path / "missing.so"))
    finally:
        dt._lib = saved


def test_absorption_fields_are_validated_on_the_host(lib):
    """dt_render checks a scene's absorption field (dense grid or hash
    texture) before it builds the scene table or launches anything: the
    device pointers here are never dereferenced.  A valid field lets the
    check move on to the views."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    fake = 0x10000  # 256-byte aligned, never read

    def scene_with(**kw):
        m = dt.DtMedium()
        m.d_mu = fake
        m.nx = m.ny = m.nz = 4
        for a in range(3):
            m.lo[a], m.hi[a] = -1.0, 1.0
        m.step = 0.05
        for k, v in kw.items():
            if k == "res":
                for i, r in enumerate(v):
                    m.res[i] = r
            else:
                setattr(m, k, v)
        sc = dt.DtScene(fake, fake, 3, 1, fake, fake, fake, fake, fake, 8, 4)
        sc.medium = ctypes.pointer(m)
        return sc, m

    def status(**kw):
        sc, m = scene_with(**kw)
        st = L.dt_render(ctypes.byref(sc), ctypes.byref(dt.DtViews()), ctypes.byref(dt.DtParams()), None, None,
                         0, None)
        return st, L.dt_last_error().decode()

    for kw, words in [(dict(nx=1), "2 nodes per axis"), (dict(step=0.0), "step"), (dict(levels=17), "levels"),
                      (dict(levels=-1), "levels"), (dict(levels=2, log2_table=3, res=[4, 8]), "log2_table"),
                      (dict(levels=2, log2_table=25, res=[4, 8]), "log2_table"),
                      (dict(levels=2, log2_table=10, res=[4, 1]), "level 1"),
                      (dict(levels=1, log2_table=10, res=[(1 << 20) + 1]), "level 0"),
                      (dict(d_mu=fake + 8), "aligned")]:
        st, msg = status(**kw)
        assert st == dt.DT_ERR_INVALID_ARG and words in msg, (kw, msg)
    # valid fields: the dense grid, and a hash texture whose dense-grid sizes are ignored
    for kw in (dict(), dict(levels=3, log2_table=12, res=[4, 16, 64], nx=0, ny=0, nz=0)):
        st, msg = status(**kw)
        assert st == dt.DT_ERR_INVALID_ARG and "d_cams" in msg, (kw, msg)


def test_views_params_and_batches_are_validated_on_the_host(lib):
    """The views, the parameters, the batch size, the output and the
    workspace are checked before anything is launched (the device pointers
    here are never dereferenced); the message names the entry."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    fake = 0x10000

    def entry(**kw):
        e = dt.DtBatchEntry()
        e.scene = dt.DtScene(fake, fake, 3, 1, fake, fake, fake, fake, fake, 8, 4)
        e.views = dt.DtViews(fake, 1, 4, 4)
        e.params = dt.DtParams(4, 1, 0, 0, 0, 1e-5, 0)
        e.d_out = fake
        for k, v in kw.items():
            owner, name = k.split("__")
            setattr(getattr(e, owner) if owner != "e" else e, name, v)
        return e

    def status(entries, ws=fake, ws_bytes=1 << 30):
        arr = (dt.DtBatchEntry * len(entries))(*entries)
        st = L.dt_render_batch(arr, len(entries), ws, ws_bytes, None)
        return st, L.dt_last_error().decode()

    cases = [(dict(views__n_views=0), "n_views"), (dict(views__width=0), "n_views"),
             (dict(params__max_depth=31), "max_depth"), (dict(params__max_depth=-1), "max_depth"),
             (dict(params__spp=0), "spp"), (dict(params__t_min=-1.0), "t_min"),
             (dict(params__tape_mode=3), "tape_mode must be 0, 1 or 2"), (dict(params__tape_mode=1), "level_capacity"),
             (dict(views__n_views=1 << 12, views__width=1 << 10, views__height=1 << 10), "too many primary rays"),
             (dict(e__d_out=None), "d_out"), (dict(scene__nf=0), "nf >= 1")]
    for kw, words in cases:
        st, msg = status([entry(), entry(**kw)])
        assert st == dt.DT_ERR_INVALID_ARG and words in msg and "entry 1" in msg, (kw, msg)
    # every entry valid on its own, but a full tape beside a moments tape
    st, msg = status([entry(), entry(params__tape_mode=2)])
    assert st == dt.DT_ERR_INVALID_ARG and "share tape_mode" in msg and "entry 1" in msg, msg
    st, msg = status([])
    assert st == dt.DT_ERR_INVALID_ARG and "batch size" in msg
    st, msg = status([entry()] * 257)
    assert st == dt.DT_ERR_INVALID_ARG and "batch size" in msg
    st, msg = status([entry()], ws=None)
    assert st == dt.DT_ERR_INVALID_ARG and "workspace is NULL" in msg
    st, msg = status([entry()], ws=fake + 16)
    assert st == dt.DT_ERR_INVALID_ARG and "256-byte aligned" in msg
    st, msg = status([entry(views__n_views=64)], ws_bytes=dt.render_workspace_size(100))
    assert st == dt.DT_ERR_INVALID_ARG and "fewer than the 1024 camera rays" in msg


def test_mesh_update_and_loss_entries_check_their_arguments_on_the_host(lib):
    """Size queries of the mesh update grow with the mesh and the iteration
    count; the entry points refuse bad meshes, NULL or misaligned buffers,
    short scratch and out-of-range hyper-parameters before any launch (the
    device pointers here are never dereferenced)."""
    import paper_2603_00413_gb300 as dt
    L = dt.load_library()
    fake = 0x10000
    b, s = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.dt_topology_size(642, 1280, ctypes.byref(b)) == dt.DT_OK
    small = b.value
    assert L.dt_topology_size(2562, 5120, ctypes.byref(b)) == dt.DT_OK and b.value > small
    for nv, nf in ((2, 1), (3, 0), (3, 1 << 29)):
        assert L.dt_topology_size(nv, nf, ctypes.byref(b)) == dt.DT_ERR_INVALID_ARG
    assert L.dt_smooth_scratch_size(642, 100, ctypes.byref(s)) == dt.DT_OK
    s100 = s.value
    assert L.dt_smooth_scratch_size(642, 200, ctypes.byref(s)) == dt.DT_OK and s.value >= s100
    assert L.dt_smooth_scratch_size(0, 100, ctypes.byref(s)) == dt.DT_ERR_INVALID_ARG
    st_b = ctypes.c_size_t()
    assert L.dt_large_steps_sizes(642, 100, ctypes.byref(st_b), ctypes.byref(s)) == dt.DT_OK
    assert st_b.value >= 642 * 3 * 4 and s.value >= s100
    assert L.dt_large_steps_sizes(642, 0, ctypes.byref(st_b), ctypes.byref(s)) == dt.DT_ERR_INVALID_ARG
    L.dt_topology_size(642, 1280, ctypes.byref(b))
    topo_bytes = b.value
    assert L.dt_build_topology(fake, 1280, 642, fake + 16, topo_bytes, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_build_topology(fake, 1280, 642, fake, topo_bytes - 1, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_build_topology(None, 1280, 642, fake, topo_bytes, None) == dt.DT_ERR_INVALID_ARG
    L.dt_smooth_scratch_size(642, 100, ctypes.byref(s))
    sb = s.value
    for lam, iters, scratch, nbytes in ((-1.0, 100, fake, sb), (float("nan"), 100, fake, sb), (10.0, 0, fake, sb),
                                        (10.0, 100, fake, sb - 1), (10.0, 100, fake + 16, sb)):
        assert L.dt_smooth_solve(fake, 642, 1280, lam, fake, fake, iters, scratch, nbytes, None) == \
            dt.DT_ERR_INVALID_ARG
    L.dt_large_steps_sizes(642, 100, ctypes.byref(st_b), ctypes.byref(s))
    good = dict(lam=10.0, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, iters=100, state=fake, scratch=fake, nbytes=s.value)
    for bad in (dict(b1=1.0), dict(b2=-0.1), dict(eps=0.0), dict(lam=-1.0), dict(state=fake + 8),
                dict(nbytes=s.value - 1), dict(iters=100001)):
        a = dict(good, **bad)
        assert L.dt_large_steps_update(fake, 642, 1280, a["lam"], a["lr"], a["b1"], a["b2"], a["eps"], a["iters"],
                                       fake, fake, a["state"], a["scratch"], a["nbytes"], None) == \
            dt.DT_ERR_INVALID_ARG, bad
    assert L.dt_edge_loss_grad(fake, 642, 1280, fake, None, fake, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_paper_loss_grad(fake, fake, -1, 1.0, 1.0, fake, fake, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_paper_loss_grad(None, fake, 10, 1.0, 1.0, fake, fake, None) == dt.DT_ERR_INVALID_ARG
    assert L.dt_paper_loss_grad(fake, fake, 10, 1.0, 1.0, fake, None, None) == dt.DT_ERR_INVALID_ARG
