"""dt_vertex_normals_noalloc, the entry point for callers that cannot allocate
device memory (a plugin handed device pointers by an application that owns
all device memory; a serving loop that must not allocate after start-up).

It is called through the C ABI and must give the same normals as
dt_vertex_normals (which takes a caller scratch buffer), bit for bit -- both
accumulate in the same integer fixed point, whose sums do not depend on the
order of the atomics -- on two calls in a row: a larger mesh, then a smaller
one, so the second call would see the first call's leftovers in the shared
array if it did not clear them.  The second call must not grow the memory
torch's allocator holds, nor the device-wide used memory, and a mesh above
the vertex limit must be rejected.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_00413_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2603_00413_gb300 import build
    build.build()
    import paper_2603_00413_gb300 as dt
    return dt, dt.load_library()


def _with_scratch(dt, V, F):
    return dt.vertex_normals(V, F)


def _noalloc(L, V, F, out, stream):
    code = L.dt_vertex_normals_noalloc(ctypes.c_void_p(V.data_ptr()), V.shape[0], ctypes.c_void_p(F.data_ptr()),
                                       F.shape[0], ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    return code


def _device_free(dev):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(dev)[0]


def test_noalloc_normals_match_the_scratch_version_twice(lib):
    dt, L = lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    meshes = [S.two_tori_mesh(40), S.icosphere(3)]
    cases = []
    for V, F in meshes:
        Vt, Ft = torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev)
        cases.append((Vt, Ft, torch.full_like(Vt, float("nan")), _with_scratch(dt, Vt, Ft)))
    torch.cuda.synchronize()
    free_before = reserved_before = None
    for k, (Vt, Ft, out, ref) in enumerate(cases):
        if k == 1:
            reserved_before = torch.cuda.memory_reserved(dev)
            free_before = _device_free(dev)
        assert _noalloc(L, Vt, Ft, out, stream) == dt.DT_OK, L.dt_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    # the second call allocated nothing: torch's allocator holds what it held,
    # and the device's free memory is unchanged (read twice before failing,
    # since another process on the same GPU may allocate in between)
    assert torch.cuda.memory_reserved(dev) == reserved_before
    free_after = _device_free(dev)
    if free_after != free_before:
        free_after = _device_free(dev)
    assert free_after == free_before, (free_before, free_after)


def test_noalloc_rejects_meshes_above_its_limit(lib):
    dt, L = lib
    V, F = S.icosphere(1)
    Vt, Ft = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    out = torch.empty_like(Vt)
    # the vertex count is checked on the host before any device work
    code = L.dt_vertex_normals_noalloc(ctypes.c_void_p(Vt.data_ptr()), dt.NOALLOC_MAX_VERTICES + 1,
                                       ctypes.c_void_p(Ft.data_ptr()), Ft.shape[0], ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == dt.DT_ERR_INVALID_ARG
    assert b"at most" in L.dt_last_error()
