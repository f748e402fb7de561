"""The read-back entry point that allocates nothing.

ipc_read_gel_surface_all_noalloc serves callers that cannot allocate device
memory when they read results back: it stages through a fixed device array
compiled into the library instead of workspace scratch.  It must return the
same coated-surface positions as ipc_read_gel_surface_all, call after call
(the shared staging array keeps the previous call's contents).

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402

build()


def _step(genv, scs, k):
    for e, s in enumerate(scs):
        t = genv.rest_y(e)
        t[:, :3] += s.delta(k)[:, :3]
        genv.set_targets(e, t)
    status, _ = genv.step()
    assert np.all(status == 0)


def test_noalloc_read_back_matches_workspace_read_back():
    # an uneven batch so that the envs' rows interleave differently in HBM
    scs = [scenes.config0(), scenes.config2(1), scenes.config0()]
    genv = ipc.Envs([s.scene for s in scs], scenes.SolverParams())
    n_rows = sum(s_[2] for s_ in genv.sizes)
    assert 0 < n_rows <= 262144
    for k in range(2):          # two calls in a row, the state changing between them
        _step(genv, scs, k)
        ref = genv.read_gel_surface_all()
        got = genv.read_gel_surface_all_noalloc()
        assert got.shape == ref.shape == (n_rows, 3)
        # the same FP64 values moved through a different staging buffer
        assert np.array_equal(got, ref)
        # and a second call right after returns them again
        again = genv.read_gel_surface_all_noalloc(np.full_like(ref, np.nan))
        assert np.array_equal(again, ref)
    # a capacity smaller than the row count copies only the leading rows
    part = genv.read_gel_surface_all_noalloc(np.zeros((7, 3)))
    assert np.array_equal(part, ref[:7])
    genv.close()


def test_noalloc_capacity_zero_reports_count_and_writes_nothing():
    import ctypes as C
    scs = [scenes.config0(), scenes.config0()]
    genv = ipc.Envs([s.scene for s in scs], scenes.SolverParams())
    n_all = sum(s_[2] for s_ in genv.sizes)
    out = np.full((4, 3), np.nan)
    w = C.c_size_t(12345)
    st = ipc.lib().ipc_read_gel_surface_all_noalloc(genv._ctx, out.ctypes.data_as(C.POINTER(C.c_double)), 0,
                                                     C.byref(w))
    assert st == ipc.IPC_OK
    assert w.value == n_all
    assert np.all(np.isnan(out))
    genv.close()


def test_noalloc_rejects_more_rows_than_its_fixed_array():
    # 14 unpinned two-layer 100 x 100 pads: every vertex is on the coated
    # surface, 14 x 20000 = 280000 rows > 262144
    sc = scenes.free_fall_scene(nx=100, ny=100, nz=2, with_body=False).scene
    genv = ipc.Envs([sc] * 14, scenes.SolverParams())
    n_all = sum(s_[2] for s_ in genv.sizes)
    assert n_all == 280000
    with pytest.raises(ipc.IpcError) as ei:
        genv.read_gel_surface_all_noalloc()
    assert ei.value.status == ipc.IPC_EINVAL
    assert "262144" in str(ei.value) and "exceed" in str(ei.value)
    # the workspace read-back has no such limit
    ref = genv.read_gel_surface_all()
    assert ref.shape == (n_all, 3) and np.all(np.isfinite(ref))
    genv.close()
