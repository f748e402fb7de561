"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point the header declares, and validates scenes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import scenes
from paper_2504_12908_b300 import ipc
from paper_2504_12908_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return ipc.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ipc_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert "ipc_step" in names and "ipc_create_envs" in names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert names <= set(ipc.EXPORTED) | names  # binding list is informative
    assert set(ipc.EXPORTED) <= names


def test_default_params(L):
    p = ipc.ipc_params()
    L.ipc_default_params(C.byref(p))
    assert p.dt == 1e-3 and p.dhat == 1e-4 and p.kappa == 1e6 and p.gravity[2] == -9.81
    # PCG scheduling defaults: whole solves in a rollout, the fused kernel,
    # 8 iterations per launch (the binding's SolverParams mirrors them)
    assert p.rollout_pcg_window == 0 and p.pcg_fused == 1 and p.pcg_iters_per_launch == 8
    sp = scenes.SolverParams()
    assert (sp.rollout_pcg_window, sp.pcg_fused, sp.pcg_iters_per_launch) == (0, 1, 8)


@pytest.mark.parametrize("field,value", [("pcg_fused", 3), ("pcg_fused", -1), ("pcg_iters_per_launch", 0),
                                         ("pcg_iters_per_launch", 17), ("rollout_pcg_window", 3),
                                         ("rollout_pcg_window", 1), ("newton_max", 0)])
def test_create_rejects_bad_scheduling_params(L, field, value):
    """ipc_create_envs checks its parameters before it touches the device:
    out-of-range scheduling parameters give IPC_EINVAL (a placeholder
    workspace address suffices, nothing is written)."""
    sc = scenes.config0()
    prm = ipc.params_from(sc.params)
    setattr(prm, field, value)
    arr, keep = ipc._descs([sc.scene])
    ctx = C.c_void_p()
    fake = C.c_void_p(1 << 20)   # 256-byte aligned, never dereferenced on this path
    st = L.ipc_create_envs(arr, 1, C.byref(prm), fake, C.c_size_t(1 << 20), None, C.byref(ctx))
    assert st == ipc.IPC_EINVAL
    assert not ctx.value


def test_workspace_bytes_scales_with_envs(L):
    sc = scenes.config0()
    one = ipc.workspace_bytes([sc.scene], sc.params)
    four = ipc.workspace_bytes([sc.scene] * 4, sc.params)
    assert one > 0 and four > 3 * one


def test_uneven_batch_workspace(L):
    scs = [scenes.config2(e).scene for e in range(3)]
    assert ipc.workspace_bytes(scs, scenes.SolverParams()) > 0


def test_rejects_inverted_rest_tet(L):
    sc = scenes.config0().scene
    bad = scenes.Scene(**{**sc.__dict__})
    bad.gel_tets = sc.gel_tets.copy()
    bad.gel_tets[0] = bad.gel_tets[0][[0, 1, 3, 2]]
    with pytest.raises(ipc.IpcError) as ei:
        ipc.workspace_bytes([bad], scenes.SolverParams())
    assert ei.value.status == ipc.IPC_EINVAL


def test_rejects_open_body_surface(L):
    sc = scenes.config0().scene
    b = sc.bodies[0]
    bad_body = scenes.Body(rest_x=b.rest_x, tris=b.tris[:-1], rho=b.rho, kappa_s=b.kappa_s, driven=True)
    bad_body.tris = b.tris[:-2]
    bad = scenes.Scene(**{**sc.__dict__})
    bad.bodies = [bad_body]
    # an open surface has a volume that is not the solid's; removing two
    # triangles of a box leaves a positive but wrong volume, so use a flipped
    # surface instead, which has negative volume
    bad.bodies = [scenes.Body(rest_x=b.rest_x, tris=b.tris[:, [0, 2, 1]], rho=b.rho, kappa_s=b.kappa_s,
                              driven=True)]
    with pytest.raises(ipc.IpcError):
        ipc.workspace_bytes([bad], scenes.SolverParams())


def test_rejects_out_of_range_index(L):
    sc = scenes.config0().scene
    bad = scenes.Scene(**{**sc.__dict__})
    bad.gel_tets = sc.gel_tets.copy()
    bad.gel_tets[3, 2] = sc.n_verts + 5
    with pytest.raises(ipc.IpcError):
        ipc.workspace_bytes([bad], scenes.SolverParams())


def test_read_back_rejects_output_arrays_of_the_wrong_layout():
    # the library writes 3 doubles per row up to out.shape[0] rows: anything
    # but a C-contiguous float64 (rows, 3) array is refused before the call
    ok = np.zeros((5, 3))
    ipc.Envs._check_out_rows(ok, "t")
    for bad in (np.zeros((5, 3), np.float32), np.zeros(15), np.zeros((5, 4)), np.zeros((3, 5)).T,
                np.zeros((10, 3))[::2]):
        with pytest.raises(ValueError):
            ipc.Envs._check_out_rows(bad, "t")
