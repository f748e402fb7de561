"""Tactile outputs on the GPU (Sec. 4.2) against the oracle's brute-force
definition, on the same deformed positions: depth maps element by element,
hit masks exactly, normals where a pixel's triangle is unique (else one of
the triangles that contain the pixel), markers and flows."""
import numpy as np
import pytest

import scenes
from oracle import tactile as tc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12908_b300 import ipc  # noqa: E402
from paper_2504_12908_b300.build import build  # noqa: E402

build()

H = W = 40


def _sensor(env, pad, origin, eu, ev, n, pitch):
    return {"env": env, "pad": pad, "origin": origin, "axis_u": eu, "axis_v": ev, "normal": n, "pitch": pitch}


def _scenarios():
    r3 = 0.01 + 2e-5
    return [
        (scenes.config0(), [(0, (-0.01, -0.01, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1), 0.5e-3)]),
        (scenes.config2(1), [(0, (-0.01, -0.01, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1), 0.5e-3)]),
        (scenes.small_contact_scene(body="sphere", level=2, depth=3e-4, n_steps=4),
         [(0, (-0.005, -0.005, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1), 0.25e-3)]),
        (scenes.config3(0, n=5, nz=3, level=1, gap=2e-5),
         [(0, (-r3, -0.01, -0.01), (0, 1, 0), (0, 0, 1), (1, 0, 0), 0.5e-3),
          (1, (r3, -0.01, -0.01), (0, 1, 0), (0, 0, 1), (-1, 0, 0), 0.5e-3)]),
    ]


def _advance(genv, scs, n_steps):
    for k in range(n_steps):
        for e, sc in enumerate(scs):
            t = genv.rest_y(e)
            t[:, :3] += sc.delta(k)[:, :3]
            genv.set_targets(e, t)
        st, _ = genv.step()
        assert np.all(st == 0)


def _containing_normals(x, T, sd, r, c):
    o, eu, ev, n = (np.asarray(sd[k], float) for k in ("origin", "axis_u", "axis_v", "normal"))
    pu, pv = (c + 0.5) * sd["pitch"], (r + 0.5) * sd["pitch"]
    out = []
    for t in T:
        P = x[t]
        U, V = (P - o) @ eu, (P - o) @ ev
        det = (U[1] - U[0]) * (V[2] - V[0]) - (U[2] - U[0]) * (V[1] - V[0])
        if det == 0.0:
            continue
        b1 = ((pu - U[0]) * (V[2] - V[0]) - (U[2] - U[0]) * (pv - V[0])) / det
        b2 = ((U[1] - U[0]) * (pv - V[0]) - (pu - U[0]) * (V[1] - V[0])) / det
        if min(1 - b1 - b2, b1, b2) >= -1e-9:
            nn = np.cross(P[1] - P[0], P[2] - P[0])
            out.append(nn / np.linalg.norm(nn))
    return out


def test_depth_normal_maps_match_the_oracle_on_deformed_states():
    cases = _scenarios()
    scs = [sc for sc, _ in cases]
    prm = scenes.SolverParams()
    genv = ipc.Envs([sc.scene for sc in scs], prm)
    _advance(genv, scs, 4)
    sensors = [_sensor(e, pad, o, eu, ev, n, p) for e, (_, lst) in enumerate(cases) for (pad, o, eu, ev, n, p) in lst]
    prep = genv.prepare_sensors(sensors, H, W)
    depth, normal, hit = genv.tactile_maps(prep)
    torch.cuda.synchronize()
    depth, normal, hit = depth.cpu().numpy(), normal.cpu().numpy(), hit.cpu().numpy().astype(bool)
    pressed = 0
    for i, sd in enumerate(sensors):
        s = scs[sd["env"]].scene
        x = genv.get_state(sd["env"])[0]
        coated = ~s.pinned & (s.attach < 0)
        T = tc.front_triangles(s.gel_tets, s.gel_x, coated, s.gel_obj, sd["pad"], np.asarray(sd["normal"], float))
        assert len(T) == len(genv.sensor_triangles(sd))
        d0, n0, h0 = tc.depth_normal_map(x, T, sd["origin"], sd["axis_u"], sd["axis_v"], sd["normal"], sd["pitch"],
                                         H, W)
        assert np.array_equal(hit[i], h0), i
        assert np.allclose(depth[i], d0, rtol=0, atol=1e-15), (i, np.abs(depth[i] - d0).max())
        bad = np.argwhere(np.abs(normal[i] - n0).max(axis=2) > 1e-12)
        for r, c in bad:
            cands = _containing_normals(x, T, sd, r, c)
            assert any(np.abs(normal[i][r, c] - nn).max() <= 1e-12 for nn in cands), (i, r, c)
        assert len(bad) < 0.05 * H * W
        pressed += int((d0 > 1e-7).sum())
    assert pressed > 0                     # some sensor saw an indentation
    genv.close()


def test_markers_and_flows_match_the_oracle():
    cases = _scenarios()[:3]
    scs = [sc for sc, _ in cases]
    genv = ipc.Envs([sc.scene for sc in scs], scenes.SolverParams())
    rng = np.random.default_rng(11)
    preps, refs = [], []
    for e, sc in enumerate(scs):
        s = sc.scene
        coated = ~s.pinned & (s.attach < 0)
        T = tc.front_triangles(s.gel_tets, s.gel_x, coated, s.gel_obj, 0, np.array([0.0, 0.0, 1.0]))
        k = rng.integers(0, len(T), 64)
        bary = rng.dirichlet([1, 1, 1], 64)
        preps.append(genv.prepare_markers(e, T[k], bary))
        refs.append((T[k], bary, tc.marker_positions(s.gel_x, T[k], bary)))
    _advance(genv, scs, 4)
    moved = 0.0
    for e in range(len(scs)):
        pos, flow = genv.markers(preps[e])
        torch.cuda.synchronize()
        x = genv.get_state(e)[0]
        tri, bary, rest = refs[e]
        p = tc.marker_positions(x, tri, bary)
        assert np.allclose(pos.cpu().numpy(), p, rtol=0, atol=1e-15)
        assert np.allclose(flow.cpu().numpy(), p - rest, rtol=0, atol=1e-15)
        moved = max(moved, float(np.abs(p - rest).max()))
    assert moved > 1e-7
    genv.close()
