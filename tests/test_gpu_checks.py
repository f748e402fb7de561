"""The bounds-checked build (libipc_b300_checks.so, -DIPC_CHECKS): on valid
inputs it records no violation and its steps match the release build's.
The checked build runs in a child process (the library is chosen when the
binding loads it); both runs take the same uneven batch through lock-step
steps and a rollout, in FP64 at the parity tolerances, where the two
results agree to the FP64 multi-step bar (1e-6 of the bbox diagonal per
step; the checks change no arithmetic, only the order of atomics can
differ)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, sys.argv[2])
    import scenes
    from paper_2504_12908_b300 import ipc

    scs = [scenes.config2(e, n_steps=12) for e in (0, 1, 2, 5)]
    prm = scenes.SolverParams().parity()
    g = ipc.Envs([sc.scene for sc in scs], prm, stream=torch.cuda.Stream())
    mb = max(g.max_bodies, 1)

    def table(k0, n):
        t = np.zeros((n, len(scs), mb, 12))
        for k in range(n):
            for e, sc in enumerate(scs):
                y = g.rest_y(e)
                y[:, :3] += np.asarray(sc.delta(k0 + k)).reshape(-1, 3)[: y.shape[0]]
                t[k, e, : y.shape[0]] = y
        return t
    status = []
    for k in range(2):
        g.set_targets_all(table(k, 1)[0])
        st, _ = g.step()
        status += list(st)
    st, steps, _ = g.rollout(2, torch.as_tensor(table(2, 2), device="cuda"))
    status += list(st)
    rep = g.check_report()
    x = [g.get_state(e)[0] for e in range(len(scs))]
    y = [g.get_state(e)[2] for e in range(len(scs))]
    np.savez(sys.argv[1], status=np.array(status), steps=steps, built=rep["checks_built"], code=rep["code"],
             index=rep["index"], **{f"x{e}": x[e] for e in range(len(scs))}, **{f"y{e}": y[e] for e in range(len(scs))})
""")


def _run(tmp_path, checks):
    out = str(tmp_path / ("checks.npz" if checks else "release.npz"))
    env = dict(os.environ)
    env["IPC_B300_CHECKS"] = "1" if checks else "0"
    r = subprocess.run([sys.executable, "-c", RUN, out, ROOT], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_checked_build_records_no_violation_and_matches_release(tmp_path):
    from paper_2504_12908_b300.build import build
    build()
    build(checks=True)
    a = _run(tmp_path, checks=False)
    b = _run(tmp_path, checks=True)
    assert int(a["built"]) == 0 and int(b["built"]) == 1
    assert int(a["code"]) == 0 and int(b["code"]) == 0, (int(b["code"]), int(b["index"]))
    assert np.all(a["status"] == 0) and np.all(b["status"] == 0)
    assert np.all(b["steps"] == 2)
    for e in range(4):
        xa, xb = a[f"x{e}"], b[f"x{e}"]
        diag = float(np.linalg.norm(xa.max(0) - xa.min(0)))
        assert np.abs(xa - xb).max() <= 1e-6 * 4 * diag, e
        assert np.abs(a[f"y{e}"][:, :3] - b[f"y{e}"][:, :3]).max() <= 1e-6 * 4 * diag, e
