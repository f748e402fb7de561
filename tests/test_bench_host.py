"""Host-side checks of the bench's measurement arithmetic (no GPU): the
algorithmic bytes per kernel class, the roofline line of the dominant class
and the source hashes that guard the stored ncu counts."""
import os
import types

import pytest

import bench


class _FakeEnvs:
    """The few fields of ipc.Envs that the bytes model reads: one env of the
    bench's gel 40x40x6 + icosphere L2 in the mixed mode."""

    def __init__(self, precision=1):
        body = types.SimpleNamespace(rest_x=[None] * 162)
        self.scenes = [types.SimpleNamespace(bodies=[body])]
        self.sizes = [(9600, 1, 2800)]
        self.params = types.SimpleNamespace(precision=precision)

    def system_sizes(self, env):
        return {"real_blocks": 112508, "stored_blocks": 120000, "rows": 9604, "tets": 38025}


def _tot(**kw):
    t = {"pcg_iters": 1000, "newton_env_iters": 20, "ls_trials": 30, "env_steps": 4, "pair_evals": 5000,
         "swept_pairs": 4000, "act_pair_iters": 22000}
    t.update(kw)
    return t


def test_kernel_bytes_per_env_iteration():
    """The SELL mat-vec moves blocks x (9 values + a column) and 4 FP32 rows
    per row per env-iteration (4.96 MB for this env: the figure the design
    notes and the ncu summaries use); the update 156 B per row; the fused
    class is the sum of the mat-vec, contact and update classes."""
    kb = bench.kernel_bytes(_FakeEnvs(), _tot(pcg_iters=1))
    assert kb["pcg_matvec"] == 112508 * (9 * 4 + 4) + 9604 * 4 * 12
    assert abs(kb["pcg_matvec"] / 1e6 - 4.96) < 0.01
    assert kb["pcg_update"] == 9604 * (96 + 24 + 24 + 12)
    assert kb["pcg_iter"] == kb["pcg_matvec"] + kb["pair_matvec"] + kb["pcg_update"]
    # FP64 mode: 8-byte values and 24-byte rows
    kb64 = bench.kernel_bytes(_FakeEnvs(precision=0), _tot(pcg_iters=1))
    assert kb64["pcg_matvec"] == 112508 * (9 * 8 + 4) + 9604 * 4 * 24


def test_roofline_line_of_the_dominant_class():
    """achieved = algorithmic bytes / the class's profiled time, frac =
    achieved / the measured HBM peak; the traffic figure scales the stored
    ncu bytes by the env-iterations per launch."""
    tot = _tot(pcg_iters=33_835)                       # 338.35 env-iterations per launch, 100 launches
    prof = {"pcg_iter": (100, 68.3), "tet_elastic": (10, 31.0), "ls_energy": (50, 12.0)}
    roof, kernels = bench.roofline_of(_FakeEnvs(), prof, tot)
    kb = bench.kernel_bytes(_FakeEnvs(), tot)
    peak, kind = bench.measured_peaks()
    assert roof["kernel"] == roof["dominant_kernel"] == "pcg_iter"
    assert roof["achieved"] == pytest.approx(kb["pcg_iter"] / 68.3e-3 / 1e9, rel=1e-3)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak, rel=1e-3)
    assert roof["env_iters_per_launch"] == pytest.approx(338.35)
    if bench.pcg_iter_traffic_per_launch(1.0) is not None:
        per = bench.PCG_ITER_TRAFFIC["bytes"] / bench.PCG_ITER_TRAFFIC["env_iters"]
        assert roof["traffic"] == pytest.approx(per * 338.35, rel=1e-9)
    assert sum(k["share"] for k in kernels.values()) == pytest.approx(1.0, abs=1e-3)


def test_source_hash_covers_the_measured_functions():
    """Each hashed part names a function that exists in the sources, and its
    extracted text runs from the signature to the function's closing brace;
    any edit of that text changes the hash (the stored counts are then not
    reported)."""
    csrc = os.path.join(bench.ROOT, "paper_2504_12908_b300", "csrc")
    parts = list(bench.PCG_ITER_PARTS) + list(bench.MATVEC_PARTS)
    for k in bench.ALU_PARTS.values():
        parts += list(k)
    for f, sig in parts:
        src = open(os.path.join(csrc, f)).read()
        if sig is None:
            continue
        text = bench._function_text(src, sig)
        assert text.startswith(sig) and text.endswith("\n}\n") and text.count("{") == text.count("}"), (f, sig)
    h = bench._kernel_source_hash(bench.PCG_ITER_PARTS)
    edited = [(f, s) for f, s in bench.PCG_ITER_PARTS]
    edited[0] = ("kernels_pcg.cu", None)               # another text for the first part
    assert bench._kernel_source_hash(edited) != h
