"""Plain FP64 CPU oracle for one implicit ABD-IPC time step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the two
meet only through the seeded scene generators in ``scenes``.

What it computes (Taccel, arXiv 2504.12908):

* the incremental potential of Sec. 3.2 / App. A.2 (backward Euler,
  ``x^{n+1} = argmin E_IP``) with lumped mass and gravity,
* the neo-Hookean elastic energy ``Phi = int Psi`` (Sec. 3.1, App. A.1),
* the IPC log barrier ``b(d)`` of Eq. (ipc_energy) summed with area weights
  over point-triangle and edge-edge pairs (Eq. fullspace_ipc, App. A.3),
* the affine-body (ABD) reduced coordinates ``y`` with ``M^y = J^T M J`` and
  a stiff orthogonality term (Sec. 3.3, Eq. unified_ipc),
* the kinematic constraints ``S x = s`` of Sec. 3.4 (Eq. unified_ipc_AL),
  handled with an augmented Lagrangian,
* minimised by projected Newton: per-element Hessians made PSD with
  ``numpy.linalg.eigh`` (negative eigenvalues clamped to zero; optionally
  replaced by their absolute values once a step's Newton iterations reach
  ``newton_abs_after``), a sparse direct solve instead of PCG, brute-force
  all-pairs contact candidates, additive CCD and backtracking line search.

Readings of the paper where it is silent or garbled are listed in the design
notes of the repository and restated in the docstrings here.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, finite differences, brute force or library routines,
except the whole contact step, which has no printed worked example in the
paper and is pinned only through invariants (min distance > 0, det F > 0,
monotone energy, CCD conservativeness against exact cubic roots).
"""
from .rest import GelRest, BodyRest, SurfaceData, gel_rest, body_rest, surface_data
from .step import OracleEnv, StepStats

__all__ = ["GelRest", "BodyRest", "SurfaceData", "gel_rest", "body_rest",
           "surface_data", "OracleEnv", "StepStats"]
