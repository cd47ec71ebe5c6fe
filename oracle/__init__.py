"""CPU FP64 oracle for batched articulated-body rollouts and their adjoints.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path; both read their inputs from the separate ``workloads`` module.

What it computes (Qiao et al., "Efficient Differentiable Simulation of
Articulated Bodies", ICML 2021):

* forward dynamics qdd = FD(q, qd, tau) two independent ways: the plain
  definition qdd = M(q)^-1 (tau - C(q, qd)) with M from the composite-rigid-body
  algorithm and C from the recursive Newton-Euler algorithm, and the direct
  Articulated Body Algorithm (Sec. 2 "Articulated body dynamics"; the three
  tree passes of Sec. 3.1 and Fig. 1), all with dense 6x6 spatial matrices;
* semi-implicit (and plain explicit) Euler time integration (Sec. 3.1);
* the gradient of an objective through the rollout by the adjoint recurrence
  R^k = dPhi/dx^k + (df/dx^k)^T R^{k+1} (Eq. 3-4) with only the per-step
  initial state kept and one step recomputed during backprop (Sec. 3.2,
  Eq. 7); the per-step vector-Jacobian product is reverse-mode AD of the
  plain step (a library primitive), not a hand-written rule.

Parity pins live in ``tests/test_oracle_*.py``.
"""
from .spatial import (crossm, crossf, xform, spatial_inertia, quat_to_E, quat_mul,  # noqa: F401
                      skew)
from .dynamics import OracleModel, crba, rnea, aba, fd_crba, jcalc, link_world_poses  # noqa: F401
from .rollout import step, rollout, rollout_backward, energy, spatial_momentum  # noqa: F401
