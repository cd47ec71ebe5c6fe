"""The kernels' per-operation adjoint rules (tests/adjoint_rules.cpp), their whole
adjoint step (tests/step_adjoint.cpp), the world-aligned step and its adjoint
(tests/wstep_check.cpp: its forward against the link-frame step, its adjoint
against central differences) and their constrained step with contacts
and limits (tests/contact_adjoint.cpp), built for the host in FP64 from
csrc/spatial.cuh, csrc/aba_step.cuh and csrc/contact.cuh, against central
differences; the pipelined kernels' compact tapes and split forward step against
the one-warp formulation (tests/layout_parity.cpp); the dot-product test of the
forward-mode JVP against the adjoint (tests/jvp_dot.cpp); and the
closed forms of a joint about e_z against the general formulas.  These pins do
not involve the oracle."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

RULES = {"crossm_adj", "crossf_adj", "apply_adj", "applyT_adj", "congruence_adj", "rbi_dmass",
         "rbi_dmass_bilinear", "rot_axis_T_dq", "rotz_T_dq", "crossm_z_adj", "quat_R_adj", "spd_solve_adj"}
IDENTITIES = {"rotz_T_mm_equals_general", "rotz_T_dq_equals_general", "crossm_z_col_z_equal_general"}


def test_adjoint_rules_match_central_differences(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "adjoint_rules"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "adjoint_rules.cpp")],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    assert set(res) == RULES | IDENTITIES
    for name in RULES:
        assert res[name] < 1e-7, (name, res[name])          # O(h^2) central differences, h = 1e-6
    for name in IDENTITIES:
        assert res[name] < 1e-14, (name, res[name])


def test_whole_adjoint_step_matches_central_differences(tmp_path):
    """step_adjoint of the kernels (host build, FP64) against central differences of
    their own forward step with respect to q, qd, tau and the link masses: a
    floating base with a branched revolute tree, a damped chain, a revolute tree
    with explicit Euler and a lone free body."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "step_adjoint"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "step_adjoint.cpp")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    assert set(res) == {"floating_base_tree", "damped_chain", "revolute_tree_explicit", "free_body_explicit"}
    for name, err in res.items():
        assert err < 1e-7, (name, err)       # a 0.1 % error in one gradient block shows as ~1e-5


def test_constrained_step_adjoint_matches_central_differences(tmp_path):
    """The contact + joint-limit step (sphere-ground MLCP by projected Gauss-Seidel)
    and its adjoint, in the order the adjoint kernels run it, against central
    differences: a floating base on four penetrating feet with two knees past a
    limit (14 active rows), both integrators."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "contact_adjoint"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "contact_adjoint.cpp")],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {line.split()[0]: (float(line.split()[1]), int(line.split()[2])) for line in out.strip().splitlines()}
    assert set(res) == {"contacts_limits_semi_implicit", "contacts_limits_explicit"}
    for name, (err, rows) in res.items():
        assert rows == 14, (name, rows)          # 4 contacts x 3 rows + 2 limit rows active in every trial
        assert err < 1e-6, (name, err)           # a 0.1 % error in the constraint path shows as ~1e-3


def test_pipelined_layouts_and_split_forward_are_bit_identical(tmp_path):
    """What the two-warp kernels compute differently (compact producer/consumer
    tapes; the forward step split into an inertia half and a bias half) equals the
    one-warp formulation bit for bit on chains of 1 to 7 links (host FP64 build with
    the field checks on)."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "layout_parity"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "layout_parity.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 21
    assert all(" adjoint_diff 0 forward_diff 0 " in line for line in lines)


def test_jvp_and_adjoint_are_transposes(tmp_path):
    """Dot-product test: the forward-mode JVP (the step on dual numbers) and
    step_adjoint satisfy <ybar, J xdot> = <J^T ybar, xdot> to round-off on a
    floating-base tree and a damped chain, both integrators."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "jvp_dot"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "jvp_dot.cpp")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    assert len(res) == 4
    for name, err in res.items():
        assert err < 1e-12, (name, err)


def test_world_aligned_step(tmp_path):
    """The world-aligned formulation of the step (host build, FP64): its joint
    accelerations equal the link-frame step's to rounding, and its adjoint matches
    central differences of its own forward step in q, qd, tau and the masses along
    random directions and along each block alone (chains, branched trees, random
    trees, a forest, a star, a caterpillar whose stack of parent values is 8 deep,
    damping, both integrators).  The models are stored in the library's
    depth-first order with a stack exactly as deep as that order says, followed by
    NaN guard entries that must stay untouched; the order's own invariants are
    checked on random trees and forests.  Both loop orders of the adjoint run
    (the plain one and the interleaved one of the FP32 global-tape kernels, two
    links' independent work per loop body) and agree.  A 0.1 % error planted in one
    adjoint term shows as 5e-7 to 6e-5 here."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "wstep_check"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(HERE, "wstep_check.cpp")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    cases = {"chain", "damped_chain", "branched_tree", "tree_explicit", "single_link", "two_roots",
             "random_tree_bf2", "random_tree_bf3", "star", "caterpillar"}
    assert set(res) == {f"{k}_{c}" for k in ("forward", "adjoint", "depth", "guards", "ilp") for c in cases} | {
        "order_invariants"}
    assert res["order_invariants"] == 1
    for c in cases:
        assert res[f"forward_{c}"] < 1e-13, (c, res[f"forward_{c}"])
        assert res[f"adjoint_{c}"] < 1e-7, (c, res[f"adjoint_{c}"])
        assert res[f"guards_{c}"] == 1, c
        assert res[f"ilp_{c}"] < 1e-12, (c, res[f"ilp_{c}"])   # the two loop orders agree
    depth = {"chain": 0, "damped_chain": 0, "single_link": 0, "branched_tree": 2, "star": 1, "two_roots": 1,
             "caterpillar": 8}
    for c, d in depth.items():
        assert res[f"depth_{c}"] == d, (c, res[f"depth_{c}"])
