"""The C-ABI library loads, exports every declared entry point, and its host-side
model validation rejects malformed trees (no GPU needed: validation runs before
any device call)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "abasim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2109_07719_gb300 as p
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(p.lib, n), n


def _desc(model, precision=0, integrator=0, **override):
    import paper_2109_07719_gb300 as p
    arrs = dict(sys_link_offset=np.ascontiguousarray(model.sys_link_offset, np.int32),
                parent=np.ascontiguousarray(model.parent, np.int32),
                joint_type=np.ascontiguousarray(model.joint_type, np.int32),
                axis=np.ascontiguousarray(model.axis, np.float64),
                X_tree=np.ascontiguousarray(model.X_tree, np.float64),
                mass=np.ascontiguousarray(model.mass, np.float64),
                com=np.ascontiguousarray(model.com, np.float64),
                I_com=np.ascontiguousarray(model.I_com, np.float64))
    for k, v in override.items():
        if k in arrs:
            arrs[k] = np.ascontiguousarray(v, arrs[k].dtype)
        elif k in ("damping", "contact", "limits"):
            arrs[k] = np.ascontiguousarray(v, np.float64)
    if "contact" not in override and getattr(model, "contact", None) is not None:
        arrs["contact"] = np.ascontiguousarray(model.contact, np.float64)
    d = p._Desc()
    d.n_systems = override.get("n_systems", len(arrs["sys_link_offset"]) - 1)
    d.precision = precision
    d.integrator = integrator
    d.dt = override.get("dt", model.dt)
    d.friction = override.get("friction", 0.8)
    d.erp = override.get("erp", 0.2)
    d.pgs_iterations = override.get("pgs_iterations", 20)
    d.flags = override.get("flags", 0)
    for i in range(3):
        d.gravity[i] = model.gravity[i]
    for k, v in arrs.items():
        setattr(d, k, v.ctypes.data)
    return d, arrs


def _create(d):
    import paper_2109_07719_gb300 as p
    h = ctypes.c_void_p()
    rc = p.lib.sim_create(ctypes.byref(d), ctypes.byref(h))
    if rc == 0:
        p.lib.sim_destroy(h)
    return rc, p.lib.sim_last_error(None).decode()


def _bad_cases():
    m = wl.config(2, B=2, T=1).model
    q = wl.config(3, B=1, T=1).model
    par = m.parent.copy(); par[3] = 3
    ax = m.axis.copy(); ax[2] *= 1.5
    Xt = m.X_tree.copy(); Xt[1, 0] = 2.0
    ms = m.mass.copy(); ms[4] = -1.0
    jt = m.joint_type.copy(); jt[2] = 1
    jt2 = m.joint_type.copy(); jt2[0] = 7
    ic = m.I_com.copy(); ic[1, 0] = -0.5
    off = m.sys_link_offset.copy(); off[1] = 0
    qc = wl.config(3, B=1, T=1, contacts=True).model
    many = qc.contact.copy(); many[:5, 3] = 0.02                      # five spheres in one system
    nan = qc.contact.copy(); nan[3, 0] = np.nan
    inf2 = np.tile([[-np.inf, np.inf]], (q.n_links_total, 1))
    lim_free = inf2.copy(); lim_free[0] = (-1.0, 1.0)                   # a limit on the floating base
    lim_order = inf2.copy(); lim_order[2] = (0.5, -0.5)
    lim_many = np.tile([[-1.0, 1.0]], (m.n_links_total, 1))
    ch = wl.config(4, B=1, T=1, dof_lo=14, dof_hi=14).model            # 14 limited joints in one system
    lim_14 = np.tile([[-1.0, 1.0]], (ch.n_links_total, 1))
    return [
        (m, dict(parent=par), "parent"),
        (m, dict(axis=ax), "axis"),
        (m, dict(X_tree=Xt), "orthonormal"),
        (m, dict(mass=ms), "mass"),
        (m, dict(joint_type=jt), "free joint"),
        (m, dict(joint_type=jt2), "joint type"),
        (m, dict(I_com=ic), "inertia"),
        (m, dict(sys_link_offset=off), "links"),
        (m, dict(dt=0.0), "dt"),
        (m, dict(n_systems=0), "n_systems"),
        (m, dict(damping=-np.ones(m.n_links_total)), "damping"),
        (q, dict(), None),
        (qc, dict(contact=many), "contact spheres"),
        (qc, dict(contact=nan), "contact sphere"),
        (qc, dict(friction=-0.1), "friction"),
        (qc, dict(erp=1.5), "erp"),
        (qc, dict(pgs_iterations=0), "pgs_iterations"),
        (qc, dict(pgs_iterations=65), "pgs_iterations"),
        (qc, dict(), None),
        (q, dict(limits=lim_free), "revolute joints only"),
        (q, dict(limits=lim_order), "lo < hi"),
        (ch, dict(limits=lim_14), "limited joints"),
        (m, dict(limits=lim_many), None),
    ]


@pytest.mark.parametrize("case", range(23))
def test_model_validation(case):
    model, over, needle = _bad_cases()[case]
    d, _keep = _desc(model, **over)
    rc, msg = _create(d)
    if needle is None:       # a valid model: without a GPU only the device step may fail
        assert rc in (0, -2, -3), (rc, msg)
    else:
        assert rc == -1, (rc, msg)
        assert needle in msg, msg


def test_bad_precision_and_integrator_rejected():
    m = wl.config(2, B=1, T=1).model
    for kw in (dict(precision=5), dict(integrator=3)):
        d, _keep = _desc(m, **kw)
        rc, msg = _create(d)
        assert rc == -1 and ("precision" in msg or "integrator" in msg), msg


def test_null_arguments():
    import paper_2109_07719_gb300 as p
    assert p.lib.sim_ckpt_bytes(None, 10, 1) == 0
    assert p.lib.sim_work_bytes(None, 10) == 0
    assert p.lib.sim_rollout(None, None, None, None, 1, 1, None, None, None, None, None) == -1
    assert p.lib.sim_create(None, None) == -1
    # the launch and precision controls refuse a null handle before touching it
    assert p.lib.sim_set_state_accumulation(None, 1) == -1
    assert p.lib.sim_set_tape_space(None, 4) == -1
    assert p.lib.sim_set_replay(None, 0) == -1
    assert p.lib.sim_set_prefetch(None, 2) == -1


def test_unknown_creation_flags_rejected():
    m = wl.config(4, B=3, T=1).model
    d, _keep = _desc(m, flags=2)
    rc, msg = _create(d)
    assert rc == -1 and "flag" in msg, msg
    d, _keep = _desc(m, flags=1)          # SIM_KEEP_SYSTEM_ORDER: valid
    rc, msg = _create(d)
    assert rc in (0, -2, -3), (rc, msg)
