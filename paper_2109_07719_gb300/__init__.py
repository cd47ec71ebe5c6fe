"""Batched differentiable articulated-body simulation on one GB300 (Python binding).

A thin ctypes layer over the C ABI in ``include/abasim.h``: it marshals torch
device tensors into pointers and streams; every step of the computation runs in
the CUDA kernels of ``libabasim.so``.  There is no CPU fallback: importing the
binding raises if the library cannot be loaded.

    sim = Simulator(model, precision="fp32")          # sim_create
    qT, qdT = Rollout.apply(sim, q0, qd0, tau, mass)  # sim_rollout / sim_backward_rollout

Paper: Qiao et al., "Efficient Differentiable Simulation of Articulated Bodies"
(ICML 2021): ABA forward dynamics (Sec. 2), the adjoint of the simulation step
(Sec. 3.1) and per-step checkpointing with recompute (Sec. 3.2).
"""
from __future__ import annotations

import ctypes
import hashlib
import os

import numpy as np
import torch

from . import build as _build

__all__ = ["Simulator", "Rollout", "RolloutTrajectory", "lib", "SimError", "PRECISIONS"]

SIM_OK = 0
SIM_ENONFINITE = -4
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_d64": 2}
INTEGRATORS = {"semi": 0, "explicit": 1}


class SimError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [("n_systems", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("sys_link_offset", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("joint_type", ctypes.c_void_p), ("axis", ctypes.c_void_p),
                ("X_tree", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("com", ctypes.c_void_p),
                ("I_com", ctypes.c_void_p), ("damping", ctypes.c_void_p),
                ("contact", ctypes.c_void_p), ("friction", ctypes.c_double), ("erp", ctypes.c_double),
                ("pgs_iterations", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("limits", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGS = {
    "sim_create": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]),
    "sim_destroy": (None, [_P]),
    "sim_dims": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "sim_ckpt_bytes": (ctypes.c_size_t, [_P, ctypes.c_int64, ctypes.c_int32]),
    "sim_work_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "sim_set_masses": (ctypes.c_int, [_P, _P, _P]),
    "sim_last_storage": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "sim_step_batch": (ctypes.c_int, [_P] * 7),
    "sim_step_batch_static": (ctypes.c_int, [_P] * 7),
    "sim_rollout": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "sim_backward_rollout": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P,
                                            _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "sim_status": (ctypes.c_int, [_P, _P]),
    "sim_clear_status": (ctypes.c_int, [_P, _P]),
    "sim_set_launch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "sim_slot_order": (ctypes.c_int, [_P, _P]),
    "sim_set_tape_space": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sim_set_replay": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sim_set_prefetch": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sim_set_state_accumulation": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sim_jvp_work_bytes": (ctypes.c_size_t, [_P]),
    "sim_step_jvp": (ctypes.c_int, [_P] * 11 + [_P, ctypes.c_size_t, _P]),
    "sim_last_error": (ctypes.c_char_p, [_P]),
}


def _load():
    path = _build.LIB
    if _build.stale():
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Simulator:
    """One batch of articulated systems on the current CUDA device (sim_create).

    ``model`` is any object with the model-description arrays (sys_link_offset,
    parent, joint_type, axis, X_tree, mass, com, I_com, dt, gravity) laid out as
    documented in ``include/abasim.h``.
    """

    def __init__(self, model, precision: str = "fp64", integrator: str = "semi", keep_order: bool = False):
        if not torch.cuda.is_available():
            raise SimError("no CUDA device: the simulator runs only on the GPU")
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        keep = dict(
            sys_link_offset=np.ascontiguousarray(model.sys_link_offset, np.int32),
            parent=np.ascontiguousarray(model.parent, np.int32),
            joint_type=np.ascontiguousarray(model.joint_type, np.int32),
            axis=np.ascontiguousarray(model.axis, np.float64),
            X_tree=np.ascontiguousarray(model.X_tree, np.float64),
            mass=np.ascontiguousarray(model.mass, np.float64),
            com=np.ascontiguousarray(model.com, np.float64),
            I_com=np.ascontiguousarray(model.I_com, np.float64))
        if getattr(model, "damping", None) is not None:
            keep["damping"] = np.ascontiguousarray(model.damping, np.float64)
        if getattr(model, "contact", None) is not None:
            keep["contact"] = np.ascontiguousarray(model.contact, np.float64)
        if getattr(model, "limits", None) is not None:
            keep["limits"] = np.ascontiguousarray(model.limits, np.float64)
        d = _Desc()
        d.friction = float(getattr(model, "friction", 0.8))
        d.erp = float(getattr(model, "erp", 0.2))
        d.pgs_iterations = int(getattr(model, "pgs_iterations", 20))
        d.n_systems = len(keep["sys_link_offset"]) - 1
        d.precision = PRECISIONS[precision]
        d.integrator = INTEGRATORS[integrator]
        d.flags = 1 if keep_order else 0          # SIM_KEEP_SYSTEM_ORDER: no sort by link count
        d.dt = float(model.dt)
        for i in range(3):
            d.gravity[i] = float(model.gravity[i])
        for k, v in keep.items():
            setattr(d, k, v.ctypes.data)
        h = ctypes.c_void_p()
        rc = lib.sim_create(ctypes.byref(d), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(f"sim_create failed ({rc}): {lib.sim_last_error(None).decode()}")
        self._h = h
        dims = [ctypes.c_int32() for _ in range(4)]
        lib.sim_dims(h, *[ctypes.byref(x) for x in dims])
        self.B, self.nq_max, self.nv_max, self.n_links = [x.value for x in dims]
        self.mass0 = torch.as_tensor(keep["mass"], dtype=self.dtype, device=self.device)
        self.launch = (32, False)
        hist = np.bincount(np.diff(keep["sys_link_offset"])).astype(np.int64)
        self.signature = (self.B, self.nq_max, self.nv_max, self.n_links, precision,
                          hashlib.sha1(hist.tobytes()).hexdigest()[:16])

    # ------------------------------------------------------------ plumbing
    def _check(self, rc, what):
        if rc != SIM_OK:
            raise SimError(f"{what} failed ({rc}): {lib.sim_last_error(self._h).decode()}")

    def _arg(self, t, shape, name):
        if t is None:
            return None
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise SimError(f"{name}: need a contiguous {self.dtype} tensor on {self.device}")
        if tuple(t.shape) != tuple(shape):
            raise SimError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
        return t

    def empty(self, *shape):
        return torch.empty(shape, dtype=self.dtype, device=self.device)

    def close(self):
        if getattr(self, "_h", None):
            lib.sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ calls
    @property
    def nx(self):
        return self.nq_max + self.nv_max

    def ckpt_bytes(self, T, k=1):
        return lib.sim_ckpt_bytes(self._h, T, k)

    def work_bytes(self, k):
        return lib.sim_work_bytes(self._h, k)

    def set_launch(self, threads: int = 0, persistent: bool = False):
        """Threads per block (one work unit each) and grid vs persistent scheduling."""
        self._check(lib.sim_set_launch(self._h, int(threads), 1 if persistent else 0), "sim_set_launch")
        self.launch = (int(threads) or 32, bool(persistent))

    def set_tape_space(self, space: str = "auto"):
        """'auto' (the world-aligned kernels for revolute models without contacts
        or limits; otherwise the pipelined kernels or shared memory when they fit),
        'global', 'shared' (one warp per tile, tape on chip), 'pipelined' (two warps
        per tile), 'one_warp' (as 'auto' without the pipelined and world-aligned
        kernels), 'aligned' (the world-aligned kernels) or 'aligned_pipelined' (the
        world-aligned kernels with the two-warp pipelined adjoint)."""
        code = {"auto": 0, "global": 1, "shared": 2, "pipelined": 3, "one_warp": 4, "aligned": 5,
                "aligned_pipelined": 6}[space]
        self._check(lib.sim_set_tape_space(self._h, code), "sim_set_tape_space")

    STORAGE = ("global", "hybrid", "shared", "pipelined", "aligned_shared", "aligned_global",
               "aligned_pipelined_shared", "aligned_pipelined_global")

    def last_storage(self):
        """(rollout, backward) storage modes of the last launches: 'global', 'hybrid',
        'shared', 'pipelined', or the world-aligned kernels' 'aligned_shared' /
        'aligned_global'."""
        f, b = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib.sim_last_storage(self._h, ctypes.byref(f), ctypes.byref(b)), "sim_last_storage")
        return self.STORAGE[f.value], self.STORAGE[b.value]

    def set_prefetch(self, links_ahead: int = 2):
        """How many links ahead the world-aligned global-tape passes prefetch (0: off)."""
        self._check(lib.sim_set_prefetch(self._h, int(links_ahead)), "sim_set_prefetch")

    def set_replay(self, mode: str = "segment"):
        """k > 1 state rebuild: 'segment' (replay once) or 'quadratic' (from the checkpoint)."""
        code = {"segment": 0, "quadratic": 1}[mode]
        self._check(lib.sim_set_replay(self._h, code), "sim_set_replay")

    def set_state_accumulation(self, precision: str = "fp32"):
        """Running-state precision of rollouts in the 'fp32_d64' mode: 'fp64' sums q
        and qd in FP64 between steps (stored as FP32), 'fp32' (default) does not."""
        code = {"fp32": 0, "fp64": 1}[precision]
        self._check(lib.sim_set_state_accumulation(self._h, code), "sim_set_state_accumulation")

    def slot_order(self):
        """System index run by each slot (thread), longest systems first."""
        out = np.zeros(self.B, np.int32)
        self._check(lib.sim_slot_order(self._h, out.ctypes.data), "sim_slot_order")
        return out

    def autotune(self, q0, qd0, **kw):
        """Pick the launch shape by timing short rollouts (see autotune.py)."""
        from .autotune import autotune
        return autotune(self, q0, qd0, **kw)

    def set_masses(self, mass):
        self._arg(mass, (self.n_links,), "mass")
        self._check(lib.sim_set_masses(self._h, _ptr(mass), _stream()), "sim_set_masses")

    def step(self, q, qd, tau, q_out=None, qd_out=None):
        B = self.B
        self._arg(q, (self.nq_max, B), "q")
        self._arg(qd, (self.nv_max, B), "qd")
        self._arg(tau, (self.nv_max, B), "tau")
        q_out = self.empty(self.nq_max, B) if q_out is None else q_out
        qd_out = self.empty(self.nv_max, B) if qd_out is None else qd_out
        self._check(lib.sim_step_batch(self._h, _ptr(q), _ptr(qd), _ptr(tau), _ptr(q_out),
                                       _ptr(qd_out), _stream()), "sim_step_batch")
        return q_out, qd_out

    def step_static(self, q, qd, tau, q_out=None, qd_out=None):
        """One step through sim_step_batch_static: no allocation by the library;
        its scratch is a fixed-size static device array (SIM_STATIC_SCRATCH_BYTES)."""
        B = self.B
        self._arg(q, (self.nq_max, B), "q")
        self._arg(qd, (self.nv_max, B), "qd")
        self._arg(tau, (self.nv_max, B), "tau")
        q_out = self.empty(self.nq_max, B) if q_out is None else q_out
        qd_out = self.empty(self.nv_max, B) if qd_out is None else qd_out
        self._check(lib.sim_step_batch_static(self._h, _ptr(q), _ptr(qd), _ptr(tau), _ptr(q_out),
                                              _ptr(qd_out), _stream()), "sim_step_batch_static")
        return q_out, qd_out

    def jvp(self, q, qd, tau, dq=None, dqd=None, dtau=None, work=None):
        """One step and its forward-mode derivative (sim_step_jvp): returns
        (q', qd', dq', dqd') with (dq', dqd') = J_x (dq, dqd) + J_tau dtau."""
        B = self.B
        self._arg(q, (self.nq_max, B), "q")
        self._arg(qd, (self.nv_max, B), "qd")
        self._arg(tau, (self.nv_max, B), "tau")
        self._arg(dq, (self.nq_max, B), "dq")
        self._arg(dqd, (self.nv_max, B), "dqd")
        self._arg(dtau, (self.nv_max, B), "dtau")
        outs = [self.empty(self.nq_max, B), self.empty(self.nv_max, B), self.empty(self.nq_max, B),
                self.empty(self.nv_max, B)]
        if work is None:
            work = torch.empty(lib.sim_jvp_work_bytes(self._h), dtype=torch.uint8, device=self.device)
        have = work.numel() * work.element_size()
        self._check(lib.sim_step_jvp(self._h, _ptr(q), _ptr(qd), _ptr(tau), _ptr(dq), _ptr(dqd),
                                     _ptr(dtau), *[_ptr(o) for o in outs], _ptr(work), have, _stream()),
                    "sim_step_jvp")
        return tuple(outs)

    def rollout(self, q0, qd0, tau, k=1, ckpt=True, traj=False, out=None):
        """Returns (qT, qdT, ckpt or None, traj or None)."""
        B, T = self.B, int(tau.shape[0])
        self._arg(q0, (self.nq_max, B), "q0")
        self._arg(qd0, (self.nv_max, B), "qd0")
        self._arg(tau, (T, self.nv_max, B), "tau")
        nck = (T + k - 1) // k
        if out is None:
            qT, qdT = self.empty(self.nq_max, B), self.empty(self.nv_max, B)
            ck = self.empty(nck, self.nx, B) if ckpt is True else ckpt
            tr = self.empty(T + 1, self.nx, B) if traj is True else (traj if traj is not False else None)
        else:
            qT, qdT, ck, tr = out
        if ck is False:
            ck = None
        self._check(lib.sim_rollout(self._h, _ptr(q0), _ptr(qd0), _ptr(tau), T, k, _ptr(ck),
                                    _ptr(qT), _ptr(qdT), _ptr(tr), _stream()), "sim_rollout")
        return qT, qdT, ck, tr

    def backward(self, ckpt, tau, gqT, gqdT, k=1, g_traj=None, mass_grad=True, work=None, out=None):
        """Returns (gq0, gqd0, gtau, gmass or None)."""
        B, T = self.B, int(tau.shape[0])
        self._arg(ckpt, ((T + k - 1) // k, self.nx, B), "ckpt")
        self._arg(gqT, (self.nq_max, B), "gqT")
        self._arg(gqdT, (self.nv_max, B), "gqdT")
        self._arg(g_traj, (T + 1, self.nx, B), "g_traj")
        if out is None:
            gq0, gqd0 = self.empty(self.nq_max, B), self.empty(self.nv_max, B)
            gtau = self.empty(T, self.nv_max, B)
            gm = self.empty(self.n_links) if mass_grad else None
        else:
            gq0, gqd0, gtau, gm = out
        wb = self.work_bytes(k)
        if wb and work is None:
            work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        have = 0 if work is None else work.numel() * work.element_size()
        self._check(lib.sim_backward_rollout(
            self._h, _ptr(ckpt), _ptr(tau), T, k, _ptr(gqT), _ptr(gqdT), _ptr(g_traj), _ptr(gq0),
            _ptr(gqd0), _ptr(gtau), _ptr(gm), _ptr(work), have, _stream()), "sim_backward_rollout")
        return gq0, gqd0, gtau, gm

    def status(self):
        flags = np.zeros(self.B, np.int32)
        rc = lib.sim_status(self._h, flags.ctypes.data)
        if rc not in (SIM_OK, SIM_ENONFINITE):
            self._check(rc, "sim_status")
        return flags

    def clear_status(self):
        self._check(lib.sim_clear_status(self._h, _stream()), "sim_clear_status")


class Rollout(torch.autograd.Function):
    """(q0, qd0, tau, mass) -> (qT, qdT) with gradients w.r.t. all four inputs.

    The forward keeps only the states x^0, x^k, ... (Sec. 3.2); the backward
    recomputes every step from them and runs the hand-derived adjoint
    (Sec. 3.1).  ``mass`` [n_links] (or None for the model's masses) is loaded
    with sim_set_masses before the rollout.
    """

    @staticmethod
    def forward(ctx, sim: Simulator, q0, qd0, tau, mass=None, k: int = 1):
        q0, qd0, tau = q0.contiguous(), qd0.contiguous(), tau.contiguous()
        if mass is not None:
            sim.set_masses(mass.detach().contiguous())
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k, ckpt=True)
        ctx.sim, ctx.k, ctx.has_mass = sim, k, mass is not None
        ctx.save_for_backward(ck, tau, mass.detach() if mass is not None else None)
        return qT, qdT

    @staticmethod
    def backward(ctx, gqT, gqdT):
        ck, tau, mass = ctx.saved_tensors
        sim = ctx.sim
        if mass is not None:
            sim.set_masses(mass.contiguous())
        gqT = torch.zeros(sim.nq_max, sim.B, dtype=sim.dtype, device=sim.device) if gqT is None else gqT.contiguous()
        gqdT = torch.zeros(sim.nv_max, sim.B, dtype=sim.dtype, device=sim.device) if gqdT is None else gqdT.contiguous()
        gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT, gqdT, k=ctx.k, mass_grad=ctx.has_mass)
        return None, gq0, gqd0, gtau, gm, None


class RolloutTrajectory(torch.autograd.Function):
    """(q0, qd0, tau, mass) -> every state x^0..x^T as [T+1, nq_max + nv_max, B].

    For objectives over the whole trajectory (per-step costs, Sec. 2: Phi(x, u)):
    the backward receives dPhi/dx^t for every t and passes it to
    sim_backward_rollout as per-step seeds (g_traj), so the same one-step
    recompute adjoint runs once for all terms.
    """

    @staticmethod
    def forward(ctx, sim: Simulator, q0, qd0, tau, mass=None, k: int = 1):
        q0, qd0, tau = q0.contiguous(), qd0.contiguous(), tau.contiguous()
        if mass is not None:
            sim.set_masses(mass.detach().contiguous())
        _, _, ck, traj = sim.rollout(q0, qd0, tau, k=k, ckpt=True, traj=True)
        ctx.sim, ctx.k, ctx.has_mass = sim, k, mass is not None
        ctx.save_for_backward(ck, tau, mass.detach() if mass is not None else None)
        return traj

    @staticmethod
    def backward(ctx, g_traj):
        ck, tau, mass = ctx.saved_tensors
        sim = ctx.sim
        if mass is not None:
            sim.set_masses(mass.contiguous())
        zq = torch.zeros(sim.nq_max, sim.B, dtype=sim.dtype, device=sim.device)
        zqd = torch.zeros(sim.nv_max, sim.B, dtype=sim.dtype, device=sim.device)
        gq0, gqd0, gtau, gm = sim.backward(ck, tau, zq, zqd, k=ctx.k, g_traj=g_traj.contiguous(),
                                           mass_grad=ctx.has_mass)
        return None, gq0, gqd0, gtau, gm, None
