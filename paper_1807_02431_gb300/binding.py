"""Thin ctypes binding of libgrp.so (include/grp.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library.  Loading fails loudly (GrpError) when the compiled
library is missing: there is no CPU fallback.  Device pointers may be given as ints or as CUDA
torch tensors; host arrays are numpy arrays.  `stream` is a cudaStream_t handle (int), a
torch.cuda.Stream, or None for the legacy default stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgrp.so")

GRP_OK = 0
GRP_EINVAL, GRP_ENOMEM, GRP_ECUDA, GRP_ENAN, GRP_EOVERFLOW, GRP_ETIMEOUT, GRP_ENOTIMPL = -1, -2, -3, -4, -5, -6, -7
GRP_NOEXIT = 1
GRP_FP64, GRP_MIXED = 0, 1
GRP_MAX_OBS, GRP_MAX_GROUPS = 8, 4
(EV_TRANSIENT, EV_REF_EXIT, EV_FV_CONVERGED, EV_PARALLEL_EXIT, EV_FV_ALL_EXITED, EV_DECORRELATED,
 EV_DEPHASED) = range(7)

_lib = None


class GrpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"grp status {status}: {msg}")
        self.status = status


class SystemDesc(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("dim", C.c_int32), ("potential", C.c_int32), ("precision", C.c_int32),
        ("mass", C.POINTER(C.c_double)), ("dw_a", C.c_double), ("dw_b", C.c_double),
        ("sigma", C.POINTER(C.c_double)), ("epsilon", C.POINTER(C.c_double)), ("charge", C.POINTER(C.c_double)),
        ("n_excl", C.c_int32), ("excl", C.POINTER(C.c_int32)),
        ("cutoff", C.c_double), ("coulomb_k", C.c_double),
        ("n_bonds", C.c_int32), ("bond_atoms", C.POINTER(C.c_int32)),
        ("bond_k", C.POINTER(C.c_double)), ("bond_r0", C.POINTER(C.c_double)),
        ("n_angles", C.c_int32), ("angle_atoms", C.POINTER(C.c_int32)),
        ("angle_k", C.POINTER(C.c_double)), ("angle_theta0", C.POINTER(C.c_double)),
        ("n_dihedrals", C.c_int32), ("dihedral_atoms", C.POINTER(C.c_int32)),
        ("dihedral_n", C.POINTER(C.c_int32)),
        ("dihedral_k", C.POINTER(C.c_double)), ("dihedral_delta", C.POINTER(C.c_double)),
        ("kT", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
        ("cv_kind", C.c_int32), ("cv_atoms", C.c_int32 * 8), ("cv_params", C.c_double * 8),
        ("n_groups", C.c_int32), ("group_offsets", C.c_int32 * (GRP_MAX_GROUPS + 1)),
        ("group_atoms", C.POINTER(C.c_int32)),
        ("n_obs", C.c_int32), ("obs_kind", C.c_int32 * GRP_MAX_OBS), ("obs_arg", (C.c_int32 * 4) * GRP_MAX_OBS),
        ("coulomb_mode", C.c_int32), ("rf_dielectric", C.c_double),
        ("gb_radius", C.POINTER(C.c_double)), ("gb_scale", C.POINTER(C.c_double)),
        ("gb_solute_dielectric", C.c_double), ("gb_solvent_dielectric", C.c_double),
        ("n_constraints", C.c_int32), ("constraint_atoms", C.POINTER(C.c_int32)),
        ("constraint_length", C.POINTER(C.c_double)), ("constraint_tol", C.c_double),
        ("constraint_max_iter", C.c_int32),
        ("box", C.c_double * 3), ("ewald_beta", C.c_double), ("pme_grid", C.c_int32 * 3),
        ("pme_order", C.c_int32),
    ]


class Counters(C.Structure):
    _fields_ = [("t_global", C.c_int64), ("t_phase", C.c_int64)]


class Exit(C.Structure):
    _fields_ = [("M", C.c_int64), ("k", C.c_int32), ("label_to", C.c_int32), ("tau_steps", C.c_int64)]


class DeviceView(C.Structure):
    _fields_ = [("q", C.c_void_p), ("p", C.c_void_p), ("f", C.c_void_p), ("acc", C.c_void_p),
                ("labels", C.c_void_p), ("exited", C.c_void_p)]


class RunParams(C.Structure):
    _fields_ = [("t_gr", C.c_int32), ("t_check", C.c_int32), ("tol", C.c_double), ("min_fv_steps", C.c_int64),
                ("max_steps", C.c_int64), ("max_exits", C.c_int32)]


class OriginalParams(C.Structure):
    _fields_ = [("t_check", C.c_int32), ("max_exits", C.c_int32), ("t_corr", C.c_int64), ("t_phase", C.c_int64),
                ("max_steps", C.c_int64)]


class FvStatus(C.Structure):
    _fields_ = [("ref_exited", C.c_int32), ("label0", C.c_int32), ("n_branched", C.c_int32),
                ("converged", C.c_int32), ("gr_evaluated", C.c_int32), ("pad", C.c_int32),
                ("t_phase", C.c_int64), ("rhat", C.c_double * GRP_MAX_OBS)]


class Loss(C.Structure):
    _fields_ = [("obs", C.c_int32), ("transform", C.c_int32), ("center", C.c_double), ("width", C.c_double)]


GRP_LOSS_IDENTITY, GRP_LOSS_LOGISTIC = 0, 1


class Event(C.Structure):
    _fields_ = [("kind", C.c_int32), ("omega", C.c_int32), ("label_to", C.c_int32), ("k", C.c_int32),
                ("M", C.c_int64), ("steps", C.c_int64), ("t_sim", C.c_int64), ("n_branch", C.c_int64)]


# exported symbols and their signatures
_VP, _D, _I32P = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
SIGNATURES = {
    "grp_last_error": (C.c_char_p, []),
    "grp_create_system": (C.c_int32, [C.POINTER(SystemDesc), C.POINTER(_VP)]),
    "grp_destroy_system": (None, [_VP]),
    "grp_init_replicas": (C.c_int32, [_VP, C.c_int32, C.c_uint64, _D, _D, C.c_int32, _VP, C.POINTER(_VP)]),
    "grp_destroy_replicas": (None, [_VP]),
    "grp_step_k": (C.c_int32, [_VP, C.c_int64, C.c_int32, C.c_int32, _VP]),
    "grp_check_states": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP]),
    "grp_fv_branch": (C.c_int32, [_VP, _VP, _VP, _I32P, _VP]),
    "grp_gelman_rubin": (C.c_int32, [_VP, C.c_double, _D, _I32P, _VP]),
    "grp_run_parallel_phase": (C.c_int32, [_VP, C.c_int32, C.c_int32, C.c_int64, C.POINTER(Exit), _VP]),
    "grp_broadcast": (C.c_int32, [_VP, C.c_int32, _VP]),
    "grp_fv_check": (C.c_int32, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int64,
                                 C.POINTER(FvStatus), _VP]),
    "grp_run": (C.c_int32, [_VP, C.POINTER(RunParams), C.POINTER(Event), C.c_int32, _I32P,
                            C.POINTER(C.c_int64), _VP]),
    "grp_batch_run": (C.c_int32, [_VP, C.POINTER(RunParams), C.POINTER(Event), C.c_int32, _I32P,
                                  C.POINTER(C.c_int64), _VP]),
    "grp_batch_stats": (C.c_int32, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "grp_run_original": (C.c_int32, [_VP, C.POINTER(OriginalParams), C.POINTER(Event), C.c_int32, _I32P,
                                     C.POINTER(C.c_int64), _VP]),
    "grp_get_state": (C.c_int32, [_VP, _D, _D, _D, C.POINTER(Counters), _VP]),
    "grp_set_state": (C.c_int32, [_VP, _D, _D, _D, C.POINTER(Counters), _VP]),
    "grp_get_device_view": (C.c_int32, [_VP, C.POINTER(DeviceView)]),
    "grp_energy_forces": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP, _VP]),
    "grp_param_count": (C.c_int32, [_VP, _I32P]),
    "grp_get_params": (C.c_int32, [_VP, _VP, _VP]),
    "grp_set_params": (C.c_int32, [_VP, _VP, _VP]),
    "grp_energy_grad": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP]),
    "grp_adjoint_segment": (C.c_int32, [_VP, C.c_int32, C.c_int32, C.c_int32, C.POINTER(Loss), _D, _VP, _VP, _VP,
                                        _VP]),
    "grp_fv_branch_noalloc": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP, _VP, _VP, C.c_uint64, C.c_int64, _I32P,
                                          _VP]),
    "grp_batch_create": (C.c_int32, [C.POINTER(_VP), C.c_int32, C.POINTER(_VP)]),
    "grp_batch_destroy": (None, [_VP]),
    "grp_batch_step_k": (C.c_int32, [_VP, C.c_int64, C.c_int32, _VP]),
    "grp_batch_fv_check": (C.c_int32, [_VP, _I32P, C.c_int32, C.c_int32, C.c_double, C.c_int64,
                                       C.POINTER(FvStatus), _VP]),
    "grp_batch_autotune": (C.c_int32, [_VP, C.c_int32, _VP, _I32P]),
    "grp_set_shard": (C.c_int32, [_VP, C.c_int32, C.c_int32]),
    "grp_fv_plan": (C.c_int32, [_VP, _VP, _VP, _VP]),
    "grp_pack_rows": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP]),
    "grp_unpack_rows": (C.c_int32, [_VP, C.c_int32, _VP, _VP, _VP]),
    "grp_gr_partials": (C.c_int32, [_VP, C.c_int32, _D, _D, _VP]),
    "grp_gr_combine": (C.c_int32, [C.c_int32, _D, _D, C.c_double, _D, _I32P]),
}


def load(path: str | None = None):
    """Load libgrp.so (building it first when the sources are newer and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise GrpError(GRP_ENOTIMPL, f"CUDA library not built: {path} is missing (run build())")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status):
    if status < 0:
        raise GrpError(status, _lib.grp_last_error().decode())
    return status


def _ptr(x):
    """Device pointer of an int, None or a CUDA tensor."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _dp(a):
    return a.ctypes.data_as(_D)


class SystemHandle:
    """A grp_system plus the host arrays its description pointed to."""

    def __init__(self, system: W.System, precision: int):
        load()
        s = system
        self.system, self.precision = s, precision
        ea = s.empty_arrays()
        keep = {}

        def d(name, arr):
            keep[name] = np.ascontiguousarray(arr, dtype=np.float64)
            return _dp(keep[name])

        def i(name, arr):
            keep[name] = np.ascontiguousarray(arr, dtype=np.int32)
            return keep[name].ctypes.data_as(_I32P)

        desc = SystemDesc()
        desc.n_atoms, desc.dim, desc.potential, desc.precision = s.n_atoms, s.dim, s.potential, precision
        desc.mass = d("mass", s.mass)
        desc.dw_a, desc.dw_b = s.dw_a, s.dw_b
        desc.sigma, desc.epsilon, desc.charge = d("sg", ea["sigma"]), d("ep", ea["epsilon"]), d("ch", ea["charge"])
        desc.n_excl, desc.excl = len(ea["excl"]), i("excl", ea["excl"])
        desc.cutoff, desc.coulomb_k = s.cutoff, s.coulomb_k
        desc.coulomb_mode, desc.rf_dielectric = s.coulomb_mode, s.rf_dielectric
        if s.gb_radius is not None:
            desc.gb_radius, desc.gb_scale = d("gbr", s.gb_radius), d("gbs", s.gb_scale)
        desc.gb_solute_dielectric, desc.gb_solvent_dielectric = s.gb_solute_dielectric, s.gb_solvent_dielectric
        if s.constraints is not None and len(s.constraints):
            desc.n_constraints = len(s.constraints)
            desc.constraint_atoms = i("con", s.constraints)
            desc.constraint_length = d("conl", s.constraint_length)
        desc.constraint_tol, desc.constraint_max_iter = s.constraint_tol, s.constraint_max_iter
        if s.box is not None:
            for x in range(3):
                desc.box[x], desc.pme_grid[x] = s.box[x], s.pme_grid[x]
        desc.ewald_beta, desc.pme_order = s.ewald_beta, s.pme_order
        desc.n_bonds, desc.bond_atoms = len(ea["bonds"]), i("b", ea["bonds"])
        desc.bond_k, desc.bond_r0 = d("bk", ea["bond_k"]), d("br", ea["bond_r0"])
        desc.n_angles, desc.angle_atoms = len(ea["angles"]), i("a", ea["angles"])
        desc.angle_k, desc.angle_theta0 = d("ak", ea["angle_k"]), d("at", ea["angle_theta0"])
        desc.n_dihedrals, desc.dihedral_atoms = len(ea["dihedrals"]), i("dh", ea["dihedrals"])
        desc.dihedral_n = i("dn", ea["dihedral_n"])
        desc.dihedral_k, desc.dihedral_delta = d("dk", ea["dihedral_k"]), d("dd", ea["dihedral_delta"])
        desc.kT, desc.gamma, desc.dt = s.kT, s.gamma, s.dt
        desc.cv_kind = s.cv_kind
        for t, a in enumerate(s.cv_atoms):
            desc.cv_atoms[t] = a
        for t, v in enumerate(s.cv_params):
            desc.cv_params[t] = v
        groups = list(s.groups)
        desc.n_groups = len(groups)
        offs = [0]
        for g in groups:
            offs.append(offs[-1] + len(g))
        for t in range(GRP_MAX_GROUPS + 1):
            desc.group_offsets[t] = offs[min(t, len(offs) - 1)]
        flat = np.concatenate([np.asarray(g, np.int32) for g in groups]) if groups else np.zeros(1, np.int32)
        desc.group_atoms = i("g", flat)
        desc.n_obs = len(s.observables)
        for j, (kind, args) in enumerate(s.observables):
            desc.obs_kind[j] = kind
            for t, a in enumerate(args):
                desc.obs_arg[j][t] = a
        self._keep, self._desc = keep, desc
        h = C.c_void_p()
        _check(_lib.grp_create_system(C.byref(desc), C.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.grp_destroy_system(self.handle)
            self.handle = None


class ReplicasHandle:
    def __init__(self, sysh: SystemHandle, n_replicas: int, seed: int, q0, p0, per_replica=False, stream=None):
        self.sysh = sysh
        self.R = n_replicas
        s = sysh.system
        self.shape = (n_replicas, s.n_atoms, s.dim)
        self.n_obs = len(s.observables)
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
        h = C.c_void_p()
        _check(_lib.grp_init_replicas(sysh.handle, n_replicas, seed, _dp(q0), _dp(p0), int(per_replica),
                                      _stream(stream), C.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.grp_destroy_replicas(self.handle)
            self.handle = None


# ---- entry points with the C names
def grp_create_system(system: W.System, precision: int = GRP_FP64) -> SystemHandle:
    return SystemHandle(system, precision)


def grp_init_replicas(sysh: SystemHandle, n_replicas: int, seed: int, q0, p0, per_replica=False, stream=None):
    return ReplicasHandle(sysh, n_replicas, seed, q0, p0, per_replica, stream)


def grp_step_k(r: ReplicasHandle, k: int, t_gr: int = 0, n_active: int = 0, stream=None):
    _check(_lib.grp_step_k(r.handle, k, t_gr, n_active, _stream(stream)))


def grp_check_states(r: ReplicasHandle, omega: int, d_labels=None, d_exited=None, stream=None):
    _check(_lib.grp_check_states(r.handle, omega, _ptr(d_labels), _ptr(d_exited), _stream(stream)))


def grp_fv_branch(r: ReplicasHandle, d_exited=None, d_src=None, stream=None, count=True):
    """Branch the exited workers; returns how many were branched, or None with count=False (then the
    call does not synchronise the stream)."""
    nb = C.c_int32(0)
    _check(_lib.grp_fv_branch(r.handle, _ptr(d_exited), _ptr(d_src), C.byref(nb) if count else None,
                              _stream(stream)))
    return nb.value if count else None


def grp_gelman_rubin(r: ReplicasHandle, tol: float, stream=None):
    rhat = np.zeros(max(r.n_obs, 1))
    conv = C.c_int32(0)
    _check(_lib.grp_gelman_rubin(r.handle, tol, _dp(rhat), C.byref(conv), _stream(stream)))
    return rhat[:r.n_obs], bool(conv.value)


def grp_run_parallel_phase(r: ReplicasHandle, omega: int, t_check: int, max_checks: int, stream=None):
    out = Exit()
    st = _check(_lib.grp_run_parallel_phase(r.handle, omega, t_check, max_checks, C.byref(out), _stream(stream)))
    if st == GRP_NOEXIT:
        return None
    return {"M": out.M, "k": out.k, "label_to": out.label_to, "tau_steps": out.tau_steps}


def grp_broadcast(r: ReplicasHandle, src: int = 0, stream=None):
    _check(_lib.grp_broadcast(r.handle, src, _stream(stream)))


def grp_fv_check(r: ReplicasHandle, omega: int, t_check: int, t_gr: int, tol: float, min_fv_steps: int = 0,
                 stream=None, out: FvStatus | None = None) -> FvStatus:
    """One exit test of the convergence step; returns the status structure (reused when given)."""
    out = FvStatus() if out is None else out
    _check(_lib.grp_fv_check(r.handle, omega, t_check, t_gr, tol, min_fv_steps, C.byref(out), _stream(stream)))
    return out


def grp_run(r: ReplicasHandle, t_gr: int, t_check: int, tol: float, min_fv_steps: int, max_steps: int,
            max_exits: int, max_events: int = 100000, stream=None):
    p = RunParams(t_gr, t_check, tol, min_fv_steps, max_steps, max_exits)
    ev = (Event * max_events)()
    n = C.c_int32(0)
    tsim = C.c_int64(0)
    _check(_lib.grp_run(r.handle, C.byref(p), ev, max_events, C.byref(n), C.byref(tsim), _stream(stream)))
    events = [{"kind": e.kind, "omega": e.omega, "label_to": e.label_to, "k": e.k, "M": e.M, "steps": e.steps,
               "t_sim": e.t_sim, "n_branch": e.n_branch} for e in ev[:n.value]]
    return events, tsim.value


def grp_run_original(r: ReplicasHandle, t_check: int, t_corr: int, t_phase: int, max_steps: int, max_exits: int,
                     max_events: int = 100000, stream=None):
    p = OriginalParams(t_check, max_exits, t_corr, t_phase, max_steps)
    ev = (Event * max_events)()
    n = C.c_int32(0)
    tsim = C.c_int64(0)
    _check(_lib.grp_run_original(r.handle, C.byref(p), ev, max_events, C.byref(n), C.byref(tsim),
                                 _stream(stream)))
    events = [{"kind": e.kind, "omega": e.omega, "label_to": e.label_to, "k": e.k, "M": e.M, "steps": e.steps,
               "t_sim": e.t_sim, "n_branch": e.n_branch} for e in ev[:n.value]]
    return events, tsim.value


def grp_get_state(r: ReplicasHandle, stream=None, q=None, p=None, acc=None, copy=("q", "p", "acc")):
    """Copy the state to host arrays (allocated when not given); returns (q, p, acc, counters).  Only
    the parts named in `copy` are read (the others are returned as None)."""
    q = (np.empty(r.shape) if q is None else q) if "q" in copy else None
    p = (np.empty(r.shape) if p is None else p) if "p" in copy else None
    acc = (np.empty((r.R, r.n_obs, 4)) if acc is None else acc) if "acc" in copy else None
    ctr = Counters()
    _check(_lib.grp_get_state(r.handle, None if q is None else _dp(q), None if p is None else _dp(p),
                              _dp(acc) if (acc is not None and r.n_obs) else None, C.byref(ctr),
                              _stream(stream)))
    return q, p, acc, {"t_global": ctr.t_global, "t_phase": ctr.t_phase}


def grp_set_state(r: ReplicasHandle, q=None, p=None, acc=None, counters=None, stream=None):
    qa = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
    pa = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
    aa = None if acc is None else np.ascontiguousarray(acc, dtype=np.float64)
    ctr = None
    if counters is not None:
        ctr = Counters(counters["t_global"], counters["t_phase"])
    _check(_lib.grp_set_state(r.handle, None if qa is None else _dp(qa), None if pa is None else _dp(pa),
                              None if aa is None else _dp(aa), None if ctr is None else C.byref(ctr),
                              _stream(stream)))


def grp_get_device_view(r: ReplicasHandle) -> dict:
    v = DeviceView()
    _check(_lib.grp_get_device_view(r.handle, C.byref(v)))
    return {"q": v.q, "p": v.p, "f": v.f, "acc": v.acc, "labels": v.labels, "exited": v.exited}


def grp_energy_forces(sysh: SystemHandle, n_conf: int, d_q, d_energy=None, d_forces=None, stream=None):
    _check(_lib.grp_energy_forces(sysh.handle, n_conf, _ptr(d_q), _ptr(d_energy), _ptr(d_forces), _stream(stream)))


def grp_param_count(sysh: SystemHandle) -> int:
    n = C.c_int32(0)
    _check(_lib.grp_param_count(sysh.handle, C.byref(n)))
    return n.value


def grp_get_params(sysh: SystemHandle, d_theta, stream=None):
    _check(_lib.grp_get_params(sysh.handle, _ptr(d_theta), _stream(stream)))


def grp_set_params(sysh: SystemHandle, d_theta, stream=None):
    _check(_lib.grp_set_params(sysh.handle, _ptr(d_theta), _stream(stream)))


def grp_energy_grad(sysh: SystemHandle, n_conf: int, d_q, d_w=None, d_energy=None, d_grad_q=None,
                    d_grad_theta=None, stream=None):
    _check(_lib.grp_energy_grad(sysh.handle, n_conf, _ptr(d_q), _ptr(d_w), _ptr(d_energy), _ptr(d_grad_q),
                                _ptr(d_grad_theta), _stream(stream)))


def grp_adjoint_segment(r: ReplicasHandle, k: int, t_gr: int, checkpoint: int, obs: int, transform: int = 0,
                        center: float = 0.0, width: float = 1.0, d_grad_theta=None, d_grad_q0=None, d_grad_p0=None,
                        stream=None) -> float:
    """Advance k steps and differentiate the segment loss (see include/grp.h); returns the loss."""
    loss = Loss(obs, transform, center, width)
    out = C.c_double(0.0)
    _check(_lib.grp_adjoint_segment(r.handle, k, t_gr, checkpoint, C.byref(loss), C.byref(out), _ptr(d_grad_theta),
                                    _ptr(d_grad_q0), _ptr(d_grad_p0), _stream(stream)))
    return out.value


class BatchHandle:
    """A grp_batch over replica sets (kept alive by this object)."""

    def __init__(self, runs):
        self.runs = list(runs)
        arr = (C.c_void_p * len(self.runs))(*[r.handle for r in self.runs])
        h = C.c_void_p()
        _check(_lib.grp_batch_create(arr, len(self.runs), C.byref(h)))
        self.handle = h
        self.status = (FvStatus * len(self.runs))()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.grp_batch_destroy(self.handle)
            self.handle = None


def grp_batch_create(runs) -> BatchHandle:
    return BatchHandle(runs)


def grp_batch_step_k(b: BatchHandle, k: int, t_gr: int = 0, stream=None):
    _check(_lib.grp_batch_step_k(b.handle, k, t_gr, _stream(stream)))


def grp_batch_fv_check(b: BatchHandle, omegas, t_check: int, t_gr: int, tol: float, min_fv_steps: int = 0,
                       stream=None):
    om = np.ascontiguousarray(omegas, dtype=np.int32)
    _check(_lib.grp_batch_fv_check(b.handle, om.ctypes.data_as(_I32P), t_check, t_gr, tol, min_fv_steps, b.status,
                                   _stream(stream)))
    return b.status


def grp_batch_run(b: BatchHandle, t_gr: int, t_check: int, tol: float, min_fv_steps: int, max_steps: int,
                  max_exits: int, max_events: int = 10000, stream=None):
    """The loop of Fig. 1 for every run of the batch; returns ([events of run i], [t_sim of run i])."""
    nr = len(b.runs)
    p = RunParams(t_gr, t_check, tol, min_fv_steps, max_steps, max_exits)
    ev = (Event * (max_events * nr))()
    n = (C.c_int32 * nr)()
    tsim = (C.c_int64 * nr)()
    _check(_lib.grp_batch_run(b.handle, C.byref(p), ev, max_events, n, tsim, _stream(stream)))
    out = []
    for i in range(nr):
        out.append([{"kind": e.kind, "omega": e.omega, "label_to": e.label_to, "k": e.k, "M": e.M,
                     "steps": e.steps, "t_sim": e.t_sim, "n_branch": e.n_branch}
                    for e in ev[i * max_events:i * max_events + n[i]]])
    return out, list(tsim)


def grp_batch_stats(b: BatchHandle):
    """(ticks, ticks replayed as a CUDA graph) of the last grp_batch_run."""
    t, g = C.c_int64(0), C.c_int64(0)
    _check(_lib.grp_batch_stats(b.handle, C.byref(t), C.byref(g)))
    return t.value, g.value


def grp_batch_autotune(b: BatchHandle, t_gr: int = 0, stream=None) -> int:
    t = C.c_int32(0)
    _check(_lib.grp_batch_autotune(b.handle, t_gr, _stream(stream), C.byref(t)))
    return t.value


def grp_fv_branch_noalloc(sysh: SystemHandle, n_rep: int, d_q, d_p, d_f, d_acc, d_exited, seed: int,
                          t_global: int, stream=None) -> int:
    """Fleming-Viot branching on caller-owned device arrays; the library allocates nothing."""
    nb = C.c_int32(0)
    _check(_lib.grp_fv_branch_noalloc(sysh.handle, n_rep, _ptr(d_q), _ptr(d_p), _ptr(d_f), _ptr(d_acc),
                                      _ptr(d_exited), seed, t_global, C.byref(nb), _stream(stream)))
    return nb.value


def grp_set_shard(r: ReplicasHandle, first: int, n_global: int):
    """Make r the shard [first, first + R) of a run of n_global replicas."""
    _check(_lib.grp_set_shard(r.handle, first, n_global))


def grp_fv_plan(r: ReplicasHandle, d_exited_global, d_src, stream=None):
    """Fleming-Viot sources (global indices, -1 = kept) of the shard's replicas."""
    _check(_lib.grp_fv_plan(r.handle, _ptr(d_exited_global), _ptr(d_src), _stream(stream)))


def row_len(r: ReplicasHandle) -> int:
    """Doubles per packed row: q, p, F (n dim each) and 4 n_obs accumulator words."""
    R, n, dim = r.shape
    return 3 * n * dim + 4 * r.n_obs


def grp_pack_rows(r: ReplicasHandle, n: int, d_idx, d_buf, stream=None):
    _check(_lib.grp_pack_rows(r.handle, n, _ptr(d_idx), _ptr(d_buf), _stream(stream)))


def grp_unpack_rows(r: ReplicasHandle, n: int, d_idx, d_buf, stream=None):
    _check(_lib.grp_unpack_rows(r.handle, n, _ptr(d_idx), _ptr(d_buf), _stream(stream)))


def grp_gr_partials(r: ReplicasHandle, pass_: int, sums1=None, stream=None) -> np.ndarray:
    """Gelman-Rubin sums of the shard's workers: pass 1 -> [n_obs][3], pass 2 (sums1 = the pass-1
    sums of all shards) -> [n_obs][2]."""
    out = np.zeros((r.n_obs, 3 if pass_ == 1 else 2))
    s1 = None if sums1 is None else np.ascontiguousarray(sums1, dtype=np.float64)
    _check(_lib.grp_gr_partials(r.handle, pass_, None if s1 is None else _dp(s1), _dp(out), _stream(stream)))
    return out


def grp_gr_combine(sums1, sums2, tol: float):
    """Ratios of Eq. 3 and the convergence flag of Eq. 4 from the sums added over every shard."""
    s1 = np.ascontiguousarray(sums1, dtype=np.float64)
    s2 = np.ascontiguousarray(sums2, dtype=np.float64)
    n_obs = s1.shape[0]
    rhat = np.zeros(n_obs)
    conv = C.c_int32(0)
    _check(_lib.grp_gr_combine(n_obs, _dp(s1), _dp(s2), tol, _dp(rhat), C.byref(conv)))
    return rhat, bool(conv.value)


class _CudaArray:
    """__cuda_array_interface__ wrapper so that torch.as_tensor can view library-owned memory."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 2, "strides": None}
        self._owner = owner


def device_tensors(r: ReplicasHandle):
    """Zero-copy torch views of the replica set's device arrays (q, p, f, acc, labels, exited)."""
    import torch

    v = grp_get_device_view(r)
    R, n, dim = r.shape
    mk = lambda ptr, shape, ts: torch.as_tensor(_CudaArray(ptr, shape, ts, r), device="cuda")
    return {"q": mk(v["q"], r.shape, "<f8"), "p": mk(v["p"], r.shape, "<f8"), "f": mk(v["f"], r.shape, "<f8"),
            "acc": mk(v["acc"], (R, r.n_obs, 4), "<f8"), "labels": mk(v["labels"], (R,), "|i1"),
            "exited": mk(v["exited"], (R,), "|u1")}
