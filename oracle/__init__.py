"""Python access to the FP64 C oracle — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It compiles ``oracle.c`` with gcc (no contraction of multiply-adds, so x86 and Arm
hosts give the same bits) and exposes each C function through ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MAX_OBS = 8
MAX_GROUPS = 4

EV_TRANSIENT, EV_REF_EXIT, EV_FV_CONVERGED, EV_PARALLEL_EXIT, EV_FV_ALL_EXITED, EV_DECORRELATED, EV_DEPHASED = range(7)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, -ffp-contract=off)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcSystem(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("dim", C.c_int32), ("potential", C.c_int32),
        ("mass", C.POINTER(C.c_double)),
        ("dw_a", C.c_double), ("dw_b", C.c_double),
        ("sigma", C.POINTER(C.c_double)), ("epsilon", C.POINTER(C.c_double)),
        ("charge", C.POINTER(C.c_double)),
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
        ("n_groups", C.c_int32), ("group_offsets", C.c_int32 * (MAX_GROUPS + 1)),
        ("group_atoms", C.POINTER(C.c_int32)),
        ("n_obs", C.c_int32), ("obs_kind", C.c_int32 * MAX_OBS),
        ("obs_arg", (C.c_int32 * 4) * MAX_OBS),
        ("coulomb_mode", C.c_int32), ("rf_dielectric", C.c_double),
        ("gb_radius", C.POINTER(C.c_double)), ("gb_scale", C.POINTER(C.c_double)),
        ("gb_solute_dielectric", C.c_double), ("gb_solvent_dielectric", C.c_double),
        ("n_constraints", C.c_int32), ("constraint_atoms", C.POINTER(C.c_int32)),
        ("constraint_length", C.POINTER(C.c_double)), ("constraint_tol", C.c_double),
        ("constraint_max_iter", C.c_int32),
        ("box", C.c_double * 3), ("ewald_beta", C.c_double), ("pme_grid", C.c_int32 * 3),
        ("pme_order", C.c_int32), ("ewald_kmax", C.c_int32),
    ]


class OrcExit(C.Structure):
    _fields_ = [("M", C.c_int64), ("k", C.c_int32), ("label_to", C.c_int32), ("tau_steps", C.c_int64)]


class OrcEvent(C.Structure):
    _fields_ = [("kind", C.c_int32), ("omega", C.c_int32), ("label_to", C.c_int32), ("k", C.c_int32),
                ("M", C.c_int64), ("steps", C.c_int64), ("t_sim", C.c_int64), ("n_branch", C.c_int64)]


class OrcRunParams(C.Structure):
    _fields_ = [("n_rep", C.c_int32), ("seed", C.c_uint64), ("t_gr", C.c_int32), ("t_check", C.c_int32),
                ("tol", C.c_double), ("min_fv_steps", C.c_int64), ("max_steps", C.c_int64),
                ("max_exits", C.c_int32)]


class OrcOriginalParams(C.Structure):
    _fields_ = [("n_rep", C.c_int32), ("seed", C.c_uint64), ("t_check", C.c_int32), ("t_corr", C.c_int64),
                ("t_phase", C.c_int64), ("max_steps", C.c_int64), ("max_exits", C.c_int32)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcSystem)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_gb_born.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_ewald_parts.argtypes = [C.c_void_p, _D, _D]
        L.orc_unconverged.restype = C.c_int64
        L.orc_unconverged.argtypes = [C.c_void_p]
        L.orc_potential.restype = C.c_double
        L.orc_potential.argtypes = [C.c_void_p, _D]
        L.orc_forces.argtypes = [C.c_void_p, _D, _D]
        L.orc_param_grad.argtypes = [C.c_void_p, _D, _D]
        L.orc_adjoint_segment.restype = C.c_double
        L.orc_adjoint_segment.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _D, _D, _D, C.c_uint64, C.c_int64, C.c_int64,
                                          C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                          _D, _D, _D]
        L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.orc_normals.argtypes = [C.c_uint64, C.c_int64, C.c_int32, C.c_int32, _D]
        L.orc_branch_word.restype = C.c_uint32
        L.orc_branch_word.argtypes = [C.c_uint64, C.c_int64, C.c_int32]
        L.orc_baoab_step.argtypes = [C.c_void_p, _D, _D, _D, C.c_uint64, C.c_int32, C.c_int64]
        L.orc_state_of.restype = C.c_int32
        L.orc_state_of.argtypes = [C.c_void_p, _D]
        L.orc_exited.restype = C.c_int32
        L.orc_exited.argtypes = [C.c_void_p, _D, C.c_int32]
        L.orc_cv.argtypes = [C.c_void_p, _D, _D]
        L.orc_observable.restype = C.c_double
        L.orc_observable.argtypes = [C.c_void_p, C.c_int32, _D, _D]
        L.orc_gelman_rubin.restype = C.c_double
        L.orc_gelman_rubin.argtypes = [C.c_int32, C.c_int32, _D]
        L.orc_fv_branch.restype = C.c_int32
        L.orc_fv_branch.argtypes = [C.c_uint64, C.c_int64, C.c_int32, _U8, _I32]
        L.orc_step_k.restype = C.c_int32
        L.orc_step_k.argtypes = [C.c_void_p, C.c_int32, _D, _D, _D, C.c_uint64, C.c_int64, C.c_int64,
                                 C.c_int64, C.c_int32, _D, C.c_int32]
        L.orc_step_k_from.restype = C.c_int32
        L.orc_step_k_from.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _D, _D, _D, C.c_uint64, C.c_int64,
                                      C.c_int64, C.c_int64, C.c_int32, _D, C.c_int32]
        L.orc_parallel_phase.restype = C.c_int32
        L.orc_parallel_phase.argtypes = [C.c_void_p, C.c_int32, _D, _D, _D, C.c_uint64, C.c_int64,
                                         C.c_int32, C.c_int32, C.c_int64, C.POINTER(OrcExit)]
        L.orc_run_original.restype = C.c_int32
        L.orc_run_original.argtypes = [C.c_void_p, C.POINTER(OrcOriginalParams), _D, _D, C.POINTER(OrcEvent),
                                       C.c_int32, _I64]
        L.orc_run_genparrep.restype = C.c_int32
        L.orc_run_genparrep.argtypes = [C.c_void_p, C.POINTER(OrcRunParams), _D, _D,
                                        C.POINTER(OrcEvent), C.c_int32, _I64]
        L.orc_run_bruteforce.restype = C.c_int32
        L.orc_run_bruteforce.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, _D, _D, C.c_int64, _I64,
                                         _I32, C.c_int32]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One system loaded into the oracle.  Arrays are kept alive for the lifetime of the object."""

    def __init__(self, system):
        s = system
        self.system = s
        ea = s.empty_arrays()
        keep = {}

        def d(name, arr):
            keep[name] = _c64(arr)
            return _dp(keep[name])

        def i(name, arr):
            keep[name] = np.ascontiguousarray(arr, dtype=np.int32)
            return keep[name].ctypes.data_as(_I32)

        st = OrcSystem()
        st.n_atoms, st.dim, st.potential = s.n_atoms, s.dim, s.potential
        st.mass = d("mass", s.mass)
        st.dw_a, st.dw_b = s.dw_a, s.dw_b
        st.sigma, st.epsilon, st.charge = d("sigma", ea["sigma"]), d("eps", ea["epsilon"]), d("q", ea["charge"])
        st.n_excl, st.excl = len(ea["excl"]), i("excl", ea["excl"])
        st.cutoff, st.coulomb_k = s.cutoff, s.coulomb_k
        st.coulomb_mode, st.rf_dielectric = s.coulomb_mode, s.rf_dielectric
        if s.gb_radius is not None:
            st.gb_radius, st.gb_scale = d("gbr", s.gb_radius), d("gbs", s.gb_scale)
        st.gb_solute_dielectric, st.gb_solvent_dielectric = s.gb_solute_dielectric, s.gb_solvent_dielectric
        if s.constraints is not None and len(s.constraints):
            st.n_constraints = len(s.constraints)
            st.constraint_atoms = i("con", s.constraints)
            st.constraint_length = d("conl", s.constraint_length)
        st.constraint_tol, st.constraint_max_iter = s.constraint_tol, s.constraint_max_iter
        if s.box is not None:
            for x in range(3):
                st.box[x], st.pme_grid[x] = s.box[x], s.pme_grid[x]
        st.ewald_beta, st.pme_order, st.ewald_kmax = s.ewald_beta, s.pme_order, s.ewald_kmax
        st.n_bonds, st.bond_atoms = len(ea["bonds"]), i("bonds", ea["bonds"])
        st.bond_k, st.bond_r0 = d("bk", ea["bond_k"]), d("br0", ea["bond_r0"])
        st.n_angles, st.angle_atoms = len(ea["angles"]), i("angles", ea["angles"])
        st.angle_k, st.angle_theta0 = d("ak", ea["angle_k"]), d("at0", ea["angle_theta0"])
        st.n_dihedrals, st.dihedral_atoms = len(ea["dihedrals"]), i("dih", ea["dihedrals"])
        st.dihedral_n = i("dn", ea["dihedral_n"])
        st.dihedral_k, st.dihedral_delta = d("dk", ea["dihedral_k"]), d("dd", ea["dihedral_delta"])
        st.kT, st.gamma, st.dt = s.kT, s.gamma, s.dt
        st.cv_kind = s.cv_kind
        for t, a in enumerate(s.cv_atoms):
            st.cv_atoms[t] = a
        for t, v in enumerate(s.cv_params):
            st.cv_params[t] = v
        groups = list(s.groups)
        st.n_groups = len(groups)
        offs = [0]
        for g in groups:
            offs.append(offs[-1] + len(g))
        for t, o in enumerate(offs):
            st.group_offsets[t] = o
        flat = np.concatenate([np.asarray(g, np.int32) for g in groups]) if groups else np.zeros(1, np.int32)
        st.group_atoms = i("groups", flat)
        st.n_obs = len(s.observables)
        for j, (kind, args) in enumerate(s.observables):
            st.obs_kind[j] = kind
            for t, a in enumerate(args):
                st.obs_arg[j][t] = a
        self._keep = keep
        self._st = st
        self.ctx = lib().orc_create(C.byref(st))
        if not self.ctx:
            raise MemoryError("orc_create failed")
        self.nd = s.n_atoms * s.dim

    def __del__(self):
        if getattr(self, "ctx", None) and _lib is not None:
            _lib.orc_destroy(self.ctx)
            self.ctx = None

    # -- single-configuration functions
    def potential(self, q):
        q = _c64(q)
        return lib().orc_potential(self.ctx, _dp(q))

    def forces(self, q):
        q = _c64(q)
        f = np.zeros_like(q)
        lib().orc_forces(self.ctx, _dp(q), _dp(f))
        return f

    def param_grad(self, q):
        """dV/d theta: [sigma_i (n), epsilon_i (n), dihedral k_t (n_dihedrals)]."""
        q = _c64(q)
        s = self.system
        nd = 0 if s.dihedrals is None else len(s.dihedrals)
        g = np.zeros(2 * s.n_atoms + nd)
        lib().orc_param_grad(self.ctx, _dp(q), _dp(g))
        return g

    def adjoint_segment(self, q, p, f, seed, t0, tp0, k, t_gr, obs, transform=0, center=0.0, width=1.0,
                        replica0=0):
        """Advance (q, p, f) [R, n, dim] in place by k steps (row r draws the noise of replica replica0 + r);
        returns (L, dL/dtheta, dL/dq0, dL/dp0)."""
        s = self.system
        nd = 0 if s.dihedrals is None else len(s.dihedrals)
        gth = np.zeros(2 * s.n_atoms + nd)
        gq = np.zeros_like(q)
        gp = np.zeros_like(p)
        loss = lib().orc_adjoint_segment(self.ctx, q.shape[0], replica0, _dp(q), _dp(p), _dp(f), seed, t0, tp0, k, t_gr, obs,
                                         transform, center, width, _dp(gth), _dp(gq), _dp(gp))
        return loss, gth, gq, gp

    def unconverged(self):
        """Constraint projections so far whose sweeps ran out before the tolerance."""
        return lib().orc_unconverged(self.ctx)

    def ewald_parts(self, q):
        """The five parts of the periodic Coulomb energy (real space, excluded pairs, self,
        reciprocal, background) of one configuration."""
        out = np.zeros(5)
        lib().orc_ewald_parts(self.ctx, _dp(_c64(q)), _dp(out))
        return out

    def gb_born(self, q):
        """Generalized Born radii B_i and descreening sums I_i of configuration q."""
        n = self.system.n_atoms
        born, integral = np.zeros(n), np.zeros(n)
        lib().orc_gb_born(self.ctx, _dp(_c64(q)), _dp(born), _dp(integral))
        return born, integral

    def state_of(self, q):
        return lib().orc_state_of(self.ctx, _dp(_c64(q)))

    def exited(self, q, omega):
        return lib().orc_exited(self.ctx, _dp(_c64(q)), omega)

    def cv(self, q):
        """The state definition's collective variables: (phi, psi), (x, 0), (d, 0), or the m rotamer
        torsions (degrees)."""
        out = np.zeros(4)
        lib().orc_cv(self.ctx, _dp(_c64(q)), _dp(out))
        if self.system.cv_kind == 3:
            return out[: int(self.system.cv_params[0])]
        return out[:2]

    def observable(self, j, q, p):
        return lib().orc_observable(self.ctx, j, _dp(_c64(q)), _dp(_c64(p)))

    def observables(self, q, p):
        return np.array([self.observable(j, q, p) for j in range(len(self.system.observables))])

    def baoab_step(self, q, p, f, seed, replica, step):
        lib().orc_baoab_step(self.ctx, _dp(q), _dp(p), _dp(f), seed, replica, step)

    # -- replica-batch functions (arrays [R, n, dim], modified in place)
    def step_k(self, q, p, f, seed, t0, tp0, k, t_gr, cap=0):
        R = q.shape[0]
        no = len(self.system.observables)
        samples = np.zeros((R, max(cap, 1), max(no, 1)))
        ns = lib().orc_step_k(self.ctx, R, _dp(q), _dp(p), _dp(f), seed, t0, tp0, k, t_gr,
                              _dp(samples), cap)
        return samples[:, :min(ns, cap), :no]

    def step_k_from(self, q, p, f, seed, replica0, t0, tp0, k, t_gr, cap=0):
        """step_k for rows that are the replicas replica0.. of a larger set (their noise indices)."""
        R = q.shape[0]
        no = len(self.system.observables)
        samples = np.zeros((R, max(cap, 1), max(no, 1)))
        ns = lib().orc_step_k_from(self.ctx, R, replica0, _dp(q), _dp(p), _dp(f), seed, t0, tp0, k, t_gr,
                                   _dp(samples), cap)
        return samples[:, :min(ns, cap), :no]

    def parallel_phase(self, q, p, f, seed, t0, omega, t_check, max_checks):
        out = OrcExit()
        found = lib().orc_parallel_phase(self.ctx, q.shape[0], _dp(q), _dp(p), _dp(f), seed, t0, omega,
                                         t_check, max_checks, C.byref(out))
        return bool(found), {"M": out.M, "k": out.k, "label_to": out.label_to, "tau_steps": out.tau_steps}

    def run_genparrep(self, n_rep, seed, t_gr, t_check, tol, min_fv_steps, max_steps, max_exits,
                      q0=None, p0=None, max_events=100000):
        s = self.system
        q0 = _c64(s.q0 if q0 is None else q0)
        p0 = _c64(s.p0 if p0 is None else p0)
        rp = OrcRunParams(n_rep, seed, t_gr, t_check, tol, min_fv_steps, max_steps, max_exits)
        ev = (OrcEvent * max_events)()
        tg = C.c_int64(0)
        n = lib().orc_run_genparrep(self.ctx, C.byref(rp), _dp(q0), _dp(p0), ev, max_events, C.byref(tg))
        events = [{"kind": e.kind, "omega": e.omega, "label_to": e.label_to, "k": e.k, "M": e.M,
                   "steps": e.steps, "t_sim": e.t_sim, "n_branch": e.n_branch} for e in ev[:n]]
        return events, tg.value

    def run_original(self, n_rep, seed, t_check, t_corr, t_phase, max_steps, max_exits, q0=None, p0=None,
                     max_events=100000):
        """The original ParRep loop (decorrelation, dephasing, parallel step); returns (events, t_global)."""
        s = self.system
        q0 = _c64(s.q0 if q0 is None else q0)
        p0 = _c64(s.p0 if p0 is None else p0)
        rp = OrcOriginalParams(n_rep, seed, t_check, t_corr, t_phase, max_steps, max_exits)
        ev = (OrcEvent * max_events)()
        tg = C.c_int64(0)
        n = lib().orc_run_original(self.ctx, C.byref(rp), _dp(q0), _dp(p0), ev, max_events, C.byref(tg))
        events = [{"kind": e.kind, "omega": e.omega, "label_to": e.label_to, "k": e.k, "M": e.M,
                   "steps": e.steps, "t_sim": e.t_sim, "n_branch": e.n_branch} for e in ev[:n]]
        return events, tg.value

    def run_bruteforce(self, seed, t_check, max_steps, max_res, q0=None, p0=None):
        s = self.system
        q0 = _c64(s.q0 if q0 is None else q0)
        p0 = _c64(s.p0 if p0 is None else p0)
        res = np.zeros(max_res, np.int64)
        frm = np.zeros(max_res, np.int32)
        n = lib().orc_run_bruteforce(self.ctx, seed, t_check, _dp(q0), _dp(p0), max_steps,
                                     res.ctypes.data_as(_I64), frm.ctypes.data_as(_I32), max_res)
        return res[:n], frm[:n]


# -- free functions
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def normals(seed, step, replica, atom):
    out = np.zeros(4)
    lib().orc_normals(seed, step, replica, atom, _dp(out))
    return out


def branch_word(seed, step, replica):
    return int(lib().orc_branch_word(seed, step, replica))


def gelman_rubin(samples):
    x = _c64(samples)
    return lib().orc_gelman_rubin(x.shape[0], x.shape[1], _dp(x))


def fv_branch(seed, step, exited):
    ex = np.ascontiguousarray(exited, dtype=np.uint8)
    src = np.zeros(len(ex), np.int32)
    nb = lib().orc_fv_branch(seed, step, len(ex), ex.ctypes.data_as(_U8), src.ctypes.data_as(_I32))
    return nb, src
