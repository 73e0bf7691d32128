"""ctypes wrapper of the FP64 CPU oracle (oracle/sph_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by __graft_entry__.smoke()
and by bench.py's CPU baseline leg; the product path never imports it.
The oracle shares no code with the CUDA library: only the seeded input
generators (paper_2510_25702_gb300.cases) feed both.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_HDR = os.path.join(_HERE, "sph_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

MAX_BUFFERS = 16
MAX_THETA = 64
DT_MODES = {"dual": 0, "single": 1, "fixed": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        # OpenMP over particles: every per-particle result is a sum in that
        # particle's own neighbour order, so the thread count changes nothing
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp",
               "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(cmd).returncode != 0:
            subprocess.check_call([x for x in cmd if x != "-fopenmp"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("rans", C.c_int), ("dt_mode", C.c_int), ("n_ac_fixed", C.c_int),
        ("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double), ("c0", C.c_double),
        ("nu_l", C.c_double), ("eta", C.c_double), ("U_ref", C.c_double),
        ("dt_ad_fixed", C.c_double), ("g", C.c_double * 3), ("lo", C.c_double * 3),
        ("hi", C.c_double * 3), ("periodic", C.c_int * 3), ("seed", C.c_uint32),
        ("gen_offset", C.c_double), ("id_check", C.c_int), ("contain_check", C.c_int),
        ("mirror_B", C.c_int), ("compensation", C.c_int), ("neighbor_mode", C.c_int),
        ("rkgc", C.c_int), ("freeze_turb", C.c_int), ("comp_B", C.c_int), ("bhat_buffer", C.c_int),
        ("density_sum", C.c_int), ("wall_fn", C.c_int), ("tvf_pbuf", C.c_int), ("tvf_alpha", C.c_double),
    ]


class OrcBuffer(C.Structure):
    _fields_ = [
        ("type", C.c_int), ("turb_bc", C.c_int), ("n_theta", C.c_int), ("pad0", C.c_int),
        ("origin", C.c_double * 3), ("frame", C.c_double * 9), ("length", C.c_double),
        ("half", C.c_double * 2), ("p_ob", C.c_double), ("noise", C.c_double),
        ("k_in", C.c_double), ("eps_in", C.c_double), ("theta", C.c_double * MAX_THETA),
    ]


_PD = C.POINTER(C.c_double)


class OrcState(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("cap", C.c_int64), ("nw", C.c_int64),
        ("pos", _PD), ("vel", _PD), ("pos0", _PD), ("rho", _PD), ("mass", _PD), ("drho", _PD),
        ("k", _PD), ("eps", _PD), ("nut", _PD), ("label", C.POINTER(C.c_int32)),
        ("uid", C.POINTER(C.c_uint32)), ("dead", C.POINTER(C.c_uint8)),
        ("p", _PD), ("B", _PD), ("acc_nu", _PD), ("acc_p", _PD), ("gradv", _PD),
        ("wpos", _PD), ("wvel", _PD),
        ("next_uid", C.c_uint32), ("nbuf", C.c_int32), ("step", C.c_int64), ("t", C.c_double),
        ("dt_ad", C.c_double), ("dt_ac", C.c_double), ("dt", C.c_double), ("n_ac", C.c_int32),
        ("pad0", C.c_int32), ("n_spawned", C.c_int64), ("n_deleted", C.c_int64),
        ("buf", OrcBuffer * MAX_BUFFERS),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        cfgp, stp = C.POINTER(OrcConfig), C.POINTER(OrcState)
        L.orc_W.restype = C.c_double
        L.orc_W.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_dW.restype = C.c_double
        L.orc_dW.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_uniform_pm1.restype = C.c_double
        L.orc_uniform_pm1.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_cell_key.restype = C.c_int64
        L.orc_cell_key.argtypes = [cfgp, _PD]
        L.orc_pairs.restype = C.c_int64
        L.orc_pairs.argtypes = [cfgp, stp, C.POINTER(C.c_int64), C.c_int64]
        for name in ("orc_compact_sort", "orc_configure", "orc_label", "orc_time_step",
                     "orc_viscous", "orc_momentum", "orc_continuity", "orc_transport", "orc_density_sum"):
            getattr(L, name).argtypes = [cfgp, stp]
        L.orc_bmatrix.argtypes = [cfgp, stp, _PD]
        for name in ("orc_rans", "orc_half1", "orc_kick", "orc_density"):
            getattr(L, name).argtypes = [cfgp, stp, C.c_double]
        L.orc_apply_bc.argtypes = [cfgp, stp, C.c_int64, C.c_uint32]
        L.orc_buffer_update.argtypes = [cfgp, stp, C.c_int64]
        L.orc_step.argtypes = [cfgp, stp, C.c_int]
        L.orc_kernel_gradient_sum.argtypes = [cfgp, stp, _PD]
        L.orc_kernel_sum.argtypes = [cfgp, stp, _PD]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_wall_utau.restype = C.c_double
        L.orc_wall_utau.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int)]
        _lib = L
    return _lib


def num_threads() -> int:
    """Threads the oracle's per-particle loops run on (OMP_NUM_THREADS)."""
    return int(lib().orc_num_threads())


def wall_utau(ut: float, y: float, nu: float):
    """(u_tau, log_layer) of the step-wise wall law."""
    lg = C.c_int()
    u = lib().orc_wall_utau(float(ut), float(y), float(nu), C.byref(lg))
    return float(u), bool(lg.value)


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} returned {rc}")


# (rkgc, mirror_B, comp_B, bhat_buffer) of the open-boundary treatments
# compared in Sec. 4.1 (Table of the four cases): 1 the original VIPO (no
# kernel correction), 2 VIPO with the correction applied directly (truncated
# support, own B_j at buffer neighbours), 3 VIPO with the corrected RKGC
# (mirror support and B_k = B_i, compensation without B_i), 4 the improved
# VIPO (the default); "minimal_mirror" is case 4 with B_i from the truncated
# support (B_k = B_i and the corrected compensation only).
OBC_SWITCHES = {"improved": None, "vipo": (0, 0, 0, 0), "vipo_rkgc": (1, 0, 0, 0),
                "vipo_rkgc_mirror": (1, 1, 0, 1), "minimal_mirror": (1, 0, 1, 1)}


class OracleSim:
    """State of the FP64 oracle for one case.

    switches: gen_offset (0.5), id_check, contain_check, mirror_B,
    compensation (all 1 = the paper's improved scheme), neighbor_mode
    (0 brute force, 1 cell grid).
    """

    def __init__(self, case, capacity: Optional[int] = None, neighbor_mode: int = 1,
                 gen_offset: float = 0.5, id_check: int = 1, contain_check: int = 1,
                 mirror_B: int = 1, compensation: int = 1, rkgc: int = 1, freeze_turb: int = 0,
                 comp_B: int = 1, bhat_buffer: int = 1):
        self.case = case
        cap = int(capacity or case.capacity or case.n + 16)
        n, nw = case.n, case.nw
        if n > cap:
            raise ValueError("capacity below particle count")
        self.cfg = OrcConfig()
        c = self.cfg
        c.dim, c.rans = case.dim, int(bool(case.rans))
        c.dt_mode = DT_MODES[case.dt_mode]
        c.n_ac_fixed = int(case.n_ac_fixed)
        c.dp, c.h, c.rho0, c.c0, c.nu_l = case.dp, case.h, case.rho0, case.c0, case.nu_l
        c.eta, c.U_ref, c.dt_ad_fixed = case.eta, case.U_ref, case.dt_ad_fixed
        for a in range(3):
            c.g[a] = float(case.g[a])
            c.lo[a] = float(case.lo[a])
            c.hi[a] = float(case.hi[a])
            c.periodic[a] = int(case.periodic[a])
        c.seed = int(case.seed) & 0xFFFFFFFF
        c.gen_offset = gen_offset
        c.id_check, c.contain_check = id_check, contain_check
        c.mirror_B, c.compensation = mirror_B, compensation
        c.neighbor_mode = neighbor_mode
        c.rkgc = rkgc
        c.freeze_turb = freeze_turb
        c.comp_B, c.bhat_buffer = comp_B, bhat_buffer
        c.tvf_alpha = float(getattr(case, "tvf", 0.0))
        c.tvf_pbuf = int(bool(getattr(case, "tvf_pbuf", False)))
        c.density_sum = int(bool(getattr(case, "density_sum", False)))
        c.wall_fn = int(bool(getattr(case, "wall_function", False)))
        # the open-boundary treatment of the case (Table of Sec. 4.1) sets
        # the switches it names; the improved scheme keeps the arguments
        obc = OBC_SWITCHES[getattr(case, "obc", "improved")]
        if obc is not None:
            c.rkgc, c.mirror_B, c.comp_B, c.bhat_buffer = obc

        z3 = lambda m: np.zeros((m, 3))
        self.a: Dict[str, np.ndarray] = dict(
            pos=z3(cap), vel=z3(cap), pos0=z3(cap), rho=np.zeros(cap), mass=np.zeros(cap),
            drho=np.zeros(cap), k=np.zeros(cap), eps=np.zeros(cap), nut=np.zeros(cap),
            label=np.zeros(cap, np.int32), uid=np.zeros(cap, np.uint32),
            dead=np.zeros(cap, np.uint8), p=np.zeros(cap), B=np.zeros((cap, 9)),
            acc_nu=z3(cap), acc_p=z3(cap), gradv=np.zeros((cap, 9)),
            wpos=np.ascontiguousarray(case.wpos, dtype=np.float64).reshape(-1, 3).copy(),
            wvel=np.ascontiguousarray(case.wvel, dtype=np.float64).reshape(-1, 3).copy(),
        )
        a = self.a
        a["pos"][:n] = case.pos
        a["pos0"][:n] = case.pos
        a["vel"][:n] = case.vel
        a["rho"][:n] = case.rho
        a["mass"][:n] = case.mass
        a["k"][:n] = case.k
        a["eps"][:n] = case.eps
        if case.rans:
            a["nut"][:n] = 0.09 * a["k"][:n] ** 2 / a["eps"][:n]
        a["uid"][:n] = np.arange(n, dtype=np.uint32)
        a["p"][:n] = case.rho0 * case.c0 ** 2 * (a["rho"][:n] / case.rho0 - 1.0)
        self.st = OrcState()
        s = self.st
        s.n, s.cap, s.nw = n, cap, nw
        for name in ("pos", "vel", "pos0", "rho", "mass", "drho", "k", "eps", "nut", "p", "B",
                     "acc_nu", "acc_p", "gradv", "wpos", "wvel"):
            setattr(s, name, _ptr(a[name], C.c_double))
        s.label = _ptr(a["label"], C.c_int32)
        s.uid = _ptr(a["uid"], C.c_uint32)
        s.dead = _ptr(a["dead"], C.c_uint8)
        s.next_uid = n
        if len(case.buffers) > MAX_BUFFERS:
            raise ValueError("too many buffers")
        s.nbuf = len(case.buffers)
        for b, spec in enumerate(case.buffers):
            ob = s.buf[b]
            ob.type = 0 if spec.kind == "velocity" else 1
            ob.turb_bc = 1 if spec.turb == "freestream" else 0
            th = list(spec.theta)
            if not 1 <= len(th) <= MAX_THETA:
                raise ValueError("theta length")
            ob.n_theta = len(th)
            for q, v in enumerate(th):
                ob.theta[q] = float(v)
            fr = np.asarray(spec.frame, dtype=np.float64).reshape(9)
            for q in range(9):
                ob.frame[q] = float(fr[q])
            for q in range(3):
                ob.origin[q] = float(spec.origin[q])
            ob.length = float(spec.length)
            ob.half[0], ob.half[1] = float(spec.half[0]), float(spec.half[1])
            ob.p_ob, ob.noise = float(spec.p_ob), float(spec.noise)
            ob.k_in, ob.eps_in = float(spec.k_in), float(spec.eps_in)
        self._cp = C.byref(self.cfg)
        self._sp = C.byref(self.st)

    # ------------------------------------------------------------ stages
    @property
    def n(self) -> int:
        return int(self.st.n)

    def step(self, nsteps: int = 1):
        _check(lib().orc_step(self._cp, self._sp, int(nsteps)), "orc_step")

    def set_profile(self, buffer_id: int, theta):
        """Replace the velocity profile of a buffer (theta across the width)."""
        th = np.asarray(theta, np.float64).reshape(-1)
        if not 1 <= th.size <= MAX_THETA:
            raise ValueError("theta length")
        b = self.st.buf[buffer_id]
        b.n_theta = th.size
        for q, v in enumerate(th):
            b.theta[q] = float(v)

    def compact_sort(self):
        _check(lib().orc_compact_sort(self._cp, self._sp), "orc_compact_sort")

    def configure(self):
        _check(lib().orc_configure(self._cp, self._sp), "orc_configure")

    def label(self):
        _check(lib().orc_label(self._cp, self._sp), "orc_label")

    def time_step(self):
        _check(lib().orc_time_step(self._cp, self._sp), "orc_time_step")
        return float(self.st.dt_ad), float(self.st.dt_ac), int(self.st.n_ac)

    def bmatrix(self, want_A: bool = False):
        A = np.zeros((self.st.cap, 9)) if want_A else None
        _check(lib().orc_bmatrix(self._cp, self._sp, _ptr(A, C.c_double) if want_A else None),
               "orc_bmatrix")
        return A[: self.n].reshape(-1, 3, 3) if want_A else None

    def viscous(self):
        _check(lib().orc_viscous(self._cp, self._sp), "orc_viscous")

    def density_sum(self):
        _check(lib().orc_density_sum(self._cp, self._sp), "orc_density_sum")

    def lattice_kernel_sum(self) -> float:
        L = lib()
        L.orc_lattice_kernel_sum.restype = C.c_double
        L.orc_lattice_kernel_sum.argtypes = [C.POINTER(OrcConfig)]
        return float(L.orc_lattice_kernel_sum(self._cp))

    def transport(self):
        _check(lib().orc_transport(self._cp, self._sp), "orc_transport")

    def rans(self, dt: float):
        _check(lib().orc_rans(self._cp, self._sp, float(dt)), "orc_rans")

    def half1(self, dt: float):
        _check(lib().orc_half1(self._cp, self._sp, float(dt)), "orc_half1")

    def momentum(self):
        _check(lib().orc_momentum(self._cp, self._sp), "orc_momentum")

    def kick(self, dt: float):
        _check(lib().orc_kick(self._cp, self._sp, float(dt)), "orc_kick")

    def continuity(self):
        _check(lib().orc_continuity(self._cp, self._sp), "orc_continuity")

    def density(self, dt: float):
        _check(lib().orc_density(self._cp, self._sp, float(dt)), "orc_density")

    def apply_bc(self, step: int, sub: int):
        _check(lib().orc_apply_bc(self._cp, self._sp, int(step), int(sub) & 0xFFFFFFFF),
               "orc_apply_bc")

    def buffer_update(self, step: int):
        _check(lib().orc_buffer_update(self._cp, self._sp, int(step)), "orc_buffer_update")

    def pairs(self) -> np.ndarray:
        """(i, j, is_wall) rows of the frozen configuration, ascending."""
        m = lib().orc_pairs(self._cp, self._sp, None, 0)
        out = np.zeros((max(m, 1), 3), np.int64)
        lib().orc_pairs(self._cp, self._sp, _ptr(out, C.c_int64), m)
        return out[:m]

    def kernel_gradient_sum(self) -> np.ndarray:
        out = np.zeros((self.n, 3))
        _check(lib().orc_kernel_gradient_sum(self._cp, self._sp, _ptr(out, C.c_double)), "kgs")
        return out

    def kernel_sum(self) -> np.ndarray:
        out = np.zeros(self.n)
        _check(lib().orc_kernel_sum(self._cp, self._sp, _ptr(out, C.c_double)), "ks")
        return out

    def cell_keys(self) -> np.ndarray:
        pos = self.a["pos"]
        return np.array([lib().orc_cell_key(self._cp, _ptr(pos[i], C.c_double)) for i in range(self.n)],
                        dtype=np.int64)

    # ------------------------------------------------------------ read-out
    def fields(self, live_only: bool = True, by_uid: bool = True) -> Dict[str, np.ndarray]:
        n = self.n
        keep = np.ones(n, bool)
        if live_only:
            keep = self.a["dead"][:n] == 0
        out = {}
        for name in ("pos", "vel", "rho", "mass", "drho", "k", "eps", "nut", "label", "uid", "p",
                     "B", "acc_nu", "acc_p", "gradv"):
            out[name] = self.a[name][:n][keep].copy()
        if by_uid:
            o = np.argsort(out["uid"], kind="stable")
            out = {k: v[o] for k, v in out.items()}
        return out

    @property
    def stats(self):
        s = self.st
        return dict(step=int(s.step), t=float(s.t), dt_ad=float(s.dt_ad), dt_ac=float(s.dt_ac),
                    n_ac=int(s.n_ac), n=int(s.n), n_spawned=int(s.n_spawned),
                    n_deleted=int(s.n_deleted), next_uid=int(s.next_uid))
