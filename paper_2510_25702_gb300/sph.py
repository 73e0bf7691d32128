"""Thin ctypes binding of the C ABI in include/sph.h.

Argument marshalling only: every stage of the step runs in the CUDA library
(_build/libsph_gb300.so).  There is no CPU fallback; constructing a
Simulation without the built library raises.  PyTorch, when present,
supplies the CUDA stream and the caching device allocator.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from . import build as _build

MAX_THETA = 64

OK = 0
ERRORS = {
    -1: "SPH_ERR_ARG", -2: "SPH_ERR_CUDA", -3: "SPH_ERR_CAPACITY", -4: "SPH_ERR_NONFINITE",
    -5: "SPH_ERR_TIMEOUT", -6: "SPH_ERR_OVERLAP", -7: "SPH_ERR_STATE", -8: "SPH_ERR_ALLOC",
}
PREC = {"fp64": 0, "fp32": 1}
DT = {"dual": 0, "single": 1, "fixed": 2}

F_POS, F_VEL, F_RHO, F_MASS, F_DRHO, F_P, F_K, F_EPS, F_NUT = (1 << i for i in range(9))
F_LABEL, F_UID, F_B, F_ACC_NU, F_INST, F_KEY = (1 << i for i in range(9, 15))
FIELDS = {  # name -> (bit, dtype, width)
    "pos": (F_POS, np.float64, 3), "vel": (F_VEL, np.float64, 3), "rho": (F_RHO, np.float64, 1),
    "mass": (F_MASS, np.float64, 1), "drho": (F_DRHO, np.float64, 1), "p": (F_P, np.float64, 1),
    "k": (F_K, np.float64, 1), "eps": (F_EPS, np.float64, 1), "nut": (F_NUT, np.float64, 1),
    "label": (F_LABEL, np.int32, 1), "uid": (F_UID, np.uint32, 1), "B": (F_B, np.float64, 9),
    "acc_nu": (F_ACC_NU, np.float64, 3), "inst": (F_INST, np.int32, 1), "key": (F_KEY, np.int64, 1),
}
WRITABLE = ("pos", "vel", "rho", "mass", "drho", "k", "eps")


class SphError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} {detail}".strip())


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("rans", C.c_int32), ("precision", C.c_int32), ("dt_mode", C.c_int32),
        ("n_ac_fixed", C.c_int32), ("kinematic", C.c_int32), ("periodic", C.c_int32 * 3),
        ("seed", C.c_uint32), ("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double),
        ("c0", C.c_double), ("nu_l", C.c_double), ("eta", C.c_double), ("U_ref", C.c_double),
        ("dt_ad_fixed", C.c_double), ("gravity", C.c_double * 3), ("domain_lo", C.c_double * 3),
        ("domain_hi", C.c_double * 3), ("obc", C.c_int32), ("density_sum", C.c_int32),
        ("tvf_alpha", C.c_double), ("wall_function", C.c_int32), ("tvf_pbuf", C.c_int32),
    ]


OBC = {"improved": 0, "vipo": 1, "vipo_rkgc": 2, "vipo_rkgc_mirror": 3, "minimal_mirror": 4}


class Particles(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("nw", C.c_int64), ("capacity", C.c_int64), ("on_device", C.c_int32),
        ("reserved", C.c_int32), ("pos", C.c_void_p), ("vel", C.c_void_p), ("rho", C.c_void_p),
        ("mass", C.c_void_p), ("k", C.c_void_p), ("eps", C.c_void_p), ("uid", C.c_void_p),
        ("wall_pos", C.c_void_p), ("wall_vel", C.c_void_p),
    ]


class BufferDesc(C.Structure):
    _fields_ = [
        ("type", C.c_int32), ("turb_bc", C.c_int32), ("n_theta", C.c_int32), ("reserved", C.c_int32),
        ("origin", C.c_double * 3), ("frame", C.c_double * 9), ("length", C.c_double),
        ("half", C.c_double * 2), ("p_ob", C.c_double), ("noise", C.c_double),
        ("k_in", C.c_double), ("eps_in", C.c_double), ("theta", C.c_double * MAX_THETA),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class AdjointDesc(C.Structure):
    _fields_ = [("instance", C.c_int32), ("profile_buffer", C.c_int32), ("steps", C.c_int32),
                ("checkpoint_every", C.c_int32), ("n_outlets", C.c_int32), ("outlets", C.c_int32 * 16),
                ("n_theta", C.c_int32), ("slab", C.c_double), ("theta", C.c_double * 64)]


class Alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p), ("stream", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("step", C.c_int64), ("t", C.c_double), ("dt_ad", C.c_double),
        ("dt_ac", C.c_double), ("n_ac", C.c_int32), ("n_instances", C.c_int32),
        ("spawned", C.c_int64), ("deleted", C.c_int64), ("capacity", C.c_int64),
        ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64), ("status", C.c_int32),
        ("reserved", C.c_int32),
    ]


_lib = None

EXPORTS = ("sph_create", "sph_add_buffer", "sph_set_profile", "sph_step", "sph_read_fields",
           "sph_write_fields", "sph_get_stats", "sph_debug_pairs", "sph_debug_list", "sph_destroy", "sph_error_string",
           "sph_last_error", "sph_abi_version", "sph_set_profiling", "sph_get_stage_times", "sph_stage_name",
           "sph_cell_sort_noalloc", "sph_set_graph", "sph_set_launch", "sph_get_launch", "sph_autotune",
           "sph_save_state", "sph_restore_state", "sph_drop_state", "sph_adjoint_forward",
           "sph_adjoint_backward", "sph_adjoint_release", "sph_debug_convert", "sph_step_async",
           "sph_reduce_mass_momentum", "sph_reduce_mass_momentum_async", "sph_measure_fma_peak",
           "sph_debug_barrier_timeout")
NOALLOC_MAX_POINTS = 1 << 19
N_STAGES = 10


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the built library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.sph_create.argtypes = [C.POINTER(Config), C.c_int32, C.POINTER(Particles), C.POINTER(Alloc),
                                 C.POINTER(vp)]
        L.sph_add_buffer.argtypes = [vp, C.c_int32, C.POINTER(BufferDesc), C.POINTER(C.c_int32)]
        L.sph_set_profile.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_int32]
        L.sph_step.argtypes = [vp, C.c_int32, C.POINTER(C.c_double)]
        L.sph_step_async.argtypes = [vp, C.c_int32]
        L.sph_reduce_mass_momentum.argtypes = [vp, vp, vp]
        L.sph_reduce_mass_momentum_async.argtypes = [vp, vp]
        L.sph_read_fields.argtypes = [vp, C.c_uint32, C.POINTER(vp), C.c_int32, C.POINTER(C.c_int64)]
        L.sph_write_fields.argtypes = [vp, C.c_uint32, C.POINTER(vp), C.c_int32, C.c_int64]
        L.sph_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.sph_debug_pairs.argtypes = [vp, C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64)]
        L.sph_debug_list.argtypes = [vp, C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64)]
        L.sph_debug_convert.argtypes = [vp, vp, vp, vp, C.c_int64]
        L.sph_destroy.argtypes = [vp]
        L.sph_destroy.restype = None
        L.sph_set_profiling.argtypes = [vp, C.c_int32]
        L.sph_get_stage_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32,
                                          C.POINTER(C.c_int32)]
        L.sph_stage_name.restype = C.c_char_p
        L.sph_cell_sort_noalloc.argtypes = [C.POINTER(Config), vp, C.c_int32, vp, vp, C.c_int64,
                                            C.POINTER(C.c_int64), vp]
        L.sph_set_graph.argtypes = [vp, C.c_int32]
        L.sph_set_launch.argtypes = [vp, C.POINTER(C.c_int32)]
        L.sph_get_launch.argtypes = [vp, C.POINTER(C.c_int32)]
        L.sph_autotune.argtypes = [vp, C.c_int32, C.c_char_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.sph_save_state.argtypes = [vp, C.POINTER(C.c_int32)]
        L.sph_restore_state.argtypes = [vp, C.c_int32]
        L.sph_drop_state.argtypes = [vp, C.c_int32]
        L.sph_adjoint_forward.argtypes = [vp, C.POINTER(AdjointDesc), C.POINTER(C.c_double)]
        L.sph_adjoint_backward.argtypes = [vp, C.POINTER(C.c_double), C.c_int32]
        L.sph_adjoint_release.argtypes = [vp]
        L.sph_measure_fma_peak.argtypes = [C.c_int32, C.POINTER(C.c_double)]
        L.sph_debug_barrier_timeout.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_uint32)]
        L.sph_error_string.restype = C.c_char_p
        L.sph_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise SphError(rc, what, lib().sph_last_error().decode(errors="replace"))


def _dptr(a: np.ndarray) -> int:
    return a.ctypes.data


def measure_fma_peak(precision: str = "fp32") -> float:
    """FMA throughput of the current GPU in FLOP/s (sph_measure_fma_peak)."""
    out = C.c_double()
    _check(lib().sph_measure_fma_peak(PREC[precision], C.byref(out)), "sph_measure_fma_peak")
    return out.value


def debug_convert(x64: np.ndarray, x32: np.ndarray):
    """The FP32 form's integer-pipe conversions on the device (test aid):
    returns (x64 rounded to binary32, x32 widened to binary64)."""
    x64 = np.ascontiguousarray(x64, dtype=np.float64)
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    if x64.size != x32.size:
        raise ValueError("x64 and x32 must have the same size")
    o32 = np.empty(x64.size, dtype=np.float32)
    o64 = np.empty(x32.size, dtype=np.float64)
    _check(lib().sph_debug_convert(x64.ctypes.data, o32.ctypes.data, x32.ctypes.data, o64.ctypes.data, x64.size),
           "sph_debug_convert")
    return o32, o64


def make_config(case, precision: str = "fp64", kinematic: bool = False) -> Config:
    c = Config()
    c.dim, c.rans = case.dim, int(bool(case.rans))
    c.precision = PREC[precision]
    c.dt_mode = DT[case.dt_mode]
    c.n_ac_fixed = int(case.n_ac_fixed)
    c.kinematic = int(bool(kinematic))
    for a in range(3):
        c.periodic[a] = int(case.periodic[a])
        c.gravity[a] = float(case.g[a])
        c.domain_lo[a] = float(case.lo[a])
        c.domain_hi[a] = float(case.hi[a])
    c.seed = int(case.seed) & 0xFFFFFFFF
    c.dp, c.h, c.rho0, c.c0, c.nu_l = case.dp, case.h, case.rho0, case.c0, case.nu_l
    c.eta, c.U_ref, c.dt_ad_fixed = case.eta, case.U_ref, case.dt_ad_fixed
    c.obc = OBC[getattr(case, "obc", "improved")]
    c.density_sum = int(bool(getattr(case, "density_sum", False)))
    c.tvf_alpha = float(getattr(case, "tvf", 0.0))
    c.tvf_pbuf = int(bool(getattr(case, "tvf_pbuf", False)))
    c.wall_function = int(bool(getattr(case, "wall_function", False)))
    return c


def make_buffer(spec) -> BufferDesc:
    b = BufferDesc()
    b.type = 0 if spec.kind == "velocity" else 1
    b.turb_bc = 1 if spec.turb == "freestream" else 0
    th = list(spec.theta)
    b.n_theta = len(th)
    for q, v in enumerate(th):
        b.theta[q] = float(v)
    fr = np.asarray(spec.frame, dtype=np.float64).reshape(9)
    for q in range(9):
        b.frame[q] = float(fr[q])
    for q in range(3):
        b.origin[q] = float(spec.origin[q])
    b.length = float(spec.length)
    b.half[0], b.half[1] = float(spec.half[0]), float(spec.half[1])
    b.p_ob, b.noise, b.k_in, b.eps_in = float(spec.p_ob), float(spec.noise), float(spec.k_in), float(spec.eps_in)
    return b


class _TorchAlloc:
    """Device allocator and stream from PyTorch (caching allocator)."""

    def __init__(self):
        import torch

        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream()
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = Alloc(self._alloc, self._free, None, C.c_void_p(self.stream.cuda_stream))

    def _do_alloc(self, user, nbytes, stream):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:
            return 0

    def _do_free(self, user, ptr, stream):
        self.torch.cuda.caching_allocator_delete(int(ptr))


class Simulation:
    """One C-ABI context over one or more instances (cases)."""

    def __init__(self, cases, precision: str = "fp64", kinematic: bool = False,
                 use_torch: bool = True, capacity: Optional[Sequence[int]] = None):
        if not isinstance(cases, (list, tuple)):
            cases = [cases]
        self.cases = list(cases)
        L = lib()
        self._keep = []
        ni = len(cases)
        cfgs = (Config * ni)(*[make_config(c, precision, kinematic) for c in cases])
        parts = (Particles * ni)()
        for i, c in enumerate(cases):
            arrs = {
                "pos": np.ascontiguousarray(c.pos, np.float64), "vel": np.ascontiguousarray(c.vel, np.float64),
                "rho": np.ascontiguousarray(c.rho, np.float64), "mass": np.ascontiguousarray(c.mass, np.float64),
                "k": np.ascontiguousarray(c.k, np.float64), "eps": np.ascontiguousarray(c.eps, np.float64),
                "wpos": np.ascontiguousarray(c.wpos, np.float64).reshape(-1, 3),
                "wvel": np.ascontiguousarray(c.wvel, np.float64).reshape(-1, 3),
            }
            self._keep.append(arrs)
            p = parts[i]
            p.n, p.nw = c.n, arrs["wpos"].shape[0]
            cap = capacity[i] if capacity else (c.capacity or c.n + 16)
            p.capacity = int(cap)
            p.on_device = 0
            p.pos, p.vel, p.rho, p.mass = (_dptr(arrs[k]) for k in ("pos", "vel", "rho", "mass"))
            p.k, p.eps = _dptr(arrs["k"]), _dptr(arrs["eps"])
            p.uid = None
            p.wall_pos = _dptr(arrs["wpos"]) if p.nw else None
            p.wall_vel = _dptr(arrs["wvel"]) if p.nw else None
        self._alloc = None
        alloc_p = None
        if use_torch:
            try:
                import torch

                if torch.cuda.is_available():
                    self._alloc = _TorchAlloc()
                    alloc_p = C.byref(self._alloc.struct)
            except ImportError:
                pass
        ctx = C.c_void_p()
        _check(L.sph_create(cfgs, ni, parts, alloc_p, C.byref(ctx)), "sph_create")
        self.ctx = ctx
        self._keep = None  # inputs were copied in
        for i, c in enumerate(cases):
            for b in c.buffers:
                bid = C.c_int32()
                _check(L.sph_add_buffer(self.ctx, i, C.byref(make_buffer(b)), C.byref(bid)), "sph_add_buffer")

    # ------------------------------------------------------------------
    def step(self, nsteps: int = 1) -> float:
        t = C.c_double()
        _check(lib().sph_step(self.ctx, int(nsteps), C.byref(t)), "sph_step")
        return t.value

    def step_async(self, nsteps: int = 1):
        """Enqueue steps without waiting; stats()["status"] reports device errors."""
        _check(lib().sph_step_async(self.ctx, int(nsteps)), "sph_step_async")

    def mass_momentum(self):
        """FP64 total mass [n_instances] and momentum [n_instances][3]."""
        m = np.zeros(len(self.cases), np.float64)
        p = np.zeros((len(self.cases), 3), np.float64)
        _check(lib().sph_reduce_mass_momentum(self.ctx, m.ctypes.data, p.ctypes.data), "sph_reduce_mass_momentum")
        return m, p

    def mass_momentum_async(self, out):
        """Enqueue the FP64 totals into out (a float64 torch tensor of
        4 * n_instances elements: mass, momentum x y z per instance; on the
        device or in page-locked host memory the reduction writes it
        directly) on the context's stream, without waiting; read out after
        the stream has passed this point (an event recorded after it)."""
        import torch

        if out.dtype != torch.float64 or out.numel() < 4 * len(self.cases) or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of 4 * n_instances elements")
        _check(lib().sph_reduce_mass_momentum_async(self.ctx, out.data_ptr()), "sph_reduce_mass_momentum_async")

    def step_rc(self, nsteps: int = 1) -> int:
        """sph_step's return code (no exception)."""
        return int(lib().sph_step(self.ctx, int(nsteps), None))

    def count(self) -> int:
        n = C.c_int64()
        _check(lib().sph_read_fields(self.ctx, 0, None, 0, C.byref(n)), "sph_read_fields")
        return n.value

    def read(self, names: Iterable[str] = ("pos", "vel", "rho", "uid")) -> Dict[str, np.ndarray]:
        names = sorted(set(names), key=lambda k: FIELDS[k][0])
        n = self.count()
        mask = 0
        outs = []
        for k in names:
            bit, dt, w = FIELDS[k]
            mask |= bit
            outs.append(np.zeros((n, w) if w > 1 else (n,), dtype=dt))
        ptrs = (C.c_void_p * max(len(outs), 1))(*[o.ctypes.data for o in outs])
        n2 = C.c_int64()
        _check(lib().sph_read_fields(self.ctx, mask, ptrs, 0, C.byref(n2)), "sph_read_fields")
        assert n2.value == n
        return dict(zip(names, outs))

    def read_device(self, names, tensors) -> int:
        """Read into device tensors (torch) in field-bit order; returns rows."""
        names = sorted(set(names), key=lambda k: FIELDS[k][0])
        mask = 0
        for k in names:
            mask |= FIELDS[k][0]
        ptrs = (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
        n = C.c_int64()
        _check(lib().sph_read_fields(self.ctx, mask, ptrs, 1, C.byref(n)), "sph_read_fields")
        return n.value

    def write(self, fields: Dict[str, np.ndarray]):
        names = sorted(fields, key=lambda k: FIELDS[k][0])
        mask = 0
        arrs = []
        for k in names:
            if k not in WRITABLE:
                raise ValueError(f"{k} is not writable")
            mask |= FIELDS[k][0]
            w = FIELDS[k][2]
            a = np.ascontiguousarray(fields[k], np.float64)
            arrs.append(a.reshape(-1, w) if w > 1 else a.reshape(-1))
        n = arrs[0].shape[0]
        ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        _check(lib().sph_write_fields(self.ctx, mask, ptrs, 0, n), "sph_write_fields")

    def write_device(self, names, tensors, n: int):
        names = sorted(set(names), key=lambda k: FIELDS[k][0])
        mask = 0
        for k in names:
            mask |= FIELDS[k][0]
        ptrs = (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
        _check(lib().sph_write_fields(self.ctx, mask, ptrs, 1, int(n)), "sph_write_fields")

    def stats(self) -> Dict[str, float]:
        s = Stats()
        _check(lib().sph_get_stats(self.ctx, C.byref(s)), "sph_get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def set_profiling(self, enable: int):
        _check(lib().sph_set_profiling(self.ctx, int(enable)), "sph_set_profiling")

    def stage_times(self) -> Dict[str, tuple]:
        ms = (C.c_double * N_STAGES)()
        cnt = (C.c_int64 * N_STAGES)()
        n = C.c_int32()
        _check(lib().sph_get_stage_times(self.ctx, ms, cnt, N_STAGES, C.byref(n)), "sph_get_stage_times")
        return {lib().sph_stage_name(s).decode(): (ms[s], cnt[s]) for s in range(n.value)}

    def set_profile(self, instance: int, buffer_id: int, theta):
        th = np.ascontiguousarray(theta, np.float64)
        _check(lib().sph_set_profile(self.ctx, instance, buffer_id, th.ctypes.data_as(C.POINTER(C.c_double)),
                                     th.size), "sph_set_profile")

    def set_graph(self, enable: bool = True):
        _check(lib().sph_set_graph(self.ctx, int(bool(enable))), "sph_set_graph")

    def set_launch(self, blocks: Sequence[int]):
        b = (C.c_int32 * 4)(*[int(x) for x in blocks])
        _check(lib().sph_set_launch(self.ctx, b), "sph_set_launch")

    def get_launch(self) -> List[int]:
        b = (C.c_int32 * 4)()
        _check(lib().sph_get_launch(self.ctx, b), "sph_get_launch")
        return list(b)

    def autotune(self, steps: int = 3, cache_path: Optional[str] = None):
        """Pick the sweep block sizes (list, advection, momentum, continuity);
        returns (blocks, from_cache).  The simulation state is unchanged."""
        b = (C.c_int32 * 4)()
        hit = C.c_int32()
        path = cache_path.encode() if cache_path else None
        _check(lib().sph_autotune(self.ctx, int(steps), path, b, C.byref(hit)), "sph_autotune")
        return list(b), bool(hit.value)

    def save_state(self) -> int:
        slot = C.c_int32()
        _check(lib().sph_save_state(self.ctx, C.byref(slot)), "sph_save_state")
        return slot.value

    def restore_state(self, slot: int):
        _check(lib().sph_restore_state(self.ctx, int(slot)), "sph_restore_state")

    def drop_state(self, slot: int):
        _check(lib().sph_drop_state(self.ctx, int(slot)), "sph_drop_state")

    def adjoint_forward(self, theta, instance: int, profile_buffer: int, outlets: Sequence[int], steps: int,
                        checkpoint_every: int, slab: float) -> float:
        """Run a differentiated window (C ABI sph_adjoint_forward); returns J."""
        th = np.ascontiguousarray(theta, np.float64).reshape(-1)
        d = AdjointDesc()
        d.instance, d.profile_buffer, d.steps, d.checkpoint_every = instance, profile_buffer, steps, checkpoint_every
        d.n_outlets = len(outlets)
        for q, b in enumerate(outlets):
            d.outlets[q] = int(b)
        d.n_theta = th.size
        d.slab = float(slab)
        for q, v in enumerate(th):
            d.theta[q] = float(v)
        J = C.c_double()
        _check(lib().sph_adjoint_forward(self.ctx, C.byref(d), C.byref(J)), "sph_adjoint_forward")
        self._adj_n = th.size
        return J.value

    def adjoint_backward(self) -> np.ndarray:
        g = np.zeros(self._adj_n, np.float64)
        _check(lib().sph_adjoint_backward(self.ctx, g.ctypes.data_as(C.POINTER(C.c_double)), g.size),
               "sph_adjoint_backward")
        return g

    def adjoint_release(self):
        _check(lib().sph_adjoint_release(self.ctx), "sph_adjoint_release")

    def _debug_rows(self, fn, name: str, max_rows: Optional[int]) -> np.ndarray:
        cnt = C.c_int64()
        if max_rows is None:
            _check(fn(self.ctx, None, 0, C.byref(cnt)), name)
            max_rows = cnt.value
        out = np.zeros((max(max_rows, 1), 4), np.int64)
        _check(fn(self.ctx, out.ctypes.data_as(C.POINTER(C.c_int64)), max_rows, C.byref(cnt)), name)
        return out[: min(cnt.value, max_rows)]

    def debug_barrier_timeout(self):
        """(status, barrier words after) of a cooperative launch whose grid
        barrier can never complete (sph_debug_barrier_timeout)."""
        st = C.c_int32()
        words = (C.c_uint32 * 4)()
        _check(lib().sph_debug_barrier_timeout(self.ctx, C.byref(st), words), "sph_debug_barrier_timeout")
        return int(st.value), [int(w) for w in words]

    def debug_pairs(self, max_pairs: Optional[int] = None) -> np.ndarray:
        """(uid_i, uid_j | wall index, is_wall, instance) of the FP64 pair test."""
        return self._debug_rows(lib().sph_debug_pairs, "sph_debug_pairs", max_pairs)

    def debug_list(self, max_rows: Optional[int] = None) -> np.ndarray:
        """The same rows read from the neighbour list the sweeps walk."""
        return self._debug_rows(lib().sph_debug_list, "sph_debug_list", max_rows)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
