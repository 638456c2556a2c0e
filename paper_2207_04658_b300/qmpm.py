"""Thin Python binding of ``libqmpm.so`` (the C ABI in ``include/qmpm.h``).

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels.  The functions keep the C names (``qmpm_init``, ``qmpm_step``, ...); ``Scene``
wraps a handle.  Loading fails loudly if the library is missing: there is no CPU
fallback.  PyTorch is used only for device buffers and streams.
"""
import ctypes as ct
import os

import numpy as np

from . import scenes as _scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqmpm.so")

MAX_COMP = 24
MATERIALS = {"neohookean": 0, "corotated": 1, "fluid": 2}
FLAG_STATS, FLAG_STRICT, FLAG_PROFILE, FLAG_SPECIALIZE = 1, 2, 4, 8
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "SCHEME", -4: "CUDA", -5: "TIMEOUT",
          -6: "OVERFLOW", -7: "QUEUE_FULL"}
ERR_INVALID_ARG, ERR_OOM, ERR_SCHEME, ERR_CUDA, ERR_TIMEOUT, ERR_OVERFLOW, ERR_QUEUE_FULL = -1, -2, -3, -4, -5, -6, -7
FAULT_DEVICE_ALLOC, FAULT_HOST_ALLOC, FAULT_WAIT = 0, 1, 2


class QmpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qmpm error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class qmpm_scene_t(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("material", ct.c_int32), ("grid_log2", ct.c_int32),
                ("bound", ct.c_int32), ("n_particles", ct.c_int64), ("dt", ct.c_double),
                ("E", ct.c_double), ("nu", ct.c_double), ("bulk", ct.c_double),
                ("p_vol", ct.c_double), ("p_mass", ct.c_double), ("gravity", ct.c_double * 3),
                ("seed", ct.c_uint64), ("dither", ct.c_int32), ("resort_every", ct.c_int32),
                ("chunk", ct.c_int32), ("flags", ct.c_int32)]


class qmpm_field_t(ct.Structure):
    _fields_ = [("bits", ct.c_int32), ("frac", ct.c_int32), ("offset", ct.c_int64),
                ("container", ct.c_int32)]


class qmpm_scheme_t(ct.Structure):
    _fields_ = [("quantized", ct.c_int32), ("field", qmpm_field_t * 4), ("n_words", ct.c_int32),
                ("bitpos", ct.c_int32 * MAX_COMP)]


class qmpm_stats_t(ct.Structure):
    _fields_ = [("saturations", ct.c_int64 * 4), ("round_ups", ct.c_int64 * 4),
                ("round_downs", ct.c_int64 * 4), ("out_of_grid", ct.c_int64),
                ("out_of_tile", ct.c_int64), ("steps", ct.c_int64), ("active_blocks", ct.c_int64),
                ("error_word", ct.c_int32), ("n_words", ct.c_int32)]

    def as_dict(self):
        return {"saturations": list(self.saturations), "round_ups": list(self.round_ups),
                "round_downs": list(self.round_downs), "out_of_grid": self.out_of_grid,
                "out_of_tile": self.out_of_tile, "steps": self.steps,
                "active_blocks": self.active_blocks, "error_word": self.error_word,
                "n_words": self.n_words}


class qmpm_profile_t(ct.Structure):
    _fields_ = [("step_ms", ct.c_double), ("step_launches", ct.c_int64), ("clear_ms", ct.c_double),
                ("clear_launches", ct.c_int64), ("sort_ms", ct.c_double), ("sort_calls", ct.c_int64),
                ("p2g_ms", ct.c_double), ("p2g_launches", ct.c_int64),
                ("kernel_launches", ct.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qmpm_solve_in_t(ct.Structure):
    _fields_ = [("H", ct.c_int32), ("P", ct.c_double * 8), ("g", ct.c_double * 8),
                ("lo", ct.c_double * 8), ("hi", ct.c_double * 8), ("kappa", ct.c_double),
                ("z", ct.c_double), ("eps", ct.c_double), ("mode", ct.c_int32),
                ("rounding", ct.c_int32), ("max_bits", ct.c_int32), ("refine", ct.c_int32),
                ("beta", ct.c_double * 8), ("margin_gain", ct.c_double * 8), ("margin_src", ct.c_int32 * 8)]


class qmpm_solve_out_t(ct.Structure):
    _fields_ = [("delta_cont", ct.c_double * 8), ("bits_paper", ct.c_int32 * 8),
                ("bits", ct.c_int32 * 8), ("frac", ct.c_int32 * 8), ("offset", ct.c_int64 * 8),
                ("pred_err", ct.c_double), ("total_bits", ct.c_double), ("pred_bias", ct.c_double),
                ("pred_var_dither", ct.c_double), ("capped", ct.c_int32), ("refined", ct.c_int32)]


class qmpm_adjoint_out_t(ct.Structure):
    _fields_ = [("z", ct.c_double), ("g", ct.c_double * 4), ("lo", ct.c_double * 4),
                ("hi", ct.c_double * 4), ("P", ct.c_int64 * 4), ("forward_steps", ct.c_int64),
                ("state_buffers", ct.c_int32), ("pad", ct.c_int32)]

    def as_dict(self):
        return {"z": self.z, "g": list(self.g), "lo": list(self.lo), "hi": list(self.hi),
                "P": list(self.P), "forward_steps": self.forward_steps,
                "state_buffers": self.state_buffers}


class qmpm_noise_out_t(ct.Structure):
    _fields_ = [("z0", ct.c_double), ("shift", ct.c_double), ("shift_se", ct.c_double), ("spread", ct.c_double),
                ("spread_se", ct.c_double), ("pairs", ct.c_int32), ("pad", ct.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class qmpm_rev_op_t(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("from_", ct.c_int32), ("to", ct.c_int32), ("t0", ct.c_int32),
                ("t1", ct.c_int32)]


CKPT_BISECTION = 0
ADJ_QUANTIZED_FORWARD = 0x100
OP_ADVANCE, OP_REVERSE = 0, 1


MEASURE_MEAN_SQ_POS, MEASURE_USER, MEASURE_KINETIC_ENERGY, MEASURE_POSITIONS = 0, 1, 2, 3
NOISE_MATCHED = 0x200
BATCH_GRAPHS = 1
SUBMIT_KEEP_STATE, SUBMIT_BORROW = 1, 2
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class qmpm_batch_info_t(ct.Structure):
    _fields_ = [("n_members", ct.c_int32), ("n_classes", ct.c_int32), ("resort_every", ct.c_int32),
                ("n_solo", ct.c_int32), ("particles", ct.c_int64), ("steps", ct.c_int64),
                ("kernel_launches", ct.c_int64), ("graph_launches", ct.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class qmpm_tune_t(ct.Structure):
    _fields_ = [("chunk", ct.c_int32), ("resort_every", ct.c_int32), ("best_ms_per_step", ct.c_double),
                ("n_candidates", ct.c_int32), ("from_cache", ct.c_int32),
                ("chunk_cand", ct.c_int32 * 16), ("resort_cand", ct.c_int32 * 16),
                ("ms_per_step", ct.c_double * 16)]

    def as_dict(self):
        n = self.n_candidates
        return {"chunk": self.chunk, "resort_every": self.resort_every,
                "best_ms_per_step": self.best_ms_per_step, "from_cache": bool(self.from_cache),
                "candidates": [(self.chunk_cand[i], self.resort_cand[i], self.ms_per_step[i])
                               for i in range(n)]}


class qmpm_engine_config_t(ct.Structure):
    _fields_ = [("budget_bytes", ct.c_int64), ("resort_every", ct.c_int32), ("max_active", ct.c_int32),
                ("flags", ct.c_int32), ("max_queued", ct.c_int32)]


class qmpm_request_t(ct.Structure):
    _fields_ = [("id", ct.c_int64), ("status", ct.c_int32), ("error", ct.c_int32), ("steps", ct.c_int32),
                ("pad", ct.c_int32), ("particles", ct.c_int64), ("resident_bytes", ct.c_int64),
                ("t_submit", ct.c_double), ("t_admit", ct.c_double), ("t_done", ct.c_double),
                ("z", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class qmpm_engine_stats_t(ct.Structure):
    _fields_ = [("queued", ct.c_int64), ("active", ct.c_int64), ("finished", ct.c_int64),
                ("bytes_in_use", ct.c_int64), ("particle_steps", ct.c_int64), ("iterations", ct.c_int64),
                ("kernel_launches", ct.c_int64), ("graph_launches", ct.c_int64), ("elapsed", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

_lib = None

# (name, restype, argtypes) of every entry point declared in include/qmpm.h
class qmpm_smoke_config_t(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("jacobi", ct.c_int32), ("dt", ct.c_float), ("buoyancy", ct.c_float),
                ("v_in", ct.c_float), ("src", ct.c_double * 4), ("dither", ct.c_int32), ("flags", ct.c_int32)]


class qmpm_smoke_scheme_t(ct.Structure):
    _fields_ = [("bits", ct.c_int32 * 2), ("frac", ct.c_int32 * 2), ("offset", ct.c_int64 * 2)]


class qmpm_smoke_info_t(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("jacobi", ct.c_int32), ("n_scenes", ct.c_int32), ("quantized", ct.c_int32),
                ("steps", ct.c_int64), ("state_bytes", ct.c_int64), ("state_bytes_fp32", ct.c_int64),
                ("device_bytes", ct.c_int64), ("kernel_launches", ct.c_int64), ("graph_launches", ct.c_int64),
                ("launches_per_step", ct.c_int32), ("pad", ct.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_P = ct.POINTER
_SIGNATURES = [
    ("qmpm_scheme_layout", ct.c_int, [ct.c_int32, ct.c_int32, _P(qmpm_scheme_t)]),
    ("qmpm_scheme_solve", ct.c_int, [_P(qmpm_solve_in_t), _P(qmpm_solve_out_t)]),
    ("qmpm_init", ct.c_int, [_P(qmpm_scene_t), _P(qmpm_scheme_t), _P(ct.c_double), ct.c_void_p,
                             _P(ct.c_void_p)]),
    ("qmpm_step", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("qmpm_readback", ct.c_int, [ct.c_void_p, _P(ct.c_double), _P(ct.c_uint32), _P(ct.c_int64),
                                 _P(qmpm_stats_t)]),
    ("qmpm_measure", ct.c_int, [ct.c_void_p, _P(ct.c_double)]),
    ("qmpm_step_host", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p]),
    ("qmpm_step_host_stream", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32]),
    ("qmpm_scheme_shift", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32]),
    ("qmpm_scheme_widen", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("qmpm_scheme_window", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_double, ct.c_double, ct.c_double,
                                      ct.c_int32, ct.c_double, ct.c_int32]),
    ("qmpm_scheme_fill_words", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32,
                                          ct.POINTER(ct.c_int32)]),
    ("qmpm_specialize_compile", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_int32,
                                           ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]),
    ("qmpm_step_kernel_info", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_double)]),
    ("qmpm_profile", ct.c_int, [ct.c_void_p, _P(qmpm_profile_t), ct.c_int32]),
    ("qmpm_state_device", ct.c_int, [ct.c_void_p, _P(ct.c_void_p), _P(ct.c_int64),
                                     _P(ct.c_void_p)]),
    ("qmpm_destroy", ct.c_int, [ct.c_void_p]),
    ("qmpm_last_error", ct.c_char_p, []),
    ("qmpm_adjoint", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                                ct.c_void_p, _P(qmpm_adjoint_out_t)]),
    ("qmpm_noise_moments", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, _P(ct.c_double), ct.c_uint64,
                                      ct.c_int32, _P(qmpm_noise_out_t)]),
    ("qmpm_footprint", ct.c_int, [_P(qmpm_scene_t), _P(qmpm_scheme_t), _P(ct.c_int64), _P(ct.c_int64)]),
    ("qmpm_bisection_schedule", ct.c_int, [ct.c_int32, _P(qmpm_rev_op_t), ct.c_int64, _P(ct.c_int64),
                                           _P(ct.c_int32)]),
    ("qmpm_batch_create", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, _P(ct.c_void_p)]),
    ("qmpm_batch_add", ct.c_int, [ct.c_void_p, ct.c_void_p]),
    ("qmpm_batch_remove", ct.c_int, [ct.c_void_p, ct.c_void_p]),
    ("qmpm_batch_step", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("qmpm_batch_info", ct.c_int, [ct.c_void_p, _P(qmpm_batch_info_t)]),
    ("qmpm_batch_destroy", ct.c_int, [ct.c_void_p]),
    ("qmpm_autotune", ct.c_int, [_P(qmpm_scene_t), _P(qmpm_scheme_t), _P(ct.c_double), ct.c_int32, ct.c_int32,
                                 _P(qmpm_tune_t)]),
    ("qmpm_engine_create", ct.c_int, [_P(qmpm_engine_config_t), _P(ct.c_void_p)]),
    ("qmpm_engine_submit", ct.c_int, [ct.c_void_p, _P(qmpm_scene_t), _P(qmpm_scheme_t), _P(ct.c_double),
                                      ct.c_int32, ct.c_int32, _P(ct.c_int64)]),
    ("qmpm_engine_start", ct.c_int, [ct.c_void_p]),
    ("qmpm_engine_stop", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("qmpm_engine_run", ct.c_int, [ct.c_void_p, ct.c_int32, _P(ct.c_int32)]),
    ("qmpm_engine_wait", ct.c_int, [ct.c_void_p, ct.c_double, _P(ct.c_int32)]),
    ("qmpm_fault_inject", ct.c_int, [ct.c_int32, ct.c_int64, ct.c_int64]),
    ("qmpm_fault_hits", ct.c_int, [ct.c_int32, _P(ct.c_int64)]),
    ("qmpm_fault_clear", ct.c_int, []),
    ("qmpm_engine_poll", ct.c_int, [ct.c_void_p, _P(qmpm_request_t), ct.c_int32, _P(ct.c_int32)]),
    ("qmpm_engine_result", ct.c_int, [ct.c_void_p, ct.c_int64, _P(ct.c_double), _P(ct.c_int64)]),
    ("qmpm_engine_release", ct.c_int, [ct.c_void_p, ct.c_int64]),
    ("qmpm_engine_stats", ct.c_int, [ct.c_void_p, _P(qmpm_engine_stats_t)]),
    ("qmpm_engine_destroy", ct.c_int, [ct.c_void_p]),
    ("qmpm_pack_f32", ct.c_int, [ct.c_int32, ct.c_int32, _P(qmpm_scheme_t), ct.c_uint64, ct.c_int32,
                                 ct.c_uint32, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int64,
                                 _P(qmpm_stats_t), ct.c_void_p]),
    ("qmpm_unpack_f32", ct.c_int, [ct.c_int32, ct.c_int32, _P(qmpm_scheme_t), ct.c_void_p,
                                   ct.c_int64, ct.c_int64, ct.c_void_p, ct.c_void_p]),
]
_SIGNATURES += [
    ("qmpm_smoke_create", ct.c_int, [_P(qmpm_smoke_config_t), _P(qmpm_smoke_scheme_t), ct.c_int32,
                                     _P(ct.c_uint64), ct.c_void_p, _P(ct.c_void_p)]),
    ("qmpm_smoke_set_state", ct.c_int, [ct.c_void_p, ct.c_int32, _P(ct.c_float), _P(ct.c_float), _P(ct.c_float)]),
    ("qmpm_smoke_set_states", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    ("qmpm_smoke_get_states", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    ("qmpm_smoke_set_noise", ct.c_int, [ct.c_void_p, _P(ct.c_float), _P(ct.c_uint64), _P(ct.c_float)]),
    ("qmpm_smoke_step", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int64]),
    ("qmpm_smoke_measure", ct.c_int, [ct.c_void_p, _P(ct.c_double)]),
    ("qmpm_smoke_readback", ct.c_int, [ct.c_void_p, ct.c_int32, _P(ct.c_float), _P(ct.c_float), _P(ct.c_float),
                                       _P(ct.c_float)]),
    ("qmpm_smoke_ranges", ct.c_int, [ct.c_void_p, _P(ct.c_float), _P(ct.c_float), _P(ct.c_int64)]),
    ("qmpm_smoke_info", ct.c_int, [ct.c_void_p, _P(qmpm_smoke_info_t)]),
    ("qmpm_smoke_profile", ct.c_int, [ct.c_void_p, _P(ct.c_double), _P(ct.c_double), _P(ct.c_int64)]),
    ("qmpm_smoke_stage", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_uint32] + [_P(ct.c_float)] * 6
     + [_P(ct.c_uint32)]),
    ("qmpm_smoke_destroy", ct.c_int, [ct.c_void_p]),
]
OPTIONAL_SIGNATURES = [
    ("qmpm_tile_order_static", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, _P(qmpm_scheme_t),
                                          ct.c_void_p, ct.c_int64, ct.c_int64, ct.c_void_p,
                                          ct.c_void_p]),
]
STATIC_SORT_MAX = 262144


def lib():
    """Load libqmpm.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2207_04658_b300.build`")
        L = ct.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES + OPTIONAL_SIGNATURES:
            if not hasattr(L, name):
                continue
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise QmpmError(rc, lib().qmpm_last_error().decode())
    return rc


def _dptr(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


# ---------------------------------------------------------------------------- structs
def make_scene_struct(scene, n_particles, flags=0):
    s = qmpm_scene_t()
    s.dim = scene["dim"]
    s.material = MATERIALS[scene["material"]]
    s.grid_log2 = scene["grid_log2"]
    s.bound = scene.get("bound", 3)
    s.n_particles = int(n_particles)
    s.dt = scene["dt"]
    s.E = scene.get("E", 0.0)
    s.nu = scene.get("nu", 0.0)
    s.bulk = scene.get("bulk", 0.0)
    s.p_vol = scene["p_vol"]
    s.p_mass = scene["p_vol"] * scene.get("rho", 1.0)
    g = list(scene.get("gravity", (0.0, -9.8, 0.0))) + [0.0, 0.0, 0.0]
    for a in range(3):
        s.gravity[a] = g[a]
    s.seed = int(scene.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    s.dither = int(bool(scene.get("dither", True)))
    s.resort_every = int(scene.get("resort_every", 8))
    s.chunk = int(scene.get("chunk", 0))
    s.flags = int(flags)
    return s


FIELD_NAMES = ("x", "v", "C", "F")


def make_scheme_struct(scheme, dim=None, material=None):
    """Per-field scheme {"x": {bits, frac, offset, container}, "v", "C", "F" or "J"}; None
    gives the FP32 state.  The layout is filled in when dim and material are given."""
    sch = qmpm_scheme_t()
    if scheme is None:
        sch.quantized = 0
    else:
        sch.quantized = 1
        for h, name in enumerate(FIELD_NAMES):
            f = scheme[name] if name in scheme else scheme["J"]
            sch.field[h].bits = int(f["bits"])
            sch.field[h].frac = int(f["frac"])
            sch.field[h].offset = int(f["offset"])
            sch.field[h].container = int(f.get("container", 0))
    if dim is not None:
        qmpm_scheme_layout(dim, MATERIALS[material], sch)
    return sch


# ---------------------------------------------------------------------------- C names
def qmpm_scheme_layout(dim, material, scheme_struct):
    _check(lib().qmpm_scheme_layout(dim, material, ct.byref(scheme_struct)))
    return scheme_struct


def qmpm_scheme_solve(P, g, lo, hi, z, eps, mode="error", rounding="paper", kappa=2.0, max_bits=0, beta=None,
                      margins=None):
    """The bit-allocation solve (Eq. 10 / Algorithm 1 or the memory-bound form) with its
    options: max_bits caps a type's bits (window kept, resolution coarser); beta (one per
    type) turns on the second-order refinement; margins = {h: (src, gain)} widens type h's
    window by gain times the resolution of type src."""
    si = qmpm_solve_in_t()
    si.H = len(P)
    for h in range(len(P)):
        si.P[h], si.g[h], si.lo[h], si.hi[h] = P[h], g[h], lo[h], hi[h]
    si.kappa, si.z, si.eps = kappa, z, eps
    si.mode = 0 if mode == "error" else 1
    si.rounding = 0 if rounding == "paper" else 1
    si.max_bits = int(max_bits)
    if beta is not None:
        si.refine = 1
        for h, b in enumerate(beta):
            si.beta[h] = float(b)
    for h, (src, gain) in (margins or {}).items():
        si.margin_src[h], si.margin_gain[h] = int(src), float(gain)
    so = qmpm_solve_out_t()
    _check(lib().qmpm_scheme_solve(ct.byref(si), ct.byref(so)))
    H = len(P)
    return {"delta_cont": list(so.delta_cont)[:H], "bits_paper": list(so.bits_paper)[:H],
            "bits": list(so.bits)[:H], "frac": list(so.frac)[:H],
            "offset": [int(v) for v in so.offset][:H], "pred_err": so.pred_err,
            "total_bits": so.total_bits, "pred_bias": so.pred_bias, "pred_var_dither": so.pred_var_dither,
            "capped_mask": so.capped, "refined": so.refined}


def qmpm_init(scene_struct, scheme_struct, h_state, stream=0):
    h = ct.c_void_p()
    st = np.ascontiguousarray(h_state, dtype=np.float64)
    _check(lib().qmpm_init(ct.byref(scene_struct), ct.byref(scheme_struct), _dptr(st, ct.c_double),
                           ct.c_void_p(stream), ct.byref(h)))
    return h


def qmpm_step(h, nsteps):
    _check(lib().qmpm_step(h, int(nsteps)))


def qmpm_readback(h, h_state=None, h_words=None, h_ids=None, stats=None):
    _check(lib().qmpm_readback(
        h,
        _dptr(h_state, ct.c_double) if h_state is not None else None,
        _dptr(h_words, ct.c_uint32) if h_words is not None else None,
        _dptr(h_ids, ct.c_int64) if h_ids is not None else None,
        ct.byref(stats) if stats is not None else None))


def qmpm_measure(h):
    z = ct.c_double(0.0)
    _check(lib().qmpm_measure(h, ct.byref(z)))
    return z.value


def qmpm_step_host(h, nsteps, h_words_in_ptr, h_words_out_ptr):
    _check(lib().qmpm_step_host(h, int(nsteps), ct.c_void_p(h_words_in_ptr),
                                ct.c_void_p(h_words_out_ptr)))


def qmpm_step_host_stream(h, nsteps, h_words_ptr, chunks=0):
    _check(lib().qmpm_step_host_stream(h, int(nsteps), ct.c_void_p(h_words_ptr), int(chunks)))


def qmpm_specialize_compile(dim, material, scheme, stats=False, dither=True):
    """Compile (or find) the step kernel specialised to this scheme; no device needed.
    Returns (seconds of the first compile, cubin bytes)."""
    sch = make_scheme_struct(scheme)  # None: FP32 state
    sec, nb = ct.c_double(), ct.c_int64()
    _check(lib().qmpm_specialize_compile(int(dim), MATERIALS[material], ct.byref(sch), int(bool(stats)),
                                         int(bool(dither)), ct.byref(sec), ct.byref(nb)))
    return sec.value, nb.value


def qmpm_step_kernel_info(h):
    on, sec = ct.c_int32(), ct.c_double()
    _check(lib().qmpm_step_kernel_info(h, ct.byref(on), ct.byref(sec)))
    return {"specialized": bool(on.value), "compile_seconds": sec.value}


def qmpm_profile(h, reset=True):
    p = qmpm_profile_t()
    _check(lib().qmpm_profile(h, ct.byref(p), int(reset)))
    return p.as_dict()


def qmpm_state_device(h):
    w, ld, ids = ct.c_void_p(), ct.c_int64(), ct.c_void_p()
    _check(lib().qmpm_state_device(h, ct.byref(w), ct.byref(ld), ct.byref(ids)))
    return w.value, ld.value, ids.value


def qmpm_destroy(h):
    _check(lib().qmpm_destroy(h))


def qmpm_pack_f32(dim, material, scheme_struct, seed, dither, step, d_vals_ptr, N, d_words_ptr, ld,
                  stats=None, stream=0):
    _check(lib().qmpm_pack_f32(dim, material, ct.byref(scheme_struct), int(seed) & (2**64 - 1),
                               int(dither), int(step), ct.c_void_p(d_vals_ptr), int(N),
                               ct.c_void_p(d_words_ptr), int(ld),
                               ct.byref(stats) if stats is not None else None, ct.c_void_p(stream)))


def qmpm_unpack_f32(dim, material, scheme_struct, d_words_ptr, N, ld, d_vals_ptr, stream=0):
    _check(lib().qmpm_unpack_f32(dim, material, ct.byref(scheme_struct), ct.c_void_p(d_words_ptr),
                                 int(N), int(ld), ct.c_void_p(d_vals_ptr), ct.c_void_p(stream)))


def qmpm_adjoint(h, T, ckpt_every=32, measure=MEASURE_MEAN_SQ_POS, d_seed_ptr=0, d_grad0_ptr=0):
    out = qmpm_adjoint_out_t()
    _check(lib().qmpm_adjoint(h, int(T), int(ckpt_every), int(measure), ct.c_void_p(d_seed_ptr),
                              ct.c_void_p(d_grad0_ptr), ct.byref(out)))
    return out.as_dict()


def qmpm_noise_moments(h, T, measure, sigma, seed0=1, n_pairs=16):
    sg = (ct.c_double * 4)(*[float(v) for v in sigma])
    out = qmpm_noise_out_t()
    _check(lib().qmpm_noise_moments(h, int(T), int(measure), sg, int(seed0), int(n_pairs), ct.byref(out)))
    return out.as_dict()


def qmpm_tile_order_static(dim, material, scheme_struct, grid_log2, d_words_ptr, N, ld, d_order_ptr,
                           stream=0):
    """The tile order of N packed records without any device allocation (scratch in a
    static device array of the library; N <= STATIC_SORT_MAX)."""
    _check(lib().qmpm_tile_order_static(dim, material, grid_log2,
                                        ct.byref(scheme_struct) if scheme_struct is not None else None,
                                        ct.c_void_p(d_words_ptr), int(N), int(ld),
                                        ct.c_void_p(d_order_ptr), ct.c_void_p(stream)))


def qmpm_fault_inject(kind, after=0, count=1):
    """Arm a host-side fault (FAULT_*): `after` occurrences pass, then `count` fail."""
    _check(lib().qmpm_fault_inject(int(kind), int(after), int(count)))


def qmpm_fault_hits(kind):
    out = ct.c_int64()
    _check(lib().qmpm_fault_hits(int(kind), ct.byref(out)))
    return out.value


def qmpm_fault_clear():
    _check(lib().qmpm_fault_clear())


def qmpm_footprint(scene_struct, scheme_struct):
    r, p = ct.c_int64(), ct.c_int64()
    _check(lib().qmpm_footprint(ct.byref(scene_struct), ct.byref(scheme_struct), ct.byref(r), ct.byref(p)))
    return r.value, p.value


def qmpm_bisection_schedule(T):
    """The bisection reverse schedule over T steps: (ops as (kind, from, to, t0, t1), slots)."""
    n, slots = ct.c_int64(), ct.c_int32()
    _check(lib().qmpm_bisection_schedule(int(T), None, 0, ct.byref(n), ct.byref(slots)))
    buf = (qmpm_rev_op_t * max(1, n.value))()
    _check(lib().qmpm_bisection_schedule(int(T), buf, n.value, ct.byref(n), ct.byref(slots)))
    return [(o.kind, o.from_, o.to, o.t0, o.t1) for o in buf[:n.value]], slots.value


def qmpm_autotune(scene_struct, scheme_struct, h_state, trial_steps=32, use_cache=True):
    st = np.ascontiguousarray(h_state, dtype=np.float64)
    out = qmpm_tune_t()
    _check(lib().qmpm_autotune(ct.byref(scene_struct), ct.byref(scheme_struct), _dptr(st, ct.c_double),
                               int(trial_steps), int(bool(use_cache)), ct.byref(out)))
    return out.as_dict()


# ---------------------------------------------------------------------------- Scene
class Scene:
    """One simulation resident on the device (a qmpm handle)."""

    def __init__(self, scene, scheme, state0, stream=0, stats=False, strict=False, profile=False, specialize=False):
        self.scene = dict(scene)
        self.dim = scene["dim"]
        self.material = scene["material"]
        state0 = np.ascontiguousarray(state0, dtype=np.float64)
        self.N = state0.shape[0]
        self.n_comp = _scenes.n_comp(self.dim, self.material)
        assert state0.shape[1] == self.n_comp
        flags = ((FLAG_STATS if stats else 0) | (FLAG_STRICT if strict else 0)
                 | (FLAG_PROFILE if profile else 0) | (FLAG_SPECIALIZE if specialize else 0))
        self._scene_struct = make_scene_struct(scene, self.N, flags)
        self._scheme_struct = make_scheme_struct(scheme, self.dim, self.material)
        self.quantized = scheme is not None
        self.n_words = self._scheme_struct.n_words
        self.h = qmpm_init(self._scene_struct, self._scheme_struct, state0, stream)

    def step(self, n=1):
        qmpm_step(self.h, n)

    def measure(self):
        return qmpm_measure(self.h)

    def readback(self, state=True, words=False, ids=True):
        out = {}
        hs = np.empty((self.N, self.n_comp)) if state else None
        hw = np.empty((self.n_words, self.N), dtype=np.uint32) if words else None
        hi = np.empty(self.N, dtype=np.int64) if ids else None
        st = qmpm_stats_t()
        qmpm_readback(self.h, hs, hw, hi, st)
        if state:
            out["state"] = hs
        if words:
            out["words"] = hw
        if ids:
            out["ids"] = hi
        out["stats"] = st.as_dict()
        return out

    def state_by_id(self):
        r = self.readback(state=True, ids=True)
        s = np.empty_like(r["state"])
        s[r["ids"]] = r["state"]
        return s

    def profile(self, reset=True):
        return qmpm_profile(self.h, reset)

    def packed_bytes_per_particle(self):
        return 4 * self.n_words

    def close(self):
        if self.h is not None:
            qmpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------- differentiation
def _torch():
    import torch
    return torch


class Rollout:
    """Differentiable FP32 rollout: ``Rollout.apply(state0, scene, T, ckpt_every)`` returns
    the state after T steps (rows in the input particle order).  Forward: qmpm_init and
    qmpm_step on FP32 state; backward: qmpm_adjoint (Sec. 6) with the incoming gradient
    as seed, checkpointing every ``ckpt_every`` steps.  After a backward pass
    ``Rollout.last`` holds the adjoint's z, g_h (Eq. 8), ranges and variable counts."""

    last = None

    @staticmethod
    def _fn():
        torch = _torch()

        class _Rollout(torch.autograd.Function):
            @staticmethod
            def forward(ctx, state0, scene, T, ckpt_every):
                s0 = state0.detach().cpu().double().numpy()
                sc = dict(scene, resort_every=0)
                g = Scene(sc, None, s0)
                g.step(int(T))
                out = g.state_by_id()
                g.close()
                ctx.save_for_backward(state0)
                ctx.scene, ctx.T, ctx.k = sc, int(T), int(ckpt_every)
                return torch.from_numpy(out).to(state0.dtype).to(state0.device)

            @staticmethod
            def backward(ctx, grad_out):
                (state0,) = ctx.saved_tensors
                s0 = state0.detach().cpu().double().numpy()
                g = Scene(ctx.scene, None, s0)
                ids = g.readback(state=False, ids=True)["ids"]
                seed = grad_out.detach().float().cpu().numpy()[ids]  # slot order
                d_seed = torch.from_numpy(np_ascontig(seed)).cuda()
                d_grad = torch.empty_like(d_seed)
                info = qmpm_adjoint(g.h, ctx.T, ctx.k, MEASURE_USER, d_seed.data_ptr(),
                                    d_grad.data_ptr())
                g.close()
                Rollout.last = info
                grad_slot = d_grad.cpu().numpy()
                grad = np.empty_like(grad_slot)
                grad[ids] = grad_slot
                return torch.from_numpy(grad).to(state0.dtype).to(state0.device), None, None, None

        return _Rollout

    @classmethod
    def apply(cls, state0, scene, T, ckpt_every=32):
        return cls._fn().apply(state0, scene, T, ckpt_every)


def np_ascontig(a):
    return np.ascontiguousarray(a, dtype=np.float32)


FIELD_KEYS = ("x", "v", "C", "F")


def sensitivities(scene, state0, T, ckpt_every=32, measure=MEASURE_MEAN_SQ_POS):
    """Algorithm 1's forward and backward pass on FP32 state: z (mean |x_T|^2 or the
    kinetic energy), the accumulated squared gradients g_h (Eq. 8) and the recorded range
    of each field."""
    g = Scene(dict(scene, resort_every=0), None, state0)
    info = qmpm_adjoint(g.h, T, ckpt_every, measure)
    g.close()
    return info


def _type_names(material):
    return ["x", "v", "C", "J" if material == "fluid" else "F"]


def _scheme_dict(st, scheme, material):
    names = _type_names(material)
    return {names[h]: dict(bits=int(st.field[h].bits), frac=int(st.field[h].frac), offset=int(st.field[h].offset),
                           container=int(scheme[names[h]].get("container", 0))) for h in range(4)}


def _type_index(material, t):
    return t if isinstance(t, int) else _type_names(material).index(t)


def scheme_shift(scheme, material, t, k):
    """Type t (name or index) k fraction bits finer (k < 0: coarser) over the same window
    (qmpm_scheme_shift); returns the new scheme dict."""
    st = make_scheme_struct(scheme)
    _check(lib().qmpm_scheme_shift(ct.byref(st), _type_index(material, t), int(k)))
    return _scheme_dict(st, scheme, material)


def scheme_widen(scheme, material, t):
    """Type t's window doubled about its middle at the same resolution (qmpm_scheme_widen)."""
    st = make_scheme_struct(scheme)
    _check(lib().qmpm_scheme_widen(ct.byref(st), _type_index(material, t)))
    return _scheme_dict(st, scheme, material)


def scheme_window(scheme, material, t, lo, hi, kappa=2.0, src=-1, gain=0.0, grow=False):
    """Type t's window from the recorded range [lo, hi] as qmpm_scheme_solve makes it, widened
    by gain x the resolution of type src (qmpm_scheme_window); grow keeps the union."""
    st = make_scheme_struct(scheme)
    _check(lib().qmpm_scheme_window(ct.byref(st), _type_index(material, t), float(lo), float(hi), float(kappa),
                                    _type_index(material, src) if src != -1 else -1, float(gain), int(bool(grow))))
    return _scheme_dict(st, scheme, material)


def scheme_fill_words(scheme, dim, material, types):
    """The last packed word's free bits spent on wider windows of the given types
    (qmpm_scheme_fill_words); returns (scheme dict, number of doublings)."""
    st = make_scheme_struct(scheme)
    mask = 0
    for t in types:
        if t in _type_names(material) or isinstance(t, int):
            mask |= 1 << _type_index(material, t)
    n = ct.c_int32()
    _check(lib().qmpm_scheme_fill_words(int(dim), MATERIALS[material], ct.byref(st), mask, ct.byref(n)))
    return _scheme_dict(st, scheme, material), n.value


def solve_scheme(info, eps, mode="error", rounding="paper", kappa=2.0, containers=(0, 0, 0, 0),
                 material="corotated", max_bits=24, margins=None, beta=None):
    """Scheme from the adjoint's sensitivities (Eq. 10 / Algorithm 1, or the memory-bound
    form): returns the per-field scheme dict consumed by Scene and the solve report.  A
    field the solve gives more than max_bits (the FP32 compute limit) keeps its window at
    max_bits, one power of two coarser per bit dropped; the report lists such fields in
    "capped" (their share of the error bound is then not met).  margins and beta are the
    solve's window-margin and second-order options (qmpm_scheme_solve)."""
    res = qmpm_scheme_solve(info["P"], info["g"], info["lo"], info["hi"], info["z"], eps, mode=mode,
                            rounding=rounding, kappa=kappa, max_bits=max_bits, margins=margins, beta=beta)
    names = ["x", "v", "C", "J" if material == "fluid" else "F"]
    scheme = {names[h]: dict(bits=int(res["bits"][h]), frac=int(res["frac"][h]), offset=int(res["offset"][h]),
                             container=int(containers[h])) for h in range(4)}
    res["capped"] = [names[h] for h in range(4) if res["capped_mask"] >> h & 1]
    return scheme, res


# ---------------------------------------------------------------------------- Batch
class Batch:
    """Several scenes stepped together by multi-scene launches (qmpm_batch_*)."""

    def __init__(self, resort_every=8, graphs=True, stream=0):
        self.h = ct.c_void_p()
        _check(lib().qmpm_batch_create(ct.c_void_p(stream), int(resort_every),
                                       BATCH_GRAPHS if graphs else 0, ct.byref(self.h)))
        self.members = []

    def add(self, scene):
        _check(lib().qmpm_batch_add(self.h, scene.h))
        self.members.append(scene)

    def remove(self, scene):
        _check(lib().qmpm_batch_remove(self.h, scene.h))
        self.members.remove(scene)

    def step(self, n=1):
        _check(lib().qmpm_batch_step(self.h, int(n)))

    def info(self):
        out = qmpm_batch_info_t()
        _check(lib().qmpm_batch_info(self.h, ct.byref(out)))
        return out.as_dict()

    def close(self):
        if self.h is not None:
            _check(lib().qmpm_batch_destroy(self.h))
            self.h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------- Engine
class Engine:
    """The serving loop (qmpm_engine_*): submit scenes, poll finished requests."""

    def __init__(self, budget_bytes=120 * 2 ** 30, resort_every=8, max_active=64, graphs=True, max_queued=0):
        cfg = qmpm_engine_config_t()
        cfg.budget_bytes = int(budget_bytes)
        cfg.resort_every = int(resort_every)
        cfg.max_active = int(max_active)
        cfg.flags = BATCH_GRAPHS if graphs else 0
        cfg.max_queued = int(max_queued)
        self.h = ct.c_void_p()
        self._borrowed = {}
        _check(lib().qmpm_engine_create(ct.byref(cfg), ct.byref(self.h)))

    def submit(self, scene, scheme, state0, steps, keep_state=False, flags=0, borrow=False):
        """Queue a request.  borrow=True lets the engine read state0 at admission instead of
        copying it now; the array is held here until the request has been polled."""
        state0 = np.ascontiguousarray(state0, dtype=np.float64)
        sc = make_scene_struct(scene, state0.shape[0], flags)
        sch = make_scheme_struct(scheme, scene["dim"], scene["material"])
        rid = ct.c_int64()
        sub = (SUBMIT_KEEP_STATE if keep_state else 0) | (SUBMIT_BORROW if borrow else 0)
        _check(lib().qmpm_engine_submit(self.h, ct.byref(sc), ct.byref(sch), _dptr(state0, ct.c_double),
                                        int(steps), sub, ct.byref(rid)))
        if borrow:
            self._borrowed[rid.value] = state0
        return rid.value

    def start(self):
        _check(lib().qmpm_engine_start(self.h))

    def stop(self, drain=True):
        _check(lib().qmpm_engine_stop(self.h, int(bool(drain))))

    def run(self, iterations=1):
        busy = ct.c_int32()
        _check(lib().qmpm_engine_run(self.h, int(iterations), ct.byref(busy)))
        return bool(busy.value)

    def wait(self, timeout_s):
        """Wait (host clock, bounded) until every submitted request has finished; raises
        QmpmError(QMPM_ERR_TIMEOUT) if the deadline passes first."""
        busy = ct.c_int32()
        _check(lib().qmpm_engine_wait(self.h, float(timeout_s), ct.byref(busy)))
        return bool(busy.value)

    def poll(self, max_n=256):
        buf = (qmpm_request_t * max_n)()
        n = ct.c_int32()
        _check(lib().qmpm_engine_poll(self.h, buf, int(max_n), ct.byref(n)))
        out = [buf[i].as_dict() for i in range(n.value)]
        for r in out:
            self._borrowed.pop(r["id"], None)
        return out

    def result(self, rid, N, n_comp):
        st = np.empty((N, n_comp), dtype=np.float64)
        ids = np.empty(N, dtype=np.int64)
        _check(lib().qmpm_engine_result(self.h, int(rid), _dptr(st, ct.c_double), _dptr(ids, ct.c_int64)))
        out = np.empty_like(st)
        out[ids] = st
        return out

    def release(self, rid):
        _check(lib().qmpm_engine_release(self.h, int(rid)))

    def stats(self):
        out = qmpm_engine_stats_t()
        _check(lib().qmpm_engine_stats(self.h, ct.byref(out)))
        return out.as_dict()

    def close(self):
        if self.h is not None:
            _check(lib().qmpm_engine_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
