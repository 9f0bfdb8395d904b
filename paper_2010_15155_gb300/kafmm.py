"""Thin Python binding of the C ABI in include/kafmm.h (argument marshalling only).

Every call forwards to ``libkafmm.so``; all arithmetic runs in the library's CUDA kernels.
There is no CPU path: if the library is missing, :func:`lib` raises.

Arrays may be CUDA tensors (PyTorch), CPU tensors or numpy arrays; their data pointers are
passed through unchanged (the library copies host arrays itself).  The dtype (float32 or
float64) must be the same for points, sources and results of one call.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkafmm.so")

# enums of include/kafmm.h
LAPLACE, STOKESLET, RPY, STOKES_DL, STOKES_REG, LAPLACE_QD, STOKES_PVEL = 0, 1, 2, 3, 4, 5, 6
STOKES_PVEL_GRAD, STOKES_PVEL_LAPL, STOKES_PVEL_TRACTION = 7, 8, 9
STOKES_DL_GRAD, STOKES_DL_LAPL, STOKES_DL_TRACTION = 10, 11, 12
LAPLACE_QUAD = 13
BC_OPEN, BC_PX, BC_PXY, BC_PXYZ, BC_WALL, BC_WALL_PX, BC_WALL_PXY = 0, 1, 2, 3, 4, 5, 6
F32, F64 = 0, 1
OPT_PRECISION, OPT_ML_VARIANT, OPT_STREAM, OPT_NEAR_ONLY, OPT_KAHAN, OPT_TC_SPLIT = 1, 2, 3, 4, 5, 6
OPT_SYNC, OPT_TC_STAGES, OPT_TC_RANGES, OPT_RPY_CONTACT, OPT_TC_TILING = 7, 8, 9, 10, 11
OPT_WAIT_LIMIT_US, OPT_WAIT_REPORT_US, OPT_TEST_STALL, OPT_COMPRESS, OPT_LEAF_STAGE = 12, 13, 14, 15, 16
OPT_TC_TILES = 17
TC_TF32X3, TC_BF16X3, TC_AUTO = 0, 1, 2
PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
ML_G, ML_L4 = 0, 1
KDIM = {LAPLACE: (1, 1), STOKESLET: (3, 3), RPY: (4, 6), STOKES_DL: (9, 4), STOKES_REG: (4, 3), LAPLACE_QD: (4, 10),
        STOKES_PVEL: (4, 4), STOKES_PVEL_GRAD: (4, 16), STOKES_PVEL_LAPL: (4, 7), STOKES_PVEL_TRACTION: (4, 9),
        STOKES_DL_GRAD: (9, 16), STOKES_DL_LAPL: (9, 7), STOKES_DL_TRACTION: (9, 9), LAPLACE_QUAD: (9, 10)}
ERRORS = {-1: "KAFMM_ERR_ARG", -2: "KAFMM_ERR_DOMAIN", -3: "KAFMM_ERR_CUDA",
          -4: "KAFMM_ERR_TIMEOUT", -5: "KAFMM_ERR_NOMEM", -6: "KAFMM_ERR_STATE"}

_lib = None


class KafmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Loads libkafmm.so (built by paper_2010_15155_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_2010_15155_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "kafmm_plan": ([i32, i32, i32, i32, ctypes.POINTER(vp)], i32),
            "kafmm_set_option": ([vp, i32, i64], i32),
            "kafmm_set_domain": ([vp, ctypes.POINTER(dbl), dbl], i32),
            "kafmm_set_points": ([vp, vp, i64, vp, i64, i32], i32),
            "kafmm_set_points_batched": ([vp, i32, vp, vp, vp, vp, i32], i32),
            "kafmm_eval": ([vp, vp, vp, i32], i32),
            "kafmm_status": ([vp], i32),
            "kafmm_autotune": ([vp, vp, vp, i32, ctypes.POINTER(i64)], i32),
            "kafmm_rpy_velocity": ([vp, vp, vp, vp, vp, i32], i32),
            "kafmm_rpy_velocity_noalloc": ([vp, vp, vp, vp, vp, i32], i32),
            "kafmm_tree_info": ([vp, ctypes.POINTER(i64), i32], i32),
            "kafmm_get_tree": ([vp, vp, vp, vp, vp], i32),
            "kafmm_get_list": ([vp, i32, vp, vp, vp], i32),
            "kafmm_phase_times": ([vp, ctypes.POINTER(dbl), i32], i32),
            "kafmm_get_counters": ([vp, ctypes.POINTER(i64), i32], i32),
            "kafmm_get_operator": ([vp, i32, vp], i32),
            "kafmm_measure_peak": ([i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)], i32),
            "kafmm_destroy": ([vp], i32),
            "kafmm_last_error": ([vp], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (must be C-contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a):
    name = str(a.dtype)
    if name.endswith("float64"):
        return F64
    if name.endswith("float32"):
        return F32
    raise TypeError(f"dtype must be float32 or float64, got {a.dtype}")


def _numel(a):
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


def _check(plan, rc):
    if rc != 0:
        msg = lib().kafmm_last_error(plan)
        raise KafmmError(rc, msg.decode() if msg else "")


# ---- the C ABI, name for name ---------------------------------------------------------------
def kafmm_plan(kernel, bc, p, max_pts_per_leaf):
    out = ctypes.c_void_p()
    _check(None, lib().kafmm_plan(kernel, bc, p, max_pts_per_leaf, ctypes.byref(out)))
    return out


def kafmm_set_option(plan, key, value):
    _check(plan, lib().kafmm_set_option(plan, key, int(value)))


def kafmm_set_domain(plan, origin, L):
    o = (ctypes.c_double * 3)(*[float(v) for v in origin])
    _check(plan, lib().kafmm_set_domain(plan, o, float(L)))


def kafmm_set_points(plan, y, n_src, x, n_trg, dtype):
    _check(plan, lib().kafmm_set_points(plan, _ptr(y), n_src, _ptr(x), n_trg, dtype))


def kafmm_set_points_batched(plan, n_prob, src_offsets, trg_offsets, y, x, dtype):
    so = np.ascontiguousarray(src_offsets, dtype=np.int64)
    to = np.ascontiguousarray(trg_offsets, dtype=np.int64)
    if so.size != n_prob + 1 or to.size != n_prob + 1:
        raise ValueError("offsets must have n_prob + 1 entries")
    _check(plan, lib().kafmm_set_points_batched(plan, n_prob, so.ctypes.data, to.ctypes.data,
                                                _ptr(y), _ptr(x), dtype))


def kafmm_eval(plan, s, g, dtype):
    _check(plan, lib().kafmm_eval(plan, _ptr(s), _ptr(g), dtype))


def kafmm_autotune(plan, s, g, dtype):
    chosen = (ctypes.c_int64 * 5)()
    _check(plan, lib().kafmm_autotune(plan, _ptr(s), _ptr(g), dtype, chosen))
    return {"tc_stages": int(chosen[0]), "tc_ranges": int(chosen[1]), "tc_tiling": int(chosen[2]),
            "leaf_stage": int(chosen[3]), "tc_tiles": int(chosen[4])}


def kafmm_status(plan):
    _check(plan, lib().kafmm_status(plan))


def kafmm_rpy_velocity(plan, s, a, g, ua, dtype):
    _check(plan, lib().kafmm_rpy_velocity(plan, _ptr(s), _ptr(a), _ptr(g), _ptr(ua), dtype))


def kafmm_rpy_velocity_noalloc(plan, s, a, g, ua, dtype):
    _check(plan, lib().kafmm_rpy_velocity_noalloc(plan, _ptr(s), _ptr(a), _ptr(g), _ptr(ua), dtype))


def kafmm_tree_info(plan):
    info = (ctypes.c_int64 * 16)()
    _check(plan, lib().kafmm_tree_info(plan, info, 16))
    keys = ["nbox", "nleaf", "nlevels", "n_u", "n_v", "n_w", "n_x", "near_pairs", "max_leaf_pts",
            "n_prob"]
    return {k: int(info[i]) for i, k in enumerate(keys)}


def kafmm_get_tree(plan, nbox):
    level = np.zeros(nbox, np.int32)
    anchor = np.zeros((nbox, 3), np.int32)
    parent = np.zeros(nbox, np.int32)
    leaf = np.zeros(nbox, np.int8)
    _check(plan, lib().kafmm_get_tree(plan, level.ctypes.data, anchor.ctypes.data,
                                      parent.ctypes.data, leaf.ctypes.data))
    return level, anchor, parent, leaf


def kafmm_get_list(plan, kind, nbox):
    off = np.zeros(nbox + 1, np.int64)
    _check(plan, lib().kafmm_get_list(plan, kind, off.ctypes.data, None, None))
    ent = np.zeros(max(int(off[-1]), 1), np.int32)
    sh = np.zeros(max(int(off[-1]), 1), np.int8)
    _check(plan, lib().kafmm_get_list(plan, kind, off.ctypes.data, ent.ctypes.data, sh.ctypes.data))
    return off, ent[:off[-1]], sh[:off[-1]]


def kafmm_phase_times(plan):
    t = (ctypes.c_double * 8)()
    _check(plan, lib().kafmm_phase_times(plan, t, 8))
    names = ["tree", "lists", "upward", "m2l", "downward", "leaves", "eval", "host_worklists"]
    return {k: float(t[i]) for i, k in enumerate(names)}


def kafmm_get_counters(plan):
    c = (ctypes.c_int64 * 12)()
    _check(plan, lib().kafmm_get_counters(plan, c, 12))
    return {"launches_points": int(c[0]), "launches_eval": int(c[1]),
            "tensor_core_m2l": int(c[2]), "launches_per_step": int(c[3]),
            "tc_split": {0: "tf32x3", 1: "bf16x3"}.get(int(c[4])),
            "m2l_tiling": {1: "whole V lists", 2: "per parent neighbour"}.get(int(c[5])),
            "m2l_tiles": int(c[6]), "device_allocations": int(c[7]),
            "compressed_rows": int(c[8]), "rank_up": int(c[9]), "rank_dn": int(c[10])}


def kafmm_get_operator(plan, slot, R):
    out = np.zeros((R, R))
    _check(plan, lib().kafmm_get_operator(plan, slot, out.ctypes.data))
    return out


PEAK_FFMA, PEAK_RSQRT, PEAK_DFMA, PEAK_MMA_TF32, PEAK_MMA_BF16 = 0, 1, 2, 3, 4


def kafmm_measure_peak(what):
    """(operations per second, ms of the timed launch) of one micro-benchmark."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(None, lib().kafmm_measure_peak(what, ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value


def kafmm_destroy(plan):
    if plan:
        lib().kafmm_destroy(plan)


def kafmm_last_error(plan):
    m = lib().kafmm_last_error(plan)
    return m.decode() if m else ""


# ---- convenience wrapper --------------------------------------------------------------------
class Plan:
    """One evaluator plan: ``Plan(STOKESLET, p=10, q=128).set_points(y).eval(f)``."""

    def __init__(self, kernel, p, q, bc=BC_OPEN, precision=PREC_MIXED, variant=ML_L4,
                 near_only=False, kahan=False, stream=None, origin=(0.0, 0.0, 0.0), L=1.0,
                 tc_split=TC_AUTO, sync=True, tc_stages=None, compress=2):
        self.kernel = kernel
        self.ks, self.kt = KDIM[kernel]
        self.h = kafmm_plan(kernel, bc, p, q)
        kafmm_set_option(self.h, OPT_PRECISION, precision)
        kafmm_set_option(self.h, OPT_ML_VARIANT, variant)
        kafmm_set_option(self.h, OPT_NEAR_ONLY, int(near_only))
        kafmm_set_option(self.h, OPT_KAHAN, int(kahan))
        kafmm_set_option(self.h, OPT_TC_SPLIT, tc_split)
        kafmm_set_option(self.h, OPT_SYNC, int(sync))
        kafmm_set_option(self.h, OPT_COMPRESS, int(compress))
        if tc_stages is not None:
            kafmm_set_option(self.h, OPT_TC_STAGES, tc_stages)
        if stream is not None:
            kafmm_set_option(self.h, OPT_STREAM, int(stream))
        kafmm_set_domain(self.h, origin, L)
        self.n_src = self.n_trg = 0

    def set_points(self, y, x=None):
        dt = _dtype_code(y)
        ns = _numel(y) // 3
        if x is None:
            x, nt = y, ns
        else:
            nt = _numel(x) // 3
        kafmm_set_points(self.h, y, ns, x, nt, dt)
        self.n_src, self.n_trg = ns, nt
        return self

    def set_points_batched(self, y, offsets, x=None, trg_offsets=None):
        """Batch of independent problems: problem k owns rows offsets[k]:offsets[k+1]."""
        dt = _dtype_code(y)
        offsets = np.asarray(offsets, dtype=np.int64)
        n_prob = offsets.size - 1
        if x is None:
            x, trg_offsets = y, offsets
        trg_offsets = np.asarray(trg_offsets, dtype=np.int64)
        kafmm_set_points_batched(self.h, n_prob, offsets, trg_offsets, y, x, dt)
        self.n_src, self.n_trg = int(offsets[-1]), int(trg_offsets[-1])
        return self

    def eval(self, s, g=None):
        dt = _dtype_code(s)
        if g is None:
            if hasattr(s, "new_zeros"):
                g = s.new_zeros((self.n_trg, self.kt))
            else:
                g = np.zeros((self.n_trg, self.kt), dtype=s.dtype)
        kafmm_eval(self.h, s, g, dt)
        return g

    def info(self):
        return kafmm_tree_info(self.h)

    def phase_times(self):
        return kafmm_phase_times(self.h)

    def close(self):
        if self.h:
            kafmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
