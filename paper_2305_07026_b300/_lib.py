"""ctypes binding of the C ABI in include/daba.h (argument marshalling only).

Every function of the header is exposed under the same name. Array arguments may be
numpy arrays (host memory) or torch tensors (host or CUDA); they are passed to the
library as raw pointers, and `stream` defaults to torch's current CUDA stream. No
computation happens here: if the CUDA library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdaba_b300.so")

DABA_OK, DABA_ERR_ARG, DABA_ERR_INDEX, DABA_ERR_DEGENERATE, DABA_ERR_NONFINITE, DABA_ERR_CUDA, DABA_ERR_OOM, \
    DABA_ERR_STATE, DABA_ERR_TIMEOUT = range(9)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_INDEX", "ERR_DEGENERATE", "ERR_NONFINITE", "ERR_CUDA", "ERR_OOM", "ERR_STATE",
                "ERR_TIMEOUT"]
LOSSES = {"trivial": 0, "huber": 1, "cauchy": 2, "welsch": 3}
PREC = {"fp64": 0, "mixed": 1}
RESTART = {"block": 0, "global": 1}
CAM_SOLVERS = {"scam": 0, "lm": 1}
BLK_MAX_CAMS = 512   # cameras per coarse block (daba_set_partition)

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library {LIB_PATH} is not built; run `python -m paper_2305_07026_b300.build`")

lib = ctypes.CDLL(LIB_PATH)


class daba_options(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_int), ("loss_scale_px", ctypes.c_double), ("xi", ctypes.c_double),
                ("eta", ctypes.c_double), ("accelerated", ctypes.c_int), ("cam_alternations", ctypes.c_int),
                ("pixel_scale", ctypes.c_double), ("prec", ctypes.c_int), ("chunk_obs", ctypes.c_int32),
                ("tile_obs", ctypes.c_int32), ("tile_lms", ctypes.c_int32), ("restart_mode", ctypes.c_int32),
                ("momentum_reset", ctypes.c_int32), ("cam_solver", ctypes.c_int32)]


class daba_pipeline(ctypes.Structure):
    _fields_ = [("ranges", ctypes.c_int32), ("cpass_warps", ctypes.c_int32), ("lpass_ctas", ctypes.c_int32),
                ("prio", ctypes.c_int32 * 3)]


_p = ctypes.c_void_p
_i32, _i64, _st = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
_SIGS = {
    "daba_default_options": (None, [ctypes.POINTER(daba_options)]),
    "daba_create": (_st, [_i32, _i32, _i64, ctypes.POINTER(daba_options), ctypes.POINTER(_p)]),
    "daba_set_observations": (_st, [_p, _p, _p, _p, _p]),
    "daba_set_state": (_st, [_p, _p, _p, _p]),
    "daba_run": (_st, [_p, _i32, _p, _p, _p]),
    "daba_objective": (_st, [_p, _p, _p]),
    "daba_get_state": (_st, [_p, _p, _p, _p]),
    "daba_get_block_metrics": (_st, [_p, _p, _p, _p, _p, _p, _p, _p]),
    "daba_get_sort": (_st, [_p, _p, _p, _p, _p, _p]),
    "daba_set_scenes": (_st, [_p, _i32, _p]),
    "daba_objective_grad": (_st, [_p, _p, _p, _p, _p, _p]),
    "daba_set_pixels": (_st, [_p, _p, _p]),
    "daba_unrolled_grad": (_st, [_p, _i32, _p, _p, _p, _p, _p, _p]),
    "daba_scene_objectives": (_st, [_p, _p, _p]),
    "daba_export_checkpoint": (_st, [_p, _p, ctypes.POINTER(ctypes.c_size_t)]),
    "daba_import_checkpoint": (_st, [_p, _p, ctypes.c_size_t]),
    "daba_set_wait_limit": (_st, [_p, _i64]),
    "daba_set_persistent": (_st, [_p, ctypes.c_int]),
    "daba_set_pipeline": (_st, [_p, ctypes.POINTER(daba_pipeline)]),
    "daba_set_partition": (_st, [_p, _i32, _p, _p]),
    "daba_get_partition_metrics": (_st, [_p, _p, _p, _p, _p]),
    "daba_set_block_ctas": (_st, [_p, _i32]),
    "daba_set_timing": (_st, [_p, ctypes.c_int]),
    "daba_get_timing": (_st, [_p, _p]),
    "daba_last_launch_count": (_i64, [_p]),
    "daba_device_bytes": (_st, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "daba_objective_noalloc": (_st, [_i32, _i32, _i64, _p, _p, _p, _p, _p, _i32, ctypes.c_double, ctypes.c_double,
                                     _p, _p]),
    "daba_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "daba_last_error": (ctypes.c_char_p, [_p]),
    "daba_destroy": (None, [_p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class DabaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def ptr(a):
    """Raw data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def options(loss="huber", loss_scale_px=1.0, xi=1e-10, eta=0.5, accelerated=True, cam_alternations=2,
            pixel_scale=0.0, prec="mixed", chunk_obs=0, tile_obs=0, tile_lms=0, restart="block",
            momentum_reset=False, cam_solver="scam") -> daba_options:
    o = daba_options()
    daba_default_options(ctypes.byref(o))
    o.loss = LOSSES[loss] if isinstance(loss, str) else int(loss)
    o.loss_scale_px = float(loss_scale_px)
    o.xi = float(xi)
    o.eta = float(eta)
    o.accelerated = int(bool(accelerated))
    o.cam_alternations = int(cam_alternations)
    o.pixel_scale = float(pixel_scale)
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.chunk_obs, o.tile_obs, o.tile_lms = int(chunk_obs), int(tile_obs), int(tile_lms)
    o.restart_mode = RESTART[restart] if isinstance(restart, str) else int(restart)
    o.momentum_reset = int(bool(momentum_reset))
    o.cam_solver = CAM_SOLVERS[cam_solver] if isinstance(cam_solver, str) else int(cam_solver)
    return o


class Daba:
    """Owns one daba_ctx; methods are the ABI calls with this context bound."""

    def __init__(self, M, N, nnz, **opts):
        self.M, self.N, self.nnz = int(M), int(N), int(nnz)
        self.opts = options(**opts)
        h = _p()
        st = daba_create(self.M, self.N, self.nnz, ctypes.byref(self.opts), ctypes.byref(h))
        if st != DABA_OK:
            raise DabaError(st, "daba_create failed")
        self._h = h

    def _check(self, st):
        if st != DABA_OK:
            raise DabaError(st, daba_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            daba_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_observations(self, cam_idx, lm_idx, uv, stream=None):
        self._check(daba_set_observations(self._h, ptr(cam_idx), ptr(lm_idx), ptr(uv),
                                          current_stream() if stream is None else stream))

    def set_state(self, cams, lms, stream=None):
        self._check(daba_set_state(self._h, ptr(cams), ptr(lms), current_stream() if stream is None else stream))

    def run(self, iters, obj_trace=None, restarts=None, stream=None):
        self._check(daba_run(self._h, int(iters), ptr(obj_trace), ptr(restarts),
                             current_stream() if stream is None else stream))

    def objective(self, out=None, stream=None):
        host = out is None
        if host:
            out = np.zeros(1)
        self._check(daba_objective(self._h, ptr(out), current_stream() if stream is None else stream))
        return float(out[0]) if host else out

    def get_state(self, cams=None, lms=None, stream=None):
        if cams is None and lms is None:
            cams, lms = np.zeros((self.M, 9)), np.zeros((self.N, 3))
        self._check(daba_get_state(self._h, ptr(cams), ptr(lms), current_stream() if stream is None else stream))
        return cams, lms

    def get_block_metrics(self, landmarks=True, stream=None):
        out = {"F_cam": np.zeros(self.M), "Fbar_cam": np.zeros(self.M), "rs_cam": np.zeros(self.M, np.uint8),
               "rs_lm": np.zeros(self.N, np.uint8)}
        if landmarks:
            out["F_lm"] = np.zeros(self.N)
            out["Fbar_lm"] = np.zeros(self.N)
        self._check(daba_get_block_metrics(self._h, ptr(out["F_cam"]), ptr(out["Fbar_cam"]), ptr(out.get("F_lm")),
                                           ptr(out.get("Fbar_lm")), ptr(out["rs_cam"]), ptr(out["rs_lm"]),
                                           current_stream() if stream is None else stream))
        return out

    def get_sort(self, stream=None):
        co, cp = np.zeros(self.nnz, np.int32), np.zeros(self.M + 1, np.int32)
        lo, lp = np.zeros(self.nnz, np.int32), np.zeros(self.N + 1, np.int32)
        self._check(daba_get_sort(self._h, ptr(co), ptr(cp), ptr(lo), ptr(lp),
                                  current_stream() if stream is None else stream))
        return co, cp, lo, lp

    def objective_grad(self, F=None, g_cams=None, g_lms=None, g_uv=None, stream=None):
        """F(x^k) and its gradients w.r.t. cameras (M x 9), landmarks (N x 3) and pixels (nnz x 2);
        with no arguments, host arrays of all four are returned."""
        if F is None and g_cams is None and g_lms is None and g_uv is None:
            F, g_cams, g_lms, g_uv = np.zeros(1), np.zeros((self.M, 9)), np.zeros((self.N, 3)), np.zeros((self.nnz, 2))
            self._check(daba_objective_grad(self._h, ptr(F), ptr(g_cams), ptr(g_lms), ptr(g_uv),
                                            current_stream() if stream is None else stream))
            return float(F[0]), g_cams, g_lms, g_uv
        self._check(daba_objective_grad(self._h, ptr(F), ptr(g_cams), ptr(g_lms), ptr(g_uv),
                                        current_stream() if stream is None else stream))
        return F, g_cams, g_lms, g_uv

    def unrolled_grad(self, K, seed_cams, seed_lms, g_cams=None, g_lms=None, g_uv=None, stream=None):
        """Vector-Jacobian product of K iterations from the state last set: the gradient of
        <seed_cams, cams_K> + <seed_lms, lms_K> w.r.t. the set cameras (M x 9), landmarks
        (N x 3) and pixels (nnz x 2). Leaves the state after K iterations. With no output
        arguments, host arrays are returned."""
        host = g_cams is None and g_lms is None and g_uv is None
        if host:
            g_cams, g_lms, g_uv = np.zeros((self.M, 9)), np.zeros((self.N, 3)), np.zeros((self.nnz, 2))
            seed_cams = np.ascontiguousarray(seed_cams, dtype=np.float64)
            seed_lms = np.ascontiguousarray(seed_lms, dtype=np.float64)
        self._check(daba_unrolled_grad(self._h, int(K), ptr(seed_cams), ptr(seed_lms), ptr(g_cams), ptr(g_lms),
                                       ptr(g_uv), current_stream() if stream is None else stream))
        return g_cams, g_lms, g_uv

    def set_pixels(self, uv, stream=None):
        self._check(daba_set_pixels(self._h, ptr(uv), current_stream() if stream is None else stream))

    def set_scenes(self, cam_begin):
        cb = np.ascontiguousarray(cam_begin, dtype=np.int32)
        self._check(daba_set_scenes(self._h, int(cb.size - 1), ptr(cb)))
        self.n_scenes = int(cb.size - 1)

    def scene_objectives(self, out=None, stream=None):
        host = out is None
        if host:
            out = np.zeros(self.n_scenes)
        self._check(daba_scene_objectives(self._h, ptr(out), current_stream() if stream is None else stream))
        return out

    def export_checkpoint(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._check(daba_export_checkpoint(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(daba_export_checkpoint(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def import_checkpoint(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(daba_import_checkpoint(self._h, buf, len(data)))

    def set_partition(self, cam_block=None, lm_block=None, n_blocks=None):
        """Coarse blocks: camera i in block cam_block[i] (at most BLK_MAX_CAMS per block), landmark
        j in block lm_block[j]; n_blocks defaults to one more than the largest block id. None
        clears (one block per camera and per landmark)."""
        if cam_block is None:
            self._check(daba_set_partition(self._h, 0, None, None))
            self.n_blocks = 0
            return
        cb = np.ascontiguousarray(cam_block, dtype=np.int32)
        lb = np.ascontiguousarray(lm_block, dtype=np.int32)
        if n_blocks is None:
            n_blocks = int(max(cb.max(initial=-1), lb.max(initial=-1))) + 1
        self._check(daba_set_partition(self._h, int(n_blocks), ptr(cb), ptr(lb)))
        self.n_blocks = int(n_blocks)

    def set_block_ctas(self, ctas=0):
        """CTAs per coarse block at the next set_partition: 0 automatic, 1 one CTA per block,
        2..16 a thread-block cluster of at most that many."""
        self._check(daba_set_block_ctas(self._h, int(ctas)))

    def get_partition_metrics(self, stream=None):
        F, Fb, rs = np.zeros(self.n_blocks), np.zeros(self.n_blocks), np.zeros(self.n_blocks, np.uint8)
        self._check(daba_get_partition_metrics(self._h, ptr(F), ptr(Fb), ptr(rs),
                                               current_stream() if stream is None else stream))
        return F, Fb, rs

    def set_persistent(self, enable=True):
        self._check(daba_set_persistent(self._h, int(bool(enable))))

    def set_pipeline(self, ranges=1, cpass_warps=0, lpass_ctas=0, prio=(1, 0, 1)):
        p = daba_pipeline(int(ranges), int(cpass_warps), int(lpass_ctas), (ctypes.c_int32 * 3)(*prio))
        self._check(daba_set_pipeline(self._h, ctypes.byref(p)))

    def set_wait_limit(self, first_wait_ns):
        self._check(daba_set_wait_limit(self._h, int(first_wait_ns)))

    def set_timing(self, enable=True):
        self._check(daba_set_timing(self._h, int(bool(enable))))

    def get_timing(self):
        out = np.zeros(5)
        self._check(daba_get_timing(self._h, ptr(out)))
        return out

    def last_launch_count(self) -> int:
        return int(daba_last_launch_count(self._h))

    def device_bytes(self):
        """(bytes of device buffers held now, the most held at once) by this context."""
        b, pk = ctypes.c_int64(), ctypes.c_int64()
        self._check(daba_device_bytes(self._h, ctypes.byref(b), ctypes.byref(pk)))
        return int(b.value), int(pk.value)


def probe_fma_rate(kind):
    """Measured FMA rate of the current GPU in FLOP/s (daba_probe_fma_rate): kind "f32", "f32x2"
    (packed FP32) or "f64"."""
    out = ctypes.c_double(0.0)
    rc = daba_probe_fma_rate({"f32": 0, "f32x2": 1, "f64": 2}[kind], ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"daba_probe_fma_rate({kind}) failed with code {rc}")
    return out.value
