"""Python binding of libfhash (include/fhash.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but
convert arguments (torch CUDA tensors or numpy host arrays -> raw pointers, the current
torch stream -> cudaStream_t) and turn a non-zero status into FHashError.  All
computation runs in the CUDA library; if libfhash.so is missing, importing this package
fails - there is no fallback.  Build it with ``python paper_2507_03836_gb300/build.py``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfhash.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libfhash.so is not built (run python paper_2507_03836_gb300/build.py): %s" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

MAX_LEVELS = 24
MAX_HIDDEN = 4
FP32, BF16 = 0, 1
SCHED_FOLD, SCHED_EXPLICIT, SCHED_GEOMETRIC = 0, 1, 2
LEVELS_MAX, LEVELS_MIN = 0, 1
STATE_PARAM, STATE_GRAD, STATE_ADAM_M, STATE_ADAM_V = 0, 1, 2, 3
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EDEVICE", 5: "ETIMEOUT", 6: "EBUSY", 7: "EIO"}


class FHashError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class fhash_schedule(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("fold", ctypes.c_int32), ("levels_rule", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("res", (ctypes.c_int32 * 4) * MAX_LEVELS),
                ("r0", ctypes.c_int32 * 4), ("r1", ctypes.c_int32 * 4)]


class fhash_build_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("nt", ctypes.c_int64),
                ("mask", ctypes.c_void_p), ("sched", fhash_schedule), ("F", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("mlp_hidden_layers", ctypes.c_int32), ("mlp_width", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("init_range", ctypes.c_float), ("layout", ctypes.c_int32), ("masks", ctypes.c_void_p),
                ("n_masks", ctypes.c_int32)]


class fhash_info(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("F", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("n_mlp_layers", ctypes.c_int32), ("mlp_dims", ctypes.c_int32 * (MAX_HIDDEN + 2)),
                ("res", (ctypes.c_int32 * 4) * MAX_LEVELS), ("base", ctypes.c_uint64 * MAX_LEVELS),
                ("total_rows", ctypes.c_uint64), ("n_table_params", ctypes.c_uint64),
                ("n_mlp_params", ctypes.c_uint64), ("fbb_lo", ctypes.c_int64 * 3), ("fbb_size", ctypes.c_int64 * 3),
                ("nt", ctypes.c_int64), ("step", ctypes.c_int64), ("device_bytes", ctypes.c_uint64)]


class fhash_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class fhash_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fwd", ctypes.c_float * 3)]


class fhash_render_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("samples_evaluated", ctypes.c_int64),
                ("samples_composited", ctypes.c_int64), ("steps_marched", ctypes.c_int64)]


class fhash_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("model", ctypes.c_int32), ("t_norm", ctypes.c_float), ("cam", fhash_camera),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32), ("max_pace", ctypes.c_int32), ("tf", ctypes.c_void_p),
                ("upsample", ctypes.c_int32), ("out", ctypes.c_void_p), ("counts", ctypes.c_void_p)]


class fhash_server_stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("samples", ctypes.c_int64), ("model_launches", ctypes.c_int64),
                ("live", ctypes.c_int64), ("queued", ctypes.c_int64), ("pool_bytes", ctypes.c_uint64),
                ("pool_used", ctypes.c_uint64), ("packed_launches", ctypes.c_int64)]


class fhash_adam_stats(ctypes.Structure):
    _fields_ = [("first_deferred_level", ctypes.c_int32), ("deferred_params", ctypes.c_uint64),
                ("step", ctypes.c_int64), ("clean_step", ctypes.c_int64), ("last_replayed_groups", ctypes.c_uint64),
                ("last_replayed_steps", ctypes.c_uint64), ("last_ms", ctypes.c_float * 7),
                ("group_params", ctypes.c_uint32), ("last_side_ms", ctypes.c_float)]


ADAM_DEFER_DEFAULT_ROWS = 1 << 25

_vp, _i64, _u64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
_SIGS = {
    "fhash_build": [ctypes.POINTER(fhash_build_desc), _vp, ctypes.POINTER(_vp)],
    "fhash_destroy": [_vp],
    "fhash_get_info": [_vp, ctypes.POINTER(fhash_info)],
    "fhash_lookup": [_vp, _vp, _i64, _vp, _vp, _vp],
    "fhash_encode": [_vp, _vp, _i64, _vp, _vp],
    "fhash_encode_backward": [_vp, _vp, _vp, _i64, _vp],
    "fhash_forward": [_vp, _vp, _i64, _vp, _vp],
    "fhash_set_forward_path": [_vp, _i32],
    "fhash_coreset_build": [_vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_int64), _vp],
    "fhash_coreset_batch": [_vp, _u64, _i64, _i64, _i64, _vp, _vp, ctypes.POINTER(ctypes.c_int64), _vp],
    "fhash_coreset_train_step": [_vp, _u64, _i64, _i64, _i64, ctypes.POINTER(fhash_adam), _vp, _vp],
    "fhash_compute_grads": [_vp, _vp, _vp, _i64, _vp, _vp],
    "fhash_apply_adam": [_vp, ctypes.POINTER(fhash_adam), _vp],
    "fhash_train_step": [_vp, _vp, _vp, _i64, ctypes.POINTER(fhash_adam), _vp, _vp],
    "fhash_set_adam_deferral": [_vp, _u64, _vp],
    "fhash_set_timing": [_vp, _i32],
    "fhash_get_adam_stats": [_vp, ctypes.POINTER(fhash_adam_stats)],
    "fhash_read_state": [_vp, _i32, _u64, _u64, _vp, _vp],
    "fhash_get_params": [_vp, _vp, _vp, _vp],
    "fhash_set_params": [_vp, _vp, _vp, _vp],
    "fhash_level_info": [_vp, ctypes.POINTER(_i32), _vp, _vp, _vp],
    "fhash_write_state": [_vp, _i32, _u64, _u64, _vp, _vp],
    "fhash_read_occupancy": [_vp, _i64, _vp, _vp],
    "fhash_read_active": [_vp, _i32, _u64, _u64, _vp, _vp],
    "fhash_active_range": [_i64, _i64, _i64, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "fhash_plan": [ctypes.POINTER(fhash_schedule), _vp, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(_i32), _vp,
                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
    "fhash_check": [_vp, _vp],
    "fhash_save": [_vp, ctypes.c_char_p],
    "fhash_diag_wait_timeout": [_vp, _u64, _vp],
    "fhash_diag_random_gather": [_vp, _u64, _i32, _i64, _u64, _vp, _vp],
    "fhash_load": [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)],
    "fhash_compute_grads_noalloc": [_vp, _vp, _vp, _i64, _vp, _vp],
    "fhash_render": [_vp, ctypes.POINTER(fhash_camera), ctypes.c_float, _vp, _i32, _i32, _i32, _vp, _vp,
                     ctypes.POINTER(fhash_render_stats), _vp],
    "fhash_decode_dims": [_vp, _i32, ctypes.POINTER(ctypes.c_int64 * 3)],
    "fhash_decode": [_vp, ctypes.c_float, _i32, _vp, _vp],
    "fhash_server_create": [ctypes.POINTER(_vp), _i32, _u64, _i32, _i64, _vp, ctypes.POINTER(_vp)],
    "fhash_server_submit": [_vp, ctypes.POINTER(fhash_request), ctypes.POINTER(_u64)],
    "fhash_server_tick": [_vp, _vp, ctypes.POINTER(_i32)],
    "fhash_server_poll": [_vp, _u64, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)],
    "fhash_server_cancel": [_vp, _u64],
    "fhash_server_get_stats": [_vp, ctypes.POINTER(fhash_server_stats)],
    "fhash_server_destroy": [_vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = None if _name in ("fhash_destroy", "fhash_server_destroy") else ctypes.c_int
_lib.fhash_last_error.restype = ctypes.c_char_p
_lib.fhash_last_error.argtypes = []


def fhash_last_error():
    return _lib.fhash_last_error().decode()


def _ok(status):
    if status != 0:
        raise FHashError(status, fhash_last_error())


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or a numpy array; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def _stream(stream=None):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


class Model:
    """Owning handle of an fhash_model*; released by fhash_destroy."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.fhash_destroy(self.handle)
            self.handle = None

    @property
    def _as_parameter_(self):
        return self.handle


def make_schedule(mode="explicit", res=None, fold=2, levels_rule=LEVELS_MAX, n_levels=0, r0=None, r1=None):
    s = fhash_schedule()
    s.mode = {"fold": SCHED_FOLD, "explicit": SCHED_EXPLICIT, "geometric": SCHED_GEOMETRIC}[mode]
    s.fold = fold
    s.levels_rule = levels_rule
    if res is not None:
        s.n_levels = len(res)
        for l, R in enumerate(res):
            for d in range(4):
                s.res[l][d] = int(R[d])
    else:
        s.n_levels = n_levels
    for d in range(4):
        s.r0[d] = int(r0[d]) if r0 is not None else 0
        s.r1[d] = int(r1[d]) if r1 is not None else 0
    return s


LAYOUT_LINEAR, LAYOUT_BRICK, LAYOUT_MASKED = 0, 1, 2


def fhash_active_range(v, S, R, is_time=False):
    """Vertices [lo, hi] of a level axis that voxel (or time step) v makes active in a masked model."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    _ok(_lib.fhash_active_range(int(v), int(S), int(R), 1 if is_time else 0, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def fhash_plan(fbb, nt, schedule=None, F=2, dtype=FP32, mlp_hidden_layers=2, mlp_width=64):
    """Levels, table rows, parameters and device state bytes fhash_build would use (host only)."""
    sched = schedule if schedule is not None else make_schedule()
    fb = (ctypes.c_int64 * 3)(*[int(x) for x in fbb])
    L = _i32()
    res = ((ctypes.c_int32 * 4) * MAX_LEVELS)()
    rows, npar, nbytes = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _ok(_lib.fhash_plan(ctypes.byref(sched), ctypes.cast(fb, _vp), int(nt), int(F), int(dtype), int(mlp_hidden_layers),
                        int(mlp_width), ctypes.byref(L), ctypes.cast(res, _vp), ctypes.byref(rows), ctypes.byref(npar),
                        ctypes.byref(nbytes)))
    return dict(res=[list(res[l]) for l in range(L.value)], table_rows=rows.value, n_params=npar.value,
                state_bytes=nbytes.value)


def fhash_build(nx, ny, nz, nt, mask=None, schedule=None, F=2, dtype=FP32, mlp_hidden_layers=2, mlp_width=64,
                seed=0, init_range=1e-4, layout=LAYOUT_LINEAR, stream=None, masks=None):
    """fhash_build: mask is a host numpy uint8 array [nt][nz][ny][nx] or None; masks, a list of such arrays
    (several features, merged), replaces it."""
    d = fhash_build_desc()
    d.nx, d.ny, d.nz, d.nt = int(nx), int(ny), int(nz), int(nt)

    def _mask(a):
        a = np.ascontiguousarray(a, np.uint8)
        if a.shape != (nt, nz, ny, nx):
            raise ValueError("mask shape %s != (nt, nz, ny, nx)" % (a.shape,))
        return a
    if mask is not None:
        mask = _mask(mask)
    d.mask = _ptr(mask)
    keep = []
    if masks is not None:
        keep = [_mask(a) for a in masks]
        arr = (_vp * max(1, len(keep)))(*[a.ctypes.data for a in keep])
        d.masks = ctypes.cast(arr, _vp)
        d.n_masks = len(keep)
    d.sched = schedule if schedule is not None else make_schedule()
    d.F, d.dtype = int(F), int(dtype)
    d.mlp_hidden_layers, d.mlp_width = int(mlp_hidden_layers), int(mlp_width)
    d.seed, d.init_range = int(seed), float(init_range)
    d.layout = int(layout)
    h = _vp()
    _ok(_lib.fhash_build(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
    return Model(h.value)


def fhash_get_info(model):
    info = fhash_info()
    _ok(_lib.fhash_get_info(model.handle, ctypes.byref(info)))
    L = info.n_levels
    return dict(n_levels=L, F=info.F, dtype=info.dtype, mlp_dims=list(info.mlp_dims[:info.n_mlp_layers + 1]),
                res=[list(info.res[l]) for l in range(L)], base=[int(info.base[l]) for l in range(L)],
                total_rows=int(info.total_rows), n_table_params=int(info.n_table_params),
                n_mlp_params=int(info.n_mlp_params), fbb_lo=list(info.fbb_lo), fbb_size=list(info.fbb_size),
                nt=int(info.nt), step=int(info.step), device_bytes=int(info.device_bytes))


def fhash_lookup(model, coords, rows, weights=None, stream=None):
    _ok(_lib.fhash_lookup(model.handle, _ptr(coords), coords.shape[0], _ptr(rows), _ptr(weights), _stream(stream)))


def fhash_encode(model, coords, enc, stream=None):
    _ok(_lib.fhash_encode(model.handle, _ptr(coords), coords.shape[0], _ptr(enc), _stream(stream)))


def fhash_encode_backward(model, coords, d_enc, stream=None):
    _ok(_lib.fhash_encode_backward(model.handle, _ptr(coords), _ptr(d_enc), coords.shape[0], _stream(stream)))


FORWARD_AUTO, FORWARD_FUSED, FORWARD_SPLIT = 0, 1, 2


def fhash_set_forward_path(model, path):
    _ok(_lib.fhash_set_forward_path(model.handle, path))


def fhash_forward(model, coords, out, stream=None):
    _ok(_lib.fhash_forward(model.handle, _ptr(coords), coords.shape[0], _ptr(out), _stream(stream)))


def _adam(adam):
    a = fhash_adam()
    a.lr, a.beta1, a.beta2, a.eps = adam if adam is not None else (1e-2, 0.9, 0.99, 1e-8)
    return a


def fhash_compute_grads(model, coords, target, loss=None, stream=None):
    _ok(_lib.fhash_compute_grads(model.handle, _ptr(coords), _ptr(target), coords.shape[0], _ptr(loss),
                                 _stream(stream)))


def fhash_apply_adam(model, adam=None, stream=None):
    a = _adam(adam)
    _ok(_lib.fhash_apply_adam(model.handle, ctypes.byref(a), _stream(stream)))


def fhash_train_step(model, coords, target, adam=None, loss=None, stream=None):
    a = _adam(adam)
    _ok(_lib.fhash_train_step(model.handle, _ptr(coords), _ptr(target), coords.shape[0], ctypes.byref(a),
                              _ptr(loss), _stream(stream)))


def fhash_set_adam_deferral(model, min_level_rows, stream=None):
    _ok(_lib.fhash_set_adam_deferral(model.handle, int(min_level_rows), _stream(stream)))


def fhash_set_timing(model, enable=True):
    _ok(_lib.fhash_set_timing(model.handle, 1 if enable else 0))


def fhash_get_adam_stats(model):
    st = fhash_adam_stats()
    _ok(_lib.fhash_get_adam_stats(model.handle, ctypes.byref(st)))
    return {"first_deferred_level": st.first_deferred_level, "deferred_params": st.deferred_params,
            "step": st.step, "clean_step": st.clean_step, "last_replayed_groups": st.last_replayed_groups,
            "last_replayed_steps": st.last_replayed_steps, "last_ms": list(st.last_ms),
            "group_params": st.group_params, "last_side_ms": st.last_side_ms}


def fhash_coreset_build(model, volume, key_frames, stream=None):
    """Returns the number of coreset samples."""
    keys = np.ascontiguousarray(key_frames, np.int32)
    n = ctypes.c_int64(0)
    _ok(_lib.fhash_coreset_build(model.handle, _ptr(volume), keys.ctypes.data, keys.size, ctypes.byref(n),
                                 _stream(stream)))
    return int(n.value)


def fhash_coreset_batch(model, seed, epoch, batch, batch_size, coords, target, stream=None):
    """Returns the number of samples written."""
    n = ctypes.c_int64(0)
    _ok(_lib.fhash_coreset_batch(model.handle, seed, epoch, batch, batch_size, _ptr(coords), _ptr(target),
                                 ctypes.byref(n), _stream(stream)))
    return int(n.value)


def fhash_coreset_train_step(model, seed, epoch, batch, batch_size, adam=None, loss=None, stream=None):
    a = _adam(adam)
    _ok(_lib.fhash_coreset_train_step(model.handle, seed, epoch, batch, batch_size, ctypes.byref(a), _ptr(loss),
                                      _stream(stream)))


def fhash_get_params(model, tables=None, mlp=None, stream=None):
    _ok(_lib.fhash_get_params(model.handle, _ptr(tables), _ptr(mlp), _stream(stream)))


def fhash_set_params(model, tables=None, mlp=None, stream=None):
    _ok(_lib.fhash_set_params(model.handle, _ptr(tables), _ptr(mlp), _stream(stream)))


def fhash_level_info(model):
    """Returns (res [L][4], base [L], fbb [6]) as lists."""
    L = ctypes.c_int32(0)
    res = (ctypes.c_int32 * (4 * MAX_LEVELS))()
    base = (ctypes.c_uint64 * MAX_LEVELS)()
    fbb = (ctypes.c_int64 * 6)()
    _ok(_lib.fhash_level_info(model.handle, ctypes.byref(L), res, base, fbb))
    n = L.value
    return [list(res[4 * l:4 * l + 4]) for l in range(n)], [int(b) for b in base[:n]], list(fbb)


def fhash_read_state(model, which, offset, buf, stream=None):
    n = buf.numel() if hasattr(buf, "numel") else buf.size
    _ok(_lib.fhash_read_state(model.handle, which, int(offset), int(n), _ptr(buf), _stream(stream)))


def fhash_write_state(model, which, offset, buf, stream=None):
    n = buf.numel() if hasattr(buf, "numel") else buf.size
    _ok(_lib.fhash_write_state(model.handle, which, int(offset), int(n), _ptr(buf), _stream(stream)))


def fhash_read_occupancy(model, t, out, stream=None):
    _ok(_lib.fhash_read_occupancy(model.handle, int(t), _ptr(out), _stream(stream)))


def fhash_read_active(model, level, word0, out, stream=None):
    """Active-vertex bit words [word0, word0 + len(out)) of a masked level into `out` (uint64)."""
    n = out.numel() if hasattr(out, "numel") else out.size
    _ok(_lib.fhash_read_active(model.handle, int(level), int(word0), int(n), _ptr(out), _stream(stream)))


def fhash_compute_grads_noalloc(model, coords, target, loss=None, stream=None):
    _ok(_lib.fhash_compute_grads_noalloc(model.handle, _ptr(coords), _ptr(target), coords.shape[0], _ptr(loss),
                                         _stream(stream)))


NOALLOC_MAX_SAMPLES = 4096


def make_camera(eye, right, up, fwd):
    c = fhash_camera()
    for a in range(3):
        c.eye[a], c.right[a], c.up[a], c.fwd[a] = float(eye[a]), float(right[a]), float(up[a]), float(fwd[a])
    return c


def fhash_render(model, cam, t_norm, tf, w, h, rgba, counts=None, max_pace=64, stream=None):
    """cam: fhash_camera or (eye, right, up, fwd); tf, rgba, counts: device tensors.  Returns stats dict."""
    if not isinstance(cam, fhash_camera):
        cam = make_camera(*cam)
    st = fhash_render_stats()
    _ok(_lib.fhash_render(model.handle, ctypes.byref(cam), float(t_norm), _ptr(tf), int(w), int(h), int(max_pace),
                          _ptr(rgba), _ptr(counts), ctypes.byref(st), _stream(stream)))
    return dict(rounds=st.rounds, samples_evaluated=st.samples_evaluated,
                samples_composited=st.samples_composited, steps_marched=st.steps_marched)


def fhash_decode_dims(model, upsample):
    d = (ctypes.c_int64 * 3)()
    _ok(_lib.fhash_decode_dims(model.handle, int(upsample), ctypes.byref(d)))
    return [int(d[0]), int(d[1]), int(d[2])]


def fhash_decode(model, t_norm, upsample, out, stream=None):
    _ok(_lib.fhash_decode(model.handle, float(t_norm), int(upsample), _ptr(out), _stream(stream)))


def fhash_save(model, path):
    _ok(_lib.fhash_save(model.handle, str(path).encode()))


def fhash_load(path, stream=None):
    h = _vp()
    _ok(_lib.fhash_load(str(path).encode(), _stream(stream), ctypes.byref(h)))
    return Model(h.value)


def fhash_diag_wait_timeout(model, limit_ns, stream=None):
    _ok(_lib.fhash_diag_wait_timeout(model.handle, int(limit_ns), _stream(stream)))


def fhash_diag_random_gather(table, width, n, seed, sum_out, stream=None):
    nbytes = table.numel() * table.element_size()
    _ok(_lib.fhash_diag_random_gather(_ptr(table), nbytes, width, n, seed, _ptr(sum_out), _stream(stream)))


def fhash_check(model, stream=None):
    _ok(_lib.fhash_check(model.handle, _stream(stream)))


REQ_RENDER, REQ_DECODE = 0, 1
REQ_QUEUED, REQ_LIVE, REQ_DONE, REQ_CANCELLED = 0, 1, 2, 3


class Server:
    """Owning handle of an fhash_server*; keeps its models alive."""

    def __init__(self, handle, models):
        self.handle, self.models = handle, list(models)

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.fhash_server_destroy(self.handle)
            self.handle = None


def fhash_server_create(models, budget_bytes, max_live=64, tick_samples=1 << 22, stream=None):
    arr = (_vp * len(models))(*[m.handle for m in models])
    h = _vp()
    _ok(_lib.fhash_server_create(arr, len(models), int(budget_bytes), int(max_live), int(tick_samples),
                                 _stream(stream), ctypes.byref(h)))
    return Server(h.value, models)


def make_request(kind, model=0, t_norm=0.0, cam=None, w=0, h=0, max_pace=64, tf=None, upsample=1, out=None,
                 counts=None):
    r = fhash_request()
    r.kind, r.model, r.t_norm = int(kind), int(model), float(t_norm)
    if cam is not None:
        r.cam = cam if isinstance(cam, fhash_camera) else make_camera(*cam)
    r.w, r.h, r.max_pace = int(w), int(h), int(max_pace)
    r.tf, r.upsample, r.out, r.counts = _ptr(tf), int(upsample), _ptr(out), _ptr(counts)
    return r


def fhash_server_submit(server, req):
    i = _u64()
    _ok(_lib.fhash_server_submit(server.handle, ctypes.byref(req), ctypes.byref(i)))
    return int(i.value)


def fhash_server_tick(server, stream=None):
    n = _i32()
    _ok(_lib.fhash_server_tick(server.handle, _stream(stream), ctypes.byref(n)))
    return int(n.value)


def fhash_server_poll(server, rid):
    st, lat = _i32(), ctypes.c_double()
    _ok(_lib.fhash_server_poll(server.handle, int(rid), ctypes.byref(st), ctypes.byref(lat)))
    return int(st.value), float(lat.value)


def fhash_server_cancel(server, rid):
    _ok(_lib.fhash_server_cancel(server.handle, int(rid)))


def fhash_server_get_stats(server):
    st = fhash_server_stats()
    _ok(_lib.fhash_server_get_stats(server.handle, ctypes.byref(st)))
    return {k: int(getattr(st, k)) for k, _ in fhash_server_stats._fields_}
