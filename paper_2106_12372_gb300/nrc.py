"""Thin Python binding of the C ABI in ``include/nrc.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA library ``libnrc.so``; this module
passes tensor data pointers, sizes and the current CUDA stream through ctypes.
PyTorch is used for device memory and streams only.  There is no fallback: if
the library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# NRC_LIB_VARIANT=san|debug selects a variant build (build.py) instead of libnrc.so
VARIANT = os.environ.get("NRC_LIB_VARIANT", "")
LIB_PATH = os.path.join(HERE, f"libnrc_{VARIANT}.so" if VARIANT else "libnrc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "nrc.h")

NRC_OK, NRC_ERR_INVALID_ARG, NRC_ERR_CUDA, NRC_ERR_OOM, NRC_ERR_TIMEOUT, NRC_ERR_UNSUPPORTED, NRC_ERR_BUSY, \
    NRC_ERR_BOUNDS = range(8)
FP32, FP16, BF16, FP8 = 0, 1, 2, 3
ENC_CHEAP, ENC_EXACT = 0, 1
LOSS_LUMINANCE, LOSS_PER_CHANNEL = 0, 1
PATH_FUSED, PATH_PLAIN = 0, 1
OPT_ADAM, OPT_SHAMPOO = 0, 1
DTYPES = {"fp32": FP32, "fp16": FP16, "bf16": BF16, "fp8": FP8}

_lock = threading.Lock()
_lib = None


class NrcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nrc status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("hidden_layers", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("enc_mode", ctypes.c_int32),
        ("loss_mode", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("pad_value", ctypes.c_float),
        ("lr", ctypes.c_float),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("adam_eps", ctypes.c_float),
        ("loss_eps", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("ema", ctypes.c_int32),
        ("ema_alpha", ctypes.c_float),
        ("refl_factor", ctypes.c_int32),
        ("optimizer", ctypes.c_int32),
        ("shampoo_interval", ctypes.c_int32),
        ("shampoo_eps", ctypes.c_float),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("memory_budget", ctypes.c_uint64),
        ("max_viewports", ctypes.c_int32),
        ("max_inflight", ctypes.c_int32),
        ("train_steps", ctypes.c_int32),
        ("train_batch", ctypes.c_int32),
        ("train_tiles", ctypes.c_int32),
        ("unit_tiles", ctypes.c_int32),
    ]


class FrameDone(ctypes.Structure):
    _fields_ = [
        ("viewport", ctypes.c_int32),
        ("slot", ctypes.c_int32),
        ("tag", ctypes.c_int64),
        ("n_queries", ctypes.c_int64),
        ("arrival_ns", ctypes.c_int64),
        ("submit_ns", ctypes.c_int64),
        ("launch_ns", ctypes.c_int64),
        ("done_ns", ctypes.c_int64),
        ("batch_frames", ctypes.c_int32),
        ("failed", ctypes.c_int32),
    ]


class ServerInfo(ctypes.Structure):
    _fields_ = [
        ("memory_used", ctypes.c_uint64),
        ("memory_budget", ctypes.c_uint64),
        ("frames_done", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("queries_done", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("viewports", ctypes.c_int32),
        ("inflight", ctypes.c_int32),
    ]


def declared_functions() -> list[str]:
    """Names of the entry points declared in include/nrc.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^NRC_API [^(]*?\b(nrc_\w+)\(", text, flags=re.M)))


def lib() -> ctypes.CDLL:
    """Loads libnrc.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        sig = {
            "nrc_default_config": (None, [P]),
            "nrc_create": (i32, [P, P, P]),
            "nrc_destroy": (i32, [P]),
            "nrc_param_count": (i64, [P]),
            "nrc_encode": (i32, [P, P, i64, P, i32, P]),
            "nrc_infer": (i32, [P, P, i64, P, P]),
            "nrc_gather": (i32, [P, P, i64, i64, u64, i32, P, P, P]),
            "nrc_train_step": (i32, [P, P, P, i64, i64, u64, i32, P, P]),
            "nrc_frame": (i32, [P, P, i64, P, P, P, i64, i64, i32, u64, P, P]),
            "nrc_frame_host": (i32, [P, P, i64, P, P, P, i64, i64, i32, u64, P, P]),
            "nrc_set_frame_ctas": (i32, [P, i32]),
            "nrc_frame_ctas": (i32, [P, i64, i64, i32]),
            "nrc_get_state": (i32, [P, P, P, P, P, P]),
            "nrc_set_state": (i32, [P, P, P, P, i64, P]),
            "nrc_set_path": (i32, [P, i32]),
            "nrc_check_error": (i32, [P, P]),
            "nrc_debug_fail_device_allocs": (None, [i32, i32]),
            "nrc_debug_wait_timeout": (i32, [P, i32, P]),
            "nrc_launch_count": (i64, [P]),
            "nrc_last_error_string": (ctypes.c_char_p, []),
            "nrc_train_step_noalloc": (i32, [P, P, P, P, P, P, P, i64, i64, u64, i32, P, P, P]),
            "nrc_batch_create": (i32, [P, i32, P]),
            "nrc_batch_destroy": (i32, [P]),
            "nrc_batch_infer": (i32, [P, P, P, P, P]),
            "nrc_batch_train_step": (i32, [P, P, P, P, P, P, i32, P, P]),
            "nrc_batch_train_step_dev": (i32, [P, P, P, P, P, P, i32, P, P]),
            "nrc_batch_set_unit_tiles": (i32, [P, i32]),
            "nrc_batch_autotune": (i32, [P, P, P, P, P, P]),
            "nrc_batch_set_train_tiles": (i32, [P, i32]),
            "nrc_get_ema": (i32, [P, P, P]),
            "nrc_paths_tile_count": (i64, [i32, i32, i32]),
            "nrc_paths_adapt_tile": (i32, [i32, i64, i64]),
            "nrc_paths_offsets_count": (i64, [i64]),
            "nrc_paths_terminate": (i32, [P, P, P, P, P, P, P, P]),
            "nrc_paths_records": (i32, [P, P, P, P, P, P, i64, P, P, P]),
            "nrc_paths_composite": (i32, [P, P, P, i64, P, P]),
            "nrc_set_ema": (i32, [P, P, P]),
            "nrc_server_default_config": (None, [P]),
            "nrc_now_ns": (i64, []),
            "nrc_server_create": (i32, [P, P, P]),
            "nrc_server_destroy": (i32, [P]),
            "nrc_server_open_viewport": (i32, [P, P, i64, i64, i32, P]),
            "nrc_server_close_viewport": (i32, [P, i32]),
            "nrc_server_viewport_buffers": (i32, [P, i32, i32, P, P, P]),
            "nrc_server_viewport_pool": (i32, [P, i32, P, P, P]),
            "nrc_server_submit": (i32, [P, i32, i32, i64, u64, i64, i64]),
            "nrc_server_poll": (i32, [P, P, i32, i32, P]),
            "nrc_server_pause": (i32, [P, i32]),
            "nrc_server_drain": (i32, [P]),
            "nrc_server_query": (i32, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int) -> None:
    if status != NRC_OK:
        msg = lib().nrc_last_error_string()
        raise NrcError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def default_config(**kw) -> Config:
    cfg = Config()
    lib().nrc_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "dtype" and isinstance(v, str):
            v = DTYPES[v]
        setattr(cfg, k, v)
    return cfg


def gather(pool, target, batch: int, frame_seed: int, step: int, stream=None):
    """Device gather of training batch ``step`` (Sec. 3.5): returns (records, targets)."""
    import torch

    rec = torch.empty((batch, 16), dtype=torch.float32, device=pool.device)
    tgt = torch.empty((batch, 3), dtype=torch.float32, device=pool.device)
    _check(lib().nrc_gather(_ptr(pool), _ptr(target), pool.shape[0], batch, frame_seed & (2**64 - 1), step,
                            _ptr(rec), _ptr(tgt), _stream(stream)))
    return rec, tgt


def train_step_noalloc(cfg: Config, weights, adam_m, adam_v, step_counter, pool, target, batch: int,
                       frame_seed: int, step: int, loss_out=None, err_out=None, stream=None) -> None:
    """Allocation-free training step on caller-owned device state (see include/nrc.h)."""
    _check(lib().nrc_train_step_noalloc(ctypes.byref(cfg), _ptr(weights), _ptr(adam_m), _ptr(adam_v),
                                        _ptr(step_counter), _ptr(pool), _ptr(target), pool.shape[0], batch,
                                        frame_seed & (2**64 - 1), step, _ptr(loss_out), _ptr(err_out),
                                        _stream(stream)))


class Cache:
    """One neural radiance cache (weights, Adam state) owned by the CUDA library."""

    def __init__(self, stream=None, **cfg_kw):
        self.cfg = default_config(**cfg_kw)
        h = ctypes.c_void_p()
        _check(lib().nrc_create(ctypes.byref(self.cfg), _stream(stream), ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().nrc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def n_params(self) -> int:
        return lib().nrc_param_count(self._h)

    @property
    def launches(self) -> int:
        return lib().nrc_launch_count(self._h)

    def set_path(self, path: int) -> None:
        _check(lib().nrc_set_path(self._h, path))

    def encode(self, rec, out_dtype: str = "fp32", stream=None):
        import torch

        tdt = {"fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}[out_dtype]
        out = torch.empty((rec.shape[0], 64), dtype=tdt, device=rec.device)
        _check(lib().nrc_encode(self._h, _ptr(rec), rec.shape[0], _ptr(out), DTYPES[out_dtype], _stream(stream)))
        return out

    def infer(self, rec, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty((rec.shape[0], 3), dtype=torch.float32, device=rec.device)
        _check(lib().nrc_infer(self._h, _ptr(rec), rec.shape[0], _ptr(out), _stream(stream)))
        return out

    def train_step(self, pool, target, batch: int, frame_seed: int, step: int, loss_out=None, stream=None):
        _check(lib().nrc_train_step(self._h, _ptr(pool), _ptr(target), pool.shape[0], batch,
                                    frame_seed & (2**64 - 1), step, _ptr(loss_out), _stream(stream)))

    def frame(self, queries, rgb, pool, target, batch: int, n_steps: int, frame_seed: int, loss_out=None,
              stream=None):
        _check(lib().nrc_frame(self._h, _ptr(queries), queries.shape[0], _ptr(rgb), _ptr(pool), _ptr(target),
                               pool.shape[0], batch, n_steps, frame_seed & (2**64 - 1), _ptr(loss_out),
                               _stream(stream)))

    def set_frame_ctas(self, train_ctas: int) -> None:
        """Training CTAs of the fused frame launch: 0 automatic, -1 separate launches."""
        _check(lib().nrc_set_frame_ctas(self._h, int(train_ctas)))

    def frame_ctas(self, n_queries: int, batch: int, n_steps: int) -> int:
        """Training CTAs nrc_frame would use for this shape (-1: not the fused launch)."""
        return int(lib().nrc_frame_ctas(self._h, int(n_queries), int(batch), int(n_steps)))

    def frame_host(self, queries, rgb, pool, target, batch: int, n_steps: int, frame_seed: int, loss_out=None,
                   stream=None):
        """As :meth:`frame` with host (ideally pinned) tensors; copies are inside the call."""
        _check(lib().nrc_frame_host(self._h, _ptr(queries), queries.shape[0], _ptr(rgb), _ptr(pool), _ptr(target),
                                    pool.shape[0], batch, n_steps, frame_seed & (2**64 - 1), _ptr(loss_out),
                                    _stream(stream)))

    def get_state(self, stream=None):
        n = self.n_params
        w, m, v = (np.zeros(n, dtype=np.float32) for _ in range(3))
        t = ctypes.c_int64()
        _check(lib().nrc_get_state(self._h, w.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(t),
                                   _stream(stream)))
        return w, m, v, t.value

    def set_state(self, w, m=None, v=None, step: int = 0, stream=None):
        n = self.n_params
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == n
        m = None if m is None else np.ascontiguousarray(m, dtype=np.float32)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        _check(lib().nrc_set_state(self._h, w.ctypes.data, None if m is None else m.ctypes.data,
                                   None if v is None else v.ctypes.data, step, _stream(stream)))

    def get_ema(self, stream=None):
        """The weight average (cfg.ema = 1) as an FP32 host array."""
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().nrc_get_ema(self._h, out.ctypes.data, _stream(stream)))
        return out

    def set_ema(self, ema, stream=None) -> None:
        a = np.ascontiguousarray(ema, dtype=np.float32)
        _check(lib().nrc_set_ema(self._h, a.ctypes.data, _stream(stream)))

    def debug_wait_timeout(self, limit_us: int, stream=None) -> None:
        """Fault injection: a bounded device wait that runs out after limit_us
        (the next check_error raises NRC_ERR_TIMEOUT)."""
        _check(lib().nrc_debug_wait_timeout(self._h, int(limit_us), _stream(stream)))

    def check_error(self, stream=None) -> None:
        _check(lib().nrc_check_error(self._h, _stream(stream)))


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t)
    return arr


class Batch:
    """Several caches served together: one persistent query launch, one training launch per step."""

    def __init__(self, caches):
        self.caches = list(caches)
        handles = (ctypes.c_void_p * len(self.caches))(*[c.handle for c in self.caches])
        h = ctypes.c_void_p()
        _check(lib().nrc_batch_create(handles, len(self.caches), ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().nrc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def infer(self, records, rgb, stream=None) -> None:
        n = (ctypes.c_int64 * len(records))(*[r.shape[0] for r in records])
        _check(lib().nrc_batch_infer(self._h, _ptr_array(records), n, _ptr_array(rgb), _stream(stream)))

    def train_step(self, pools, targets, batches, frame_seeds, step: int, losses=None, stream=None) -> None:
        k = len(pools)
        n_pool = (ctypes.c_int64 * k)(*[p.shape[0] for p in pools])
        bs = (ctypes.c_int64 * k)(*batches)
        fs = (ctypes.c_uint64 * k)(*[s & (2**64 - 1) for s in frame_seeds])
        lo = _ptr_array(losses) if losses is not None else None
        _check(lib().nrc_batch_train_step(self._h, _ptr_array(pools), _ptr_array(targets), n_pool, bs, fs, step, lo,
                                          _stream(stream)))

    def train_step_dev(self, pools, targets, batches, seeds_dev, step: int, losses=None, stream=None) -> None:
        """train_step with the frame seeds in a device tensor (int64 bits, one per cache), read when the kernel
        runs: the call is capturable in a CUDA graph with the query launch."""
        k = len(pools)
        n_pool = (ctypes.c_int64 * k)(*[p.shape[0] for p in pools])
        bs = (ctypes.c_int64 * k)(*batches)
        lo = _ptr_array(losses) if losses is not None else None
        _check(lib().nrc_batch_train_step_dev(self._h, _ptr_array(pools), _ptr_array(targets), n_pool, bs,
                                              _ptr(seeds_dev), step, lo, _stream(stream)))

    def set_unit_tiles(self, u: int) -> None:
        _check(lib().nrc_batch_set_unit_tiles(self._h, u))

    def set_train_tiles(self, t: int) -> None:
        _check(lib().nrc_batch_set_train_tiles(self._h, t))

    def autotune(self, records, rgb, stream=None) -> int:
        n = (ctypes.c_int64 * len(records))(*[r.shape[0] for r in records])
        chosen = ctypes.c_int32()
        _check(lib().nrc_batch_autotune(self._h, _ptr_array(records), n, _ptr_array(rgb), _stream(stream),
                                        ctypes.byref(chosen)))
        return chosen.value


class _BorrowedCache(Cache):
    """A cache handle owned elsewhere (a server's viewport): never destroyed from here."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def close(self) -> None:
        self._h = None


class _DeviceView:
    """A float32 device buffer owned by the library, viewable as a torch tensor."""

    def __init__(self, ptr: int, shape: tuple):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": "<f4", "data": (ptr, False), "version": 2,
                                         "strides": None}


def _view(ptr: int, shape: tuple):
    import torch

    return torch.as_tensor(_DeviceView(ptr, shape), device="cuda")


def now_ns() -> int:
    return lib().nrc_now_ns()


class Server:
    """Continuous-batching server of several viewports' caches (see include/nrc.h)."""

    def __init__(self, cache_cfg: Config | None = None, **kw):
        cfg = ServerConfig()
        lib().nrc_server_default_config(ctypes.byref(cfg))
        for k, v in kw.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.cache_cfg = cache_cfg if cache_cfg is not None else default_config(dtype="fp16")
        h = ctypes.c_void_p()
        _check(lib().nrc_server_create(ctypes.byref(cfg), ctypes.byref(self.cache_cfg), ctypes.byref(h)))
        self._h = h
        self._vp = {}

    def close(self) -> None:
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _check(lib().nrc_server_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_viewport(self, max_queries: int, n_pool: int, n_slots: int = 2, seed: int | None = None) -> int:
        """Admits a viewport (raises NrcError with status NRC_ERR_BUSY if it does not fit the budget)."""
        c = Config.from_buffer_copy(self.cache_cfg)
        if seed is not None:
            c.seed = seed
        vid = ctypes.c_int32()
        _check(lib().nrc_server_open_viewport(self._h, ctypes.byref(c), max_queries, n_pool, n_slots,
                                              ctypes.byref(vid)))
        self._vp[vid.value] = (max_queries, n_pool, n_slots)
        return vid.value

    def close_viewport(self, vid: int) -> None:
        _check(lib().nrc_server_close_viewport(self._h, vid))
        self._vp.pop(vid, None)

    def buffers(self, vid: int, slot: int):
        """(records [max_queries,16], rgb [max_queries,3], losses [train_steps]) of a slot, as device tensors."""
        r, g, l = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().nrc_server_viewport_buffers(self._h, vid, slot, ctypes.byref(r), ctypes.byref(g),
                                                 ctypes.byref(l)))
        mq = self._vp[vid][0]
        return (_view(r.value, (mq, 16)), _view(g.value, (mq, 3)), _view(l.value, (max(1, self.cfg.train_steps),)))

    def pool(self, vid: int):
        """(pool [n_pool,16], target [n_pool,3]) device tensors and the viewport's cache handle."""
        p, t, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().nrc_server_viewport_pool(self._h, vid, ctypes.byref(p), ctypes.byref(t), ctypes.byref(c)))
        n = self._vp[vid][1]
        return _view(p.value, (n, 16)), _view(t.value, (n, 3)), c.value

    def cache(self, vid: int) -> "Cache":
        """The viewport's cache (owned by the server; use get_state / set_state after drain)."""
        return _BorrowedCache(self.pool(vid)[2])

    def submit(self, vid: int, slot: int, n_queries: int, frame_seed: int, arrival_ns: int | None = None,
               tag: int = 0) -> bool:
        """Queues a frame; False if the slot's previous frame is still in flight."""
        st = lib().nrc_server_submit(self._h, vid, slot, n_queries, frame_seed & (2**64 - 1),
                                     now_ns() if arrival_ns is None else arrival_ns, tag)
        if st == NRC_ERR_BUSY:
            return False
        _check(st)
        return True

    def poll(self, max_out: int = 256, timeout_ms: int = 0) -> list:
        buf = (FrameDone * max_out)()
        n = ctypes.c_int32()
        _check(lib().nrc_server_poll(self._h, buf, max_out, timeout_ms, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    def pause(self, paused: bool = True) -> None:
        """Holds (or releases) the scheduler: held frames are batched together on release."""
        _check(lib().nrc_server_pause(self._h, int(bool(paused))))

    def drain(self) -> None:
        _check(lib().nrc_server_drain(self._h))

    def info(self) -> ServerInfo:
        out = ServerInfo()
        _check(lib().nrc_server_query(self._h, ctypes.byref(out)))
        return out


class _Paths(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("n_vertices", ctypes.c_int32), ("camera", ctypes.c_float * 3)]


class PathParams(ctypes.Structure):
    _fields_ = [("c", ctypes.c_float), ("tile", ctypes.c_int32), ("tile_ox", ctypes.c_int32),
                ("tile_oy", ctypes.c_int32), ("unbiased_phase", ctypes.c_int32), ("rr_survive", ctypes.c_float)]


def debug_fail_device_allocs(after: int, count: int) -> None:
    """Fault injection: after `after` more device allocations by the library,
    the next `count` fail as if out of memory; (0, 0) switches it off."""
    lib().nrc_debug_fail_device_allocs(int(after), int(count))


def paths_tile_count(width: int, height: int, tile: int) -> int:
    return lib().nrc_paths_tile_count(width, height, tile)


def paths_offsets_count(n_tiles: int) -> int:
    return lib().nrc_paths_offsets_count(n_tiles)


def paths_adapt_tile(tile: int, generated: int, target: int) -> int:
    return lib().nrc_paths_adapt_tile(tile, generated, target)


def _paths(vertices, width, height, camera):
    return _Paths(_ptr(vertices), width, height, vertices.shape[1], (ctypes.c_float * 3)(*camera))


def paths_terminate(vertices, width: int, height: int, camera, params: PathParams, stream=None, out=None):
    """(render_queries, render_emitted, render_throughput, tiles, tail_queries) as device tensors;
    `out` may hold these five tensors, preallocated (the tail queries of tiles without a
    training pixel are left as they are, so zero them once)."""
    import torch

    d = vertices.device
    P = width * height
    nt = paths_tile_count(width, height, params.tile)
    if out is None:
        out = (torch.empty((P, 16), device=d), torch.empty((P, 3), device=d), torch.empty((P, 3), device=d),
               torch.empty((nt, 4), dtype=torch.int32, device=d), torch.zeros((nt, 16), device=d))
    rq, em, tp, tiles, tq = out
    if rq.shape[0] < P or em.shape[0] < P or tp.shape[0] < P or tiles.shape[0] < nt or tq.shape[0] < nt:
        raise ValueError("paths_terminate: output tensors too small")
    ps = _paths(vertices, width, height, camera)
    _check(lib().nrc_paths_terminate(ctypes.byref(ps), ctypes.byref(params), _ptr(rq), _ptr(em), _ptr(tp),
                                     _ptr(tiles), _ptr(tq), _stream(stream)))
    return rq, em, tp, tiles, tq


def paths_records(vertices, width: int, height: int, camera, params: PathParams, tiles, tail_rgb, max_records: int,
                  stream=None, out=None):
    """(pool [max,16], targets [max,3], count device int64 [1]); `out` may hold
    (pool, targets, offsets [paths_offsets_count(n_tiles)] int64, count [1] int64), preallocated."""
    import torch

    d = vertices.device
    if out is None:
        out = (torch.zeros((max_records, 16), device=d), torch.zeros((max_records, 3), device=d),
               torch.empty(paths_offsets_count(tiles.shape[0]), dtype=torch.int64, device=d),
               torch.zeros(1, dtype=torch.int64, device=d))
    pool, tg, offsets, count = out
    if (pool.shape[0] < max_records or tg.shape[0] < max_records
            or offsets.shape[0] < paths_offsets_count(tiles.shape[0])):
        raise ValueError("paths_records: output tensors too small")
    ps = _paths(vertices, width, height, camera)
    _check(lib().nrc_paths_records(ctypes.byref(ps), ctypes.byref(params), _ptr(tiles), _ptr(tail_rgb), _ptr(pool),
                                   _ptr(tg), max_records, _ptr(offsets), _ptr(count), _stream(stream)))
    return pool, tg, count


def paths_composite(emitted, throughput, rgb, stream=None, out=None):
    import torch

    img = torch.empty_like(emitted) if out is None else out
    _check(lib().nrc_paths_composite(_ptr(emitted), _ptr(throughput), _ptr(rgb), emitted.shape[0], _ptr(img),
                                     _stream(stream)))
    return img
