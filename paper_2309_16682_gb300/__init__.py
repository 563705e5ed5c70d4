"""GB300-native V-family generators (arXiv 2309.16682): Python binding.

A thin ctypes layer over the C ABI of ``_build/libvmt.so`` (declared in
``include/vmt.h``).  It only marshals arguments: seeding, jump-ahead, twist,
tempering, interleave, conversion and stores all run in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing the calls raise.

    >>> import torch, paper_2309_16682_gb300 as vmt
    >>> g = vmt.VGenerator("mt32", lanes=16, seeds=[5489])
    >>> x = g.generate(1 << 20, "u32")          # torch.uint32 tensor on cuda
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

# The server keeps many streams busy at once (per batch slot one stream per
# variant's initialisation and one for generation).  CUDA multiplexes streams
# onto a fixed number of hardware work queues, 8 by default, and kernels of
# unrelated streams that share a queue wait for each other: a small request's
# launches then queue behind a long request's jump chain.  The count is read
# when the process creates its CUDA context, so it is set here, on import,
# unless the caller has chosen one (32 is CUDA's maximum).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvmt.so")
CACHE_DIR = os.path.join(HERE, "_cache")

VARIANTS = {"mt32": 0, "mt64": 1, "sfmt": 2}
DTYPES = {"u32": 0, "u64": 1, "f32": 2, "f64": 3}
UNITS = {0: 624, 1: 312, 2: 156}

VMT_OK, VMT_EINVAL, VMT_ENOMEM, VMT_ECUDA, VMT_ETIMEOUT, VMT_EBUSY, VMT_ESTATE = 0, -1, -2, -3, -4, -5, -6
VMT_ECANCELED = -7
VMT_INJECT_ALLOC = 1

_lib = None
_lock = threading.Lock()


class VMTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vmt error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libvmt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2309_16682_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        PP = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "vmt_init": (I, [PP, I, I, U64, U64, P]),
            "vmt_init_batch": (I, [PP, I, I, I64, P, P, P]),
            "vmt_jump": (I, [P, P, I64, P]),
            "vmt_jump_poly": (I, [I, U64, I, P, I64]),
            "vmt_prepare": (I, [I, P]),
            "vmt_generate": (I, [P, I64, I, P, P]),
            "vmt_generate_multi": (I, [P, I, P, P, P, P]),
            "vmt_generate_host": (I, [P, I64, I, P, P]),
            "vmt_state_bytes": (I64, [P]),
            "vmt_state_export": (I, [P, P, ctypes.c_size_t, P]),
            "vmt_state_import": (I, [P, P, ctypes.c_size_t, P]),
            "vmt_state_info": (I, [P, P, P, P, P]),
            "vmt_state_device_ptr": (P, [P]),
            "vmt_free": (None, [P]),
            "vmt_last_error": (ctypes.c_char_p, []),
            "vmt_set_cache_dir": (I, [ctypes.c_char_p]),
            "vmt_poly_minpoly": (I, [P, I64, P, I64]),
            "vmt_poly_mulmod": (I, [P, P, P, P, I64]),
            "vmt_poly_x2pow": (I, [P, I64, I, I, P]),
            "vmt_device_status": (I, [I]),
            "vmt_generate_ragged": (I, [P, P, I, P, P]),
            "vmt_batch_create": (I, [PP]),
            "vmt_batch_add": (I, [P, P, I64, I, P]),
            "vmt_batch_run": (I, [P, P]),
            "vmt_batch_run_graph": (I, [P, P]),
            "vmt_batch_clear": (I, [P]),
            "vmt_batch_destroy": (None, [P]),
            "vmt_server_create": (I, [PP, P]),
            "vmt_server_submit": (I, [P, P, P]),
            "vmt_server_poll": (I, [P, U64, P, P, P, P]),
            "vmt_server_wait": (I, [P, U64, I]),
            "vmt_server_release": (I, [P, U64]),
            "vmt_server_copy": (I, [P, U64, P, I64]),
            "vmt_server_stats": (I, [P, P]),
            "vmt_server_cancel": (I, [P, U64]),
            "vmt_server_next_done": (I, [P, I64, P]),
            "vmt_server_inject": (I, [P, I, I]),
            "vmt_selftest_wait": (I, [I64, P]),
            "vmt_scalar_create": (I, [PP, I, I, U64, U64, I, I64]),
            "vmt_scalar_next": (I, [P, P]),
            "vmt_scalar_take": (I, [P, I64, P]),
            "vmt_scalar_drain": (I, [P, I64, P]),
            "vmt_scalar_destroy": (None, [P]),
            "vmt_server_destroy": (None, [P]),
            "vmt_tune_set": (I, [I, I, I]),
            "vmt_tune_get": (I, [I, I]),
            "vmt_tune_save": (I, [ctypes.c_char_p]),
            "vmt_tune_load": (I, [ctypes.c_char_p]),
            "vmt_tune_jump_set": (I, [I, I64]),
            "vmt_measure_store_bw": (I, [I64, I, P, P]),
            "vmt_stream_generate": (I, [I, U64, U64, I64, I, P, P]),
            "vmt_tune_jump_get": (I64, [I]),
            "vmt_autotune": (I, [I, I, I64, I64, I, I, P, P, P]),
            "vmt_autotune_multi": (I, [I, I, I64, I, P, P, I, P, P, P]),
            "vmt_tune_kernels": (I, [I, I, P, I]),
            "vmt_tune_pass_cut": (I, [I, I, I, P]),
            "vmt_tune_jump_compact": (I, [I, I]),
            "vmt_tgfsr_jump": (I, [P, I64, P, P, I64, I, P]),
            "vmt_server_submit_many": (I, [P, P, I64, P]),
            "vmt_server_next_done_many": (I64, [P, I64, P, P, P, I64]),
            "vmt_server_release_many": (I, [P, P, I64]),
            "vmt_tgfsr_generate": (I, [P, I64, I, P, I64, P, P]),
            "vmt_tune_set_kernel": (I, [I, I, I]),
            "vmt_tune_get_kernel": (I, [I, I]),
            "vmt_autotune_grid": (I, [I, I, I64, I, P, P, I, P, P, I, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        os.makedirs(CACHE_DIR, exist_ok=True)
        L.vmt_set_cache_dir(CACHE_DIR.encode())
        _lib = L
        return L


def _check(rc: int) -> int:
    if rc < 0:
        raise VMTError(rc, lib().vmt_last_error().decode(errors="replace"))
    return rc


def _stream_handle(stream=None) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np_ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _torch_dtype(dtype: str):
    import torch
    return {"u32": torch.uint32, "u64": torch.uint64, "f32": torch.float32, "f64": torch.float64}[dtype]


class VGenerator:
    """``count`` V-family generators (one vmt_state) advancing in lock-step."""

    def __init__(self, variant: str, lanes: int, seeds, jumps=None, stream=None):
        self.variant = variant
        self.v = VARIANTS[variant]
        self.lanes = int(lanes)
        seeds = np.ascontiguousarray(np.atleast_1d(np.asarray(seeds, dtype=np.uint64)))
        self.count = int(seeds.size)
        js = None
        if jumps is not None:
            js = np.ascontiguousarray(np.broadcast_to(np.asarray(jumps, dtype=np.uint64), seeds.shape))
        h = ctypes.c_void_p()
        _check(lib().vmt_init_batch(ctypes.byref(h), self.v, self.lanes, self.count, _np_ptr(seeds),
                                    _np_ptr(js) if js is not None else None, _stream_handle(stream)))
        self._h = h

    # -- generation ---------------------------------------------------------
    def generate(self, n: int, dtype: str = "u32", out=None, stream=None):
        """Next n outputs per generator; returns a [count, n] tensor on the device."""
        import torch
        if out is None:
            out = torch.empty((self.count, n), dtype=_torch_dtype(dtype), device="cuda")
        _check(lib().vmt_generate(self._h, int(n), DTYPES[dtype], ctypes.c_void_p(out.data_ptr()),
                                  _stream_handle(stream)))
        return out

    def generate_multi(self, segments, outs=None, stream=None):
        """segments: [(n, dtype), ...] consecutive outputs fused into one pass."""
        import torch
        nseg = len(segments)
        if outs is None:
            outs = [torch.empty((self.count, n), dtype=_torch_dtype(dt), device="cuda") for n, dt in segments]
        counts = (ctypes.c_int64 * nseg)(*[int(n) for n, _ in segments])
        dts = (ctypes.c_int * nseg)(*[DTYPES[dt] for _, dt in segments])
        ptrs = (ctypes.c_void_p * nseg)(*[o.data_ptr() for o in outs])
        _check(lib().vmt_generate_multi(self._h, nseg, counts, dts, ptrs, _stream_handle(stream)))
        return outs

    def generate_host(self, n: int, dtype: str = "u32", out=None, stream=None):
        """Next n outputs per generator into host memory (numpy or pinned torch tensor)."""
        import torch
        if out is None:
            out = torch.empty((self.count, n), dtype=_torch_dtype(dtype), pin_memory=True)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        _check(lib().vmt_generate_host(self._h, int(n), DTYPES[dtype], ctypes.c_void_p(ptr), _stream_handle(stream)))
        return out

    def generate_ragged(self, n, dtype: str = "u32", outs=None, stream=None):
        """Generator g takes its next n[g] outputs; returns the list of tensors."""
        import torch
        n = [int(x) for x in n]
        assert len(n) == self.count
        if outs is None:
            outs = [torch.empty(max(k, 1), dtype=_torch_dtype(dtype), device="cuda")[:k] for k in n]
        na = np.ascontiguousarray(n, dtype=np.int64)
        ptrs = (ctypes.c_void_p * self.count)(*[o.data_ptr() for o in outs])
        _check(lib().vmt_generate_ragged(self._h, _np_ptr(na), DTYPES[dtype], ptrs, _stream_handle(stream)))
        return outs

    # -- jump / state ---------------------------------------------------------
    def jump(self, poly: np.ndarray, nbits: int | None = None, stream=None):
        poly = np.ascontiguousarray(poly, dtype=np.uint64)
        nb = int(nbits if nbits is not None else poly.size * 64)
        _check(lib().vmt_jump(self._h, _np_ptr(poly), nb, _stream_handle(stream)))

    def info(self):
        v, m = ctypes.c_int(), ctypes.c_int()
        c, p = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().vmt_state_info(self._h, ctypes.byref(v), ctypes.byref(m), ctypes.byref(c), ctypes.byref(p)))
        return dict(variant=v.value, lanes=m.value, count=c.value, block_pos=p.value)

    def export_state(self, stream=None) -> bytes:
        n = _check(lib().vmt_state_bytes(self._h))
        buf = np.empty(n, np.uint8)
        _check(lib().vmt_state_export(self._h, _np_ptr(buf), n, _stream_handle(stream)))
        return buf.tobytes()

    def import_state(self, blob: bytes, stream=None):
        buf = np.frombuffer(blob, np.uint8).copy()
        _check(lib().vmt_state_import(self._h, _np_ptr(buf), buf.size, _stream_handle(stream)))

    def device_states(self):
        """The combined states as a torch uint8 view-copy [count, bytes] (tests)."""
        import torch
        n = _check(lib().vmt_state_bytes(self._h))
        hdr = 48
        buf = np.empty(n, np.uint8)
        _check(lib().vmt_state_export(self._h, _np_ptr(buf), n, _stream_handle(None)))
        return buf[hdr:n - 8 * self.count].reshape(self.count, -1)

    def close(self):
        if getattr(self, "_h", None):
            lib().vmt_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several generator sets produced in one pass (vmt_batch_*)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().vmt_batch_create(ctypes.byref(h)))
        self._h = h
        self._keep = []

    def add(self, gen: VGenerator, n: int, dtype: str, out):
        _check(lib().vmt_batch_add(self._h, gen._h, int(n), DTYPES[dtype], ctypes.c_void_p(out.data_ptr())))
        self._keep.append((gen, out))

    def run(self, stream=None, graph: bool = False):
        f = lib().vmt_batch_run_graph if graph else lib().vmt_batch_run
        _check(f(self._h, _stream_handle(stream)))

    def clear(self):
        _check(lib().vmt_batch_clear(self._h))
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            lib().vmt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVER_QUEUED, SERVER_RUNNING, SERVER_DONE = 0, 1, 2


class _ServerConfig(ctypes.Structure):
    _fields_ = [("state_budget_bytes", ctypes.c_int64), ("output_budget_bytes", ctypes.c_int64),
                ("max_batch", ctypes.c_int), ("reserve", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("lanes", ctypes.c_int), ("dtype", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("jump", ctypes.c_uint64), ("n", ctypes.c_int64)]


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("queued", "in_flight_batches", "batches", "completed", "failed",
                                             "bytes_out", "state_bytes_in_use", "output_bytes_in_use",
                                             "peak_state_bytes", "peak_output_bytes")] + \
        [(n, ctypes.c_double) for n in ("host_launch_s", "init_gpu_s", "batch_gpu_s")] + [("cancelled", ctypes.c_int64)] + \
        [(n, ctypes.c_int64) for n in ("express_batches", "express_completed")] + \
        [(n, ctypes.c_double) for n in ("queued_s", "running_s", "express_queued_s", "express_running_s",
                                        "express_init_gpu_s", "express_batch_gpu_s")]


class Server:
    """Continuous-batching request server (vmt_server_*)."""

    def __init__(self, state_budget: int = 8 << 30, output_budget: int = 32 << 30, max_batch: int = 4096,
                 reserve: bool = False):
        cfg = _ServerConfig(int(state_budget), int(output_budget), int(max_batch), int(bool(reserve)))
        h = ctypes.c_void_p()
        _check(lib().vmt_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h

    def submit(self, variant: str, lanes: int, dtype: str, seed: int, jump: int, n: int) -> int:
        r = _Request(VARIANTS[variant], int(lanes), DTYPES[dtype], int(seed) & (2**64 - 1), int(jump) & (2**64 - 1),
                     int(n))
        rid = ctypes.c_uint64(0)
        _check(lib().vmt_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def poll(self, rid: int):
        st, ptr, nb, lat = ctypes.c_int(), ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().vmt_server_poll(self._h, rid, ctypes.byref(st), ctypes.byref(ptr), ctypes.byref(nb),
                                     ctypes.byref(lat)))
        return st.value, ptr.value, nb.value, lat.value

    def wait(self, rid: int, timeout_ms: int = 60000) -> int:
        """0 when done; raises VMTError (VMT_ETIMEOUT, or the request's own error)."""
        return _check(lib().vmt_server_wait(self._h, rid, int(timeout_ms)))

    def copy(self, rid: int, dtype: str) -> np.ndarray:
        st, ptr, nb, lat = self.poll(rid)
        npdt = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32, "f64": np.float64}[dtype]
        out = np.empty(nb // np.dtype(npdt).itemsize, npdt)
        _check(lib().vmt_server_copy(self._h, rid, _np_ptr(out), nb))
        return out

    def release(self, rid: int) -> None:
        _check(lib().vmt_server_release(self._h, rid))

    def next_done(self, timeout_us: int = 0):
        """Id of the next request that finished (in completion order), or None
        if none finished within timeout_us."""
        rid = ctypes.c_uint64(0)
        rc = lib().vmt_server_next_done(self._h, int(timeout_us), ctypes.byref(rid))
        if rc == VMT_ETIMEOUT:
            return None
        _check(rc)
        return rid.value

    @staticmethod
    def requests(rows) -> "ctypes.Array":
        """A request array for submit_many from (variant, lanes, dtype, seed,
        jump, n) rows (built once, ahead of the submissions)."""
        arr = (_Request * len(rows))()
        for i, (v, m, dt, seed, jump, n) in enumerate(rows):
            arr[i] = _Request(VARIANTS[v], int(m), DTYPES[dt], int(seed) & (2**64 - 1), int(jump) & (2**64 - 1),
                              int(n))
        return arr

    def submit_many(self, reqs: "ctypes.Array", first: int, count: int) -> np.ndarray:
        """Submit reqs[first:first + count] in one call; returns their ids."""
        ids = np.empty(count, np.uint64)
        if count:
            ptr = ctypes.cast(ctypes.byref(reqs, first * ctypes.sizeof(_Request)), ctypes.c_void_p)
            _check(lib().vmt_server_submit_many(self._h, ptr, int(count), _np_ptr(ids)))
        return ids

    def next_done_many(self, timeout_us: int = 0, cap: int = 4096):
        """Up to cap finished requests in completion order: (ids, status,
        latency seconds); empty arrays when none finished within timeout_us."""
        ids = np.empty(cap, np.uint64)
        st = np.empty(cap, np.int32)
        lat = np.empty(cap, np.float64)
        k = lib().vmt_server_next_done_many(self._h, int(timeout_us), _np_ptr(ids), _np_ptr(st), _np_ptr(lat), int(cap))
        if k < 0:
            _check(int(k))
        return ids[:k], st[:k], lat[:k]

    def release_many(self, ids: np.ndarray) -> None:
        ids = np.ascontiguousarray(ids, np.uint64)
        _check(lib().vmt_server_release_many(self._h, _np_ptr(ids), int(ids.size)))

    def cancel(self, rid: int) -> None:
        """Withdraw a queued request (its status becomes VMT_ECANCELED)."""
        _check(lib().vmt_server_cancel(self._h, rid))

    def inject_alloc_failures(self, count: int) -> None:
        """Fault injection: the next `count` output allocations fail."""
        _check(lib().vmt_server_inject(self._h, VMT_INJECT_ALLOC, int(count)))

    def stats(self) -> dict:
        c = _Counters()
        _check(lib().vmt_server_stats(self._h, ctypes.byref(c)))
        return {n: getattr(c, n) for n, _ in _Counters._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().vmt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_status(reset: bool = False) -> int:
    """0, or raises VMTError(VMT_ETIMEOUT) if a kernel gave up a bounded wait."""
    return _check(lib().vmt_device_status(1 if reset else 0))


def tune_set(variant: str, lanes: int, threads: int) -> None:
    _check(lib().vmt_tune_set(VARIANTS[variant], int(lanes), int(threads)))


def tune_jump(variant: str, split_below: int | None = None) -> int:
    """Jump launches of the variant with fewer lane-jumps than split_below use
    one CTA per lane-jump; returns the value in force before the call (None:
    just read)."""
    old = int(lib().vmt_tune_jump_get(VARIANTS[variant]))
    if split_below is not None:
        _check(lib().vmt_tune_jump_set(VARIANTS[variant], int(split_below)))
    return old


def tune_jump_compact(variant: str, on: bool | None = None) -> bool:
    """Every jump launch of the variant in the compact CTA form (on=True), or
    the default choice (False); returns the setting before the call (None:
    just read)."""
    return bool(_check(lib().vmt_tune_jump_compact(VARIANTS[variant], -1 if on is None else int(bool(on)))))


class Tgfsr(ctypes.Structure):
    """Parameters of a twisted GFSR with run-time constants (vmt_tgfsr)."""
    _fields_ = [("w", ctypes.c_int), ("n", ctypes.c_int), ("m", ctypes.c_int), ("r", ctypes.c_int),
                ("a", ctypes.c_uint32), ("temper", ctypes.c_int), ("u", ctypes.c_int), ("s", ctypes.c_int),
                ("t", ctypes.c_int), ("l", ctypes.c_int), ("d", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("c", ctypes.c_uint32)]


def tgfsr_jump(params: Tgfsr, states, poly: np.ndarray, nbits: int | None = None, kernel: str = "warp",
               stream=None) -> None:
    """Every state (a uint32 tensor [count, n] on the GPU) by c(F) X (Sec. 3.1)."""
    poly = np.ascontiguousarray(poly, dtype=np.uint64)
    nb = poly.size * 64 if nbits is None else int(nbits)
    _check(lib().vmt_tgfsr_jump(ctypes.byref(params), int(states.shape[0]), ctypes.c_void_p(states.data_ptr()),
                                _np_ptr(poly), nb, {"warp": 0, "cta": 1}[kernel], _stream_handle(stream)))


def tgfsr_generate(params: Tgfsr, states, lanes: int, n: int, out=None, stream=None):
    """n outputs of every state, interleaved over `lanes` (tensor [groups, n * lanes])."""
    import torch
    groups = int(states.shape[0]) // int(lanes)
    if out is None:
        out = torch.empty((groups, n * lanes), dtype=torch.int32, device=states.device)   # uint32 words
    _check(lib().vmt_tgfsr_generate(ctypes.byref(params), int(states.shape[0]), int(lanes),
                                    ctypes.c_void_p(states.data_ptr()), int(n), ctypes.c_void_p(out.data_ptr()),
                                    _stream_handle(stream)))
    return out


def tune_save(path: str) -> None:
    """Write the tuning table (entries that differ from the defaults)."""
    _check(lib().vmt_tune_save(os.fspath(path).encode()))


def tune_load(path: str) -> None:
    """Apply a tuning table written by tune_save."""
    _check(lib().vmt_tune_load(os.fspath(path).encode()))


def tune_cache_path() -> str:
    """Where the autotuner's table is kept for the current GPU model."""
    import re
    import torch
    name = re.sub(r"[^A-Za-z0-9]+", "_", torch.cuda.get_device_name())
    return os.path.join(CACHE_DIR, f"tune_{name}.txt")


def tune_get(variant: str, lanes: int) -> int:
    return _check(lib().vmt_tune_get(VARIANTS[variant], int(lanes)))


FORMS = {0: "phase", 1: "chain", 2: "inplace"}


def tune_kernels(variant: str, lanes: int) -> list[dict]:
    """The compiled generation-kernel configurations of (variant, lanes), in
    index order (entry 0 is the default)."""
    n = _check(lib().vmt_tune_kernels(VARIANTS[variant], int(lanes), None, 0))
    buf = (ctypes.c_int * max(1, 4 * n))()
    _check(lib().vmt_tune_kernels(VARIANTS[variant], int(lanes), buf, n))
    return [{"form": FORMS[buf[4 * i]], "lanes_per_cta": buf[4 * i + 1], "threads": buf[4 * i + 2],
             "store_bytes": buf[4 * i + 3]} for i in range(n)]


def tune_pass_cut(variant: str, lanes: int, index: int) -> dict:
    """The pass schedule of a phase-form or in-place configuration
    (vmt_tune_pass_cut), in vectors of one row's VW lane words."""
    out = (ctypes.c_int * 8)()
    _check(lib().vmt_tune_pass_cut(VARIANTS[variant], int(lanes), int(index), out))
    keys = ("vectors", "step", "row_vectors", "n_minus_m_vectors", "m_vectors", "threads", "in_place", "early")
    return dict(zip(keys, list(out)))


def tune_set_kernel(variant: str, lanes: int, index: int) -> None:
    _check(lib().vmt_tune_set_kernel(VARIANTS[variant], int(lanes), int(index)))


def tune_get_kernel(variant: str, lanes: int) -> int:
    return _check(lib().vmt_tune_get_kernel(VARIANTS[variant], int(lanes)))


def autotune_grid(variant: str, lanes: int, count: int, segments, reps: int = 3, stream=None):
    """Time every compiled configuration of (variant, lanes) on `count`
    generators producing `segments` [(n per generator, dtype), ...]; selects
    the fastest.  Returns (best index, [ms per call of each configuration])."""
    cands = tune_kernels(variant, lanes)
    ms = (ctypes.c_double * max(1, len(cands)))()
    best = ctypes.c_int(0)
    counts = (ctypes.c_int64 * len(segments))(*[int(n) for n, _ in segments])
    dts = (ctypes.c_int * len(segments))(*[DTYPES[d] for _, d in segments])
    _check(lib().vmt_autotune_grid(VARIANTS[variant], int(lanes), int(count), len(segments), counts, dts, int(reps),
                                   _stream_handle(stream), ms, len(cands), ctypes.byref(best)))
    return best.value, [float(ms[i]) for i in range(len(cands))]


def autotune(variant: str, lanes: int, count: int, n_per_gen: int, dtype: str = "u32", reps: int = 3, stream=None,
             segments=None):
    """Time every compiled CTA size and keep the fastest; returns (threads, ms
    per call).  `segments` [(n, dtype), ...] times that fused output mix
    instead of n_per_gen outputs of one type."""
    t = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    if segments:
        counts = (ctypes.c_int64 * len(segments))(*[int(n) for n, _ in segments])
        dts = (ctypes.c_int * len(segments))(*[DTYPES[d] for _, d in segments])
        _check(lib().vmt_autotune_multi(VARIANTS[variant], int(lanes), int(count), len(segments), counts, dts,
                                        int(reps), _stream_handle(stream), ctypes.byref(t), ctypes.byref(ms)))
    else:
        _check(lib().vmt_autotune(VARIANTS[variant], int(lanes), int(count), int(n_per_gen), DTYPES[dtype],
                                  int(reps), _stream_handle(stream), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def stream_generate(variant: str, seed: int, n: int, dtype: str = "u32", jump: int = 0, out=None, stream=None):
    """The base generator's own stream (M = 1) from offset `jump`, n outputs,
    generated in parallel chunks (vmt_stream_generate)."""
    import torch
    if out is None:
        out = torch.empty(max(int(n), 1), dtype=_torch_dtype(dtype), device="cuda")[:int(n)]
    _check(lib().vmt_stream_generate(VARIANTS[variant], int(seed) & (2**64 - 1), int(jump) & (2**64 - 1), int(n),
                                     DTYPES[dtype], ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


class ScalarGenerator:
    """Buffered scalar queries on the host from one V-generator
    (vmt_scalar_*): next() returns one output, take(n) the next n."""

    def __init__(self, variant: str, lanes: int, seed: int, jump: int = 0, dtype: str = "u32",
                 buffer_outputs: int = 1 << 20):
        h = ctypes.c_void_p()
        _check(lib().vmt_scalar_create(ctypes.byref(h), VARIANTS[variant], int(lanes), int(seed) & (2**64 - 1),
                                       int(jump) & (2**64 - 1), DTYPES[dtype], int(buffer_outputs)))
        self._h = h
        self.dtype = dtype
        self._np = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32, "f64": np.float64}[dtype]

    def next(self):
        v = np.zeros(1, self._np)
        _check(lib().vmt_scalar_next(self._h, _np_ptr(v)))
        return v[0]

    def take(self, n: int) -> np.ndarray:
        out = np.empty(int(n), self._np)
        _check(lib().vmt_scalar_take(self._h, int(n), _np_ptr(out)))
        return out

    def drain(self, count: int) -> int:
        c = ctypes.c_uint64(0)
        _check(lib().vmt_scalar_drain(self._h, int(count), ctypes.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "_h", None):
            lib().vmt_scalar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_wait(limit_ns: int = 1_000_000) -> tuple[int, int]:
    """Run a bounded device wait that nothing satisfies; returns (status,
    elapsed ns) -- status VMT_ETIMEOUT when the wait gave up as designed."""
    el = ctypes.c_int64(0)
    rc = lib().vmt_selftest_wait(int(limit_ns), ctypes.byref(el))
    if rc not in (VMT_OK, VMT_ETIMEOUT):
        _check(rc)
    return rc, el.value


def measure_store_bw(nbytes: int = 8 << 30, reps: int = 5, stream=None) -> float:
    """HBM write bandwidth of a store-only kernel, GB/s (best of reps)."""
    out = ctypes.c_double(0.0)
    _check(lib().vmt_measure_store_bw(int(nbytes), int(reps), ctypes.byref(out), _stream_handle(stream)))
    return out.value


def prepare(variant: str, stream=None) -> None:
    """Build the variant's polynomial tables now instead of on first use."""
    _check(lib().vmt_prepare(VARIANTS[variant], _stream_handle(stream)))


def jump_poly(variant: str, d: int, log2_extra: int = 0) -> np.ndarray:
    out = np.zeros(320, np.uint64)
    n = _check(lib().vmt_jump_poly(VARIANTS[variant], int(d), int(log2_extra), _np_ptr(out), out.size))
    return out[:n].copy()


def poly_minpoly(bits: np.ndarray) -> tuple[int, np.ndarray]:
    """Berlekamp-Massey on a 0/1 array (host helper of the library)."""
    b = np.asarray(bits, dtype=np.uint8)
    packed = np.zeros((b.size + 63) // 64, np.uint64)
    idx = np.nonzero(b)[0]
    np.bitwise_or.at(packed, idx // 64, np.left_shift(np.uint64(1), (idx % 64).astype(np.uint64)))
    mu = np.zeros(packed.size + 2, np.uint64)
    d = _check(lib().vmt_poly_minpoly(_np_ptr(packed), b.size, _np_ptr(mu), mu.size))
    return d, mu


def poly_mulmod(a: np.ndarray, b: np.ndarray, mu: np.ndarray) -> np.ndarray:
    nw = mu.size
    a = np.ascontiguousarray(a[:nw], np.uint64)
    b = np.ascontiguousarray(b[:nw], np.uint64)
    mu = np.ascontiguousarray(mu, np.uint64)
    out = np.zeros(nw, np.uint64)
    _check(lib().vmt_poly_mulmod(_np_ptr(a), _np_ptr(b), _np_ptr(mu), _np_ptr(out), nw))
    return out


def poly_x2pow(mu: np.ndarray, q_lo: int, q_hi: int) -> np.ndarray:
    mu = np.ascontiguousarray(mu, np.uint64)
    out = np.zeros((q_hi - q_lo + 1, mu.size), np.uint64)
    _check(lib().vmt_poly_x2pow(_np_ptr(mu), mu.size, q_lo, q_hi, _np_ptr(out)))
    return out
