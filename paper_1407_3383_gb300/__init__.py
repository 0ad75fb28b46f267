"""GB300 (sm_103a) exact modular NTT library: Python binding of libgbntt.so.

Argument marshalling only: every step of every transform and product runs in
the library's CUDA kernels.  Device buffers are torch tensors (uint32 words
for p < 2^32, uint64 words for 2^32 <= p < 2^62); streams are torch CUDA
streams.  The binding never computes a result itself and never falls back to
another implementation: if the shared library is missing, every call raises.

The calls and their semantics are those declared in include/gbntt.h, after
van der Hoeven, Lecerf and Quintin, "Modular SIMD arithmetic in Mathemagix"
(2014): the transform of Section 5.1, the polynomial product of Section 5.2
and the modular products of Sections 2-3.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libgbntt.so")
HEADER = os.path.join(ROOT, "include", "gbntt.h")

NTT_OK = 0
NTT_FLAG_PLAIN = 0x1
NTT_FLAG_CHECK = 0x2
NTT_FLAG_FP64 = 0x4
NTT_SCHED_FUSED = 0
NTT_SCHED_PLAIN = 1
NTT_MM_BARRETT = 0
NTT_MM_SHOUP = 1
NTT_MM_MONTGOMERY = 2
NTT_MM_FMA = 3
NTT_MM_MONT_FIXED = 4
NTT_MM_MONT_PRODUCT = 5
NTT_MM_ADD = 6
NTT_MM_SUB = 7
NTT_MM_MONT_FIXED_W = 8
NTT_MM_MONT_PRODUCT_W = 9
NTT_BATCH_DIRECT = 0
NTT_BATCH_STREAMS = 1
NTT_BATCH_GRAPH = 2
NTT_REQ_INTMUL = 0
NTT_REQ_POLYMUL = 1
NTT_REQ_DEVICE = 0x1
NTT_PROBE_IMAD = 0
NTT_PROBE_ALU = 1
NTT_PROBE_MIXED = 2
NTT_PROBE_WIDE = 3

_lock = threading.Lock()
_lib = None

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t
_vp = ctypes.c_void_p
_int = ctypes.c_int
_uint = ctypes.c_uint


class NttError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _load()
        name = lib.ntt_status_str(status).decode()
        detail = lib.ntt_last_error().decode()
        super().__init__(f"{where}: {name} ({status}) {detail}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("p", _u64), ("g", _u64), ("omega", _u64), ("omega_inv", _u64),
                ("n_inv", _u64), ("log2n", _u32), ("word_bytes", _u32), ("v2", _u32),
                ("tile_max_log", _u32)]


def header_functions() -> list[str]:
    """Names of every function include/gbntt.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgbntt.so is not built ({LIB_PATH}); "
                               "run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "ntt_find_prime": (_int, [_uint, _uint, _uint, ctypes.POINTER(_u64)]),
            "ntt_root_of_unity": (_int, [_u64, _uint, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
            "ntt_fixed_companion": (_int, [_u64, _uint, _uint, _vp, _vp, _sz]),
            "ntt_plan_create": (_int, [_u64, _uint, _uint, ctypes.POINTER(_vp)]),
            "ntt_plan_destroy": (_int, [_vp]),
            "ntt_plan_get_info": (_int, [_vp, ctypes.POINTER(PlanInfo)]),
            "ntt_forward": (_int, [_vp, _vp, _sz, _vp]),
            "ntt_inverse": (_int, [_vp, _vp, _sz, _vp]),
            "polymul_workspace_size": (_sz, [_vp, _sz, _uint]),
            "polymul_mod_p_batch": (_int, [_vp, _vp, _sz, _vp, _sz, _sz, _vp, _uint, _vp, _sz, _vp]),
            "polymul_mod_p": (_int, [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp]),
            "polymul_mod_p_batch_static": (_int, [_vp, _vp, _sz, _vp, _sz, _sz, _vp, _vp]),
            "polymul_host_stage_size": (_sz, [_vp, _sz, _sz, _sz]),
            "polymul_mod_p_batch_host": (_int, [_vp, _vp, _sz, _vp, _sz, _sz, _vp, _sz, _vp, _sz, _vp]),
            "ntt_modmul_vec": (_int, [_u64, _uint, _uint, _vp, _vp, _vp, _vp, _sz, _vp]),
            "ntt_modmul_rate": (_int, [_u64, _uint, _uint, _int, ctypes.POINTER(ctypes.c_double)]),
            "polymat_workspace_size": (_sz, [_vp, _uint]),
            "polymat_mul": (_int, [_vp, _vp, _vp, _uint, _sz, _vp, _vp, _sz, _vp]),
            "polymul_batch_plan_create": (_int, [_vp, _uint, _vp, _sz, _uint, ctypes.POINTER(_vp)]),
            "polymul_batch_plan_destroy": (_int, [_vp]),
            "polymul_batch_workspace_size": (_sz, [_vp]),
            "polymul_batch_run": (_int, [_vp, _vp, _vp, _vp, _vp, _sz, _uint, _vp]),
            "ntt_autotune": (_int, [_vp, _sz, _vp, ctypes.POINTER(ctypes.c_float)]),
            "ntt_tune_get": (_int, [_uint, _uint, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                    ctypes.POINTER(_int)]),
            "ntt_tune_export": (_int, [ctypes.c_char_p, _sz, ctypes.POINTER(_sz)]),
            "ntt_tune_import": (_int, [ctypes.c_char_p]),
            "ntt_tune_reset": (_int, []),
            "ntt_device_status": (_int, []),
            "ntt_int_probe": (_int, [_uint, _int, _int, _int, _vp, ctypes.POINTER(ctypes.c_double)]),
            "ntt_profile_begin": (_int, []),
            "ntt_profile_end": (_int, [_int, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(_int)]),
            "ntt_server_create": (_int, [_vp, ctypes.POINTER(_vp)]),
            "ntt_server_submit": (_int, [_vp, _uint, _uint, _vp, _sz, _vp, _sz, _vp, _uint,
                                         ctypes.POINTER(_u64)]),
            "ntt_server_poll": (_int, [_vp, _u64, ctypes.POINTER(_int),
                                       ctypes.POINTER(ctypes.c_double)]),
            "ntt_server_wait": (_int, [_vp, _u64, _int, ctypes.POINTER(ctypes.c_double)]),
            "ntt_server_release": (_int, [_vp, _u64]),
            "ntt_server_stats": (_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                        ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
            "ntt_server_destroy": (_int, [_vp]),
            "intmul_plan_create": (_int, [_sz, ctypes.POINTER(_vp)]),
            "intmul_plan_destroy": (_int, [_vp]),
            "intmul_workspace_size": (_sz, [_vp, _sz, _sz]),
            "intmul_crt": (_int, [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp]),
            "intmat_workspace_size": (_sz, [_vp, _uint, _sz, _sz]),
            "intmat_mul": (_int, [_vp, _vp, _sz, _vp, _sz, _uint, _vp, _vp, _sz, _vp]),
            "ntt_status_str": (ctypes.c_char_p, [_int]),
            "ntt_last_error": (ctypes.c_char_p, []),
            "ntt_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def lib():
    return _load()


def _check(status: int, where: str):
    if status != NTT_OK:
        raise NttError(status, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- host planning

def ntt_find_prime(bits: int, min_l: int, index: int) -> int:
    out = _u64()
    _check(_load().ntt_find_prime(bits, min_l, index, ctypes.byref(out)), "ntt_find_prime")
    return out.value


def ntt_root_of_unity(p: int, log2n: int) -> tuple[int, int]:
    g, w = _u64(), _u64()
    _check(_load().ntt_root_of_unity(p, log2n, ctypes.byref(g), ctypes.byref(w)), "ntt_root_of_unity")
    return g.value, w.value


def ntt_fixed_companion(p: int, kind: int, word_bytes: int, y):
    """Host companions (numpy uint64 in, numpy uint64 out)."""
    import numpy as np
    y = np.ascontiguousarray(np.asarray(y, dtype=np.uint64))
    out = np.empty_like(y)
    _check(_load().ntt_fixed_companion(p, kind, word_bytes, y.ctypes.data, out.ctypes.data,
                                       y.size), "ntt_fixed_companion")
    return out


# ---------------------------------------------------------------- plans

class Plan:
    """An ntt_plan: modulus p, transform length 2^log2n, device tables."""

    def __init__(self, p: int, log2n: int, flags: int = 0):
        h = _vp()
        _check(_load().ntt_plan_create(p, log2n, flags, ctypes.byref(h)), "ntt_plan_create")
        self.handle = h.value
        info = PlanInfo()
        _check(_load().ntt_plan_get_info(self.handle, ctypes.byref(info)), "ntt_plan_get_info")
        self.info = info
        self.p = info.p
        self.log2n = info.log2n
        self.n = 1 << info.log2n
        self.word_bytes = info.word_bytes
        self.omega = info.omega

    @property
    def dtype(self):
        import torch
        return torch.uint32 if self.word_bytes == 4 else torch.uint64

    def close(self):
        if getattr(self, "handle", None):
            _load().ntt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ntt_plan_create(p: int, log2n: int, flags: int = 0) -> Plan:
    return Plan(p, log2n, flags)


def ntt_forward(plan: Plan, data, batch: int | None = None, stream=None):
    batch = data.numel() // plan.n if batch is None else batch
    _check(_load().ntt_forward(plan.handle, _ptr(data), batch, _stream(stream)), "ntt_forward")


def ntt_inverse(plan: Plan, data, batch: int | None = None, stream=None):
    batch = data.numel() // plan.n if batch is None else batch
    _check(_load().ntt_inverse(plan.handle, _ptr(data), batch, _stream(stream)), "ntt_inverse")


def polymul_workspace_size(plan: Plan, batch: int, schedule: int = NTT_SCHED_FUSED) -> int:
    return int(_load().polymul_workspace_size(plan.handle, batch, schedule))


def polymul_mod_p_batch(plan: Plan, a, na: int, b, nb: int, batch: int, c,
                        schedule: int = NTT_SCHED_FUSED, ws=None, ws_bytes: int | None = None,
                        stream=None):
    if ws_bytes is None:
        ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_load().polymul_mod_p_batch(plan.handle, _ptr(a), na, _ptr(b), nb, batch, _ptr(c),
                                       schedule, _ptr(ws), ws_bytes, _stream(stream)),
           "polymul_mod_p_batch")


def polymul_mod_p(plan: Plan, a, na: int, b, nb: int, c, ws=None, ws_bytes: int | None = None,
                  stream=None):
    if ws_bytes is None:
        ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_load().polymul_mod_p(plan.handle, _ptr(a), na, _ptr(b), nb, _ptr(c), _ptr(ws),
                                 ws_bytes, _stream(stream)), "polymul_mod_p")


def polymul_mod_p_batch_static(plan: Plan, a, na: int, b, nb: int, batch: int, c, stream=None):
    """polymul_mod_p_batch (fused) with the library's fixed scratch array:
    for callers that cannot allocate device memory (see include/gbntt.h)."""
    _check(_load().polymul_mod_p_batch_static(plan.handle, _ptr(a), na, _ptr(b), nb, batch,
                                              _ptr(c), _stream(stream)),
           "polymul_mod_p_batch_static")


def ntt_modmul_vec(p: int, kind: int, word_bytes: int, x, y, yc, z, n: int | None = None,
                   stream=None):
    n = x.numel() if n is None else n
    _check(_load().ntt_modmul_vec(p, kind, word_bytes, _ptr(x), _ptr(y), _ptr(yc), _ptr(z), n,
                                  _stream(stream)), "ntt_modmul_vec")


# ---------------------------------------------------------------- polynomial matrices

def polymat_workspace_size(plan: Plan, n: int) -> int:
    return int(_load().polymat_workspace_size(plan.handle, n))


def polymat_mul(plan: Plan, A, B, n: int, d: int, C, ws, stream=None):
    ws_bytes = ws.numel() * ws.element_size()
    _check(_load().polymat_mul(plan.handle, _ptr(A), _ptr(B), n, d, _ptr(C), _ptr(ws), ws_bytes,
                               _stream(stream)), "polymat_mul")


# ---------------------------------------------------------------- uneven batches

class PolymulDesc(ctypes.Structure):
    _fields_ = [("a_off", _u64), ("b_off", _u64), ("c_off", _u64), ("na", _u32), ("nb", _u32),
                ("prime", _u32), ("reserved", _u32)]


class BatchPlan:
    """A polymul_batch_plan over `primes` for products given as arrays of
    operand lengths na, nb and modulus indices; operands and outputs are laid
    out back to back in the order given (offsets in words)."""

    def __init__(self, primes, na, nb, prime_idx):
        import numpy as np
        na = np.asarray(na, dtype=np.int64)
        nb = np.asarray(nb, dtype=np.int64)
        pi = np.asarray(prime_idx, dtype=np.int64)
        count = na.size
        nc = na + nb - 1
        self.a_off = np.concatenate([[0], np.cumsum(na)[:-1]]).astype(np.int64)
        self.b_off = np.concatenate([[0], np.cumsum(nb)[:-1]]).astype(np.int64)
        self.c_off = np.concatenate([[0], np.cumsum(nc)[:-1]]).astype(np.int64)
        self.na, self.nb, self.nc, self.prime_idx = na, nb, nc, pi
        self.a_words, self.b_words, self.c_words = int(na.sum()), int(nb.sum()), int(nc.sum())
        descs = (PolymulDesc * max(1, count))()
        for t in range(count):
            descs[t] = PolymulDesc(int(self.a_off[t]), int(self.b_off[t]), int(self.c_off[t]),
                                   int(na[t]), int(nb[t]), int(pi[t]), 0)
        arr = (_u64 * len(primes))(*[int(p) for p in primes])
        h = _vp()
        _check(_load().polymul_batch_plan_create(ctypes.cast(arr, _vp), len(primes),
                                                 ctypes.cast(descs, _vp), count, 0, ctypes.byref(h)),
               "polymul_batch_plan_create")
        self.handle = h.value
        self.primes = [int(p) for p in primes]
        self.word_bytes = 8 if max(self.primes) >> 32 else 4
        self.count = count

    def workspace_size(self) -> int:
        return int(_load().polymul_batch_workspace_size(self.handle))

    def run(self, a, b, c, ws, mode: int = NTT_BATCH_GRAPH, stream=None):
        ws_bytes = ws.numel() * ws.element_size()
        _check(_load().polymul_batch_run(self.handle, _ptr(a), _ptr(b), _ptr(c), _ptr(ws), ws_bytes,
                                         mode, _stream(stream)), "polymul_batch_run")

    def close(self):
        if getattr(self, "handle", None):
            _load().polymul_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------- serving loop

class ServerConfig(ctypes.Structure):
    _fields_ = [("max_limbs", _sz), ("mem_bytes", _sz), ("slots", _uint), ("reserved", _uint)]


class Server:
    """ntt_server: continuous batching of integer / polynomial products."""

    def __init__(self, max_limbs: int, mem_bytes: int, slots: int = 4):
        cfg = ServerConfig(max_limbs, mem_bytes, slots, 0)
        h = _vp()
        _check(_load().ntt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ntt_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, kind: int, a, b, c, prime: int = 0, flags: int = 0, na=None, nb=None) -> int:
        """a, b, c: tensors (pinned host, or device with NTT_REQ_DEVICE)."""
        na = a.numel() if na is None else na
        nb = b.numel() if nb is None else nb
        rid = _u64()
        _check(_load().ntt_server_submit(self.handle, kind, prime, _ptr(a), na, _ptr(b), nb, _ptr(c),
                                         flags, ctypes.byref(rid)), "ntt_server_submit")
        self._keep[rid.value] = (a, b, c)
        return rid.value

    def poll(self, rid: int):
        st, lat = _int(), ctypes.c_double()
        _check(_load().ntt_server_poll(self.handle, rid, ctypes.byref(st), ctypes.byref(lat)),
               "ntt_server_poll")
        return st.value, lat.value

    def wait(self, rid: int, timeout_ms: int = 60000) -> float:
        lat = ctypes.c_double()
        _check(_load().ntt_server_wait(self.handle, rid, timeout_ms, ctypes.byref(lat)), "ntt_server_wait")
        return lat.value

    def release(self, rid: int):
        _check(_load().ntt_server_release(self.handle, rid), "ntt_server_release")
        self._keep.pop(rid, None)

    def stats(self):
        v = [_u64() for _ in range(4)]
        _check(_load().ntt_server_stats(self.handle, *[ctypes.byref(x) for x in v]), "ntt_server_stats")
        return dict(zip(["completed", "pending", "running", "peak_inflight"], [x.value for x in v]))

    def close(self):
        if getattr(self, "handle", None):
            _load().ntt_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------- autotuning

def ntt_autotune(plan: Plan, batch: int, stream=None) -> float:
    best = ctypes.c_float()
    _check(_load().ntt_autotune(plan.handle, batch, _stream(stream), ctypes.byref(best)), "ntt_autotune")
    return best.value


def ntt_tune_get(word_bytes: int, log2n: int) -> tuple[int, int, int]:
    a, b, c = _int(), _int(), _int()
    _check(_load().ntt_tune_get(word_bytes, log2n, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "ntt_tune_get")
    return a.value, b.value, c.value


def ntt_tune_export() -> str:
    n = _sz()
    _check(_load().ntt_tune_export(None, 0, ctypes.byref(n)), "ntt_tune_export")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(_load().ntt_tune_export(buf, n.value + 1, ctypes.byref(n)), "ntt_tune_export")
    return buf.value.decode()


def ntt_tune_import(text: str):
    _check(_load().ntt_tune_import(text.encode()), "ntt_tune_import")


def ntt_device_status():
    """Raise NttError(NTT_ERR_TIMEOUT) if a kernel's bounded TMA wait ran out."""
    _check(_load().ntt_device_status(), "ntt_device_status")


def ntt_tune_reset():
    """Forget every tuned or imported launch shape."""
    _check(_load().ntt_tune_reset(), "ntt_tune_reset")


# ---------------------------------------------------------------- integer products

class IntmulPlan:
    """An intmul_plan: three 62-bit primes and their transform plans."""

    def __init__(self, max_limbs: int):
        h = _vp()
        _check(_load().intmul_plan_create(max_limbs, ctypes.byref(h)), "intmul_plan_create")
        self.handle = h.value
        self.max_limbs = max_limbs

    def close(self):
        if getattr(self, "handle", None):
            _load().intmul_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def intmul_plan_create(max_limbs: int) -> IntmulPlan:
    return IntmulPlan(max_limbs)


def intmul_workspace_size(plan: IntmulPlan, na: int, nb: int) -> int:
    return int(_load().intmul_workspace_size(plan.handle, na, nb))


def intmul_crt(plan: IntmulPlan, a, na: int, b, nb: int, c, ws, ws_bytes: int | None = None,
               stream=None):
    if ws_bytes is None:
        ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_load().intmul_crt(plan.handle, _ptr(a), na, _ptr(b), nb, _ptr(c), _ptr(ws), ws_bytes,
                              _stream(stream)), "intmul_crt")


def ntt_modmul_rate(p: int, kind: int, word_bytes: int, iters: int = 2048) -> float:
    out = ctypes.c_double()
    _check(_load().ntt_modmul_rate(p, kind, word_bytes, iters, ctypes.byref(out)), "ntt_modmul_rate")
    return out.value


def ntt_int_probe(kind: int, blocks: int, threads: int = 256, iters: int = 4096, stream=None) -> float:
    """Integer operations per second of the throughput probe `kind`
    (NTT_PROBE_IMAD, _ALU, _MIXED or _WIDE); synchronous."""
    out = ctypes.c_double()
    _check(_load().ntt_int_probe(kind, blocks, threads, iters, _stream(stream), ctypes.byref(out)),
           "ntt_int_probe")
    return out.value


def ntt_profile_begin():
    _check(_load().ntt_profile_begin(), "ntt_profile_begin")


def ntt_profile_end(cap: int = 256) -> list[tuple[str, float]]:
    """(kernel name, device ms) of every launch since ntt_profile_begin()."""
    ms = (ctypes.c_float * cap)()
    names = (ctypes.c_char_p * cap)()
    cnt = ctypes.c_int()
    _check(_load().ntt_profile_end(cap, ms, names, ctypes.byref(cnt)), "ntt_profile_end")
    return [(names[i].decode(), float(ms[i])) for i in range(min(cnt.value, cap))]


def intmat_workspace_size(plan: IntmulPlan, n: int, na: int, nb: int) -> int:
    return int(_load().intmat_workspace_size(plan.handle, n, na, nb))


def intmat_mul(plan: IntmulPlan, A, na: int, B, nb: int, n: int, C, ws, stream=None):
    ws_bytes = ws.numel() * ws.element_size()
    _check(_load().intmat_mul(plan.handle, _ptr(A), na, _ptr(B), nb, n, _ptr(C), _ptr(ws), ws_bytes,
                              _stream(stream)), "intmat_mul")


# ---------------------------------------------------------------- conveniences

def alloc_workspace(plan: Plan, batch: int, schedule: int = NTT_SCHED_FUSED, device="cuda"):
    """A uint8 device tensor of polymul_workspace_size bytes (None if 0)."""
    import torch
    nbytes = polymul_workspace_size(plan, batch, schedule)
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def polymul_host_stage_size(plan: Plan, na: int, nb: int, chunk: int) -> int:
    return int(_load().polymul_host_stage_size(plan.handle, na, nb, chunk))


def polymul_mod_p_batch_host(plan: Plan, h_a, na: int, h_b, nb: int, batch: int, h_c,
                             chunk: int, d_stage, stream=None):
    """polymul_mod_p_batch on HOST operands (CPU tensors, page-locked for
    overlap): the library uploads, multiplies and downloads in chunks of
    `chunk` products on overlapping streams; d_stage is a device tensor of
    polymul_host_stage_size bytes.  Asynchronous on `stream`."""
    stage_bytes = d_stage.numel() * d_stage.element_size()
    _check(_load().polymul_mod_p_batch_host(plan.handle, _ptr(h_a), na, _ptr(h_b), nb, batch,
                                            _ptr(h_c), chunk, _ptr(d_stage), stage_bytes,
                                            _stream(stream)), "polymul_mod_p_batch_host")
