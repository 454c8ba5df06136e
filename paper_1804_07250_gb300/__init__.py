"""GB300 sampler for random tilings by colour-class-parallel heat-bath
Glauber dynamics (Keating & Sridhar, "Random Tilings with the GPU").

Thin ctypes binding over ``libtiling.so`` (the C-ABI in ``include/tiling.h``):
argument marshalling only.  Every step of the sampler runs in the library's
CUDA kernels; there is no CPU fallback, and importing this package fails if
the library has not been built (``python paper_1804_07250_gb300/_build.py``).

Buffers may be numpy arrays (host) or torch tensors (host or CUDA); streams
may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer or None (the
legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TL_DEBUG=1 selects the bounds-checked build (_build.py --debug)
DEBUG_BUILD = os.environ.get("TL_DEBUG") == "1"
LIB_PATH = os.path.join(_HERE, "libtiling_debug.so" if DEBUG_BUILD else "libtiling.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("%s is missing: build it with "
                      "`python paper_1804_07250_gb300/_build.py%s` (needs nvcc)"
                      % (os.path.basename(LIB_PATH), " --debug" if DEBUG_BUILD else ""))

_lib = ctypes.CDLL(LIB_PATH)

TL_OK, TL_EINVAL, TL_ENOTSIMPLY, TL_ENOTTILEABLE, TL_ENOMEM = 0, 1, 2, 3, 4
TL_EBUDGET, TL_ECUDA, TL_ETIMEOUT, TL_EBUSY, TL_EUNSUPPORTED = 5, 6, 7, 8, 9
DOMINO, LOZENGE, SIXV = 0, 1, 2
T_SCALAR, T_SITE, T_TABLE16 = 0, 1, 2

_ERRNAMES = {1: "EINVAL", 2: "ENOTSIMPLY", 3: "ENOTTILEABLE", 4: "ENOMEM", 5: "EBUDGET",
             6: "ECUDA", 7: "ETIMEOUT", 8: "EBUSY", 9: "EUNSUPPORTED"}


class TilingError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, code), msg))
        self.code = code


class DomainInfo(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("planes", ctypes.c_int), ("passes", ctypes.c_int), ("sites", ctypes.c_uint64),
                ("edges", ctypes.c_uint64), ("canon_bytes", ctypes.c_uint64),
                ("packed_bytes", ctypes.c_uint64), ("site_box", ctypes.c_uint64),
                ("height_count", ctypes.c_uint64), ("height_width", ctypes.c_int),
                ("height_height", ctypes.c_int)]


class Plan(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("sweeps_per_launch", ctypes.c_int),
                ("halo", ctypes.c_int), ("threads", ctypes.c_int), ("npre", ctypes.c_int),
                ("ctas", ctypes.c_int), ("smem_bytes", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchPlan(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int), ("sweeps_per_launch", ctypes.c_int),
                ("graph_block", ctypes.c_int), ("grid", ctypes.c_int), ("smem_bytes", ctypes.c_int),
                ("ntiles", ctypes.c_int), ("threads", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Blob(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("size", ctypes.c_size_t)]


class Thresholds(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("scalar", ctypes.c_uint32),
                ("site", ctypes.c_void_p), ("table16", ctypes.c_uint32 * 16)]


_vp, _u64, _u32, _i = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_SIG = {
    "tl_last_error": (ctypes.c_char_p, []),
    "tl_version": (ctypes.c_char_p, []),
    "tl_ctx_create": (_i, [_i, ctypes.POINTER(_vp)]),
    "tl_ctx_destroy": (None, [_vp]),
    "tl_domain_aztec": (_i, [_i, ctypes.POINTER(_vp)]),
    "tl_domain_rect": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "tl_domain_hexagon": (_i, [_i, _i, _i, ctypes.POINTER(_vp)]),
    "tl_domain_dwbc": (_i, [_i, ctypes.POINTER(_vp)]),
    "tl_domain_destroy": (None, [_vp]),
    "tl_domain_get_info": (_i, [_vp, ctypes.POINTER(DomainInfo)]),
    "tl_domain_initial_state": (_i, [_vp, _vp, ctypes.c_size_t]),
    "tl_domain_extreme_state": (_i, [_vp, _i, _vp, ctypes.c_size_t]),
    "tl_domain_from_boundary": (_i, [_i, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "tl_thresholds_domino_edge_weights": (_i, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]),
    "tl_thresholds_lozenge_q": (_i, [ctypes.c_double, _vp, _vp]),
    "tl_thresholds_volume": (_i, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]),
    "tl_thresholds_lognormal_device": (_i, [_vp, ctypes.c_double, _u64, _vp, ctypes.c_size_t, _vp]),
    "tl_thresholds_6v": (_i, [_vp, _vp]),
    "tl_chain_create": (_i, [_vp, _vp, _vp, _u64, _u32, ctypes.POINTER(Thresholds),
                             ctypes.POINTER(_vp)]),
    "tl_chain_destroy": (None, [_vp]),
    "tl_chain_reset": (_i, [_vp, _vp]),
    "tl_chain_sweep": (_u64, [_vp]),
    "tl_chain_seek": (_i, [_vp, _u64]),
    "tl_chain_set_order": (_i, [_vp, _i]),
    "tl_aztec_shuffle": (_i, [_vp, _i, _u64, _u32, _vp, ctypes.c_size_t, _vp]),
    "tl_cftp": (_i, [_vp, _vp, _u64, _u32, ctypes.POINTER(Thresholds), _u64, _u64, _vp, ctypes.c_size_t,
                     ctypes.POINTER(_u64), _vp]),
    "tl_chain_launches": (_u64, [_vp]),
    "tl_chain_set_plan": (_i, [_vp, ctypes.POINTER(Plan)]),
    "tl_chain_get_plan": (_i, [_vp, ctypes.POINTER(Plan)]),
    "tl_chain_sync": (_i, [_vp, _vp]),
    "tl_debug_raise_status": (_i, [_vp, _vp]),
    "tl_debug_build": (_i, []),
    "tl_debug_checks": (_i, [ctypes.c_int, _vp, _vp, _vp, _vp]),
    "tl_debug_selftest": (_i, []),
    "tl_checkpoint": (_i, [_vp, _vp]),
    "tl_autotune_cache_clear": (None, []),
    "tl_chain_count_flips": (_i, [_vp, ctypes.c_int]),
    "tl_chain_flips": (_i, [_vp, _vp]),
    "tl_ctx_create_opts": (_i, [ctypes.c_int, _vp, _vp]),
    "tl_restore": (_i, [_vp, _vp, _vp]),
    "tl_blob_free": (None, [_vp]),
    "tl_run_sweeps": (_i, [_vp, _u64, _vp]),
    "tl_run_sweeps_hashed": (_i, [_vp, _u64, _vp, _vp]),
    "tl_read_state": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "tl_write_state": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "tl_state_hash": (_i, [_vp, _vp, _vp]),
    "tl_read_height": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "tl_read_height_noalloc": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "tl_density_begin": (_i, [_vp, _u32, _u64]),
    "tl_batch_create": (_i, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "tl_batch_destroy": (None, [_vp]),
    "tl_batch_run": (_i, [_vp, _u64, _vp]),
    "tl_batch_run_per_chain": (_i, [_vp, _u64, _vp]),
    "tl_batch_hashes": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "tl_batch_set_plan": (_i, [_vp, ctypes.POINTER(BatchPlan)]),
    "tl_batch_get_plan": (_i, [_vp, ctypes.POINTER(BatchPlan)]),
    "tl_batch_autotune": (_i, [_vp, _u64, _vp, ctypes.POINTER(BatchPlan)]),
    "tl_batch_launches": (_u64, [_vp]),
    "tl_batch_add": (_i, [_vp, _vp]),
    "tl_batch_remove": (_i, [_vp, _vp]),
    "tl_batch_size": (ctypes.c_size_t, [_vp]),
    "tl_read_density": (_i, [_vp, _vp, ctypes.c_size_t, _vp, _vp]),
    "tl_read_domino_nsew": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
}
for _name, (_res, _args) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIG)


def lib():
    return _lib


def debug_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(_lib.tl_debug_build())


def debug_checks(clear: bool = True) -> dict:
    """Failed bounds checks of the checked build since the last clear
    (tl_debug_checks): count, and id / index / bound of the first."""
    n = _u64(0)
    fid = ctypes.c_int(0)
    ix = ctypes.c_int64(0)
    bd = ctypes.c_int64(0)
    _check(_lib.tl_debug_checks(1 if clear else 0, ctypes.byref(n), ctypes.byref(fid), ctypes.byref(ix),
                                ctypes.byref(bd)))
    return {"failures": int(n.value), "id": fid.value, "index": ix.value, "bound": bd.value}


def debug_selftest():
    """Run one out-of-range check whose access is skipped (tl_debug_selftest)."""
    _check(_lib.tl_debug_selftest())


def _check(rc):
    if rc != TL_OK:
        raise TilingError(rc, _lib.tl_last_error().decode(errors="replace"))


def version() -> str:
    return _lib.tl_version().decode()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(getattr(s, "cuda_stream"))


def _ptr(buf):
    """Data pointer and byte size of a numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"], "buffer must be contiguous"
        return buf.ctypes.data, buf.nbytes
    if hasattr(buf, "data_ptr"):
        assert buf.is_contiguous(), "buffer must be contiguous"
        return buf.data_ptr(), buf.numel() * buf.element_size()
    raise TypeError("expected a numpy array or a torch tensor")


class CtxOpts(ctypes.Structure):
    _fields_ = [("max_sms", ctypes.c_int)]


class Context:
    def __init__(self, device: int = 0, max_sms: int = 0):
        h = _vp()
        if max_sms:
            o = CtxOpts(max_sms)
            _check(_lib.tl_ctx_create_opts(device, ctypes.byref(o), ctypes.byref(h)))
        else:
            _check(_lib.tl_ctx_create(device, ctypes.byref(h)))
        self._h = h
        self.device = device

    def close(self):
        if self._h:
            _lib.tl_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    def __init__(self, handle):
        self._h = handle
        info = DomainInfo()
        _check(_lib.tl_domain_get_info(self._h, ctypes.byref(info)))
        self.info = info

    @classmethod
    def aztec(cls, n):
        h = _vp(); _check(_lib.tl_domain_aztec(n, ctypes.byref(h))); return cls(h)

    @classmethod
    def rect(cls, w, h_):
        h = _vp(); _check(_lib.tl_domain_rect(w, h_, ctypes.byref(h))); return cls(h)

    @classmethod
    def hexagon(cls, a, b, c):
        h = _vp(); _check(_lib.tl_domain_hexagon(a, b, c, ctypes.byref(h))); return cls(h)

    @classmethod
    def dwbc(cls, N):
        h = _vp(); _check(_lib.tl_domain_dwbc(N, ctypes.byref(h))); return cls(h)

    @classmethod
    def from_boundary(cls, lattice, steps):
        """Domain enclosed by a closed lattice path: lattice DOMINO (steps 0..3 =
        +x, +y, -x, -y) or LOZENGE (0..5 = +x, +y, +x+y, -x, -y, -x-y)."""
        st = np.ascontiguousarray(steps, dtype=np.int8)
        h = _vp()
        _check(_lib.tl_domain_from_boundary(int(lattice), st.ctypes.data, st.size, ctypes.byref(h)))
        return cls(h)

    @property
    def canon_shape(self):
        return (self.info.planes, self.info.height, self.info.width)

    @property
    def height_shape(self):
        return (self.info.height_height, self.info.height_width)

    def initial_state(self) -> np.ndarray:
        out = np.zeros(self.canon_shape, dtype=np.uint8)
        p, n = _ptr(out)
        _check(_lib.tl_domain_initial_state(self._h, p, n))
        return out

    def extreme_state(self, which: str) -> np.ndarray:
        """'top' (every rotatable site UP) or 'bottom' (every one DOWN)."""
        out = np.zeros(self.canon_shape, dtype=np.uint8)
        p, n = _ptr(out)
        _check(_lib.tl_domain_extreme_state(self._h, {"bottom": 0, "top": 1}[which], p, n))
        return out

    def domino_thresholds(self, w: np.ndarray) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        t = np.zeros((self.info.height, self.info.width), dtype=np.uint32)
        pw, _ = _ptr(w)
        pt, _ = _ptr(t)
        _check(_lib.tl_thresholds_domino_edge_weights(self._h, pw, w.size, pt, t.size))
        return t

    def volume_thresholds(self, q: np.ndarray) -> np.ndarray:
        """Per-site thresholds from volume weights q[H, W] (one per box vertex)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        t = np.zeros((self.info.height, self.info.width), dtype=np.uint32)
        pq, _ = _ptr(q)
        pt, _ = _ptr(t)
        _check(_lib.tl_thresholds_volume(self._h, pq, q.size, pt, t.size))
        return t

    def lognormal_thresholds_device(self, sigma: float, seed: int, out, stream=None):
        """Per-site thresholds from device-generated log-normal weights (device buffer)."""
        p, n = _ptr(out)
        _check(_lib.tl_thresholds_lognormal_device(self._h, sigma, seed, p, n // 4, _stream(stream)))
        return out

    def close(self):
        if self._h:
            _lib.tl_domain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lozenge_thresholds(q: float):
    a = np.zeros(1, dtype=np.uint32)
    r = np.zeros(1, dtype=np.uint32)
    _check(_lib.tl_thresholds_lozenge_q(q, a.ctypes.data, r.ctypes.data))
    return int(a[0]), int(r[0])


def sixv_thresholds(w6) -> np.ndarray:
    w = np.ascontiguousarray(w6, dtype=np.float64)
    t = np.zeros(16, dtype=np.uint32)
    _check(_lib.tl_thresholds_6v(w.ctypes.data, t.ctypes.data))
    return t


def thresholds(scalar=None, site=None, table16=None) -> Thresholds:
    th = Thresholds()
    if table16 is not None:
        th.kind = T_TABLE16
        for i, v in enumerate(np.asarray(table16, dtype=np.uint32)):
            th.table16[i] = int(v)
    elif site is not None:
        th.kind = T_SITE
        if isinstance(site, np.ndarray):
            th._site = np.ascontiguousarray(site, dtype=np.uint32)
            th.site = th._site.ctypes.data
        else:                                   # a device tensor
            th._site = site
            th.site, _ = _ptr(site)
    else:
        th.kind = T_SCALAR
        th.scalar = int(scalar if scalar is not None else 1 << 31)
    return th


def cftp(ctx, domain, *, seed: int, stream_id: int = 0, th, t0: int = 64, tmax: int = 1 << 31,
         out=None, stream=None):
    """Exact sample by coupling from the past; returns (configuration, T)."""
    if out is None:
        out = np.zeros(domain.canon_shape, dtype=np.uint8)
    p, n = _ptr(out)
    t = _u64()
    _check(_lib.tl_cftp(ctx._h, domain._h, seed, stream_id, ctypes.byref(th), t0, tmax, p, n, ctypes.byref(t),
                        _stream(stream)))
    return out, int(t.value)


def aztec_shuffle(ctx, n: int, *, seed: int, stream_id: int = 0, out=None, stream=None):
    """Exact uniform tiling of the Aztec diamond of order n by domino shuffling."""
    if out is None:
        out = np.zeros((2, 2 * n + 1, 2 * n + 1), dtype=np.uint8)
    p, size = _ptr(out)
    _check(_lib.tl_aztec_shuffle(ctx._h, n, seed, stream_id, p, size, _stream(stream)))
    return out


class Chain:
    """One Markov chain resident on the GPU."""

    def __init__(self, ctx: Context, domain: Domain, *, seed: int, stream_id: int = 0,
                 th: Thresholds | None = None, init: np.ndarray | None = None):
        self.ctx, self.domain = ctx, domain
        self._th = th if th is not None else thresholds()
        p = None
        if init is not None:
            init = np.ascontiguousarray(init, dtype=np.uint8)
            assert init.shape == domain.canon_shape
            p = init.ctypes.data
        h = _vp()
        _check(_lib.tl_chain_create(ctx._h, domain._h, p, seed, stream_id,
                                    ctypes.byref(self._th), ctypes.byref(h)))
        self._h = h

    @property
    def sweep(self) -> int:
        return int(_lib.tl_chain_sweep(self._h))

    @property
    def launches(self) -> int:
        return int(_lib.tl_chain_launches(self._h))

    def reset(self, stream=None):
        _check(_lib.tl_chain_reset(self._h, _stream(stream)))

    def seek(self, sweep: int):
        _check(_lib.tl_chain_seek(self._h, sweep))

    def count_flips(self, on: bool = True):
        """Start (and reset) or stop the accepted-flip counter."""
        _check(_lib.tl_chain_count_flips(self._h, 1 if on else 0))

    @property
    def flips(self) -> int:
        v = ctypes.c_uint64()
        _check(_lib.tl_chain_flips(self._h, ctypes.byref(v)))
        return int(v.value)

    def set_order(self, random: bool):
        """Fixed colour order per sweep, or a random colour for every pass slot."""
        _check(_lib.tl_chain_set_order(self._h, 1 if random else 0))

    def set_plan(self, kernel: int = 0, sweeps_per_launch: int = 0, halo: int = 0,
                 threads: int = 0, npre: int = 0):
        """kernel 0 auto / 1 per-pass global / 2 shared-memory resident / 3
        register-resident (dominoes at t = 2^31); results never depend on it."""
        p = Plan(kernel, sweeps_per_launch, halo, threads, npre, 0, 0)
        _check(_lib.tl_chain_set_plan(self._h, ctypes.byref(p)))

    def plan(self) -> dict:
        p = Plan()
        _check(_lib.tl_chain_get_plan(self._h, ctypes.byref(p)))
        return p.as_dict()

    def sync(self, stream=None):
        _check(_lib.tl_chain_sync(self._h, _stream(stream)))

    def checkpoint(self) -> bytes:
        """The chain's inputs, start, state and sweep index as bytes
        (tl_checkpoint); waits for the device."""
        b = Blob()
        _check(_lib.tl_checkpoint(self._h, ctypes.byref(b)))
        try:
            return ctypes.string_at(b.data, b.size)
        finally:
            _lib.tl_blob_free(ctypes.byref(b))

    @classmethod
    def restore(cls, ctx: "Context", blob: bytes, domain: "Domain | None" = None) -> "Chain":
        """A new chain on `ctx` continuing exactly where the checkpointed one
        stood (tl_restore).  `domain` (the same domain, optional) only gives
        read_state and friends their default output shapes."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        b = Blob(ctypes.cast(buf, ctypes.c_void_p), len(blob))
        h = _vp()
        _check(_lib.tl_restore(ctx._h, ctypes.byref(b), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.ctx, self.domain, self._th, self._h = ctx, domain, None, h
        return self

    def debug_raise_status(self):
        """Test hook: make the resident kernel's next launch stop at its first
        boundary exchange as if a bounded wait had run out."""
        _check(_lib.tl_debug_raise_status(self._h, None))

    def run(self, k: int, stream=None):
        _check(_lib.tl_run_sweeps(self._h, k, _stream(stream)))

    def run_hashed(self, k: int, ring=None, stream=None):
        if ring is None:
            ring = np.zeros(k, dtype=np.uint64)
        p, n = _ptr(ring)
        assert n >= 8 * k
        _check(_lib.tl_run_sweeps_hashed(self._h, k, p, _stream(stream)))
        return ring

    def read_state(self, out=None, stream=None):
        if out is None:
            out = np.zeros(self.domain.canon_shape, dtype=np.uint8)
        p, n = _ptr(out)
        _check(_lib.tl_read_state(self._h, p, n, _stream(stream)))
        return out

    def write_state(self, state, stream=None):
        if isinstance(state, np.ndarray):
            state = np.ascontiguousarray(state, dtype=np.uint8)
        p, n = _ptr(state)
        _check(_lib.tl_write_state(self._h, p, n, _stream(stream)))

    def state_hash(self, out=None, stream=None) -> int:
        if out is not None:
            p, _ = _ptr(out)
            _check(_lib.tl_state_hash(self._h, p, _stream(stream)))
            return None
        v = np.zeros(1, dtype=np.uint64)
        _check(_lib.tl_state_hash(self._h, v.ctypes.data, _stream(stream)))
        return int(v[0])

    def read_height(self, out=None, stream=None):
        if out is None:
            out = np.zeros(self.domain.height_shape, dtype=np.int32)
        p, n = _ptr(out)
        _check(_lib.tl_read_height(self._h, p, n // 4, _stream(stream)))
        return out

    def read_height_noalloc(self, out, stream=None):
        """Heights into a device buffer without any allocation (static scratch)."""
        p, n = _ptr(out)
        _check(_lib.tl_read_height_noalloc(self._h, p, n // 4, _stream(stream)))
        return out

    def density_begin(self, stride: int, burn_in: int = 0):
        _check(_lib.tl_density_begin(self._h, stride, burn_in))

    def read_density(self, out=None, stream=None):
        if out is None:
            out = np.zeros(self.domain.canon_shape, dtype=np.float64)
        p, n = _ptr(out)
        s = np.zeros(1, dtype=np.uint64)
        _check(_lib.tl_read_density(self._h, p, n // 8, s.ctypes.data, _stream(stream)))
        return out, int(s[0])

    def read_nsew(self, out=None, stream=None):
        H, W = self.domain.info.height, self.domain.info.width
        if out is None:
            out = np.zeros((4, H - 1, W - 1), dtype=np.float64)
        p, n = _ptr(out)
        _check(_lib.tl_read_domino_nsew(self._h, p, n // 8, _stream(stream)))
        return out

    def close(self):
        if self._h:
            _lib.tl_chain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many chains advanced together (one work list, CUDA-graph blocks)."""

    def __init__(self, ctx: Context, chains=()):
        self.ctx, self.chains = ctx, list(chains)
        arr = (_vp * max(1, len(self.chains)))(*[c._h for c in self.chains])
        h = _vp()
        _check(_lib.tl_batch_create(ctx._h, ctypes.cast(arr, _vp), len(self.chains), ctypes.byref(h)))
        self._h = h

    def add(self, chain: Chain):
        _check(_lib.tl_batch_add(self._h, chain._h))
        self.chains.append(chain)

    def remove(self, chain: Chain):
        _check(_lib.tl_batch_remove(self._h, chain._h))
        self.chains.remove(chain)

    def __len__(self):
        return int(_lib.tl_batch_size(self._h))

    def run(self, k: int, stream=None):
        _check(_lib.tl_batch_run(self._h, k, _stream(stream)))

    def run_per_chain(self, k: int, stream=None):
        _check(_lib.tl_batch_run_per_chain(self._h, k, _stream(stream)))

    def debug_raise_status(self):
        """Test hook: make the batched kernel's next launch stop before its
        next tile as if a bounded wait had run out."""
        _check(_lib.tl_debug_raise_status(None, self._h))

    def hashes(self, out=None, stream=None):
        if out is None:
            out = np.zeros(len(self.chains), dtype=np.uint64)
        p, n = _ptr(out)
        _check(_lib.tl_batch_hashes(self._h, p, n // 8, _stream(stream)))
        return out

    def set_plan(self, tile_rows=0, sweeps_per_launch=0, graph_block=0, threads=0):
        p = BatchPlan(tile_rows, sweeps_per_launch, graph_block, 0, 0, 0, threads)
        _check(_lib.tl_batch_set_plan(self._h, ctypes.byref(p)))

    def plan(self) -> dict:
        p = BatchPlan()
        _check(_lib.tl_batch_get_plan(self._h, ctypes.byref(p)))
        return p.as_dict()

    def autotune(self, trial_sweeps: int = 8, stream=None) -> dict:
        p = BatchPlan()
        _check(_lib.tl_batch_autotune(self._h, trial_sweeps, _stream(stream), ctypes.byref(p)))
        return p.as_dict()

    @staticmethod
    def autotune_cache_clear():
        _lib.tl_autotune_cache_clear()

    @property
    def launches(self) -> int:
        return int(_lib.tl_batch_launches(self._h))

    def close(self):
        if self._h:
            _lib.tl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

