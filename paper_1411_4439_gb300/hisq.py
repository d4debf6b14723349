"""Python binding of libhisq: the C ABI of include/hisq.h, same names.

Argument marshalling only: every step of the Dslash and the CG runs in the
CUDA library. Device buffers are torch CUDA tensors (their data pointers are
passed through), host buffers are numpy arrays or CPU tensors. The stream
defaults to torch's current CUDA stream. If the compiled library is missing
every call raises: there is no fallback.

Element types of spinors ([V_h][3] complex per rhs):
  F64: complex128; F32: complex64; F16: float16 with a trailing (re, im)
  axis of length 2.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhisq.so")

# status codes
HISQ_OK, HISQ_EINVAL, HISQ_ERECON, HISQ_ENOCONV = 0, 1, 2, 3
HISQ_EBREAKDOWN, HISQ_ENAN, HISQ_ECUDA, HISQ_ETIMEOUT, HISQ_ENOMEM = 4, 5, 6, 7, 8
# precisions and compressions
HISQ_F64, HISQ_F32, HISQ_F16 = 0, 1, 2
HISQ_R18, HISQ_R12, HISQ_R14 = 18, 12, 14
HISQ_AOS, HISQ_SOA, HISQ_BUNDLE = 0, 1, 2

STATUS_NAMES = {0: "HISQ_OK", 1: "HISQ_EINVAL", 2: "HISQ_ERECON", 3: "HISQ_ENOCONV",
                4: "HISQ_EBREAKDOWN", 5: "HISQ_ENAN", 6: "HISQ_ECUDA", 7: "HISQ_ETIMEOUT",
                8: "HISQ_ENOMEM"}
MAX_RHS = 16

HISQ_OP_M, HISQ_OP_MDAG, HISQ_OP_DM_DMU = 0, 1, 2
HISQ_OP_D2M_DMU2, HISQ_OP_D3M_DMU3, HISQ_OP_D4M_DMU4 = 3, 4, 5
HISQ_MAP_PACKED, HISQ_MAP_L2_PREFETCH, HISQ_MAP_STAGED = 1, 2, 4
HISQ_MAP_PIPELINED, HISQ_MAP_PIPELINED2 = 8, 16
HISQ_MAP_COMPACT = 128
HISQ_MAP_TILE_XY = 256

EXPORTED = ["hisq_version", "hisq_last_error", "hisq_gauge_load", "hisq_gauge_free",
            "hisq_gauge_info", "hisq_set_dslash_mapping", "hisq_get_dslash_mapping",
            "hisq_get_dslash_mapping_ex",
            "hisq_autotune_dslash", "hisq_gauge_load_tuned", "hisq_autotune_bundle",
            "hisq_link_compress",
            "hisq_link_reconstruct", "hisq_dslash", "hisq_dslash_ex", "hisq_bundle_pack",
            "hisq_bundle_unpack", "hisq_mdagm",
            "hisq_apply_m", "hisq_link_force", "hisq_cdot", "hisq_cdot_noalloc",
            "hisq_cg_default_params", "hisq_cg_solve", "hisq_cg_solve_batched"]


class HisqError(RuntimeError):
    def __init__(self, status: int, message: str, stats=None):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.stats = stats


class hisq_cg_params(ctypes.Structure):
    _fields_ = [("maxiter", ctypes.c_int), ("reliable_every", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("inner_prec", ctypes.c_int),
                ("use_x0", ctypes.c_int), ("even_odd", ctypes.c_int),
                ("check_every", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("rhs_per_thread", ctypes.c_int), ("spinor_layout", ctypes.c_int),
                ("device_loop", ctypes.c_int), ("profile_kernels", ctypes.c_int)]


class hisq_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * MAX_RHS), ("total_iters", ctypes.c_int),
                ("reliable_updates", ctypes.c_int),
                ("true_rel_res", ctypes.c_double * MAX_RHS), ("seconds", ctypes.c_double),
                ("profiled_iters", ctypes.c_int), ("kernel_us", ctypes.c_double * 4)]


class hisq_cg_problem(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("mass", ctypes.c_double), ("mu", ctypes.c_double),
                ("b", ctypes.POINTER(ctypes.c_void_p)), ("x", ctypes.POINTER(ctypes.c_void_p)),
                ("n", ctypes.c_int), ("tol", ctypes.c_double)]


_lib = None


def library() -> ctypes.CDLL:
    """The loaded libhisq (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise HisqError(HISQ_ECUDA, f"{LIB_PATH} is missing; build it with "
                        "`python -m paper_1411_4439_gb300.build_lib`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, c_int, c_double = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
    sig = {
        "hisq_version": (c_int, []),
        "hisq_last_error": (ctypes.c_char_p, []),
        "hisq_gauge_load": (c_int, [ip, vp, vp, c_int, c_int, c_int, c_int, c_double, vp,
                                    ctypes.POINTER(vp)]),
        "hisq_gauge_free": (c_int, [vp]),
        "hisq_gauge_info": (c_int, [vp, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_size_t)]),
        "hisq_set_dslash_mapping": (c_int, [vp, c_int, c_int, c_int]),
        "hisq_get_dslash_mapping": (c_int, [vp, c_int, c_int, ip, ip, ip]),
        "hisq_get_dslash_mapping_ex": (c_int, [vp, c_int, c_int, c_int, ip, ip, ip]),
        "hisq_autotune_dslash": (c_int, [vp, c_int, c_int, c_int, c_int, ip, ip, ip,
                                         ctypes.POINTER(c_double)]),
        "hisq_gauge_load_tuned": (c_int, [ip, vp, vp, c_int, c_int, c_int, c_double, vp, ctypes.POINTER(vp)]),
        "hisq_autotune_bundle": (c_int, [vp, c_int, c_int, c_int, c_int, ip, ctypes.POINTER(c_double)]),
        "hisq_link_compress": (c_int, [ip, vp, c_int, vp, ctypes.POINTER(c_double), vp]),
        "hisq_link_reconstruct": (c_int, [ip, vp, c_int, vp, vp]),
        "hisq_dslash": (c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, c_int, c_int, vp]),
        "hisq_dslash_ex": (c_int, [vp, c_double, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, c_int,
                                   c_int, c_int, vp]),
        "hisq_mdagm": (c_int, [vp, c_double, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, c_int, vp]),
        "hisq_bundle_pack": (c_int, [vp, ctypes.POINTER(vp), c_int, c_int, vp, vp]),
        "hisq_bundle_unpack": (c_int, [vp, vp, c_int, c_int, ctypes.POINTER(vp), vp]),
        "hisq_apply_m": (c_int, [vp, c_double, c_double, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 c_int, c_int, vp]),
        "hisq_link_force": (c_int, [vp, c_double, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int,
                                    c_double, vp, vp]),
        "hisq_cdot": (c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, ctypes.c_longlong,
                              ctypes.POINTER(c_double), vp]),
        "hisq_cdot_noalloc": (c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, ctypes.c_longlong,
                                      ctypes.POINTER(c_double), vp]),
        "hisq_cg_default_params": (None, [ctypes.POINTER(hisq_cg_params)]),
        "hisq_cg_solve_batched": (c_int, [ctypes.POINTER(hisq_cg_problem), c_int,
                                          ctypes.POINTER(hisq_cg_params), ctypes.POINTER(hisq_cg_stats),
                                          vp]),
        "hisq_cg_solve": (c_int, [vp, c_double, c_double, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int,
                                  c_double, ctypes.POINTER(hisq_cg_params),
                                  ctypes.POINTER(hisq_cg_stats), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, stats=None):
    if status != HISQ_OK:
        msg = library().hisq_last_error().decode(errors="replace")
        raise HisqError(status, msg, stats)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _ptr(buf) -> int:
    """Address of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffer must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, int):
        return buf
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _is_device(buf) -> bool:
    return hasattr(buf, "is_cuda") and bool(buf.is_cuda)


def _stream_handle(stream, *bufs) -> int | None:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if any(_is_device(b) for b in bufs):
        return int(_torch().cuda.current_stream().cuda_stream)
    return None


def _ptr_array(bufs):
    arr = (ctypes.c_void_p * len(bufs))()
    for i, b in enumerate(bufs):
        arr[i] = _ptr(b)
    return arr


def _lattice(L):
    L = [int(a) for a in L]
    if len(L) != 4:
        raise ValueError("L must have 4 extents")
    return (ctypes.c_int * 4)(*L)


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def hisq_version() -> int:
    return library().hisq_version()


def hisq_last_error() -> str:
    return library().hisq_last_error().decode(errors="replace")


@dataclass
class Gauge:
    """Owner of a hisq_gauge handle; free with hisq_gauge_free or `with`."""
    handle: int
    L: tuple
    prec: int
    recon_U: int
    recon_N: int
    _freed: bool = field(default=False, repr=False)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        hisq_gauge_free(self)

    def __del__(self):
        try:
            hisq_gauge_free(self)
        except Exception:
            pass


def hisq_gauge_load(L, U, N, prec=HISQ_F32, recon_U=HISQ_R18, recon_N=HISQ_R18,
                    recon_tol=1e-10, stream=None) -> Gauge:
    """Load canonical complex128 [4][V][3][3] links (device tensor or host array)."""
    on_dev = _is_device(U)
    if on_dev != _is_device(N):
        raise ValueError("U and N must both be on the device or both on the host")
    for a in (U, N):
        dt = getattr(a, "dtype", None)
        if str(dt) not in ("complex128", "torch.complex128"):
            raise TypeError("links must be complex128")
    h = ctypes.c_void_p()
    st = library().hisq_gauge_load(_lattice(L), _ptr(U), _ptr(N), int(on_dev), int(prec),
                                   int(recon_U), int(recon_N), float(recon_tol),
                                   _stream_handle(stream, U, N), ctypes.byref(h))
    _check(st)
    return Gauge(h.value, tuple(int(a) for a in L), int(prec), int(recon_U), int(recon_N))


def hisq_gauge_load_tuned(L, U, N, prec=HISQ_F32, n=8, recon_tol=1e-10, stream=None) -> Gauge:
    """Load the links with the compression pair whose tuned Dslash for n rhs is fastest."""
    on_dev = _is_device(U)
    if on_dev != _is_device(N):
        raise ValueError("U and N must both be on the device or both on the host")
    h = ctypes.c_void_p()
    _check(library().hisq_gauge_load_tuned(_lattice(L), _ptr(U), _ptr(N), int(on_dev), int(prec), int(n),
                                           float(recon_tol), _stream_handle(stream, U, N), ctypes.byref(h)))
    g = Gauge(h.value, tuple(int(a) for a in L), int(prec), 0, 0)
    info = hisq_gauge_info(g)
    g.recon_U, g.recon_N = info["recon_U"], info["recon_N"]
    return g


def hisq_gauge_free(g: Gauge) -> None:
    if g is None or g._freed:
        return
    g._freed = True
    _check(library().hisq_gauge_free(g.handle))


def hisq_gauge_info(g: Gauge) -> dict:
    L = (ctypes.c_int * 4)()
    prec, ru, rn = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nbytes = ctypes.c_size_t()
    _check(library().hisq_gauge_info(g.handle, L, ctypes.byref(prec), ctypes.byref(ru),
                                     ctypes.byref(rn), ctypes.byref(nbytes)))
    return dict(L=tuple(L), prec=prec.value, recon_U=ru.value, recon_N=rn.value,
                device_bytes=nbytes.value)


def hisq_set_dslash_mapping(g: Gauge, rhs_per_thread: int, min_blocks: int = 0,
                            flags: int = 0) -> None:
    """Dslash rhs per thread, register budget (min blocks per SM) and HISQ_MAP_* flags
    (packed f32x2 arithmetic, L2 link prefetch, staged links, pipelined hops);
    0 = automatic."""
    _check(library().hisq_set_dslash_mapping(g.handle, int(rhs_per_thread), int(min_blocks),
                                             int(flags)))


def hisq_get_dslash_mapping(g: Gauge, n: int, prec: int) -> tuple:
    """(rhs per thread, min blocks, HISQ_MAP_* flags) a Dslash of n rhs will use."""
    r, b, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(library().hisq_get_dslash_mapping(g.handle, int(n), int(prec), ctypes.byref(r),
                                             ctypes.byref(b), ctypes.byref(f)))
    return r.value, b.value, f.value


def hisq_get_dslash_mapping_ex(g: Gauge, n: int, prec: int, layout: int) -> tuple:
    """(rhs per thread, min blocks, HISQ_MAP_* flags) a Dslash of n rhs in `layout` will use."""
    r, b, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(library().hisq_get_dslash_mapping_ex(g.handle, int(n), int(prec), int(layout), ctypes.byref(r),
                                                ctypes.byref(b), ctypes.byref(f)))
    return r.value, b.value, f.value


def hisq_autotune_dslash(g: Gauge, n: int, prec: int, layout: int = HISQ_SOA, reps: int = 5) -> dict:
    """Time every built Dslash mapping for (n, prec, layout), keep the fastest on g."""
    r, b, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    sec = ctypes.c_double()
    _check(library().hisq_autotune_dslash(g.handle, int(n), int(prec), int(layout), int(reps),
                                          ctypes.byref(r), ctypes.byref(b), ctypes.byref(f),
                                          ctypes.byref(sec)))
    return dict(rhs_per_thread=r.value, min_blocks=b.value, flags=f.value, seconds=sec.value)


def hisq_autotune_bundle(g: Gauge, n_max: int, prec: int, layout: int = HISQ_SOA, reps: int = 5) -> dict:
    """Bundle size (power of two <= n_max) with the lowest tuned Dslash time per rhs."""
    bn, sec = ctypes.c_int(), ctypes.c_double()
    _check(library().hisq_autotune_bundle(g.handle, int(n_max), int(prec), int(layout), int(reps),
                                          ctypes.byref(bn), ctypes.byref(sec)))
    return dict(n=bn.value, seconds_per_rhs=sec.value)


def hisq_link_compress(L, links, recon, packed, stream=None) -> float:
    """Device complex128 [4][V][3][3] -> device float64 [4][V][recon]; returns max error."""
    err = ctypes.c_double()
    _check(library().hisq_link_compress(_lattice(L), _ptr(links), int(recon), _ptr(packed),
                                        ctypes.byref(err), _stream_handle(stream, links)))
    return err.value


def hisq_link_reconstruct(L, packed, recon, links, stream=None) -> None:
    _check(library().hisq_link_reconstruct(_lattice(L), _ptr(packed), int(recon), _ptr(links),
                                           _stream_handle(stream, packed)))


def hisq_dslash(g: Gauge, v, w, parity: int, prec: int, stream=None) -> None:
    """w[k] = D_{p,1-p} v[k] (Eq. 3, Eq. 4); v, w lists of device tensors."""
    hisq_dslash_ex(g, 0.0, v, w, parity, prec, HISQ_AOS, stream)


def hisq_dslash_ex(g: Gauge, mu: float, v, w, parity: int, prec: int, layout: int = HISQ_AOS,
                   stream=None, n: int | None = None) -> None:
    """Dslash with a chemical potential on the temporal hops.

    AoS or SoA: v, w lists of one device tensor per rhs. HISQ_BUNDLE: v, w are
    single device tensors holding the bundle of all ``n`` rhs.
    """
    if layout == HISQ_BUNDLE:
        if n is None:
            raise ValueError("the bundle layout needs n")
        _check_bundle_tensor(v, prec, n, g)
        _check_bundle_tensor(w, prec, n, g)
        _check(library().hisq_dslash_ex(g.handle, float(mu), _ptr_array([v]), _ptr_array([w]), int(n),
                                        int(parity), int(prec), int(layout), _stream_handle(stream, v)))
        return
    if len(v) != len(w):
        raise ValueError("v and w need the same number of rhs")
    _check(library().hisq_dslash_ex(g.handle, float(mu), _ptr_array(v), _ptr_array(w), len(v),
                                    int(parity), int(prec), int(layout), _stream_handle(stream, *v)))


def bundle_bytes(g: Gauge, n: int, prec: int) -> int:
    """Bytes of a bundle of n rhs on one parity of g's lattice."""
    vh = int(np.prod(g.L)) // 2
    return n * 3 * vh * (8 if prec == HISQ_F32 else 4)


def _check_bundle_tensor(t, prec: int, n: int, g: Gauge):
    if not _is_device(t):
        raise ValueError("bundle buffers must be CUDA tensors")
    if t.numel() * t.element_size() != bundle_bytes(g, n, prec):
        raise ValueError(f"bundle buffer has {t.numel() * t.element_size()} bytes, "
                         f"{bundle_bytes(g, n, prec)} expected for n = {n}")


def hisq_bundle_pack(g: Gauge, src, prec: int, bundle, stream=None) -> None:
    """Pack FP64 complex vectors src[k] ([V_h][3], device) into one bundle of prec."""
    _check_fp64_vectors(src)
    _check_bundle_tensor(bundle, prec, len(src), g)
    _check(library().hisq_bundle_pack(g.handle, _ptr_array(src), len(src), int(prec), _ptr(bundle),
                                      _stream_handle(stream, bundle)))


def hisq_bundle_unpack(g: Gauge, bundle, prec: int, dst, stream=None) -> None:
    """Unpack one bundle of prec into FP64 complex vectors dst[k] ([V_h][3], device)."""
    _check_fp64_vectors(dst)
    _check_bundle_tensor(bundle, prec, len(dst), g)
    _check(library().hisq_bundle_unpack(g.handle, _ptr(bundle), len(dst), int(prec), _ptr_array(dst),
                                        _stream_handle(stream, bundle)))


def _check_fp64_vectors(vs):
    """Every vector a CUDA complex128 (or float64 pairs) tensor of one device and length."""
    torch = _torch()
    if len(vs) == 0:
        raise ValueError("no vectors")
    for t in vs:
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            raise ValueError("vectors must be CUDA tensors")
        if t.dtype not in (torch.complex128, torch.float64):
            raise ValueError(f"vectors must be complex128 or float64, got {t.dtype}")
        if t.dtype != vs[0].dtype or t.device != vs[0].device or t.numel() != vs[0].numel():
            raise ValueError("vectors must share dtype, device and length")


def hisq_mdagm(g: Gauge, mass: float, v, w, prec: int, stream=None) -> None:
    """w[k] = (4 m^2 - D_eo D_oe) v[k] on even sites."""
    if len(v) != len(w):
        raise ValueError("v and w need the same number of rhs")
    _check(library().hisq_mdagm(g.handle, float(mass), _ptr_array(v), _ptr_array(w), len(v),
                                int(prec), _stream_handle(stream, *v)))


def hisq_apply_m(g: Gauge, mass: float, mu: float, op: int, v, w, prec: int, stream=None) -> None:
    """w[k] = M(mu) v[k], M(mu)^dag v[k] or dM/dmu v[k] on parity-blocked [2 V_h][3] vectors."""
    if len(v) != len(w):
        raise ValueError("v and w need the same number of rhs")
    _check(library().hisq_apply_m(g.handle, float(mass), float(mu), int(op), _ptr_array(v),
                                  _ptr_array(w), len(v), int(prec), _stream_handle(stream, *v)))


def hisq_link_force(g: Gauge, mu: float, hop: int, a, b, coef: float, out, stream=None) -> None:
    """out[mu][x] += coef * sum_k [f a_k(x) b_k(x+hop mu)^dag - b_k(x) a_k(x+hop mu)^dag / f]."""
    if len(a) != len(b):
        raise ValueError("a and b need the same number of rhs")
    _check(library().hisq_link_force(g.handle, float(mu), int(hop), _ptr_array(a), _ptr_array(b),
                                     len(a), float(coef), _ptr(out), _stream_handle(stream, out)))


def hisq_cdot(g: Gauge, a, b, stream=None) -> np.ndarray:
    """<a_k, b_k> for FP64 complex device vectors; returns complex128 array of n values."""
    if len(a) != len(b):
        raise ValueError("a and b need the same number of rhs")
    n = len(a)
    _check_fp64_vectors(list(a) + list(b))
    length = int(a[0].numel()) // (2 if str(a[0].dtype).endswith("float64") else 1)
    out = (ctypes.c_double * (2 * n))()
    _check(library().hisq_cdot(g.handle, _ptr_array(a), _ptr_array(b), n, length, out,
                               _stream_handle(stream, *a)))
    arr = np.frombuffer(out, dtype=np.float64).copy()
    return arr[0::2] + 1j * arr[1::2]


def hisq_cdot_noalloc(a, b, stream=None) -> np.ndarray:
    """<a_k, b_k> like hisq_cdot, with no device allocation (static library scratch)."""
    if len(a) != len(b):
        raise ValueError("a and b need the same number of rhs")
    n = len(a)
    _check_fp64_vectors(list(a) + list(b))
    length = int(a[0].numel()) // (2 if str(a[0].dtype).endswith("float64") else 1)
    out = (ctypes.c_double * (2 * max(n, 1)))()
    _check(library().hisq_cdot_noalloc(_ptr_array(a), _ptr_array(b), n, length, out,
                                       _stream_handle(stream, *a)))
    arr = np.frombuffer(out, dtype=np.float64).copy()
    return arr[0::2] + 1j * arr[1::2]


def hisq_cg_default_params() -> hisq_cg_params:
    p = hisq_cg_params()
    library().hisq_cg_default_params(ctypes.byref(p))
    return p


def cg_params(**kw) -> hisq_cg_params:
    """Defaults of the library with the given fields replaced."""
    p = hisq_cg_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"hisq_cg_params has no field {k}")
        setattr(p, k, v)
    return p


def hisq_cg_solve(g: Gauge, mass: float, mu: float, b, x, tol: float, params=None,
                  stream=None) -> hisq_cg_stats:
    """Solve the normal equations per rhs; b, x lists of complex128 buffers.

    Raises HisqError on any status but HISQ_OK (the stats ride on the error).
    """
    if len(b) != len(x):
        raise ValueError("b and x need the same number of rhs")
    stats = hisq_cg_stats()
    p = params if params is not None else hisq_cg_default_params()
    st = library().hisq_cg_solve(g.handle, float(mass), float(mu), _ptr_array(b), _ptr_array(x),
                                 len(b), float(tol), ctypes.byref(p), ctypes.byref(stats),
                                 _stream_handle(stream, *b, *x))
    _check(st, stats)
    return stats


def hisq_cg_solve_batched(problems, params=None, stream=None):
    """Independent solves advanced together through one CUDA graph per chunk.

    problems: list of dicts with keys g (Gauge), mass, mu, b, x (lists of
    complex128 buffers), tol. Returns one hisq_cg_stats per problem; raises
    HisqError (with the stats list) on any status but HISQ_OK.
    """
    arr = (hisq_cg_problem * len(problems))()
    keep = []
    bufs = []
    for i, pr in enumerate(problems):
        if len(pr["b"]) != len(pr["x"]):
            raise ValueError("b and x need the same number of rhs")
        pb, px = _ptr_array(pr["b"]), _ptr_array(pr["x"])
        keep += [pb, px]
        bufs += list(pr["b"]) + list(pr["x"])
        arr[i] = hisq_cg_problem(pr["g"].handle, float(pr["mass"]), float(pr.get("mu", 0.0)),
                                 ctypes.cast(pb, ctypes.POINTER(ctypes.c_void_p)),
                                 ctypes.cast(px, ctypes.POINTER(ctypes.c_void_p)), len(pr["b"]),
                                 float(pr["tol"]))
    stats = (hisq_cg_stats * len(problems))()
    p = params if params is not None else hisq_cg_default_params()
    st = library().hisq_cg_solve_batched(arr, len(problems), ctypes.byref(p), stats,
                                         _stream_handle(stream, *bufs))
    out = [stats[i] for i in range(len(problems))]
    _check(st, out)
    return out
