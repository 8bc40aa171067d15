"""Thin Python binding of libgbrank.so (argument marshalling only).

Every function has the name of the C entry point it calls (``include/gbrank.h``)
and does nothing but convert arguments: torch CUDA tensors become device
pointers, host arrays become host pointers, the current torch stream becomes
the stream argument, and a non-zero status becomes a ``GbrError`` carrying
``gbr_last_error()``.  There is no fallback: without the compiled library
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbrank.so")
_lock = threading.Lock()
_lib = None

GBR_OK, GBR_EINVAL, GBR_ENOMEM, GBR_ECUDA, GBR_ENOTFOUND, GBR_ETIMEOUT, GBR_EBREAKDOWN, GBR_ENONFINITE = range(8)
GBR_RANK_STAGGERED, GBR_RANK_CNS = 0, 1
GBR_HV_AUTO, GBR_HV_FUSED, GBR_HV_FACTORED = 0, 1, 2
GBR_PREC_FP64, GBR_PREC_MIXED = 0, 1
NOT_FOUND_U32 = 0xFFFFFFFF
NOT_FOUND_U64 = 0xFFFFFFFFFFFFFFFF


class GbrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gbrank error {code}: {msg}")
        self.code = code


class LanczosOpts(C.Structure):
    _fields_ = [("iters", C.c_int), ("reorth", C.c_int), ("prec", C.c_int), ("refine", C.c_int),
                ("store_basis", C.c_int), ("use_graph", C.c_int), ("profile", C.c_int), ("tol", C.c_double),
                ("ritz_tail", C.c_double)]


class LanczosResult(C.Structure):
    _fields_ = [("E0", C.c_double), ("E_ritz", C.c_double), ("residual", C.c_double), ("iters_done", C.c_int),
                ("breakdown", C.c_int), ("stored_basis", C.c_int), ("seconds", C.c_double),
                ("hv_seconds", C.c_double), ("stage_seconds", C.c_double * 4), ("stage_launches", C.c_int * 4),
                ("converged", C.c_int), ("ritz_terms", C.c_int), ("basis_head", C.c_int)]


class Term(C.Structure):
    """Tuple (v, m, l, r, x, s) of Eqs. Talpha1/Talpha2."""
    _fields_ = [("v", C.c_double), ("m", C.c_uint64), ("l", C.c_uint64), ("r", C.c_uint64), ("x", C.c_uint64),
                ("s", C.c_uint64)]


class ModelDesc(C.Structure):
    _fields_ = [("L", C.c_int), ("h", C.c_void_p), ("U", C.c_void_p)]


def lib():
    """The loaded library; raises if it was not built (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64
            sig = {
                "gbr_last_error": (C.c_char_p, []),
                "gbr_version": (i32, []),
                "gbr_comb_create": (i32, [i32, i32, i32, vp]),
                "gbr_comb_destroy": (None, [vp]),
                "gbr_comb_info": (i32, [vp, vp, vp]),
                "gbr_comb_rank": (i32, [vp, vp, vp, i32, i64, i32, vp]),
                "gbr_comb_unrank": (i32, [vp, vp, i32, vp, i64, vp]),
                "gbr_trie_create": (i32, [vp, i64, i32, i32, vp]),
                "gbr_trie_create_ordered": (i32, [vp, i64, i32, i32, i32, vp]),
                "gbr_trie_build_host_ordered": (i32, [vp, i64, i32, i32, i32, vp, i64, vp]),
                "gbr_trie_destroy": (None, [vp]),
                "gbr_trie_create_from_table": (i32, [vp, i64, i32, i32, i32, vp, i64, vp]),
                "gbr_trie_info": (i32, [vp, vp, vp, vp, vp]),
                "gbr_trie_build_host": (i32, [vp, i64, i32, i32, vp, i64, vp]),
                "gbr_trie_rank": (i32, [vp, vp, vp, i32, i64, i32, vp]),
                "gbr_trie_unrank": (i32, [vp, vp, i32, vp, i64, vp]),
                "gbr_trie_rank_bisect": (i32, [vp, vp, vp, i32, i64, i32, vp]),
                "gbr_ham_create": (i32, [i32, vp, vp, i32, i32, i32, vp]),
                "gbr_ham_destroy": (None, [vp]),
                "gbr_ham_info": (i32, [vp, vp, vp]),
                "gbr_ham_set_path": (i32, [vp, i32]),
                "gbr_check_rcp64": (i32, [i64, C.POINTER(C.c_double)]),
                "gbr_release_cache": (i32, []),
                "gbr_ham_get_path": (i32, [vp, C.POINTER(i32)]),
                "gbr_hv": (i32, [vp, vp, vp, i32, vp]),
                "gbr_ham_tune": (i32, [vp, i32, vp]),
                "gbr_ham_set_shape": (i32, [vp, i32, vp]),
                "gbr_ham_get_shape": (i32, [vp, i32, vp]),
                "gbr_device_status": (i32, [i32, vp]),
                "gbr_hv_stage": (i32, [vp, vp, vp, i32, i32, vp]),
                "gbr_hv_static": (i32, [vp, vp, vp, i32, vp]),
                "gbr_launch_count": (i64, []),
                "gbr_lanczos": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
                "gbr_setham_lanczos": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
                "gbr_termham_lanczos": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
                "gbr_term_product": (i32, [vp, i32, C.c_double, vp]),
                "gbr_term_mul": (i32, [vp, vp, vp]),
                "gbr_termham_create": (i32, [i32, vp, i32, vp, i64, i32, vp]),
                "gbr_termham_destroy": (None, [vp]),
                "gbr_termham_info": (i32, [vp, vp, vp, vp]),
                "gbr_termham_hv": (i32, [vp, vp, vp, i32, i32, vp]),
                "gbr_termham_set_bisect": (i32, [vp, i32]),
                "gbr_setham_create": (i32, [i32, vp, vp, vp, i64, i32, vp]),
                "gbr_setham_create_ordered": (i32, [i32, vp, vp, vp, i64, i32, i32, vp]),
                "gbr_setham_destroy": (None, [vp]),
                "gbr_setham_info": (i32, [vp, vp, vp, vp]),
                "gbr_setham_set_bisect": (i32, [vp, i32]),
                "gbr_setham_hv": (i32, [vp, vp, vp, i32, i32, vp]),
                "gbr_batch_layout": (i32, [i32, vp, vp, vp]),
                "gbr_batch_solve": (i32, [i32, vp, vp, i32, vp, vp, vp, vp]),
                "gbr_batch_set_shape": (i32, [i32, i32]),
                "gbr_batch_get_shape": (i32, [vp, vp]),
                "gbr_batch_tune": (i32, [i32, vp, vp, i32, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def gbr_last_error() -> str:
    return lib().gbr_last_error().decode(errors="replace")


def gbr_version() -> int:
    return lib().gbr_version()


def _check(rc: int):
    if rc != GBR_OK:
        raise GbrError(rc, gbr_last_error())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, dtypes=None):
    """Device pointer of a contiguous torch CUDA tensor."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtypes is not None and t.dtype not in dtypes:
        raise ValueError(f"dtype {t.dtype} not in {dtypes}")
    return C.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _rank_bits(t) -> int:
    import torch
    if t.dtype == torch.int32:
        return 32
    if t.dtype == torch.int64:
        return 64
    raise ValueError("rank tensors are int32 (32-bit ranks) or int64 (64-bit ranks)")


class _Handle:
    _destroy = None

    def __init__(self, ptr: C.c_void_p):
        self.ptr = ptr

    def close(self):
        if self.ptr and self.ptr.value:
            getattr(lib(), self._destroy)(self.ptr)
            self.ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Comb(_Handle):
    _destroy = "gbr_comb_destroy"


class Trie(_Handle):
    _destroy = "gbr_trie_destroy"


class Ham(_Handle):
    _destroy = "gbr_ham_destroy"


class SetHam(_Handle):
    _destroy = "gbr_setham_destroy"


class TermHam(_Handle):
    _destroy = "gbr_termham_destroy"


# ---------------------------------------------------------------- combinations

def gbr_comb_create(M: int, N: int, R: int = 8) -> Comb:
    p = C.c_void_p()
    _check(lib().gbr_comb_create(M, N, R, C.byref(p)))
    return Comb(p)


def gbr_comb_info(c: Comb):
    dim, tb = C.c_uint64(), C.c_int64()
    _check(lib().gbr_comb_info(c, C.byref(dim), C.byref(tb)))
    return dim.value, tb.value


def gbr_comb_rank(c: Comb, pat, out, check: int = 0, stream=None):
    import torch
    _check(lib().gbr_comb_rank(c, _dptr(pat, (torch.int64,)), _dptr(out), _rank_bits(out), pat.numel(), int(check),
                               _stream(stream)))
    return out


def gbr_comb_unrank(c: Comb, rank, out, stream=None):
    import torch
    _check(lib().gbr_comb_unrank(c, _dptr(rank), _rank_bits(rank), _dptr(out, (torch.int64,)), rank.numel(),
                                 _stream(stream)))
    return out


# ----------------------------------------------------------------------- tries

def gbr_trie_create(sorted_members: np.ndarray, M: int, R: int = 8, msb_first: bool = False) -> Trie:
    a = np.ascontiguousarray(sorted_members, dtype=np.uint64)
    p = C.c_void_p()
    if msb_first:
        _check(lib().gbr_trie_create_ordered(_hptr(a), a.size, M, R, 1, C.byref(p)))
    else:
        _check(lib().gbr_trie_create(_hptr(a), a.size, M, R, C.byref(p)))
    return Trie(p)


def gbr_trie_create_from_table(sorted_members: np.ndarray, M: int, R: int, table: np.ndarray,
                               msb_first: bool = False) -> Trie:
    a = np.ascontiguousarray(sorted_members, dtype=np.uint64)
    t = np.ascontiguousarray(table, dtype=np.uint64)
    p = C.c_void_p()
    _check(lib().gbr_trie_create_from_table(_hptr(a), a.size, M, R, int(bool(msb_first)), _hptr(t), t.size,
                                            C.byref(p)))
    return Trie(p)


def gbr_trie_info(t: Trie):
    nm, ne, eb, lv = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
    _check(lib().gbr_trie_info(t, C.byref(nm), C.byref(ne), C.byref(eb), C.byref(lv)))
    return dict(n_members=nm.value, n_elements=ne.value, entry_bytes=eb.value, levels=lv.value)


def gbr_trie_build_host(sorted_members: np.ndarray, M: int, R: int, msb_first: bool = False):
    """(size without padding, table with padding as uint64)."""
    a = np.ascontiguousarray(sorted_members, dtype=np.uint64)
    size = C.c_int64()
    o = int(bool(msb_first))
    _check(lib().gbr_trie_build_host_ordered(_hptr(a), a.size, M, R, o, None, 0, C.byref(size)))
    t = np.zeros(size.value + (1 << R), dtype=np.uint64)
    _check(lib().gbr_trie_build_host_ordered(_hptr(a), a.size, M, R, o, _hptr(t), t.size, C.byref(size)))
    return size.value, t


def gbr_trie_rank(t: Trie, pat, out, check: int = 0, stream=None):
    import torch
    _check(lib().gbr_trie_rank(t, _dptr(pat, (torch.int64,)), _dptr(out), _rank_bits(out), pat.numel(), int(check),
                               _stream(stream)))
    return out


def gbr_trie_rank_bisect(t: Trie, pat, out, check: int = 0, stream=None):
    import torch
    _check(lib().gbr_trie_rank_bisect(t, _dptr(pat, (torch.int64,)), _dptr(out), _rank_bits(out), pat.numel(),
                                      int(check), _stream(stream)))
    return out


def gbr_trie_unrank(t: Trie, rank, out, stream=None):
    import torch
    _check(lib().gbr_trie_unrank(t, _dptr(rank), _rank_bits(rank), _dptr(out, (torch.int64,)), rank.numel(),
                                 _stream(stream)))
    return out


# ----------------------------------------------------------------- Hamiltonian

def gbr_ham_create(L: int, h, U, Nup: int, Ndn: int, rank_method: int = GBR_RANK_STAGGERED) -> Ham:
    hh = np.ascontiguousarray(h, dtype=np.float64).reshape(L * L)
    uu = None if U is None else np.ascontiguousarray(U, dtype=np.float64).reshape(L)
    p = C.c_void_p()
    _check(lib().gbr_ham_create(L, _hptr(hh), None if uu is None else _hptr(uu), Nup, Ndn, rank_method, C.byref(p)))
    return Ham(p)


def gbr_ham_info(H: Ham):
    d, e = C.c_int64(), C.c_int64()
    _check(lib().gbr_ham_info(H, C.byref(d), C.byref(e)))
    return d.value, e.value


def gbr_ham_set_path(H: Ham, path: int):
    _check(lib().gbr_ham_set_path(H, path))


def gbr_release_cache():
    """Frees the stored-basis buffer the library keeps between Lanczos calls."""
    _check(lib().gbr_release_cache())


def gbr_check_rcp64(n: int = 1 << 22) -> float:
    """Largest relative error of the library's FP64 reciprocal against the division."""
    e = C.c_double()
    _check(lib().gbr_check_rcp64(n, C.byref(e)))
    return e.value


def gbr_ham_get_path(H: Ham) -> int:
    p = C.c_int(0)
    _check(lib().gbr_ham_get_path(H, C.byref(p)))
    return p.value


def gbr_ham_tune(H: Ham, fp: int = 32, stream=None):
    _check(lib().gbr_ham_tune(H, fp, _stream(stream)))


def gbr_ham_set_shape(H: Ham, fp: int, window: int, rows_dn: int = 0, rows_up: int = 0, rows_lz: int = 0,
                      chunk_bits: int = 0, threads_per_state: int = 0, threads_dn: int = 0, threads_up: int = 0,
                      threads_lz: int = 0):
    sh = np.array([window, rows_dn, rows_up, rows_lz, chunk_bits, threads_per_state, threads_dn, threads_up,
                   threads_lz], dtype=np.int32)
    _check(lib().gbr_ham_set_shape(H, fp, _hptr(sh)))


def gbr_ham_get_shape(H: Ham, fp: int) -> dict:
    sh = np.zeros(9, dtype=np.int32)
    _check(lib().gbr_ham_get_shape(H, fp, _hptr(sh)))
    return dict(window=int(sh[0]), rows_dn=int(sh[1]), rows_up=int(sh[2]), rows_lz=int(sh[3]),
                chunk_bits=int(sh[4]), threads_per_state=int(sh[5]), threads_dn=int(sh[6]),
                threads_up=int(sh[7]), threads_lz=int(sh[8]))


def gbr_device_status(clear: bool = True) -> int:
    """The device status word (0 = no bounded wait ran out); raises GbrError
    with GBR_ETIMEOUT when it is non-zero."""
    v = C.c_int(0)
    _check(lib().gbr_device_status(int(bool(clear)), C.byref(v)))
    return v.value


def gbr_hv(H: Ham, x, y, stream=None):
    import torch
    if x.dtype != y.dtype:
        raise ValueError("x and y must have the same dtype")
    fp = {torch.float32: 32, torch.float64: 64}.get(x.dtype)
    if fp is None:
        raise ValueError("x must be float32 or float64")
    _check(lib().gbr_hv(H, _dptr(x), _dptr(y), fp, _stream(stream)))
    return y


def gbr_hv_static(H: Ham, x, y, stream=None):
    """gbr_hv that allocates nothing (scratch in a static device array)."""
    import torch
    if x.dtype != y.dtype:
        raise ValueError("x and y must have the same dtype")
    fp = {torch.float32: 32, torch.float64: 64}.get(x.dtype)
    if fp is None:
        raise ValueError("x must be float32 or float64")
    _check(lib().gbr_hv_static(H, _dptr(x), _dptr(y), fp, _stream(stream)))
    return y


def gbr_hv_stage(H: Ham, x, y, stage: int, stream=None):
    import torch
    fp = {torch.float32: 32, torch.float64: 64}.get(x.dtype)
    if fp is None or y.dtype != x.dtype:
        raise ValueError("x and y must both be float32 or float64")
    _check(lib().gbr_hv_stage(H, _dptr(x), _dptr(y), fp, stage, _stream(stream)))
    return y


def gbr_launch_count() -> int:
    return lib().gbr_launch_count()


def _lanczos(fn, handle, v0, iters, reorth, prec, refine, store_basis, use_graph, want_ritz, profile, tol,
             ritz_tail, stream) -> dict:
    import torch
    o = LanczosOpts(iters, int(bool(reorth)), prec, int(bool(refine)), store_basis, int(bool(use_graph)),
                    int(bool(profile)), float(tol), float(ritz_tail))
    r = LanczosResult()
    a = np.zeros(iters, dtype=np.float64)
    b = np.zeros(max(iters, 1), dtype=np.float64)
    rz = np.zeros(iters, dtype=np.float64) if want_ritz else None
    _check(fn(handle, C.byref(o), _dptr(v0, (torch.float64,)), C.byref(r), _hptr(a), _hptr(b),
              None if rz is None else _hptr(rz), _stream(stream)))
    k = r.iters_done
    return dict(E0=r.E0, E_ritz=r.E_ritz, residual=r.residual, iters=k, breakdown=bool(r.breakdown),
                stored_basis=bool(r.stored_basis), seconds=r.seconds, hv_seconds=r.hv_seconds,
                stage_seconds=list(r.stage_seconds), stage_launches=list(r.stage_launches),
                converged=bool(r.converged), ritz_terms=r.ritz_terms, basis_head=r.basis_head,
                alpha=a[:k].copy(), beta=b[:max(k - 1, 0)].copy(), ritz=None if rz is None else rz[:k].copy())


def gbr_lanczos(H: Ham, v0, iters: int, reorth: bool = False, prec: int = GBR_PREC_MIXED, refine: bool = True,
                store_basis: int = -1, use_graph: bool = False, want_ritz: bool = False, profile: bool = False,
                tol: float = 0.0, ritz_tail: float = 0.0, stream=None) -> dict:
    return _lanczos(lib().gbr_lanczos, H, v0, iters, reorth, prec, refine, store_basis, use_graph, want_ritz,
                    profile, tol, ritz_tail, stream)


def gbr_setham_lanczos(Sh, v0, iters: int, reorth: bool = False, prec: int = GBR_PREC_MIXED, refine: bool = True,
                       store_basis: int = -1, use_graph: bool = False, want_ritz: bool = False, tol: float = 0.0,
                       ritz_tail: float = 0.0, stream=None) -> dict:
    return _lanczos(lib().gbr_setham_lanczos, Sh, v0, iters, reorth, prec, refine, store_basis, use_graph,
                    want_ritz, False, tol, ritz_tail, stream)


def gbr_termham_lanczos(Th, v0, iters: int, reorth: bool = False, prec: int = GBR_PREC_MIXED, refine: bool = True,
                        store_basis: int = -1, use_graph: bool = False, want_ritz: bool = False, tol: float = 0.0,
                        ritz_tail: float = 0.0, stream=None) -> dict:
    return _lanczos(lib().gbr_termham_lanczos, Th, v0, iters, reorth, prec, refine, store_basis, use_graph,
                    want_ritz, False, tol, ritz_tail, stream)


# ------------------------------------------------------ set Hamiltonians

def gbr_setham_create(L: int, h, U, states: np.ndarray, R: int = 8, msb_first: bool = True) -> SetHam:
    hh = np.ascontiguousarray(h, dtype=np.float64).reshape(L * L)
    uu = None if U is None else np.ascontiguousarray(U, dtype=np.float64).reshape(L)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    p = C.c_void_p()
    _check(lib().gbr_setham_create_ordered(L, _hptr(hh), None if uu is None else _hptr(uu), _hptr(st), st.size, R,
                                           int(bool(msb_first)), C.byref(p)))
    return SetHam(p)


def gbr_setham_info(S: SetHam):
    d, e, t = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().gbr_setham_info(S, C.byref(d), C.byref(e), C.byref(t)))
    return dict(dim=d.value, elements=e.value, trie_elements=t.value)


def gbr_setham_set_bisect(S: SetHam, bisect: bool):
    _check(lib().gbr_setham_set_bisect(S, int(bool(bisect))))


def gbr_setham_hv(S: SetHam, x, y, check: int = 1, stream=None):
    import torch
    if x.dtype != y.dtype:
        raise ValueError("x and y must have the same dtype")
    fp = {torch.float32: 32, torch.float64: 64}.get(x.dtype)
    if fp is None:
        raise ValueError("x must be float32 or float64")
    _check(lib().gbr_setham_hv(S, _dptr(x), _dptr(y), fp, int(check), _stream(stream)))
    return y


# -------------------------------------------------------- operator terms

def gbr_term_product(ops, coef: float = 1.0) -> Term:
    o = np.ascontiguousarray(ops, dtype=np.int32)
    t = Term()
    _check(lib().gbr_term_product(_hptr(o) if o.size else None, o.size, float(coef), C.byref(t)))
    return t


def gbr_term_mul(a: Term, b: Term) -> Term:
    t = Term()
    _check(lib().gbr_term_mul(C.byref(a), C.byref(b), C.byref(t)))
    return t


def gbr_termham_create(M: int, terms, states: np.ndarray, R: int = 8) -> TermHam:
    """terms: a sequence of Term tuples."""
    arr = (Term * len(terms))(*terms)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    p = C.c_void_p()
    _check(lib().gbr_termham_create(M, arr, len(terms), _hptr(st), st.size, R, C.byref(p)))
    return TermHam(p)


def gbr_termham_set_bisect(T: TermHam, bisect: bool):
    _check(lib().gbr_termham_set_bisect(T, int(bool(bisect))))


def gbr_termham_info(T: TermHam):
    d, e, t = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().gbr_termham_info(T, C.byref(d), C.byref(e), C.byref(t)))
    return dict(dim=d.value, elements=e.value, trie_elements=t.value)


def gbr_termham_hv(T: TermHam, x, y, check: int = 1, stream=None):
    import torch
    if x.dtype != y.dtype:
        raise ValueError("x and y must have the same dtype")
    fp = {torch.float32: 32, torch.float64: 64}.get(x.dtype)
    if fp is None:
        raise ValueError("x must be float32 or float64")
    _check(lib().gbr_termham_hv(T, _dptr(x), _dptr(y), fp, int(check), _stream(stream)))
    return y


# ---------------------------------------------------------------------- batch

def _models(models):
    keep = []
    arr = (ModelDesc * len(models))()
    for i, (h, U) in enumerate(models):
        h = np.ascontiguousarray(h, dtype=np.float64)
        L = h.shape[0]
        u = np.ascontiguousarray(np.zeros(L) if U is None else U, dtype=np.float64)
        keep += [h, u]
        arr[i] = ModelDesc(L, h.ctypes.data, u.ctypes.data)
    return arr, keep


def gbr_batch_layout(models):
    arr, keep = _models(models)
    ns, nst = C.c_int64(), C.c_int64()
    _check(lib().gbr_batch_layout(len(models), arr, C.byref(ns), C.byref(nst)))
    return ns.value, nst.value


def gbr_batch_solve(models, start, iters: int, stream=None) -> dict:
    import torch
    arr, keep = _models(models)
    ns, nst = gbr_batch_layout(models)
    if start.numel() != nst:
        raise ValueError(f"start has {start.numel()} entries, the batch has {nst} states")
    E0 = np.zeros(len(models))
    arg = np.zeros(2 * len(models), dtype=np.int32)
    sec = np.zeros(ns)
    _check(lib().gbr_batch_solve(len(models), arr, _dptr(start, (torch.float64,)), iters, _hptr(E0), _hptr(arg),
                                 _hptr(sec), _stream(stream)))
    return dict(E0=E0, arg=arg.reshape(-1, 2), sector_E=sec)


def gbr_batch_set_shape(threads: int, ctas_per_sm: int = 0):
    _check(lib().gbr_batch_set_shape(threads, ctas_per_sm))


def gbr_batch_get_shape() -> dict:
    t, p = C.c_int(), C.c_int()
    _check(lib().gbr_batch_get_shape(C.byref(t), C.byref(p)))
    return dict(threads=t.value, ctas_per_sm=p.value)


def gbr_batch_tune(models, start, iters: int, stream=None) -> dict:
    import torch
    arr, keep = _models(models)
    ns, nst = gbr_batch_layout(models)
    if start.numel() != nst:
        raise ValueError(f"start has {start.numel()} entries, the batch has {nst} states")
    sh = np.zeros(2, dtype=np.int32)
    ms = np.zeros(9, dtype=np.float32)
    _check(lib().gbr_batch_tune(len(models), arr, _dptr(start, (torch.float64,)), iters, _hptr(sh), _hptr(ms),
                                _stream(stream)))
    return dict(threads=int(sh[0]), ctas_per_sm=int(sh[1]), candidate_ms=ms.tolist())
