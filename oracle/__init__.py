"""ORACLE -- test infrastructure only.

Plain, slow, obviously-correct CPU reference for the ranking, H·v and Lanczos
quantities of Wallerberger & Held, "Trie-based ranking of quantum many-body
states".  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import it; the product path (the CUDA library and its binding)
never does, and shares no code with it.

The C part (``oracle.c``) is compiled with plain gcc on first use.  The Python
part adds what numpy does best: dense diagonalisation (``numpy.linalg.eigvalsh``)
of small sectors and the non-interacting closed form.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NOT_FOUND = -1


def build(force: bool = False) -> str:
    """Compile oracle.c to a shared library with gcc (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u64, i64, i32, dbl = C.c_uint64, C.c_int64, C.c_int, C.c_double
            vp = C.c_void_p
            L.ora_binom.restype = u64; L.ora_binom.argtypes = [i32, i32]
            L.ora_enumerate.restype = i64; L.ora_enumerate.argtypes = [i32, i32, vp, i64]
            L.ora_rank_bisect.restype = i64; L.ora_rank_bisect.argtypes = [vp, i64, u64]
            L.ora_rank_count.restype = u64; L.ora_rank_count.argtypes = [i32, u64]
            L.ora_unrank_greedy.restype = u64; L.ora_unrank_greedy.argtypes = [i32, i32, u64]
            L.ora_trie_build.restype = i64; L.ora_trie_build.argtypes = [vp, i64, i32, i32, vp, i64]
            L.ora_trie_rank.restype = i64; L.ora_trie_rank.argtypes = [vp, i64, i32, i32, u64]
            L.ora_sector_dim.restype = i64; L.ora_sector_dim.argtypes = [i32, i32, i32]
            L.ora_sector_states.restype = i32; L.ora_sector_states.argtypes = [i32, i32, i32, vp]
            L.ora_sector_rank_of.restype = i64; L.ora_sector_rank_of.argtypes = [i32, i32, i32, u64]
            L.ora_hv_full.restype = i32; L.ora_hv_full.argtypes = [i32, vp, vp, i32, i32, vp, vp]
            L.ora_hv_rows.restype = i32; L.ora_hv_rows.argtypes = [i32, vp, vp, i32, i32, vp, vp, i64, vp]
            L.ora_hv_rows_seeded.restype = i32
            L.ora_hv_rows_seeded.argtypes = [i32, vp, vp, i32, i32, u64, vp, i64, vp]
            L.ora_seeded_uniform.restype = dbl; L.ora_seeded_uniform.argtypes = [u64, u64]
            L.ora_hv_set.restype = i32; L.ora_hv_set.argtypes = [i32, vp, vp, vp, i64, vp, vp, vp]
            L.ora_hv_ops.restype = i32
            L.ora_hv_ops.argtypes = [vp, vp, vp, vp, i32, vp, i64, vp, vp, vp]
            L.ora_apply_ops.restype = i32; L.ora_apply_ops.argtypes = [vp, i32, u64, vp]
            L.ora_count_elements.restype = i64; L.ora_count_elements.argtypes = [i32, vp, i32, i32, i64, i64]
            L.ora_dense.restype = i32; L.ora_dense.argtypes = [i32, vp, vp, i32, i32, vp]
            L.ora_tridiag_lowest.restype = dbl; L.ora_tridiag_lowest.argtypes = [vp, vp, i32]
            L.ora_lanczos.restype = i32
            L.ora_lanczos.argtypes = [i32, vp, vp, i32, i32, vp, i32, i32, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ ranking

def binom(n: int, k: int) -> int:
    return int(lib().ora_binom(n, k))


def enumerate_sector(M: int, N: int) -> np.ndarray:
    """C^M_N in lexicographic (= increasing numeric) order, by brute force."""
    n = binom(M, N)
    out = np.empty(n, dtype=np.uint64)
    got = lib().ora_enumerate(M, N, _p(out), n)
    if got != n:
        raise RuntimeError("enumeration count differs from C(M, N)")
    return out


def rank_bisect(sorted_list: np.ndarray, alpha: int) -> int:
    a = np.ascontiguousarray(sorted_list, dtype=np.uint64)
    return int(lib().ora_rank_bisect(_p(a), a.size, int(alpha)))


def rank_bisect_many(sorted_list: np.ndarray, alphas) -> np.ndarray:
    a = np.ascontiguousarray(sorted_list, dtype=np.uint64)
    f = lib().ora_rank_bisect
    return np.array([f(_p(a), a.size, int(x)) for x in np.asarray(alphas, dtype=np.uint64)], dtype=np.int64)


def rank_count(M: int, alpha: int) -> int:
    return int(lib().ora_rank_count(M, int(alpha)))


def unrank(M: int, N: int, i: int) -> int:
    return int(lib().ora_unrank_greedy(M, N, int(i)))


def trie_build(sorted_members: np.ndarray, M: int, R: int, with_table: bool = True):
    """Packed trie of Sec. IV (depth-first layout).  Returns (size, t or None)."""
    a = np.ascontiguousarray(sorted_members, dtype=np.uint64)
    size = int(lib().ora_trie_build(_p(a), a.size, M, R, None, 0))
    if size < 0:
        raise ValueError("bad trie input")
    if not with_table:
        return size, None
    t = np.empty(size, dtype=np.int64)
    lib().ora_trie_build(_p(a), a.size, M, R, _p(t), size)
    return size, t


def trie_rank(t: np.ndarray, M: int, R: int, alpha: int) -> int:
    return int(lib().ora_trie_rank(_p(t), t.size, M, R, int(alpha)))


# ----------------------------------------------------------------- sectors

def sector_dim(L: int, Nup: int, Ndn: int) -> int:
    return int(lib().ora_sector_dim(L, Nup, Ndn))


def sector_states(L: int, Nup: int, Ndn: int) -> np.ndarray:
    out = np.empty(sector_dim(L, Nup, Ndn), dtype=np.uint64)
    if lib().ora_sector_states(L, Nup, Ndn, _p(out)):
        raise ValueError("bad sector")
    return out


def sector_rank(L: int, Nup: int, Ndn: int, alpha: int) -> int:
    return int(lib().ora_sector_rank_of(L, Nup, Ndn, int(alpha)))


# -------------------------------------------------------------------- H·v

def _hU(L, h, U):
    h = _f64(h).reshape(L, L)
    U = _f64(np.zeros(L) if U is None else U).reshape(L)
    return h, U


def hv(L, h, U, Nup, Ndn, x) -> np.ndarray:
    """y = H x over the whole sector (scatter form, Eq. mvblock)."""
    h, U = _hU(L, h, U)
    x = _f64(x)
    y = np.empty_like(x)
    rc = lib().ora_hv_full(L, _p(h), _p(U), Nup, Ndn, _p(x), _p(y))
    if rc:
        raise RuntimeError(f"ora_hv_full failed: {rc}")
    return y


def hv_rows(L, h, U, Nup, Ndn, x, rows) -> np.ndarray:
    """Rows ``rows`` of H x (gather form)."""
    h, U = _hU(L, h, U)
    x = _f64(x)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(r.size, dtype=np.float64)
    rc = lib().ora_hv_rows(L, _p(h), _p(U), Nup, Ndn, _p(x), _p(r), r.size, _p(y))
    if rc:
        raise RuntimeError(f"ora_hv_rows failed: {rc}")
    return y


def hv_rows_seeded(L, h, U, Nup, Ndn, seed: int, rows) -> np.ndarray:
    """Rows of H x with x_j = uniform[-1,1)(seed, j) generated on demand."""
    h, U = _hU(L, h, U)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(r.size, dtype=np.float64)
    rc = lib().ora_hv_rows_seeded(L, _p(h), _p(U), Nup, Ndn, int(seed), _p(r), r.size, _p(y))
    if rc:
        raise RuntimeError(f"ora_hv_rows_seeded failed: {rc}")
    return y


def seeded_uniform(seed: int, i: int) -> float:
    return float(lib().ora_seeded_uniform(int(seed), int(i)))


def hv_set(L, h, U, states, x):
    """y = P H P x over the sorted set ``states``; returns (y, dropped terms)."""
    h, U = _hU(L, h, U)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    x = _f64(x)
    y = np.empty(st.size, dtype=np.float64)
    dropped = C.c_int64(0)
    lib().ora_hv_set(L, _p(h), _p(U), _p(st), st.size, _p(x), _p(y), C.byref(dropped))
    return y, dropped.value


def fixed_N_states(L: int, N: int) -> np.ndarray:
    """All 2L-bit states with N particles in total (every S_z), sorted."""
    return enumerate_sector(2 * L, N)


def _flatten_terms(terms):
    coef = np.array([c for c, _ in terms], dtype=np.float64)
    nops = np.array([len(o) for _, o in terms], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(nops)[:-1]]).astype(np.int32)
    ops = np.array([code for _, o in terms for code in o] or [0], dtype=np.int32)
    return coef, nops, off, ops


def hv_ops(terms, states, x):
    """y = P H P x for H = sum of operator products ``terms`` = [(coef, [op codes
    left to right])], op code = 2*orbital + creator; returns (y, dropped)."""
    coef, nops, off, ops = _flatten_terms(terms)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    x = _f64(x)
    y = np.empty(st.size)
    dropped = C.c_int64(0)
    lib().ora_hv_ops(_p(coef), _p(nops), _p(off), _p(ops), len(terms), _p(st), st.size, _p(x), _p(y),
                     C.byref(dropped))
    return y, dropped.value


def apply_ops(ops, alpha: int):
    """Literal product application: (sign, resulting pattern)."""
    o = np.ascontiguousarray(ops, dtype=np.int32)
    b = C.c_uint64(0)
    sgn = lib().ora_apply_ops(_p(o), o.size, int(alpha), C.byref(b))
    return sgn, b.value


def dense_ops(terms, states) -> np.ndarray:
    """Dense matrix of P H P on the set (columns by applying H to unit vectors)."""
    n = len(states)
    Hm = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        Hm[:, j] = hv_ops(terms, states, e)[0]
    return Hm


def count_elements(L, h, Nup, Ndn, row0: int = 0, row1: int = 0) -> int:
    h, _ = _hU(L, h, None)
    return int(lib().ora_count_elements(L, _p(h), Nup, Ndn, row0, row1))


def dense(L, h, U, Nup, Ndn) -> np.ndarray:
    h, U = _hU(L, h, U)
    D = sector_dim(L, Nup, Ndn)
    Hm = np.empty((D, D), dtype=np.float64)
    if lib().ora_dense(L, _p(h), _p(U), Nup, Ndn, _p(Hm)):
        raise RuntimeError("ora_dense failed")
    return Hm


def dense_E0(L, h, U, Nup, Ndn) -> float:
    """Lowest eigenvalue of the dense sector matrix (numpy eigvalsh)."""
    return float(np.linalg.eigvalsh(dense(L, h, U, Nup, Ndn))[0])


def free_E0(h, Nup: int, Ndn: int) -> float:
    """U = 0 closed form: sum of the lowest N_up plus lowest N_dn one-body levels."""
    e = np.linalg.eigvalsh(_f64(h))
    return float(e[:Nup].sum() + e[:Ndn].sum())


def tridiag_lowest(a, b) -> float:
    a = _f64(a); b = _f64(b if len(b) else [0.0])
    return float(lib().ora_tridiag_lowest(_p(a), _p(b), a.size))


def lanczos(L, h, U, Nup, Ndn, s0, iters: int, reorth: bool):
    """FP64 Lanczos; returns dict(E0, alpha, beta, k, ritz)."""
    h, U = _hU(L, h, U)
    s0 = _f64(s0)
    a = np.zeros(iters); b = np.zeros(max(iters, 1)); e = np.zeros(iters)
    k = C.c_int(0); E0 = C.c_double(0.0)
    rc = lib().ora_lanczos(L, _p(h), _p(U), Nup, Ndn, _p(s0), iters, int(bool(reorth)), _p(a), _p(b),
                           C.byref(k), C.byref(E0), _p(e))
    if rc:
        raise RuntimeError(f"ora_lanczos failed: {rc}")
    kk = k.value
    return dict(E0=E0.value, alpha=a[:kk].copy(), beta=b[:max(kk - 1, 0)].copy(), k=kk, ritz=e[:kk].copy())


def bethe_ansatz_E0(L: int, Nup: int, Ndn: int, U: float, t: float = 1.0, shift: int = 0, tol: float = 1e-14):
    """Ground-state energy of the periodic Hubbard ring, H = -t sum (c+_{i+1} c_i + h.c.) + U sum n_up n_dn,
    from the Lieb-Wu Bethe-ansatz equations (textbook; not in the paper), for U > 0.

    With N = Nup + Ndn electrons, M = min(Nup, Ndn) rapidities Lambda and
    theta(x) = 2 arctan(x), the logarithmic equations are
        L k_j = 2 pi I_j - sum_b theta((sin k_j - Lambda_b) / (U / 4t)),
        sum_j theta((Lambda_a - sin k_j) / (U / 4t)) = 2 pi J_a + sum_b theta((Lambda_a - Lambda_b) / (U / 2t)),
    and E = -2t sum_j cos k_j.  Taking logarithms of the product form fixes
    the quantum numbers' parity: I_j is an integer for even M and half an odd
    integer for odd M; J_a is an integer for odd N - M and half an odd
    integer for even N - M.  The ground state takes consecutive I_j and J_a
    centred on zero; when the parity forbids exact centring (the open-shell
    fillings) the I_j are centred on +1/2 (shift = 0) or -1/2 (shift = 1).
    (These consecutive quantum numbers give the ground state at the fillings
    the tests compare with dense diagonalisation; not at every filling.)
    Solved by Newton's method (finite-difference Jacobian), first at U = 4t
    from the U = 0 momenta, then continued in small steps of U when U is
    elsewhere.  Returns (E0, k, Lambda).
    """
    N, M = Nup + Ndn, min(Nup, Ndn)
    if U <= 0 or M < 0 or N > 2 * L:
        raise ValueError("needs U > 0 and a valid filling")
    i_half = 0.5 if M % 2 else 0.0
    j_half = 0.0 if (N - M) % 2 else 0.5

    def centred(n, half, s):
        base = np.arange(n) - (n - 1) / 2.0
        if n and abs((base[0] - half) - round(base[0] - half)) > 1e-9:   # parity forbids centring
            base = base + (0.5 if s == 0 else -0.5)
        return base

    I = centred(N, i_half, shift)
    J = centred(M, j_half, 0)
    th = lambda x: 2.0 * np.arctan(x)

    def resid(z, c):
        kk, ll = z[:N], z[N:]
        sk = np.sin(kk)
        r1 = L * kk - 2.0 * np.pi * I + th((sk[:, None] - ll[None, :]) / c).sum(axis=1)
        r2 = (th((ll[:, None] - sk[None, :]) / c).sum(axis=1) - 2.0 * np.pi * J
              - th((ll[:, None] - ll[None, :]) / (2 * c)).sum(axis=1))
        return np.concatenate([r1, r2])

    def solve(z, c):
        for _ in range(100):
            r = resid(z, c)
            if np.max(np.abs(r)) < tol:
                break
            h = 1e-7
            Jm = np.empty((z.size, z.size))
            for q in range(z.size):
                dz = np.zeros(z.size)
                dz[q] = h
                Jm[:, q] = (resid(z + dz, c) - resid(z - dz, c)) / (2 * h)
            step = np.linalg.solve(Jm, -r)
            lamb = 1.0
            while lamb > 1e-4 and np.max(np.abs(resid(z + lamb * step, c))) > np.max(np.abs(r)):
                lamb *= 0.5
            z = z + lamb * step
        return z, float(np.max(np.abs(resid(z, c))))

    z = np.concatenate([2.0 * np.pi * I / L, np.linspace(-0.5, 0.5, M)])
    z, res = solve(z, 1.0)                        # U = 4t
    Us = [4.0 * t]
    if U != 4.0 * t:
        n = max(1, int(np.ceil(abs(np.log(U / (4.0 * t))) / 0.05)))
        Us = list(4.0 * t * (U / (4.0 * t)) ** (np.arange(1, n + 1) / n))
    for Ui in Us:
        z, res = solve(z, Ui / (4.0 * t))
    if res > 1e-10:
        raise RuntimeError(f"Bethe-ansatz equations did not converge (residual {res:.2e})")
    kk = z[:N]
    return float(-2.0 * t * np.cos(kk).sum()), kk, z[N:]
