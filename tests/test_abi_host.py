"""CPU checks of the C ABI: the library loads, exports every symbol the
header declares, rejects bad arguments on the host, and its host-side trie
builder reproduces the paper's trie sizes and walks."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import gbr_synth as S
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbrank.h")


@pytest.fixture(scope="module")
def G():
    from paper_2203_04158_gb300 import build as gbuild
    gbuild.build()
    import paper_2203_04158_gb300 as G
    return G


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_api():
    syms = declared_symbols()
    for s in ("gbr_comb_rank", "gbr_trie_rank", "gbr_hv", "gbr_lanczos", "gbr_batch_solve", "gbr_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(G):
    lib = C.CDLL(G.gbrank.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert G.gbr_version() == 1


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs (options, results, term
    tuples, model descriptions) have the C layout: sizes and every field's
    offset, from a C program compiled against the header."""
    import subprocess
    from paper_2203_04158_gb300 import gbrank as B
    pairs = [("gbr_lanczos_opts", B.LanczosOpts), ("gbr_lanczos_result", B.LanczosResult),
             ("gbr_term", B.Term), ("gbr_model_desc", B.ModelDesc)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gbrank.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("%zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for _, py in pairs:
        want.append(C.sizeof(py))
        want += [getattr(py, f[0]).offset for f in py._fields_]
    assert got == want


def test_null_handles_are_rejected_on_the_host(G):
    lib = C.CDLL(G.gbrank.LIB_PATH)
    assert lib.gbr_release_cache() == G.GBR_OK          # nothing cached: no device call
    path = C.c_int(-1)
    assert lib.gbr_ham_get_path(None, C.byref(path)) == G.GBR_EINVAL and path.value == -1
    assert lib.gbr_ham_set_path(None, 0) == G.GBR_EINVAL
    assert lib.gbr_ham_info(None, None, None) == G.GBR_EINVAL


def test_shape_status_and_operator_lanczos_validate_on_the_host(G):
    """The launch-shape, device-status and set/term Lanczos entry points
    reject NULL arguments before touching a device."""
    lib = C.CDLL(G.gbrank.LIB_PATH)
    shape = (C.c_int * 9)(1, 64, 64, 64, 8, 1, 0, 0, 0)
    assert lib.gbr_ham_set_shape(None, 32, shape) == G.GBR_EINVAL
    assert lib.gbr_ham_get_shape(None, 32, shape) == G.GBR_EINVAL
    assert lib.gbr_device_status(0, None) == G.GBR_EINVAL
    opts = G.gbrank.LanczosOpts(10, 0, 1, 1, 0, 0, 0, 0.0, 0.0)
    res = G.gbrank.LanczosResult()
    for fn in (lib.gbr_setham_lanczos, lib.gbr_termham_lanczos):
        fn.argtypes = [C.c_void_p] * 8
        assert fn(None, C.byref(opts), None, C.byref(res), None, None, None, None) == G.GBR_EINVAL
        assert b"NULL" in lib_last_error(lib)


def lib_last_error(lib):
    lib.gbr_last_error.restype = C.c_char_p
    return lib.gbr_last_error()


def test_new_entry_points_validate_on_the_host(G):
    lib = C.CDLL(G.gbrank.LIB_PATH)
    members = np.array([1, 5, 9], dtype=np.uint64)
    pm = members.ctypes.data_as(C.c_void_p)
    out = C.c_void_p()
    size = C.c_int64()
    assert lib.gbr_trie_create_ordered(pm, C.c_int64(3), 8, 4, 2, C.byref(out)) == G.GBR_EINVAL
    assert lib.gbr_trie_build_host_ordered(pm, C.c_int64(3), 8, 4, -1, None, C.c_int64(0), C.byref(size)) == G.GBR_EINVAL
    assert lib.gbr_trie_build_host_ordered(pm, C.c_int64(3), 8, 4, 1, None, C.c_int64(0), C.byref(size)) == G.GBR_OK
    assert size.value > 0
    err = C.c_double()
    assert lib.gbr_check_rcp64(C.c_int64(0), C.byref(err)) == G.GBR_EINVAL
    assert lib.gbr_setham_set_bisect(None, 1) == G.GBR_EINVAL


def test_host_argument_errors(G):
    with pytest.raises(G.GbrError) as e:
        G.gbr_comb_create(65, 3, 8)
    assert e.value.code == G.GBR_EINVAL and "M=65" in str(e.value)
    with pytest.raises(G.GbrError):
        G.gbr_comb_create(10, 11, 8)
    with pytest.raises(G.GbrError):
        G.gbr_comb_create(10, 3, 0)
    # unsorted, duplicate and too-wide trie members are rejected before any device work
    for bad in ([3, 1], [1, 1], [1 << 12]):
        with pytest.raises(G.GbrError) as e:
            G.gbr_trie_build_host(np.array(bad, dtype=np.uint64), 12, 4)
        assert e.value.code == G.GBR_EINVAL
    with pytest.raises(G.GbrError):
        G.gbr_ham_create(4, np.array([[0, 1, 0, 0], [0.5, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]), None, 2, 2)
    with pytest.raises(G.GbrError):
        G.gbr_ham_create(33, np.zeros((33, 33)), None, 2, 2)


def walk(t, M, R, a, msb_first=False):
    """Fig. trielookup over the host-built table, with the wrap-around pointer
    arithmetic of the unsigned entries and clamping into the table; with
    msb_first the chunks are taken from the top bits down (the short chunk
    first, at the top)."""
    w0 = M % R or R
    widths = [w0] + [R] * ((M - w0) // R)
    k, done = 0, 0
    for w in widths:
        sh = M - done - w if msb_first else done
        idx = (k + ((a >> sh) & ((1 << w) - 1))) % (1 << 64)
        idx = min(idx, t.size - 1)
        k = int(t[idx])
        done += w
    return k


def test_host_trie_matches_worked_example_size_and_walk(G):
    lst = oracle.enumerate_sector(6, 2)
    size, t = G.gbr_trie_build_host(lst, 6, 2)
    osize, _ = oracle.trie_build(lst, 6, 2)
    assert size == osize == 30
    for i, a in enumerate(lst):
        assert walk(t, 6, 2, int(a)) == i


@pytest.mark.parametrize("M,R", [(7, 3), (10, 4), (12, 5), (16, 8), (20, 8), (11, 12)])
def test_host_trie_random_sets(G, M, R):
    rng = np.random.default_rng(M + 7 * R)
    members = np.sort(rng.choice(1 << M, size=min(300, 1 << (M - 1)), replace=False).astype(np.uint64))
    size, t = G.gbr_trie_build_host(members, M, R)
    osize, _ = oracle.trie_build(members, M, R)
    assert size == osize
    for i, a in enumerate(members):
        assert walk(t, M, R, int(a)) == i


@pytest.mark.parametrize("M,R", [(7, 3), (10, 4), (12, 5), (16, 8), (20, 8), (11, 12), (40, 8)])
def test_host_trie_most_significant_first(G, M, R):
    """The most-significant-first order ranks every member correctly, reads
    nothing for non-members beyond the table, and on a fixed-popcount sector
    has the size of the paper's order."""
    rng = np.random.default_rng(M + 11 * R)
    if M <= 20:
        members = np.sort(rng.choice(1 << M, size=min(300, 1 << (M - 1)), replace=False).astype(np.uint64))
    else:
        members = np.unique(rng.integers(0, 1 << M, size=3000, dtype=np.uint64))
    size, t = G.gbr_trie_build_host(members, M, R, msb_first=True)
    for i, a in enumerate(members):
        assert walk(t, M, R, int(a), msb_first=True) == i
    others = np.setdiff1d(rng.integers(0, 1 << min(M, 20), size=200, dtype=np.uint64), members)
    for a in others:
        walk(t, M, R, int(a), msb_first=True)          # stays inside the table (clamped)
    sector = oracle.enumerate_sector(14, 5)
    assert G.gbr_trie_build_host(sector, 14, 4, msb_first=True)[0] == G.gbr_trie_build_host(sector, 14, 4)[0]


@pytest.mark.slow
def test_host_trie_overhead_factors(G):
    # the breadth-first table has exactly the oracle's element count, hence the paper's f
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_examples.json")))["trie_overhead"]
    lists = {}
    for row in gold["rows"]:
        if row["N"] not in lists:
            lists[row["N"]] = oracle.enumerate_sector(28, row["N"])
        lst = lists[row["N"]]
        size = G.gbr_trie_build_host(lst, 28, row["R"])[0] if row["R"] != 4 or row["N"] == 5 else None
        if size is None:
            continue
        assert round(size / lst.size, 2) == row["f"], row


def test_seeded_generator_twins_agree():
    idx = np.array([0, 1, 2, 12345, 2**40 + 3], dtype=np.uint64)
    py = S.uniform(1, idx)
    for i, v in zip(idx, py):
        assert oracle.seeded_uniform(1, int(i)) == v


def tuple_apply_right(t, a):
    """Eq. Talpha1 on a basis state: (coefficient, result) or (0, None)."""
    if (a & t.m) != t.r or t.v == 0.0:
        return 0.0, None
    sgn = -1.0 if bin(a & t.s).count("1") & 1 else 1.0
    return t.v * sgn, a ^ t.x


def tuple_apply_left(t, a):
    """Eq. Talpha2: <a| T = coefficient <result|."""
    if (a & t.m) != t.l or t.v == 0.0:
        return 0.0, None
    sgn = -1.0 if bin(a & t.s).count("1") & 1 else 1.0
    return t.v * sgn, a ^ t.x


def test_building_blocks_follow_eqs_ci(G):
    for i in (0, 3, 17, 63):
        c = G.gbr_term_product([2 * i])
        cd = G.gbr_term_product([2 * i + 1])
        b = 1 << i
        assert (c.v, c.m, c.l, c.r, c.x, c.s) == (1.0, b, 0, b, b, b - 1)
        assert (cd.v, cd.m, cd.l, cd.r, cd.x, cd.s) == (1.0, b, b, 0, b, b - 1)


@pytest.mark.parametrize("seed", range(6))
def test_product_rule_matches_literal_operator_application(G, seed):
    """Fig. mul, built up operator by operator, reproduces Eq. cee applied
    literally for every basis state -- from the right (Talpha1) and, for the
    transpose matrix element, from the left (Talpha2)."""
    rng = np.random.default_rng(seed)
    M = 7
    for _ in range(60):
        k = int(rng.integers(1, 7))
        ops = [int(rng.integers(0, 2 * M)) for _ in range(k)]
        coef = float(rng.normal())
        t = G.gbr_term_product(ops, coef)
        for a in range(1 << M):
            sgn, b = oracle.apply_ops(ops, a)
            cv, cb = tuple_apply_right(t, a)
            if sgn == 0:
                assert cv == 0.0
            else:
                assert cb == b and cv == pytest.approx(coef * sgn, abs=1e-15)
                # <b| T |a> = coef*sgn: the left application of T to <b| lands on <a|
                lv, lb = tuple_apply_left(t, b)
                assert lb == a and lv == pytest.approx(coef * sgn, abs=1e-15)


def test_mul_is_the_product_of_terms(G):
    rng = np.random.default_rng(9)
    for _ in range(100):
        A = [int(x) for x in rng.integers(0, 12, size=int(rng.integers(1, 4)))]
        B = [int(x) for x in rng.integers(0, 12, size=int(rng.integers(1, 4)))]
        ab = G.gbr_term_mul(G.gbr_term_product(A, 2.0), G.gbr_term_product(B, -0.5))
        ref = G.gbr_term_product(A + B, -1.0)
        if ref.v == 0.0:
            assert ab.v == 0.0
        else:
            assert (ab.v, ab.m, ab.l, ab.r, ab.x, ab.s) == (ref.v, ref.m, ref.l, ref.r, ref.x, ref.s)


def test_term_and_set_hamiltonians_reject_bad_input_on_the_host(G):
    t = G.gbr_term_product([2 * 9 + 1, 2 * 0])                 # touches orbital 9
    with pytest.raises(G.GbrError) as e:
        G.gbr_termham_create(8, [t], np.array([1, 2], dtype=np.uint64))
    assert e.value.code == G.GBR_EINVAL and "orbitals" in str(e.value)
    with pytest.raises(G.GbrError):
        G.gbr_term_product([200])                               # orbital 100
    with pytest.raises(G.GbrError):
        G.gbr_termham_create(65, [t], np.array([1], dtype=np.uint64))
    hbad = np.zeros((3, 3)); hbad[0, 1] = 1.0                   # not symmetric
    with pytest.raises(G.GbrError):
        G.gbr_setham_create(3, hbad, None, np.array([1, 2], dtype=np.uint64))
