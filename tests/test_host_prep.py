"""The host-side layout (paper_2511_13894_gb300/csrc/host_prep.cpp) on the CPU.

host_prep.cpp is plain C++: the test compiles it with g++ together with a
small dump driver (tests/host_prep_dump.cpp), runs it on an LP with every
row class (CTA, warp and SELL-32 rows, empty rows, ties in length) and checks
the layout against its definition: the permutations sort rows and columns
by decreasing length, stably; the internal A is the user's A permuted with
'<' rows negated; A' is its transpose; every SELL slot maps to the right CSR
entry and every SELL row entry appears exactly once; the blocks cover the
slices; and invalid inputs get the documented error codes.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_13894_gb300", "csrc")

EQ, LE, GE = ord("="), ord("<"), ord(">")


def _constants():
    src = open(os.path.join(CSRC, "host_prep.h")).read()
    get = lambda name: int(re.search(rf"constexpr int {name} = (\d+);", src).group(1))  # noqa: E731
    block, sell_h, cols_per_warp, warp_max = get("kBlock"), get("kSellH"), get("kColsPerWarp"), get("kWarpMaxLen")
    return dict(warps=block // 32, sell_h=sell_h, cols_per_warp=cols_per_warp,
                sell_max=cols_per_warp * (block // 32), warp_max=warp_max)


K = _constants()


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hp") / "host_prep_dump")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host_prep_dump.cpp"),
                    os.path.join(CSRC, "host_prep.cpp"), "-o", out], check=True, capture_output=True)
    return out


def _run(exe, tmp_path, lp, chunk=None, sms=None):
    m, n = lp["m"], lp["n"]
    rp = np.asarray(lp["row_ptr"], dtype=np.int64)
    nnz = int(lp.get("nnz", rp[-1]))
    flags = (1 if lp.get("lb") is not None else 0) | (2 if lp.get("ub") is not None else 0) | \
        (4 if lp.get("sense") is not None else 0)
    path_in, path_out = str(tmp_path / "lp.bin"), str(tmp_path / "layout.bin")
    with open(path_in, "wb") as f:
        np.array([m, n, nnz, flags], dtype=np.int64).tofile(f)
        rp.tofile(f)
        np.asarray(lp["col_idx"], dtype=np.int32)[:nnz].tofile(f)
        np.asarray(lp["val"], dtype=np.float64)[:nnz].tofile(f)
        np.asarray(lp["b"], dtype=np.float64).tofile(f)
        np.asarray(lp["c"], dtype=np.float64).tofile(f)
        for key, dt in (("lb", np.float64), ("ub", np.float64), ("sense", np.int8)):
            if lp.get(key) is not None:
                np.asarray(lp[key], dtype=dt).tofile(f)
    extra = [str(chunk), str(sms)] if chunk is not None else []
    subprocess.run([exe, path_in, path_out, *extra], check=True)
    data = open(path_out, "rb").read()
    rc = int(np.frombuffer(data, np.int64, 1, 0)[0])
    dl = int(np.frombuffer(data, np.int64, 1, 8)[0])
    pos = 16 + dl
    arrays = {}
    types = {0: np.int32, 1: np.float64, 2: np.int8}
    while pos < len(data):
        ln = int(np.frombuffer(data, np.int32, 1, pos)[0])
        name = data[pos + 4:pos + 4 + ln].decode()
        pos += 4 + ln
        ty = types[int(np.frombuffer(data, np.int32, 1, pos)[0])]
        cnt = int(np.frombuffer(data, np.int64, 1, pos + 4)[0])
        pos += 12
        arrays[name] = np.frombuffer(data, ty, cnt, pos).copy()
        pos += cnt * np.dtype(ty).itemsize
    return rc, arrays


def _layout_lp(seed=0):
    """300 x 6000: one row of 5000 nonzeros (a CTA row), rows of 300-1000 (warp
    rows), short rows of 0-60 with many ties (SELL-32, empty rows), column 0 in
    every row (a warp row of A'); entries of a row in random column order."""
    rng = np.random.default_rng(seed)
    m, n = 300, 6000
    lens = rng.integers(1, 61, size=m)
    lens[[3, 50, 77, 120, 200, 250]] = rng.integers(300, 1001, size=6)  # warp rows
    lens[17] = 5000                                                     # a CTA row
    lens[[8, 9, 60, 61, 130, 131, 210, 211, 280, 299]] = 0              # empty rows
    cols, rp = [], [0]
    for i in range(m):
        c = rng.choice(np.arange(1, n), size=lens[i], replace=False) if lens[i] else np.zeros(0, np.int64)
        if lens[i]:
            c[rng.integers(0, lens[i])] = 0  # column 0 in every non-empty row
        cols.append(c)
        rp.append(rp[-1] + len(c))
    col = np.concatenate(cols).astype(np.int32)
    sense = rng.choice(np.array([EQ, LE, GE], dtype=np.int8), size=m)
    lb = np.where(rng.random(n) < 0.3, -np.inf, rng.uniform(-2, 0, n))
    ub = np.where(rng.random(n) < 0.4, np.inf, rng.uniform(1, 3, n))
    return dict(m=m, n=n, row_ptr=np.array(rp, dtype=np.int64), col_idx=col,
                val=rng.standard_normal(len(col)), b=rng.standard_normal(m), c=rng.standard_normal(n),
                lb=lb, ub=ub, sense=sense)


def _dense(rp, col, val, rows, cols):
    D = np.zeros((rows, cols))
    for r in range(rows):
        for e in range(rp[r], rp[r + 1]):
            D[r, col[e]] += val[e]
    return D


def _check_csr_segments(prefix, a):
    rp, seg = a[prefix + ".row_ptr"], a[prefix + ".seg"]
    cta_rows, long_rows, nslices = (int(v) for v in seg)
    lens = np.diff(rp)
    R = len(lens)
    assert np.all(lens[:cta_rows] > K["warp_max"])
    assert np.all((lens[cta_rows:long_rows] > K["sell_max"]) & (lens[cta_rows:long_rows] <= K["warp_max"]))
    assert np.all(lens[long_rows:] <= K["sell_max"])
    assert nslices == -(-(R - long_rows) // K["sell_h"])
    sp, sw, smap = a[prefix + ".slice_ptr"], a[prefix + ".slice_w"], a[prefix + ".sell_map"]
    seen = np.zeros(rp[-1], dtype=np.int64)
    for s in range(nslices):
        rows = np.arange(long_rows + s * K["sell_h"], min(R, long_rows + (s + 1) * K["sell_h"]))
        assert sw[s] == lens[rows].max() == lens[rows[0]]
        assert sp[s + 1] - sp[s] == sw[s] * K["sell_h"]
        for t in range(K["sell_h"]):
            for j in range(sw[s]):
                slot = smap[sp[s] + j * K["sell_h"] + t]
                if t < len(rows) and j < lens[rows[t]]:
                    assert slot == rp[rows[t]] + j
                    seen[slot] += 1
                else:
                    assert slot == -1
    sell_entries = np.zeros(rp[-1], dtype=bool)
    sell_entries[rp[long_rows]:] = True
    assert np.all(seen[sell_entries] == 1) and np.all(seen[~sell_entries] == 0)
    # blocks: consecutive, K warps per slice (the least power of two giving
    # each warp at most cols_per_warp columns, capped at the CTA's warps)
    blocks = a[prefix + ".sell_blocks"].reshape(-1, 4)
    nxt = 0
    for first, count, k, _ in blocks:
        assert first == nxt and count >= 1 and k in (1, 2, 4, 8) and count * k <= K["warps"]
        for s in range(first, first + count):
            want = 1
            while want < K["warps"] and want * K["cols_per_warp"] < sw[s]:
                want *= 2
            assert k == want
        nxt = first + count
    assert nxt == nslices
    return cta_rows, long_rows


def test_layout_matches_its_definition(dump_exe, tmp_path):
    lp = _layout_lp()
    rc, a = _run(dump_exe, tmp_path, lp)
    assert rc == 0
    m, n = lp["m"], lp["n"]
    rlen = np.diff(lp["row_ptr"])
    clen = np.bincount(lp["col_idx"], minlength=n)
    # stable order by decreasing length
    assert np.array_equal(a["row_perm"], np.argsort(-rlen, kind="stable"))
    assert np.array_equal(a["col_perm"], np.argsort(-clen, kind="stable"))
    assert np.array_equal(a["row_inv"][a["row_perm"]], np.arange(m))
    assert np.array_equal(a["col_inv"][a["col_perm"]], np.arange(n))
    # internal A = sign * user A, rows and columns permuted; entries keep the
    # user's order within a row
    user = _dense(lp["row_ptr"], lp["col_idx"], lp["val"], m, n)
    sign = np.where(lp["sense"][a["row_perm"]] == LE, -1.0, 1.0)
    A = _dense(a["A.row_ptr"], a["A.col"], a["A.val"], m, n)
    assert np.array_equal(A, sign[:, None] * user[np.ix_(a["row_perm"], a["col_perm"])])
    for r in (0, 5, 150, m - 1):
        i = a["row_perm"][r]
        e0, e1 = lp["row_ptr"][i], lp["row_ptr"][i + 1]
        assert np.array_equal(a["A.col"][a["A.row_ptr"][r]:a["A.row_ptr"][r + 1]],
                              a["col_inv"][lp["col_idx"][e0:e1]])
    # A' is the transpose, each row in increasing internal row order
    AT = _dense(a["AT.row_ptr"], a["AT.col"], a["AT.val"], n, m)
    assert np.array_equal(AT, A.T)
    for j in range(n):
        seg = a["AT.col"][a["AT.row_ptr"][j]:a["AT.row_ptr"][j + 1]]
        assert np.all(np.diff(seg) > 0)
    # vectors
    assert np.array_equal(a["sign"], sign)
    assert np.array_equal(a["b_int"], sign * lp["b"][a["row_perm"]])
    assert np.array_equal(a["ge"], (lp["sense"][a["row_perm"]] != EQ).astype(np.int8))
    assert np.array_equal(a["c"], lp["c"][a["col_perm"]])
    assert np.array_equal(a["l"], lp["lb"][a["col_perm"]]) and np.array_equal(a["u"], lp["ub"][a["col_perm"]])
    assert a["norms"][0] == pytest.approx(np.linalg.norm(lp["b"]), rel=1e-14)
    assert a["norms"][1] == pytest.approx(np.linalg.norm(lp["c"]), rel=1e-14)
    # every row class is present and laid out by its definition
    cta, long_ = _check_csr_segments("A", a)
    assert cta == 1 and long_ == 7
    cta_t, long_t = _check_csr_segments("AT", a)
    assert cta_t == 0 and long_t == 1  # column 0 of A is the only A' row above the SELL limit


def test_defaults_without_bounds_or_senses(dump_exe, tmp_path):
    lp = _layout_lp(1)
    lp["lb"] = lp["ub"] = lp["sense"] = None
    rc, a = _run(dump_exe, tmp_path, lp)
    assert rc == 0
    assert np.all(a["l"] == 0.0) and np.all(np.isposinf(a["u"]))
    assert np.all(a["sign"] == 1.0) and np.all(a["ge"] == 0)


def _small():
    return dict(m=2, n=3, row_ptr=np.array([0, 2, 3]), col_idx=np.array([0, 2, 1], dtype=np.int32),
                val=np.array([1.0, -2.0, 3.0]), b=np.array([1.0, 2.0]), c=np.array([1.0, 0.0, -1.0]),
                lb=np.zeros(3), ub=np.full(3, 5.0), sense=np.array([EQ, GE], dtype=np.int8))


@pytest.mark.parametrize("edit, code", [
    (lambda lp: lp.__setitem__("row_ptr", np.array([1, 2, 3])), -2),               # row_ptr[0] != 0
    (lambda lp: lp.__setitem__("row_ptr", np.array([0, 3, 2])) or lp.__setitem__("nnz", 2), -2),  # decreasing
    (lambda lp: lp["col_idx"].__setitem__(1, 3), -2),                              # column out of range
    (lambda lp: lp["val"].__setitem__(0, np.nan), -3),                             # non-finite value
    (lambda lp: lp["b"].__setitem__(1, np.inf), -3),                               # non-finite b
    (lambda lp: lp["lb"].__setitem__(2, np.inf), -3),                              # l = +inf
    (lambda lp: lp["lb"].__setitem__(0, 6.0), -4),                                 # l > u
    (lambda lp: lp["sense"].__setitem__(0, ord("x")), -1),                         # bad sense
])
def test_invalid_inputs_get_their_error_codes(dump_exe, tmp_path, edit, code):
    lp = _small()
    rc, _ = _run(dump_exe, tmp_path, lp)
    assert rc == 0
    edit(lp)
    rc, _ = _run(dump_exe, tmp_path, lp)
    assert rc == code


def _chunk_constants():
    src = open(os.path.join(CSRC, "host_prep.h")).read()
    def get(name):  # an integer literal or a product of two
        expr = re.search(rf"constexpr int {name} = ([0-9 *]+);", src).group(1)
        out = 1
        for f in expr.split("*"):
            out *= int(f)
        return out
    return dict(threads=get("kChunkThreads"), maxu=get("kChunkMaxUnits"), long_len=get("kChunkLongLen"),
                bytes=get("kChunkBytes"))


def test_chunk_plan_matches_its_definition(dump_exe, tmp_path):
    # the chunked primal pass's plan of A' with a small chunk (many chunks):
    # every entry of A' sits in exactly one slot of its row's unit and its
    # chunk, at its index within the chunk; padding slots are marked; every
    # unit is on exactly one warp, at most kChunkMaxUnits per warp; the grid
    # is a multiple of the SM count
    KC = _chunk_constants()
    lp = _layout_lp(3)
    chunk, sms = 37, 3
    rc, a = _run(dump_exe, tmp_path, lp, chunk, sms)
    assert rc == 0
    n, m = lp["n"], lp["m"]
    C, nch, blocks, nunits = (int(v) for v in a["ch.hdr"])
    assert C == chunk and nch == -(-m // chunk) and blocks % sms == 0
    rp, col = a["AT.row_ptr"], a["AT.col"]
    units = a["ch.units"].reshape(-1, 3)
    assert units.shape[0] == nunits
    # units cover the rows in order: long rows one each, then slices of 32
    row = 0
    for row0, nrows, is_long in units:
        assert row0 == row
        ln = rp[row0 + 1] - rp[row0]
        if is_long:
            assert nrows == 1 and ln > KC["long_len"]
        else:
            assert 1 <= nrows <= 32 and all(rp[r + 1] - rp[r] <= KC["long_len"] for r in range(row0, row0 + nrows))
        row += nrows
    assert row == n
    smap, sidx = a["ch.slot_map"], a["ch.slot_idx"]
    off = a["ch.uc_off"].reshape(nunits, nch)
    cnt = a["ch.uc_cnt"].reshape(nunits, nch)
    seen = np.zeros(len(col), dtype=np.int64)
    for u, (row0, nrows, is_long) in enumerate(units):
        for c in range(nch):
            o, w = off[u, c], cnt[u, c]
            if is_long:
                e_in = [e for e in range(rp[row0], rp[row0 + 1]) if col[e] // chunk == c]
                assert w == len(e_in) and list(smap[o:o + w]) == e_in
                slots = range(o, o + w)
            else:
                widths = [sum(1 for e in range(rp[r], rp[r + 1]) if col[e] // chunk == c)
                          for r in range(row0, row0 + nrows)]
                assert w == max(widths)
                slots = range(o, o + 32 * w)
                for t in range(32):
                    es = [smap[o + 32 * j + t] for j in range(w)]
                    if t < nrows:
                        want = [e for e in range(rp[row0 + t], rp[row0 + t + 1]) if col[e] // chunk == c]
                        assert es[:len(want)] == want and all(x == -1 for x in es[len(want):])
                    else:
                        assert all(x == -1 for x in es)
            for sl in slots:
                e = smap[sl]
                if e < 0:
                    assert sidx[sl] == 0xFFFF
                else:
                    assert sidx[sl] == col[e] - c * chunk
                    seen[e] += 1
    assert np.all(seen == 1)
    wu = a["ch.warp_units"].reshape(blocks * KC["threads"] // 32, KC["maxu"])
    listed = wu[wu >= 0]
    assert sorted(listed.tolist()) == list(range(nunits))


def test_column_order_is_chunk_aware(dump_exe, tmp_path):
    # with more rows than one FP64 chunk, columns of equal length are ordered
    # by their entry counts in the first three chunks of the (internal) rows
    rng = np.random.default_rng(7)
    KC = _chunk_constants()
    c64 = KC["bytes"] // 8
    m, n = c64 * 3 + 500, 400
    counts = rng.integers(1, 6, size=n)
    rows = np.concatenate([rng.choice(m, size=k, replace=False) for k in counts])
    cols = np.repeat(np.arange(n), counts)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=rp[1:])
    lp = dict(m=m, n=n, row_ptr=rp, col_idx=cols.astype(np.int32), val=np.ones(len(cols)), b=np.zeros(m),
              c=np.ones(n), lb=None, ub=None, sense=None)
    rc, a = _run(dump_exe, tmp_path, lp)
    assert rc == 0
    rlen = np.diff(rp)
    row_inv = a["row_inv"]
    q = np.zeros((n, 3), dtype=np.int64)
    for r, cc in zip(rows, cols):
        k = row_inv[r] // c64
        if k < 3:
            q[cc, k] += 1
    want = np.lexsort((np.arange(n), -q[:, 2], -q[:, 1], -q[:, 0], -counts))
    assert np.array_equal(a["col_perm"], want)
    assert np.array_equal(a["row_perm"], np.argsort(-rlen, kind="stable"))


def test_large_layout_matches_its_definition(dump_exe, tmp_path):
    # an LP large enough that the layout is built on several host threads (one
    # per 64k entries) and that rows reach the second staged chunk: the same
    # definition, checked with sparse arithmetic
    import scipy.sparse as sp
    import lpgen
    lp = lpgen.power_law_lp(30000, 60000, 2000, 7, kmax=3000)
    rc, a = _run(dump_exe, tmp_path, lp)
    assert rc == 0
    m, n = lp["m"], lp["n"]
    rp = np.asarray(lp["row_ptr"])
    col = np.asarray(lp["col_idx"])
    val = np.asarray(lp["val"])
    nnz = int(rp[-1])
    assert nnz > 4 * 65536
    rlen = np.diff(rp)
    clen = np.bincount(col, minlength=n)
    assert np.array_equal(a["row_perm"], np.argsort(-rlen, kind="stable"))
    row_inv = a["row_inv"]
    assert np.array_equal(row_inv[a["row_perm"]], np.arange(m))
    # columns: decreasing length, then decreasing counts in the row chunks
    # [0, C), [C, 2C), [2C, 3C) of the internal row numbering, stable
    C = int(re.search(r"kChunkBytes = (\d+) \* 1024", open(os.path.join(CSRC, "host_prep.h")).read()).group(1)) * 1024 // 8
    chunk_of_entry = row_inv[np.repeat(np.arange(m), rlen)] // C
    q = np.zeros((n, 3), dtype=np.int64)
    for k in range(3):
        q[:, k] = np.bincount(col[chunk_of_entry == k], minlength=n)
    assert q[:, 1].sum() > 0  # the second chunk is populated
    want = np.lexsort((np.arange(n), -q[:, 2], -q[:, 1], -q[:, 0], -clen))
    assert np.array_equal(a["col_perm"], want)
    col_inv = a["col_inv"]
    # internal A: permuted rows, sign-flipped '<' rows, entries in the user's order
    sign = np.where(lp["sense"][a["row_perm"]] == LE, -1.0, 1.0)
    order = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in a["row_perm"]])
    assert np.array_equal(a["A.row_ptr"], np.concatenate([[0], np.cumsum(rlen[a["row_perm"]])]))
    assert np.array_equal(a["A.col"], col_inv[col[order]])
    assert np.array_equal(a["A.val"], np.repeat(sign, rlen[a["row_perm"]]) * val[order])
    # A': the transpose, each row in increasing internal row order
    A = sp.csr_matrix((a["A.val"], a["A.col"], a["A.row_ptr"]), shape=(m, n))
    T = A.T.tocsr()
    T.sort_indices()
    assert np.array_equal(a["AT.row_ptr"], T.indptr)
    assert np.array_equal(a["AT.col"], T.indices)
    assert np.array_equal(a["AT.val"], T.data)
    _check_csr_segments("A", a)
    _check_csr_segments("AT", a)
