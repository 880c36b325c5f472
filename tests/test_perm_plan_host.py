"""Host check of the permute plans (the block bookkeeping behind every leg permutation): the boxes
that make_perm_plan (Z2 block matrices) and make_graded_perm_plan (graded matrices of complex
tensors) build must send each element of the input's storage to the position the layout gives it
in the output (tests/perm_plan_check.cu prints a plan's map; the expected map is computed here
from the layout's definition).

The layouts. A fused group of legs enumerates its parity tuples grouped by total parity, even
group first, tuples in lexicographic order, local indices row-major inside a tuple. Z2 block
matrix (Sec. II.B: a Z2-symmetric tensor is block diagonal in the parity of its fused legs):
block p holds the rows of parity p times the columns of parity p, row-major, rows padded to `pad`
elements, block 0 first. Graded matrix (Sec. II.C): all rows times all columns, each in that
order, as one dense row-major matrix with rows padded to `pad` elements."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2410_11596_gb300 import _lib as L, build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2410_11596_gb300", "csrc")


def _group_index(sects, idx):
    """(parity, position in its parity group) of the leg indices idx of one fused group."""
    bits = [int(i >= e) for (e, _), i in zip(sects, idx)]
    loc = [i - b * e for (e, _), i, b in zip(sects, idx, bits)]
    par = sum(bits) % 2
    off = 0
    for t in itertools.product((0, 1), repeat=len(sects)):
        if sum(t) % 2 != par:
            continue
        if list(t) == bits:
            break
        off += int(np.prod([s[b] for s, b in zip(sects, t)]))
    ext = [s[b] for s, b in zip(sects, bits)]
    return par, off + int(np.ravel_multi_index(loc, ext)) if ext else off


def _group_size(sects, par):
    return sum(int(np.prod([s[b] for s, b in zip(sects, t)]))
               for t in itertools.product((0, 1), repeat=len(sects)) if sum(t) % 2 == par)


def _flat(rows, cols, pad, idx):
    """Flat position of the element with leg indices idx in the block storage, or None if its
    total parity is odd (no such block)."""
    pr, ri = _group_index(rows, idx[:len(rows)])
    pc, ci = _group_index(cols, idx[len(rows):])
    if pr != pc:
        return None
    ld = [-(-_group_size(cols, p) // pad) * pad for p in (0, 1)]
    off = 0 if pr == 0 else _group_size(rows, 0) * ld[0]
    return off + ri * ld[pr] + ci


def _elems(rows, cols, pad):
    return sum(_group_size(rows, p) * (-(-_group_size(cols, p) // pad) * pad) for p in (0, 1))


def _graded_ld(cols, pad):
    return -(-(_group_size(cols, 0) + _group_size(cols, 1)) // pad) * pad


def _graded_flat(rows, cols, pad, idx):
    """Flat position of the element with leg indices idx in a graded matrix."""
    pr, ri = _group_index(rows, idx[:len(rows)])
    pc, ci = _group_index(cols, idx[len(rows):])
    r = (_group_size(rows, 0) if pr else 0) + ri
    c = (_group_size(cols, 0) if pc else 0) + ci
    return r * _graded_ld(cols, pad) + c


def _graded_elems(rows, cols, pad):
    return (_group_size(rows, 0) + _group_size(rows, 1)) * _graded_ld(cols, pad)


def _expected(mode, kr, sects, kro, perm, pad):
    rows, cols = sects[:kr], sects[kr:]
    so = [sects[p] for p in perm]
    orows, ocols = so[:kro], so[kro:]
    flat, elems = (_flat, _elems) if mode == 0 else (_graded_flat, _graded_elems)
    m = np.full(elems(rows, cols, 1), -1, dtype=np.int64)
    for idx in itertools.product(*[range(e + o) for e, o in sects]):
        fi = flat(rows, cols, 1, idx)
        if fi is None:
            continue
        m[fi] = flat(orows, ocols, pad, [idx[p] for p in perm])
    return m, elems(orows, ocols, pad)


# (mode, kr, sectors, kr_out, perm, pad_out); mode 0: Z2 block matrices. The permutations of the
# C4v and directional moves ([(a, x) | (y, b)] -> [(a, b) | (y, x)], [(a, b) | (d, r)] ->
# [(a, d) | (b, r)], the transposes, the edge's [(b, x) | a] -> [(x, a) | b], the split operands'
# padded rows); empty odd sectors (D = 1, a boundary with no odd states) and empty even ones;
# three- to six-leg groupings.
CASES = [
    (0, 2, [(3, 2), (2, 1), (2, 1), (3, 2)], 2, [0, 3, 2, 1], 1),
    (0, 2, [(3, 2), (2, 1), (2, 1), (3, 2)], 2, [0, 2, 1, 3], 1),
    (0, 2, [(3, 2), (2, 1), (3, 2), (2, 1)], 2, [2, 3, 0, 1], 1),
    (0, 2, [(3, 2), (2, 1), (3, 2), (2, 1)], 2, [0, 3, 1, 2], 32),
    (0, 1, [(4, 3), (5, 2)], 1, [1, 0], 1),
    (0, 2, [(4, 3), (3, 1), (4, 3)], 2, [1, 2, 0], 1),
    (0, 2, [(4, 3), (3, 1), (4, 3)], 1, [0, 2, 1], 32),
    (0, 2, [(3, 0), (1, 0), (1, 0), (3, 0)], 2, [0, 3, 2, 1], 1),
    (0, 2, [(2, 2), (3, 0), (3, 0), (2, 2)], 2, [0, 2, 1, 3], 32),
    (0, 2, [(0, 3), (2, 1), (2, 1), (0, 3)], 2, [2, 3, 0, 1], 1),
    (0, 1, [(6, 0), (6, 0)], 1, [1, 0], 32),
    (0, 3, [(2, 1), (1, 2), (2, 2), (1, 1), (2, 1)], 2, [4, 0, 3, 1, 2], 1),
    (0, 3, [(2, 1), (1, 1), (2, 1), (1, 2), (1, 1), (2, 1)], 3, [5, 4, 3, 2, 1, 0], 1),
    (0, 2, [(2, 1), (1, 1), (2, 1), (1, 2), (1, 1), (2, 1)], 4, [1, 3, 5, 0, 2, 4], 32),
]


# Graded matrices (mode 1, at most five legs): the complex path's permutations of the corner and
# edge chains, with empty and uneven sectors.
GRADED_CASES = [
    (1, 2, [(3, 2), (2, 1), (2, 1), (3, 2)], 2, [0, 3, 2, 1], 1),
    (1, 2, [(3, 2), (2, 1), (3, 2), (2, 1)], 2, [0, 2, 1, 3], 32),
    (1, 2, [(4, 3), (3, 1), (4, 3)], 2, [1, 2, 0], 1),
    (1, 2, [(4, 3), (3, 1), (4, 3)], 1, [2, 0, 1], 32),
    (1, 1, [(4, 3), (5, 2)], 1, [1, 0], 1),
    (1, 2, [(3, 0), (2, 1), (2, 1), (3, 0)], 2, [2, 3, 0, 1], 1),
    (1, 3, [(2, 1), (1, 2), (2, 2), (1, 1), (2, 1)], 2, [4, 0, 3, 1, 2], 32),
]


def _random_cases(n, seed, mode=0, max_legs=6):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        legs = int(rng.integers(2, max_legs + 1))
        kr = int(rng.integers(1, min(legs - 1, 4) + 1))
        if legs - kr > 4:
            continue
        kro = int(rng.integers(1, min(legs - 1, 4) + 1))
        if legs - kro > 4:
            continue
        sects = [(int(rng.integers(0, 4)), int(rng.integers(0, 3))) for _ in range(legs)]
        if any(e + o == 0 for e, o in sects):
            continue
        out.append((mode, kr, sects, kro, [int(x) for x in rng.permutation(legs)], int(rng.choice([1, 4, 32]))))
    return out


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    if not os.path.exists(L.LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(L.LIB_PATH) for s in build.sources()):
        build.build()
    libdir = os.path.dirname(L.LIB_PATH)
    path = tmp_path_factory.mktemp("perm") / "perm_plan_check"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, os.path.join(HERE, "perm_plan_check.cu"), "-o", str(path),
                    "-L", libdir, "-lhs", "-Xlinker", "-rpath=" + libdir], check=True, capture_output=True)
    return path


def _plan_maps(exe, cases):
    text = "".join(f"{mode} {kr} {len(s) - kr} " + " ".join(f"{e} {o}" for e, o in s) + f" {kro} " +
                   " ".join(map(str, perm)) + f" {pad}\n" for mode, kr, s, kro, perm, pad in cases)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-500:] + out.stderr
    lines = out.stdout.splitlines()
    assert len(lines) == len(cases)
    maps = []
    for line in lines:
        assert line != "unsupported"
        v = np.array(line.split(), dtype=np.int64)
        maps.append((v[2:], int(v[1])))
        assert len(v) - 2 == v[0]
    return maps


@pytest.mark.parametrize("which", ["move_layouts", "random", "graded", "graded_random"])
def test_perm_plan_matches_the_block_layout(exe, which):
    cases = {"move_layouts": CASES, "random": _random_cases(60, 11596), "graded": GRADED_CASES,
             "graded_random": _random_cases(40, 11597, mode=1, max_legs=5)}[which]
    for case, (got, nout) in zip(cases, _plan_maps(exe, cases)):
        want, nout_want = _expected(*case)
        assert nout == nout_want, case
        np.testing.assert_array_equal(got, want, err_msg=str(case))
        # a bijection onto the output's non-padding entries
        assert len(np.unique(got)) == len(got) and (got >= 0).all(), case


def test_expected_map_on_a_hand_example():
    """The layout definition itself on a two-leg matrix small enough to write out: legs (2 even,
    1 odd) x (1 even, 1 odd). Block 0 = rows {e0, e1} x cols {e0}; block 1 = row {o0} x col {o0};
    the transpose sends (r, c) to (c, r)."""
    want, n = _expected(0, 1, [(2, 1), (1, 1)], 1, [1, 0], 1)
    # input storage: [ (e0,e0), (e1,e0) | (o0,o0) ]; output (transposed) storage:
    # block 0 = row e0 x cols {e0, e1}: [(e0,e0), (e0,e1)], block 1 = [(o0,o0)]
    assert n == 3
    assert list(want) == [0, 1, 2]
    want, n = _expected(0, 1, [(2, 1), (1, 1)], 1, [1, 0], 4)
    assert n == 4 + 4       # each block's row padded to 4
    assert list(want) == [0, 1, 4]


def _pack(tensor, rows, cols, pad):
    """Z2 block storage of a tensor whose first len(rows) legs are the rows (odd-total entries
    dropped), by the layout definition."""
    out = np.zeros(_elems(rows, cols, pad))
    for idx in itertools.product(*[range(e + o) for e, o in rows + cols]):
        f = _flat(rows, cols, pad, idx)
        if f is not None:
            out[f] = tensor[idx]
    return out


def _even_random(sects, rng):
    t = rng.standard_normal([e + o for e, o in sects])
    for idx in itertools.product(*[range(e + o) for e, o in sects]):
        if sum(int(i >= e) for (e, _), i in zip(sects, idx)) % 2:
            t[idx] = 0.0
    return t


# (R legs, K legs, N legs, pads of A, B, C): the move's corner and edge products (two-leg groups,
# ragged sectors, an empty odd sector), one-leg groups, three-leg groups, padded operands.
GEMM_CASES = [
    ([(3, 2), (2, 1)], [(2, 1), (3, 2)], [(3, 2), (2, 1)], 1, 1, 1),
    ([(3, 2)], [(3, 2), (2, 1)], [(2, 1), (2, 1)], 32, 32, 1),
    ([(4, 0), (1, 0)], [(1, 0), (4, 0)], [(2, 0)], 1, 4, 1),
    ([(2, 1), (1, 1), (1, 2)], [(2, 2)], [(1, 1), (2, 1)], 4, 1, 32),
    ([(0, 2), (2, 1)], [(1, 2), (2, 0)], [(2, 2)], 1, 1, 4),
]


def test_block_gemm_descriptors_give_the_dense_contraction(exe):
    """make_z2_gemm's problems (sizes, strides, offsets), applied with numpy to the packed operands,
    give the packed dense contraction C[R, N] = sum_K A[R, K] B[N, K]; their flop count is the
    sum over parity blocks of 2 M N K."""
    rng = np.random.default_rng(2410)
    text = "".join(f"2 {len(r)} {len(k)} {len(n)} " + " ".join(f"{e} {o}" for e, o in r + k + n) +
                   f" {pa} {pb} {pc}\n" for r, k, n, pa, pb, pc in GEMM_CASES)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-500:] + out.stderr
    lines = out.stdout.splitlines()
    assert len(lines) == len(GEMM_CASES)
    for (r, k, n, pa, pb, pc), line in zip(GEMM_CASES, lines):
        v = [int(x) for x in line.split()]
        nprob, ea, eb, ec = v[:4]
        assert (ea, eb, ec) == (_elems(r, k, pa), _elems(n, k, pb), _elems(r, n, pc))
        a = _even_random(r + k, rng)
        b = _even_random(n + k, rng)
        A, B = _pack(a, r, k, pa), _pack(b, n, k, pb)
        C = np.zeros(ec)
        flops = 0
        for i in range(nprob):
            M, N, K, lda, ldb, ldc, ao, bo, co = v[4 + 9 * i: 13 + 9 * i]
            Ab = A[ao:ao + M * lda].reshape(M, lda)[:, :K]
            Bb = B[bo:bo + N * ldb].reshape(N, ldb)[:, :K]
            C[co:co + M * ldc].reshape(M, ldc)[:, :N] = Ab @ Bb.T
            flops += 2 * M * N * K
        dense = np.tensordot(a, b, axes=(list(range(len(r), len(r) + len(k))),
                                          list(range(len(n), len(n) + len(k)))))
        np.testing.assert_allclose(C, _pack(dense, r, n, pc), atol=1e-12, err_msg=str((r, k, n)))
        want = sum(2 * _group_size(r, p) * _group_size(n, p) * _group_size(k, p) for p in (0, 1)
                   if _group_size(r, p) and _group_size(n, p))
        assert flops == want


def _block(off, rows, cols, ld):
    """Flat indices of a rows x cols block with row stride ld starting at off."""
    return off + np.arange(rows)[:, None] * ld + np.arange(cols)[None, :]


def _graded_pack(t, rows, cols, pad):
    out = np.zeros(_graded_elems(rows, cols, pad))
    for idx in itertools.product(*[range(e + o) for e, o in rows + cols]):
        out[_graded_flat(rows, cols, pad, idx)] = t[idx]
    return out


def _parity(sects, idx):
    return sum(int(i >= e) for (e, _), i in zip(sects, idx)) % 2


def test_graded_gemm_descriptors_give_the_complex_product(exe):
    """make_graded_gemm's four sub-GEMMs per product, with the diagonal blocks reading the copy of
    B~ whose odd-total entries are negated (stored right after B~), applied with numpy to packed
    graded operands, give the graded form of the complex product: for complex X with
    X[r, c] = i^[p(r) != p(c)] X~[r, c] (X~ real, Sec. II.C), C = A B^T and C~ = C / i^[p(r) != p(k)]."""
    rng = np.random.default_rng(2411)
    text = "".join(f"3 {len(r)} {len(k)} {len(n)} " + " ".join(f"{e} {o}" for e, o in r + k + n) +
                   f" {pa} {pb} {pc}\n" for r, k, n, pa, pb, pc in GEMM_CASES)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-500:] + out.stderr
    for (r, k, n, pa, pb, pc), line in zip(GEMM_CASES, out.stdout.splitlines()):
        v = [int(x) for x in line.split()]
        nprob, ea, eb, ec = v[:4]
        assert (ea, eb, ec) == (_graded_elems(r, k, pa), _graded_elems(n, k, pb), _graded_elems(r, n, pc))
        at = rng.standard_normal([e + o for e, o in r + k])      # A~ over (R, K)
        bt = rng.standard_normal([e + o for e, o in n + k])      # B~ over (N, K): the operand B^T
        A = _graded_pack(at, r, k, pa)
        Bs = _graded_pack(bt, n, k, pb)
        conj = bt.copy()
        for idx in itertools.product(*[range(e + o) for e, o in n + k]):
            if _parity(n, idx[:len(n)]) != _parity(k, idx[len(n):]):
                conj[idx] = -conj[idx]
        B = np.concatenate([Bs, _graded_pack(conj, n, k, pb)])
        C = np.zeros(ec)
        for i in range(nprob):
            M, N, K, lda, ldb, ldc, ao, bo, co = v[4 + 9 * i: 13 + 9 * i]
            C[_block(co, M, N, ldc)] = A[_block(ao, M, K, lda)] @ B[_block(bo, N, K, ldb)].T
        # the complex product, written out
        ac = at.astype(complex)
        for idx in itertools.product(*[range(e + o) for e, o in r + k]):
            if _parity(r, idx[:len(r)]) != _parity(k, idx[len(r):]):
                ac[idx] *= 1j
        bc = bt.astype(complex)
        for idx in itertools.product(*[range(e + o) for e, o in n + k]):
            if _parity(n, idx[:len(n)]) != _parity(k, idx[len(n):]):
                bc[idx] *= 1j
        cc = np.tensordot(ac, bc, axes=(list(range(len(r), len(r) + len(k))), list(range(len(n), len(n) + len(k)))))
        ct = np.empty(cc.shape)
        for idx in itertools.product(*[range(e + o) for e, o in r + n]):
            z = cc[idx] / (1j if _parity(r, idx[:len(r)]) != _parity(n, idx[len(r):]) else 1)
            assert abs(z.imag) <= 1e-12
            ct[idx] = z.real
        np.testing.assert_allclose(C, _graded_pack(ct, r, n, pc), atol=1e-12, err_msg=str((r, k, n)))
