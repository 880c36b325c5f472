"""Helpers for the GPU tests: library build/load and the FSO packing of hs.h (layout only)."""
import json
import os

import numpy as np

from paper_2410_11596_gb300 import _lib as L, build

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ensure_library():
    if not os.path.exists(L.LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(L.LIB_PATH) for s in build.sources()):
        build.build()
    return L.load()


def fso_order(sects, k):
    """Fused sector order of k legs with sectors sects[j] = (n_even, n_odd): list per parity of
    (tuple, local index arrays) giving, for each fused position, the per-leg basis indices."""
    out = {0: [], 1: []}
    for t in range(1 << k):
        bits = [(t >> (k - 1 - j)) & 1 for j in range(k)]
        P = sum(bits) & 1
        ranges = []
        for j, b in enumerate(bits):
            ne, no = sects[j]
            ranges.append(np.arange(ne) if b == 0 else ne + np.arange(no))
        grid = np.meshgrid(*ranges, indexing="ij")
        out[P].append(np.stack([g.reshape(-1) for g in grid], axis=1) if grid[0].size else
                      np.zeros((0, k), dtype=int))
    return {P: (np.concatenate(v, axis=0) if v else np.zeros((0, k), dtype=int)) for P, v in out.items()}


def fso_pack(t, row_sects, col_sects):
    """Pack a dense tensor (legs = row legs then col legs, each in sector order) into FSO blocks."""
    kr, kc = len(row_sects), len(col_sects)
    R, Cc = fso_order(row_sects, kr), fso_order(col_sects, kc)
    blocks = []
    for P in (0, 1):
        r, c = R[P], Cc[P]
        if len(r) == 0 or len(c) == 0:
            continue
        # (rows x cols) block by broadcast advanced indexing on every leg
        sub = t[tuple(r[:, j][:, None] for j in range(kr)) + tuple(c[:, j][None, :] for j in range(kc))]
        blocks.append(sub.reshape(-1))
    return np.concatenate(blocks) if blocks else np.zeros(0)


def golden(k):
    with open(os.path.join(GOLDEN, f"ctmrg_w{k}.json")) as f:
        return json.load(f)


def graded_pack(t, row_sects, col_sects):
    """Dense graded matrix of hs.h (complex tensors): all rows in FSO order (both parities),
    all columns likewise; entries of odd total parity give their imaginary part, even ones
    their real part."""
    kr, kc = len(row_sects), len(col_sects)
    R, Cc = fso_order(row_sects, kr), fso_order(col_sects, kc)
    r = np.concatenate([R[0], R[1]], axis=0)
    c = np.concatenate([Cc[0], Cc[1]], axis=0)
    sub = t[tuple(r[:, j][:, None] for j in range(kr)) + tuple(c[:, j][None, :] for j in range(kc))]
    nr0, nc0 = len(R[0]), len(Cc[0])
    pr = (np.arange(len(r)) >= nr0)[:, None]
    pc = (np.arange(len(c)) >= nc0)[None, :]
    return np.where(pr != pc, np.imag(sub), np.real(sub))
