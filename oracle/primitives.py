"""Plain definitions of the HISA building blocks (Section 4), for kernel-level
parity tests.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Each function is the
definition written out with numpy primitives as steps; nothing is blocked,
fused or reordered.  Tuples of a k-ary relation are rows of an (n, k) uint32
array (the data array of Section 4.1).
"""
from __future__ import annotations

import numpy as np


def _rows(a) -> np.ndarray:
    """View ``a`` as an (n, k) uint32 array of tuples (k = 2 when ``a`` is empty and flat)."""
    a = np.asarray(a, dtype=np.uint32)
    if a.ndim == 2:
        return a
    return a.reshape(0, 2) if a.size == 0 else a.reshape(len(a), -1)


def reorder_columns(rows: np.ndarray, join_cols) -> np.ndarray:
    """Algorithm 1, first loop: every tuple rewritten as join columns ++ the
    remaining columns (in their original order)."""
    rows = _rows(rows)
    rest = [c for c in range(rows.shape[1]) if c not in join_cols]
    return rows[:, list(join_cols) + rest]


def sorted_index_array(rows: np.ndarray, join_cols) -> np.ndarray:
    """Algorithm 1 / Section 4.2: positions of the tuples in lexicographic order of
    the reordered tuples, built as one stable sort per column from the rightmost
    (least significant) column to the leftmost."""
    r = reorder_columns(rows, join_cols)
    idx = np.arange(len(r))
    for c in reversed(range(r.shape[1])):
        idx = idx[np.argsort(r[idx, c], kind="stable")]
    return idx


def sort_unique(rows: np.ndarray) -> np.ndarray:
    """Section 4.2 "Deduplication": the tuples sorted lexicographically, each
    distinct tuple kept once (adjacent duplicates removed after the sort)."""
    rows = _rows(rows)
    if len(rows) == 0:
        return rows
    return np.unique(rows, axis=0)


def run_index(sorted_rows: np.ndarray, nkey: int):
    """Section 4.3: for every distinct value of the first ``nkey`` columns of a
    sorted relation, the smallest position holding it and the length of its run.
    Returns (keys (r, nkey), begin (r,), length (r,))."""
    s = _rows(sorted_rows)
    if len(s) == 0:
        return s[:, :nkey], np.zeros(0, np.int64), np.zeros(0, np.int64)
    keys, begin, length = np.unique(s[:, :nkey], axis=0, return_index=True, return_counts=True)
    return keys, begin.astype(np.int64), length.astype(np.int64)


def set_difference(new_rows: np.ndarray, full_rows: np.ndarray) -> np.ndarray:
    """Section 5.1 "Populating delta": the distinct tuples of new that are not in
    full, in lexicographic order."""
    new_rows = sort_unique(new_rows)
    full = {tuple(r) for r in _rows(full_rows).tolist()}
    keep = [i for i, r in enumerate(new_rows.tolist()) if tuple(r) not in full]
    return new_rows[keep]


def merge(full_rows: np.ndarray, delta_rows: np.ndarray) -> np.ndarray:
    """Section 4.2 "Merge operation": the sorted union of two sorted relations."""
    both = np.concatenate([_rows(full_rows), _rows(delta_rows)])
    return sort_unique(both)


def join(outer: np.ndarray, outer_cols, inner: np.ndarray, inner_cols, project):
    """Algorithm 3: every pair (outer tuple, inner tuple) whose join columns are
    equal yields one result tuple; ``project`` lists the result columns as
    ("o", c) or ("i", c).  Returned as a multiset in outer-major order."""
    outer = _rows(outer)
    inner = _rows(inner)
    out = []
    for o in outer.tolist():
        for i in inner.tolist():
            if all(o[a] == i[b] for a, b in zip(outer_cols, inner_cols)):
                out.append([o[c] if side == "o" else i[c] for side, c in project])
    return np.array(out, dtype=np.uint32).reshape(len(out), len(project))


# ---- the same definitions on packed codes (c0 << b) | c1 ------------------------------

def decode_codes(codes, b: int) -> np.ndarray:
    """Packed codes -> (n, 2) tuples."""
    c = np.asarray(codes, dtype=np.uint64)
    mask = np.uint64((1 << b) - 1)
    return np.stack([(c >> np.uint64(b)) & mask, c & mask], axis=1).astype(np.uint32)


def encode_rows(rows, b: int, dtype=np.uint64) -> np.ndarray:
    r = _rows(rows).astype(np.uint64)
    return ((r[:, 0] << np.uint64(b)) | r[:, 1]).astype(dtype)


def sort_codes(codes) -> np.ndarray:
    """The sorted data array: codes in ascending order (order of tuples)."""
    return np.sort(np.asarray(codes), kind="stable")


def sort_unique_codes(codes) -> np.ndarray:
    return np.unique(np.asarray(codes))


def difference_merge_codes(full, fresh):
    """(delta, full U delta) on codes: Section 5.1 populate delta, then merge."""
    full = np.asarray(full)
    fresh = np.asarray(fresh)
    delta = np.setdiff1d(np.unique(fresh), full, assume_unique=True)
    return delta, np.union1d(full, delta)


def join_codes(outer, inner, b: int, outer_col: int, proj0: int, proj1: int, neq=None, dtype=np.uint64):
    """Algorithm 3 on codes: the inner relation joins on its column 0; result
    sources 0 = outer c0, 1 = outer c1, 2 = inner c0 (the key), 3 = inner c1;
    ``neq`` = (a, b) keeps results with source a != source b."""
    o = decode_codes(outer, b).tolist()
    groups = {}                       # inner tuples by join value, in inner order
    for k, x in decode_codes(np.sort(np.asarray(inner)), b).tolist():
        groups.setdefault(k, []).append(x)
    out = []
    for t in o:
        k = t[outer_col]
        for x in groups.get(k, ()):
            src = (t[0], t[1], k, x)
            if neq is not None and src[neq[0]] == src[neq[1]]:
                continue
            out.append((src[proj0], src[proj1]))
    return encode_rows(np.array(out, np.uint32).reshape(len(out), 2), b, dtype)
