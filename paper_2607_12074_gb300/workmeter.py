"""Host work meter: exact algorithmic work and bytes of each counting kernel for a given graph.

"Algorithmic bytes" are the bytes an ideal implementation of each step must move between the SMs
and memory (every needed list element, offset and statistic read or written once), independent of
how many of them the L2 serves.  They are the numerators of the roofline figures (per unit below).
This module is plain numpy on the host and is not on the counting path (bench.py uses it to turn
kernel times into bandwidth).

Per unit (int32 ids and counters = 4 B, int64 offsets = 8 B):
  orientation   read offsets + cols + perm gather, write relabelled cols and offsets, out-CSR copy:
                24 (n+1) + 12 * 2m + 8 m
  triangle      per anchor u: its list N+(u) (4 d+), per row v in N+(u): offsets (16) and the probed
                part of N+(v) up to max N+(u) (4 each); per triangle: 3 t_e updates (8 each, RMW);
                per out-arc: its own t_e update (8)
  wedge (C4)    per root u: N-(u) read once (4 d-) + the row bounds of each w (16 d-); per wedge
                element x of degree >= 2: 4.  The windowed kernel re-reads N-(u) and the row
                bounds once per further x-window; those bytes are this design's overhead and are
                reported apart ("overhead_bytes"), not counted as algorithmic
  reduction     t_e read: 4 m
"""
from __future__ import annotations

import numpy as np

WARP_MAX_TRI = 32
CTA_SMALL_MAX = 256
CTA_MAX = 1024
WIN_WORDS = {1: 51200, 2: 25600, 3: 16384, 4: 12288}  # counter words per wedge window by resident blocks per SM


def window_words(c4_window_bytes, n=0):
    """Counter words of the wedge window the kernel picks for plan.c4_window_bytes (the largest that
    fits; 0 = by graph: 200 KiB above 2^22 vertices, else 100 KiB)."""
    if c4_window_bytes == 0:
        c4_window_bytes = 4 * WIN_WORDS[1] if n > (1 << 22) else 4 * WIN_WORDS[2]
    for minb in (1, 2, 3):
        if c4_window_bytes >= 4 * WIN_WORDS[minb]:
            return WIN_WORDS[minb]
    return WIN_WORDS[4]


def _simple_edges(n, src, dst):
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    s, d = s[keep], d[keep]
    lo = np.minimum(s, d)
    hi = np.maximum(s, d)
    key = np.unique(lo * n + hi)
    return key // n, key % n


def rank_space(n, src, dst):
    """Degrees and the rank-ordered sorted CSR used by the kernels (rank = (degree, id))."""
    lo, hi = _simple_edges(n, src, dst)
    deg0 = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    order = np.lexsort((np.arange(n), deg0))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    a, b = rank[lo], rank[hi]
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    o = np.lexsort((cols, rows))
    rows, cols = rows[o], cols[o]
    deg = deg0[order]
    indptr = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=indptr[1:])
    pos = np.arange(cols.size, dtype=np.int64) - indptr[rows]
    split = np.bincount(rows[cols < rows], minlength=n)   # |N-(u)|
    return {"n": n, "m": int(lo.size), "deg": deg, "indptr": indptr, "rows": rows, "cols": cols, "pos": pos,
            "split": split, "dplus": deg - split}


def _merged_windows(bounds, widths, mask, u, words):
    """Grid windows that intersect [n1, u) per root u when band b merges into band b + 1 (and takes
    its wider counters) for every bit b set in mask; bounds = band starts followed by n."""
    total = np.zeros(len(u), np.int64)
    gs = bounds[0]
    for b, width in enumerate(widths):
        if b + 1 < len(widths) and (mask >> b) & 1:
            continue
        e = np.minimum(bounds[b + 1], u)
        span = words * (32 // width)
        total += np.where(e > gs, (e - gs + span - 1) // span, 0)
        gs = bounds[b + 1]
    return total


def meter(n, src, dst, c4_warp_max=512, c4_window_bytes=0, c4_mid_max=2048):
    """Per-kernel work and algorithmic bytes (dict of dicts) under the given wedge plan fields."""
    G = rank_space(n, src, dst)
    m = G["m"]
    deg, indptr, rows, cols, pos = G["deg"], G["indptr"], G["rows"], G["cols"], G["pos"]
    split, dplus = G["split"], G["dplus"]
    out = {"n": n, "m": m}
    out["orient"] = {"bytes": 24 * (n + 1) + 12 * 2 * m + 8 * m}

    # ---- triangle anchors: out-arcs (u -> v), u < v
    up = cols > rows
    au, av = rows[up], cols[up]                      # oriented arcs in row order
    offp = np.zeros(n + 1, np.int64)
    np.cumsum(dplus, out=offp[1:])
    last = np.full(n, -1, np.int64)
    has = dplus > 0
    last[has] = cols[indptr[1:][has] - 1]            # max of N+(u) = last element of row u
    # probed part of N+(v) for each out-arc (u, v): elements y of N+(v) with y <= last[u]
    keys = au * n + av                               # sorted: out-arcs grouped by source, ascending
    q = av * n + last[au]
    probed = np.searchsorted(keys, q, side="right") - offp[av]
    probed = np.maximum(probed, 0)
    cls = np.where(dplus < 2, -1, np.where(dplus <= WARP_MAX_TRI, 0, np.where(dplus <= CTA_SMALL_MAX, 1,
                   np.where(dplus <= CTA_MAX, 2, 3))))
    arc_cls = cls[au]
    # rows i < d-1 only: the last element of N+(u) starts no row
    is_last = np.zeros(au.size, bool)
    ends = offp[1:][has] - 1
    is_last[ends] = True
    row_bytes = np.where(is_last, 0, 16 + 4 * probed)
    tri_units = {}
    for c, name in ((0, "tri_warp"), (1, "tri_cta_small"), (2, "tri_cta_large"), (3, "tri_fallback")):
        sel = arc_cls == c
        tri_units[name] = {"anchors": int((cls == c).sum()), "probes": int(probed[sel & ~is_last].sum()),
                           "bytes": int(row_bytes[sel].sum() + 4 * sel.sum() + 8 * sel.sum())}
    out.update(tri_units)
    out["tri_probes_total"] = int(probed[~is_last].sum())

    # ---- wedge anchors: root u, w in N-(u) (arcs (u -> w), w < u).  Leaves (degree 1) never close a
    # 4-cycle, so a segment runs from fpos[w] (first neighbour of degree >= 2) to pos_w(u).
    down = cols < rows
    ru, rw = rows[down], cols[down]
    rev = np.searchsorted(rows * n + cols, rw * n + ru)
    n1 = int(np.searchsorted(deg, 2))                 # first rank of degree >= 2
    band_widths = (3, 4, 5, 6, 8, 16, 32)              # x bands by d(x): d < 2^width
    band_starts = [n1] + [max(int(np.searchsorted(deg, 1 << w)), n1) for w in band_widths[:-1]]
    fpos = np.bincount(rows[cols < n1], minlength=n)  # neighbours of degree <= 1 lead every row
    seg = np.maximum(pos[rev] - fpos[rw], 0)
    W = np.bincount(ru, weights=seg, minlength=n).astype(np.int64)
    dm = split
    # warp-local hash mode for W <= c4_warp_max (1024 slots), the middle tier for W <= c4_mid_max (4096
    # slots), windowed counters above
    wmax = min(c4_warp_max, 512)
    mmax = max(min(c4_mid_max, 2048), wmax)
    tier = np.where((dm < 2) | (W == 0), -1, np.where(W <= wmax, 0, np.where(W <= mmax, 1, 2)))
    words = window_words(c4_window_bytes, n)
    bounds = band_starts + [n]
    # narrow bands may merge into the next wider one: the mask with the fewest degree-weighted windows
    # over 64 roots spread evenly over the ranks of degree >= 64 (lowest mask on a tie)
    s0 = int(np.searchsorted(deg, 64))
    s0 = 0 if s0 >= n else s0
    samples = s0 + ((n - s0) * (2 * np.arange(64, dtype=np.int64) + 1)) // 128
    weights = deg[samples].astype(np.float64) if n > s0 else np.zeros(0)
    costs = [float((weights * _merged_windows(bounds, band_widths, mask, samples, words)).sum())
             for mask in range(1 << (len(band_widths) - 1))]
    best = int(np.argmin(costs))
    nwin = _merged_windows(bounds, band_widths, best, np.arange(n, dtype=np.int64), words)
    nwin = np.where(tier == 2, nwin, 1)
    for t, name in ((0, "c4_small"), (1, "c4_mid"), (2, "c4_window")):
        sel = tier == t
        passes = nwin[sel]
        out[name] = {"roots": int(sel.sum()), "wedges": int(W[sel].sum()),
                     "items": int(passes.sum()),
                     "bytes": int((20 * dm[sel]).sum() + 4 * W[sel].sum()),
                     "overhead_bytes": int((20 * dm[sel] * (passes - 1)).sum())}
    out["c4_wedges_total"] = int(W.sum())
    out["reduce"] = {"bytes": 4 * m}
    return out
