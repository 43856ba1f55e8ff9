"""Closed-form graph families shared by the oracle pins and the GPU parity tests.

Each entry: (name, n, (src, dst), expected counts) with the counts derived from the definition of an
induced occurrence (Section II); order [star3, path4, paw, cycle4, diamond, clique4].
"""
import itertools
import math

import numpy as np

C = math.comb


def edges_of(pairs):
    pairs = list(pairs)
    if not pairs:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.array([a for a, b in pairs], np.int32), np.array([b for a, b in pairs], np.int32)


def complete(n):
    return edges_of(itertools.combinations(range(n), 2))


def star(k):
    return edges_of((0, i) for i in range(1, k + 1))


def cycle(n):
    return edges_of((i, (i + 1) % n) for i in range(n))


def path(n):
    return edges_of((i, i + 1) for i in range(n - 1))


def kbip(a, b):
    return edges_of((i, a + j) for i in range(a) for j in range(b))


def wheel(n):
    rim = [(i, (i + 1) % n) for i in range(n)]
    return edges_of(rim + [(n, i) for i in range(n)])


def cocktail(k):
    return edges_of((i, j) for i in range(2 * k) for j in range(i + 1, 2 * k) if j != i + k)


def closed_forms(scale=1):
    """Closed forms; scale > 1 adds large members that exercise every GPU execution mode."""
    out = []
    for n in (4, 5, 6, 9, 12):
        out.append((f"K{n}", n, complete(n), [0, 0, 0, 0, 0, C(n, 4)]))
    for k in (3, 4, 7, 11):
        out.append((f"K1,{k}", k + 1, star(k), [C(k, 3), 0, 0, 0, 0, 0]))
    out.append(("C4", 4, cycle(4), [0, 0, 0, 1, 0, 0]))
    for n in (5, 6, 9, 17):
        out.append((f"C{n}", n, cycle(n), [0, n, 0, 0, 0, 0]))
    for n in (4, 5, 10, 23):
        out.append((f"P{n}", n, path(n), [0, n - 3, 0, 0, 0, 0]))
    for a, b in ((2, 2), (2, 5), (3, 4), (5, 6)):
        out.append((f"K{a},{b}", a + b, kbip(a, b), [a * C(b, 3) + b * C(a, 3), 0, 0, C(a, 2) * C(b, 2), 0, 0]))
    for n in (5, 6, 8, 13):
        out.append((f"W{n}", n + 1, wheel(n), [n * C(n - 3, 3) // (n - 3), n, n * (n - 4), 0, n, 0]))
    for k in (2, 3, 4, 6):
        out.append((f"CP{k}", 2 * k, cocktail(k), [0, 0, 0, C(k, 2), 4 * k * C(k - 1, 2), 16 * C(k, 4)]))
    if scale > 1:
        for n in (40, 300, 700, 1100):   # warp, CTA (256 / 512 / 1024) and fallback triangle modes
            out.append((f"K{n}", n, complete(n), [0, 0, 0, 0, 0, C(n, 4)]))
        out.append(("K1,5000", 5001, star(5000), [C(5000, 3), 0, 0, 0, 0, 0]))   # hub row sort
        n = 5000
        out.append((f"W{n}", n + 1, wheel(n), [n * C(n - 3, 3) // (n - 3), n, n * (n - 4), 0, n, 0]))
        for a, b in ((40, 60), (300, 500)):   # dense 4-cycles: CTA and windowed wedge modes
            out.append((f"K{a},{b}", a + b, kbip(a, b), [a * C(b, 3) + b * C(a, 3), 0, 0, C(a, 2) * C(b, 2), 0, 0]))
        for k in (40, 600):
            out.append((f"CP{k}", 2 * k, cocktail(k), [0, 0, 0, C(k, 2), 4 * k * C(k - 1, 2), 16 * C(k, 4)]))
        out.append(("C100000", 100000, cycle(100000), [0, 100000, 0, 0, 0, 0]))
    return out
