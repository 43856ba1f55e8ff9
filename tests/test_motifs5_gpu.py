"""Connected induced 5-vertex motif counts on the GPU (harp_count5) against the 5-vertex oracle,
bit-exact: each class's own graph, closed forms (cliques, stars, cycles, paths, complete bipartite
graphs), random graphs against the brute force over every 5-subset, and BA / ER / RGG graphs against
the oracle's ESU."""
import itertools
import os
import sys

import numpy as np
import pytest

import graphgen
from oracle import motifs5 as M5

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import complete, cycle, edges_of, kbip, path, star  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def harp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_12074_gb300 import _build, harp as H
    _build.build()
    H.lib()
    return H


def gpu5(H, n, src, dst):
    g = H.harp_build_csr(n, torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda())
    try:
        return H.harp_count5(g)
    finally:
        g.close()


def test_each_class_graph_alone(harp):
    for c in range(21):
        s, d = edges_of(M5.class_edges(c))
        want = np.zeros(21, np.uint64)
        want[c] = 1
        assert gpu5(harp, 5, s, d).tolist() == want.tolist(), c


FAMILIES = [("K7", 7, complete(7)), ("K12", 12, complete(12)), ("K1,9", 10, star(9)), ("C9", 9, cycle(9)),
            ("C30", 30, cycle(30)), ("P12", 12, path(12)), ("K3,5", 8, kbip(3, 5)), ("K6,7", 13, kbip(6, 7))]


@pytest.mark.parametrize("name,n,e", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_closed_forms(harp, name, n, e):
    s, d = e
    assert gpu5(harp, n, s, d).tolist() == M5.count5_brute(n, s, d).tolist()


def test_random_graphs_against_brute_force(harp):
    rng = np.random.default_rng(55)
    for trial in range(25):
        n = int(rng.integers(5, 16))
        p = float(rng.uniform(0.1, 0.8))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        s, d = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        assert gpu5(harp, n, s, d).tolist() == M5.count5_brute(n, s, d).tolist(), (trial, n, p)


@pytest.mark.parametrize("make", [lambda: graphgen.ba(250, 2, 2), lambda: graphgen.er(250, 6, 3),
                                  lambda: graphgen.rgg(300, 8, 4)], ids=["ba250", "er250", "rgg300"])
def test_generated_graphs_against_esu(harp, make):
    g = make()
    assert gpu5(harp, g.n, g.src, g.dst).tolist() == M5.count5_esu(g.n, g.src, g.dst).tolist()


def test_fewer_than_five_vertices_or_edges(harp):
    s, d = edges_of([(0, 1), (1, 2), (2, 3)])
    assert gpu5(harp, 4, s, d).tolist() == [0] * 21
    assert gpu5(harp, 9, s, d).tolist() == [0] * 21
