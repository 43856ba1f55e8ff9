"""Per-vertex orbit counts on the GPU (harp_count4_orbits) against the per-vertex oracle, bit-exact.

* every motif graph alone and closed-form families (cliques, stars, cycles, paths, complete
  bipartite graphs, wheels, cocktail parties) against oracle.orbits.orbits4_brute / orbits4_combo;
* random graphs against the brute force over every 4-subset;
* BA, ER, RGG and Chung-Lu graphs (hubs whose wedge work takes the block kernel with dense
  counters) against orbits4_combo;
* on larger graphs (R-MAT 14, 16) every role summed over the vertices equals the GPU's global count
  times the role's vertices in its motif;
* the device-output form equals the host one;
* per-edge orbit counts (harp_count4_edge_orbits) the same way against oracle.edge_orbits.
"""
import os
import sys

import numpy as np
import pytest

import graphgen
from oracle import edge_orbits as EB
from oracle import orbits as OB

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from graph_families import closed_forms, complete, cocktail, edges_of, kbip, star, wheel  # noqa: E402

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


def gpu_orbits(H, n, src, dst):
    g = H.harp_build_csr(n, torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda())
    try:
        return H.harp_count4_orbits(g), H.harp_count4(g)
    finally:
        g.close()


MOTIF_GRAPHS = {
    "star": edges_of([(0, 1), (0, 2), (0, 3)]), "path": edges_of([(0, 1), (1, 2), (2, 3)]),
    "paw": edges_of([(0, 1), (1, 2), (0, 2), (2, 3)]), "cycle": edges_of([(0, 1), (1, 2), (2, 3), (3, 0)]),
    "diamond": edges_of([(0, 1), (1, 2), (2, 0), (0, 3), (1, 3)]), "clique": complete(4),
}


@pytest.mark.parametrize("name", list(MOTIF_GRAPHS))
def test_each_motif_graph_alone(harp, name):
    s, d = MOTIF_GRAPHS[name]
    got, _ = gpu_orbits(harp, 4, s, d)
    assert got.tolist() == OB.orbits4_brute(4, s, d).tolist()


EXTRA = [("K40", 40, complete(40)), ("K1,700", 701, star(700)), ("W600", 601, wheel(600)),
         ("K30,45", 75, kbip(30, 45)), ("CP25", 50, cocktail(25))]
FAMILIES = [(c[0], c[1], c[2]) for c in closed_forms(scale=1)] + EXTRA


@pytest.mark.parametrize("name,n,e", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_closed_form_families(harp, name, n, e):
    s, d = e
    got, _ = gpu_orbits(harp, n, s, d)
    want = OB.orbits4_brute(n, s, d) if n <= 14 else OB.orbits4_combo(n, s, d)
    assert got.tolist() == want.tolist()


def test_random_graphs_against_brute_force(harp):
    rng = np.random.default_rng(77)
    for trial in range(30):
        n = int(rng.integers(5, 22))
        p = float(rng.uniform(0.1, 0.7))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        s, d = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        got, _ = gpu_orbits(harp, n, s, d)
        assert got.tolist() == OB.orbits4_brute(n, s, d).tolist(), (trial, n, p)


@pytest.mark.parametrize("make", [lambda: graphgen.ba(2000, 4, 1), lambda: graphgen.er(1500, 10, 3),
                                  lambda: graphgen.rgg(2000, 12, 4), lambda: graphgen.chung_lu(3000, 2.1, 150, 6, 5)],
                         ids=["ba2000", "er1500", "rgg2000", "chunglu3000"])
def test_generated_graphs_against_the_per_vertex_oracle(harp, make):
    g = make()
    got, _ = gpu_orbits(harp, g.n, g.src, g.dst)
    assert got.tolist() == OB.orbits4_combo(g.n, g.src, g.dst).tolist()


@pytest.mark.parametrize("scale", [14, 16])
def test_role_sums_equal_global_counts(harp, scale):
    g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, seed=3)
    got, counts = gpu_orbits(harp, g.n, g.src, g.dst)
    sums = got.sum(axis=0, dtype=np.uint64)
    for r in range(11):
        assert int(sums[r]) == (int(counts[OB.ORBIT_MOTIF[r]]) * OB.ORBIT_SIZE[r]) % 2**64, OB.ORBITS[r]


def test_device_output_equals_host_output(harp):
    g = graphgen.ba(3000, 5, 9)
    csr = harp.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
    try:
        host = harp.harp_count4_orbits(csr)
        dev = torch.full((g.n * harp.HARP_NORBITS,), -1, dtype=torch.int64, device="cuda")
        harp.harp_count4_orbits(csr, dev)
        torch.cuda.synchronize()
        assert dev.cpu().numpy().view(np.uint64).reshape(g.n, -1).tolist() == host.tolist()
    finally:
        csr.close()



def gpu_edge_orbits(H, n, src, dst):
    g = H.harp_build_csr(n, torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda())
    try:
        return H.harp_count4_edge_orbits(g), H.harp_count4(g)
    finally:
        g.close()


@pytest.mark.parametrize("name", list(MOTIF_GRAPHS))
def test_edge_orbits_each_motif_graph_alone(harp, name):
    s, d = MOTIF_GRAPHS[name]
    got, _ = gpu_edge_orbits(harp, 4, s, d)
    assert got.tolist() == EB.edge_orbits4_brute(4, s, d).tolist()


@pytest.mark.parametrize("name,n,e", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_edge_orbits_closed_form_families(harp, name, n, e):
    s, d = e
    got, _ = gpu_edge_orbits(harp, n, s, d)
    want = EB.edge_orbits4_brute(n, s, d) if n <= 14 else EB.edge_orbits4_combo(n, s, d)
    assert got.tolist() == want.tolist()


def test_edge_orbits_random_graphs_against_brute_force(harp):
    rng = np.random.default_rng(78)
    for trial in range(30):
        n = int(rng.integers(5, 22))
        p = float(rng.uniform(0.1, 0.7))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        s, d = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
        if s.size == 0:
            continue
        got, _ = gpu_edge_orbits(harp, n, s, d)
        assert got.tolist() == EB.edge_orbits4_brute(n, s, d).tolist(), (trial, n, p)


@pytest.mark.parametrize("make", [lambda: graphgen.ba(1500, 4, 1), lambda: graphgen.er(1200, 10, 3),
                                  lambda: graphgen.rgg(1500, 12, 4), lambda: graphgen.chung_lu(2500, 2.1, 150, 6, 5)],
                         ids=["ba1500", "er1200", "rgg1500", "chunglu2500"])
def test_edge_orbits_generated_graphs_against_the_per_edge_oracle(harp, make):
    g = make()
    got, _ = gpu_edge_orbits(harp, g.n, g.src, g.dst)
    assert got.tolist() == EB.edge_orbits4_combo(g.n, g.src, g.dst).tolist()


@pytest.mark.parametrize("scale", [14, 16])
def test_edge_role_sums_equal_global_counts(harp, scale):
    g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, seed=3)
    got, counts = gpu_edge_orbits(harp, g.n, g.src, g.dst)
    sums = got.sum(axis=0, dtype=np.uint64)
    for r in range(10):
        want = (int(counts[EB.EDGE_ORBIT_MOTIF[r]]) * EB.EDGE_ORBIT_SIZE[r]) % 2**64
        assert int(sums[r]) == want, EB.EDGE_ORBITS[r]
