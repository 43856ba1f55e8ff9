"""The 5-vertex class table of the library (built by its host code from the definition: smallest
10-bit adjacency mask over the 120 permutations, classes in increasing (edge count, key) order) equals
the oracle's, and needs no GPU."""
from oracle import motifs5 as M5


def test_library_class_keys_equal_the_oracles():
    from paper_2607_12074_gb300 import _build, harp
    _build.build()
    keys = harp.harp_motif5_classes()
    assert len(keys) == 21
    assert tuple(keys) == M5.CLASSES
