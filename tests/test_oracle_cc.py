"""Pins for the automatic subdomain-levelset oracle (connected components of
each subdomain's levelset classes): against scipy.ndimage.label on each
(subdomain, class) mask, hand-built layered and checkerboard fields, and the
plain SLD labels when every region is connected.  CPU only."""
import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W


@pytest.fixture(scope="module")
def cc():
    import oracle
    from oracle import sld_cc
    oracle.build()
    return oracle, sld_cc


def _partition_equal(a, b):
    """Two labelings describe the same partition of the cells."""
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_scipy_components_per_region(cc, seed):
    import scipy.ndimage as ndi
    oracle, C = cc
    rng = np.random.default_rng(seed)
    K = np.exp(2.5 * rng.standard_normal((7, 9, 11)))
    S, tau, L = (2, 3, 2), (0.3, 3.0), 3
    lab, d = C.cc_labels(K, S, tau, L)
    base = oracle.labels(K, S, tau, L)
    ref = np.full(K.size, -1, dtype=np.int64)
    nxt = 0
    for v in np.unique(base):
        comp, nc = ndi.label((base == v).reshape(K.shape))  # 6-connectivity (default structure)
        comp = comp.reshape(-1)
        m = comp > 0
        ref[m] = comp[m] - 1 + nxt
        nxt += nc
    assert d == nxt
    assert _partition_equal(lab, ref)
    # canonical order: by (SLD label, smallest cell index)
    first = np.array([np.flatnonzero(lab == k)[0] for k in range(d)])
    keys = list(zip(base[first].tolist(), first.tolist()))
    assert keys == sorted(keys)
    # a component never spans two SLD labels
    for k in range(d):
        assert np.unique(base[lab == k]).size == 1


def test_layers_become_one_vector_each(cc):
    """The paper's manual vectors for layered reservoirs: one per layer."""
    oracle, C = cc
    K = W.layered(10, 6, 12, 4, 1.0, 1e-6)  # 4 layers of 3 cells in z, alternating
    lab, d = C.cc_labels(K, (1, 1, 1), (1e-3,), 2)
    assert d == 4
    z_of = np.repeat(np.arange(12), 60)
    for k in range(4):
        assert np.array_equal(np.unique(z_of[lab == k] // 3), [np.unique(z_of[lab == k] // 3)[0]])
        assert np.count_nonzero(lab == k) == 180
    # two subdomains in z: layers split at the subdomain face
    lab2, d2 = C.cc_labels(K, (1, 1, 2), (1e-3,), 2)
    assert d2 == 4  # the 6-cell subdomains hold 2 layers each, no layer crosses z = 6


def test_checkerboard_every_cell_alone(cc):
    oracle, C = cc
    z, y, x = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    K = np.where((x + y + z) % 2 == 0, 1.0, 1e-6)
    lab, d = C.cc_labels(K, (1, 1, 1), (1e-3,), 2)
    assert d == K.size
    flat = K.reshape(-1)
    low = np.flatnonzero(flat < 1e-3)
    high = np.flatnonzero(flat >= 1e-3)
    expect = np.empty(K.size, dtype=np.int32)
    expect[low] = np.arange(low.size)                  # class 0 first, in index order
    expect[high] = low.size + np.arange(high.size)
    assert np.array_equal(lab, expect)


def test_connected_regions_keep_the_sld_labels(cc):
    oracle, C = cc
    K = np.full((6, 8, 10), 2.0)
    lab, d = C.cc_labels(K, (2, 2, 3), (), 1)
    assert d == 12
    assert np.array_equal(lab, oracle.labels(K, (2, 2, 3), (), 1))
