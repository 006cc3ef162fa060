"""Static decomposition (Sec. 5, Sec. 6.1) on the GPU, checked against the
oracle: SLAB_OCT must give exactly the undecomposed candidate list; ALT_BANDS
must give the undecomposed list restricted to pairs joined in the
potential-collision graph (Def 9: padded radial ranges intersect)."""
import numpy as np
import pytest
import torch

import oracle as O
import population as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scd():
    import paper_1901_10475_gb300 as m
    torch.cuda.set_device(0)
    return m


def _same(got, want):
    g = np.asarray(got).view(np.int32).reshape(-1, 4)
    w = np.asarray(want).view(np.int32).reshape(-1, 4)
    return g.shape == w.shape and bool((g == w).all())


def _oracle_plain(sc):
    lo, hi, obj = (x.cpu().numpy() for x in sc.boxes())
    return O.canonicalize(O.raw_cells_sweep(lo, hi, obj.view(np.uint32)))


@pytest.mark.parametrize("n_slabs", [1, 7, 16])
def test_slab_oct_equals_plain(scd, n_slabs):
    els = P.catalog_mixture(n=700, seed=41, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 20000.0, 1.0, pol).build_boxes()
    plain = sc.find_pairs()
    dec = sc.find_pairs((scd.SCD_DECOMP_SLAB_OCT, 0, n_slabs))
    want = _oracle_plain(sc)
    assert _same(plain, want)
    assert _same(dec, want), (len(dec), len(want))
    assert len(want) > 100
    sc.close()


def test_slab_oct_band_table_and_more_slabs_than_ticks(scd):
    els = P.uniform_leo(120, seed=43, radius_km=60.0)
    edges, fr = P.band_table_config3()
    pol = scd.make_step_policy(scd.SCD_STEP_BAND_TABLE, band_edges_km=edges, band_fractions=fr)
    sc = scd.Scene(els, 300.0, 1.0, pol).build_boxes()
    want = _oracle_plain(sc)
    for n_slabs in (16, 400):
        assert _same(sc.find_pairs((scd.SCD_DECOMP_SLAB_OCT, 0, n_slabs)), want)
    sc.close()


@pytest.mark.parametrize("p", [1, 4, 16])
def test_alt_bands_equals_filtered_plain(scd, p):
    els = P.catalog_mixture(n=800, seed=42, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 20000.0, 1.0, pol).build_boxes()
    dec = sc.find_pairs((scd.SCD_DECOMP_ALT_BANDS, p, 0))
    want = O.potential_collision_filter(els, _oracle_plain(sc))
    assert _same(dec, want), (len(dec), len(want))
    assert len(want) > 50
    sc.close()


def test_decomposition_argument_checks(scd):
    els = P.uniform_leo(20, seed=44)
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, 100.0, 1.0, pol).build_boxes()
    for bad in [(scd.SCD_DECOMP_SLAB_OCT, 0, 0), (scd.SCD_DECOMP_ALT_BANDS, 0, 0),
                (scd.SCD_DECOMP_ALT_BANDS, 21, 0), (7, 1, 1)]:
        with pytest.raises(scd.ScdError) as e:
            sc.find_pairs(bad)
        assert e.value.status == scd._binding.SCD_ERR_INVALID_ARG
    sc.close()


@pytest.mark.parametrize("decomp", [None, "slab", "bands"])
def test_four_wide_nodes_give_the_same_lists(scd, decomp):
    """Node width 4 (grandchildren in one line, cell subtrees rooted at
    binary nodes) gives the same lists as binary nodes, plain and
    decomposed, eagerly and replayed as a CUDA graph."""
    els = P.catalog_mixture(n=700, seed=44, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    d = {None: None, "slab": (scd.SCD_DECOMP_SLAB_OCT, 0, 16),
         "bands": (scd.SCD_DECOMP_ALT_BANDS, 8, 0)}[decomp]
    ref = scd.Scene(els, 20000.0, 1.0, pol).build_boxes()
    want = ref.find_pairs(d)
    ref.close()
    assert len(want) > 100
    for graph in (0, 1):
        sc = scd.Scene(els, 20000.0, 1.0, pol, tuning=dict(node_width=4, use_graph=graph))
        for _ in range(3):  # a graph is captured on the first call and replayed after
            sc.build_boxes()
            assert _same(sc.find_pairs(d), want)
        sc.close()
