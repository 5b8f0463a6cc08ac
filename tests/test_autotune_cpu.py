"""Host logic of the autotuner (CPU): shape features, class keys, candidate
sets, the stored table and the lookup guards."""
import json

import numpy as np

from paper_1004_4548_gb300 import autotune as at
from workloads import Poly, random_poly, random_pseries, workload_cfg2


def test_features_give_the_product_box():
    f, g = workload_cfg2()
    feat = at.features(f, g)
    assert not feat["poisson"]
    assert feat["pairs"] == 10626 * 10626
    assert feat["W"] == 41.0 ** 4            # widths of the output box (each variable 0..40)
    p = random_pseries(2, 2, 50, 3, 4, 11)
    q = random_pseries(2, 2, 40, 3, 4, 12)
    feat = at.features(p, q)
    w_poly = np.prod((p.exps.max(1).astype(np.int64) + q.exps.max(1)) - (p.exps.min(1) + q.exps.min(1)) + 1)
    R = np.abs(p.trig).max(1).astype(np.int64) + np.abs(q.trig).max(1)
    assert feat["poisson"] and feat["W"] == float(w_poly * np.prod(2 * R + 1))


def test_class_keys_bin_by_size_and_density():
    k = at.class_key({"poisson": False, "pairs": 1 << 20, "W": float(1 << 24)})
    assert k == "poly|p20|d4"
    assert at.class_key({"poisson": False, "pairs": 1 << 20, "W": 1.0}) == "poly|p20|d-10"   # clamped
    assert at.class_key({"poisson": False, "pairs": 1 << 10, "W": 2.0 ** 40}) == "poly|p10|d14"
    assert at.class_key({"poisson": True, "pairs": 3000, "W": 1e9}) == "pois|p12"


def test_candidates_keep_the_dense_path_to_arrays_that_fit():
    small = at.candidates({"poisson": False, "pairs": 1000, "W": 1e6})
    assert [c["block_slots"] for c in small if c["path"] == 1] == list(at.DENSE_S)
    assert [c["load_factor"] for c in small if c["path"] == 2] == list(at.HASH_ALPHA)
    assert all(c["path"] == 2 for c in at.candidates({"poisson": False, "pairs": 1000, "W": 1e12}))
    assert all(c["path"] == 2 for c in at.candidates({"poisson": True, "pairs": 1000, "W": 1e3}))


def test_stored_table_holds_only_candidates():
    with open(at.TABLE) as fh:
        table = json.load(fh)["classes"]
    assert len(table) > 0
    for key, o in table.items():
        assert key.startswith(("poly|p", "pois|p")), key
        if o["path"] == 1:
            assert o["block_slots"] in at.DENSE_S and key.startswith("poly"), (key, o)
        else:
            assert o["path"] == 2 and o["load_factor"] in at.HASH_ALPHA, (key, o)


def test_lookup_guards():
    f = random_poly(3, 200, -3, 3, 21)
    g = random_poly(3, 150, -3, 3, 22)
    key = at.class_key(at.features(f, g))
    assert at.opts_for(f, g, table={}) == {}                                  # never tuned
    assert at.opts_for(f, g, table={key: {"path": 2, "load_factor": 0.3}}) == {"path": 2, "load_factor": 0.3}
    # a dense entry is dropped for a product whose array would not fit
    big = Poly(np.array([[0, 1 << 20], [0, 1 << 20], [0, 1 << 10]], np.int32), np.array([1, 2], np.int64))
    kb = at.class_key(at.features(big, big))
    assert at.opts_for(big, big, table={kb: {"path": 1, "block_slots": 4096}}) == {}
