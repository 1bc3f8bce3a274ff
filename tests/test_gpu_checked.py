"""The checked build (``-m gpu``, library built and loaded with IVHD_CHECKED=1).

The memory checker is closed on this machine; the checked library stands in for
it.  Its step kernels test every gathered index and row extent before use, and
the conftest fixture asserts after every GPU test that none was out of range.
Here a layout entry is overwritten with an out-of-range id: each step must
count it once, skip it, and keep the embedding finite, through the
multi-launch kernel and the cluster kernel alike.  With the normal library
the corruption hook refuses and these tests are skipped.
"""
import os

import numpy as np
import pytest

from paper_2303_05455_gb300 import _lib, ivhd, synth

pytestmark = [pytest.mark.gpu, pytest.mark.plants_violations]

CHECKED = os.environ.get("IVHD_CHECKED", "") not in ("", "0")


def test_normal_library_refuses_corruption():
    if CHECKED:
        pytest.skip("checked library loaded")
    emb = ivhd.Embedding(synth.random_knn_graph(500, 3, 1), r=1, c=0.1, seed=1)
    assert _lib.load().ivhd_test_corrupt_layout(emb._h, 0, 0xFFFFFFF) == -1
    assert ivhd.check_violations() == -1
    emb.close()


@pytest.mark.skipif(not CHECKED, reason="needs the checked library (IVHD_CHECKED=1)")
@pytest.mark.parametrize("resident", [False, "cluster"])
def test_out_of_range_id_is_counted_and_skipped(resident):
    L = _lib.load()
    M = 3000
    knn = synth.random_knn_graph(M, 4, 2, hub_frac=0.1, n_hubs=8)
    emb = ivhd.Embedding(knn, r=1, c=0.05, seed=3, resident=resident, hub_threshold=16)
    ivhd.check_violations(reset=True)
    emb.step(5)
    assert ivhd.check_violations(reset=True) == 0
    assert L.ivhd_test_corrupt_layout(emb._h, 0, M + 7) == 0
    emb.step(10)
    assert ivhd.check_violations(reset=True) == 10      # one skipped gather per step
    assert np.all(np.isfinite(emb.positions(host=True)))
    assert L.ivhd_test_corrupt_layout(emb._h, emb.info()["layout_slots"], 0) == -1
    emb.close()
