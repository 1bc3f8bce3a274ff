"""The largest layouts the step accepts, and the first one it refuses.

The symmetric layout addresses its id slots with 32-bit offsets, so a graph
whose padded layout needs 2^31 - 1 slots or more is refused (IVHD_ERR_ARG)
before anything is allocated for it.  A circulant kNN graph with k = 7 and
r = 0 gives every vertex 14 symmetric entries (7 out, 7 in, no mutual pair),
stored as 4 int4 groups of a SELL slice: 16 slots per vertex, 512 per slice,
the last slice padded like the others.

* M = 2^27 - 37: 4,194,303 slices, 2^31 - 512 slots (offsets reach the top of
  the int32 range; the last slice is ragged, 27 rows).  One momentum step
  (Sec. 3.3.3, Eq. 3.34) and the forces after it are checked element by
  element against the FP64 oracle on sampled vertices (the first and last
  rows, the wrap-around neighbourhood, the ragged last slice), with the
  oracle's terms restricted to those touching the sample (all of a sampled
  vertex's terms, so its force is exact).  The initial positions are compared
  with the oracle's on every vertex.
* M = 2^27 - 31: 2^22 slices, exactly 2^31 slots: refused by the layout build
  (the host-side size check, 2 M (k + r) < 2^31, passes).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd
from paper_2303_05455_gb300._lib import IvhdError
from step_bounds import close_elem, force_error_bound, step_bound

pytestmark = pytest.mark.gpu

OFFS = np.array([1, 2, 3, 5, 8, 13, 21], np.int64)
A, B, C, SEED = 0.9, 0.01, 0.01, 27


def circulant(M):
    knn = np.empty((M, OFFS.size), np.int32)
    i = np.arange(M, dtype=np.int64)
    for q, o in enumerate(OFFS):
        knn[:, q] = (i + o) % M
    return knn


def terms_touching(sample, M):
    """The nn terms (row u, slot q) -> (u, u + OFFS[q]) that touch a sampled vertex."""
    keys = set()
    for v in sample:
        for q, o in enumerate(OFFS):
            keys.add((int(v), q))                  # v's own entry
            keys.add((int((v - o) % M), q))        # the entry of the row that lists v
    u = np.array([k[0] for k in keys], np.int64)
    q = np.array([k[1] for k in keys], np.int64)
    return oracle.Terms(u, (u + OFFS[q]) % M, np.zeros(u.size, np.int8), M)


def test_layout_at_the_top_of_the_32_bit_offsets_steps_like_the_oracle():
    M = 2 ** 27 - 37
    emb = ivhd.Embedding(circulant(M), r=0, c=C, a=A, b=B, seed=SEED)
    inf = emb.info()
    assert inf["layout_slots"] == 2 ** 31 - 512
    assert inf["n_terms"] == 7 * M and inf["nnz_sym"] == 14 * M and inf["n_hub"] == 0
    y0 = emb.positions(host=True)
    assert np.array_equal(y0, oracle.init_positions(M, SEED).astype(np.float32))
    last = 32 * (M // 32)                           # first row of the ragged last slice
    S = np.unique(np.array([0, 1, 2, 20, 21, 22, 12345, M // 2, last - 1, last, last + 13,
                            M - 22, M - 21, M - 2, M - 1], np.int64))
    terms = terms_touching(S, M)
    y0d = y0.astype(np.float64)
    F0 = oracle.forces(y0d, terms, C)
    st = oracle.State.fresh(y0d)
    oracle.step(st, terms, C, oracle.OPT_MOMENTUM, a=A, b=B)
    emb.step(1)
    y1 = emb.positions(host=True)
    d_ref = (st.Y - y0d)[S]
    bound = step_bound("momentum", st.Y[S], d_ref, F0[S],
                       force_error_bound(y0d, terms, C)[S], A, B)
    close_elem(y1[S].astype(np.float64) - y0d[S], d_ref, bound, "displacement")
    y1d = y1.astype(np.float64)
    F1 = emb.forces(host=True)
    close_elem(F1[S], oracle.forces(y1d, terms, C)[S],
               force_error_bound(y1d, terms, C)[S] + 1e-30, "forces")
    emb.close()


def test_layout_of_2_to_the_31_slots_is_refused():
    M = 2 ** 27 - 31
    assert 2 * M * (OFFS.size + 0) < 2 ** 31 - 1       # passes the host-side check
    with pytest.raises(IvhdError) as e:
        ivhd.Embedding(circulant(M), r=0, c=C, a=A, b=B, seed=SEED)
    assert e.value.status == -1
    # the device is still usable
    small = ivhd.Embedding(circulant(1000), r=0, c=C, a=A, b=B, seed=SEED)
    small.step(2)
    assert np.isfinite(small.positions(host=True)).all()
    small.close()
