"""fc_partition (host only, no GPU): patches ordered along the Morton curve of their
centres, cut into runs of about equal active point counts."""
import numpy as np
import pytest

from paper_2506_16076_gb300 import fcsdnn, workloads as W


def _centres(w):
    out = []
    for p in w.patches:
        x, y = W.patch_xy(p)
        out.append((x.mean(), y.mean()))
    return np.array(out)


def _morton(c):
    lo, span = c.min(axis=0), max(np.ptp(c[:, 0]), np.ptp(c[:, 1]))
    q = np.minimum(65535, np.floor((c - lo) / span * 65535)).astype(np.int64)
    key = np.zeros(len(c), dtype=np.int64)
    for b in range(16):
        key |= ((q[:, 0] >> b) & 1) << (2 * b)
        key |= ((q[:, 1] >> b) & 1) << (2 * b + 1)
    return key


@pytest.mark.parametrize("nranks", [1, 2, 4, 8])
def test_balanced_contiguous_runs(nranks):
    w = W.cyl_m25_32()
    owner = np.array(fcsdnn.partition(w, nranks))
    assert owner.min() == 0 and owner.max() == nranks - 1
    # contiguous along the Morton curve: owners never decrease in curve order
    order = np.lexsort((np.arange(len(owner)), _morton(_centres(w))))
    assert np.all(np.diff(owner[order]) >= 0)
    # balanced: the hole blanks only a few patches' points, so n1 n2 is close to the weight
    load = np.bincount(owner, weights=[p.n1 * p.n2 for p in w.patches], minlength=nranks)
    assert load.max() / load.mean() < 1.03, load
    assert fcsdnn.partition(w, nranks) == list(owner)  # deterministic


def test_more_ranks_than_patches_and_bad_counts():
    w = W.small_multipatch()
    owner = fcsdnn.partition(w, 8)
    assert len(owner) == 5 and min(owner) >= 0 and max(owner) < 8
    with pytest.raises(fcsdnn.FcError):
        fcsdnn.partition(w, 0)
