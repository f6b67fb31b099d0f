"""The allocation-free labelling entry point, om_label_connectivity_noalloc.

Some callers cannot allocate device memory: their GPU memory is held by
another allocator, or their memory plan is fixed at start-up.  This entry
point gives them the same labelling as om_label_connectivity_dev with its
scratch in a static device array.  The test calls both through the C ABI,
twice in a row on different masks (the shared scratch keeps the previous
call's contents, so the second call shows it is cleared), and compares
labels, transport flags and connectivity exactly -- the labelling is integer
work and the parity bar for it is bit-exact.  It lives in its own file,
collected last, and needs nothing from the other tests.
"""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _both(om, m):
    dom = om.domain(m.shape)
    md = torch.from_numpy(np.ascontiguousarray(m)).cuda()
    lab_a = torch.empty(m.size, dtype=torch.int32, device="cuda")
    tr_a = torch.empty(m.size, dtype=torch.uint8, device="cuda")
    lab_b = torch.full((m.size,), -7, dtype=torch.int32, device="cuda")
    tr_b = torch.full((m.size,), 9, dtype=torch.uint8, device="cuda")
    conn_a = om.om_label_connectivity_dev(md, dom, lab_a, tr_a)
    conn_b = om.om_label_connectivity_noalloc(md, dom, lab_b, tr_b)
    torch.cuda.synchronize()
    return (lab_a.cpu().numpy(), tr_a.cpu().numpy(), conn_a), (lab_b.cpu().numpy(), tr_b.cpu().numpy(), conn_b)


def test_noalloc_matches_allocating_entry_point_twice(om, orc):
    first = S.blob_mask((40, 33, 29), 3, n=9, rmin=2.0, rmax=6.0)
    second = S.random_mask((24, 20, 36), 0.55, 8)  # different shape and components
    for m in (first, second):
        (la, ta, ca), (lb, tb, cb) = _both(om, m)
        assert np.array_equal(la, lb)
        assert np.array_equal(ta, tb)
        assert ca == cb
        # and the oracle's 18-neighbour labelling (Sec. 4.1), directly
        lo, to, co = orc.label18(m)
        assert np.array_equal(lb, lo.reshape(-1)) and np.array_equal(tb, to.reshape(-1)) and cb == co
    assert ta.sum() > 0


def test_noalloc_at_the_largest_box_it_accepts(om):
    # 256^3 = 2^24 voxels: the packed flags fill every word of the static
    # array and the counters sit right behind them
    m = S.random_mask((256, 256, 256), 0.6, 11)
    (la, ta, ca), (lb, tb, cb) = _both(om, m)
    assert np.array_equal(la, lb) and np.array_equal(ta, tb) and ca == cb
    assert ta.sum() > 0


def test_noalloc_rejects_boxes_beyond_the_static_limit(om):
    dom = om.domain((257, 256, 256))
    dummy = torch.zeros(1, dtype=torch.uint8, device="cuda")
    lab = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(om.OmError) as e:
        om.om_label_connectivity_noalloc(dummy, dom, lab)
    assert e.value.status == om.OM_EINVAL and "16777216" in str(e.value)
