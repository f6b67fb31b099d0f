"""Checkpoint and resume (om_*_save_state / om_*_load_state): a solver
restored from a saved state continues bit for bit as the saved one does, in
every storage format, for the flow and both diffusion lattices, through
single steps and captured check windows; images of another solver are
refused and leave the solver unchanged."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


def _pops(obj, q, n):
    out = torch.empty(q * n, dtype=torch.float64, device="cuda")
    obj.get_populations(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


NODE = S.blob_mask((20, 24, 40), 11, n=9)
D_NM = (S.random_field(NODE.shape, 5, 3.0, 90.0) * NODE).astype(np.float32)


def _flow(om, ns, prec):
    return om.Flow(ns, om.flow_params(tau=0.9, body_force=1e-5, precision=prec, check_every=4))


def _diff(om, ns, prec, q):
    return om.Diffusion(ns, _dev(D_NM), om.diff_params(precision=prec, check_every=4, lattice=q, c_in=0.9, c_out=0.1))


@pytest.mark.parametrize("prec", ["OM_F64", "OM_F32", "OM_F16DEV", "OM_BF16DEV"])
@pytest.mark.parametrize("model", ["flow", "d3q7", "d3q19"])
def test_resume_is_bit_identical(om, prec, model):
    P = getattr(om, prec)
    ns = om.NodeSet(_dev(NODE), om.domain(NODE.shape))
    make = (lambda: _flow(om, ns, P)) if model == "flow" else (lambda: _diff(om, ns, P, 7 if model == "d3q7" else 19))
    q = 19 if model != "d3q7" else 7
    a = make()
    a.step(9)  # odd time: the image carries the parity
    img = a.save_state()
    a.step(13)  # single sweeps, then whole windows from the next even time
    b = make()
    b.step(2)  # some other state, overwritten by the image
    b.load_state(img)
    assert b.time == 9
    b.step(13)
    assert a.time == b.time == 22
    assert np.array_equal(_pops(a, q, NODE.size), _pops(b, q, NODE.size))
    # and the convergence state: both observe the same change
    assert a.observe() == b.observe()


def test_foreign_images_are_refused(om):
    ns = om.NodeSet(_dev(NODE), om.domain(NODE.shape))
    fl = _flow(om, ns, om.OM_F32)
    fl.step(3)
    before = _pops(fl, 19, NODE.size)
    other = _flow(om, ns, om.OM_F16DEV).save_state()
    diff = _diff(om, ns, om.OM_F32, 7).save_state()
    node2 = NODE.copy()
    node2[0, 0, 0] ^= 1
    small = _flow(om, om.NodeSet(_dev(node2), om.domain(NODE.shape)), om.OM_F32).save_state()
    own = fl.save_state()
    for bad in (other, diff, small, own[:100], np.zeros_like(own)):
        with pytest.raises(om.OmError):
            fl.load_state(bad)
    assert fl.time == 3
    assert np.array_equal(_pops(fl, 19, NODE.size), before)
