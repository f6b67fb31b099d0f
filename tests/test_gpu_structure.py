"""Parity of the CUDA structure steps with the oracle, bit for bit: the
pore-sphere reconstruction (Sec. 2), the 18-neighbour labelling and transport
set (Sec. 4.1), the 13-direction pore size (Sec. 4.1) and the inscribed-sphere
pore size -- at small sizes, ragged shapes and the full workload sizes."""
import numpy as np
import pytest

import synthetic as S
from conftest import recon_args, recon_params

pytestmark = pytest.mark.gpu

SMALL = [
    S.small_structure(1).with_(shape=(24, 24, 24)),
    S.small_structure(2).with_(shape=(20, 33, 37), porosity=0.3),
    S.Recon(5, (16, 16, 16), 1.0, 6.0, 1.5, 3.0, 10.0, 0.45, 0.5, p0=0.2, dist=1),
    S.Recon(7, (40, 24, 30), 1.5, 9.0, 2.0, 4.5, 15.0, 0.25, 0.1, p0=0.8),
    S.small_structure(3),
]


def _recon_both(orc, om, cfg):
    rc, mask_o, sph, eps_o, _ = orc.reconstruct(*recon_args(cfg))
    st, mask_g, eps_g, n_g = om.om_reconstruct(cfg.seed, om.domain(cfg.shape, cfg.dx_nm), recon_params(om, cfg))
    return rc, mask_o, len(sph), eps_o, st, mask_g, n_g, eps_g


@pytest.mark.parametrize("cfg", SMALL)
def test_reconstruct_bit_exact(orc, om, cfg):
    rc, mo, no, eo, st, mg, ng, eg = _recon_both(orc, om, cfg)
    assert rc == 0 and st == om.OM_OK
    assert np.array_equal(mo, mg)
    assert no == ng and eo == eg


def test_reconstruct_infeasible_status(orc, om):
    cfg = S.Recon(2, (16, 16, 16), 1.0, 8.0, 0.5, 7.0, 9.0, 0.8, 0.0, p0=0.0, max_trials=20000)
    rc, mo, no, eo, st, mg, ng, eg = _recon_both(orc, om, cfg)
    assert rc == orc.ORC_EINFEASIBLE and st == om.OM_EINFEASIBLE
    assert np.array_equal(mo, mg) and no == ng


def test_reconstruct_rejects_bad_arguments(om):
    with pytest.raises(om.OmError) as e:
        om.om_reconstruct(1, om.domain((8, 8, 8)), om.recon_params(5, 1, 2, 8, 1.5, 0.2))
    assert e.value.status == om.OM_EINVAL
    with pytest.raises(om.OmError):
        om.om_reconstruct(1, om.domain((0, 8, 8)), om.recon_params(5, 1, 2, 8, 0.3, 0.2))


@pytest.mark.parametrize("cfg", SMALL[:4])
def test_labels_bit_exact(orc, om, cfg):
    _, mask, *_ = orc.reconstruct(*recon_args(cfg))
    lo, to, co = orc.label18(mask)
    lg, tg, cg = om.om_label_connectivity(mask)
    assert np.array_equal(lo, lg) and np.array_equal(to, tg) and co == cg


@pytest.mark.parametrize("seed,shape,p", [(1, (5, 4, 3), 0.45), (2, (9, 7, 33), 0.4), (3, (1, 6, 6), 0.5),
                                          (4, (12, 2, 1), 0.6), (5, (31, 17, 65), 0.35)])
def test_labels_random_masks(orc, om, seed, shape, p):
    m = S.random_mask(shape, p, seed)
    lo, to, co = orc.label18(m)
    lg, tg, cg = om.om_label_connectivity(m)
    assert np.array_equal(lo, lg) and np.array_equal(to, tg) and co == cg


def test_labels_empty_and_full(orc, om):
    for m in (np.zeros((4, 5, 6), np.uint8), np.ones((4, 5, 6), np.uint8)):
        lo, to, co = orc.label18(m)
        lg, tg, cg = om.om_label_connectivity(m)
        assert np.array_equal(lo, lg) and np.array_equal(to, tg) and co == cg


@pytest.mark.parametrize("cfg", SMALL[:4])
def test_chord13_bit_exact(orc, om, cfg):
    _, mask, *_ = orc.reconstruct(*recon_args(cfg))
    do, co = orc.chord13(mask, cfg.dx_nm)
    dg, cg = om.om_local_pore_diameter(mask, om.domain(cfg.shape, cfg.dx_nm), om.OM_PORE_CHORD13, witness=True)
    assert np.array_equal(co, cg)
    assert np.array_equal(do, dg)


def test_chord13_closed_loops(orc, om):
    # all-pore box: every line wraps; counts are the loop periods
    m = np.ones((3, 4, 6), np.uint8)
    do, co = orc.chord13(m)
    dg, cg = om.om_local_pore_diameter(m, om.domain(m.shape), om.OM_PORE_CHORD13, witness=True)
    assert np.array_equal(co, cg) and np.array_equal(do, dg)


@pytest.mark.parametrize("cfg", [SMALL[0], SMALL[2], SMALL[1].with_(shape=(14, 17, 19))])
def test_mis_bit_exact(orc, om, cfg):
    _, mask, *_ = orc.reconstruct(*recon_args(cfg))
    rc, do, r2o = orc.mis(mask, cfg.dx_nm)
    dg, r2g = om.om_local_pore_diameter(mask, om.domain(cfg.shape, cfg.dx_nm), om.OM_PORE_MIS, witness=True)
    assert rc == 0
    assert np.array_equal(r2o, r2g)
    assert np.array_equal(do, dg)


def test_mis_no_solid_rejected(om):
    with pytest.raises(om.OmError) as e:
        om.om_local_pore_diameter(np.ones((4, 4, 4), np.uint8), None, om.OM_PORE_MIS)
    assert e.value.status == om.OM_EINVAL


@pytest.mark.slow
def test_small_workload_structure_bit_exact(orc, om):
    """The 48^3, 2 nm, porosity 0.40 workload: mask, labels and the
    inscribed-sphere pore size that feeds its diffusion solve."""
    cfg = S.small_structure(1)
    rc, mo, no, eo, st, mg, ng, eg = _recon_both(orc, om, cfg)
    assert rc == 0 and st == 0 and np.array_equal(mo, mg) and no == ng
    lo, to, co = orc.label18(mo)
    lg, tg, cg = om.om_label_connectivity(mo)
    assert np.array_equal(lo, lg) and np.array_equal(to, tg)
    rc, do, r2o = orc.mis(mo, cfg.dx_nm)
    dg, r2g = om.om_local_pore_diameter(mo, om.domain(cfg.shape, cfg.dx_nm), om.OM_PORE_MIS, witness=True)
    assert np.array_equal(r2o, r2g) and np.array_equal(do, dg)


@pytest.mark.slow
@pytest.mark.parametrize("eps", S.SWEEP_POROSITIES)
def test_sweep_workload_structure_bit_exact(orc, om, eps):
    """The 256^3, 1 nm porosity-sweep structures at full size: mask, labels,
    transport set and 13-direction pore size, every voxel."""
    cfg = S.sweep_structure(eps)
    rc, mo, no, eo, st, mg, ng, eg = _recon_both(orc, om, cfg)
    assert rc == 0 and st == 0 and np.array_equal(mo, mg) and no == ng and eo == eg
    lo, to, co = orc.label18(mo)
    lg, tg, cg = om.om_label_connectivity(mo)
    assert np.array_equal(lo, lg) and np.array_equal(to, tg) and co == cg
    do, _ = orc.chord13(mo, cfg.dx_nm, counts=False)
    dg, _ = om.om_local_pore_diameter(mo, om.domain(cfg.shape, cfg.dx_nm), om.OM_PORE_CHORD13)
    assert np.array_equal(do, dg)


@pytest.mark.parametrize("shape,seed", [((40, 33, 29), 3), ((64, 48, 40), 5), ((96, 64, 64), 9)])
def test_labels_repeatable_under_contention(orc, om, shape, seed):
    """Union-find labels must be the canonical ones on every run, not only on
    most: thin one-voxel channels with many concurrent links are where a
    racy root compression shows up.  Repeated runs against the oracle."""
    m = S.blob_mask(shape, seed, n=12, rmin=2.0, rmax=7.0)
    lo, to, co = orc.label18(m)
    for _ in range(40):
        lg, tg, cg = om.om_label_connectivity(m)
        assert np.array_equal(lo, lg) and np.array_equal(to, tg) and co == cg
