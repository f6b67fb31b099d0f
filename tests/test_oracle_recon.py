"""Oracle pins for random numbers and the pore-sphere reconstruction (Sec. 2).

The reconstruction has no printed worked example in the paper, so its pins
are invariants that any correct implementation of Sec. 2 satisfies: the
porosity stop rule, the pairwise overlap tolerance, the overlap requirement,
the mask being the union of the accepted balls, and the diameter law.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import synthetic as S


def test_splitmix64_known_answers(orc):
    # published SplitMix64 reference outputs (Vigna's splitmix64.c)
    assert orc.splitmix64(1234567, 5) == [6457827717110365317, 3203168211198807973,
                                          9817491932198370423, 4593380528125082431,
                                          16408922859458223821]
    assert orc.splitmix64(1477776061723855037, 3) == [1985237415132408290, 2979275885539914483,
                                                      13511426838097143398]


def test_uniforms_in_unit_interval(orc):
    u = orc.uniforms(42, 20000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.003


def _lens_by_quadrature(r1, r2, d):
    # coaxial cross-sections: at abscissa x both balls cut discs centred on
    # the axis, so the intersection's area is pi * min(a1, a2)^2
    lo, hi = max(-r1, d - r2), min(r1, d + r2)
    if hi <= lo:
        return 0.0

    def area(x):
        a1 = r1 * r1 - x * x
        a2 = r2 * r2 - (x - d) ** 2
        return math.pi * max(0.0, min(a1, a2))

    v, _ = integrate.quad(area, lo, hi, epsabs=1e-13, epsrel=1e-12, limit=200)
    return v


@pytest.mark.parametrize("r1,r2,d", [(5, 5, 3), (5, 5, 9.99), (7, 3, 6), (7, 3, 4.5), (2, 6, 5.5),
                                      (4, 4, 0.5), (3, 8, 4.0), (3, 8, 12), (6, 2.5, 8.4)])
def test_lens_volume_matches_quadrature(orc, r1, r2, d):
    v = orc.lens_volume(r1, r2, d)
    q = _lens_by_quadrature(r1, r2, d)
    assert v == pytest.approx(q, rel=1e-9, abs=1e-12)
    assert orc.lens_volume(r2, r1, d) == pytest.approx(v, rel=1e-14)


def test_sphere_volume(orc):
    assert orc.sphere_volume(2.0) == pytest.approx(4.0 / 3.0 * math.pi * 8.0, rel=1e-15)


def _union_of_balls(shape, spheres):
    nx, ny, nz = shape
    X, Y, Z = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5, indexing="ij")
    m = np.zeros(shape, bool)
    for cx, cy, cz, r in spheres:
        for ky in (-1, 0, 1):
            for kz in (-1, 0, 1):
                m |= (X - cx) ** 2 + (Y - (cy + ky * ny)) ** 2 + (Z - (cz + kz * nz)) ** 2 <= r * r
    return m


def _min_image_dist(a, b, ny, nz):
    dx = a[0] - b[0]
    dy = a[1] - b[1]
    dz = a[2] - b[2]
    dy -= ny * round(dy / ny)
    dz -= nz * round(dz / nz)
    return math.sqrt(dx * dx + dy * dy + dz * dz)


RECON_CASES = [
    S.Recon(3, (24, 24, 24), 2.0, 10.0, 3.0, 4.0, 20.0, 0.30, 0.3),
    S.Recon(11, (20, 28, 16), 1.5, 9.0, 2.0, 4.5, 15.0, 0.25, 0.1, p0=0.8),
    S.Recon(5, (16, 16, 16), 1.0, 6.0, 1.5, 3.0, 10.0, 0.45, 0.5, p0=0.2, dist=1),
]


@pytest.mark.parametrize("cfg", RECON_CASES)
def test_reconstruction_invariants(orc, cfg):
    rc, mask, sph, eps, trials = orc.reconstruct(cfg.seed, cfg.shape, cfg.dx_nm, cfg.mean_nm,
                                                 cfg.sd_nm, cfg.dmin_nm, cfg.dmax_nm, cfg.porosity,
                                                 cfg.xi, cfg.p0, cfg.dist)
    assert rc == 0
    N = mask.size
    # step 3: stop at the first acceptance that reaches the porosity
    assert eps == mask.sum() / N and eps >= cfg.porosity
    before = _union_of_balls(cfg.shape, sph[:-1])
    assert before.sum() / N < cfg.porosity
    # the mask is exactly the union of the accepted balls (periodic in y, z)
    assert np.array_equal(mask.astype(bool), _union_of_balls(cfg.shape, sph))
    # pairwise overlap tolerance, against both spheres' volumes
    nx, ny, nz = cfg.shape
    for i in range(len(sph)):
        for j in range(i):
            d = _min_image_dist(sph[i], sph[j], ny, nz)
            v = _lens_by_quadrature(sph[i][3], sph[j][3], d) if d < sph[i][3] + sph[j][3] else 0.0
            assert v <= cfg.xi * (4 / 3 * math.pi * sph[i][3] ** 3) * (1 + 1e-9)
            assert v <= cfg.xi * (4 / 3 * math.pi * sph[j][3] ** 3) * (1 + 1e-9)
    # diameters within the clip range (Normal) or the uniform range
    dnm = 2 * sph[:, 3] * cfg.dx_nm
    if cfg.dist == 0:
        assert dnm.min() >= cfg.dmin_nm - 1e-12 and dnm.max() <= cfg.dmax_nm + 1e-12
    else:
        assert dnm.min() >= cfg.mean_nm - cfg.sd_nm - 1e-12
        assert dnm.max() <= cfg.mean_nm + cfg.sd_nm + 1e-12
    assert trials >= len(sph)


def test_reconstruction_is_deterministic(orc):
    c = RECON_CASES[0]
    a = orc.reconstruct(c.seed, c.shape, c.dx_nm, c.mean_nm, c.sd_nm, c.dmin_nm, c.dmax_nm,
                        c.porosity, c.xi, c.p0)
    b = orc.reconstruct(c.seed, c.shape, c.dx_nm, c.mean_nm, c.sd_nm, c.dmin_nm, c.dmax_nm,
                        c.porosity, c.xi, c.p0)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    d = orc.reconstruct(c.seed + 1, c.shape, c.dx_nm, c.mean_nm, c.sd_nm, c.dmin_nm, c.dmax_nm,
                        c.porosity, c.xi, c.p0)
    assert not np.array_equal(a[1], d[1])


def test_overlap_required_when_p0_is_one(orc):
    # step 2a: with p0 = 1 every sphere after the first touches an earlier one
    rc, mask, sph, eps, _ = orc.reconstruct(9, (24, 24, 24), 1.0, 6.0, 1.0, 3.0, 9.0, 0.3, 0.3, p0=1.0)
    assert rc == 0
    for i in range(1, len(sph)):
        assert any(_min_image_dist(sph[i], sph[j], 24, 24) < sph[i][3] + sph[j][3] for j in range(i))


def test_no_overlap_when_tolerance_zero(orc):
    rc, mask, sph, eps, _ = orc.reconstruct(4, (24, 24, 24), 1.0, 5.0, 1.0, 3.0, 8.0, 0.15, 0.0, p0=0.0)
    assert rc == 0
    for i in range(len(sph)):
        for j in range(i):
            assert _min_image_dist(sph[i], sph[j], 24, 24) >= sph[i][3] + sph[j][3]


def test_normal_diameter_law(orc):
    # with tolerance 1 and p0 = 0 every trial is accepted, so the diameters
    # are independent draws of Normal(mean, sd) clipped to [dmin, dmax]
    mean, sd = 20.0, 4.0
    rc, mask, sph, eps, trials = orc.reconstruct(21, (64, 64, 64), 1.0, mean, sd, 0.0, 100.0,
                                                 0.999, 1.0, p0=0.0)
    d = 2 * sph[:, 3]
    assert trials == len(sph) and len(d) > 200
    assert abs(d.mean() - mean) < 4 * sd / math.sqrt(len(d))
    assert abs(d.std() - sd) < 0.15 * sd
    # centres uniform over the box
    c = sph[:, :3] / 64.0
    assert abs(c.mean() - 0.5) < 0.05


def test_infeasible_reconstruction_reports(orc):
    rc, mask, sph, eps, trials = orc.reconstruct(2, (16, 16, 16), 1.0, 8.0, 0.5, 7.0, 9.0, 0.8, 0.0,
                                                 p0=0.0, max_trials=20000)
    assert rc == orc.ORC_EINFEASIBLE and trials == 20000 and eps < 0.8
