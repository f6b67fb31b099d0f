"""Oracle pins for the structure characterisation of Sec. 4.1: 18-neighbour
connected-phase labelling, the 13-direction pore size and the maximal
inscribed sphere pore size.  Pins: exhaustive and random brute force on tiny
masks, and closed forms for slabs and ducts."""
import itertools
import math

import numpy as np
import pytest

import synthetic as S

NB18 = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
        if 1 <= abs(dx) + abs(dy) + abs(dz) <= 2]


def _brute_labels(mask):
    """All-pairs union-find: two pore voxels are joined when their offset,
    wrapped in y and z only, is one of the 18 D3Q19 neighbour offsets."""
    nx, ny, nz = mask.shape
    vox = [v for v in itertools.product(range(nx), range(ny), range(nz)) if mask[v]]
    parent = {v: v for v in vox}

    def find(v):
        while parent[v] != v:
            v = parent[v]
        return v

    for a in vox:
        for b in vox:
            dx = b[0] - a[0]
            ok = False
            for dy in {(b[1] - a[1]) % ny, (b[1] - a[1]) % ny - ny}:
                for dz in {(b[2] - a[2]) % nz, (b[2] - a[2]) % nz - nz}:
                    if (dx, dy, dz) in NB18:
                        ok = True
            if ok:
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[ra] = rb
    comps = {}
    for v in vox:
        comps.setdefault(find(v), []).append(v)
    lab = -np.ones(mask.shape, np.int64)
    tr = np.zeros(mask.shape, np.uint8)
    for members in comps.values():
        canon = min((x * ny + y) * nz + z for x, y, z in members)
        xs = {m[0] for m in members}
        for m in members:
            lab[m] = canon
            tr[m] = 1 if (0 in xs and nx - 1 in xs) else 0
    return lab, tr


def test_label18_exhaustive_3x2x2(orc):
    shape = (3, 2, 2)
    for bits in range(1 << 12):
        m = np.array([(bits >> k) & 1 for k in range(12)], np.uint8).reshape(shape)
        lab, tr, conn = orc.label18(m)
        blab, btr = _brute_labels(m)
        assert np.array_equal(lab, blab), bits
        assert np.array_equal(tr, btr), bits


@pytest.mark.parametrize("seed,shape,p", [(1, (5, 4, 3), 0.4), (2, (4, 5, 5), 0.3), (3, (6, 3, 4), 0.5),
                                          (4, (3, 6, 6), 0.25), (5, (7, 4, 4), 0.35)])
def test_label18_random_bruteforce(orc, seed, shape, p):
    m = S.random_mask(shape, p, seed)
    lab, tr, conn = orc.label18(m)
    blab, btr = _brute_labels(m)
    assert np.array_equal(lab, blab)
    assert np.array_equal(tr, btr)
    npore = int(m.sum())
    assert conn == pytest.approx(btr.sum() / npore if npore else 0.0)


def test_label18_ignores_corner_only_contacts(orc):
    # two voxels touching only at a corner are not 18-neighbours
    m = np.zeros((2, 5, 5), np.uint8)
    m[0, 1, 1] = 1
    m[1, 2, 2] = 1
    lab, tr, _ = orc.label18(m)
    assert lab[0, 1, 1] != lab[1, 2, 2] and tr.sum() == 0
    m[1, 2, 1] = 1  # edge contact (1,1,0) joins them
    lab, tr, _ = orc.label18(m)
    assert lab[0, 1, 1] == lab[1, 2, 2] == lab[1, 2, 1] and tr.sum() == 3


D13 = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1),
       (0, 1, -1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)]


def _duct_chords(nx, a, x, y, z):
    """Closed form for a square duct (pore y, z in 1..a, all x): steps to the
    first non-pore cell along +e and -e are the minimum over axes of the
    distance to that axis' bound; x is bounded by the domain faces."""
    out = []
    for e in D13:
        n = 1
        for s in (1, -1):
            lim = []
            for ax, (c, lo, hi) in enumerate(((x, 0, nx - 1), (y, 1, a), (z, 1, a))):
                d = s * e[ax]
                if d > 0:
                    lim.append(hi - c)
                elif d < 0:
                    lim.append(c - lo)
            n += min(lim)
        out.append(n)
    return out


def test_chord13_square_duct_closed_form(orc):
    nx, a = 7, 5
    m = S.square_duct(nx, a)
    d, cnt = orc.chord13(m, dx_nm=1.5)
    for x in range(nx):
        for y in range(1, a + 1):
            for z in range(1, a + 1):
                exp = _duct_chords(nx, a, x, y, z)
                assert list(cnt[:, x, y, z]) == exp
                sa, sf, sb = sum(exp[:3]), sum(exp[3:9]), sum(exp[9:])
                dd = 1.5 * (sa + math.sqrt(2) * sf + math.sqrt(3) * sb) / 13
                assert d[x, y, z] == pytest.approx(dd, rel=1e-6)
    assert np.all(d[m == 0] == 0) and np.all(cnt[:, m == 0] == 0)


def test_chord13_slab_closed_form(orc):
    # pore slab normal to x, thickness t: every line leaving the y-z plane
    # spans t cells; the in-plane lines wrap and count one full period
    nx, ny, nz, t = 9, 4, 6, 3
    m = np.zeros((nx, ny, nz), np.uint8)
    m[3:3 + t] = 1
    d, cnt = orc.chord13(m)
    lcm = ny * nz // math.gcd(ny, nz)
    exp = [t, ny, nz, t, t, t, t, lcm, lcm, t, t, t, t]
    for v in zip(*np.nonzero(m)):
        assert list(cnt[(slice(None),) + v]) == exp
    dd = (t + ny + nz + math.sqrt(2) * (4 * t + 2 * lcm) + math.sqrt(3) * 4 * t) / 13
    assert np.allclose(d[m == 1], dd, rtol=1e-6)


def _walk_count(m, v, e):
    nx, ny, nz = m.shape
    n = 1
    for s in (1, -1):
        x, y, z = v
        while True:
            x += s * e[0]
            if x < 0 or x >= nx:
                break
            y = (y + s * e[1]) % ny
            z = (z + s * e[2]) % nz
            if (x, y, z) == tuple(v):
                return n  # closed all-pore loop: counted once
            if not m[x, y, z]:
                break
            n += 1
    return n


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_chord13_random_bruteforce(orc, seed):
    m = S.random_mask((5, 4, 6), 0.6, seed)
    d, cnt = orc.chord13(m)
    for v in zip(*np.nonzero(m)):
        for k, e in enumerate(D13):
            assert cnt[(k,) + v] == _walk_count(m, v, e)


def _brute_mis(m):
    nx, ny, nz = m.shape
    P = np.argwhere(m == 1)
    Sd = np.argwhere(m == 0)

    def d2(a, b):
        dx = a[:, None, 0] - b[None, :, 0]
        dy = np.abs(a[:, None, 1] - b[None, :, 1]); dy = np.minimum(dy, ny - dy)
        dz = np.abs(a[:, None, 2] - b[None, :, 2]); dz = np.minimum(dz, nz - dz)
        return dx * dx + dy * dy + dz * dz

    r2 = d2(P, Sd).min(axis=1)
    inball = d2(P, P) < r2[None, :]  # [v, c]
    val = np.where(inball, 2 * np.sqrt(r2)[None, :] - 1, 0).max(axis=1)
    return P, r2, val


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_mis_random_bruteforce(orc, seed):
    m = S.random_mask((6, 5, 7), 0.7, seed)
    rc, d, r2 = orc.mis(m, dx_nm=2.0)
    assert rc == 0
    P, br2, val = _brute_mis(m)
    for k, v in enumerate(map(tuple, P)):
        assert r2[v] == br2[k]
        assert d[v] == np.float32(2.0 * val[k])


def test_mis_slab_closed_form(orc):
    # pore slab of odd thickness t normal to x, solid elsewhere: every slab
    # voxel lies in a ball of diameter t
    for t in (1, 3, 5):
        m = np.zeros((t + 4, 5, 5), np.uint8)
        m[2:2 + t] = 1
        rc, d, r2 = orc.mis(m)
        assert rc == 0
        assert np.all(d[m == 1] == t)


def test_mis_duct_centre_closed_form(orc):
    for W in (3, 5, 7):
        m = S.square_duct(4, W)
        rc, d, _ = orc.mis(m)
        c = (W + 1) // 2
        assert np.all(d[:, c, c] == W)
        assert d.max() == W


def test_mis_rejects_all_pore(orc):
    rc, _, _ = orc.mis(np.ones((3, 3, 3), np.uint8))
    assert rc == orc.ORC_EINVAL
