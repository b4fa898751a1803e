"""Geometry behind the sector wiring of the enlarged corner (Fig. 1c,d; Fig. 3).

The drawings are not in the paper's text, so the wiring the oracle and the
kernels use is checked here on explicit honeycomb coordinates:

* six 60-degree sectors around a hexagon centre partition the sites;
* each sector is a quadrant of radial dimers (m, n >= 0) on the Bravais
  vectors a1, a2 (60 degrees apart), i.e. an effective square-lattice patch;
* inside a sector, the outer site of dimer (m, n) bonds to the inner sites of
  (m+1, n) and (m, n+1) -- the legs u, l (or w) of the outer-site tensor;
* the inner site's other two legs go to (m-1, n) and (m, n-1), or, on the
  sector's first row/column, cross the boundary ray to the inner site of the
  neighbouring sector's first column/row at the same position -- the open legs
  x, y of the enlarged corner and the outer side of the edge tensor.
"""
import math

import numpy as np

S3 = math.sqrt(3.0)
A1 = np.array([S3 / 2, 1.5])
A2 = np.array([-S3 / 2, 1.5])
Z = np.array([0.0, 1.0])        # radial bond of the sector at 60..120 degrees


def _rot(v, deg):
    t = math.radians(deg)
    c, s = math.cos(t), math.sin(t)
    return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1]])


def _key(p):
    return (round(p[0] * 1e3), round(p[1] * 1e3))


def _honeycomb(R):
    """All sites within radius R of the hexagon centre at the origin, with bonds."""
    sites = {}
    N = int(R) + 3
    for m in range(-N, N + 1):
        for n in range(-N, N + 1):
            base = m * A1 + n * A2
            for p in (Z + base, 2 * Z + base):
                if np.hypot(*p) < R:
                    sites[_key(p)] = p
    # inner-type sites (x, y) have bonds at 90, 210, 330 degrees; outer-type at 270, 30, 150
    bonds = {k: [] for k in sites}
    for k, p in sites.items():
        for ang in (90, 210, 330, 270, 30, 150):
            q = p + _rot(np.array([1.0, 0.0]), ang)
            if _key(q) in sites and k != _key(q):
                bonds[k].append(_key(q))
    return sites, bonds


def _sector_dimers(sector, R):
    """Dimers (m, n) -> (inner, outer) coordinates of sector k (60k .. 60k+60 degrees)."""
    out = {}
    rot = 60 * (sector - 1)
    for m in range(0, int(R) + 2):
        for n in range(0, int(R) + 2):
            inner = _rot(Z + m * A1 + n * A2, rot)
            outer = _rot(2 * Z + m * A1 + n * A2, rot)
            out[(m, n)] = (inner, outer)
    return out


def test_sectors_partition_the_lattice():
    R = 13.7
    sites, bonds = _honeycomb(R)
    owner = {}
    for sec in range(6):
        for (m, n), (inner, outer) in _sector_dimers(sec, R + 4).items():
            for p in (inner, outer):
                if np.hypot(*p) < R:
                    k = _key(p)
                    assert k in sites
                    assert k not in owner, "site claimed by two sectors"
                    owner[k] = (sec, m, n)
                    ang = math.degrees(math.atan2(p[1], p[0])) % 360.0
                    assert 60 * sec < ang < 60 * sec + 60 + 1e-9
    assert set(owner) == set(sites), "every site belongs to exactly one sector"


def test_sector_wiring_matches_the_contraction():
    R = 15.7
    sites, bonds = _honeycomb(R)
    dim = {sec: _sector_dimers(sec, R + 4) for sec in range(6)}
    where = {}
    for sec in range(6):
        for (m, n), (inner, outer) in dim[sec].items():
            where[_key(inner)] = (sec, m, n, "inner")
            where[_key(outer)] = (sec, m, n, "outer")
    checked = 0
    for (m, n), (inner, outer) in dim[1].items():
        if np.hypot(*outer) > R - 3:
            continue
        ki, ko = _key(inner), _key(outer)
        assert ko in bonds[ki] and len(bonds[ki]) == 3 and len(bonds[ko]) == 3
        # outer site: radial bond + inner sites of (m+1, n) and (m, n+1)
        nb_o = {where[q] for q in bonds[ko] if q != ki}
        assert nb_o == {(1, m + 1, n, "inner"), (1, m, n + 1, "inner")}
        # inner site: radial bond + outer sites of (m-1, n), (m, n-1), or a boundary crossing
        nb_i = {where[q] for q in bonds[ki] if q != ko}
        expect = set()
        expect.add((1, m - 1, n, "outer") if m >= 1 else (2, n, 0, "inner"))
        expect.add((1, m, n - 1, "outer") if n >= 1 else (0, 0, m, "inner"))
        assert nb_i == expect
        checked += 1
    assert checked > 20
