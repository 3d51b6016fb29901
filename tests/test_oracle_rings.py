"""Pins of the oracle's ring statistics (primitive rings of the C bond
graph, 6-ring orientation modulo 60 degrees), from combinatorics and
geometry the paper and the lattice fix:

* perfect graphene: every atom lies on three hexagons, so N/2 six-rings and
  no other ring up to size 8; every hexagon has a vertical C-C bond, so its
  diagonals point at 30, 90 and 150 degrees: orientation 30;
* one Stone-Wales defect turns four hexagons into two pentagons and two
  heptagons;
* a lone regular n-gon is one n-ring; two squares sharing an edge are two
  4-rings (their 6-atom perimeter has the shared edge as a shortcut);
* rotating a flake about z by phi turns every orientation by phi (mod 60);
* a path around a periodic box is not a ring.
"""
import math

import numpy as np
import pytest

from oracle import ctbop_oracle as O
from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")
SCC = P1["pair"]["CC"]["S"]
OPEN = np.array([False] * 3)


def _polygon(n, b=1.42):
    R = b / (2.0 * math.sin(math.pi / n))
    a = 2 * math.pi * np.arange(n) / n
    return np.stack([R * np.cos(a), R * np.sin(a), np.zeros(n)], 1) + 20.0


def test_perfect_graphene():
    s = st.graphene_sheet(200, seed=1, n_stone_wales=0, disp=0.0)
    rl = O.rings(s.x, s.types, s.box, s.pbc, SCC)
    c = O.ring_counts(rl)
    assert c[3] == s.n // 2 and c.sum() == c[3]
    ang = np.array([o for n, _, o in rl if n == 6])
    assert np.allclose(ang, 30.0, atol=1e-9)


def test_stone_wales_defect():
    s = st.graphene_sheet(200, seed=3, n_stone_wales=1, disp=0.0)
    c = O.ring_counts(O.rings(s.x, s.types, s.box, s.pbc, 1.7))
    assert (c[2], c[3], c[4]) == (2, s.n // 2 - 4, 2) and c.sum() == s.n // 2


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_single_polygon(n):
    x = _polygon(n)
    rl = O.rings(x, np.ones(n, int), np.full(3, 40.0), OPEN, 1.6)
    assert [r[0] for r in rl] == [n]
    assert np.allclose(rl[0][1], x.mean(axis=0), atol=1e-12)


def test_two_squares_share_an_edge():
    b = 1.42
    x = np.array([[0, 0, 0], [b, 0, 0], [2 * b, 0, 0], [0, b, 0], [b, b, 0], [2 * b, b, 0]], float) + 20.0
    rl = O.rings(x, np.ones(6, int), np.full(3, 40.0), OPEN, 1.6)
    assert sorted(r[0] for r in rl) == [4, 4]


def test_rotation_turns_orientation():
    xy = st.graphene_flake(150, seed=2, vac_frac=0.0, n_stone_wales=0)
    x = np.concatenate([xy, np.zeros((len(xy), 1))], 1) + 30.0
    t = np.ones(len(x), int)
    a0 = [o for n, _, o in O.rings(x, t, np.full(3, 60.0), OPEN, SCC) if n == 6]
    phi = 17.0
    c, s_ = math.cos(math.radians(phi)), math.sin(math.radians(phi))
    xr = (x - 30.0) @ np.array([[c, s_, 0], [-s_, c, 0], [0, 0, 1]]) + 30.0
    a1 = [o for n, _, o in O.rings(xr, t, np.full(3, 60.0), OPEN, SCC) if n == 6]
    assert len(a0) == len(a1) > 10
    d = (np.array(a1) - np.array(a0) - phi) % 60.0
    assert np.all(np.minimum(d, 60.0 - d) < 1e-9)


def test_path_around_a_periodic_box_is_not_a_ring():
    # a straight C chain across a 4-atom periodic cell: closed in the graph,
    # displaced by one box length
    x = np.array([[0.7 + 1.4 * k, 5.0, 5.0] for k in range(4)])
    rl = O.rings(x, np.ones(4, int), np.array([5.6, 10.0, 10.0]), np.array([True, False, False]), 1.6)
    assert rl == []
    assert O.rings(*(lambda s: (s.x, s.types, s.box, s.pbc))(st.sic_3c(2, 4.36, 0.05, seed=1)), SCC) == []
