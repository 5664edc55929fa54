"""The flop counts behind the bench line's roofline, checked against an
enumeration of the stencil: the method's count per face (the left and right
states at q Gauss points from dot products over the blocky diamond
|a| + |b| <= R, q HLLC fluxes, the Gauss sum) and the executed count of the
parity-sum kernel (sums over the diamond's mirror orbits, one dot product per
pair of Gauss points, butterflies)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def diamond(R):
    return [(a, b) for b in range(-R, R + 1) for a in range(-R, R + 1) if abs(a) + abs(b) <= R]


def mirror_orbits(R):
    """orbits of the diamond under x -> -x and y -> -y"""
    seen, orbits = set(), []
    for a, b in diamond(R):
        if (a, b) in seen:
            continue
        orb = {(sa * a, sb * b) for sa in (1, -1) for sb in (1, -1)}
        seen |= orb
        orbits.append(orb)
    return orbits


def test_method_count_per_face():
    for R in (1, 2, 3):
        N, q = len(diamond(R)), R + 1
        assert N == 2 * R * R + 2 * R + 1
        # 2 states x 4 variables x q points x N FMA (2 flop), q HLLC, Gauss sum
        assert bench.algorithmic_flops_per_face(R) == 2 * (2 * 4 * q * N) + q * 78 + 2 * 4 * q
    assert bench.algorithmic_flops_per_face(3) == 1944


def test_parity_sum_count_matches_the_orbits():
    for R in (1, 2, 3):
        orbits = mirror_orbits(R)
        # an orbit of size s gives s parity components
        assert sum(len(o) for o in orbits) == len(diamond(R))
        # forming them: nothing for the centre, a sum and a difference for a
        # pair, two levels of sums and differences (8 adds) for a quadruple
        adds = sum({1: 0, 2: 2, 4: 8}[len(o)] for o in orbits)
        N, q = len(diamond(R)), R + 1
        pairs, middle = q // 2, q % 2
        dots = 4 * (2 * N * (pairs + middle) + 8 * pairs + 2 * middle)
        split = bench.faces_flops_per_face(R)
        assert split == 4 * adds + dots + q * (78 + 8)


def test_fused_count_is_the_split_count_over_the_owned_faces():
    R = 3
    N, q = len(diamond(R)), R + 1
    sums = 4 * sum({1: 0, 2: 2, 4: 8}[len(o)] for o in mirror_orbits(R))
    dots = 4 * (2 * N * (q // 2) + 8 * (q // 2))
    # a block of 8 x 32 cells forms the sums of all 256 cells, x states on
    # the 7 rows that own x faces (224 cells), y states on all 256, and owns
    # 7 x 31 faces of each direction
    per_face = (256 * sums + (224 + 256) * dots) / (2 * 7 * 31) + q * (78 + 8)
    assert abs(bench.faces_flops_per_face(R, fused=True) - per_face) < 1e-9
    assert round(per_face, 1) == 942.1
