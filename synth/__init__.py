"""Seeded synthetic inputs for the M-scheme block Hamiltonian product and its solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the method itself: it only describes model spaces (which
single-particle m-states exist), draws the seeded Gaussian interaction
parameters, places them in dense coefficient arrays, and draws seeded random
blocks of vectors.  Building determinants, applying operators, signs and
eigensolves live elsewhere (the oracle on one side, the CUDA library on the
other).

Conventions (the paper fixes none of them):

* m-states of a species are listed shell by shell in the order the shells are
  given, and inside a shell by ascending 2m.  Bit i of a determinant's bit
  string is m-state i.
* One-body energies are assigned to the shells in the order listed.
* The two-body parameters are drawn with ``numpy.random.default_rng(seed)``
  as standard normals, in the order AA, BB, AB.  Inside each set, the pair
  index I runs over pairs in lexicographic order ((i<j) for like particles,
  (a, b) a-major for the cross-species set) and, for each I, J runs over pairs
  J >= I with the same total 2m.  The drawn value fills V[I,J] and V[J,I], so
  every interaction is symmetric, and storing like-particle pairs only as i<j
  makes it antisymmetric by construction.

The model Hamiltonian is the one of the paper's Sec. II (one-body plus
two-body terms, h(1)_ac c+_a c_c and sum over a<b, c<d of
h(2)_abcd c+_a c+_b c_d c_c), split by species as in App. B.2 (Eq. for the
proton-neutron two-body term as a product of two one-body operators).
"""
from __future__ import annotations

import dataclasses
import json
import os
from typing import Dict, List, Sequence, Tuple

import numpy as np

__all__ = [
    "ModelSpace",
    "make_space",
    "SPACE12_SHELLS",
    "SPACE20_SHELLS",
    "TABLE1_SHELLS",
    "Workload",
    "WORKLOADS",
    "workload",
    "like_pairs",
    "cross_pairs",
    "draw_interaction",
    "Interaction",
    "random_block",
    "splitmix64",
]


# ----------------------------------------------------------------------------
# Model spaces
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class ModelSpace:
    """Single-particle m-states of one species.

    twoj[i], twom[i]: 2j and 2m of m-state i; orbit[i]: index of its shell;
    eps[i]: one-body energy of its shell.
    """

    twoj: Tuple[int, ...]
    twom: Tuple[int, ...]
    orbit: Tuple[int, ...]
    eps: Tuple[float, ...]

    @property
    def n(self) -> int:
        return len(self.twom)


def make_space(shells: Sequence[Tuple[int, float]]) -> ModelSpace:
    """Build a ModelSpace from (2j, energy) shells in the listed order."""
    twoj, twom, orbit, eps = [], [], [], []
    for k, (tj, e) in enumerate(shells):
        for tm in range(-tj, tj + 1, 2):
            twoj.append(tj)
            twom.append(tm)
            orbit.append(k)
            eps.append(float(e))
    return ModelSpace(tuple(twoj), tuple(twom), tuple(orbit), tuple(eps))


# 12 m-states: j = 1/2, 3/2, 5/2 with energies 0, 1, 2 (sd-shell-sized space).
SPACE12_SHELLS = ((1, 0.0), (3, 1.0), (5, 2.0))
# 20 m-states: j = 1/2, 3/2, 5/2, 7/2 with energies 0, 0.5, 1.5, 3.0 (pf-sized).
SPACE20_SHELLS = ((1, 0.0), (3, 0.5), (5, 1.5), (7, 3.0))
# Table I of the paper: d5/2 then s1/2 (8 m-states), used with 3 particles, 2M=1.
TABLE1_SHELLS = ((5, 0.0), (1, 0.0))


# ----------------------------------------------------------------------------
# Interaction parameters
# ----------------------------------------------------------------------------

def like_pairs(space: ModelSpace) -> List[Tuple[int, int]]:
    """All (i, j) with i < j, lexicographic."""
    n = space.n
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def cross_pairs(sa: ModelSpace, sb: ModelSpace) -> List[Tuple[int, int]]:
    """All (a, b), a in species A, b in species B, a-major."""
    return [(a, b) for a in range(sa.n) for b in range(sb.n)]


def _pair_twom(pairs, ma, mb) -> np.ndarray:
    return np.array([ma[x] + mb[y] for (x, y) in pairs], dtype=np.int64)


def _param_slots(pairs, twom_of_pair) -> List[Tuple[int, int]]:
    """(I, J) slots, I <= J with equal pair 2m, I-major then J ascending."""
    slots = []
    npair = len(pairs)
    for I in range(npair):
        for J in range(I, npair):
            if twom_of_pair[I] == twom_of_pair[J]:
                slots.append((I, J))
    return slots


@dataclasses.dataclass
class Interaction:
    """Dense coefficient arrays of one Hamiltonian.

    h1A[a, c], h1B[b, d]: one-body coefficients h(1) of c+_a c_c.
    VAA[a, b, c, d]: h(2) of a+_a a+_b a_d a_c, nonzero only for a<b, c<d.
    VBB likewise for species B.
    VAB[a, b, c, d]: coefficient of a+_a b+_b b_d a_c (a, c in A; b, d in B).
    The parameter vector ``theta`` lists the independent values in the
    canonical order (one-body A, one-body B, AA, BB, AB); ``param_index``
    gives, per parameter, its kind and slot.
    """

    spaceA: ModelSpace
    spaceB: ModelSpace
    h1A: np.ndarray
    h1B: np.ndarray
    VAA: np.ndarray
    VBB: np.ndarray
    VAB: np.ndarray
    theta: np.ndarray
    param_index: List[Tuple[str, Tuple[int, ...]]]


def draw_interaction(sa: ModelSpace, sb: ModelSpace, seed: int,
                     two_body_scale: float = 1.0) -> Interaction:
    """Seeded Gaussian interaction on the two species' spaces.

    One-body: h1 diagonal = shell energies, off-diagonals 0 (they are still
    listed as parameters for m_a = m_c, a < c).  Two-body values are
    N(0,1) * two_body_scale, placed symmetrically.
    """
    rng = np.random.default_rng(seed)
    nA, nB = sa.n, sb.n
    h1A = np.diag(np.array(sa.eps, dtype=np.float64))
    h1B = np.diag(np.array(sb.eps, dtype=np.float64))
    params: List[Tuple[str, Tuple[int, ...]]] = []
    theta: List[float] = []
    for name, sp, h1 in (("h1A", sa, h1A), ("h1B", sb, h1B)):
        for a in range(sp.n):
            for c in range(a, sp.n):
                if sp.twom[a] == sp.twom[c]:
                    params.append((name, (a, c)))
                    theta.append(h1[a, c])

    VAA = np.zeros((nA, nA, nA, nA))
    VBB = np.zeros((nB, nB, nB, nB))
    VAB = np.zeros((nA, nB, nA, nB))

    sets = (
        ("VAA", like_pairs(sa), sa.twom, sa.twom, VAA),
        ("VBB", like_pairs(sb), sb.twom, sb.twom, VBB),
        ("VAB", cross_pairs(sa, sb), sa.twom, sb.twom, VAB),
    )
    for name, pairs, ma, mb, V in sets:
        pm = _pair_twom(pairs, ma, mb)
        slots = _param_slots(pairs, pm)
        vals = rng.standard_normal(len(slots)) * two_body_scale
        for (I, J), x in zip(slots, vals):
            (i, j), (k, l) = pairs[I], pairs[J]
            V[i, j, k, l] = x
            V[k, l, i, j] = x
            params.append((name, (i, j, k, l)))
            theta.append(x)
    return Interaction(sa, sb, h1A, h1B, VAA, VBB, VAB,
                       np.array(theta, dtype=np.float64), params)


def interaction_from_theta(sa: ModelSpace, sb: ModelSpace, theta: np.ndarray,
                           param_index) -> Interaction:
    """Place a parameter vector into dense arrays (inverse of ``theta``)."""
    nA, nB = sa.n, sb.n
    arr = {
        "h1A": np.zeros((nA, nA)), "h1B": np.zeros((nB, nB)),
        "VAA": np.zeros((nA,) * 4), "VBB": np.zeros((nB,) * 4),
        "VAB": np.zeros((nA, nB, nA, nB)),
    }
    for (name, idx), x in zip(param_index, theta):
        A = arr[name]
        if name.startswith("h1"):
            a, c = idx
            A[a, c] = x
            A[c, a] = x
        else:
            i, j, k, l = idx
            A[i, j, k, l] = x
            A[k, l, i, j] = x
    return Interaction(sa, sb, arr["h1A"], arr["h1B"], arr["VAA"], arr["VBB"],
                       arr["VAB"], np.asarray(theta, dtype=np.float64),
                       list(param_index))


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    shells: Tuple[Tuple[int, float], ...]
    nA: int
    nB: int
    twoM: int
    seed: int
    q: int
    nev: int
    max_basis: int
    tol: float
    width_scaled: bool = False


WORKLOADS: Dict[str, Workload] = {
    # 12 m-states, 2+2 particles: the small case, checked against dense eigh.
    "s12_2p2n": Workload("s12_2p2n", SPACE12_SHELLS, 2, 2, 0, 0, 4, 10, 40, 1e-10),
    # 12 m-states, 4+4 particles (D = 28,503), two-body width scaled to 50.
    "s12_4p4n": Workload("s12_4p4n", SPACE12_SHELLS, 4, 4, 0, 1, 8, 100, 256, 1e-10,
                         width_scaled=True),
    # 20 m-states, 4+4 particles (D = 1,963,461).
    "s20_4p4n": Workload("s20_4p4n", SPACE20_SHELLS, 4, 4, 0, 2, 16, 200, 1024, 1e-6),
    # 20 m-states, 5+5 particles (D = 18,600,516).
    "s20_5p5n": Workload("s20_5p5n", SPACE20_SHELLS, 5, 5, 0, 3, 32, 500, 1024, 1e-6),
}

_SCALES_FILE = os.path.join(os.path.dirname(__file__), "scales.json")


def two_body_scale(w: Workload) -> float:
    """Two-body scale factor of a workload (1 unless width-scaled).

    The width-scaled factor is the ratio 50 / (spectral width of the two-body
    part alone); it is an input constant stored in scales.json, which is
    written by the oracle's make_scales script.
    """
    if not w.width_scaled:
        return 1.0
    with open(_SCALES_FILE) as f:
        return float(json.load(f)[w.name])


def workload(name: str):
    """(Workload, spaceA, spaceB, Interaction) for a named workload."""
    w = WORKLOADS[name]
    sp = make_space(w.shells)
    inter = draw_interaction(sp, sp, w.seed, two_body_scale(w))
    return w, sp, sp, inter


# ----------------------------------------------------------------------------
# Random blocks
# ----------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def random_block(D: int, q: int, seed: int, dtype=np.float64) -> np.ndarray:
    """D x q block, entry (i, j) = uniform(-1, 1) from splitmix64(seed*2^32 + i*q + j).

    The top 53 bits of the hash give u in [0, 1); the entry is 2u - 1.
    """
    idx = np.arange(D * q, dtype=np.uint64) + np.uint64((seed & 0xFFFFFFFF) << 32)
    h = splitmix64(idx)
    u = (h >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (2.0 * u - 1.0).reshape(D, q).astype(dtype)
