"""Seeded synthetic RVE inputs: Voronoi seeds, Haar orientations and twin draws.

This module only draws random numbers and turns them into the plain inputs a
polycrystal RVE is described by (seed points, Bunge Euler angles, which grains
carry a twin and about which {111} normal).  It holds none of the solver's or
the constitutive law's arithmetic, so both the CUDA library and the FP64
oracle can be fed from it.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles from the top 53 bits.

Microstructure recipe (paper Section 2 uses a Matern-hardcore Voronoi model; the
synthetic workloads here use uniform seeds):

* seeds s_n uniform in the unit cube, one per grain (Voronoi generators, Sec. 2.1);
* orientations Haar-uniform on SO(3) (Sec. 2.2, "uniform distribution on the
  space of rotations"), drawn directly in Bunge angles: phi1, phi2 uniform on
  [0, 2 pi), cos(Phi) uniform on [-1, 1], which is the Haar measure in that chart;
* twins: each grain is twinned with probability p; its twin normal is one of the
  four crystal {111} plane normals, chosen uniformly; the twin orientation is the
  parent rotated by 180 degrees about that normal.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK64 = (1 << 64) - 1

# The four {111} plane normals of the crystal (same planes as the paper's Table 1).
TWIN_PLANE_NORMALS = np.array(
    [[1.0, 1.0, -1.0], [-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, 1.0]]
) / math.sqrt(3.0)


class SplitMix64:
    """SplitMix64 stream; `uniform()` returns doubles in [0, 1) with 53 random bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)


def _bunge_matrix(e: np.ndarray) -> np.ndarray:
    """Crystal-to-sample rotation Rz(phi1) Rx(Phi) Rz(phi2) for the twin draw only."""
    c1, s1 = math.cos(e[0]), math.sin(e[0])
    c, s = math.cos(e[1]), math.sin(e[1])
    c2, s2 = math.cos(e[2]), math.sin(e[2])
    return np.array([
        [c1 * c2 - s1 * c * s2, -c1 * s2 - s1 * c * c2, s1 * s],
        [s1 * c2 + c1 * c * s2, -s1 * s2 + c1 * c * c2, -c1 * s],
        [s * s2, s * c2, c],
    ])


def _bunge_angles(R: np.ndarray) -> np.ndarray:
    """Inverse of `_bunge_matrix` (Phi in [0, pi], phi1 and phi2 in [0, 2 pi))."""
    Phi = math.acos(max(-1.0, min(1.0, R[2, 2])))
    if abs(math.sin(Phi)) > 1e-12:
        phi1 = math.atan2(R[0, 2], -R[1, 2])
        phi2 = math.atan2(R[2, 0], R[2, 1])
    else:  # gimbal lock: fold everything into phi1
        phi1 = math.atan2(R[1, 0], R[0, 0])
        phi2 = 0.0
    two_pi = 2.0 * math.pi
    return np.array([phi1 % two_pi, Phi, phi2 % two_pi])


@dataclass
class RVEInputs:
    """Everything needed to label voxels and to create an RVE.

    shape      (nz, ny, nx); voxel (i, j, k) has centre ((i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz)
    seeds      (n_parent, 3) float64 in [0, 1): Voronoi generators (x, y, z)
    euler      (2*n_parent, 3) float64 Bunge angles in rad; row p is parent p,
               row n_parent + p the twin domain of parent p (parent's angles if untwinned)
    twinned    (n_parent,) uint8, 1 if parent p is split into parent and twin
    twin_normal(n_parent, 3) float64, unit twin-plane normal in the sample frame
    """

    shape: tuple
    seeds: np.ndarray
    euler: np.ndarray
    twinned: np.ndarray
    twin_normal: np.ndarray

    @property
    def n_parent(self) -> int:
        return self.seeds.shape[0]

    @property
    def n_grains(self) -> int:
        return self.euler.shape[0]


def make_inputs(shape, n_parent: int, p_twin: float, seed: int) -> RVEInputs:
    """Draw one RVE description.

    Draw order (fixed, so any consumer can replay it): 3 seed coordinates per
    grain, then 3 orientation uniforms per grain, then per grain one uniform
    deciding the twin and one choosing the {111} normal.
    """
    if n_parent < 1:
        raise ValueError("need at least one grain")
    rng = SplitMix64(seed)
    seeds = rng.uniforms(3 * n_parent).reshape(n_parent, 3)
    u = rng.uniforms(3 * n_parent).reshape(n_parent, 3)
    euler_parent = np.stack(
        [2.0 * math.pi * u[:, 0], np.arccos(1.0 - 2.0 * u[:, 1]), 2.0 * math.pi * u[:, 2]],
        axis=1,
    )
    twinned = np.zeros(n_parent, dtype=np.uint8)
    twin_normal = np.zeros((n_parent, 3))
    euler = np.concatenate([euler_parent, euler_parent.copy()], axis=0)
    for p in range(n_parent):
        u_twin = rng.uniform()
        u_normal = rng.uniform()
        if u_twin < p_twin:
            twinned[p] = 1
            nc = TWIN_PLANE_NORMALS[min(3, int(u_normal * 4.0))]
            R = _bunge_matrix(euler_parent[p])
            ns = R @ nc
            ns /= np.linalg.norm(ns)
            twin_normal[p] = ns
            half_turn = 2.0 * np.outer(ns, ns) - np.eye(3)
            euler[n_parent + p] = _bunge_angles(half_turn @ R)
    return RVEInputs(tuple(int(s) for s in shape), seeds, euler, twinned, twin_normal)


# Workload recipes used by the tests and the benchmark (material and loading are the
# defaults of the library's material and load setters).
def workload_plain_16():
    """16^3 voxels, 8 untwinned Voronoi grains, FP64 plain method."""
    return make_inputs((16, 16, 16), 8, 0.0, seed=1000 * 0 + 0)


def workload_twinned_128():
    """128^3 voxels, 200 grains, each twinned with probability 0.5 (FP32 fields)."""
    return make_inputs((128, 128, 128), 200, 0.5, seed=1000 * 1 + 0)


ENSEMBLE_SIZES = (64, 96, 128, 160)
ENSEMBLE_GRAINS = (50, 125, 241, 400)  # 50 at 64^3 to 400 at 160^3 (see workload_ensemble)


def workload_ensemble():
    """16 realizations: 4 each of 64^3, 96^3, 128^3 and 160^3 voxels; the first two of each
    size twinned (p_twin 0.5), the other two untwinned; grain counts 50, 125, 241, 400,
    i.e. n = 50 (V / 64^3)^(ln 8 / ln 15.625), the power law through (64^3, 50) and
    (160^3, 400); realization r (0..15) draws with seed 3000 + r."""
    out = []
    r = 0
    for n, g in zip(ENSEMBLE_SIZES, ENSEMBLE_GRAINS):
        for j in range(4):
            out.append(make_inputs((n, n, n), g, 0.5 if j < 2 else 0.0, seed=1000 * 3 + r))
            r += 1
    return out


def workload_twinned_256():
    """256^3 voxels, 1000 grains, each twinned with probability 0.5 (precision study)."""
    return make_inputs((256, 256, 256), 1000, 0.5, seed=1000 * 2 + 0)


# ---------------------------------------------------------------------------------
# The paper's own microstructure model (Sec. 2): Matern-hardcore Voronoi tessellation,
# neighbouring twins and inclusion twins.  Geometry and random draws only.
# ---------------------------------------------------------------------------------
TWIN_MISORIENTATION_DEG = 69.79  # the misorientation angle printed in Sec. 2.2
# habit planes of the tetragonal lattice read with c/a = 1, each with the in-plane axis the
# twin rotation turns about: (011) with [100], (101) with [010]
HABIT_NORMALS = np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0]]) / math.sqrt(2.0)
HABIT_AXES = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


def poisson(rng: SplitMix64, mean: float) -> int:
    """Poisson draw as the number of unit-rate exponential arrivals before `mean`."""
    t = 0.0
    k = 0
    while True:
        t -= math.log(1.0 - rng.uniform())
        if t > mean:
            return k
        k += 1


def matern_hardcore_seeds(rng: SplitMix64, n_expected: float, r_hard: float) -> np.ndarray:
    """Matern hard-core process of type II on the periodic unit cube (Sec. 2.1): a Poisson
    process with marks, a point removed when another point within distance r_hard has a
    smaller mark.  The parent intensity l_p solves (1 - exp(-l_p v)) / v = n_expected,
    v = 4/3 pi r_hard^3, so the thinned pattern has n_expected points on average.
    Returns (n, 3) points in [0, 1)^3; every periodic pairwise distance is >= r_hard."""
    v = 4.0 / 3.0 * math.pi * r_hard ** 3
    if n_expected * v >= 1.0:
        raise ValueError("intensity too high for this hard-core radius")
    lam_p = -math.log(1.0 - n_expected * v) / v if v > 0 else n_expected
    n_p = poisson(rng, lam_p)
    pts = rng.uniforms(3 * n_p).reshape(n_p, 3)
    marks = rng.uniforms(n_p)
    keep = np.ones(n_p, dtype=bool)
    for i in range(n_p):
        d = pts - pts[i]
        d -= np.round(d)
        close = np.einsum("ij,ij->i", d, d) < r_hard * r_hard
        close[i] = False
        if np.any(marks[close] < marks[i]):
            keep[i] = False
    return pts[keep]


def _rodrigues(axis: np.ndarray, angle: float) -> np.ndarray:
    a = axis / np.linalg.norm(axis)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def _align(h: np.ndarray, n: np.ndarray) -> np.ndarray:
    """A rotation mapping unit vector h onto unit vector n."""
    c = float(np.dot(h, n))
    ax = np.cross(h, n)
    s = float(np.linalg.norm(ax))
    if s < 1e-15:
        if c > 0:
            return np.eye(3)
        perp = np.cross(h, [1.0, 0.0, 0.0])
        if np.linalg.norm(perp) < 1e-6:
            perp = np.cross(h, [0.0, 1.0, 0.0])
        return _rodrigues(perp, math.pi)
    return _rodrigues(ax, math.atan2(s, c))


def _haar_rotation(rng: SplitMix64) -> np.ndarray:
    u = rng.uniforms(3)
    return _bunge_matrix(np.array([2.0 * math.pi * u[0], math.acos(1.0 - 2.0 * u[1]), 2.0 * math.pi * u[2]]))


def grain_adjacency(gid: np.ndarray):
    """Sorted unique pairs (a, b), a < b, of labels meeting across a voxel face (periodic)."""
    pairs = []
    for ax in range(3):
        a = gid.reshape(-1)
        b = np.roll(gid, -1, axis=ax).reshape(-1)
        m = a != b
        lo = np.minimum(a[m], b[m]).astype(np.int64)
        hi = np.maximum(a[m], b[m]).astype(np.int64)
        pairs.append(lo * (1 << 32) + hi)
    u = np.unique(np.concatenate(pairs)) if pairs else np.zeros(0, dtype=np.int64)
    return np.stack([u >> 32, u & 0xFFFFFFFF], axis=1)


@dataclass
class PaperMicrostructure:
    """gid (nz, ny, nx) uint32 labels; euler (n_grains, 3) Bunge angles (crystal -> sample);
    seeds (n_voronoi, 3); pairs: neighbouring twins (k, l, habit index, habit sign);
    inclusions: rows (parent, child id, habit index, x (3, voxel units), thickness)."""

    gid: np.ndarray
    euler: np.ndarray
    seeds: np.ndarray
    pairs: list
    inclusions: list

    @property
    def n_grains(self) -> int:
        return self.euler.shape[0]


def paper_microstructure(shape, label, n_expected: float = 1920.0, r_hard_vox: float = 5.0, p_neigh: float = 0.0,
                         p_incl: float = 0.0, delta=(0.1, 0.3), seed: int = 0) -> PaperMicrostructure:
    """The paper's stochastic microstructure (Sec. 2.1-2.3) on an (nz, ny, nx) grid.

    `label(inp)` must return the Voronoi label map of an RVEInputs without twins (the GPU
    labeller and the oracle's agree bit for bit).  Steps, in the paper's order:
    1. Matern hard-core seeds: n_expected grains on average, hard-core radius r_hard_vox
       voxels (relative to nx; the window is periodic).
    2. Neighbouring twins: N ~ Poisson(p_neigh N_W / 2), redrawn until N <= N_W / 2; pairs of
       adjacent unassigned grains (k, l) are drawn at random; O_k is Haar-uniform under the
       condition that a habit plane ((011) or (101), chosen at random) lies in the joint
       facet, whose normal is the direction between the two Voronoi seeds; O_l is O_k turned
       by the misorientation angle about [100] or [010] respectively.  Assigned grains are
       not drawn again, so no twin chains form.
    3. The remaining grains get Haar-uniform orientations.
    4. Inclusion twins: each grain, with probability p_incl, gets an inclusion I = the voxels
       of G within a slab of thickness delta ~ U[delta_- ved(G), delta_+ ved(G)] around the
       plane through a random boundary voxel of G parallel to the habit plane that the
       chosen axis ([100] or [010]) fixes; O_I = O_G turned by the misorientation angle
       about that axis; I becomes a new grain.  ved(G) = (6 V / pi)^(1/3) in voxels.
    """
    nz, ny, nx = shape
    rng = SplitMix64(seed)
    seeds = matern_hardcore_seeds(rng, n_expected, r_hard_vox / nx)
    n = seeds.shape[0]
    base = RVEInputs((nz, ny, nx), seeds, np.zeros((2 * n, 3)), np.zeros(n, dtype=np.uint8), np.zeros((n, 3)))
    gid = np.asarray(label(base)).astype(np.uint32).reshape(nz, ny, nx)
    theta = math.radians(TWIN_MISORIENTATION_DEG)
    R = [None] * n
    # 2. neighbouring twins
    adj = grain_adjacency(gid)
    nbrs = [[] for _ in range(n)]
    for a, b in adj:
        nbrs[int(a)].append(int(b))
        nbrs[int(b)].append(int(a))
    n_pairs = poisson(rng, p_neigh * n / 2.0)
    while n_pairs > n // 2:
        n_pairs = poisson(rng, p_neigh * n / 2.0)
    free = np.ones(n, dtype=bool)
    pairs = []
    while len(pairs) < n_pairs:
        cand = [g for g in range(n) if free[g] and any(free[m] for m in nbrs[g])]
        if not cand:
            break
        k = cand[min(len(cand) - 1, int(rng.uniform() * len(cand)))]
        fn = [m for m in nbrs[k] if free[m]]
        l_ = fn[min(len(fn) - 1, int(rng.uniform() * len(fn)))]
        hi = min(1, int(rng.uniform() * 2.0))
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        psi = 2.0 * math.pi * rng.uniform()
        d = seeds[l_] - seeds[k]
        d -= np.round(d)
        nrm = sign * d / np.linalg.norm(d)
        h = HABIT_NORMALS[hi]
        R[k] = _align(h, nrm) @ _rodrigues(h, psi)
        R[l_] = R[k] @ _rodrigues(HABIT_AXES[hi], theta)
        free[k] = free[l_] = False
        pairs.append((k, l_, hi, sign))
    # 3. the remaining grains
    for g in range(n):
        if R[g] is None:
            R[g] = _haar_rotation(rng)
    # 4. inclusion twins
    flat = gid.reshape(-1)
    order = np.argsort(flat, kind="stable")
    starts = np.searchsorted(flat[order], np.arange(n + 1))
    boundary = np.zeros(flat.shape, dtype=bool)
    for ax in range(3):
        boundary |= (gid != np.roll(gid, 1, axis=ax)).reshape(-1)
        boundary |= (gid != np.roll(gid, -1, axis=ax)).reshape(-1)
    inclusions = []
    new_gid = flat.copy()
    dims = np.array([nx, ny, nz], dtype=np.float64)
    for g in range(n):
        if not rng.uniform() < p_incl:
            continue
        ai = min(1, int(rng.uniform() * 2.0))
        vox = order[starts[g]:starts[g + 1]]
        bvox = vox[boundary[vox]]
        u_pt, u_th = rng.uniform(), rng.uniform()
        if bvox.size == 0:
            continue
        xv = int(bvox[min(bvox.size - 1, int(u_pt * bvox.size))])
        x = np.array([xv % nx, (xv // nx) % ny, xv // (nx * ny)], dtype=np.float64)
        ved = (6.0 * vox.size / math.pi) ** (1.0 / 3.0)
        thick = ved * (delta[0] + u_th * (delta[1] - delta[0]))
        nrm = R[g] @ HABIT_NORMALS[ai]
        yv = np.stack([vox % nx, (vox // nx) % ny, vox // (nx * ny)], axis=1).astype(np.float64)
        dd = yv - x
        dd -= dims * np.round(dd / dims)
        inside = np.abs(dd @ nrm) <= 0.5 * thick
        child = len(R)
        new_gid[vox[inside]] = child
        R.append(R[g] @ _rodrigues(HABIT_AXES[ai], theta))
        inclusions.append((g, child, ai, x, thick))
    euler = np.stack([_bunge_angles(r) for r in R])
    return PaperMicrostructure(new_gid.reshape(nz, ny, nx), euler, seeds, pairs, inclusions)
