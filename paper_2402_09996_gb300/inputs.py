"""Seeded synthetic RVE inputs: Voronoi seeds, Haar orientations and twin draws.

This module only draws random numbers and turns them into the plain inputs a
polycrystal RVE is described by (seed points, Bunge Euler angles, which grains
carry a twin and about which {111} normal).  It holds none of the solver's or
the constitutive law's arithmetic, so both the CUDA library and the FP64
oracle can be fed from it.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles from the top 53 bits.

Microstructure recipe (paper Section 2 uses a Matern-hardcore Voronoi model; the
synthetic workloads here use uniform seeds, as documented in the design doc):

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
