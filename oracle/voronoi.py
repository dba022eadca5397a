"""Brute-force periodic Voronoi labelling and centroid-plane twin split (oracle side).

TEST INFRASTRUCTURE: used only by tests, the smoke check and the benchmark's CPU
baseline leg; it shares no code with the library's labelling kernel.

Sec. 2.1 defines the grain G_n as the set of points not farther from generator s_n
than from any other generator, on a periodic window.  Choices where it is silent:

* voxel (i, j, k) is represented by its centre ((i+1/2)/nx, (j+1/2)/ny,
  (k+1/2)/nz); the squared minimum-image distance is formed in float64 as
  (dx*dx + dy*dy) + dz*dz, every product and sum rounded separately; a tie goes to
  the lowest generator index.  The minimum image folds d into [-1/2, 1/2]:
  d > 1/2 -> d - 1, d < -1/2 -> d + 1.
* twins of the synthetic workloads: a twinned parent p is split by the plane
  through its centroid c_p with normal n_p.  The centroid is taken in voxel units as
  (centre of the voxel holding s_p) + (integer sum of minimum-image voxel offsets
  from that voxel) / count, so it is independent of summation order.  A voxel of p
  goes to the twin (id n_parent + p) when the minimum-image offset (x - c_p), in
  voxel units, has (dx*nx_ + dy*ny_) + dz*nz_ > 0.

Parity: bit-exact by construction; pinned by tests/test_oracle_voronoi.py (known
two- and three-seed partitions, symmetric ties, twin halves of a slab grain).
"""
from __future__ import annotations

import numpy as np


def _fold(d):
    d = np.where(d > 0.5, d - 1.0, d)
    return np.where(d < -0.5, d + 1.0, d)


def voronoi_labels(shape, seeds, voxels=None):
    """Nearest-generator label of each voxel (or of the flat voxel indices `voxels`).

    shape = (nz, ny, nx); seeds (n, 3) in [0, 1) ordered (x, y, z).
    Returns int64 labels, shaped like the grid or like `voxels`.
    """
    nz, ny, nx = shape
    if voxels is None:
        idx = np.arange(nx * ny * nz, dtype=np.int64)
    else:
        idx = np.asarray(voxels, dtype=np.int64).reshape(-1)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    cx = (i.astype(np.float64) + 0.5) / float(nx)
    cy = (j.astype(np.float64) + 0.5) / float(ny)
    cz = (k.astype(np.float64) + 0.5) / float(nz)
    best = np.full(idx.shape, np.inf)
    label = np.zeros(idx.shape, dtype=np.int64)
    for s in range(seeds.shape[0]):
        dx = _fold(cx - seeds[s, 0])
        dy = _fold(cy - seeds[s, 1])
        dz = _fold(cz - seeds[s, 2])
        d2 = (dx * dx + dy * dy) + dz * dz
        closer = d2 < best
        best = np.where(closer, d2, best)
        label = np.where(closer, s, label)
    if voxels is None:
        return label.reshape(shape)
    return label.reshape(np.shape(voxels))


def _wrap_int(d, n):
    """Integer minimum image in [-n/2, n/2)."""
    return (d + n // 2) % n - n // 2


def twin_centroids(labels, seeds, twinned):
    """Centroids (voxel units, x/y/z) of the twinned parents, by integer offset sums."""
    nz, ny, nx = labels.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cent = np.zeros((seeds.shape[0], 3))
    for p in np.nonzero(twinned)[0]:
        mask = labels == p
        cnt = int(mask.sum())
        si = min(int(seeds[p, 0] * nx), nx - 1)
        sj = min(int(seeds[p, 1] * ny), ny - 1)
        sk = min(int(seeds[p, 2] * nz), nz - 1)
        if cnt == 0:
            cent[p] = (si + 0.5, sj + 0.5, sk + 0.5)
            continue
        ox = int(np.sum(_wrap_int(i[mask] - si, nx), dtype=np.int64))
        oy = int(np.sum(_wrap_int(j[mask] - sj, ny), dtype=np.int64))
        oz = int(np.sum(_wrap_int(k[mask] - sk, nz), dtype=np.int64))
        cent[p] = (
            (si + 0.5) + float(ox) / float(cnt),
            (sj + 0.5) + float(oy) / float(cnt),
            (sk + 0.5) + float(oz) / float(cnt),
        )
    return cent


def label_rve(inputs):
    """Grain-ID map (nz, ny, nx) of an `RVEInputs`: Voronoi parents, then twin split."""
    shape = inputs.shape
    nz, ny, nx = shape
    labels = voronoi_labels(shape, inputs.seeds)
    if not np.any(inputs.twinned):
        return labels
    cent = twin_centroids(labels, inputs.seeds, inputs.twinned)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = labels.copy()
    n_parent = inputs.seeds.shape[0]
    for p in np.nonzero(inputs.twinned)[0]:
        mask = labels == p
        if not np.any(mask):
            continue
        c = cent[p]
        nrm = inputs.twin_normal[p]
        dx = (i[mask].astype(np.float64) + 0.5) - c[0]
        dy = (j[mask].astype(np.float64) + 0.5) - c[1]
        dz = (k[mask].astype(np.float64) + 0.5) - c[2]
        dx = np.where(dx >= 0.5 * nx, dx - nx, np.where(dx < -0.5 * nx, dx + nx, dx))
        dy = np.where(dy >= 0.5 * ny, dy - ny, np.where(dy < -0.5 * ny, dy + ny, dy))
        dz = np.where(dz >= 0.5 * nz, dz - nz, np.where(dz < -0.5 * nz, dz + nz, dz))
        side = (dx * nrm[0] + dy * nrm[1]) + dz * nrm[2]
        sub = out[mask]
        sub[side > 0.0] = n_parent + p
        out[mask] = sub
    return out
