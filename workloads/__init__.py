"""Seeded synthetic workloads: lattice-gas configurations and uniform streams.

This module holds no arithmetic of the method.  It is the only code shared by
the CUDA path's callers (tests, benchmark, smoke check) and the CPU oracle.

Lattice: an E^3 simple-cubic periodic grid of spacing h = 1 (box edge a = E).
Site s = x + E*(y + E*z) sits at ((x+1/2), (y+1/2), (z+1/2)).  Charges are +1
and -1 in equal numbers (neutral), on distinct sites.

Workloads (the paper's own runs use 1/27 occupancy, 14 hop targets and
off-lattice variants, Sec. 5.3; these synthetic ones follow the benchmark
definitions used throughout this repository):

  small   16^3 sites, 1000 charges, L=3, p=8,  kT=0.1,  100 steps
  medium  64^3 sites, 32768 charges, L=4, p=12, kT=0.05, 1000 steps, recompute every 100
  large   256^3 sites, 1048576 charges, L=6, p=12, kT=0.05, 1000 steps
  batch   64 replicas, edges from {32,48,64,96,128}, occupancy U[0.02,0.15], p=10, 500 steps
  blobs   512^3 sites, 8388608 charges, 70% in 200 Gaussian blobs (sigma 8), L=7, p=10, 200 steps
  tile    128^3 sites, 131072 charges, L=5, p=12: the leaf shape of "large" (8^3 sites and 32
          charges per leaf) on 4096 leaves, for kernel profiles that span several waves
  sec53   the paper's Sec. 5.3 single-node benchmark shape: one charge per 27 sites and 14 hop
          targets (6 faces, 8 body diagonals), L=6, p=12, on 288^3 sites (884,736 charges; the
          paper's 300^3 lattice is not divisible into 32^3 leaves of whole sites)

Every workload uses the 6 face hops except sec53 (key "hops").  Hop k is HOPS[k]: the faces
(+x, -x, +y, -y, +z, -z), then the body diagonals with x fastest.
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    "small": dict(E=16, N=1000, L=3, p=8, kT=0.1, steps=100, seed=1001, recompute_every=0),
    "medium": dict(E=64, N=32768, L=4, p=12, kT=0.05, steps=1000, seed=1002, recompute_every=100),
    "large": dict(E=256, N=1048576, L=6, p=12, kT=0.05, steps=1000, seed=1003, recompute_every=0),
    "blobs": dict(E=512, N=8388608, L=7, p=10, kT=0.05, steps=200, seed=1005, recompute_every=0),
    "tile": dict(E=128, N=131072, L=5, p=12, kT=0.05, steps=100, seed=1007, recompute_every=0),
    "sec53": dict(E=288, N=884736, L=6, p=12, kT=0.05, steps=100, seed=1006, recompute_every=0, hops=14),
}
HOPS = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 1), (-1, 1, 1), (1, -1, 1), (-1, -1, 1), (1, 1, -1), (-1, 1, -1), (1, -1, -1), (-1, -1, -1)]


def lower_half_lattice(E: int, N: int, seed: int):
    """N distinct sites below the plane z = E/2 (grounded-wall systems: the library adds the
    mirror images above it) and N/2 charges of each sign, seeded."""
    rng = np.random.default_rng(seed)
    sites = rng.choice((E ** 3) // 2, N, replace=False).astype(np.int64)  # z < E/2 <=> s < E^3/2
    return sites, neutral_charges(rng, N)


def hop_vectors(nhop: int = 6) -> np.ndarray:
    """The first nhop hop vectors (6: faces; 14: faces and body diagonals), int64 (nhop, 3)."""
    assert nhop in (6, 14)
    return np.array(HOPS[:nhop], dtype=np.int64)


def hop_targets(E: int, sites: np.ndarray, nhop: int = 6) -> np.ndarray:
    """Target site of every hop, (n, nhop), event order j = nhop i + k, periodic."""
    xyz = site_xyz(E, np.asarray(sites, dtype=np.int64))
    t = (xyz[:, None, :] + hop_vectors(nhop)[None, :, :]) % E
    return t[..., 0] + E * (t[..., 1] + E * t[..., 2])
BATCH = dict(replicas=64, edges=(32, 48, 64, 96, 128), occ=(0.02, 0.15), p=10, kT=0.05, steps=500,
             seed=1004, replica_seed0=2000)


def site_xyz(E: int, sites: np.ndarray) -> np.ndarray:
    """Integer lattice coordinates (x, y, z) of linear site indices."""
    s = np.asarray(sites, dtype=np.int64)
    return np.stack([s % E, (s // E) % E, s // (E * E)], axis=-1)


def site_positions(E: int, sites: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Cartesian positions ((x+1/2)h, (y+1/2)h, (z+1/2)h), float64, shape (n, 3)."""
    return (site_xyz(E, sites).astype(np.float64) + 0.5) * h


def neutral_charges(rng: np.random.Generator, n: int) -> np.ndarray:
    if n % 2:
        raise ValueError("neutral +-1 charges need an even count")
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    return rng.permutation(q)


def uniform_lattice(E: int, N: int, seed: int):
    """N distinct uniform-random sites of an E^3 grid and neutral +-1 charges."""
    rng = np.random.default_rng(seed)
    sites = rng.choice(E ** 3, size=N, replace=False).astype(np.int64)
    q = neutral_charges(rng, N)
    return sites, q


def blob_lattice(E: int, N: int, seed: int, n_blobs: int = 200, sigma: float = 8.0, frac: float = 0.7):
    """70% of charges in Gaussian blobs (offsets N(0, sigma^2) per axis, rounded to a
    site, wrapped; draws landing on an occupied site are redrawn), 30% uniform
    over the remaining empty sites."""
    rng = np.random.default_rng(seed)
    S = E ** 3
    occ = np.zeros(S, dtype=bool)
    n_blob = int(round(frac * N))
    centres = rng.random((n_blobs, 3)) * E
    chosen = []
    need = n_blob
    while need > 0:
        b = rng.integers(0, n_blobs, size=need)
        off = rng.normal(0.0, sigma, size=(need, 3))
        xyz = np.floor(centres[b] + off).astype(np.int64) % E
        s = xyz[:, 0] + E * (xyz[:, 1] + E * xyz[:, 2])
        s = s[~occ[s]]
        s = np.unique(s)  # duplicate draws in one batch: keep one
        s = rng.permutation(s)[:need]
        occ[s] = True
        chosen.append(s)
        need -= len(s)
    n_uni = N - n_blob
    uni = []
    while n_uni > 0:
        s = rng.integers(0, S, size=2 * n_uni)
        s = np.unique(s[~occ[s]])
        s = rng.permutation(s)[:n_uni]
        occ[s] = True
        uni.append(s)
        n_uni -= len(s)
    sites = rng.permutation(np.concatenate(chosen + uni)).astype(np.int64)
    q = neutral_charges(rng, N)
    return sites, q


def workload(name: str):
    """(params, sites, charges) for a named workload."""
    w = dict(WORKLOADS[name])
    if name == "blobs":
        sites, q = blob_lattice(w["E"], w["N"], w["seed"])
    else:
        sites, q = uniform_lattice(w["E"], w["N"], w["seed"])
    return w, sites, q


def uniforms(steps: int, seed: int) -> np.ndarray:
    """(zeta, xi) pairs for each step, in (0, 1]: u[2s] = zeta_s, u[2s+1] = xi_s."""
    rng = np.random.default_rng(seed + 500_000)
    return (1.0 - rng.random(2 * steps)).reshape(steps, 2)


def batch_replicas(n: int | None = None, first: int = 0):
    """Replica list for the batched workload: dicts with E, N, sites, q, seed.
    Replicas first .. first + n - 1; the first 64 draw their edge and occupancy
    from one stream (seed 1004), later ones from a stream of their own."""
    B = BATCH
    n = B["replicas"] if n is None else n
    rng = np.random.default_rng(B["seed"])
    edges = rng.choice(np.array(B["edges"]), size=B["replicas"])
    occs = rng.uniform(B["occ"][0], B["occ"][1], size=B["replicas"])
    out = []
    for r in range(first, first + n):
        if r < B["replicas"]:
            E, occ = int(edges[r]), float(occs[r])
        else:
            rr = np.random.default_rng(B["seed"] + 1 + r)
            E, occ = int(rr.choice(np.array(B["edges"]))), float(rr.uniform(B["occ"][0], B["occ"][1]))
        N = int(round(occ * E ** 3 / 2)) * 2
        sites, q = uniform_lattice(E, N, B["replica_seed0"] + r)
        out.append(dict(E=E, N=N, sites=sites, q=q, seed=B["replica_seed0"] + r, occupancy=N / E ** 3))
    return out


def random_small(E: int, N: int, seed: int):
    """Small uniform lattice system for unit tests."""
    return uniform_lattice(E, N, seed)


# Error study of Sec. 5.1: an almost regular cubic arrangement at a density of
# 0.01 charges per unit volume, small random perturbations, proposals that add
# a further small displacement, and a fresh system every 100 proposals.
ERROR_STUDY = dict(density=0.01, jitter=0.1, step=0.3, moves_per_system=100, seed=1006)


def perturbed_cubic(n_side: int, seed: int, density: float = ERROR_STUDY["density"],
                    jitter: float = ERROR_STUDY["jitter"]):
    """n_side^3 charges on a simple-cubic grid of spacing c = density^(-1/3),
    each moved by a uniform offset in [-jitter c, jitter c]^3, inside the
    periodic box a = n_side c; neutral +-1 charges in random order.
    Returns (positions (N, 3) in [0, a)^3, charges, a, c)."""
    rng = np.random.default_rng(seed)
    c = density ** (-1.0 / 3.0)
    a = n_side * c
    g = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = (g + 0.5) * c + rng.uniform(-jitter * c, jitter * c, size=g.shape)
    pos = np.mod(pos, a)
    q = neutral_charges(rng, len(pos))
    return pos, q, a, c


def small_moves(n: int, c: float, m: int, seed: int, step: float = ERROR_STUDY["step"]):
    """m proposals (particle index, displacement): particles uniform over the n
    charges, displacement components uniform in [-step c, step c]."""
    rng = np.random.default_rng(seed)
    part = rng.integers(0, n, size=m)
    disp = rng.uniform(-step * c, step * c, size=(m, 3))
    return part.astype(np.int32), disp
