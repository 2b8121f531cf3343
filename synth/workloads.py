"""Seeded generators for the synthetic TNEP workloads.

Shapes follow the paper's workloads (Sec. III "Computational speed": liquid
water replicated up to ~7e4 atoms; Sec. IV: water, the PTAF- anion and a
12x12x12 BaZrO3 supercell).  The paper's datasets and trained models are not
available, so every input here is synthetic:

* water: molecules on a cubic grid at 1 g/cm^3 with random orientations,
  O-H 0.96 A and H-O-H 104.5 deg, plus Gaussian jitter or a random walk;
* BaZrO3: the cubic perovskite (a = 4.19 A) with Gaussian displacements;
* water clusters: the molecules of a 1 g/cm^3 grid closest to a centre;
* anions: random bonded trees of H/C/N/O/F/S atoms, non-periodic;
* model parameters: i.i.d. N(0, 0.1) in FP32, in the flat layout that the
  C header documents.

Seeds follow 2312005233 + 100 * workload + k.  Positions are float32 in
Angstrom, boxes are orthorhombic edge lengths (0 marks an open axis) and types
are int32.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2312005233
WATER_MOL_PER_A3 = 0.033428  # 1 g/cm^3
OH_BOND = 0.96
HOH_ANGLE_DEG = 104.5

__all__ = [
    "SEED_BASE", "seed_for", "HyperParams", "n_params", "model_params",
    "default_q_scaler", "random_rotation", "random_rotations", "water_molecule_frame",
    "water_box", "water_grid_box", "jitter_frames", "random_walk_frames",
    "bzo_supercell", "thermal_frames", "water_cluster", "anion",
    "poisson_arrivals", "Structure", "StructureBatch", "concat_structures",
    "water_small", "water_bulk", "bzo_perovskite", "population_structures",
    "serving_requests", "snes_update_inputs", "tensor_targets", "tensor_series", "cell_water",
]


def seed_for(workload: int, k: int = 0) -> int:
    return SEED_BASE + 100 * workload + k


# --------------------------------------------------------------------------
# model hyper-parameters and the flat parameter vector
# --------------------------------------------------------------------------
@dataclass
class HyperParams:
    """TNEP model shape.  n = 0..n_max, k = 0..basis, l = 1..l_max."""

    n_types: int = 2
    rank: int = 1
    n_max_R: int = 4
    n_max_A: int = 4
    basis_R: int = 8
    basis_A: int = 8
    l_max: int = 4
    use_4body: int = 1
    n_hidden: int = 30
    per_type_nn: int = 1

    @property
    def dim(self) -> int:
        return (self.n_max_R + 1) + (self.n_max_A + 1) * (self.l_max + (1 if self.use_4body else 0))


def n_params(hp: HyperParams) -> int:
    """Length of the flat parameter vector (layout in include/tnep.h)."""
    n_nets = hp.n_types if hp.per_type_nn else 1
    per_net = hp.n_hidden * hp.dim + 2 * hp.n_hidden + 1
    pairs = hp.n_types * hp.n_types
    c = pairs * ((hp.n_max_R + 1) * (hp.basis_R + 1) + (hp.n_max_A + 1) * (hp.basis_A + 1))
    return n_nets * per_net + c


def model_params(hp: HyperParams, rng: np.random.Generator, scale: float = 0.1) -> np.ndarray:
    return (scale * rng.standard_normal(n_params(hp))).astype(np.float32)


def default_q_scaler(hp: HyperParams) -> np.ndarray:
    """Fixed input scaling so that the hidden layer is not saturated.

    Constants chosen once for water-density inputs with N(0, 0.1) parameters:
    radial components are O(1), angular ones O(0.1), the 4-body term O(0.01).
    """
    nR, nA = hp.n_max_R + 1, hp.n_max_A + 1
    s = [0.5] * nR + [5.0] * (nA * hp.l_max)
    if hp.use_4body:
        s += [100.0] * nA
    return np.asarray(s, dtype=np.float32)


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_molecule_frame() -> np.ndarray:
    """O, H, H in a molecular frame (O at the origin)."""
    half = math.radians(HOH_ANGLE_DEG) / 2
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
        [-OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
    ])


def random_rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """n uniform random rotations [n,3,3] from normalised Gaussian quaternions."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1)[:, None]
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _place_waters(centres: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    mol = water_molecule_frame()
    R = random_rotations(len(centres), rng)
    return (centres[:, None, :] + np.einsum("ka,mba->mkb", mol, R)).reshape(-1, 3)


def water_grid_box(n_side: int, L: float, rng: np.random.Generator):
    """n_side^3 molecules on a cubic grid in a periodic cube of edge L."""
    sp = L / n_side
    g = (np.arange(n_side) + 0.5) * sp
    centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = _place_waters(centres, rng)
    types = np.tile(np.array([0, 1, 1], np.int32), len(centres))
    return pos, types, np.array([L, L, L])


def water_box(n_mol: int, rng: np.random.Generator, L: float | None = None):
    """n_mol molecules at 1 g/cm^3 on randomly chosen sites of a cubic grid."""
    if L is None:
        L = (n_mol / WATER_MOL_PER_A3) ** (1.0 / 3.0)
    n_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    sp = L / n_side
    g = (np.arange(n_side) + 0.5) * sp
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pick = np.sort(rng.choice(len(sites), size=n_mol, replace=False))
    pos = _place_waters(sites[pick], rng)
    types = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    return pos, types, np.array([L, L, L])


def wrap(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    return np.mod(pos, box)


def jitter_frames(base: np.ndarray, box: np.ndarray, n_frames: int, sigma: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Independent Gaussian jitter of every atom in every frame, wrapped."""
    out = np.empty((n_frames,) + base.shape, np.float32)
    for f in range(n_frames):
        out[f] = wrap(base + sigma * rng.standard_normal(base.shape), box)
    return out


def random_walk_frames(base: np.ndarray, box: np.ndarray, n_frames: int, sigma: float,
                       rng: np.random.Generator) -> np.ndarray:
    """Unwrapped Gaussian random walk (sigma per atom per step), wrapped per frame."""
    out = np.empty((n_frames,) + base.shape, np.float32)
    cur = base.astype(np.float64).copy()
    for f in range(n_frames):
        if f:
            cur += sigma * rng.standard_normal(base.shape)
        out[f] = wrap(cur, box)
    return out


def bzo_supercell(n: int = 12, a: float = 4.19):
    """Cubic BaZrO3, types Ba=0, Zr=1, O=2, five atoms per cell."""
    basis = np.array([[0, 0, 0], [.5, .5, .5], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]])
    btypes = np.array([0, 1, 2, 2, 2], np.int32)
    g = np.arange(n)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)
    types = np.tile(btypes, len(cells))
    L = n * a
    return pos, types, np.array([L, L, L])


def thermal_frames(base, box, n_frames, sigma, rng):
    return jitter_frames(base, box, n_frames, sigma, rng)


def water_cluster(n_mol: int, rng: np.random.Generator):
    """Open cluster: the n_mol sites of a 1 g/cm^3 grid closest to its centre."""
    sp = (1.0 / WATER_MOL_PER_A3) ** (1.0 / 3.0)
    n_side = int(math.ceil(n_mol ** (1.0 / 3.0))) + 2
    g = (np.arange(n_side) - (n_side - 1) / 2) * sp
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    d = np.linalg.norm(sites, axis=1) + 1e-9 * np.arange(len(sites))
    pick = sites[np.argsort(d, kind="stable")[:n_mol]]
    pos = _place_waters(pick, rng) + 0.05 * rng.standard_normal((3 * n_mol, 3))
    types = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    return pos, types, np.zeros(3)


ANION_TYPE_P = np.array([0.4, 0.3, 0.1, 0.1, 0.05, 0.05])  # H, C, N, O, F, S


def anion(n_atoms: int, rng: np.random.Generator):
    """Random bonded tree: bonds U(1.0, 1.5) A, no two atoms closer than 0.9 A."""
    pos = [np.zeros(3)]
    while len(pos) < n_atoms:
        parent = pos[rng.integers(len(pos))]
        v = rng.standard_normal(3)
        cand = parent + rng.uniform(1.0, 1.5) * v / np.linalg.norm(v)
        if min(np.linalg.norm(cand - p) for p in pos) >= 0.9:
            pos.append(cand)
    types = rng.choice(6, size=n_atoms, p=ANION_TYPE_P).astype(np.int32)
    return np.asarray(pos), types, np.zeros(3)


def poisson_arrivals(rate: float, n: int, rng: np.random.Generator) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


# --------------------------------------------------------------------------
# structure batches (uneven sizes, open or periodic)
# --------------------------------------------------------------------------
@dataclass
class Structure:
    pos: np.ndarray    # [n,3] float32
    types: np.ndarray  # [n] int32
    box: np.ndarray    # [3] float32, zeros = open


@dataclass
class StructureBatch:
    offsets: np.ndarray  # [S+1] int32
    pos: np.ndarray      # [N,3] float32
    types: np.ndarray    # [N] int32
    box: np.ndarray      # [S,3] float32
    sizes: list = field(default_factory=list)

    @property
    def n_structs(self) -> int:
        return len(self.offsets) - 1


def concat_structures(structs) -> StructureBatch:
    sizes = [len(s.types) for s in structs]
    offsets = np.zeros(len(structs) + 1, np.int32)
    offsets[1:] = np.cumsum(sizes)
    return StructureBatch(
        offsets=offsets,
        pos=np.concatenate([s.pos for s in structs]).astype(np.float32),
        types=np.concatenate([s.types for s in structs]).astype(np.int32),
        box=np.stack([s.box for s in structs]).astype(np.float32),
        sizes=sizes,
    )


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
def water_small(n_frames: int = 100):
    """64 H2O in a 12.42 A cube, jitter 0.05 A per frame (192 atoms)."""
    rng = np.random.default_rng(seed_for(1))
    base, types, box = water_grid_box(4, 12.42, rng)
    frames = jitter_frames(base, box, n_frames, 0.05, rng)
    return frames, types, box.astype(np.float32)


def water_bulk(n_frames: int = 2000, n_side: int = 24, L: float = 74.5, sigma: float = 0.01, seed_k: int = 0):
    """13,824 H2O (41,472 atoms) in a 74.5 A cube, random walk 0.01 A/step."""
    rng = np.random.default_rng(seed_for(2, seed_k))
    base, types, box = water_grid_box(n_side, L, rng)
    frames = random_walk_frames(base, box, n_frames, sigma, rng)
    return frames, types, box.astype(np.float32)


def bzo_perovskite(n_frames: int = 500, n: int = 12):
    """12x12x12 BaZrO3 (8,640 atoms), Gaussian displacements 0.08 A."""
    rng = np.random.default_rng(seed_for(3))
    base, types, box = bzo_supercell(n)
    frames = thermal_frames(base, box, n_frames, 0.08, rng)
    return frames, types, box.astype(np.float32)


def population_structures(n_clusters: int = 300, n_boxes: int = 300, seed_k: int = 0):
    """Open water clusters (1-100 molecules) and periodic boxes of 64-512 H2O."""
    rng = np.random.default_rng(seed_for(4, seed_k))
    out = []
    for _ in range(n_clusters):
        p, t, b = water_cluster(int(rng.integers(1, 101)), rng)
        out.append(Structure(p.astype(np.float32), t, b.astype(np.float32)))
    box_sizes = {64: 12.42, 128: 15.65, 256: 19.72, 512: 24.84}
    keys = list(box_sizes)
    for _ in range(n_boxes):
        nm = keys[int(rng.integers(len(keys)))]
        p, t, b = water_box(nm, rng, L=box_sizes[nm])
        p = wrap(p + 0.05 * rng.standard_normal(p.shape), b)
        out.append(Structure(p.astype(np.float32), t, b.astype(np.float32)))
    return out


def serving_requests(n: int, rng: np.random.Generator, max_mol: int = 8000):
    """50/50 mix of open anions (20-60 atoms, types 0-5) and periodic water
    frames of log-uniform(64, max_mol) molecules (water types: O=3, H=0)."""
    out = []
    for _ in range(n):
        if rng.random() < 0.5:
            p, t, b = anion(int(rng.integers(20, 61)), rng)
        else:
            nm = int(round(math.exp(rng.uniform(math.log(64), math.log(max_mol)))))
            p, t, b = water_box(nm, rng)
            p = wrap(p, b)
            t = np.where(t == 0, 3, 0).astype(np.int32)
        out.append(Structure(p.astype(np.float32), t.astype(np.int32), b.astype(np.float32)))
    return out


def tensor_targets(n_structs: int, width: int, rng: np.random.Generator) -> np.ndarray:
    """Reference tensors for training-style runs: N(0, 1) per component."""
    return rng.standard_normal((n_structs, width))


def snes_update_inputs(n_pop: int, dim: int, rng: np.random.Generator, ties: bool = True, nan: bool = False):
    """Inputs of one SNES update: mean, step sizes, samples and losses.  With
    `ties`, some losses repeat exactly; with `nan`, one loss is NaN."""
    mu = rng.standard_normal(dim)
    sigma = rng.uniform(0.05, 0.5, dim)
    s = rng.standard_normal((n_pop, dim))
    loss = rng.uniform(0.5, 2.0, n_pop)
    if ties and n_pop >= 4:
        loss[1] = loss[0]
        loss[n_pop - 1] = loss[2]
    if nan and n_pop >= 3:
        loss[n_pop // 2] = np.nan
    return mu, sigma, s, loss


def tensor_series(n_steps: int, rng: np.random.Generator, n_modes: int = 4, dt_fs: float = 5.0,
                  symmetric: bool = True) -> np.ndarray:
    """A synthetic polarizability / susceptibility trajectory [T][9]: a
    constant tensor plus damped, randomly re-excited oscillators (AR(2)
    processes at 100-900 cm^-1) with random tensor amplitudes, plus white
    noise; symmetric tensors unless asked otherwise."""
    c_cm_fs = 2.99792458e-5
    base = rng.standard_normal((3, 3))
    out = np.zeros((n_steps, 3, 3)) + base
    for _ in range(n_modes):
        w = 2 * np.pi * rng.uniform(100, 900) * c_cm_fs * dt_fs  # rad per step
        r = np.exp(-rng.uniform(0.002, 0.02))
        a1, a2 = 2 * r * np.cos(w), -r * r
        drive = rng.standard_normal(n_steps)
        x = np.zeros(n_steps)
        for t in range(2, n_steps):
            x[t] = a1 * x[t - 1] + a2 * x[t - 2] + drive[t]
        amp = rng.standard_normal((3, 3))
        out += x[:, None, None] * amp * 0.05
    out += 0.01 * rng.standard_normal(out.shape)
    if symmetric:
        out = 0.5 * (out + out.transpose(0, 2, 1))
    return out.reshape(n_steps, 9)


def cell_water(n_mol: int, cell: np.ndarray, rng: np.random.Generator, min_dist: float = 2.6):
    """Water molecules at random positions inside a general cell (rows =
    lattice vectors), oxygens at least min_dist apart under every image;
    returns (pos [3 n_mol][3], types, cell)."""
    H = np.asarray(cell, dtype=np.float64)
    centres = []
    tries = 0
    while len(centres) < n_mol:
        tries += 1
        if tries > 200000:
            raise RuntimeError("cell too small for the requested molecules")
        c = rng.uniform(0.0, 1.0, 3) @ H
        ok = True
        for o in centres:
            d = (c - o) @ np.linalg.inv(H)
            d -= np.round(d)
            for sh in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).T.reshape(-1, 3):
                if np.linalg.norm((d + sh) @ H) < min_dist:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            centres.append(c)
    pos = _place_waters(np.array(centres), rng)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    return pos, types, H
