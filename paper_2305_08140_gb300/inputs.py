"""Seeded synthetic inputs for the NEP-ZBL tungsten workloads.

This module is shared by the CUDA path (tests, bench) and by the FP64 oracle.
It holds none of the method's arithmetic: only bcc lattices, random
displacements, random network/descriptor parameters, Maxwell-Boltzmann
velocities and the stored descriptor scaler table (which was written by the
oracle's own script, ``oracle/make_scaler.py``).

Workloads follow the paper's tungsten systems (Sec. II.B, Table I: bcc W,
bulk boxes periodic in x, y, z; foils with open boundaries in z) at the sizes
of the five benchmark configurations:

* ``c1``: 2,000-atom bcc W, 10x10x10 cells, a = 3.165 A (Table III, exp.),
  periodic, Gaussian displacements sigma = 0.05 A (seed 0), 300 K.
* ``c2``: 128,000-atom bcc W, 40x40x40 cells, periodic, 1000 K (seed 2).
* ``c3``: 250,000-atom bcc W, 50x50x50 cells, periodic; 5% of the atoms
  (seed 3) moved into a 20 A sphere at the box centre with a minimum
  separation of 0.3 A (close-pair / load-imbalance stress), 300 K.
* ``c4``: 512 small periodic bcc W boxes of 54/128/250/432 atoms, lattice
  constant scaled by U(0.95, 1.05), displacements sigma = 0.1 A (seed 4).
* ``c5``: 8,192,000-atom bcc W slab, 160x160x160 cells, periodic in x, y,
  open in z with 30 A of vacuum on each side, 300 K (seed 5).

Several species (the multi-species form of the model): ``alloy`` puts a
random solid solution of the listed species on a bcc lattice, ``b2`` the
ordered CsCl arrangement of two species, ``hea`` the equiatomic W-Mo-Ta-Nb
solid solution.  Species data (Z, mass) are the elements' standard values.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

# --- physical constants of the workloads (not of the method) ------------------
A_W = 3.165            # bcc W lattice constant, A (Table III, experiment)
MASS_W = 183.84        # amu
Z_W = 74               # nuclear charge of W (Eq. 2)
KB_EV = 8.617333262e-5  # Boltzmann constant, eV/K
# 1 eV/amu expressed in A^2/fs^2 (CODATA e and u)
EV_PER_AMU_A2_FS2 = 1.602176634e-19 / 1.66053906660e-27 * 1e-10

# Z and standard atomic mass (amu) of the species the multi-species workloads use
SPECIES = {"W": (74, 183.84), "Mo": (42, 95.95), "Ta": (73, 180.94788), "Nb": (41, 92.90637)}

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclass
class Structure:
    """Atoms in an orthorhombic box.

    pos:   (N, 3) float64 positions in A
    box:   (3,) float64 box lengths in A (orthorhombic), or (3, 3) float64 cell
           whose rows are the cell vectors (triclinic); for an open dimension it
           is the extent of the region in which the atoms start
    pbc:   (3,) int32, 1 = periodic, 0 = open
    types: (N,) int32 species index (0 for W)
    vel:   (N, 3) float64 velocities in A/fs, or None
    mass:  mass of species 0 in amu
    """
    pos: np.ndarray
    box: np.ndarray
    pbc: np.ndarray
    types: np.ndarray
    vel: np.ndarray | None = None
    mass: float = MASS_W
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def copy(self) -> "Structure":
        return Structure(self.pos.copy(), self.box.copy(), self.pbc.copy(),
                         self.types.copy(),
                         None if self.vel is None else self.vel.copy(),
                         self.mass, self.name, dict(self.meta))


def bcc(nx: int, ny: int, nz: int, a: float = A_W) -> np.ndarray:
    """bcc positions, cell-major order (ix, iy, iz, basis), (N, 3) float64."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    corner = np.stack([ix, iy, iz], axis=-1).reshape(-1, 3).astype(np.float64)
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    pos = (corner[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos


def maxwell_boltzmann(rng: np.random.Generator, n: int, temperature: float,
                      mass=MASS_W) -> np.ndarray:
    """Velocities (A/fs) from a Maxwell-Boltzmann draw; the centre-of-mass
    velocity is removed and the set is rescaled to exactly ``temperature``
    with 3N - 3 degrees of freedom.  ``mass``: one value (the same draw as
    before per-atom masses existed) or one per atom."""
    if np.ndim(mass) == 0:
        sigma = np.sqrt(KB_EV * temperature / mass * EV_PER_AMU_A2_FS2)
        v = rng.normal(0.0, sigma, size=(n, 3))
        v -= v.mean(axis=0, keepdims=True)
        m = np.full(n, float(mass))
    else:
        m = np.asarray(mass, dtype=np.float64)
        sigma = np.sqrt(KB_EV * temperature / m * EV_PER_AMU_A2_FS2)
        v = rng.normal(0.0, 1.0, size=(n, 3)) * sigma[:, None]
        if n > 0:
            v -= (m[:, None] * v).sum(axis=0, keepdims=True) / m.sum()
    if n > 1 and temperature > 0:
        ke = 0.5 * np.sum(m[:, None] * v * v) / EV_PER_AMU_A2_FS2
        t_now = 2.0 * ke / ((3 * n - 3) * KB_EV)
        v *= np.sqrt(temperature / t_now)
    return v


def _cubic(ncell: int, a: float = A_W) -> Structure:
    pos = bcc(ncell, ncell, ncell, a)
    L = ncell * a
    return Structure(pos, np.array([L, L, L]), np.array([1, 1, 1], np.int32),
                     np.zeros(len(pos), np.int32))


def c1() -> Structure:
    """2,000-atom bcc W, sigma = 0.05 A displacements and 300 K velocities,
    both from one seed-0 generator (displacements drawn first)."""
    s = _cubic(10)
    rng = np.random.default_rng(0)
    s.pos += rng.normal(0.0, 0.05, size=s.pos.shape)
    s.vel = maxwell_boltzmann(rng, s.n, 300.0)
    s.name = "c1_bcc_W_2000"
    return s


def c2() -> Structure:
    """128,000-atom perfect bcc W lattice with 1000 K velocities (seed 2)."""
    s = _cubic(40)
    s.vel = maxwell_boltzmann(np.random.default_rng(2), s.n, 1000.0)
    s.name = "c2_bcc_W_128000"
    return s


def c3(ncell: int = 50, fraction: float = 0.05, radius: float = 20.0,
       min_sep: float = 0.3, temperature: float = 300.0, seed: int = 3) -> Structure:
    """bcc W in which ``fraction`` of the atoms (chosen by ``seed``) are moved to
    uniform random points inside a sphere of ``radius`` at the box centre.
    Each new point is rejected until it is at least ``min_sep`` from every atom
    already in place (unmoved lattice atoms and earlier moved atoms).
    Velocities at ``temperature`` come from the same generator afterwards."""
    s = _cubic(ncell)
    rng = np.random.default_rng(seed)
    n = s.n
    n_move = int(round(fraction * n))
    moved = rng.choice(n, size=n_move, replace=False)
    centre = 0.5 * s.box
    keep = np.ones(n, bool)
    keep[moved] = False
    # unmoved atoms near the sphere, the only ones that can be too close
    near = s.pos[keep][np.linalg.norm(s.pos[keep] - centre, axis=1)
                       < radius + 2 * min_sep]
    placed = np.empty((n_move, 3))
    ms2 = min_sep * min_sep
    for t in range(n_move):
        while True:
            p = rng.uniform(-radius, radius, 3)
            if p @ p > radius * radius:
                continue
            p = p + centre
            d = near - p
            if np.min(np.einsum("ij,ij->i", d, d)) < ms2:
                continue
            if t > 0:
                d = placed[:t] - p
                if np.min(np.einsum("ij,ij->i", d, d)) < ms2:
                    continue
            placed[t] = p
            break
    s.pos[moved] = placed
    s.vel = maxwell_boltzmann(rng, n, temperature)
    s.name = f"c3_bcc_W_{n}_clump"
    s.meta = {"moved": moved}
    return s


def c4(n_configs: int = 512, seed: int = 4) -> list[Structure]:
    """``n_configs`` small periodic bcc W boxes. For each box in turn the
    generator draws the size (3, 4, 5 or 6 cells per side: 54/128/250/432
    atoms), the lattice scale U(0.95, 1.05) and sigma = 0.1 A displacements."""
    rng = np.random.default_rng(seed)
    out = []
    for s_i in range(n_configs):
        nc = int(rng.choice([3, 4, 5, 6]))
        scale = float(rng.uniform(0.95, 1.05))
        s = _cubic(nc, A_W * scale)
        s.pos += rng.normal(0.0, 0.1, size=s.pos.shape)
        s.name = f"c4_{s_i}_{s.n}"
        s.meta = {"scale": scale}
        out.append(s)
    return out


def c5(ncell: int = 160, vacuum: float = 30.0, temperature: float = 300.0,
       seed: int = 5) -> Structure:
    """bcc W slab periodic in x, y and open in z (free surfaces, Sec. II.B),
    with ``vacuum`` A of empty space on each side inside the z extent."""
    pos = bcc(ncell, ncell, ncell)
    L = ncell * A_W
    pos[:, 2] += vacuum
    s = Structure(pos, np.array([L, L, L + 2 * vacuum]),
                  np.array([1, 1, 0], np.int32), np.zeros(len(pos), np.int32))
    s.vel = maxwell_boltzmann(np.random.default_rng(seed), s.n, temperature)
    s.name = f"c5_bcc_W_{s.n}_slab"
    return s


def displaced(s: Structure, sigma: float, seed: int) -> Structure:
    """Copy of ``s`` with Gaussian displacements (for parity cases)."""
    t = s.copy()
    t.pos += np.random.default_rng(seed).normal(0.0, sigma, size=t.pos.shape)
    return t


def alloy(s: Structure, fractions, seed: int) -> Structure:
    """Copy of ``s`` with species drawn per atom: exactly round(f_t N) atoms of
    species t (the last species takes the remainder), placed by a seeded
    permutation."""
    t = s.copy()
    n = t.n
    counts = [int(round(f * n)) for f in fractions[:-1]]
    counts.append(n - sum(counts))
    labels = np.concatenate([np.full(c, k, np.int32) for k, c in enumerate(counts)])
    t.types = labels[np.random.default_rng(seed).permutation(n)].astype(np.int32)
    return t


def b2(ncell: int, a: float = A_W) -> Structure:
    """Ordered CsCl (B2) crystal: species 0 on the cube corners, species 1 on
    the body centres of a periodic ncell^3 bcc lattice."""
    s = _cubic(ncell, a)
    s.types = np.tile(np.array([0, 1], np.int32), s.n // 2)
    return s


def hea(ncell: int = 40, a: float = 3.23, temperature: float = 300.0,
        seed: int = 6) -> Structure:
    """Equiatomic random bcc W-Mo-Ta-Nb (species 0..3), periodic ncell^3
    cells; the seed-6 generator draws the species permutation, then sigma =
    0.05 A displacements, then velocities at ``temperature`` with each atom's
    own mass."""
    s = _cubic(ncell, a)
    rng = np.random.default_rng(seed)
    labels = np.tile(np.arange(4, dtype=np.int32), s.n // 4 + 1)[:s.n]
    s.types = labels[rng.permutation(s.n)].astype(np.int32)
    s.pos += rng.normal(0.0, 0.05, size=s.pos.shape)
    masses = np.array([SPECIES[e][1] for e in ("W", "Mo", "Ta", "Nb")])
    s.vel = maxwell_boltzmann(rng, s.n, temperature, masses[s.types])
    s.name = f"hea_WMoTaNb_{s.n}"
    return s


def triclinic(ncell: int = 7, shear: float = 3.0, sigma: float = 0.05, seed: int = 81,
              pbc=(1, 1, 1)) -> Structure:
    """bcc W in a skewed periodic cell: H = a ncell I plus off-diagonal entries
    drawn from U(-shear, shear) (seed), the crystal's fractional sites mapped
    into it, then sigma displacements (same generator)."""
    rng = np.random.default_rng(seed)
    L = ncell * A_W
    H = np.diag([L] * 3) + rng.uniform(-shear, shear, (3, 3)) * (1 - np.eye(3))
    frac = bcc(ncell, ncell, ncell) / L
    pos = frac @ H + rng.normal(0.0, sigma, size=frac.shape)
    return Structure(pos, H, np.array(pbc, np.int32), np.zeros(len(pos), np.int32),
                     name=f"triclinic_bcc_W_{len(pos)}")


def border_group(s: Structure, width: float = 3 * A_W) -> np.ndarray:
    """uint8 flags of the atoms within ``width`` of a periodic face of the box
    (the thermostatted shell of the cascade runs, Sec. II.B: 3 a0; the free
    surfaces of a foil are not part of it)."""
    d = np.full(s.n, np.inf)
    for a in range(3):
        if s.pbc[a]:
            x = np.mod(s.pos[:, a], s.box[a])
            d = np.minimum(d, np.minimum(x, s.box[a] - x))
    return (d < width).astype(np.uint8)


def small_box(ncell: tuple[int, int, int], a: float = A_W, sigma: float = 0.0,
              seed: int = 0, pbc=(1, 1, 1)) -> Structure:
    """A bcc box of ``ncell`` cells with optional displacements."""
    pos = bcc(*ncell, a)
    s = Structure(pos, np.array(ncell, float) * a, np.array(pbc, np.int32),
                  np.zeros(len(pos), np.int32))
    if sigma > 0:
        s.pos += np.random.default_rng(seed).normal(0.0, sigma, size=pos.shape)
    return s


# --- model hyperparameters and parameters --------------------------------------

@dataclass
class NepModel:
    """NEP-ZBL model. ``params`` is the flat parameter vector in the order
    w0[H x D] (row-major), b0[H], w1[H], b1, cR[T][T][nR x KR],
    cA[T][T][nA x KA] (block (a, b): centre species a, neighbour species b;
    T = number of species); ``scaler`` multiplies the descriptor (length D)."""
    rc_radial: float = 6.0
    rc_angular: float = 4.0
    n_max_radial: int = 4
    n_max_angular: int = 4
    basis_size_radial: int = 8
    basis_size_angular: int = 8
    l_max: int = 4
    use_4body: int = 1
    n_hidden: int = 30
    species: tuple = ("W",)
    zbl_r_inner: float = 1.0
    zbl_r_outer: float = 2.0
    params: np.ndarray | None = None
    scaler: np.ndarray | None = None
    seed: int = 1

    @property
    def n_types(self) -> int:
        return len(self.species)

    @property
    def zs(self) -> list[int]:
        return [SPECIES[e][0] for e in self.species]

    @property
    def masses(self) -> list[float]:
        return [SPECIES[e][1] for e in self.species]

    @property
    def dim(self) -> int:
        nR = self.n_max_radial + 1
        nA = self.n_max_angular + 1
        return nR + nA * self.l_max + (nA if self.use_4body else 0)

    @property
    def n_params(self) -> int:
        D, H = self.dim, self.n_hidden
        nR, nA = self.n_max_radial + 1, self.n_max_angular + 1
        KR, KA = self.basis_size_radial + 1, self.basis_size_angular + 1
        return H * D + H + H + 1 + self.n_types ** 2 * (nR * KR + nA * KA)


def draw_params(model: NepModel, seed: int) -> np.ndarray:
    """All parameters from one ``default_rng(seed).uniform(-0.5, 0.5, P)``."""
    return np.random.default_rng(seed).uniform(-0.5, 0.5, model.n_params)


def random_packing(ncell: int = 4, min_sep: float = 2.2, seed: int = 200) -> Structure:
    """Liquid-like W: 2 ncell^3 atoms placed uniformly at random (rejection
    below ``min_sep`` A, minimum image) in the periodic box of an ncell^3 bcc
    crystal, i.e. at the crystal's density."""
    rng = np.random.default_rng(seed)
    L = ncell * A_W
    n = 2 * ncell ** 3
    pts = np.empty((n, 3))
    t = 0
    while t < n:
        p = rng.uniform(0.0, L, 3)
        d = pts[:t] - p
        d -= L * np.round(d / L)
        if t == 0 or np.min(np.einsum("ij,ij->i", d, d)) >= min_sep * min_sep:
            pts[t] = p
            t += 1
    return Structure(pts, np.array([L, L, L]), np.array([1, 1, 1], np.int32),
                     np.zeros(n, np.int32), name="liquid_like")


def scaler_structures(n_types: int = 1) -> list[Structure]:
    """Structures over which the descriptor scaler is taken, one of each kind
    the paper's W training set contains (Sec. III.A: bulk bcc, strongly
    disordered and liquid structures, short interatomic distances): the c1
    crystal, a hot crystal (sigma = 0.3 A), a liquid-like random packing and a
    crystal compressed to 0.9 a.  For several species each structure becomes an
    equiatomic random solid solution (seeds 210, 211, ...)."""
    out = [c1(), small_box((6, 6, 6), sigma=0.3, seed=201), random_packing(),
           small_box((6, 6, 6), a=0.9 * A_W, sigma=0.1, seed=202)]
    if n_types > 1:
        out = [alloy(s, [1.0 / n_types] * n_types, 210 + k) for k, s in enumerate(out)]
    return out


def scaler_key(seed: int, species=("W",)) -> str:
    """Key of a model's scaler in the stored table."""
    return str(seed) if tuple(species) == ("W",) else f"{seed}:{'-'.join(species)}"


def stored_scaler(seed: int, species=("W",)) -> np.ndarray:
    """Descriptor scaler for the parameter set ``seed``: s_nu = 1 / max |q_nu^i|
    over all atoms i of ``scaler_structures()``, as written by the oracle's
    scaler script."""
    with open(os.path.join(_DATA, "q_scaler.json")) as f:
        table = json.load(f)
    return np.array(table["scalers"][scaler_key(seed, species)], dtype=np.float64)


def nep_model(seed: int = 1, with_scaler: bool = True, species=("W",)) -> NepModel:
    """The random-init model: r_c 6/4 A, n_max 4/4, basis 8, l_max 4 with the
    4-body term, 30 hidden neurons, ZBL switch 1.0/2.0 A; W alone unless
    ``species`` lists several."""
    m = NepModel(seed=seed, species=tuple(species))
    m.params = draw_params(m, seed)
    m.scaler = stored_scaler(seed, species) if with_scaler else np.ones(m.dim)
    return m
