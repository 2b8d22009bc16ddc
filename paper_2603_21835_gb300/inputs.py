"""Seeded synthetic inputs for NAO uniform-grid integration.

This module only *generates inputs*: crystal geometry, radial tables sampled
from a closed-form radial shape, a periodic local potential V on the grid and a
density matrix D.  It holds none of the integration arithmetic (no orbital
evaluation, no contraction), so both the FP64 oracle and the CUDA path can take
their inputs from here without sharing any of the method.

Draw order for one seeded system (``numpy.random.default_rng(seed)``):
  1. V: 20 Gaussian centres (fractional, 20x3), widths sigma~U[1,3] (20),
     amplitudes A~N(0, 0.5) (20, 0.5 is the standard deviation);
  2. D: coefficient matrix C~N(0,1)*scale of shape (norb, nbands), D = C C^T,
     then (D + D^T)/2;
  3. atomic displacements ~N(0, sigma_disp) (natoms x 3), wrapped into the cell.

Units are atomic units (Bohr, Hartree).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Diamond basis in fractional coordinates of the cubic 8-atom cell.
DIAMOND_BASIS = np.array(
    [
        [0.0, 0.0, 0.0],
        [0.0, 0.5, 0.5],
        [0.5, 0.0, 0.5],
        [0.5, 0.5, 0.0],
        [0.25, 0.25, 0.25],
        [0.25, 0.75, 0.75],
        [0.75, 0.25, 0.75],
        [0.75, 0.75, 0.25],
    ]
)
SI_A = 10.26  # cubic lattice constant of Si (Bohr)


@dataclasses.dataclass
class Radial:
    """One radial function R_{l,zeta}(r) sampled on uniform knots r_k = k*dr.

    ``f`` holds R (including the r^l factor) and ``df`` its exact derivative.
    ``alpha`` records the Gaussian exponent it was sampled from.
    """

    l: int
    alpha: float
    rc: float
    dr: float
    f: np.ndarray
    df: np.ndarray

    @property
    def npts(self) -> int:
        return int(self.f.shape[0])


@dataclasses.dataclass
class Species:
    name: str
    radials: List[Radial]

    @property
    def norb(self) -> int:
        return sum(2 * r.l + 1 for r in self.radials)

    @property
    def rcut(self) -> float:
        return max(r.rc for r in self.radials)


@dataclasses.dataclass
class System:
    """A periodic system: cell rows a1,a2,a3 (Bohr), Cartesian positions."""

    cell: np.ndarray  # (3,3) rows are lattice vectors
    pos: np.ndarray  # (natoms,3)
    species: np.ndarray  # (natoms,) int32 index into ``sp``
    sp: List[Species]
    grid: Tuple[int, int, int]
    name: str = ""

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def norb(self) -> int:
        return int(sum(self.sp[s].norb for s in self.species))

    def atom_orb_offsets(self) -> np.ndarray:
        n = [self.sp[s].norb for s in self.species]
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def radial_shape(r: np.ndarray, l: int, alpha: float, rc: float) -> Tuple[np.ndarray, np.ndarray]:
    """R(r) = r^l exp(-alpha r^2) (1-(r/rc)^2)^3 for r < rc, 0 beyond; and dR/dr."""
    r = np.asarray(r, dtype=np.float64)
    inside = r < rc
    u = np.where(inside, 1.0 - (r / rc) ** 2, 0.0)
    e = np.exp(-alpha * r * r)
    rl = r**l
    f = np.where(inside, rl * e * u**3, 0.0)
    drl = l * r ** (l - 1) if l > 0 else np.zeros_like(r)
    df = (drl - 2.0 * alpha * r * rl) * e * u**3 + rl * e * 3.0 * u**2 * (-2.0 * r / (rc * rc))
    df = np.where(inside, df, 0.0)
    return f, df


def make_radial(l: int, alpha: float, rc: float, dr: float = 0.01) -> Radial:
    npts = int(round(rc / dr)) + 1
    r = np.arange(npts, dtype=np.float64) * dr
    f, df = radial_shape(r, l, alpha, rc)
    f[-1] = 0.0
    df[-1] = 0.0
    return Radial(l=l, alpha=alpha, rc=rc, dr=dr, f=f, df=df)


ZETA_ALPHA = (0.3, 0.8)


def species_dzp(name: str, rc: float, shells: Sequence[Tuple[int, int]], dr: float = 0.01) -> Species:
    """Species from (l, nzeta) shells; zeta k uses alpha = ZETA_ALPHA[k]."""
    rad = []
    for l, nz in sorted(shells):
        for z in range(nz):
            rad.append(make_radial(l, ZETA_ALPHA[z], rc, dr))
    return Species(name=name, radials=rad)


def si_species(rc: float = 7.0, dr: float = 0.01) -> Species:
    """Si 2s2p1d: 13 orbitals per atom."""
    return species_dzp("Si", rc, [(0, 2), (1, 2), (2, 1)], dr)


def si_projectors(rc: float = 2.5, dr: float = 0.01) -> Species:
    """Nonlocal projectors of Si (one s and one p channel, 4 functions per atom), localised like
    pseudopotential projectors: r^l exp(-6 r^2) (1 - (r/rc)^2)^3 within rc = 2.5 Bohr."""
    return Species(name="Si-proj", radials=[make_radial(0, 6.0, rc, dr), make_radial(1, 6.0, rc, dr)])


def o_species(rc: float = 6.0, dr: float = 0.01) -> Species:
    return species_dzp("O", rc, [(0, 2), (1, 2), (2, 1)], dr)


def h_species(rc: float = 6.0, dr: float = 0.01) -> Species:
    """H 2s1p: 5 orbitals per atom."""
    return species_dzp("H", rc, [(0, 2), (1, 1)], dr)


def si_supercell(n: Tuple[int, int, int], a: float = SI_A) -> Tuple[np.ndarray, np.ndarray]:
    """Diamond Si supercell; cell (i,j,k) outer with k fastest, basis inner."""
    cell = np.diag([a * n[0], a * n[1], a * n[2]]).astype(np.float64)
    frac = []
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                for b in DIAMOND_BASIS:
                    frac.append([(i + b[0]) / n[0], (j + b[1]) / n[1], (k + b[2]) / n[2]])
    pos = np.asarray(frac) @ cell
    return cell, pos


def grid_points(cell: np.ndarray, grid: Tuple[int, int, int]) -> np.ndarray:
    """Cartesian grid points r_ijk = (i/n1)a1+(j/n2)a2+(k/n3)a3, C order (k fastest)."""
    n1, n2, n3 = grid
    f = np.stack(
        np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3, indexing="ij"), axis=-1
    ).reshape(-1, 3)
    return f @ cell


def periodic_gaussians_V(
    cell: np.ndarray, grid: Tuple[int, int, int], centres_frac: np.ndarray, sigma: np.ndarray, amp: np.ndarray,
    nimg: int = 2,
) -> np.ndarray:
    """V(r) = sum_k A_k sum_{R in [-nimg,nimg]^3} exp(-|r - c_k - R|^2 / (2 sigma_k^2)) on the grid.

    For an orthorhombic cell the Gaussian factorises per axis, which makes the
    lattice sum exact per axis; other cells take the direct 3-D image sum.
    Returns a float64 array of shape grid (C order).
    """
    n1, n2, n3 = grid
    V = np.zeros((n1, n2, n3))
    diag = np.allclose(cell, np.diag(np.diag(cell)))
    if diag:
        L = np.diag(cell)
        axes = [np.arange(n) / n * L[d] for d, n in enumerate(grid)]
        for c, s, A in zip(centres_frac, sigma, amp):
            cc = c * L
            fac = []
            for d in range(3):
                x = axes[d][:, None] - cc[d] - np.arange(-nimg, nimg + 1)[None, :] * L[d]
                fac.append(np.exp(-(x * x) / (2 * s * s)).sum(axis=1))
            V += A * fac[0][:, None, None] * fac[1][None, :, None] * fac[2][None, None, :]
        return V
    pts = grid_points(cell, grid)
    rng = np.arange(-nimg, nimg + 1)
    shifts = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) @ cell
    Vf = np.zeros(pts.shape[0])
    for c, s, A in zip(centres_frac, sigma, amp):
        cc = c @ cell
        for R in shifts:
            d = pts - cc - R
            Vf += A * np.exp(-(d * d).sum(1) / (2 * s * s))
    return Vf.reshape(grid)


def draw_V(rng: np.random.Generator, cell: np.ndarray, grid, ngauss: int = 20) -> np.ndarray:
    centres = rng.random((ngauss, 3))
    sigma = rng.uniform(1.0, 3.0, ngauss)
    amp = rng.normal(0.0, 0.5, ngauss)
    return periodic_gaussians_V(cell, grid, centres, sigma, amp)


def draw_C(rng: np.random.Generator, norb: int, nbands: int, scale: float) -> np.ndarray:
    return rng.standard_normal((norb, nbands)) * scale


def density_matrix(C: np.ndarray) -> np.ndarray:
    D = C @ C.T
    return 0.5 * (D + D.T)


def wrap_positions(cell: np.ndarray, pos: np.ndarray) -> np.ndarray:
    frac = pos @ np.linalg.inv(cell)
    frac -= np.floor(frac)
    return frac @ cell


def on_species(system: System, library: Sequence[Species]) -> System:
    """The same system with its atoms' species re-indexed into ``library`` (matched by name).

    Systems that share one species list share the radial-table metadata, which is what lets a
    serving loop run them in one batched launch."""
    idx = {sp.name: k for k, sp in enumerate(library)}
    remap = np.array([idx[sp.name] for sp in system.sp], dtype=np.int32)
    return dataclasses.replace(system, species=remap[system.species].astype(np.int32), sp=list(library))


@dataclasses.dataclass
class Workload:
    system: System
    V: np.ndarray  # grid-shaped float64
    C: Optional[np.ndarray]  # coefficients (norb, nbands) or None
    D: Optional[np.ndarray]  # dense symmetric (norb, norb) or None (large cases build blocks from C)


def si_workload(
    ncell: Tuple[int, int, int], grid: Tuple[int, int, int], seed: int = 0, nbands: Optional[int] = None,
    cscale: float = 0.25, disp_sigma: float = 0.0, dense_D: bool = True, rc: float = 7.0, name: str = "",
) -> Workload:
    sp = si_species(rc)
    cell, pos = si_supercell(ncell)
    nat = pos.shape[0]
    species = np.zeros(nat, dtype=np.int32)
    norb = nat * sp.norb
    if nbands is None:
        nbands = 2 * nat
    rng = np.random.default_rng(seed)
    V = draw_V(rng, cell, grid)
    C = draw_C(rng, norb, nbands, cscale)
    D = density_matrix(C) if dense_D else None
    if disp_sigma > 0:
        pos = wrap_positions(cell, pos + rng.normal(0.0, disp_sigma, pos.shape))
    sysm = System(cell=cell, pos=pos, species=species, sp=[sp], grid=grid, name=name)
    return Workload(system=sysm, V=V, C=C, D=D)


def config_workload(name: str, dense_D: Optional[bool] = None) -> Workload:
    """The synthetic bulk-Si workloads used for parity and benchmarks.

    si8_g48    : diamond Si cubic cell (8 atoms, 104 NAOs), 48^3 grid
    si64_g96   : 2x2x2 supercell (64 atoms, 832 NAOs), 96^3 grid
    si512_g192 : 4x4x4 supercell (512 atoms, 6656 NAOs), 192^3 grid, N(0,0.05) displacements,
                 C 6656x1024 ~ N(0,1)/32
    si64_g96_d : 64 atoms with N(0,0.1) displacements, 96^3 grid (force workload)
    """
    if name == "si8_g48":
        return si_workload((1, 1, 1), (48, 48, 48), name=name, dense_D=True if dense_D is None else dense_D)
    if name == "si64_g96":
        return si_workload((2, 2, 2), (96, 96, 96), name=name, dense_D=True if dense_D is None else dense_D)
    if name == "si512_g192":
        return si_workload((4, 4, 4), (192, 192, 192), nbands=1024, cscale=1.0 / 32, disp_sigma=0.05, name=name,
                           dense_D=False if dense_D is None else dense_D)
    if name == "si64_g96_d":
        return si_workload((2, 2, 2), (96, 96, 96), disp_sigma=0.1, name=name,
                           dense_D=True if dense_D is None else dense_D)
    raise KeyError(name)


# --------------------------------------------------------------------------------------
# Water clusters in vacuum boxes (mixed-size serving requests)
# --------------------------------------------------------------------------------------
OH_BOND = 1.809
HOH_ANGLE = math.radians(104.5)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array(
        [
            [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
            [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
            [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
        ]
    )


def h2o_workload(nmol: int, seed: int, box: float = 30.0, grid: Tuple[int, int, int] = (144, 144, 144),
                 cscale: float = 0.25, dense_D: bool = True) -> Workload:
    """Rigid water molecules placed in a central sphere of a cubic vacuum box."""
    rng = np.random.default_rng(seed)
    sysm = _h2o_system(rng, nmol, box, grid)
    V = draw_V(rng, sysm.cell, grid)
    C = draw_C(rng, sysm.norb, 2 * nmol * 4 // 2, cscale)
    D = density_matrix(C) if dense_D else None
    return Workload(system=sysm, V=V, C=C, D=D)


def _h2o_system(rng: np.random.Generator, nmol: int, box: float, grid: Tuple[int, int, int]) -> System:
    spO, spH = o_species(), h_species()
    Rs = (3.0 * nmol / (4.0 * math.pi * 0.00495)) ** (1.0 / 3.0)
    centre = np.full(3, box / 2)
    Os: List[np.ndarray] = []
    tries = 0
    while len(Os) < nmol:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place water molecules")
        p = rng.uniform(-Rs, Rs, 3)
        if np.linalg.norm(p) > Rs:
            continue
        p = p + centre
        if all(np.linalg.norm(p - q) >= 4.5 for q in Os):
            Os.append(p)
    pos, spec = [], []
    half = HOH_ANGLE / 2
    h1 = OH_BOND * np.array([math.sin(half), 0.0, math.cos(half)])
    h2 = OH_BOND * np.array([-math.sin(half), 0.0, math.cos(half)])
    for o in Os:
        Rm = _random_rotation(rng)
        pos += [o, o + Rm @ h1, o + Rm @ h2]
        spec += [0, 1, 1]
    cell = np.diag([box, box, box]).astype(np.float64)
    pos = np.asarray(pos)
    species = np.asarray(spec, dtype=np.int32)
    return System(cell=cell, pos=pos, species=species, sp=[spO, spH], grid=grid, name=f"h2o{nmol}")


# --------------------------------------------------------------------------------------
# Serving mix: Si supercells of 8-216 atoms (48 grid points per cubic-cell edge) and water
# clusters of 8-64 molecules in 30 Bohr vacuum boxes (144^3), on one species list
# --------------------------------------------------------------------------------------
SERVING_SI_CELLS = tuple((a, b, c) for a in range(1, 4) for b in range(a, 4) for c in range(b, 4))  # n1<=n2<=n3
SERVING_H2O = (8, 16, 32, 64)
OCCUPIED_PAIRS = {"Si": 2.0, "O": 3.0, "H": 0.5}  # valence electron pairs per atom


def serving_library() -> List[Species]:
    return [si_species(), o_species(), h_species()]


def serving_pool(seed: int = 0) -> List[System]:
    """The geometries of the serving mix: the ten Si supercells n1 x n2 x n3 with
    1 <= n1 <= n2 <= n3 <= 3 (N(0, 0.05) Bohr displacements, grid 48 n_i), then the four water
    clusters.  serving_kinds() tells which entries are Si and which are water."""
    lib = serving_library()
    out: List[System] = []
    for k, n in enumerate(SERVING_SI_CELLS):
        cell, pos = si_supercell(n)
        rng = np.random.default_rng(seed + 1000 + k)
        pos = wrap_positions(cell, pos + rng.normal(0.0, 0.05, pos.shape))
        grid = tuple(48 * x for x in n)
        sysm = System(cell=cell, pos=pos, species=np.zeros(pos.shape[0], dtype=np.int32), sp=[lib[0]], grid=grid,
                      name=f"si{pos.shape[0]}")
        out.append(on_species(sysm, lib))
    for nmol in SERVING_H2O:
        sysm = _h2o_system(np.random.default_rng(seed + 2000 + nmol), nmol, 30.0, (144, 144, 144))
        out.append(on_species(sysm, lib))
    return out


def serving_kinds() -> Tuple[List[int], List[int]]:
    """Indices of serving_pool() entries: (Si supercells, water clusters)."""
    ns = len(SERVING_SI_CELLS)
    return list(range(ns)), list(range(ns, ns + len(SERVING_H2O)))


def serving_requests(n: int, seed: int = 1) -> List[int]:
    """Pool indices of n requests: Si or water with probability 1/2 each, then a uniform size."""
    rng = np.random.default_rng(seed)
    si, h2o = serving_kinds()
    return [int(rng.choice(si)) if rng.random() < 0.5 else int(rng.choice(h2o)) for _ in range(n)]


def serving_inputs(system: System, seed: int, cscale: float = 0.25) -> Tuple[np.ndarray, np.ndarray]:
    """One request's inputs: V (20 periodic Gaussians) and coefficients C (norb x occupied pairs)."""
    rng = np.random.default_rng(seed)
    V = draw_V(rng, system.cell, system.grid)
    nb = int(round(sum(OCCUPIED_PAIRS[system.sp[s].name] for s in system.species)))
    C = draw_C(rng, system.norb, max(nb, 1), cscale)
    return V, C
