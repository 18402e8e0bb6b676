"""Seeded synthetic inputs for the two-step Brillouin-zone propagation.

This module is shared by the CPU oracle and the GPU library's tests and
benchmark.  It holds *inputs only*: cell geometry, pseudopotential
parameters, random draws (Kleinman-Bylander energies, SCF start vectors,
random shifts) and run parameters.  It contains none of the method's
arithmetic (no k-point formula, no Hamiltonian, no propagator); each side
implements those itself.

Workloads follow the paper's silicon set-up (Sec. III: a diamond-structure
Si crystal, norm-conserving pseudopotential, LDA, real-space grid) with a
synthetic pseudopotential:
  * cubic cell a = 10.26 bohr, 8 atoms at the diamond sites, 16^3 grid,
    16 doubly occupied bands;
  * v_loc = sum over atoms of -Z erf(r/r_e)/r + C_core exp(-r^2 / 2 sigma^2)
    (Z = 4, r_e = 0.8, C_core = +10 Ha, sigma = 1 bohr: a repulsive core;
    this choice opens a gap of >= 0.07 Ha above band 16 at every sampled
    k, which the fixed-occupation ground state needs);
  * one s and three p Kleinman-Bylander projectors per atom with a Gaussian
    radial part (r_c = 1 bohr), energies E_s, E_p ~ U[0.5, 2] Ha drawn from
    the seed and shared by all atoms.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 2112009

# Unit conversions (Hartree atomic units).
AU_PER_FS = 41.341373335
HARTREE_EV = 27.211386245988

DIAMOND_FRAC = np.array(
    [
        [0.00, 0.00, 0.00],
        [0.00, 0.50, 0.50],
        [0.50, 0.00, 0.50],
        [0.50, 0.50, 0.00],
        [0.25, 0.25, 0.25],
        [0.25, 0.75, 0.75],
        [0.75, 0.25, 0.75],
        [0.75, 0.75, 0.25],
    ],
    dtype=np.float64,
)


@dataclass(frozen=True)
class CellSpec:
    """An orthorhombic cell with its synthetic pseudopotential.

    ``a`` are the three edge lengths (bohr); ``n`` the grid points per axis
    (x = axis 0 is the fastest-varying index of every array, arrays are
    stored [n3][n2][n1]).  ``proj_half`` is the half-width of the projector
    box in grid points: a projector of an atom is non-zero only where the
    minimum-image offset |o_ax| < proj_half along every axis.
    """

    name: str
    a: tuple
    n: tuple
    atom_frac: np.ndarray
    n_bands: int
    e_kb_s: float
    e_kb_p: float
    z_ion: float = 4.0
    r_erf: float = 0.8
    c_core: float = 10.0
    sigma_core: float = 1.0
    r_proj: float = 1.0
    proj_half: float = 8.0
    occ: float = 2.0
    use_projectors: bool = True

    @property
    def n_atoms(self) -> int:
        return int(self.atom_frac.shape[0])

    @property
    def n_pts(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def replace(self, **kw) -> "CellSpec":
        return dataclasses.replace(self, **kw)


def _kb_energies(seed: int) -> tuple[float, float]:
    rng = np.random.default_rng([seed, 1])
    e = rng.uniform(0.5, 2.0, size=2)
    return float(e[0]), float(e[1])


def cell_a(seed: int = MASTER_SEED, **kw) -> CellSpec:
    """8-atom cubic Si-like cell, a = 10.26 bohr, 16^3 grid, 16 bands."""
    es, ep = _kb_energies(seed)
    base = CellSpec(name="A", a=(10.26, 10.26, 10.26), n=(16, 16, 16),
                    atom_frac=DIAMOND_FRAC.copy(), n_bands=16, e_kb_s=es, e_kb_p=ep)
    return base.replace(**kw) if kw else base


def cell_a_coarse(seed: int = MASTER_SEED, n: int = 8, **kw) -> CellSpec:
    """Cell A on a coarser n^3 grid (n a multiple of 8 keeps every atom and
    the bond centre on grid points); the projector box keeps its physical
    half-width a/2."""
    return cell_a(seed, n=(n, n, n), proj_half=n / 2.0, **kw)


def cell_b(seed: int = MASTER_SEED, **kw) -> CellSpec:
    """2x2x2 supercell of cell A: a = 20.52 bohr, 32^3 grid, 64 atoms, 128 bands."""
    es, ep = _kb_energies(seed)
    fr = []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                fr.append((DIAMOND_FRAC + np.array([i, j, k], dtype=np.float64)) / 2.0)
    base = CellSpec(name="B", a=(20.52, 20.52, 20.52), n=(32, 32, 32),
                    atom_frac=np.concatenate(fr, axis=0), n_bands=128, e_kb_s=es, e_kb_p=ep)
    return base.replace(**kw) if kw else base


def cell_tiny(seed: int = MASTER_SEED, n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands: int = 4,
              atoms: str = "pair", **kw) -> CellSpec:
    """Small cells for brute-force and dense-matrix checks.

    ``atoms``: "pair" puts two atoms at (0,0,0) and (1/4,1/4,1/4) (grid
    points when n is a multiple of 4); "none" gives a free-electron cell.
    """
    es, ep = _kb_energies(seed)
    if atoms == "pair":
        fr = np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]])
    elif atoms == "one":
        fr = np.array([[0.0, 0.0, 0.0]])
    elif atoms == "offgrid":
        fr = np.array([[0.1, 0.2, 0.3], [0.55, 0.6, 0.7]])
    else:
        fr = np.zeros((0, 3))
    half = float(min(n)) / 2.0
    base = CellSpec(name="tiny", a=tuple(float(x) for x in a), n=tuple(int(x) for x in n),
                    atom_frac=fr, n_bands=n_bands, e_kb_s=es, e_kb_p=ep,
                    z_ion=2.0 if len(fr) else 0.0, c_core=-1.0 if len(fr) else 0.0,
                    proj_half=half, use_projectors=bool(len(fr)))
    return base.replace(**kw) if kw else base


def free_electron(cell: CellSpec) -> CellSpec:
    """The same grid with no ions: Z = 0, no core term, no projectors."""
    return cell.replace(atom_frac=np.zeros((0, 3)), z_ion=0.0, c_core=0.0, use_projectors=False)


# ----------------------------------------------------------------------------
# Fields
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Kick:
    """Impulsive perturbation of strength k0 along ``direction`` (Eq. 11)."""

    k0: float = 0.005
    direction: tuple = (1.0, 0.0, 0.0)


@dataclass(frozen=True)
class Pulse:
    """Laser vector potential of the HHG run (Eq. 15): peak field e0 (au),
    mean frequency omega0 (Ha), full duration t_pulse (au), polarisation."""

    e0: float = 0.005
    omega0: float = 0.057
    t_pulse: float = 1654.0
    direction: tuple = (0.0, 0.0, 1.0)


# ----------------------------------------------------------------------------
# Runs
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class SubsimSpec:
    """One independent sub-simulation of the two-step scheme.

    ``mp`` is the Monkhorst-Pack subgrid size (N1, N2, N3) and ``shift`` the
    fractional shift (q, p, r) in (0,1)^3 of Eq. 10 (zero for a plain MP grid).
    """

    cell: CellSpec
    mp: tuple
    shift: tuple
    dt: float
    n_steps: int
    field: object


@dataclass
class RunSpec:
    name: str
    subsims: list
    hxc: str = "scf"          # "scf" (self-consistent v_Hxc) or "frozen"
    shift_scheme: str = "none"
    note: str = ""

    @property
    def n_orbitals(self) -> int:
        return int(sum(s.cell.n_bands * s.mp[0] * s.mp[1] * s.mp[2] for s in self.subsims))

    @property
    def orbital_steps(self) -> int:
        return int(sum(s.cell.n_bands * s.mp[0] * s.mp[1] * s.mp[2] * s.n_steps for s in self.subsims))


def lattice_shifts(r: int) -> list:
    """Shift values (2i+1)/(2r), i = 0..r-1, on every axis (x fastest): the
    regular lattice of shifts that tiles an (r*N)^3 grid with r^3 shifted
    N^3 grids, for even r."""
    if r % 2:
        raise ValueError("lattice_shifts needs an even r")
    vals = [(2 * i + 1) / (2.0 * r) for i in range(r)]
    return [(vx, vy, vz) for vz in vals for vy in vals for vx in vals]


def random_shifts(n: int, seed: int) -> list:
    """Uniform random shifts in (0,1)^3 (the paper also allows plain random
    numbers for the second sampling)."""
    rng = np.random.default_rng([seed, 5])
    return [tuple(float(v) for v in row) for row in rng.uniform(0.0, 1.0, size=(n, 3))]


def mp2_kick_run(seed: int = MASTER_SEED, n_steps: int = 100) -> RunSpec:
    """Plain FP64 run: cell A, MP 2^3 (8 k), 16 bands, kick k0=0.005 x,
    dt=0.08, 100 steps."""
    c = cell_a(seed)
    return RunSpec("mp2-kick", [SubsimSpec(c, (2, 2, 2), (0.0, 0.0, 0.0), 0.08, n_steps, Kick())])


def twostep_kick_run(seed: int = MASTER_SEED, n_steps: int = 3000, hxc: str = "scf") -> RunSpec:
    """Two-step linear response: the 16^3 k grid split into 64 shifted 4^3
    subgrids (4096 k), 16 bands, kick 0.005 x, dt=0.08, 3000 steps."""
    c = cell_a(seed)
    subs = [SubsimSpec(c, (4, 4, 4), s, 0.08, n_steps, Kick()) for s in lattice_shifts(4)]
    return RunSpec("twostep-64x4^3-kick", subs, hxc=hxc, shift_scheme="lattice")


def twostep_hhg_run(seed: int = MASTER_SEED, n_steps: int = 41350) -> RunSpec:
    """Two-step HHG: 8 shifted 8^3 subgrids, sin^4 pulse along z,
    omega0=0.057, E0=0.005, T=1654, dt=0.04."""
    c = cell_a(seed)
    subs = [SubsimSpec(c, (8, 8, 8), s, 0.04, n_steps, Pulse()) for s in lattice_shifts(2)]
    return RunSpec("twostep-8x8^3-hhg", subs, shift_scheme="lattice")


def uneven_batch_run(seed: int = MASTER_SEED, n_a: int = 180, n_b: int = 20, max_steps: int | None = None) -> RunSpec:
    """Uneven batch: n_a cell-A and n_b cell-B sub-simulations with seeded
    subgrid sizes 2..6, random shifts, kick amplitudes log-uniform in
    [1e-4, 1e-2] along x and 500..5000 steps."""
    rng = np.random.default_rng([seed, 7])
    ca, cb = cell_a(seed), cell_b(seed)
    kinds = ["A"] * n_a + ["B"] * n_b
    order = rng.permutation(len(kinds))
    shifts = random_shifts(len(kinds), seed)
    subs = []
    for idx in order:
        kind = kinds[idx]
        nk = int(rng.integers(2, 7))
        k0 = float(10.0 ** rng.uniform(-4.0, -2.0))
        steps = int(rng.integers(500, 5001))
        if max_steps is not None:
            steps = min(steps, max_steps)
        subs.append(SubsimSpec(ca if kind == "A" else cb, (nk, nk, nk), shifts[idx], 0.08, steps,
                               Kick(k0=k0)))
    return RunSpec("uneven-batch", subs, shift_scheme="random")


def scf_start_vectors(n_k: int, n_vec: int, n_pts: int, seed: int, tag: int = 0) -> np.ndarray:
    """Seeded random complex start vectors for the ground-state solver,
    shape (n_k, n_vec, n_pts)."""
    rng = np.random.default_rng([seed, 11, tag])
    return rng.standard_normal((n_k, n_vec, n_pts)) + 1j * rng.standard_normal((n_k, n_vec, n_pts))


def random_complex(shape, seed: int, tag: int = 0) -> np.ndarray:
    rng = np.random.default_rng([seed, 13, tag])
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------
# Initial orbitals (inputs of a propagation; no method arithmetic)
# ----------------------------------------------------------------------------
def random_orbitals(n_k: int, n_b: int, n: tuple, dv: float, seed: int, tag: int = 0) -> np.ndarray:
    """Seeded random orbitals, orthonormal per k in the metric dV sum conj(u) v,
    shape (n_k, n_b, n3, n2, n1) complex128."""
    npts = int(n[0] * n[1] * n[2])
    x = random_complex((n_k, npts, n_b), seed, tag)
    out = np.empty((n_k, n_b, npts), dtype=np.complex128)
    for k in range(n_k):
        q, _ = np.linalg.qr(x[k])
        out[k] = q.T / np.sqrt(dv)
    return out.reshape((n_k, n_b, n[2], n[1], n[0]))


def plane_wave_set(n_b: int) -> np.ndarray:
    """The n_b integer triples with the smallest |n|^2 (ties lexicographic)."""
    rng = range(-4, 5)
    cands = sorted(((i * i + j * j + l * l, (i, j, l)) for i in rng for j in rng for l in rng))
    return np.array([c[1] for c in cands[:n_b]], dtype=np.int64)


def plane_wave_orbitals(a: tuple, n: tuple, gints: np.ndarray, n_k: int) -> np.ndarray:
    """u_b(r) = exp(2 pi i g_b . (i/N)) / sqrt(Omega) on the grid, the same for
    every k: shape (n_k, n_b, n3, n2, n1) complex128."""
    i1 = np.arange(n[0]) / n[0]
    i2 = np.arange(n[1]) / n[1]
    i3 = np.arange(n[2]) / n[2]
    z, y, x = np.meshgrid(i3, i2, i1, indexing="ij")
    omega = float(a[0] * a[1] * a[2])
    one = np.stack([np.exp(2j * np.pi * (g[0] * x + g[1] * y + g[2] * z)) for g in gints]) / np.sqrt(omega)
    return np.broadcast_to(one, (n_k,) + one.shape).copy()
