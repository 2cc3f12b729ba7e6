"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only -- lattices, random displacements,
velocity draws, type assignment, replica sizes -- and none of the method's
arithmetic (no forces, lists or integration).  Everything is NumPy with
``np.random.default_rng(seed)``.

The workloads stand in for the paper's benchmark systems (App. A: an LJ
liquid, "lj/cut", cut-off 2.5 sigma, and an EAM metal, cut-off 4.95 A); the
paper uses synthetic LAMMPS set-ups, not a dataset, so nothing external is
needed.  Sizes, densities, temperatures and seeds are those of the five
workloads this library is measured on:

    0  LJ liquid FP64, 4,000 atoms (10^3 fcc cells), rho 0.8442, T 1.44
    1  LJ liquid mixed, 864,000 atoms (60^3 fcc cells), rc 2.5 and 5.0
    2  EAM fcc metal, 500,000 atoms (50^3 cells), a = 3.615 A, 300 K
    3  binary LJ force matching, 32,768 atoms (16x16x32 fcc), rho 1.2
    4  512 LJ replicas, N_r log-uniform in [500, 20000]
"""
from __future__ import annotations

import math

import numpy as np

# metal units: eV, Angstrom, amu, fs.  a[A/fs^2] = FTM2V_METAL * F[eV/A] / m[amu]
FTM2V_METAL = 9.64853321e-3
KB_METAL = 8.617333262e-5  # eV/K

SEED_BASE = 1000


def fcc_lattice(nx: int, ny: int, nz: int, a: float):
    """Positions of an fcc lattice of nx*ny*nz cubic cells (4 atoms each), box origin 0.

    Atom order: cell-major (x fastest), then the 4 basis sites.  Returns
    (x (N,3) float64, box (3,) float64).  Sites sit at (c + b + 1/4) * a so
    that no atom lies exactly on a box face.
    """
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    x = (cells[:, None, :] + basis[None, :, :] + 0.25).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return np.ascontiguousarray(x), box


def fcc_constant(rho: float) -> float:
    """Cubic fcc lattice constant for number density rho (4 atoms per cell)."""
    return (4.0 / rho) ** (1.0 / 3.0)


def displace(x, box, std: float, seed: int):
    """Gaussian displacement of every coordinate (std per component), wrapped into the box."""
    rng = np.random.default_rng(seed)
    y = x + rng.normal(0.0, std, size=x.shape)
    return np.ascontiguousarray(np.mod(y, box))


def maxwell_boltzmann(n: int, temperature: float, mass_per_atom, seed: int, kb: float = 1.0,
                      ftm2v: float = 1.0):
    """Seeded Maxwell-Boltzmann velocities with zero net momentum, rescaled to exactly T.

    v ~ N(0, kB T ftm2v / m) per component; the mass-weighted mean is
    removed; then v is scaled so that sum m v^2 / (2 ftm2v) = (3N-3) kB T / 2.
    """
    rng = np.random.default_rng(seed)
    m = np.broadcast_to(np.asarray(mass_per_atom, dtype=np.float64), (n,))
    v = rng.normal(size=(n, 3)) * np.sqrt(kb * temperature * ftm2v / m)[:, None]
    p = (m[:, None] * v).sum(axis=0) / m.sum()
    v = v - p[None, :]
    ke = 0.5 * float((m[:, None] * v * v).sum()) / ftm2v
    target = 0.5 * (3 * n - 3) * kb * temperature
    if ke > 0:
        v *= math.sqrt(target / ke)
    return np.ascontiguousarray(v)


def binary_types(n: int, n_b: int, seed: int):
    """Type 0 everywhere except n_b atoms (chosen by a seeded permutation) of type 1."""
    rng = np.random.default_rng(seed)
    t = np.zeros(n, dtype=np.int32)
    t[rng.permutation(n)[:n_b]] = 1
    return t


def replica_sizes(n_rep: int, lo: int, hi: int, seed: int):
    """N_r = round(exp(U[ln lo, ln hi])) for each replica."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_rep))).astype(np.int64)


def fcc_subset(n: int, rho: float, seed: int):
    """n atoms on a cubic box of density rho: take n of the 4 m^3 fcc sites
    (m = ceil((n/4)^(1/3))) of a lattice scaled to the box, chosen at random."""
    L = (n / rho) ** (1.0 / 3.0)
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
    x, _ = fcc_lattice(m, m, m, L / m)
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.permutation(x.shape[0])[:n])
    return np.ascontiguousarray(x[keep]), np.array([L, L, L])


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

def lj_liquid(cells: int, rho: float = 0.8442, temperature: float = 1.44, seed: int = SEED_BASE,
              displacement: float = 0.0):
    """fcc LJ start (sigma = eps = m = 1) with Maxwell-Boltzmann velocities.

    ``displacement`` > 0 adds a Gaussian jitter (std per component) so that
    force/list parity is exercised away from the perfect lattice.
    """
    a = fcc_constant(rho)
    x, box = fcc_lattice(cells, cells, cells, a)
    if displacement > 0:
        x = displace(x, box, displacement, seed + 7)
    v = maxwell_boltzmann(x.shape[0], temperature, 1.0, seed)
    return {"x": x, "v": v, "box": box, "types": np.zeros(x.shape[0], dtype=np.int32), "n_types": 1,
            "eps": np.ones((1, 1)), "sig": np.ones((1, 1)), "mass": np.ones(1), "ftm2v": 1.0}


def config0(displacement: float = 0.0):
    """LJ liquid, 4,000 atoms, FP64, rc 2.5, skin 0.3, dt 0.005, 100 steps."""
    d = lj_liquid(10, seed=SEED_BASE + 0, displacement=displacement)
    d.update(rc=2.5, skin=0.3, dt=0.005, steps=100, name="lj4000_fp64")
    return d


def config1(rc: float = 2.5, cells: int = 60, displacement: float = 0.0):
    """LJ liquid, 864,000 atoms (60^3 cells), mixed precision, rc 2.5 or 5.0, skin 0.3, 1,000 steps."""
    d = lj_liquid(cells, seed=SEED_BASE + 1, displacement=displacement)
    d.update(rc=rc, skin=0.3, dt=0.005, steps=1000, name=f"lj{d['x'].shape[0]}_rc{rc:g}_mixed")
    return d


EAM_PARAMS = (4.95, 1.0, 0.5, -0.2, 0.02)  # rc, A, c0, c1, c2 (eV, A)


def config2(cells: int = 50, displacement: float = 0.0):
    """EAM-FS fcc metal, a = 3.615 A, m = 63.55 amu, 300 K, dt 1 fs, skin 0.5 A, 500 steps."""
    a = 3.615
    x, box = fcc_lattice(cells, cells, cells, a)
    seed = SEED_BASE + 2
    if displacement > 0:
        x = displace(x, box, displacement, seed + 7)
    mass = 63.55
    v = maxwell_boltzmann(x.shape[0], 300.0, mass, seed, kb=KB_METAL, ftm2v=FTM2V_METAL)
    return {"x": x, "v": v, "box": box, "types": np.zeros(x.shape[0], dtype=np.int32), "n_types": 1,
            "mass": np.array([mass]), "ftm2v": FTM2V_METAL, "eam": np.array(EAM_PARAMS),
            "rc": EAM_PARAMS[0], "skin": 0.5, "dt": 1.0, "steps": 500, "name": f"eam{x.shape[0]}_mixed"}


# true per-type-pair parameters of the binary mixture: AA, AB, BB
KA_EPS = (1.0, 1.5, 0.5)
KA_SIG = (1.0, 0.8, 0.88)


def pair_matrix(vals3):
    """(AA, AB, BB) -> symmetric 2x2 matrix."""
    aa, ab, bb = (float(v) for v in vals3)
    return np.array([[aa, ab], [ab, bb]])


def config3(shape=(16, 16, 32), rho: float = 1.2, frac_b: float = 0.2, jitter: float = 0.05):
    """Binary LJ force matching: 32,768 atoms on a 16x16x32-cell fcc box at
    rho 1.2, 6,554 type-B atoms (round(0.2 N)), Gaussian displacement 0.05."""
    seed = SEED_BASE + 3
    a = fcc_constant(rho)
    x, box = fcc_lattice(shape[0], shape[1], shape[2], a)
    n = x.shape[0]
    x = displace(x, box, jitter, seed)
    t = binary_types(n, int(round(frac_b * n)), seed + 1)
    rng = np.random.default_rng(seed + 2)
    start_eps = np.array(KA_EPS) * (1.0 + rng.uniform(-0.1, 0.1, 3))
    start_sig = np.array(KA_SIG) * (1.0 + rng.uniform(-0.1, 0.1, 3))
    return {"x": x, "box": box, "types": t, "n_types": 2, "rc": 2.5, "skin": 0.3,
            "eps_true": np.array(KA_EPS), "sig_true": np.array(KA_SIG),
            "eps0": start_eps, "sig0": start_sig, "mass": np.ones(2), "ftm2v": 1.0,
            "name": f"ka{n}_grad"}


def config4(n_rep: int = 512, lo: int = 500, hi: int = 20000, rho: float = 0.8442, temperature: float = 1.44):
    """Batched LJ replicas with log-uniform sizes; each replica is n of the
    sites of an fcc lattice in a cube of density rho, with MB velocities."""
    seed = SEED_BASE + 4
    sizes = replica_sizes(n_rep, lo, hi, seed)
    reps = []
    for r, n in enumerate(sizes):
        x, box = fcc_subset(int(n), rho, seed * 1000 + r)
        v = maxwell_boltzmann(int(n), temperature, 1.0, seed * 1000 + 500 + r)
        reps.append({"x": x, "v": v, "box": box, "types": np.zeros(int(n), dtype=np.int32)})
    return {"replicas": reps, "sizes": sizes, "rc": 2.5, "skin": 0.3, "dt": 0.005, "steps": 1000,
            "n_types": 1, "eps": np.ones((1, 1)), "sig": np.ones((1, 1)), "mass": np.ones(1), "ftm2v": 1.0,
            "name": f"lj_batch{n_rep}"}
