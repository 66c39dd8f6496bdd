"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benches.

This module only draws random numbers and writes them out: model weights,
lattice geometries and initial velocities.  It holds none of the method's
arithmetic (no switch function, no network evaluation, no tabulation), so the
oracle and the CUDA path can both take their inputs from here without sharing
any computation.

The paper's trained copper and water models, its DFT data and its
equilibrated 192-atom water box are not available; these generators stand in
for them (Sec. 4 describes the paper's systems: FCC copper with lattice
constant 3.634 A, a 192-atom water box, 330 K initial velocities).

Model file format ("DPSEAV01", little endian):
    char[8]  magic = b"DPSEAV01"
    int32    ntypes
    int32    n_emb                 number of embedding layers (3 in the paper)
    int32    emb_w[n_emb]          widths, e.g. 32 64 128; emb_w[k] = 2*emb_w[k-1]
    int32    m_lt                  M^< (first columns of G used in Eq. 2)
    int32    n_fit                 number of hidden fitting layers (3)
    int32    fit_w[n_fit]          e.g. 240 240 240
    int32    pad                   present when the int count is odd (8-byte align)
    float64  arrays, in this order:
      for ti in types, for tj in types (embedding net of the pair ti <- tj):
          W0[emb_w[0]], b0[emb_w[0]]                        (input width 1)
          for k >= 1: Wk[emb_w[k-1]][emb_w[k]], bk[emb_w[k]] (row = input)
      for ti in types (fitting net of centre type ti):
          W1[M*m_lt][fit_w[0]], b1[fit_w[0]]
          for k >= 1: Wk[fit_w[k-1]][fit_w[k]], bk[fit_w[k]]
          w_out[fit_w[-1]], b_out[1]
All weights and biases are drawn i.i.d. from N(0, std^2) with numpy's PCG64
generator, in exactly the order above.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass

import numpy as np

MAGIC = b"DPSEAV01"

# Cu and water masses in amu
MASS_CU = 63.546
MASS_O = 15.999
MASS_H = 1.008
KB_EV_PER_K = 8.617333262e-5
# 1 eV / (A amu) expressed in A / fs^2
ACC_UNIT = 9.648533212e-3


@dataclass
class ModelSpec:
    ntypes: int = 1
    emb_w: tuple = (32, 64, 128)
    m_lt: int = 16
    fit_w: tuple = (240, 240, 240)

    @property
    def M(self) -> int:
        return self.emb_w[-1]

    @property
    def din(self) -> int:
        return self.M * self.m_lt


COPPER_SPEC = ModelSpec(1, (32, 64, 128), 16, (240, 240, 240))
WATER_SPEC = ModelSpec(2, (25, 50, 100), 16, (240, 240, 240))


def model_shapes(spec: ModelSpec):
    """Names and shapes of every array in file order."""
    out = []
    for ti in range(spec.ntypes):
        for tj in range(spec.ntypes):
            prev = 1
            for k, w in enumerate(spec.emb_w):
                out.append((f"emb{ti}{tj}_W{k}", (prev, w) if k else (w,)))
                out.append((f"emb{ti}{tj}_b{k}", (w,)))
                prev = w
    for ti in range(spec.ntypes):
        prev = spec.din
        for k, w in enumerate(spec.fit_w):
            out.append((f"fit{ti}_W{k}", (prev, w)))
            out.append((f"fit{ti}_b{k}", (w,)))
            prev = w
        out.append((f"fit{ti}_wout", (prev,)))
        out.append((f"fit{ti}_bout", (1,)))
    return out


def make_model(spec: ModelSpec, seed: int, std: float = 0.1) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    arrs = {}
    for name, shape in model_shapes(spec):
        arrs[name] = rng.normal(0.0, std, size=shape)
    return arrs


def write_model(path, spec: ModelSpec, arrs: dict) -> None:
    ints = [spec.ntypes, len(spec.emb_w), *spec.emb_w, spec.m_lt,
            len(spec.fit_w), *spec.fit_w]
    if len(ints) % 2:
        ints.append(0)
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack(f"<{len(ints)}i", *ints))
        for name, shape in model_shapes(spec):
            a = np.ascontiguousarray(arrs[name], dtype="<f8")
            assert a.shape == tuple(shape), (name, a.shape, shape)
            f.write(a.tobytes())


def write_seeded_model(path, spec: ModelSpec = COPPER_SPEC, seed: int = 0,
                       std: float = 0.1) -> dict:
    arrs = make_model(spec, seed, std)
    write_model(path, spec, arrs)
    return arrs


# --------------------------------------------------------------------------
# geometries
# --------------------------------------------------------------------------
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5],
                      [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def fcc_copper(ncell, a: float = 3.634, sigma: float = 0.0, seed: int = 1):
    """FCC lattice of nx*ny*nz cubic cells (4 atoms each), orthorhombic box.

    Atoms are ordered cell by cell (x slowest, then y, then z, then basis).
    Gaussian displacements N(0, sigma^2) per component are drawn from the
    seed.  Positions are NOT wrapped back into the box.
    Returns (x [N,3] float64, types [N] int32, box [3,3] float64 row vectors).
    """
    if np.isscalar(ncell):
        ncell = (int(ncell),) * 3
    nx, ny, nz = (int(c) for c in ncell)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    x = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    if sigma > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = x + rng.normal(0.0, sigma, size=x.shape)
    box = np.diag([nx * a, ny * a, nz * a]).astype(np.float64)
    types = np.zeros(len(x), dtype=np.int32)
    return np.ascontiguousarray(x), types, box


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def replicate(x, types, box, reps: int):
    """The periodic system (x [n, 3], types [n], orthorhombic box) repeated
    reps times along each axis: copy (i, j, k) is x shifted by (i, j, k) box
    edges, one copy after another; the box grows reps-fold per edge.  Every
    atom keeps the environment it has in the original periodic system."""
    L = np.diag(np.asarray(box, np.float64))
    shifts = np.array([(i, j, k) for i in range(reps) for j in range(reps)
                       for k in range(reps)], np.float64) * L
    xr = (np.asarray(x, np.float64)[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
    tr = np.tile(np.asarray(types, np.int32), len(shifts))
    return np.ascontiguousarray(xr), tr, np.diag(L * reps)


def water_like(nmol: int = 64, L: float = 12.417, seed: int = 3,
               d_oh: float = 0.96, angle_deg: float = 104.5,
               min_oo: float = 2.5, min_inter: float = 1.4, max_tries: int = 200000):
    """Randomly packed water-like box: nmol O atoms (type 0) then 2*nmol H (type 1).

    Rigid molecules (O-H d_oh, H-O-H angle) with uniformly random orientation;
    rejection sampling keeps O-O >= min_oo and every intermolecular pair
    >= min_inter under the minimum image.  Cubic box of edge L (12.417 A
    gives 1 g/cm^3 for 64 molecules).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    half = np.deg2rad(angle_deg) / 2
    local = np.array([[0.0, 0.0, 0.0],
                      [d_oh * np.sin(half), 0.0, d_oh * np.cos(half)],
                      [-d_oh * np.sin(half), 0.0, d_oh * np.cos(half)]])
    mols = []
    tries = 0
    while len(mols) < nmol:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("water_like: packing failed; lower the density")
        c = rng.uniform(0, L, size=3)
        m = c + local @ _random_rotation(rng).T
        ok = True
        for p in mols:
            d = m[:, None, :] - p[None, :, :]
            d -= L * np.round(d / L)
            r = np.sqrt((d * d).sum(-1))
            if r[0, 0] < min_oo or r.min() < min_inter:
                ok = False
                break
        if ok:
            mols.append(m)
    mols = np.array(mols)
    x = np.concatenate([mols[:, 0, :], mols[:, 1:, :].reshape(-1, 3)], axis=0)
    types = np.concatenate([np.zeros(nmol, np.int32), np.ones(2 * nmol, np.int32)])
    box = np.diag([L, L, L]).astype(np.float64)
    return np.ascontiguousarray(x), types, box


def maxwell_velocities(masses, temperature: float, seed: int = 2):
    """Seeded Maxwell-Boltzmann velocities in A/fs, centre-of-mass motion removed
    and rescaled so that the kinetic temperature with 3N-3 degrees of freedom is
    exactly `temperature` (K)."""
    masses = np.asarray(masses, dtype=np.float64)
    n = len(masses)
    rng = np.random.Generator(np.random.PCG64(seed))
    # sigma^2 = kT/m in (eV/amu) -> (A/fs)^2 via ACC_UNIT (eV/(A amu) = ACC_UNIT A/fs^2)
    sig = np.sqrt(KB_EV_PER_K * temperature / masses * ACC_UNIT)
    v = rng.normal(size=(n, 3)) * sig[:, None]
    p = (masses[:, None] * v).sum(0) / masses.sum()
    v -= p
    ke = 0.5 * (masses[:, None] * v * v).sum() / ACC_UNIT  # eV
    t_now = 2 * ke / ((3 * n - 3) * KB_EV_PER_K)
    if t_now > 0:
        v *= np.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


def random_subset(n: int, k: int, seed: int = 7):
    """k distinct atom indices out of n, sorted (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)


_WATER_BASE = {}


def water_tiled(k: int, seed: int = 3):
    """192*k-atom water-like box: the 64-molecule box of water_like tiled k
    times (k a power of two up to 512, tiles as near a cube as possible)."""
    if seed not in _WATER_BASE:
        _WATER_BASE[seed] = water_like(64, seed=seed)
    x0, t0, box0 = _WATER_BASE[seed]
    L = box0[0, 0]
    dims = [1, 1, 1]
    kk, d = k, 0
    while kk > 1:
        dims[d % 3] *= 2
        kk //= 2
        d += 1
    shifts = np.array([[i, j, l] for i in range(dims[0]) for j in range(dims[1])
                       for l in range(dims[2])], np.float64) * L
    x = (x0[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
    types = np.tile(t0, len(shifts))
    box = np.diag([dims[0] * L, dims[1] * L, dims[2] * L]).astype(np.float64)
    return np.ascontiguousarray(x), types.astype(np.int32), box


def serve_requests(n: int, seed: int = 5, min_atoms: int = 500, max_atoms: int = 500000,
                   p_md: float = 0.5, p_water: float = 0.5, md_steps: int = 50,
                   water_md_steps: int = 50):
    """Seeded request mix for the serving loop: copper boxes of log-uniform
    size in [min_atoms, max_atoms] (FCC cells per edge rounded) and water-like
    boxes of 192*k atoms (k log-uniform over powers of two 1..128), each an
    energy/force evaluation or an MD run (md_steps steps for copper,
    water_md_steps for water), with 330 K Maxwell velocities, except that MD
    runs of water start at rest: the seeded water model holds no molecule
    together, and from 330 K its H atoms fly into close contacts within tens
    of fs (the work of a step is the same).  Returns a list of dicts (model,
    kind, x, v, types, box, masses, steps)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        water = rng.uniform() < p_water
        kind = "md" if rng.uniform() < p_md else "eval"
        if water:
            k = 2 ** int(rng.integers(0, 8))
            x, t, box = water_tiled(k, seed=3)
            masses = [MASS_O, MASS_H]
            m = np.where(t == 0, MASS_O, MASS_H)
        else:
            na = float(np.exp(rng.uniform(np.log(min_atoms), np.log(max_atoms))))
            ncell = max(5, int(round((na / 4.0) ** (1.0 / 3.0))))
            x, t, box = fcc_copper(ncell, sigma=0.05, seed=int(rng.integers(1 << 30)))
            masses = [MASS_CU]
            m = np.full(len(x), MASS_CU)
        v = maxwell_velocities(m, 330.0, seed=int(rng.integers(1 << 30)))
        if water and kind == "md":
            v = np.zeros_like(v)
        steps = (water_md_steps if water else md_steps) if kind == "md" else 0
        out.append(dict(model="water" if water else "cu", kind=kind, x=x, v=v, types=t, box=box,
                        masses=masses, steps=steps))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 6):
    """Arrival times (s) of a Poisson stream of n requests at `rate` per second."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
