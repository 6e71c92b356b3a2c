"""Seeded synthetic plane-wave cells: the inputs shared by the oracle and the CUDA path.

This module only *draws* inputs.  It computes nothing that the eigensolver computes:
no kinetic energies of the operator, no Fourier transform of the potential, no
projector Gram matrix used by either side.  Both sides receive the arrays built here
and derive everything else on their own.

Recipe (stand-ins for the paper's BaTiO3 / Ti PAW systems, whose datasets are not
available; the paper's problem statement is Section 2.1, Eq. (KS)):

* cubic cell of side ``L`` bohr, FFT grid ``N^3``, Gamma point unless ``kpt`` is given;
* G-sphere: all integer triples ``m`` with ``|k + G(m)|^2 / 2 <= E_cut`` (Section 2.1,
  "all plane waves whose kinetic energy is less than a threshold"), ordered by the
  integer norm ``m.m`` then lexicographically;
* ``V_loc(r) = sum_a d_a sum_images exp(-|r - R_a|^2 / (2 sigma^2))`` with sigma = 1
  bohr, ``d_a ~ U[-2, -0.5]`` Ha and the 27 nearest periodic images (the image sum of
  a Gaussian factorises into three 1-D image sums);
* projectors: Gaussian radial functions in reciprocal space
  ``f(|k+G|) Y(k+G) exp(-i (k+G).R_a)`` with ``f = exp(-|k+G|^2 sigma_p^2 / 2)``;
  channel set ``s`` (sigma_p = 0.5) for one projector per atom, or
  ``s(0.5), s(1.0), p(0.5) x3, p(1.0) x3`` for ``n_lmn = 8``; every column is scaled
  to unit 2-norm over the sphere;
* ``D`` per-atom blocks: upper triangle ``U[-1, 1]`` mirrored;
  ``Q`` per-atom blocks: upper triangle ``N(0, 0.05)`` (standard deviation) mirrored,
  halved until ``S = I + P Q P^H`` keeps every eigenvalue above 1/2;
* ``Y0``: complex Gaussian ``(a + i b)/sqrt(2)`` damped by ``1 / (1 + |k+G|^2 / 2)``.

Every random stream is a child of ``numpy.random.SeedSequence(seed)`` so changing one
draw does not shift the others.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
from typing import Optional

import numpy as np

__all__ = ["Cell", "make_cell", "CONFIGS", "config_cell", "random_block", "kpoint_cells"]


@dataclasses.dataclass
class Cell:
    """One synthetic problem.  Array layouts match the C-ABI.

    lattice      (3, 3) float64, rows are the lattice vectors a1, a2, a3 (bohr)
    grid         (3,) int, FFT grid N1, N2, N3
    kpt          (3,) float64, Bloch vector k in Cartesian coordinates (1/bohr)
    miller       (npw, 3) int32, integer coordinates m of each plane wave G = m . B
    vloc         (N1, N2, N3) float64, z fastest (C order)
    P            (npw, nproj) complex128, Fortran order (column j = projector j)
    proj_offsets (natoms + 1,) int32, projector columns of atom a are
                 [proj_offsets[a], proj_offsets[a + 1])
    D, Q         concatenated per-atom n_a x n_a blocks, row-major; Q is None for S = I
    Y0           (npw, nbands) complex128, Fortran order
    """

    lattice: np.ndarray
    grid: np.ndarray
    kpt: np.ndarray
    miller: np.ndarray
    vloc: np.ndarray
    P: np.ndarray
    proj_offsets: np.ndarray
    D: np.ndarray
    Q: Optional[np.ndarray]
    Y0: np.ndarray
    ecut: float
    atoms: np.ndarray
    depths: np.ndarray
    q_halvings: int = 0
    name: str = ""

    @property
    def npw(self) -> int:
        return int(self.miller.shape[0])

    @property
    def nproj(self) -> int:
        return int(self.P.shape[1])

    @property
    def natoms(self) -> int:
        return int(len(self.proj_offsets) - 1)

    @property
    def nbands(self) -> int:
        return int(self.Y0.shape[1])

    def block_sizes(self) -> np.ndarray:
        return np.diff(self.proj_offsets).astype(np.int64)


def random_block(rng: np.random.Generator, n: int, kind: str, scale: float) -> np.ndarray:
    """Symmetric n x n block: upper triangle drawn, mirrored to the lower one."""
    if kind == "uniform":
        u = rng.uniform(-scale, scale, size=(n, n))
    else:
        u = rng.normal(0.0, scale, size=(n, n))
    b = np.triu(u)
    return b + np.triu(b, 1).T


def _sphere(lattice, kpt, ecut):
    binv = 2.0 * np.pi * np.linalg.inv(lattice).T  # rows b1, b2, b3
    # bound on |m_i|: |G| <= sqrt(2 ecut) + |k|, |m_i| <= |G| |a_i| / 2pi
    gmax = np.sqrt(2.0 * ecut) + np.linalg.norm(kpt)
    mmax = [int(np.ceil(gmax * np.linalg.norm(lattice[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-m, m + 1) for m in mmax]
    m = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    kg = kpt[None, :] + m @ binv
    keep = 0.5 * np.einsum("ij,ij->i", kg, kg) <= ecut
    m = m[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.einsum("ij,ij->i", m, m)))
    return m[order].astype(np.int32), binv


def _vloc(lattice, grid, atoms, depths, sigma=1.0):
    L = np.diag(lattice)
    assert np.allclose(lattice, np.diag(L)), "the Gaussian image sum assumes a cubic/orthorhombic cell"
    v = np.zeros(tuple(grid), dtype=np.float64)
    axes = [np.arange(grid[i]) * (L[i] / grid[i]) for i in range(3)]
    for pos, d in zip(atoms, depths):
        fac = []
        for i in range(3):
            x = axes[i][:, None] - pos[i] - L[i] * np.array([-1.0, 0.0, 1.0])[None, :]
            fac.append(np.exp(-(x * x) / (2.0 * sigma * sigma)).sum(1))
        v += d * np.einsum("i,j,k->ijk", fac[0], fac[1], fac[2])
    return v


def _projectors(kg, atoms, channels):
    npw = kg.shape[0]
    g2 = np.einsum("ij,ij->i", kg, kg)
    cols = []
    for pos in atoms:
        phase = np.exp(-1j * (kg @ pos))
        for kind, sp in channels:
            radial = np.exp(-0.5 * g2 * sp * sp)
            if kind == "s":
                ang = [np.ones(npw)]
            else:
                ang = [kg[:, 0], kg[:, 1], kg[:, 2]]
            for a in ang:
                c = radial * a * phase
                cols.append(c / np.linalg.norm(c))
    return np.asfortranarray(np.stack(cols, 1))


def _blockdiag(blocks_flat, sizes):
    n = int(sizes.sum())
    out = np.zeros((n, n))
    o = 0
    f = 0
    for s in sizes:
        out[o:o + s, o:o + s] = blocks_flat[f:f + s * s].reshape(s, s)
        o += s
        f += s * s
    return out


def make_cell(L: float, grid: int, ecut: float, natoms: int, nlmn: int, nbands: int,
              paw: bool, seed: int, kpt=(0.0, 0.0, 0.0), name: str = "") -> Cell:
    """Draw one synthetic cell; see the module docstring for the recipe."""
    ss = np.random.SeedSequence(seed)
    r_pos, r_dep, r_d, r_q, r_y = [np.random.default_rng(s) for s in ss.spawn(5)]
    lattice = np.diag([float(L)] * 3)
    grid3 = np.array([grid] * 3, dtype=np.int64)
    kpt = np.asarray(kpt, dtype=np.float64)
    miller, binv = _sphere(lattice, kpt, ecut)
    assert np.all(np.abs(miller) < np.asarray(grid3)[None, :] // 2), "sphere does not fit the FFT grid"
    atoms = r_pos.uniform(0.0, L, size=(natoms, 3))
    depths = r_dep.uniform(-2.0, -0.5, size=natoms)
    vloc = _vloc(lattice, grid3, atoms, depths)
    kg = kpt[None, :] + miller @ binv
    if nlmn == 1:
        channels = [("s", 0.5)]
    elif nlmn == 8:
        channels = [("s", 0.5), ("s", 1.0), ("p", 0.5), ("p", 1.0)]
    else:
        raise ValueError("n_lmn must be 1 or 8")
    P = _projectors(kg, atoms, channels)
    offs = np.arange(natoms + 1, dtype=np.int32) * nlmn
    D = np.concatenate([random_block(r_d, nlmn, "uniform", 1.0).ravel() for _ in range(natoms)])
    Q = None
    halvings = 0
    if paw:
        Q = np.concatenate([random_block(r_q, nlmn, "normal", 0.05).ravel() for _ in range(natoms)])
        # admissibility of the draw: S = I + P Q P^H must stay well positive definite.
        # The nonzero eigenvalues of P Q P^H are those of R^H Q R with P = U R (thin QR).
        R = np.linalg.qr(P, mode="r")
        while True:
            qd = _blockdiag(Q, np.diff(offs))
            lo = np.linalg.eigvalsh(R @ qd @ R.conj().T).min()
            if lo > -0.5:
                break
            Q = Q * 0.5
            halvings += 1
    g2 = np.einsum("ij,ij->i", kg, kg)
    y = (r_y.normal(size=(miller.shape[0], nbands)) + 1j * r_y.normal(size=(miller.shape[0], nbands)))
    y *= (1.0 / np.sqrt(2.0)) / (1.0 + 0.5 * g2)[:, None]
    return Cell(lattice=lattice, grid=grid3, kpt=kpt, miller=miller, vloc=vloc, P=P,
                proj_offsets=offs, D=D, Q=Q, Y0=np.asfortranarray(y), ecut=float(ecut),
                atoms=atoms, depths=depths, q_halvings=halvings, name=name)


#: The synthetic workloads: name -> (L bohr, grid, E_cut Ha, atoms, n_lmn, bands, PAW,
#: Chebyshev degree, sweeps).  Seeds are 1000 + index.
CONFIGS = {
    "nc24": dict(L=10.0, grid=24, ecut=7.60, natoms=8, nlmn=1, nbands=32, paw=False,
                 degree=8, sweeps=5, seed=1001),
    "paw48": dict(L=20.0, grid=48, ecut=7.58, natoms=32, nlmn=8, nbands=256, paw=True,
                  degree=10, sweeps=8, seed=1002),
    "paw96": dict(L=40.0, grid=96, ecut=7.275, natoms=256, nlmn=8, nbands=2048, paw=True,
                  degree=4, sweeps=4, seed=1003),
    # same spacing and atom density at 72^3: a mid-size case for detailed profiles whose
    # wavefunction block (512 bands) still exceeds the L2 cache
    "paw72": dict(L=30.0, grid=72, ecut=7.275, natoms=108, nlmn=8, nbands=512, paw=True,
                  degree=4, sweeps=4, seed=1006),
    # paw96's FFT geometry (same cell, grid and E_cut: the same 60005-point sphere and 1861
    # columns) with 4 atoms: a small device footprint for counter captures of the FFT passes,
    # its column buffer (128 bands, 183 MB) still larger than the L2 cache
    "prof96": dict(L=40.0, grid=96, ecut=7.275, natoms=4, nlmn=8, nbands=128, paw=True,
                   degree=4, sweeps=4, seed=1007),
}


def _cache_path(key: str) -> str:
    root = os.environ.get("SYNTH_CACHE", os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), ".synth_cache"))
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, key + ".npz")


def config_cell(name: str, nbands: Optional[int] = None, cache: bool = True) -> Cell:
    """The named workload (optionally with fewer bands: Y0 keeps its first columns)."""
    c = CONFIGS[name]
    key = hashlib.sha1(repr(sorted(c.items())).encode()).hexdigest()[:12] + "_" + name
    path = _cache_path(key) if cache else None
    if path and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        cell = Cell(lattice=z["lattice"], grid=z["grid"], kpt=z["kpt"], miller=z["miller"],
                    vloc=z["vloc"], P=np.asfortranarray(z["P"]), proj_offsets=z["proj_offsets"],
                    D=z["D"], Q=(z["Q"] if z["Q"].size else None),
                    Y0=np.asfortranarray(z["Y0"]), ecut=float(z["ecut"]), atoms=z["atoms"],
                    depths=z["depths"], q_halvings=int(z["q_halvings"]), name=name)
    else:
        cell = make_cell(c["L"], c["grid"], c["ecut"], c["natoms"], c["nlmn"], c["nbands"],
                         c["paw"], c["seed"], name=name)
        if path:
            tmp = path + ".tmp.npz"
            np.savez(tmp, lattice=cell.lattice, grid=cell.grid, kpt=cell.kpt, miller=cell.miller,
                     vloc=cell.vloc, P=cell.P, proj_offsets=cell.proj_offsets, D=cell.D,
                     Q=(cell.Q if cell.Q is not None else np.zeros(0)), Y0=cell.Y0,
                     ecut=cell.ecut, atoms=cell.atoms, depths=cell.depths,
                     q_halvings=cell.q_halvings)
            os.replace(tmp, path)
    if nbands is not None:
        cell.Y0 = np.asfortranarray(cell.Y0[:, :nbands])
    return cell


def kpoint_cells(nk: int = 64, nbands: int = 128, seed: int = 1004, npw_range=(3000, 12000), L: float = 20.0,
                 grid: int = 48, natoms: int = 32, nlmn: int = 8):
    """The batched k-point workload: one PAW cell (the atoms, V_loc, D and Q of
    ``make_cell(L, grid, ., natoms, nlmn, ., True, seed)``) sampled at ``nk`` Bloch vectors k
    drawn uniformly in the first Brillouin zone, each with its own E_cut so that its G-sphere
    size is drawn uniformly in ``npw_range`` (sizes from the free-electron count
    N_pw ~ L^3 (2 E_cut)^{3/2} / (6 pi^2)).  Q is the most-halved of the per-k admissible
    draws, so every k-point sees the same S coefficients.  Returns a list of Cells."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    target = rng.uniform(npw_range[0], npw_range[1], size=nk)
    kpts = rng.uniform(-np.pi / L, np.pi / L, size=(nk, 3))
    cells = []
    for i in range(nk):
        ecut = 0.5 * (target[i] * 6.0 * np.pi ** 2 / L ** 3) ** (2.0 / 3.0)
        cells.append(make_cell(L, grid, ecut, natoms, nlmn, nbands, True, seed, kpt=kpts[i], name="k%d" % i))
    h = max(c.q_halvings for c in cells)
    for c in cells:
        c.Q = c.Q * 0.5 ** (h - c.q_halvings)
        c.q_halvings = h
    return cells
