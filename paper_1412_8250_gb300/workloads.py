"""Seeded synthetic inputs for the periodic OF-DFT hot path.

This module holds input generation only: FCC aluminium-like cells (lattice, random
displacements, vacancies) and seeded test fields. It contains none of the method's
arithmetic (no finite-difference weights, no pseudocharges, no functionals), so both the
CUDA path and the CPU oracle can be fed from it without sharing any computation.

Recipe (all lengths in bohr):
  * cubic FCC cells of lattice constant ``a`` (7.6 by default), basis at fractional
    (0,0,0), (0,1/2,1/2), (1/2,0,1/2), (1/2,1/2,0) -- the 4-atom Al unit cell used in
    Sec. 5.1 of the paper (there with a = 8.0) and the supercells of Sec. 5.3 / 5.5;
  * ``points_per_cell`` grid points per cubic cell edge (32 gives h = 0.2375);
  * every ion carries charge Z = 3 and a Gaussian pseudocharge (the charge density of the
    nuclei of Sec. 3.2 is replaced by a normalised Gaussian because the paper's
    pseudopotential tables are not available): width sigma = 0.7, cutoff r_c = 7 for TFW
    cells; sigma = 1.2, r_c = 10 (the paper's cutoff) for cells run with the linear-response
    kernel, whose energy has no minimiser with u >= 0 for the harder sigma = 0.7 ions;
  * displacements are uniform in [-d, d] per coordinate from ``numpy.random.default_rng``;
  * vacancies remove the site nearest the cell centre, or random sites when drawn.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

A_LATTICE = 7.6
Z_ION = 3.0
SIGMA = 0.7          # TFW cells
R_CUT = 7.0
SIGMA_LR = 1.2       # cells run with the linear-response (kernel) term
R_CUT_LR = 10.0
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


@dataclass
class Cell:
    """A periodic cuboid cell with ions and a uniform grid.

    ``n`` = (n1, n2, n3) grid points along x, y, z; ``L`` = side lengths; ``R`` = (M, 3)
    ion positions (cartesian, inside [0, L)); ``Z`` = (M,) ion charges; ``sigma`` and ``rc``
    the Gaussian pseudocharge width and cutoff.  Fields on this grid are stored x-fastest,
    i.e. as arrays of shape (n3, n2, n1).
    """
    n: tuple
    L: tuple
    R: np.ndarray
    Z: np.ndarray
    sigma: float = SIGMA
    rc: float = R_CUT
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def n_electrons(self) -> float:
        return float(self.Z.sum())

    @property
    def shape(self) -> tuple:
        """numpy shape of a field on this grid (x fastest)."""
        return (self.n[2], self.n[1], self.n[0])


def fcc_supercell(reps=(1, 1, 1), a=A_LATTICE, points_per_cell=32, displacement=0.0,
                  vacancy="none", seed=None, Z=Z_ION, sigma=SIGMA, rc=R_CUT, name=""):
    """FCC supercell of reps[0] x reps[1] x reps[2] cubic cells.

    vacancy: "none", "center" (remove the site nearest the cell centre) or "random".
    Displacements are drawn after the vacancy choice, from the same generator.
    """
    rng = np.random.default_rng(seed)
    reps = tuple(int(c) for c in reps)
    sites = []
    for k in range(reps[2]):
        for j in range(reps[1]):
            for i in range(reps[0]):
                for b in FCC_BASIS:
                    sites.append((np.array([i, j, k], dtype=float) + b) * a)
    R = np.array(sites)
    L = tuple(float(c * a) for c in reps)
    if vacancy == "center":
        centre = np.array(L) / 2
        R = np.delete(R, int(np.argmin(((R - centre) ** 2).sum(1))), axis=0)
    elif vacancy == "random":
        R = np.delete(R, int(rng.integers(R.shape[0])), axis=0)
    elif vacancy != "none":
        raise ValueError(vacancy)
    if displacement:
        R = R + rng.uniform(-displacement, displacement, size=R.shape)
    R = np.mod(R, np.array(L))
    n = tuple(int(c * points_per_cell) for c in reps)
    return Cell(n=n, L=L, R=R, Z=np.full(R.shape[0], float(Z)), sigma=sigma, rc=rc,
                name=name or f"fcc{reps[0]}x{reps[1]}x{reps[2]}",
                meta=dict(reps=reps, a=a, displacement=displacement, vacancy=vacancy,
                          seed=seed))


def al4_cell(points_per_cell=32, a=A_LATTICE):
    """4-atom cubic FCC cell, a = 7.6, ions exactly on grid points, 32^3 grid (TFW case)."""
    return fcc_supercell((1, 1, 1), a=a, points_per_cell=points_per_cell, name="al4")


def al4_displaced_cell(points_per_cell=32, a=A_LATTICE):
    """4-atom FCC cell with the corner atom moved to (0.80, 0.56, 0.42) (Sec. 5.1 geometry)."""
    c = fcc_supercell((1, 1, 1), a=a, points_per_cell=points_per_cell, name="al4_disp")
    c.R[0] = np.array([0.80, 0.56, 0.42])
    return c


def al108_cell(seed=2):
    """108-atom 3x3x3 FCC supercell, +-0.1 displacements, 96^3 grid (WT-type case)."""
    return fcc_supercell((3, 3, 3), points_per_cell=32, displacement=0.1, seed=seed,
                         sigma=SIGMA_LR, rc=R_CUT_LR, name="al108")


def al4_lr_cell(points_per_cell=32, seed=2):
    """4-atom FCC cell, +-0.1 displacements, soft ions: the smallest WT-type case."""
    return fcc_supercell((1, 1, 1), points_per_cell=points_per_cell, displacement=0.1,
                         seed=seed, sigma=SIGMA_LR, rc=R_CUT_LR, name="al4_lr")


def al864_cell(seed=4):
    """864-atom 6x6x6 FCC supercell, +-0.1 displacements, 192^3 grid."""
    return fcc_supercell((6, 6, 6), points_per_cell=32, displacement=0.1, seed=seed,
                         sigma=SIGMA_LR, rc=R_CUT_LR, name="al864")


def al3999_cell(seed=5):
    """10x10x10 FCC supercell with the centre site removed, +-0.1 displacements, 320^3."""
    return fcc_supercell((10, 10, 10), points_per_cell=32, displacement=0.1,
                         vacancy="center", seed=seed, sigma=SIGMA_LR, rc=R_CUT_LR,
                         name="al3999")


def batched_cells(count=64, seed=3):
    """Uneven independent cells: reps drawn per axis from {2,3,4}, half with a vacancy.

    Shapes, then which cells get a vacancy, then per-cell displacement seeds are drawn in
    that order from one generator.
    """
    rng = np.random.default_rng(seed)
    reps = rng.integers(2, 5, size=(count, 3))
    vac = np.zeros(count, dtype=bool)
    vac[rng.choice(count, count // 2, replace=False)] = True
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [fcc_supercell(tuple(reps[c]), displacement=0.1,
                          vacancy="random" if vac[c] else "none", seed=int(seeds[c]),
                          sigma=SIGMA_LR, rc=R_CUT_LR, name=f"cell{c}") for c in range(count)]


def small_cell(n=(16, 16, 16), L=(7.6, 7.6, 7.6), sigma=0.9, rc=6.0, seed=0, n_atoms=4,
               Z=Z_ION):
    """A small cell with randomly placed ions, for quick tests (non-cubic grids allowed)."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, 1, size=(n_atoms, 3)) * np.array(L)
    return Cell(n=tuple(n), L=tuple(float(x) for x in L), R=R, Z=np.full(n_atoms, float(Z)),
                sigma=sigma, rc=rc, name=f"small{n}")


def random_field(shape, seed=0, kind="white", dtype=np.float64):
    """Seeded test field of numpy shape (n3, n2, n1).

    kind: "white" (uniform in [-1, 1]) or "smooth" (a few random low-order Fourier modes
    plus a constant, positive everywhere).
    """
    rng = np.random.default_rng(seed)
    if kind == "white":
        return rng.uniform(-1.0, 1.0, size=shape).astype(dtype)
    if kind == "smooth":
        n3, n2, n1 = shape
        z, y, x = np.meshgrid(np.arange(n3) / n3, np.arange(n2) / n2, np.arange(n1) / n1,
                              indexing="ij")
        f = np.full(shape, 2.0)
        for _ in range(6):
            k = rng.integers(-3, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.uniform(0.05, 0.25)
            f += amp * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + ph)
        return f.astype(dtype)
    raise ValueError(kind)


def initial_network(seed=0, channels=16, scale=0.3):
    """Seeded initial parameters of the preconditioner network, flattened in the order of the C
    ABI (W1[16][27], b1[16], W2[16][16][27], b2[16], W3[16][27], b3), float32: normal weights
    with variance 2 / fan-in (1 / fan-in for the last layer), times `scale`; zero biases."""
    rng = np.random.default_rng(seed)
    c = channels
    W1 = rng.normal(0, np.sqrt(2.0 / 27), size=(c, 1, 27))
    W2 = rng.normal(0, np.sqrt(2.0 / (27 * c)), size=(c, c, 27))
    W3 = rng.normal(0, np.sqrt(1.0 / (27 * c)), size=(1, c, 27))
    parts = [scale * W1, np.zeros(c), scale * W2, np.zeros(c), scale * W3, np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
