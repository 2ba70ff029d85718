"""Seeded synthetic meshes and densities (shared by the CUDA path, the oracle and the bench).

This module only produces inputs: a block octree in the layout the library and the oracle both
accept, and a density per cell. It holds none of the solver's arithmetic (no masses, moments,
MACs, interactions, Ewald sums or column integrals).

Mesh layout (Sec. 2 of the paper: an amr-tree of blocks, each leaf-block holding 8^3 cells):
  level[nb]    int32, root block = 1, children one level deeper
  child[nb,8]  int32, child block of octant c = ix + 2*iy + 4*iz, or -1 for a leaf-block
  lo[nb,3]     float64, lower corner of the block
  size[nb,3]   float64, edge lengths of the block (cuboid allowed: Sec. 2, blocks may have
               different physical sizes per direction)
Block 0 is the root.  Blocks are listed in depth-first (Morton) pre-order, so leaf-blocks appear
in Morton order.  The density of leaf-block n (n-th leaf in block order) is rho[n, k, j, i]
(x fastest).
"""
from __future__ import annotations

import dataclasses
import numpy as np

NB = 8  # cells per block edge (2^l_bt with l_bt = 3)


@dataclasses.dataclass
class Mesh:
    level: np.ndarray
    child: np.ndarray
    lo: np.ndarray
    size: np.ndarray
    bc: tuple = (0, 0, 0)          # per axis: 0 isolated, 1 periodic

    @property
    def nblocks(self) -> int:
        return int(self.level.shape[0])

    @property
    def leaves(self) -> np.ndarray:
        return np.nonzero(self.child[:, 0] < 0)[0].astype(np.int64)

    @property
    def nleaf(self) -> int:
        return int((self.child[:, 0] < 0).sum())

    @property
    def ncell(self) -> int:
        return self.nleaf * NB ** 3

    @property
    def domain_lo(self) -> np.ndarray:
        return self.lo[0].copy()

    @property
    def domain_size(self) -> np.ndarray:
        return self.size[0].copy()

    def cell_centres(self) -> np.ndarray:
        """[nleaf, 8, 8, 8, 3] cell centres (k, j, i order)."""
        lf = self.leaves
        lo = self.lo[lf]
        dx = self.size[lf] / NB
        idx = (np.arange(NB) + 0.5)
        x = lo[:, None, None, None, 0] + idx[None, None, None, :] * dx[:, None, None, None, 0]
        y = lo[:, None, None, None, 1] + idx[None, None, :, None] * dx[:, None, None, None, 1]
        z = lo[:, None, None, None, 2] + idx[None, :, None, None] * dx[:, None, None, None, 2]
        out = np.empty((lf.size, NB, NB, NB, 3))
        out[..., 0] = x
        out[..., 1] = y
        out[..., 2] = z
        return out

    def cell_volume(self) -> np.ndarray:
        """[nleaf] volume of one cell of each leaf-block."""
        s = self.size[self.leaves] / NB
        return s[:, 0] * s[:, 1] * s[:, 2]


def build_mesh(refine, box=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), bc=(0, 0, 0)) -> Mesh:
    """Refine the root block recursively while refine(level, lo, size) is true (depth-first)."""
    level, child, lo, size = [], [], [], []

    def add(lev, blo, bsz):
        b = len(level)
        level.append(lev)
        child.append([-1] * 8)
        lo.append(list(blo))
        size.append(list(bsz))
        if refine(lev, np.asarray(blo), np.asarray(bsz)):
            h = np.asarray(bsz) / 2.0
            for c in range(8):
                off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=np.float64)
                child[b][c] = add(lev + 1, np.asarray(blo) + off * h, h)
        return b

    add(1, np.asarray(origin, dtype=np.float64), np.asarray(box, dtype=np.float64))
    return Mesh(level=np.asarray(level, dtype=np.int32),
                child=np.asarray(child, dtype=np.int32),
                lo=np.asarray(lo, dtype=np.float64),
                size=np.asarray(size, dtype=np.float64),
                bc=tuple(int(v) for v in bc))


def uniform_mesh(ncell_axis: int, box=(1.0, 1.0, 1.0), bc=(0, 0, 0)) -> Mesh:
    """Uniform grid of ncell_axis^3 cells (ncell_axis = 8 * 2^k) as a full block octree."""
    nblk = ncell_axis // NB
    assert nblk * NB == ncell_axis and nblk & (nblk - 1) == 0, "ncell_axis must be 8 * 2^k"
    leaf_level = 1 + int(round(np.log2(nblk)))
    return build_mesh(lambda lev, lo, sz: lev < leaf_level, box=box, bc=bc)


def uniform_to_blocks(mesh: Mesh, field: np.ndarray) -> np.ndarray:
    """Scatter a uniform [nz, ny, nx] field into [nleaf, 8, 8, 8] for a uniform mesh."""
    lf = mesh.leaves
    dom_lo, dom_sz = mesh.domain_lo, mesh.domain_size
    nz, ny, nx = field.shape
    out = np.empty((lf.size, NB, NB, NB), dtype=field.dtype)
    for n, b in enumerate(lf):
        bi = np.rint((mesh.lo[b] - dom_lo) / dom_sz * np.array([nx, ny, nz])).astype(int)
        out[n] = field[bi[2]:bi[2] + NB, bi[1]:bi[1] + NB, bi[0]:bi[0] + NB]
    return out


def gaussian_random_field(n: int, slope: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance periodic Gaussian random field on n^3 with P(k) ~ k^slope (k=0 removed)."""
    k = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(k, k, np.fft.rfftfreq(n) * n, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (slope / 2.0)
    noise = rng.standard_normal((n, n, n))
    f = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=(n, n, n), axes=(0, 1, 2))
    f -= f.mean()
    f /= f.std()
    return f


# ---------------------------------------------------------------- the five workloads

def sphere_32(seed: int = 0, ncell_axis: int = 32):
    """Isolated uniform 32^3 grid, unit box: sphere R=0.3, rho=1*(1+0.1 N(0,1)), background 1e-3."""
    rng = np.random.default_rng(seed)
    mesh = uniform_mesh(ncell_axis)
    r = mesh.cell_centres() - 0.5
    rr = np.sqrt((r ** 2).sum(-1))
    rho = np.where(rr < 0.3, 1.0 * (1.0 + 0.1 * rng.standard_normal(rr.shape)), 1e-3)
    return mesh, np.maximum(rho, 1e-3)


def plummer_refine(a: float = 0.05, thresh: float = 0.0013, min_level: int = 3, max_level: int = 6):
    c = np.array([0.5, 0.5, 0.5])

    def rho_p(r):
        return (1.0 + (r / a) ** 2) ** -2.5

    def refine(lev, lo, sz):
        if lev < min_level:
            return True
        if lev >= max_level:
            return False
        closest = np.clip(c, lo, lo + sz)
        dmin = np.sqrt(((closest - c) ** 2).sum())
        return sz.max() * np.sqrt(rho_p(dmin)) > thresh

    return refine


def plummer_amr(seed: int = 1, a: float = 0.05, max_level: int = 6, sigma: float = 0.2):
    """Isolated AMR mesh (leaf levels 3..max_level) around a Plummer sphere with log-normal noise."""
    rng = np.random.default_rng(seed)
    mesh = build_mesh(plummer_refine(a=a, max_level=max_level))
    r = mesh.cell_centres() - 0.5
    rr2 = (r ** 2).sum(-1)
    rho_p = (1.0 + rr2 / a ** 2) ** -2.5
    rho = rho_p * np.exp(sigma * rng.standard_normal(rr2.shape) - 0.5 * sigma * sigma)
    return mesh, rho


def be_sphere(n: int = 128, radius: float = 0.4, contrast: float = 14.0, ambient: float = 0.01):
    """Isolated uniform n^3 unit box holding a Bonnor-Ebert-like sphere: rho = 1 / (1 + (r/a)^2)
    inside `radius` (the isothermal profile's large-r form), with a chosen so that the centre-to-edge
    contrast is `contrast` (about 14 for the critical sphere), and `ambient` times the edge density
    outside.  Deterministic (no noise): a static single-step configuration."""
    mesh = uniform_mesh(n)
    r = np.sqrt(((mesh.cell_centres() - 0.5) ** 2).sum(-1))
    a = radius / np.sqrt(contrast - 1.0)
    rho = 1.0 / (1.0 + (r / a) ** 2)
    return mesh, np.where(r <= radius, rho, ambient / contrast)


def disk_2p1i(seed: int = 2, n: int = 256, hz: float = 0.05, amp: float = 0.3):
    """Mixed BCs (x,y periodic, z isolated), n^3 grid in a 1x1x4 box, exponential disk + GRF."""
    rng = np.random.default_rng(seed)
    mesh = uniform_mesh(n, box=(1.0, 1.0, 4.0), bc=(1, 1, 0))
    g = gaussian_random_field(n, -2.0, rng)
    z = (np.arange(n) + 0.5) * (4.0 / n)
    rho = np.exp(-np.abs(z - 2.0) / hz)[:, None, None] * (1.0 + amp * g)
    return mesh, uniform_to_blocks(mesh, np.maximum(rho, 1e-6))


def turbulent_periodic(seed: int = 3, n: int = 128, sigma_ln: float = 1.5, slope: float = -4.0):
    """Fully periodic n^3 unit box, log-normal density with ln(rho) = s*g - s^2/2, g ~ GRF k^slope."""
    rng = np.random.default_rng(seed)
    mesh = uniform_mesh(n, bc=(1, 1, 1))
    g = gaussian_random_field(n, slope, rng)
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    return mesh, uniform_to_blocks(mesh, rho)


def batched_grids(count: int = 64, base: int = 32):
    """Independent grids g = 0..count-1 of side base*2^(g mod 3) with rotating BCs and densities."""
    bcs = [(0, 0, 0), (1, 1, 1), (1, 1, 0)]
    out = []
    for g in range(count):
        n = base * 2 ** (g % 3)
        bc = bcs[(g // 3) % 3]
        rng = np.random.default_rng(g)
        mesh = uniform_mesh(n, bc=bc)
        if g % 2 == 0:
            r = mesh.cell_centres() - 0.5
            rr2 = (r ** 2).sum(-1)
            rho = (1.0 + rr2 / 0.05 ** 2) ** -2.5 * np.exp(0.2 * rng.standard_normal(rr2.shape) - 0.02)
        else:
            gg = gaussian_random_field(n, -4.0, rng)
            rho = uniform_to_blocks(mesh, np.exp(1.5 * gg - 1.125))
        out.append((mesh, rho))
    return out


def sample_cells(ncell: int, count: int, seed: int = 12345) -> np.ndarray:
    """Sorted distinct random flat cell indices (leaf*512 + k*64 + j*8 + i)."""
    rng = np.random.default_rng(seed)
    count = min(count, ncell)
    return np.sort(rng.choice(ncell, size=count, replace=False)).astype(np.int64)
