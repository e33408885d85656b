"""Seeded synthetic inputs for the FE spinor ChFSI hot path.

This module only *draws* inputs: mesh descriptions, atom positions, the
quadrature-point fields V_eff and B_xc, the values of the atom-centred
projector functions at the quadrature points of their support cells, the
2x2-spin-block SOC coupling matrices Delta_a, and the random spinor blocks.
It contains none of the method's arithmetic (no FE basis, no operator, no
filter); both the CUDA path and the CPU oracle consume what it produces.

Workload shapes follow the paper's setting (Sec. III.A: hexahedral cells,
GLL nodes of order p, Gauss quadrature; Sec. II.B, Eq. nlOP: atom-centred
separable projectors with 2x2 D blocks indexed 2*chi+alpha).  The paper does
not state the constants (well depth/width, projector Gaussian widths, cut-off
radius, B magnitude, Delta spread); the defaults of ``make_problem`` are the
values chosen for them.

Seed streams (offset added to ``seed * 100``): 0 = spinor block X,
1 = atom positions, 2 = B_xc Fourier modes, 3 = Delta matrices,
4 = Lanczos start vector, 5 = gradient weights / directions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Atom", "Problem", "make_problem", "config", "random_block", "random_start",
    "free_nodes_per_dim", "n_free_nodes", "CONFIGS", "gauss_points_1d",
]


# ----------------------------------------------------------------------------
# small helpers (geometry of the structured mesh, quadrature coordinates)
# ----------------------------------------------------------------------------
def free_nodes_per_dim(ncell: int, p: int, periodic: bool) -> int:
    """Number of free global FE nodes along one direction.

    Periodic: n*p nodes (the last face is identified with the first).
    Non-periodic (homogeneous Dirichlet on both faces): n*p - 1 interior
    nodes.
    """
    return ncell * p if periodic else ncell * p - 1


def n_free_nodes(ncell, p, periodic) -> int:
    return int(np.prod([free_nodes_per_dim(n, p, bool(b)) for n, b in zip(ncell, periodic)]))


def gauss_points_1d(nq: int):
    """Gauss-Legendre points/weights on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return x, w


def _quad_coords(ncell, h, nq):
    """Physical coordinates of every quadrature point, shape [E, nq^3, 3].

    Cell index e = (cz*ny + cy)*nx + cx; point index q = (qz*nq + qy)*nq + qx.
    """
    nx, ny, nz = ncell
    xi, _ = gauss_points_1d(nq)
    t = (xi + 1.0) * 0.5
    cx = (np.arange(nx)[:, None] + t[None, :]) * h[0]   # [nx, nq]
    cy = (np.arange(ny)[:, None] + t[None, :]) * h[1]
    cz = (np.arange(nz)[:, None] + t[None, :]) * h[2]
    # broadcast to [cz, cy, cx, qz, qy, qx]
    X = np.broadcast_to(cx[None, None, :, None, None, :], (nz, ny, nx, nq, nq, nq))
    Y = np.broadcast_to(cy[None, :, None, None, :, None], (nz, ny, nx, nq, nq, nq))
    Z = np.broadcast_to(cz[:, None, None, :, None, None], (nz, ny, nx, nq, nq, nq))
    out = np.stack([X, Y, Z], axis=-1).reshape(nx * ny * nz, nq ** 3, 3)
    return np.ascontiguousarray(out)


def _real_sph_harm(l: int, d: np.ndarray) -> np.ndarray:
    """Real spherical harmonics Y_lm(r_hat) for l <= 2, m = -l..l; d: [..., 3].

    Returns [..., 2l+1].  At r = 0 the l >= 1 functions are taken as 0 (they
    multiply r^l radial parts that vanish there anyway).
    """
    r = np.linalg.norm(d, axis=-1)
    safe = np.where(r > 0, r, 1.0)
    x, y, z = d[..., 0] / safe, d[..., 1] / safe, d[..., 2] / safe
    if l == 0:
        return np.full(d.shape[:-1] + (1,), 0.5 / math.sqrt(math.pi))
    if l == 1:
        c = math.sqrt(3.0 / (4.0 * math.pi))
        return np.stack([c * y, c * z, c * x], axis=-1)
    if l == 2:
        c1 = 0.5 * math.sqrt(15.0 / math.pi)
        c0 = 0.25 * math.sqrt(5.0 / math.pi)
        c2 = 0.25 * math.sqrt(15.0 / math.pi)
        return np.stack([c1 * x * y, c1 * y * z, c0 * (3 * z * z - 1.0),
                         c1 * x * z, c2 * (x * x - y * y)], axis=-1)
    raise ValueError("l > 2 not supported")


def _radial_norm(l: int, sigma: float, rc: float) -> float:
    """1 / sqrt( int_0^rc (r^l exp(-r^2/(2 sigma^2)))^2 r^2 dr ) on a fine grid."""
    r = np.linspace(0.0, rc, 20001)
    f = (r ** l * np.exp(-r * r / (2 * sigma * sigma))) ** 2 * r * r
    trap = getattr(np, "trapezoid", None) or getattr(np, "trapz")
    return 1.0 / math.sqrt(trap(f, r))


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------
@dataclass
class Atom:
    pos: np.ndarray                 # (3,) bohr
    npj: int                        # number of scalar projectors chi
    supp_cell: np.ndarray           # (ns,) int32 cell indices
    supp_img: np.ndarray            # (ns, 3) int32 lattice image shifts (units of box length)
    pvals: np.ndarray               # (ns, nq^3, npj) float64: p_chi(r_q - L - R)
    delta: np.ndarray               # (2npj, 2npj) complex128, Hermitian, index 2*chi+alpha


@dataclass
class Problem:
    ncell: tuple
    h: tuple
    p: int
    nq: int
    periodic: tuple
    k: np.ndarray
    veff: np.ndarray                # [E, nq^3]
    bx: np.ndarray
    by: np.ndarray
    bz: np.ndarray
    atoms: list = field(default_factory=list)
    name: str = ""
    seed: int = 0

    @property
    def ncells(self) -> int:
        return int(np.prod(self.ncell))

    @property
    def nnodes(self) -> int:
        return n_free_nodes(self.ncell, self.p, self.periodic)

    @property
    def box(self) -> np.ndarray:
        return np.array([n * hh for n, hh in zip(self.ncell, self.h)], dtype=np.float64)

    def flat_projectors(self):
        """Flattened projector arrays in the layout of gbc_set_projectors."""
        if not self.atoms:
            return dict(natoms=0, npj=np.zeros(0, np.int32), pos=np.zeros(0),
                        nsupp=np.zeros(0, np.int32), supp_cell=np.zeros(0, np.int32),
                        supp_img=np.zeros(0, np.int32), pvals=np.zeros(0),
                        delta=np.zeros(0, np.complex128))
        return dict(
            natoms=len(self.atoms),
            npj=np.array([a.npj for a in self.atoms], np.int32),
            pos=np.concatenate([a.pos for a in self.atoms]).astype(np.float64),
            nsupp=np.array([len(a.supp_cell) for a in self.atoms], np.int32),
            supp_cell=np.concatenate([a.supp_cell for a in self.atoms]).astype(np.int32),
            supp_img=np.concatenate([a.supp_img.reshape(-1) for a in self.atoms]).astype(np.int32),
            pvals=np.concatenate([a.pvals.reshape(-1) for a in self.atoms]).astype(np.float64),
            delta=np.concatenate([a.delta.reshape(-1) for a in self.atoms]).astype(np.complex128),
        )

    def with_(self, **kw) -> "Problem":
        d = dict(self.__dict__)
        d.update(kw)
        return Problem(**d)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(seed * 100 + stream)


def _support(pos, ncell, h, periodic, rc):
    """Cells (with lattice image shift) whose box intersects the ball |r-R-L| < rc."""
    nx, ny, nz = ncell
    box = np.array([nx * h[0], ny * h[1], nz * h[2]])
    imgs = [[-1, 0, 1] if periodic[d] else [0] for d in range(3)]
    cells, shifts = [], []
    for iz in imgs[2]:
        for iy in imgs[1]:
            for ix in imgs[0]:
                L = np.array([ix, iy, iz]) * box
                c = pos + L
                lo = [max(0, int(math.floor((c[d] - rc) / h[d]))) for d in range(3)]
                hi = [min(ncell[d] - 1, int(math.floor((c[d] + rc) / h[d]))) for d in range(3)]
                for cz in range(lo[2], hi[2] + 1):
                    for cy in range(lo[1], hi[1] + 1):
                        for cx in range(lo[0], hi[0] + 1):
                            cmin = np.array([cx * h[0], cy * h[1], cz * h[2]])
                            cmax = cmin + np.array(h)
                            dd = np.maximum(np.maximum(cmin - c, 0.0), c - cmax)
                            if float(np.sqrt((dd * dd).sum())) < rc:
                                cells.append((cz * ny + cy) * nx + cx)
                                shifts.append((ix, iy, iz))
    return np.array(cells, np.int32), np.array(shifts, np.int32).reshape(-1, 3)


def make_problem(ncell=(2, 2, 2), h=(1.0, 1.0, 1.0), p=2, nq=None, periodic=(1, 1, 1),
                 k=(0.0, 0.0, 0.0), atom_pos=None, natoms=0, channels=((0.5, 1),),
                 well_depth=2.0, well_width=0.8, bmax=0.1, nmodes=3, rc=2.0,
                 delta_std=0.1, seed=0, name="", well_cutoff=None) -> Problem:
    """Draw one synthetic problem.

    channels: sequence of (sigma, l) radial channels; each contributes 2l+1
      projectors r^l exp(-r^2/(2 sigma^2)) Y_lm, L2-normalised on [0, rc].
    atom_pos: explicit positions (natoms, 3) or None to draw ``natoms``
      uniformly in the box (seed stream 1).
    well_cutoff: None sums every well over every point; a radius (bohr) sums each
      well only over the cells within that distance of the atom (minimum image),
      for meshes where atoms x points is too large to sum in full.
    """
    ncell = tuple(int(n) for n in ncell)
    h = tuple(float(x) for x in h)
    periodic = tuple(bool(b) for b in periodic)
    if nq is None:
        nq = p + 2
    E = int(np.prod(ncell))
    box = np.array([n * hh for n, hh in zip(ncell, h)])
    if atom_pos is None:
        r1 = _rng(seed, 1)
        atom_pos = r1.uniform(0.0, 1.0, size=(natoms, 3)) * box
    atom_pos = np.asarray(atom_pos, np.float64).reshape(-1, 3)

    rq = _quad_coords(ncell, h, nq).reshape(-1, 3)          # [E*nq^3, 3]
    per = np.array(periodic)

    # ---- V_eff: Gaussian wells (image sum for small boxes, minimum image otherwise)
    V = np.zeros(rq.shape[0])
    small = box[per].size and box[per].min() < 8 * well_width
    for R in (atom_pos if well_cutoff is None else []):
        if small:
            for iz in ([-1, 0, 1] if per[2] else [0]):
                for iy in ([-1, 0, 1] if per[1] else [0]):
                    for ix in ([-1, 0, 1] if per[0] else [0]):
                        d = rq - R - np.array([ix, iy, iz]) * box
                        V -= well_depth * np.exp(-(d * d).sum(-1) / (2 * well_width ** 2))
        else:
            d = rq - R
            d[:, per] -= box[per] * np.round(d[:, per] / box[per])
            V -= well_depth * np.exp(-(d * d).sum(-1) / (2 * well_width ** 2))

    if well_cutoff is not None:
        nq3 = nq ** 3
        for R in atom_pos:
            sc, si = _support(R, ncell, h, periodic, well_cutoff)
            for c, L in zip(sc, si):
                pts = slice(int(c) * nq3, (int(c) + 1) * nq3)
                d = rq[pts] - R - L * box
                V[pts] -= well_depth * np.exp(-(d * d).sum(-1) / (2 * well_width ** 2))

    # ---- B_xc: a few low-frequency Fourier modes, rescaled to max |B| = bmax
    r2 = _rng(seed, 2)
    B = np.zeros((rq.shape[0], 3))
    if nmodes > 0 and bmax > 0:
        choices = [np.array(n) for n in np.ndindex(3, 3, 3) if n != (1, 1, 1)]
        for d in range(3):
            for _ in range(nmodes):
                n = choices[r2.integers(len(choices))] - 1
                G = 2 * np.pi * n / box
                a = r2.normal()
                ph = r2.uniform(0, 2 * np.pi)
                B[:, d] += a * np.cos(rq @ G + ph)
        mag = np.sqrt((B * B).sum(-1)).max()
        if mag > 0:
            B *= bmax / mag

    # ---- projectors
    r3 = _rng(seed, 3)
    atoms = []
    chan_norm = [(_radial_norm(l, s, rc), s, l) for s, l in channels]
    npj = sum(2 * l + 1 for _, l in channels)
    rq_cells = rq.reshape(E, nq ** 3, 3)
    for R in atom_pos:
        sc, si = _support(R, ncell, h, periodic, rc)
        pv = np.zeros((len(sc), nq ** 3, npj))
        for s, (c, L) in enumerate(zip(sc, si)):
            d = rq_cells[c] - R - L * box
            r = np.sqrt((d * d).sum(-1))
            inside = r < rc
            col = 0
            for nrm, sig, l in chan_norm:
                rad = nrm * r ** l * np.exp(-r * r / (2 * sig * sig)) * inside
                Y = _real_sph_harm(l, d)
                pv[s, :, col:col + 2 * l + 1] = rad[:, None] * Y
                col += 2 * l + 1
        A = r3.normal(0, delta_std, (2 * npj, 2 * npj)) + 1j * r3.normal(0, delta_std, (2 * npj, 2 * npj))
        delta = 0.5 * (A + A.conj().T)
        atoms.append(Atom(pos=R.copy(), npj=npj, supp_cell=sc, supp_img=si, pvals=pv, delta=delta))

    return Problem(ncell=ncell, h=h, p=p, nq=nq, periodic=periodic,
                   k=np.asarray(k, np.float64), veff=V.reshape(E, nq ** 3),
                   bx=np.ascontiguousarray(B[:, 0].reshape(E, nq ** 3)),
                   by=np.ascontiguousarray(B[:, 1].reshape(E, nq ** 3)),
                   bz=np.ascontiguousarray(B[:, 2].reshape(E, nq ** 3)),
                   atoms=atoms, name=name, seed=seed)


def random_block(nnodes: int, nvec: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Spinor block X[M][2][nvec], real and imaginary parts uniform in [-1, 1)."""
    r = _rng(seed, 0)
    re = r.uniform(-1.0, 1.0, size=(nnodes, 2, nvec))
    im = r.uniform(-1.0, 1.0, size=(nnodes, 2, nvec))
    return (re + 1j * im).astype(dtype)


def random_start(nnodes: int, seed: int) -> np.ndarray:
    """Lanczos start spinor v0[M][2], uniform [-1, 1) parts (stream 4)."""
    r = _rng(seed, 4)
    return r.uniform(-1, 1, (nnodes, 2)) + 1j * r.uniform(-1, 1, (nnodes, 2))


# ----------------------------------------------------------------------------
# the paper-shaped workloads
# ----------------------------------------------------------------------------
SPD_CHANNELS = ((0.5, 0), (0.65, 0), (0.5, 1), (0.65, 1), (0.5, 2), (0.65, 2))  # 18 projectors
P_CHANNEL = ((0.5, 1),)                                                            # 3 projectors


def _jittered_lattice(n, spacing, jitter, seed, origin=(0.0, 0.0, 0.0)):
    """Sites of an n (int or 3 ints) lattice of the given spacing (number or 3 numbers)
    from ``origin``, cell-centred, each moved by uniform(-jitter, jitter) (seed stream 1)."""
    r = _rng(seed, 1)
    n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    sp = np.broadcast_to(np.asarray(spacing, np.float64), (3,))
    g = np.stack(np.meshgrid(*[np.arange(m) for m in n3], indexing="ij"), -1).reshape(-1, 3)
    g = (g + 0.5) * sp + np.asarray(origin, np.float64)
    return g + r.uniform(-jitter, jitter, g.shape)


def mp_kpoints(n1, n2, n3, box):
    """Monkhorst-Pack grid k_i = (2i - n - 1)/(2n) * b, b = 2 pi / L."""
    ks = []
    for i3 in range(1, n3 + 1):
        for i2 in range(1, n2 + 1):
            for i1 in range(1, n1 + 1):
                f = np.array([(2 * i1 - n1 - 1) / (2 * n1), (2 * i2 - n2 - 1) / (2 * n2),
                              (2 * i3 - n3 - 1) / (2 * n3)])
                ks.append(f * 2 * np.pi / np.asarray(box))
    return ks


CONFIGS = {
    # 6^3 cells, p=4, nq=6, Gamma, 4 atoms with one l=1 channel, 32 vectors, m=10, 3 cycles
    "cube6_p4": dict(ncell=(6, 6, 6), p=4, nq=6, natoms=4, channels=P_CHANNEL, nvec=32, degree=10,
               cycles=3, lanczos=10, kgrid=(1, 1, 1)),
    # 16^3 cells, p=6, nq=8, 64 atoms (jittered 4^3 lattice), 18 projectors, 256 vectors, m=20, 2x2x1 k
    "cube16_p6": dict(ncell=(16, 16, 16), p=6, nq=8, lattice=(4, 4.0, 0.3), channels=SPD_CHANNELS,
               nvec=256, degree=20, cycles=1, lanczos=10, kgrid=(2, 2, 1)),
    # backward workload: the cube16_p6 mesh and atoms, 128 vectors, m=20
    "cube16_p6_grad": dict(ncell=(16, 16, 16), p=6, nq=8, lattice=(4, 4.0, 0.3), channels=SPD_CHANNELS,
               nvec=128, degree=20, cycles=0, lanczos=10, kgrid=(1, 1, 1)),
    # semi-periodic slab: 40x40x20 cells (240x240x119 = 6,854,400 free nodes), p=6, periodic in
    # x and y, Dirichlet in z with 4 vacuum cells on each side; 640 atoms on a jittered
    # 16x8x5 lattice inside the slab (z in [4, 16] bohr); 20,000 states filtered in blocks of
    # 256 at m=30, Gamma; wells summed within 6 widths of each atom
    "slab40_p6": dict(ncell=(40, 40, 20), p=6, nq=8, periodic=(1, 1, 0),
                      slab_lattice=((16, 8, 5), (2.5, 5.0, 2.4), 0.3, (0.0, 0.0, 4.0)),
                      channels=SPD_CHANNELS, nvec=256, degree=30, nstates=20000, cycles=1,
                      lanczos=10, kgrid=(1, 1, 1), well_cutoff=4.8),
}


def config(name: str, seed: int = 0, kindex: int = 0, **over) -> Problem:
    """Problem for a named workload (cube6_p4, cube16_p6, cube16_p6_grad, slab40_p6) at
    k-point ``kindex``."""
    c = dict(CONFIGS[name])
    c.update(over)
    h = (1.0, 1.0, 1.0)
    box = [n * hh for n, hh in zip(c["ncell"], h)]
    ks = mp_kpoints(*c["kgrid"], box)
    pos = None
    natoms = c.get("natoms", 0)
    if "lattice" in c:
        n, sp, jit = c["lattice"]
        pos = _jittered_lattice(n, sp, jit, seed)
    if "slab_lattice" in c:
        n, sp, jit, origin = c["slab_lattice"]
        pos = _jittered_lattice(n, sp, jit, seed, origin)
    return make_problem(ncell=c["ncell"], h=h, p=c["p"], nq=c["nq"],
                        periodic=c.get("periodic", (1, 1, 1)), k=ks[kindex], atom_pos=pos,
                        natoms=natoms, channels=c["channels"], seed=seed, name=name,
                        well_cutoff=c.get("well_cutoff"))


def batch16_systems(seed: int = 0):
    """Sixteen independent periodic systems of uneven size for the batched filter:
    8^3..14^3 cells, p in {4, 5, 6}, 64..320 vectors, 8..40 atoms with s, p, d
    projectors (18 per atom), Chebyshev degree 12..24 (seed stream 6)."""
    r = _rng(seed, 6)
    out = []
    for i in range(16):
        n = int(r.integers(8, 15))
        out.append(dict(ncell=(n, n, n), p=int(r.choice([4, 5, 6])), nvec=int(r.integers(64, 321)),
                        natoms=int(r.integers(8, 41)), degree=int(r.integers(12, 25)),
                        seed=seed * 1000 + i))
    return out


def batch16_problem(desc) -> Problem:
    """The Problem of one batch16_systems() entry (Gamma point, 1 bohr cells)."""
    return make_problem(ncell=desc["ncell"], h=(1.0, 1.0, 1.0), p=desc["p"], nq=desc["p"] + 2,
                        periodic=(1, 1, 1), k=(0.0, 0.0, 0.0), natoms=desc["natoms"],
                        channels=SPD_CHANNELS, seed=desc["seed"], name="batch16")
