"""Seeded synthetic inputs for GCMe systems.

This module is shared by the FP64 oracle (``oracle/``) and by the CUDA path
(``paper_2403_08148_gb300``).  It only draws random inputs and fixes run
parameters (box, charges, bonds, velocities, cutoff, grid, Ewald splitting
parameter); it evaluates none of the model's energies or forces.

Reduced units throughout: kT = 1, length d (the bead diameter), mass m = 1,
charges in units of e.  The workloads mirror the systems the paper studies:
bulk GCMe fluids at the paper's densities (Parametrization section) and a
polyelectrolyte / counterion / solvent mixture between planar electrodes
(Illustrative example section).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 2403081480

GEOM_BULK = 0
GEOM_SLAB_NM = 1  # nonmetal electrodes: tripled box + Yeh-Berkowitz term
GEOM_SLAB_PC = 2  # perfectly conducting electrodes: doubled box + images

GEOM_NAMES = {GEOM_BULK: "bulk", GEOM_SLAB_NM: "slab_nm", GEOM_SLAB_PC: "slab_pc"}


# ---------------------------------------------------------------------------
# Physical constants and reduced units (Parametrization section: d = 2 sigma,
# N_m = 4 water molecules per bead, rho = 2.5 d^-3, water at 300 K, eps_r=78).
# ---------------------------------------------------------------------------
_E = 1.602176634e-19
_EPS0 = 8.8541878128e-12
_KB = 1.380649e-23
_NA = 6.02214076e23


def bead_diameter_nm(rho: float = 2.5, n_m: int = 4, d_water_nm: float = 0.275) -> float:
    """d = (rho d^3 N_m)^(1/3) x 0.275 nm (Parametrization section)."""
    return (rho * n_m) ** (1.0 / 3.0) * d_water_nm


def bead_mass_gmol(n_m: int = 4, m_water: float = 18.02) -> float:
    return n_m * m_water


def time_unit_ps(rho: float = 2.5, n_m: int = 4, temp: float = 300.0) -> float:
    """tau = sqrt(m d^2 / (N_A kT)) (Parametrization section)."""
    d = bead_diameter_nm(rho, n_m) * 1e-9
    m = bead_mass_gmol(n_m) * 1e-3
    return math.sqrt(m * d * d / (_NA * _KB * temp)) * 1e12


def bjerrum_length_d(eps_r: float = 78.0, temp: float = 300.0,
                     rho: float = 2.5, n_m: int = 4) -> float:
    """lambda_B = e^2 / (4 pi eps0 eps_r kT), in units of d (~1.2053)."""
    lb_m = _E * _E / (4.0 * math.pi * _EPS0 * eps_r * _KB * temp)
    return lb_m / (bead_diameter_nm(rho, n_m) * 1e-9)


LB_WATER = bjerrum_length_d()


def ewald_kappa(rc: float, delta: float = 5e-4) -> float:
    """Splitting parameter from the tolerance rule erfc(kappa rc) ~ 2 delta.

    The paper leaves the screening width G (kappa = 1/(sqrt(2) G)) free; this
    is the conventional choice kappa = sqrt(-ln(2 delta)) / rc.
    """
    return math.sqrt(-math.log(2.0 * delta)) / rc


def smooth_size(n: int, radices=(2, 3, 5)) -> int:
    """Smallest integer >= n whose prime factors are all in ``radices``."""
    m = max(int(n), 1)
    while True:
        k = m
        for r in radices:
            while k % r == 0:
                k //= r
        if k == 1:
            return m
        m += 1


# ---------------------------------------------------------------------------
# System description
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class System:
    """One GCMe system: real beads only (images are derived, never stored)."""

    name: str
    geometry: int
    box: np.ndarray          # (3,) float64, full periodic box
    pos: np.ndarray          # (n,3) float64
    vel: np.ndarray          # (n,3) float64
    q: np.ndarray            # (n,) float64 charge numbers z_i
    bonds: np.ndarray        # (nb,2) int32
    A: float = 25.0          # Gaussian-core amplitude A_ij (kT d^3)
    sigma: float = 0.5       # mass smearing radius sigma_i (d)
    a: float = 0.5           # charge smearing radius a_i (d)
    lB: float = LB_WATER     # Bjerrum length (d)
    rc: float = 3.0          # real-space cutoff (d)
    kappa: float = 0.0       # Ewald splitting parameter (1/d)
    K: tuple = (32, 32, 32)  # PME grid
    order: int = 5           # B-spline order p
    dt: float = 0.01         # time step (tau)
    bond_k: float = 100.0    # harmonic bond force constant (kT/d^2)
    bond_r0: float = 1.0     # bond rest length (d)
    H: float = 0.0           # slab height for slab geometries (d)
    wall_A: float = 0.0      # continuum wall amplitude A n_s (kT/d^2 x d^3)
    wall_sigma2: float = 0.0  # sigma_w^2 = sigma_i^2 + sigma_e^2
    # several species (optional): type of each bead and per-type tables;
    # None means one species with the scalars A, sigma, a above
    types: Optional[np.ndarray] = None   # (n,) int32 in [0, nt)
    A_tab: Optional[np.ndarray] = None   # (nt, nt) A_ij, symmetric
    sig_tab: Optional[np.ndarray] = None  # (nt,) sigma_i
    a_tab: Optional[np.ndarray] = None   # (nt,) a_i
    frozen_mask: int = 0                 # bit t: beads of species t do not move

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ntypes(self) -> int:
        return 0 if self.types is None else int(self.A_tab.shape[0])

    @property
    def n_charged(self) -> int:
        return int(np.count_nonzero(self.q))

    def copy(self) -> "System":
        cp = lambda a: None if a is None else a.copy()
        return dataclasses.replace(
            self, box=self.box.copy(), pos=self.pos.copy(), vel=self.vel.copy(),
            q=self.q.copy(), bonds=self.bonds.copy(), types=cp(self.types),
            A_tab=cp(self.A_tab), sig_tab=cp(self.sig_tab), a_tab=cp(self.a_tab))


def _rng(index: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + index, sub]))


def _velocities(rng, n, kT=1.0, m=1.0):
    v = rng.normal(0.0, math.sqrt(kT / m), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
    return v


def _random_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _reflect(x, lo, hi):
    """Fold coordinates back into [lo, hi] by mirror reflection."""
    w = hi - lo
    y = np.mod(x - lo, 2.0 * w)
    y = np.where(y > w, 2.0 * w - y, y)
    return lo + y


def _chains(rng, n_chains, length, box, bond=1.0, zlim=None):
    """Random walks with fixed step ``bond`` from uniform starts."""
    pos = np.empty((n_chains, length, 3))
    start = rng.uniform(0.0, 1.0, size=(n_chains, 3)) * box
    if zlim is not None:
        start[:, 2] = rng.uniform(zlim[0], zlim[1], size=n_chains)
    pos[:, 0] = start
    for k in range(1, length):
        step = _random_unit(rng, n_chains) * bond
        nxt = pos[:, k - 1] + step
        if zlim is not None:
            nxt[:, 2] = _reflect(nxt[:, 2], zlim[0], zlim[1])
        pos[:, k] = nxt
    bonds = []
    for c in range(n_chains):
        b0 = c * length
        for k in range(length - 1):
            bonds.append((b0 + k, b0 + k + 1))
    return pos.reshape(-1, 3), np.asarray(bonds, dtype=np.int32).reshape(-1, 2)


def _wrap(pos, box, periodic=(True, True, True)):
    out = pos.copy()
    for ax in range(3):
        if periodic[ax]:
            out[:, ax] = np.mod(out[:, ax], box[ax])
    return out


def _wall_params(A: float, sigma: float, sigma_e: float = 0.25,
                 lattice: float = 0.5):
    """Continuum limit of one hexagonal layer of electrode beads of size d/2.

    n_s = 2/(sqrt(3) b^2) beads per unit area for a triangular layer of
    spacing b = d/2; sigma_w^2 = sigma_i^2 + sigma_e^2.  Returned as the
    pair (A n_s, sigma_w^2) consumed by the wall term.
    """
    n_s = 2.0 / (math.sqrt(3.0) * lattice * lattice)
    return A * n_s, sigma * sigma + sigma_e * sigma_e


def make_bulk(n: int, rho: float = 3.0, charged_frac: float = 0.1,
              seed_index: int = 1, K=None, spacing: float = 1.0,
              name: Optional[str] = None, rc: float = 3.0,
              order: int = 5, dt: float = 0.01, sub: int = 0) -> System:
    """Cubic periodic GCMe fluid: uniform positions, +/-1 on a random subset."""
    rng = _rng(seed_index, sub)
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * box
    nq = int(round(charged_frac * n))
    nq -= nq % 2
    perm = rng.permutation(n)
    q = np.zeros(n)
    q[perm[: nq // 2]] = 1.0
    q[perm[nq // 2: nq]] = -1.0
    vel = _velocities(rng, n)
    if K is None:
        K = tuple(smooth_size(int(math.ceil(L / spacing))) for _ in range(3))
    return System(name=name or f"bulk_n{n}", geometry=GEOM_BULK, box=box,
                  pos=pos, vel=vel, q=q, bonds=np.zeros((0, 2), np.int32),
                  rc=rc, kappa=ewald_kappa(rc), K=tuple(int(k) for k in K),
                  order=order, dt=dt)


def make_polyelectrolyte(n_chains: int = 100, chain_len: int = 50,
                         n_solvent: int = 22000, rho: float = 3.0,
                         seed_index: int = 2, K=(64, 64, 64),
                         name: str = "polyelectrolyte", sub: int = 0,
                         box=None) -> System:
    """Bulk polyanion solution: chains of -1 beads, +1 counterions, solvent."""
    rng = _rng(seed_index, sub)
    n_mono = n_chains * chain_len
    n = n_mono + n_mono + n_solvent
    if box is None:
        L = (n / rho) ** (1.0 / 3.0)
        box = np.array([L, L, L])
    box = np.asarray(box, dtype=np.float64)
    cpos, bonds = _chains(rng, n_chains, chain_len, box)
    other = rng.uniform(0.0, 1.0, size=(n - n_mono, 3)) * box
    pos = _wrap(np.concatenate([cpos, other]), box)
    q = np.zeros(n)
    q[:n_mono] = -1.0
    q[n_mono: 2 * n_mono] = 1.0
    vel = _velocities(rng, n)
    return System(name=name, geometry=GEOM_BULK, box=box, pos=pos, vel=vel,
                  q=q, bonds=bonds, kappa=ewald_kappa(3.0),
                  K=tuple(int(k) for k in K))


def make_slab(geometry: int, n_chains: int = 200, chain_len: int = 50,
              n_solvent: int = 44000, box=(30.0, 30.0, 90.0),
              K=(64, 64, 192), seed_index: int = 3, sub: int = 0,
              margin: float = 0.75, n_counter: Optional[int] = None,
              name: Optional[str] = None) -> System:
    """Polyelectrolyte between two planar electrodes at z = 0 and z = H.

    Nonmetal electrodes: the box is three times the slab height (H = Lz/3).
    Perfectly conducting electrodes: the box is twice the slab height
    (H = Lz/2); the lower half holds the mirror images.
    """
    rng = _rng(seed_index, sub)
    box = np.asarray(box, dtype=np.float64)
    H = box[2] / 3.0 if geometry == GEOM_SLAB_NM else box[2] / 2.0
    zlim = (margin, H - margin)
    n_mono = n_chains * chain_len
    if n_counter is None:
        n_counter = n_mono
    if n_mono > 0:
        cpos, bonds = _chains(rng, n_chains, chain_len, box, zlim=zlim)
    else:
        cpos, bonds = np.zeros((0, 3)), np.zeros((0, 2), np.int32)
    n_other = n_counter + n_solvent
    other = rng.uniform(0.0, 1.0, size=(n_other, 3)) * box
    other[:, 2] = rng.uniform(zlim[0], zlim[1], size=n_other)
    pos = _wrap(np.concatenate([cpos, other]), box, periodic=(True, True, False))
    n = pos.shape[0]
    q = np.zeros(n)
    q[:n_mono] = -1.0
    q[n_mono: n_mono + n_counter] = 1.0
    vel = _velocities(rng, n)
    wA, ws2 = _wall_params(25.0, 0.5)
    return System(name=name or GEOM_NAMES[geometry], geometry=geometry,
                  box=box, pos=pos, vel=vel, q=q, bonds=bonds,
                  kappa=ewald_kappa(3.0), K=tuple(int(k) for k in K), H=H,
                  wall_A=wA, wall_sigma2=ws2)


def make_slab_fluid(geometry: int, n: int, rho: float = 3.0,
                    charged_frac: float = 0.1, seed_index: int = 5,
                    sub: int = 0, spacing: float = 1.0, aspect: float = 2.0,
                    margin: float = 0.75) -> System:
    """Simple charged fluid in a slab: height H = aspect x lateral side."""
    rng = _rng(seed_index, sub)
    Lxy = (n / (rho * aspect)) ** (1.0 / 3.0)
    H = aspect * Lxy
    Lz = 3.0 * H if geometry == GEOM_SLAB_NM else 2.0 * H
    box = np.array([Lxy, Lxy, Lz])
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * box
    pos[:, 2] = rng.uniform(margin, H - margin, size=n)
    nq = int(round(charged_frac * n))
    nq -= nq % 2
    perm = rng.permutation(n)
    q = np.zeros(n)
    q[perm[: nq // 2]] = 1.0
    q[perm[nq // 2: nq]] = -1.0
    vel = _velocities(rng, n)
    K = tuple(smooth_size(int(math.ceil(b / spacing))) for b in box)
    wA, ws2 = _wall_params(25.0, 0.5)
    return System(name=f"{GEOM_NAMES[geometry]}_n{n}", geometry=geometry,
                  box=box, pos=pos, vel=vel, q=q,
                  bonds=np.zeros((0, 2), np.int32), kappa=ewald_kappa(3.0),
                  K=K, H=H, wall_A=wA, wall_sigma2=ws2)


# ---------------------------------------------------------------------------
# The five workloads
def make_mixture(n: int, fractions, charges, A_tab, sig_tab, a_tab, rho: float = 3.0,
                 seed_index: int = 9, K=None, geometry: int = GEOM_BULK,
                 sub: int = 0) -> System:
    """Fluid of several species (Supporting Information, Flory-Huggins
    section: A/B blends with A_AB = A_AA + Delta A; species may also differ
    in sigma_i and a_i).  Species t takes a fraction fractions[t] of the
    beads and charge charges[t]; the charged species' counts are adjusted so
    that the system is neutral.  Uniform positions; bulk, or a slab between
    walls at z = 0 and H (box L x L x 3H nonmetal, L x L x 2H conducting)."""
    rng = _rng(seed_index, sub)
    fr = np.asarray(fractions, float) / np.sum(fractions)
    ch = np.asarray(charges, float)
    cnt = np.floor(fr * n).astype(int)
    cnt[0] += n - cnt.sum()
    # neutrality: move beads between the first positive and first negative
    # charged species until sum(cnt * ch) = 0 (integer charges)
    pos_t = [t for t in range(len(ch)) if ch[t] > 0]
    neg_t = [t for t in range(len(ch)) if ch[t] < 0]
    if pos_t and neg_t:
        tp, tn = pos_t[0], neg_t[0]
        for _ in range(4 * n):
            net = float(np.sum(cnt * ch))
            if abs(net) < 1e-9:
                break
            if net > 0:
                cnt[tp] -= 1
                cnt[0] += 1
            else:
                cnt[tn] -= 1
                cnt[0] += 1
    types = np.repeat(np.arange(len(ch)), cnt).astype(np.int32)
    rng.shuffle(types)
    q = ch[types].copy()
    if geometry == GEOM_BULK:
        L = (n / rho) ** (1.0 / 3.0)
        box = np.array([L, L, L])
        pos = rng.uniform(0.0, 1.0, size=(n, 3)) * box
        H, wA, ws2 = 0.0, 0.0, 0.0
    else:  # slab of height H = 2 L between walls, as make_slab_fluid
        L = (n / (rho * 2.0)) ** (1.0 / 3.0)
        H = 2.0 * L
        mult = 3.0 if geometry == GEOM_SLAB_NM else 2.0
        box = np.array([L, L, mult * H])
        pos = rng.uniform(0.0, 1.0, size=(n, 3)) * np.array([L, L, 0.0])
        pos[:, 2] = rng.uniform(0.75, H - 0.75, size=n)
        wA, ws2 = _wall_params(25.0, 0.5)
    if K is None:
        K = tuple(smooth_size(int(math.ceil(b))) for b in box)
    return System(name=f"mixture_n{n}", geometry=geometry, box=box, pos=pos,
                  vel=_velocities(rng, n), q=q, bonds=np.zeros((0, 2), np.int32),
                  kappa=ewald_kappa(3.0), K=tuple(int(k) for k in K), H=H,
                  wall_A=wA, wall_sigma2=ws2, types=types,
                  A_tab=np.asarray(A_tab, float), sig_tab=np.asarray(sig_tab, float),
                  a_tab=np.asarray(a_tab, float))


def hcp_layer(nx: int, ny: int, b: float = 0.5, z: float = 0.0) -> np.ndarray:
    """Triangular (close-packed) layer of nx x ny points of spacing b in the
    x-y plane at height z; rows alternate by b/2 so that the layer is
    periodic in a box of nx b by ny b sqrt(3)/2 (ny even)."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (i + 0.5 * (j % 2)) * b
    y = j * b * math.sqrt(3.0) / 2.0
    return np.stack([x.ravel(), y.ravel(), np.full(x.size, z)], axis=1)


def make_electrode_slab(geometry: int, nx: int = 16, ny: int = 18, H: float = 20.0,
                        n_chains: int = 10, chain_len: int = 20, rho: float = 3.0,
                        sigma_q: float = 0.005 * bead_diameter_nm() ** 2,
                        seed_index: int = 10, K=None, margin: float = 0.75) -> System:
    """Fluid between explicit electrodes (Illustrative example and the
    performance table's slab systems): at z = 0 and z = H one close-packed
    layer each of beads of size d/2 (sigma = a = 0.25, species 1, frozen)
    with spacing d/2, carrying +sigma_q and -sigma_q per unit area (sigma_q
    in e/d^2; default 0.005 e/nm^2); polyanion chains (-1) with counterions
    (+1) and solvent (species 0) at density rho in between.  Box nx/2 by
    ny sqrt(3)/4 by 3H (nonmetal) or 2H (image charges); no continuum wall."""
    rng = _rng(seed_index)
    b = 0.5
    Lx, Ly = nx * b, ny * b * math.sqrt(3.0) / 2.0
    box = np.array([Lx, Ly, (3.0 if geometry == GEOM_SLAB_NM else 2.0) * H])
    lo, hi = hcp_layer(nx, ny, b, 0.0), hcp_layer(nx, ny, b, H)
    ne = lo.shape[0]
    q_e = sigma_q * (Lx * Ly) / ne
    n_fluid = int(round(rho * Lx * Ly * (H - 2 * margin)))
    n_mono = n_chains * chain_len
    zlim = (margin, H - margin)
    cpos, bonds = _chains(rng, n_chains, chain_len, box, zlim=zlim)
    n_other = n_fluid - n_mono
    other = rng.uniform(0.0, 1.0, size=(n_other, 3)) * box
    other[:, 2] = rng.uniform(zlim[0], zlim[1], size=n_other)
    fluid = _wrap(np.concatenate([cpos, other]), box, periodic=(True, True, False))
    pos = np.concatenate([fluid, lo, hi])
    n = pos.shape[0]
    q = np.zeros(n)
    q[:n_mono] = -1.0
    q[n_mono: 2 * n_mono] = 1.0
    q[n_fluid: n_fluid + ne] = q_e
    q[n_fluid + ne:] = -q_e
    types = np.zeros(n, np.int32)
    types[n_fluid:] = 1
    vel = _velocities(rng, n)
    vel[n_fluid:] = 0.0
    if K is None:
        K = tuple(smooth_size(int(math.ceil(v))) for v in box)
    return System(name=f"electrodes_{GEOM_NAMES[geometry]}_n{n}", geometry=geometry, box=box,
                  pos=pos, vel=vel, q=q, bonds=bonds, kappa=ewald_kappa(3.0),
                  K=tuple(int(k) for k in K), H=H, wall_A=0.0, wall_sigma2=0.0, types=types,
                  A_tab=np.full((2, 2), 25.0), sig_tab=np.array([0.5, 0.25]),
                  a_tab=np.array([0.5, 0.25]), frozen_mask=1 << 1)


# ---------------------------------------------------------------------------
def config1() -> System:
    """Plain GCMe fluid: N=3000, rho=3 (L=10), 10% charged, grid 32^3."""
    s = make_bulk(3000, rho=3.0, charged_frac=0.1, seed_index=1, K=(32, 32, 32),
                  name="c1_bulk_n3000")
    return s


def config2() -> System:
    """Bulk polyelectrolyte: N=32000, 100 chains x 50, 5000 counterions, 64^3."""
    return make_polyelectrolyte(100, 50, 22000, rho=3.0, seed_index=2,
                                K=(64, 64, 64), name="c2_polyelectrolyte_n32000")


def config3(geometry: int) -> System:
    """Slab: 30x30x90 box, N=64000, 200 chains x 50, grid 64x64x192."""
    return make_slab(geometry, 200, 50, 44000, box=(30.0, 30.0, 90.0),
                     K=(64, 64, 192), seed_index=3,
                     sub=0 if geometry == GEOM_SLAB_NM else 1,
                     name=f"c3_{GEOM_NAMES[geometry]}_n64000")


def config4_sizes(n_sys: int = 256, lo: int = 500, hi: int = 8000) -> List[int]:
    rng = _rng(4, 0)
    u = rng.uniform(math.log(lo), math.log(hi), size=n_sys)
    return [int(math.floor(math.exp(x))) for x in u]


def config4(n_sys: int = 256, lo: int = 500, hi: int = 8000) -> List[System]:
    """256 independent bulk systems, N log-uniform in [500, 8000]."""
    sizes = config4_sizes(n_sys, lo, hi)
    return [make_bulk(n, rho=3.0, charged_frac=0.1, seed_index=4, sub=1 + i,
                      name=f"c4_sys{i}_n{n}") for i, n in enumerate(sizes)]


def config5_requests(n_req: int, rate: float = 200.0, lo: int = 1000,
                     hi: int = 64000, steps: int = 1000, seed_sub: int = 0):
    """Poisson arrivals of trajectory-segment requests (arrival time, spec).

    Geometry mix: 50% bulk, 25% nonmetal slab, 25% conducting slab.
    Returns a list of (t_arrival_s, System, nsteps).
    """
    rng = _rng(5, seed_sub)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_req)))
    kinds = rng.choice([GEOM_BULK, GEOM_BULK, GEOM_SLAB_NM, GEOM_SLAB_PC],
                       size=n_req)
    out = []
    for i in range(n_req):
        n = int(sizes[i])
        g = int(kinds[i])
        if g == GEOM_BULK:
            s = make_bulk(n, seed_index=5, sub=1000 + i, name=f"req{i}_bulk_n{n}")
        else:
            s = make_slab_fluid(g, n, seed_index=5, sub=1000 + i)
        out.append((float(t[i]), s, int(steps)))
    return out
