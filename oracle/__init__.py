"""FP64 CPU oracle for the GCMe nonbonded force/energy path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plainly written
reference that the CUDA library is checked against.  It shares no code with
the CUDA path (``paper_2403_08148_gb300``) and neither imports the other;
the only common module is ``synth`` (seeded inputs, no model arithmetic).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use it.

The numerical core is ``gcme_oracle.c`` (plain loops, FP64, optional
OpenMP), compiled on first use with gcc.  This module assembles the pieces
of the paper's energy for each boundary condition:

* bulk periodic:  U = U_gc + U_real + U_recip + U_corr + U_self (Eq. ewald)
  + harmonic bonds (Illustrative example section);
* nonmetal slab (electrode permittivity equal to the solvent's, so image
  charges vanish): tripled box + Yeh-Berkowitz term + electrode walls;
* perfectly conducting slab (method of image charges section): a doubled
  box holding every charged bead's mirror image (x, y, -z) with charge -z_i;
  the physical electrostatic energy is half that of the doubled system,
  forces on the real beads are the doubled-system forces.

Parity status of each function is listed in its docstring; all are pinned
by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

from synth import GEOM_BULK, GEOM_SLAB_NM, GEOM_SLAB_PC, System

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcme_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile gcme_oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_bspline.restype = ctypes.c_double
            L.orc_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_pair_set.restype = ctypes.c_int64
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
# Thin wrappers over the C routines
# ---------------------------------------------------------------------------
def wrap(pos, box):
    pos = _f64(pos)
    out = np.empty_like(pos)
    lib().orc_wrap(ctypes.c_int64(pos.shape[0]), _p(pos), _p(_f64(box)), _p(out))
    return out


def bspline(p: int, u: float) -> float:
    """Cardinal B-spline M_p(u) (Essmann et al. 1995, recursion)."""
    return float(lib().orc_bspline(int(p), float(u)))


def bspline_moduli(p: int, K: int) -> np.ndarray:
    out = np.empty(K)
    lib().orc_bspline_moduli(ctypes.c_int(p), ctypes.c_int(K), _p(out))
    return out


def cell_counts(box, rc: float, factor: int = 1, margin: float = 1e-4):
    """Cells per axis: floor(L / ((rc / factor) (1 + margin))), at least 1.

    The margin keeps every cell side above rc / factor by far more than FP32
    rounding of coordinates, so the stencil of +-factor cells reaches every
    in-cutoff pair.
    """
    return np.array([max(1, int(np.floor(b / ((rc / factor) * (1.0 + margin))))) for b in box],
                    dtype=np.int32)


def cell_list(pos, box, nc, cls, ncls: int = 3):
    """Counting-sort cell list; beads inside a cell ordered by (class, index)."""
    pos = _f64(pos)
    n = pos.shape[0]
    nc = _i32(nc)
    ncell = int(np.prod(nc))
    cell_of = np.empty(n, np.int32)
    start = np.empty(ncell + 1, np.int32)
    order = np.empty(n, np.int32)
    lib().orc_cell_list(ctypes.c_int64(n), _p(pos), _p(_f64(box)), _p(nc, _I32),
                        _p(_i32(cls), _I32), ctypes.c_int32(ncls), _p(cell_of, _I32),
                        _p(start, _I32), _p(order, _I32))
    return cell_of, start, order


def pair_set(pos, box, rc: float):
    """All ordered in-cutoff triples (i, j, shift code) by brute force."""
    pos = _f64(pos)
    n = pos.shape[0]
    L = lib()
    cnt = L.orc_pair_set(ctypes.c_int64(n), _p(pos), _p(_f64(box)), ctypes.c_double(rc),
                         ctypes.c_int64(0), _p(np.zeros(3, np.int32), _I32))
    out = np.empty((max(cnt, 1), 3), np.int32)
    L.orc_pair_set(ctypes.c_int64(n), _p(pos), _p(_f64(box)), ctypes.c_double(rc),
                   ctypes.c_int64(cnt), _p(out, _I32))
    return out[:cnt]


def pairs(pos, q, types, A_tab, sig_tab, a_tab, box, rc, kappa, lB,
          do_gc=True, do_real=True, per_bead=False):
    """Real-space pair sums (Eq. u_ex and the real part of Eq. ewald)."""
    pos = _f64(pos)
    n = pos.shape[0]
    A_tab = _f64(A_tab)
    nt = int(A_tab.shape[0])
    e = np.zeros(2)
    f = np.zeros((n, 3))
    vir = np.zeros(9)
    npairs = ctypes.c_int64(0)
    eb = np.zeros((n, 2)) if per_bead else None
    lib().orc_pairs(ctypes.c_int64(n), _p(pos), _p(_f64(q)), _p(_i32(types), _I32),
                    ctypes.c_int32(nt), _p(A_tab), _p(_f64(sig_tab)), _p(_f64(a_tab)),
                    _p(_f64(box)), ctypes.c_double(rc), ctypes.c_double(kappa),
                    ctypes.c_double(lB), ctypes.c_int32(int(do_gc)),
                    ctypes.c_int32(int(do_real)), _p(e), _p(f), _p(vir),
                    ctypes.byref(npairs), _p(eb) if per_bead else None)
    out = dict(gc=e[0], real=e[1], forces=f, virial=vir.reshape(3, 3),
               npairs=int(npairs.value))
    if per_bead:
        out["per_bead"] = eb
    return out


def ewald_recip(pos, q, box, kappa, lB, tol=1e-16, forces=True):
    """Direct reciprocal k-sum of Eq. ewald (tin-foil, k != 0)."""
    pos = _f64(pos)
    n = pos.shape[0]
    e = ctypes.c_double(0.0)
    f = np.zeros((n, 3)) if forces else None
    vir = np.zeros(9)
    lib().orc_ewald_recip(ctypes.c_int64(n), _p(pos), _p(_f64(q)), _p(_f64(box)),
                          ctypes.c_double(kappa), ctypes.c_double(lB),
                          ctypes.c_double(tol), ctypes.byref(e),
                          _p(f) if forces else None, _p(vir))
    return dict(recip=e.value, forces=f, virial=vir.reshape(3, 3))


def spme(pos, q, box, K, p, kappa, lB, forces=True):
    """FP64 smooth PME (Essmann et al. 1995) with direct separable DFTs."""
    pos = _f64(pos)
    n = pos.shape[0]
    e = ctypes.c_double(0.0)
    f = np.zeros((n, 3)) if forces else None
    vir = np.zeros(9)
    lib().orc_spme(ctypes.c_int64(n), _p(pos), _p(_f64(q)), _p(_f64(box)),
                   _p(_i32(K), _I32), ctypes.c_int32(p), ctypes.c_double(kappa),
                   ctypes.c_double(lB), ctypes.byref(e), _p(f) if forces else None,
                   _p(vir))
    return dict(recip=e.value, forces=f, virial=vir.reshape(3, 3))


def ewald_constants(q, a_bead, kappa, lB):
    c = ctypes.c_double(0.0)
    s = ctypes.c_double(0.0)
    q = _f64(q)
    lib().orc_ewald_constants(ctypes.c_int64(q.shape[0]), _p(q), _p(_f64(a_bead)),
                              ctypes.c_double(kappa), ctypes.c_double(lB),
                              ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def slab_yb(pos, q, box, lB):
    pos = _f64(pos)
    e = ctypes.c_double(0.0)
    fz = np.zeros(pos.shape[0])
    lib().orc_slab_yb(ctypes.c_int64(pos.shape[0]), _p(pos), _p(_f64(q)), _p(_f64(box)),
                      ctypes.c_double(lB), ctypes.byref(e), _p(fz))
    return e.value, fz


def walls(pos, H, wallA, s_w):
    pos = _f64(pos)
    e = ctypes.c_double(0.0)
    fz = np.zeros(pos.shape[0])
    lib().orc_walls(ctypes.c_int64(pos.shape[0]), _p(pos), ctypes.c_double(H),
                    ctypes.c_double(wallA), ctypes.c_double(s_w), ctypes.byref(e),
                    _p(fz))
    return e.value, fz


def bonds(pairs_ij, pos, box, periodic, k, r0):
    pos = _f64(pos)
    pairs_ij = _i32(pairs_ij).reshape(-1, 2)
    e = ctypes.c_double(0.0)
    f = np.zeros_like(pos)
    vir = np.zeros(9)
    lib().orc_bonds(ctypes.c_int64(pairs_ij.shape[0]), _p(pairs_ij, _I32),
                    ctypes.c_int64(pos.shape[0]), _p(pos), _p(_f64(box)),
                    _p(_i32(periodic), _I32), ctypes.c_double(k), ctypes.c_double(r0),
                    ctypes.byref(e), _p(f), _p(vir))
    return e.value, f, vir.reshape(3, 3)


# ---------------------------------------------------------------------------
# Whole-model assembly per boundary condition
# ---------------------------------------------------------------------------
TERMS = ("gc", "real", "recip", "corr", "self", "slab", "wall", "bond")

# bead classes of the cell order: images, charged reals, neutral reals
CLS_IMAGE, CLS_CHARGED, CLS_NEUTRAL = 0, 1, 2


def _species(s: System):
    """Number of species and the species of every real bead (one species,
    type 0, when the system has no tables)."""
    if s.types is None:
        return 1, np.zeros(s.n, np.int32)
    return int(s.A_tab.shape[0]), np.asarray(s.types, np.int32)


def electrostatic_beads(s: System, pos=None):
    """Beads that carry the electrostatics: the reals, plus mirror images
    (x, y, -z) with charge -z_i for every charged real in the conducting-slab
    geometry.  Returns (pos, q, type, n_real).  type = the species t of a
    real bead, nt + t for the image of a bead of species t (images carry the
    smearing radius of their source and no Gaussian core)."""
    pos = s.pos if pos is None else pos
    q = s.q
    n = pos.shape[0]
    nt, types = _species(s)
    if s.geometry != GEOM_SLAB_PC:
        return pos, q, types, n
    qi = np.nonzero(q)[0]
    img = pos[qi].copy()
    img[:, 2] = -img[:, 2]
    return (np.concatenate([pos, img]), np.concatenate([q, -q[qi]]),
            np.concatenate([types, nt + types[qi]]).astype(np.int32), n)


def bead_classes(s: System):
    """Class of every bead of the (possibly doubled) electrostatic system."""
    pos, q, types, n = electrostatic_beads(s)
    cls = np.where(q != 0.0, CLS_CHARGED, CLS_NEUTRAL).astype(np.int32)
    cls[n:] = CLS_IMAGE
    return cls


def _tables(s: System):
    """Pair tables over 2 nt bead types: species 0..nt-1 (A_ij, sigma_i, a_i
    of the system) and their images nt..2nt-1 (same a_i, no Gaussian core)."""
    if s.types is None:
        A, sig, a = np.array([[s.A]]), np.array([s.sigma]), np.array([s.a])
    else:
        A, sig, a = (np.asarray(s.A_tab, float), np.asarray(s.sig_tab, float),
                     np.asarray(s.a_tab, float))
    nt = A.shape[0]
    A_tab = np.zeros((2 * nt, 2 * nt))
    A_tab[:nt, :nt] = A
    return A_tab, np.concatenate([sig, sig]), np.concatenate([a, a])


def energy_forces(s: System, pos=None, recip: str = "spme",
                  ewald_tol: float = 1e-16) -> Dict:
    """Total energy by term, forces on the real beads and the virial.

    recip = "spme" (same grid and order as the system) or "ewald" (direct
    k-sum; the converged reciprocal sum).  Returns a dict with the terms of
    ``TERMS``, "potential", "forces" (n,3), "virial" (3,3, pair + reciprocal
    + bonds) and "npairs" (unordered in-cutoff triples, images included).
    """
    pos = s.pos if pos is None else np.asarray(pos, np.float64)
    n = pos.shape[0]
    epos, eq, etype, _ = electrostatic_beads(s, pos)
    A_tab, sig, a = _tables(s)
    pr = pairs(epos, eq, etype, A_tab, sig, a, s.box, s.rc, s.kappa, s.lB)
    if recip == "spme":
        rr = spme(epos, eq, s.box, s.K, s.order, s.kappa, s.lB)
    else:
        rr = ewald_recip(epos, eq, s.box, s.kappa, s.lB, tol=ewald_tol)
    corr, self_e = ewald_constants(eq, a[etype], s.kappa, s.lB)
    half = 0.5 if s.geometry == GEOM_SLAB_PC else 1.0
    E = dict(gc=pr["gc"], real=half * pr["real"], recip=half * rr["recip"],
             corr=half * corr, self=half * self_e, slab=0.0, wall=0.0, bond=0.0)
    F = pr["forces"][:n] + rr["forces"][:n]
    vir = pr["virial"] + rr["virial"]
    if s.geometry == GEOM_SLAB_NM:
        e, fz = slab_yb(pos, s.q, s.box, s.lB)
        E["slab"] = e
        F[:, 2] += fz
    if s.geometry in (GEOM_SLAB_NM, GEOM_SLAB_PC) and s.wall_A != 0.0:  # no wall: none
        e, fz = walls(pos, s.H, s.wall_A, s.wall_sigma2)
        E["wall"] = e
        F[:, 2] += fz
    if s.bonds.shape[0] > 0:
        per = (1, 1, 1) if s.geometry == GEOM_BULK else (1, 1, 0)
        e, fb, vb = bonds(s.bonds, pos, s.box, per, s.bond_k, s.bond_r0)
        E["bond"] = e
        F += fb
        vir = vir + vb
    E["potential"] = sum(E[t] for t in TERMS)
    E["forces"] = F
    E["virial"] = vir
    E["npairs"] = pr["npairs"]
    return E


def mobile(s: System) -> np.ndarray:
    """(n, 1) weights: 1 for beads that move, 0 for beads of a frozen species
    (explicit electrodes): the integrators leave their positions and
    velocities as they are and the kinetic energy omits them."""
    m = np.ones((s.n, 1))
    if s.types is not None and s.frozen_mask:
        m[((s.frozen_mask >> np.asarray(s.types)) & 1) == 1] = 0.0
    return m


def velocity_verlet(s: System, nsteps: int, recip: str = "spme", record=None):
    """NVE velocity Verlet, unit masses, FP64:
        v += dt/2 F;  x += dt v;  F = F(x);  v += dt/2 F
    (beads of frozen species keep x and v).
    Returns (pos, vel, list of per-step dicts {potential, kinetic})."""
    pos = s.pos.copy()
    vel = s.vel.copy()
    dt = s.dt
    m = mobile(s)
    ef = energy_forces(s, pos, recip=recip)
    F = ef["forces"]
    hist = [dict(potential=ef["potential"], kinetic=0.5 * float(np.sum(m * vel * vel)))]
    for _ in range(nsteps):
        vel += m * (0.5 * dt * F)
        pos += m * (dt * vel)
        ef = energy_forces(s, pos, recip=recip)
        F = ef["forces"]
        vel += m * (0.5 * dt * F)
        hist.append(dict(potential=ef["potential"],
                         kinetic=0.5 * float(np.sum(m * vel * vel))))
    return pos, vel, hist


# ---------------------------------------------------------------------------
# Langevin dynamics (the paper integrates the Langevin equations of motion in
# the canonical ensemble, method of image charges and illustrative example
# sections; it names neither the splitting nor the friction).  Reading: the
# BAOAB splitting of Leimkuhler and Matthews (2013), unit masses, friction
# gamma, temperature kT:
#   B: v += dt/2 F;  A: x += dt/2 v;  O: v = c1 v + c2 xi;  A: x += dt/2 v;
#   F = F(x);  B: v += dt/2 F,   c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT).
# The noise xi of bead i at step n comes from a counter-based generator,
# Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): counter
# (n, i, 0, 0), key (seed, 0); its four 64-bit words give uniforms
# u_k = (floor(w_k / 2^40) + 1/2) / 2^24 and, by the Box-Muller transform,
#   xi_x = sqrt(-2 ln u_0) cos(2 pi u_1),  xi_y = sqrt(-2 ln u_0) sin(2 pi u_1),
#   xi_z = sqrt(-2 ln u_2) cos(2 pi u_3).
# Parity: the generator is pinned word for word to numpy's Philox; the
# integrator to the exact configurational sampling of BAOAB for harmonic
# forces, the free-particle velocity autocorrelation exp(-gamma t) and its
# reduction to velocity Verlet at gamma = 0.
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1
PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)   # round multipliers
PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)   # key increments (Weyl)


def _mulhilo64(a, b):
    """Full 128-bit product of uint64 arrays a * b as (hi, lo), from 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo, a_hi = a & m32, a >> s32
    b_lo, b_hi = b & m32, b >> s32
    ll = a_lo * b_lo
    hl = a_hi * b_lo
    lh = a_lo * b_hi
    hh = a_hi * b_hi
    t = hl + (ll >> s32)
    w = (t & m32) + lh
    hi = hh + (t >> s32) + (w >> s32)
    lo = a * b
    return hi, lo


def philox4x64(ctr, key, rounds: int = 10):
    """Philox4x64-R block function on arrays: ctr (..., 4) and key (..., 2)
    of uint64; returns (..., 4) uint64."""
    with np.errstate(over="ignore"):
        c = [np.asarray(ctr[..., k], dtype=np.uint64).copy() for k in range(4)]
        k0 = np.asarray(key[..., 0], dtype=np.uint64).copy()
        k1 = np.asarray(key[..., 1], dtype=np.uint64).copy()
        m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
        w0, w1 = np.uint64(PHILOX_W[0]), np.uint64(PHILOX_W[1])
        for r in range(rounds):
            if r > 0:
                k0 = k0 + w0
                k1 = k1 + w1
            hi0, lo0 = _mulhilo64(m0 * np.ones_like(c[0]), c[0])
            hi1, lo1 = _mulhilo64(m1 * np.ones_like(c[2]), c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        return np.stack(c, axis=-1)


def langevin_noise(seed: int, step: int, n: int) -> np.ndarray:
    """Standard normal noise (n, 3) of beads 0..n-1 at step `step`."""
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.uint64(step)
    ctr[:, 1] = np.arange(n, dtype=np.uint64)
    key = np.zeros((n, 2), dtype=np.uint64)
    key[:, 0] = np.uint64(seed & _M64)
    w = philox4x64(ctr, key)
    u = ((w >> np.uint64(40)).astype(np.float64) + 0.5) * 2.0 ** -24
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r2 = np.sqrt(-2.0 * np.log(u[:, 2]))
    out = np.empty((n, 3))
    out[:, 0] = r0 * np.cos(2.0 * np.pi * u[:, 1])
    out[:, 1] = r0 * np.sin(2.0 * np.pi * u[:, 1])
    out[:, 2] = r2 * np.cos(2.0 * np.pi * u[:, 3])
    return out


def langevin_baoab(s: System, nsteps: int, gamma: float, kT: float, seed: int,
                   step0: int = 0, recip: str = "spme", force_fn=None):
    """BAOAB Langevin dynamics, unit masses, FP64 (see the block comment).
    force_fn(pos) -> (forces, potential) replaces the GCMe forces if given.
    Returns (pos, vel, list of per-step dicts {potential, kinetic})."""
    pos = s.pos.copy()
    vel = s.vel.copy()
    dt = s.dt
    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt((1.0 - c1 * c1) * kT)

    def fe(x):
        if force_fn is not None:
            return force_fn(x)
        ef = energy_forces(s, x, recip=recip)
        return ef["forces"], ef["potential"]

    m = mobile(s) if hasattr(s, "types") else np.ones((pos.shape[0], 1))
    F, U = fe(pos)
    hist = [dict(potential=U, kinetic=0.5 * float(np.sum(m * vel * vel)))]
    for n in range(step0, step0 + nsteps):
        vel += m * (0.5 * dt * F)
        pos += m * (0.5 * dt * vel)
        vel = np.where(m > 0, c1 * vel + c2 * langevin_noise(seed, n, pos.shape[0]), vel)
        pos += m * (0.5 * dt * vel)
        F, U = fe(pos)
        vel += m * (0.5 * dt * F)
        hist.append(dict(potential=U, kinetic=0.5 * float(np.sum(m * vel * vel))))
    return pos, vel, hist


# ---------------------------------------------------------------------------
# Pressure and NpT (Parametrization section).  The pressure is Eq.
# pres_virial for one configuration, p = N kT / V + tr(W) / (3 V), with W the
# virial of all forces (pair, reciprocal, bonds; bulk systems).  The
# paper's NpT runs name no barostat; reading: a Monte Carlo barostat with
# isotropic moves of ln V (symmetric proposals), every bead's position
# scaled with the box:
#   V' = V exp((2 u0 - 1) dlnv),  x' = x (V'/V)^{1/3},
#   dW = U(x', V') - U(x, V) + p (V' - V) - (N + 1) kT ln(V'/V),
#   accept iff dW <= 0 or u1 < exp(-dW / kT)
# (N + 1: the configurational Jacobian V^N and the d ln V measure),
# u0, u1 = floor(w / 2^11) / 2^53 of Philox4x64-10 at counter (move, 0, 0, 0)
# with key (seed, 1) (the Langevin noise uses key word 1 = 0).
# Parity: pinned by the ideal gas, whose NpT volume has <V> = (N + 1) kT / p
# exactly, and by p_conf = tr(W)/(3V) = -dU/dV under isotropic scaling.
# ---------------------------------------------------------------------------
def pressure(s: System, pos=None, kT: float = 1.0) -> float:
    """Instantaneous virial pressure with the ideal term N kT / V."""
    pos = s.pos if pos is None else pos
    ef = energy_forces(s, pos)
    V = float(np.prod(s.box))
    return (s.n * kT + float(np.trace(ef["virial"])) / 3.0) / V


def barostat_uniforms(seed: int, move: int):
    ctr = np.array([[move, 0, 0, 0]], dtype=np.uint64)
    key = np.array([[seed & _M64, 1]], dtype=np.uint64)
    w = philox4x64(ctr, key)[0]
    return [float(int(x) >> 11) * 2.0 ** -53 for x in w[:2]]


def barostat_move(s: System, pos, box, pressure_: float, kT: float, dlnv: float, seed: int,
                  move: int, energy_fn=None):
    """One Monte Carlo volume move (see the block comment).  energy_fn(pos,
    box) -> potential energy; default: the GCMe energy of s in that box.
    Returns (pos, box, accepted)."""
    def energy(p, b):
        if energy_fn is not None:
            return energy_fn(p, b)
        t = s.copy()
        t.box = np.asarray(b, float).copy()
        return energy_forces(t, p)["potential"]

    u0, u1 = barostat_uniforms(seed, move)
    V = float(np.prod(box))
    lr = (2.0 * u0 - 1.0) * dlnv  # ln(V'/V)
    V1 = V * np.exp(lr)
    sc = np.exp(lr / 3.0)
    pos1 = pos * sc
    box1 = np.asarray(box, float) * sc
    dW = energy(pos1, box1) - energy(pos, box) + pressure_ * (V1 - V) - \
        (pos.shape[0] + 1) * kT * lr
    if dW <= 0.0 or u1 < np.exp(-dW / kT):
        return pos1, box1, True
    return pos, box, False
