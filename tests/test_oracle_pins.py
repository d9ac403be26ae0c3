"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with an
independent route (quadrature of the SI's defining integrals, textbook
constants, invariances of the Ewald split, finite differences, brute force,
analytic image laws).  Each test names the passage it follows.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LB = synth.LB_WATER


def _two_bead(r, q=(0.0, 0.0), sig=(0.5, 0.5), a=(0.5, 0.5), A=25.0, L=20.0):
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    types = np.array([0, 1], np.int32)
    A_tab = np.full((2, 2), A)
    return pos, np.array(q, float), types, A_tab, np.array(sig), np.array(a), np.array([L, L, L])


# --------------------------------------------------------------------------
# Gaussian core (Eq. u_ex and its SI derivation as an overlap integral)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,sig", [(0.0, (0.5, 0.5)), (0.4, (0.5, 0.5)),
                                   (1.1, (0.5, 0.3)), (2.0, (0.6, 0.4))])
def test_gc_equals_overlap_integral(r, sig):
    """SI 'Derivation of the excluded volume interaction potential':
    u_ex = A int rho_i rho_j d^3r with normalised Gaussians of variance
    sigma^2/3 per axis.  Evaluated here by quadrature, axis by axis."""
    pos, q, types, A_tab, s, a, box = _two_bead(r, sig=sig)
    e = oracle.pairs(pos, q, types, A_tab, s, a, box, 3.0, 0.9, LB, do_real=False)
    v = [si * si / 3.0 for si in sig]

    def g(x, var, c):
        return math.exp(-(x - c) ** 2 / (2 * var)) / math.sqrt(2 * math.pi * var)

    ix = integrate.quad(lambda x: g(x, v[0], 0.0) * g(x, v[1], r), -10, 10 + r,
                        epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    iy = integrate.quad(lambda x: g(x, v[0], 0.0) * g(x, v[1], 0.0), -10, 10,
                        epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    ref = 25.0 * ix * iy * iy
    assert e["gc"] == pytest.approx(ref, rel=1e-9)


def test_gc_contact_value():
    """Limits section (SI): u_ex(0) = A (3/(2 pi sigma_ij^2))^{3/2}; with
    A = 25, sigma_i = 0.5 this is 23.329 kT."""
    pos, q, types, A_tab, s, a, box = _two_bead(0.0)
    e = oracle.pairs(pos, q, types, A_tab, s, a, box, 3.0, 0.9, LB, do_real=False)
    assert e["gc"] == pytest.approx(23.329, abs=5e-4)


# --------------------------------------------------------------------------
# Smeared Coulomb (Eq. u_elec and the SI's Fourier-integral derivation)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r,a", [(0.3, (0.5, 0.5)), (1.0, (0.5, 0.5)),
                                 (1.7, (0.3, 0.7)), (2.5, (0.5, 0.2))])
def test_elec_equals_fourier_integral(r, a):
    """SI 'Derivation of the smeared electrostatic interaction potential':
    u = (2 lB z_i z_j / (pi r)) int_0^inf sin(k r)/k exp(-a_ij^2 k^2/(2 pi)) dk.
    The oracle's real-space kernel with kappa = 0 is exactly u_elec."""
    pos, q, types, A_tab, s, aa, box = _two_bead(r, q=(1.0, -1.0), a=a, A=0.0)
    e = oracle.pairs(pos, q, types, A_tab, s, aa, box, 3.0, 0.0, LB, do_gc=False)
    a2 = a[0] ** 2 + a[1] ** 2
    val = integrate.quad(lambda k: math.sin(k * r) / k * math.exp(-a2 * k * k / (2 * math.pi)),
                         0, 60, limit=500, epsabs=1e-13, epsrel=1e-12)[0]
    ref = 2.0 * LB * (1.0 * -1.0) / (math.pi * r) * val
    assert e["real"] == pytest.approx(ref, rel=1e-9)


def test_elec_contact_and_born_limits():
    """Gaussian core model section and SI Limits: u_elec(0) =
    z_i z_j e^2/(2^{3/2} pi eps a_ij) = sqrt(2) lB z_i z_j / a_ij (2.4106 kT for
    a = 0.5, lB = 1.2053); the Born self energy is half the contact value of a
    bead with itself (a_ii^2 = 2 a^2), i.e. the U_self term of Eq. ewald."""
    pos, q, types, A_tab, s, a, box = _two_bead(1e-9, q=(1.0, 1.0), A=0.0)
    e = oracle.pairs(pos, q, types, A_tab, s, a, box, 3.0, 0.0, LB, do_gc=False)
    assert e["real"] == pytest.approx(2.4106, abs=2e-4)
    # Born: the self term of one bead vs half the contact value of the pair
    # function with a_i = a_j = a (a_ij = sqrt(2) a)
    _, born = oracle.ewald_constants(np.array([1.0]), np.array([0.5]), 0.9, LB)
    assert born == pytest.approx(0.5 * e["real"], rel=1e-12)


def test_elec_large_r_is_coulomb():
    """SI Limits: erf(beta r) -> 1, u_elec -> lB z_i z_j / r for r >> a_ij."""
    pos, q, types, A_tab, s, a, box = _two_bead(2.9, q=(1.0, 1.0), a=(0.05, 0.05), A=0.0)
    e = oracle.pairs(pos, q, types, A_tab, s, a, box, 3.0, 0.0, LB, do_gc=False)
    assert e["real"] == pytest.approx(LB / 2.9, rel=1e-14)


# --------------------------------------------------------------------------
# Ewald decomposition (Eq. ewald)
# --------------------------------------------------------------------------
def _small_charged(n=24, L=6.0, seed=7, a=0.5):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(n, 3))
    q = np.array([1.0, -1.0] * (n // 2))
    rng.shuffle(q)
    return pos, q, np.array([L, L, L])


def _elec_total(pos, q, box, kappa, rc, a=0.5):
    n = pos.shape[0]
    types = np.zeros(n, np.int32)
    A_tab = np.zeros((1, 1))
    pr = oracle.pairs(pos, q, types, A_tab, np.array([0.5]), np.array([a]), box, rc,
                      kappa, LB, do_gc=False)
    rr = oracle.ewald_recip(pos, q, box, kappa, LB)
    corr, self_e = oracle.ewald_constants(q, np.full(n, a), kappa, LB)
    return pr["real"] + rr["recip"] + corr + self_e, pr["forces"] + rr["forces"], \
        dict(real=pr["real"], recip=rr["recip"], corr=corr, self=self_e)


def test_ewald_kappa_independence():
    """Eq. ewald: the split is exact, so the total does not depend on the
    screening width G = 1/(sqrt(2) kappa) once rc makes erfc(kappa rc)
    negligible (here the image enumeration reaches r = 7 in a box of 6)."""
    pos, q, box = _small_charged()
    vals, forces = [], []
    for kappa in (1.2, 1.5, 2.0):
        E, F, _ = _elec_total(pos, q, box, kappa, rc=7.0)
        vals.append(E)
        forces.append(F)
    assert vals[1] == pytest.approx(vals[0], rel=1e-11, abs=1e-10)
    assert vals[2] == pytest.approx(vals[0], rel=1e-11, abs=1e-10)
    assert np.max(np.abs(forces[1] - forces[0])) < 1e-9
    assert np.max(np.abs(forces[2] - forces[0])) < 1e-9


def test_ewald_fully_reciprocal_limit():
    """Model section: choosing G = a_ij / sqrt(pi) (kappa = beta for uniform
    a) moves everything to reciprocal space: the real term vanishes pair by
    pair and corr + self cancel.  SI eq. for the Fourier transform of the
    smeared density gives the same reciprocal weight exp(-a^2 k^2/pi)."""
    pos, q, box = _small_charged()
    a = 0.5
    beta = math.sqrt(math.pi) / (math.sqrt(2.0) * math.sqrt(2 * a * a))
    E_b, _, parts = _elec_total(pos, q, box, beta, rc=2.9, a=a)
    assert abs(parts["real"]) < 1e-15
    assert parts["corr"] + parts["self"] == pytest.approx(0.0, abs=1e-12)
    E_ref, _, _ = _elec_total(pos, q, box, 1.3, rc=7.0, a=a)
    assert E_b == pytest.approx(E_ref, rel=1e-11)


@pytest.mark.parametrize("reps", [1, 2])
def test_madelung_rocksalt(reps):
    """Point-charge limit (SI Limits, a -> 0): rock-salt lattice energy is
    -M lB / r_nn per ion pair with the textbook Madelung constant M."""
    M = json.load(open(os.path.join(GOLD, "madelung_nacl.json")))["madelung_rocksalt"]
    base = []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                base.append(((i, j, k), 1.0 if (i + j + k) % 2 == 0 else -1.0))
    pos, q = [], []
    for X in range(2 * reps):
        for Y in range(2 * reps):
            for Z in range(2 * reps):
                if (X + Y + Z) % 2 == 0:
                    pass
                pos.append((X, Y, Z))
                q.append(1.0 if (X + Y + Z) % 2 == 0 else -1.0)
    pos = np.array(pos, float) + 0.25
    q = np.array(q)
    L = 2.0 * reps
    box = np.array([L, L, L])
    a = 0.05
    E, F, parts = _elec_total(pos, q, box, kappa=2.2, rc=min(3.0, L), a=a)
    n_pairs = pos.shape[0] / 2
    assert E - parts["self"] == pytest.approx(-M * LB * n_pairs, rel=1e-9)
    assert np.max(np.abs(F)) < 1e-9  # every ion sits at a centre of symmetry


def test_ewald_direct_lattice_sum_small_box():
    """Eq. ewald first line (direct lattice sum) summed over whole periodic
    cells in growing spheres converges to the tin-foil Ewald value plus the
    spherical surface term 2 pi lB |M|^2 / (3 V) (de Leeuw, Perram & Smith)."""
    rng = np.random.default_rng(3)
    L = 3.0
    pos = rng.uniform(0, L, size=(4, 3))
    q = np.array([1.0, -1.0, 1.0, -1.0])
    box = np.array([L, L, L])
    a = 0.5
    E_ew, _, _ = _elec_total(pos, q, box, kappa=1.4, rc=6.0, a=a)
    Mvec = (q[:, None] * pos).sum(0)
    surf = 2 * math.pi * LB * float(Mvec @ Mvec) / (3 * L ** 3)
    beta = math.sqrt(math.pi) / (math.sqrt(2.0) * math.sqrt(2 * a * a))
    from scipy.special import erf

    def direct(R):
        rng_ = np.arange(-R, R + 1)
        n = np.stack(np.meshgrid(rng_, rng_, rng_, indexing="ij"), -1).reshape(-1, 3)
        n = n[(n ** 2).sum(1) <= R * R] * L
        tot = 0.0
        for i in range(4):
            for j in range(4):
                d = pos[j] + n - pos[i]
                r = np.sqrt((d ** 2).sum(1))
                if i == j:
                    r = r[r > 0]
                tot += 0.5 * LB * q[i] * q[j] * np.sum(erf(beta * r) / r)
        return tot + LB * np.sum(q * q / (2 * a))

    # Richardson extrapolation in 1/R of the shell sums
    R1, R2 = 24, 48
    d1, d2 = direct(R1), direct(R2)
    extrap = (R2 * d2 - R1 * d1) / (R2 - R1)
    assert extrap == pytest.approx(E_ew + surf, abs=2e-3 * abs(E_ew + surf) + 2e-3)
    # and the surface term matters: without it the gap is far larger
    assert abs(extrap - E_ew) > 10 * abs(extrap - E_ew - surf)


def test_zero_net_force_pairs_and_ewald():
    """Newton's third law for the pair terms and the direct Ewald sum."""
    pos, q, box = _small_charged(n=40, L=7.0, seed=11)
    E, F, _ = _elec_total(pos, q, box, kappa=0.9, rc=3.0)
    assert np.max(np.abs(F.sum(0))) < 1e-10
    s = synth.make_bulk(400, seed_index=9)
    A_tab = np.array([[25.0]])
    pr = oracle.pairs(s.pos, s.q, np.zeros(400, np.int32), A_tab, np.array([0.5]),
                      np.array([0.5]), s.box, 3.0, s.kappa, LB)
    assert np.max(np.abs(pr["forces"].sum(0))) < 1e-9


def _fd_check(efun, pos, idx, h=1e-5):
    """Central differences of efun at a few coordinates."""
    out = []
    for (i, a) in idx:
        p1 = pos.copy()
        p1[i, a] += h
        p2 = pos.copy()
        p2[i, a] -= h
        out.append(-(efun(p1) - efun(p2)) / (2 * h))
    return np.array(out)


def test_forces_are_energy_gradient_bulk():
    """Forces of every term (GC, real, SPME reciprocal, bonds) equal minus
    the finite-difference gradient of the total energy."""
    s = synth.make_polyelectrolyte(n_chains=4, chain_len=6, n_solvent=120, seed_index=8,
                                   K=(16, 16, 16))
    s.kappa = 0.9
    ef = oracle.energy_forces(s)
    rng = np.random.default_rng(1)
    idx = [(int(rng.integers(0, s.n)), int(rng.integers(0, 3))) for _ in range(10)]
    idx += [(0, 0), (1, 2), (3, 1)]  # charged chain beads with bonds
    fd = _fd_check(lambda p: oracle.energy_forces(s, p)["potential"], s.pos, idx)
    an = np.array([ef["forces"][i, a] for i, a in idx])
    assert np.max(np.abs(fd - an)) < 2e-6 * max(1.0, np.max(np.abs(an)))


# --------------------------------------------------------------------------
# Smooth PME (Essmann et al. 1995) against the direct k-sum
# --------------------------------------------------------------------------
def test_bspline_partition_of_unity_and_moduli():
    """Cardinal B-splines sum to one over integer shifts; |b(m)|^2 is the
    inverse power spectrum of the sampled spline (Essmann et al. 1995)."""
    for p in (4, 5, 6):
        for u in (0.0, 0.3, 0.77):
            assert sum(oracle.bspline(p, u + k) for k in range(p)) == pytest.approx(1.0, abs=1e-14)
    K = 16
    for p in (4, 6):
        b = oracle.bspline_moduli(p, K)
        samples = np.zeros(K)
        for k in range(p - 1):
            samples[k] = oracle.bspline(p, k + 1.0)
        spec = np.abs(np.fft.fft(samples)) ** 2
        assert np.allclose(b, 1.0 / spec, rtol=1e-12)


def test_spme_converges_to_ewald():
    """PME is an approximation of the reciprocal sum: its error must fall
    steeply with the grid and be tiny on a fine grid."""
    s = synth.make_bulk(300, rho=3.0, charged_frac=0.3, seed_index=12)
    ref = oracle.ewald_recip(s.pos, s.q, s.box, s.kappa, LB)
    errs = []
    for K in (8, 12, 16, 24, 32):
        r = oracle.spme(s.pos, s.q, s.box, (K, K, K), 5, s.kappa, LB)
        ferr = np.sqrt(np.mean((r["forces"] - ref["forces"]) ** 2)) / \
            np.sqrt(np.mean(ref["forces"] ** 2))
        errs.append((abs(r["recip"] - ref["recip"]) / abs(ref["recip"]), ferr))
    assert all(errs[i + 1][1] < errs[i][1] for i in range(len(errs) - 1))
    assert errs[-1][0] < 1e-6 and errs[-1][1] < 1e-5
    # high order on a fine grid reaches the direct sum to ~1e-11
    r = oracle.spme(s.pos, s.q, s.box, (48, 48, 48), 8, s.kappa, LB)
    assert abs(r["recip"] - ref["recip"]) < 1e-10 * abs(ref["recip"])
    assert np.max(np.abs(r["forces"] - ref["forces"])) < 1e-8 * np.max(np.abs(ref["forces"]))
    assert np.allclose(oracle.spme(s.pos, s.q, s.box, (32, 32, 32), 5, s.kappa, LB)["virial"],
                       ref["virial"], rtol=1e-5, atol=1e-5 * abs(ref["recip"]))


def test_spme_forces_are_gradient_of_spme_energy():
    """The SPME force is the analytic gradient of the SPME energy."""
    s = synth.make_bulk(120, rho=3.0, charged_frac=0.5, seed_index=13)
    K = (12, 10, 14)
    r = oracle.spme(s.pos, s.q, s.box, K, 5, s.kappa, LB)
    qi = np.nonzero(s.q)[0]
    idx = [(int(qi[k]), k % 3) for k in range(6)]
    fd = _fd_check(lambda p: oracle.spme(p, s.q, s.box, K, 5, s.kappa, LB, forces=False)["recip"],
                   s.pos, idx, h=1e-5)
    an = np.array([r["forces"][i, a] for i, a in idx])
    assert np.max(np.abs(fd - an)) < 1e-7


# --------------------------------------------------------------------------
# Virial (Eq. pres_virial) against the strain derivative of the energy
# --------------------------------------------------------------------------
def test_virial_is_strain_derivative():
    """W_ab = -dU/d eps_ab under an affine strain of box and positions."""
    s = synth.make_bulk(60, rho=1.0, charged_frac=0.4, seed_index=14, rc=4.5)
    s.kappa = 1.1
    ef = oracle.energy_forces(s, recip="ewald")
    W = ef["virial"]
    h = 1e-6
    for a in range(3):
        E = []
        for sgn in (+1, -1):
            t = s.copy()
            t.box = s.box.copy()
            t.box[a] *= 1 + sgn * h
            t.pos = s.pos.copy()
            t.pos[:, a] *= 1 + sgn * h
            E.append(oracle.energy_forces(t, recip="ewald")["potential"])
        dE = (E[0] - E[1]) / (2 * h)
        assert -dE == pytest.approx(W[a, a], rel=1e-6, abs=1e-6)


# --------------------------------------------------------------------------
# Slab boundary conditions (Illustrative example; method of image charges)
# --------------------------------------------------------------------------
def _slab_system(geom, Lz_factor, n=60, seed=21):
    s = synth.make_slab_fluid(geom, n, charged_frac=0.3, seed_index=seed, aspect=1.0)
    H = s.H
    s.box = np.array([s.box[0], s.box[1], Lz_factor * H])
    s.K = tuple(synth.smooth_size(int(math.ceil(b / 0.5))) for b in s.box)
    return s


def test_yeh_berkowitz_void_invariance():
    """Nonmetal electrodes: with the Yeh-Berkowitz term the slab energy no
    longer depends on the vacuum added along z; without it, it does."""
    E = {}
    for f in (3.0, 5.0):
        s = _slab_system(synth.GEOM_SLAB_NM, f)
        ef = oracle.energy_forces(s, recip="ewald")
        E[f] = (ef["potential"], ef["potential"] - ef["slab"])
    with_yb = abs(E[3.0][0] - E[5.0][0])
    without = abs(E[3.0][1] - E[5.0][1])
    assert with_yb < 2e-3
    assert without > 20 * with_yb


def test_slab_forces_are_gradient():
    """Yeh-Berkowitz and wall forces are minus the gradient of their energy."""
    s = _slab_system(synth.GEOM_SLAB_NM, 3.0)
    ef = oracle.energy_forces(s, recip="ewald")
    qi = np.nonzero(s.q)[0]
    idx = [(int(qi[0]), 2), (int(qi[1]), 2), (0, 2), (5, 0)]
    fd = _fd_check(lambda p: oracle.energy_forces(s, p, recip="ewald")["potential"],
                   s.pos, idx)
    an = np.array([ef["forces"][i, a] for i, a in idx])
    assert np.max(np.abs(fd - an)) < 1e-6 * max(1.0, np.max(np.abs(an)))


def test_wall_is_plane_integral_of_core():
    """The continuum wall is u_ex integrated over a plane of density n_s:
    2 pi n_s int_0^inf u_ex(sqrt(rho^2 + h^2)) rho d rho, with the electrode
    bead width entering through sigma_ij^2 (Eq. u_ex)."""
    s = _slab_system(synth.GEOM_SLAB_NM, 3.0, n=60)
    n_s = 2.0 / (math.sqrt(3.0) * 0.25)
    s2 = s.wall_sigma2
    for h in (0.3, 0.8):
        pos = np.array([[1.0, 1.0, h], [1.0, 1.0, s.H / 2]])
        e_w, _ = oracle.walls(pos[:1], s.H, s.wall_A, s2)
        e_far, _ = oracle.walls(np.array([[1.0, 1.0, s.H - h]]), s.H, 0.0, s2)

        def u(r2):
            return 25.0 * (3 / (2 * math.pi * s2)) ** 1.5 * math.exp(-1.5 * r2 / s2)

        ref = 2 * math.pi * n_s * integrate.quad(lambda r: u(r * r + h * h) * r, 0, 20,
                                                 epsabs=1e-13, epsrel=1e-12)[0]
        far = 2 * math.pi * n_s * integrate.quad(lambda r: u(r * r + (s.H - h) ** 2) * r, 0, 20)[0]
        assert e_w == pytest.approx(ref + far, rel=1e-9)
        assert e_far == 0.0


def _one_ion_pc(h, Lxy=60.0, H=60.0, q=1.0):
    s = synth.System(name="ion", geometry=synth.GEOM_SLAB_PC,
                     box=np.array([Lxy, Lxy, 2 * H]), pos=np.array([[7.0, 9.0, h]]),
                     vel=np.zeros((1, 3)), q=np.array([q]), bonds=np.zeros((0, 2), np.int32),
                     kappa=0.6, rc=8.0, K=(32, 32, 64), H=H, wall_A=0.0, wall_sigma2=0.3125)
    return s


def test_image_charge_law():
    """Method of image charges, perfectly conducting electrode: the image
    carries -z_i e; the force on an ion at height h >> a is the image law
    -lB z^2/(4 h^2) toward the wall, and the physical energy (half of the
    doubled system's) changes with h as -lB z^2/(4 h)."""
    E, F = {}, {}
    for h in (1.5, 3.0):
        s = _one_ion_pc(h)
        ef = oracle.energy_forces(s, recip="ewald", ewald_tol=1e-14)
        E[h] = ef["potential"]
        F[h] = ef["forces"][0]
    for h in (1.5, 3.0):
        assert F[h][2] == pytest.approx(-LB / (4 * h * h), rel=1e-2)
        assert abs(F[h][0]) < 1e-6 and abs(F[h][1]) < 1e-6
    dE = E[1.5] - E[3.0]
    assert dE == pytest.approx(-LB / 4 * (1 / 1.5 - 1 / 3.0), rel=1e-2)


# --------------------------------------------------------------------------
# Harmonic bonds (Illustrative example) and velocity Verlet
# --------------------------------------------------------------------------
def test_bond_minimum_image_and_gradient():
    box = np.array([5.0, 5.0, 5.0])
    pos = np.array([[0.2, 1.0, 1.0], [4.5, 1.3, 1.1]])  # 0.7 apart across x
    e, f, _ = oracle.bonds(np.array([[0, 1]]), pos, box, (1, 1, 1), 100.0, 1.0)
    d = np.array([-0.7, 0.3, 0.1])
    r = np.linalg.norm(d)
    assert e == pytest.approx(50.0 * (r - 1.0) ** 2, rel=1e-14)
    fd = _fd_check(lambda p: oracle.bonds(np.array([[0, 1]]), p, box, (1, 1, 1), 100.0, 1.0)[0],
                   pos, [(0, 0), (1, 1)])
    assert np.allclose(fd, [f[0, 0], f[1, 1]], atol=1e-6)
    assert np.allclose(f.sum(0), 0.0, atol=1e-12)


def test_velocity_verlet_time_reversible():
    """Velocity Verlet is time reversible: integrating forward, flipping the
    velocities and integrating again returns to the start."""
    s = synth.make_polyelectrolyte(n_chains=3, chain_len=5, n_solvent=80, seed_index=15,
                                   K=(12, 12, 12))
    s.dt = 0.01
    p1, v1, _ = oracle.velocity_verlet(s, 20)
    t = s.copy()
    t.pos, t.vel = p1, -v1
    p2, v2, _ = oracle.velocity_verlet(t, 20)
    assert np.max(np.abs(p2 - s.pos)) < 1e-9
    assert np.max(np.abs(v2 + s.vel)) < 1e-8


def test_velocity_verlet_second_order_energy_error():
    """NVE velocity Verlet: the energy error of a symplectic second-order
    scheme falls as dt^2 (ratio 4 per halving) from a random, strongly
    relaxing start of a GCMe fluid at density 3."""
    s0 = synth.make_bulk(600, seed_index=19, K=(16, 16, 16))
    errs = []
    for dt, n in ((0.01, 40), (0.005, 80), (0.0025, 160)):
        s = s0.copy()
        s.dt = dt
        _, _, hist = oracle.velocity_verlet(s, n)
        tot = np.array([h["potential"] + h["kinetic"] for h in hist])
        errs.append(np.max(np.abs(tot - tot[0])))
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


@pytest.mark.slow
def test_nve_drift_config1():
    """N=3000 fluid of the plain FP64 workload, 100 steps at dt = 0.01 tau:
    the total energy stays within 2e-3 of its start (the soft cores make a
    random start safe, the paper's argument for large steps)."""
    s = synth.config1()
    _, _, hist = oracle.velocity_verlet(s, 100)
    tot = np.array([h["potential"] + h["kinetic"] for h in hist])
    assert np.max(np.abs(tot - tot[0])) / abs(tot[0]) < 2e-3


# --------------------------------------------------------------------------
# Cell list and neighbour set (FP32 rule) by independent routes
# --------------------------------------------------------------------------
def _cell_enumeration(pos, box, rc):
    """Ordered in-cutoff triples found through the 27-cell stencil."""
    nc = oracle.cell_counts(box, rc)
    cls = np.zeros(pos.shape[0], np.int32)
    cell_of, start, order = oracle.cell_list(pos, box, nc, cls, ncls=1)
    w = oracle.wrap(pos, box).astype(np.float32)
    Lf = box.astype(np.float32)
    rc2 = np.float32(rc * rc)
    out = set()
    for c in range(int(np.prod(nc))):
        cc = np.array([c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])])
        ii = order[start[c]:start[c + 1]]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    u = cc + np.array([dx, dy, dz])
                    sh = np.floor_divide(u, nc)
                    v = u - sh * nc
                    cn = v[0] + nc[0] * (v[1] + nc[1] * v[2])
                    jj = order[start[cn]:start[cn + 1]]
                    if len(ii) == 0 or len(jj) == 0:
                        continue
                    shift = (sh.astype(np.float32) * Lf).astype(np.float32)
                    d = (w[jj][None, :, :] - w[ii][:, None, :]).astype(np.float32)
                    d = (d + shift).astype(np.float32)
                    sq = (d * d).astype(np.float32)
                    r2 = ((sq[..., 0] + sq[..., 1]).astype(np.float32) + sq[..., 2]).astype(np.float32)
                    for a_, b_ in zip(*np.nonzero(r2 < rc2)):
                        i, j = int(ii[a_]), int(jj[b_])
                        code = int((sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1))
                        if i == j and code == 13:
                            continue
                        out.add((i, j, code))
    return out


@pytest.mark.parametrize("n,rho", [(300, 3.0), (120, 3.0), (90, 3.0)])
def test_pair_set_brute_force_equals_cell_stencil(n, rho):
    """The brute-force O(N^2 x images) enumeration and the 27-cell stencil
    give the same ordered in-cutoff triples, including boxes shorter than
    2 rc where several images of a bead are within the cutoff."""
    s = synth.make_bulk(n, rho=rho, seed_index=16)
    bf = oracle.pair_set(s.pos, s.box, 3.0)
    got = {tuple(map(int, t)) for t in bf}
    assert len(got) == bf.shape[0]
    assert got == _cell_enumeration(s.pos, s.box, 3.0)
    # symmetric rule: (i,j,n) in the set iff (j,i,-n) is
    for (i, j, c) in list(got)[:2000]:
        assert (j, i, 26 - c) in got


def test_pair_count_matches_density():
    """Uniform fluid: unordered pairs ~ N^2/2 (4/3 pi rc^3)/V."""
    s = synth.make_bulk(3000, rho=3.0, seed_index=17)
    pr = oracle.pairs(s.pos, np.zeros(s.n), np.zeros(s.n, np.int32), np.array([[25.0]]),
                      np.array([0.5]), np.array([0.5]), s.box, 3.0, s.kappa, LB)
    expect = s.n * (s.n - 1) / 2 * (4 / 3 * math.pi * 27) / float(np.prod(s.box))
    assert abs(pr["npairs"] - expect) < 5 * math.sqrt(expect) + 0.01 * expect


def test_cell_list_is_a_stable_counting_sort():
    s = synth.make_bulk(500, seed_index=18)
    nc = oracle.cell_counts(s.box, 3.0)
    cls = (s.q == 0).astype(np.int32) + 1
    cell_of, start, order = oracle.cell_list(s.pos, s.box, nc, cls)
    w = oracle.wrap(s.pos, s.box)
    side = s.box / nc
    for i in range(s.n):
        c = cell_of[i]
        cc = np.array([c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])])
        assert np.all(w[i] >= cc * side - 1e-12) and np.all(w[i] <= (cc + 1) * side + 1e-12)
    keys = [(cell_of[i], cls[i], i) for i in order]
    assert keys == sorted(keys)
    assert start[-1] == s.n


# --------------------------------------------------------------------------
# Reduced units (Parametrization section)
# --------------------------------------------------------------------------
def test_reduced_units_match_paper():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    assert synth.bead_diameter_nm() == pytest.approx(g["bead_diameter_nm"]["value"],
                                                     abs=g["bead_diameter_nm"]["tol"])
    assert synth.bead_mass_gmol() == pytest.approx(g["bead_mass_gmol"]["value"],
                                                   abs=g["bead_mass_gmol"]["tol"])
    assert synth.time_unit_ps() == pytest.approx(g["time_unit_ps"]["value"],
                                                 abs=g["time_unit_ps"]["tol"])
    # water-sized beads: d = 0.275 nm, m = 18.02 g/mol -> tau ~ 0.739 ps
    d, m = 0.275e-9, 18.02e-3
    tau = math.sqrt(m * d * d / (6.02214076e23 * 1.380649e-23 * 300.0)) * 1e12
    assert tau == pytest.approx(g["water_time_unit_ps"]["value"], abs=g["water_time_unit_ps"]["tol"])


# --------------------------------------------------------------------------
# The pins discriminate: mistakes planted in the oracle's assembly fail them
# --------------------------------------------------------------------------
def test_planted_mistakes_are_caught():
    pos, q, box = _small_charged()
    tot = {}
    for kappa in (1.2, 2.0):
        _, _, p = _elec_total(pos, q, box, kappa, rc=7.0)
        tot[kappa] = p
    good = [sum(p.values()) for p in tot.values()]
    flipped_corr = [p["real"] + p["recip"] - p["corr"] + p["self"] for p in tot.values()]
    doubled_recip = [p["real"] + 2 * p["recip"] + p["corr"] + p["self"] for p in tot.values()]
    assert abs(good[0] - good[1]) < 1e-9
    assert abs(flipped_corr[0] - flipped_corr[1]) > 1e-3
    assert abs(doubled_recip[0] - doubled_recip[1]) > 1e-3
