"""Pins of the oracle's multi-species assembly (per-type A_ij, sigma_i, a_i).

The pair functions are pinned with unequal sigma and a in
test_oracle_pins.py (overlap and Fourier integrals by quadrature).  Here the
system-level pieces: the per-type tables and per-pair beta_ij = sqrt(pi) /
(sqrt(2) a_ij), image beads carrying their source's a_i, and the per-bead
Born self energy lB z_i^2 / (2 a_i), pinned by
* the kappa independence of the total electrostatic energy (Eq. ewald is an
  exact split only if every per-pair beta_ij and every per-bead self term is
  right) for mixtures of smearing radii, bulk and with image charges;
* the fully reciprocal limit kappa = beta_ij, which exists for a single
  a_ij only: a mixture with a_i = a for all species reduces to it;
* forces = minus the finite-difference gradient of the total energy;
* two species with identical tables = the one-species system (forces exactly).
"""
import math

import numpy as np
import pytest

import oracle
import synth

# species: solvent, large cation, small anion (sigma_i, a_i differ; A_ij with a blend offset)
A3 = np.array([[25.0, 27.0, 26.0], [27.0, 25.0, 30.0], [26.0, 30.0, 25.0]])
S3 = np.array([0.5, 0.6, 0.4])
a3 = np.array([0.5, 0.7, 0.35])


def _mixture(n=300, geometry=synth.GEOM_BULK, seed=40, a=a3):
    return synth.make_mixture(n, (0.6, 0.2, 0.2), (0.0, 1.0, -1.0), A3, S3, a,
                              seed_index=seed, geometry=geometry, K=(12, 12, 12))


def _elec_total(s, kappa, rc):
    t = s.copy()
    t.kappa, t.rc = kappa, rc
    ef = oracle.energy_forces(t, recip="ewald")
    return sum(ef[k] for k in ("real", "recip", "corr", "self")), ef


@pytest.mark.parametrize("geometry", [synth.GEOM_BULK, synth.GEOM_SLAB_PC])
def test_kappa_independence_with_species(geometry):
    s = _mixture(120 if geometry == synth.GEOM_BULK else 100, geometry, seed=41)
    if geometry == synth.GEOM_BULK:
        rc, ks = min(s.box) * 0.999, (1.6, 2.2)
    else:
        rc, ks = min(s.box[:2]) * 0.999, (1.9, 2.5)
    assert math.erfc(ks[0] * rc) < 1e-9
    e1, f1 = _elec_total(s, ks[0], rc)
    e2, f2 = _elec_total(s, ks[1], rc)
    assert e1 == pytest.approx(e2, rel=1e-9, abs=1e-9)
    # and the split is not trivially kappa-free: the parts move
    assert abs(f1["real"] - f2["real"]) > 1e-3


def test_one_smearing_radius_has_the_fully_reciprocal_limit():
    """With a_i = a for every species, kappa = beta = sqrt(pi)/(2a) makes the
    real term vanish pair by pair and corr + self cancel (species still
    differ in A_ij and sigma_i, which do not enter the electrostatics)."""
    a = 0.45
    s = _mixture(150, seed=42, a=np.full(3, a))
    beta = math.sqrt(math.pi) / (2.0 * a)
    e_b, ef = _elec_total(s, beta, 2.9)
    assert abs(ef["real"]) < 1e-14
    assert ef["corr"] + ef["self"] == pytest.approx(0.0, abs=1e-11)
    e_ref, _ = _elec_total(s, 1.6, min(s.box) * 0.999)
    assert e_b == pytest.approx(e_ref, rel=1e-9)


@pytest.mark.parametrize("geometry", [synth.GEOM_BULK, synth.GEOM_SLAB_PC, synth.GEOM_SLAB_NM])
def test_species_forces_are_energy_gradient(geometry):
    s = _mixture(160, geometry, seed=43)
    s.kappa = 0.9
    ef = oracle.energy_forces(s)
    rng = np.random.default_rng(2)
    charged = np.nonzero(s.q)[0]
    idx = [(int(charged[k]), k % 3) for k in range(6)]
    idx += [(int(rng.integers(0, s.n)), int(rng.integers(0, 3))) for _ in range(6)]
    h = 1e-5
    fd = []
    for i, a in idx:
        p = s.pos.copy()
        p[i, a] += h
        ep = oracle.energy_forces(s, p)["potential"]
        p[i, a] -= 2 * h
        em = oracle.energy_forces(s, p)["potential"]
        fd.append(-(ep - em) / (2 * h))
    an = np.array([ef["forces"][i, a] for i, a in idx])
    assert np.max(np.abs(np.array(fd) - an)) < 2e-6 * max(1.0, np.max(np.abs(an)))


def test_identical_species_equal_one_species():
    s = synth.make_bulk(400, seed_index=44, charged_frac=0.2, K=(10, 10, 10))
    t = s.copy()
    rng = np.random.default_rng(3)
    t.types = rng.integers(0, 2, size=s.n).astype(np.int32)
    t.A_tab = np.full((2, 2), s.A)
    t.sig_tab = np.full(2, s.sigma)
    t.a_tab = np.full(2, s.a)
    e0 = oracle.energy_forces(s)
    e1 = oracle.energy_forces(t)
    assert np.array_equal(e0["forces"], e1["forces"])
    for k in oracle.TERMS:  # energies to the last bits of the threads' reduction order
        assert e1[k] == pytest.approx(e0[k], rel=1e-13, abs=1e-13)


def test_mixture_is_neutral_and_uses_every_species():
    s = _mixture(301, seed=45)
    assert abs(np.sum(s.q)) < 1e-12
    assert set(np.unique(s.types)) == {0, 1, 2}
    assert np.array_equal(s.q, np.array([0.0, 1.0, -1.0])[s.types])
