"""Pins of explicit electrode beads (one close-packed layer of beads of size
d/2 per electrode, a frozen species) in the oracle.

* The Gaussian-core energy of a fluid bead at height h above a periodic
  close-packed layer, averaged over the layer's lateral unit cell, equals
  the continuum wall u_w(h) = A n_s (3/(2 pi s_w))^{1/2} exp(-3 h^2/(2 s_w)),
  n_s = 2/(sqrt(3) b^2), s_w = sigma_i^2 + sigma_e^2: the average of a
  periodic lattice sum over a cell is the plane integral times the areal
  density, which the continuum wall is (an exact identity; the uniform
  lateral grid makes the average converge spectrally).
* Frozen species keep positions and velocities; with them the integrator
  still conserves energy (they act as a fixed external field).
* Image-charge geometry: electrode beads in the plane z = 0 coincide with
  their images (r = 0, the smeared-charge limit), and the forces on the
  fluid stay the gradient of the energy.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _layer_energy(h, x, y, nx=16, ny=18, b=0.5):
    layer = synth.hcp_layer(nx, ny, b, 0.0)
    box = np.array([nx * b, ny * b * math.sqrt(3.0) / 2.0, 40.0])
    pos = np.concatenate([[[x, y, h + 10.0]], layer + [0.0, 0.0, 10.0]])
    types = np.concatenate([[0], np.ones(layer.shape[0], np.int32)]).astype(np.int32)
    A = np.full((2, 2), 25.0)
    A[1, 1] = 0.0  # only the fluid-electrode term
    e = oracle.pairs(pos, np.zeros(pos.shape[0]), types, A, np.array([0.5, 0.25]),
                     np.array([0.5, 0.25]), box, 3.0, 1.0, 1.0, do_real=False)
    return e["gc"]


@pytest.mark.parametrize("h", [0.3, 0.6, 1.0])
def test_layer_average_is_the_continuum_wall(h):
    b = 0.5
    cx, cy = b, b * math.sqrt(3.0)  # rectangular cell holding two lattice points
    m = 12
    vals = [_layer_energy(h, (i + 0.5) * cx / m, (j + 0.5) * cy / m)
            for i in range(m) for j in range(m)]
    wA, ws2 = synth._wall_params(25.0, 0.5)  # A n_s, sigma_i^2 + sigma_e^2
    e_wall, _ = oracle.walls(np.array([[0.0, 0.0, h]]), 1000.0, wA, ws2)
    assert np.mean(vals) == pytest.approx(e_wall, rel=1e-9)
    # the lattice is corrugated at these heights, but only slightly
    assert np.std(vals) < 0.05 * np.mean(vals)


def test_frozen_electrodes_stay_and_energy_is_conserved():
    s = synth.make_electrode_slab(synth.GEOM_SLAB_NM, nx=12, ny=14, H=9.0, n_chains=3,
                                  chain_len=8, sigma_q=0.3, K=(12, 12, 48))
    frozen = s.types == 1
    s.vel[frozen] = 0.0
    p, v, hist = oracle.velocity_verlet(s, 60)
    assert np.array_equal(p[frozen], s.pos[frozen]) and np.array_equal(v[frozen], 0 * v[frozen])
    assert np.max(np.abs(p[~frozen] - s.pos[~frozen])) > 1e-2
    e = [h["potential"] + h["kinetic"] for h in hist]
    assert max(abs(x - e[0]) for x in e) < 2e-3 * abs(e[0])
    # Langevin leaves them too
    p2, v2, _ = oracle.langevin_baoab(s, 5, gamma=1.0, kT=1.0, seed=3)
    assert np.array_equal(p2[frozen], s.pos[frozen]) and np.array_equal(v2[frozen], v[frozen])


def test_electrode_image_geometry_forces_are_gradient():
    s = synth.make_electrode_slab(synth.GEOM_SLAB_PC, nx=10, ny=12, H=7.0, n_chains=2,
                                  chain_len=6, sigma_q=0.4, K=(10, 10, 32))
    s.kappa = 0.9
    ef = oracle.energy_forces(s)
    assert np.isfinite(ef["potential"])
    fluid = np.nonzero(s.types == 0)[0]
    charged = fluid[s.q[fluid] != 0]
    idx = [(int(charged[k]), 2) for k in range(4)] + [(int(fluid[k]), k % 3) for k in range(4)]
    h = 1e-5
    for i, a in idx:
        p = s.pos.copy()
        p[i, a] += h
        ep = oracle.energy_forces(s, p)["potential"]
        p[i, a] -= 2 * h
        em = oracle.energy_forces(s, p)["potential"]
        assert abs(-(ep - em) / (2 * h) - ef["forces"][i, a]) < 2e-6 * max(1.0, abs(ef["forces"][i, a]))


def test_electrode_slab_is_neutral_with_opposite_plates():
    s = synth.make_electrode_slab(synth.GEOM_SLAB_NM, nx=16, ny=18, H=12.0, sigma_q=0.2)
    lo = (s.types == 1) & (s.pos[:, 2] < 1.0)
    hi = (s.types == 1) & (s.pos[:, 2] > 1.0)
    assert lo.sum() == hi.sum() == 288
    area = s.box[0] * s.box[1]
    assert np.sum(s.q[lo]) / area == pytest.approx(0.2, rel=1e-12)
    assert np.sum(s.q[hi]) / area == pytest.approx(-0.2, rel=1e-12)
    assert abs(np.sum(s.q)) < 1e-9
