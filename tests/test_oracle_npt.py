"""Pins of the oracle's pressure (Eq. pres_virial) and Monte Carlo barostat.

* An ideal gas in the NpT ensemble has the volume density V^N exp(-p V / kT),
  so <V> = (N + 1) kT / p exactly; the barostat must reproduce it (a
  missing or wrong Jacobian term gives N kT / p or kT / p).
* The configurational pressure tr(W)/(3V) equals -dU/dV for isotropic
  scaling of box and positions (finite differences, all force terms).
* The pressure of an ideal configuration (no interactions) is N kT / V.
"""
import types

import numpy as np
import pytest

import oracle
import synth


def test_ideal_gas_npt_volume():
    n, p, kT = 12, 0.8, 1.0
    box = np.full(3, 3.0)
    pos = np.random.default_rng(0).uniform(0, 3.0, size=(n, 3))
    s = types.SimpleNamespace()
    vols, acc = [], 0
    for m in range(40000):
        pos, box, a = oracle.barostat_move(s, pos, box, p, kT, 0.6, seed=21, move=m,
                                           energy_fn=lambda x, b: 0.0)
        acc += a
        if m >= 2000:
            vols.append(float(np.prod(box)))
    v = np.array(vols)
    ref = (n + 1) * kT / p
    # blocks of 1000 moves for the error of the mean
    blocks = v[: len(v) // 1000 * 1000].reshape(-1, 1000).mean(axis=1)
    se = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(v.mean() - ref) < 4 * se + 0.01 * ref, (v.mean(), ref, se)
    assert abs(v.mean() - n * kT / p) > 4 * se  # distinguishes the Jacobian's N + 1
    assert 0.2 < acc / 40000 < 0.9


def test_configurational_pressure_is_volume_derivative():
    s = synth.make_polyelectrolyte(n_chains=3, chain_len=6, n_solvent=150, seed_index=150,
                                   K=(16, 16, 16))
    s.kappa = 1.0
    V = float(np.prod(s.box))
    p_conf = oracle.pressure(s, kT=0.0)
    h = 1e-6

    def U(scale):
        t = s.copy()
        t.box = s.box * scale
        return oracle.energy_forces(t, s.pos * scale)["potential"]

    dU = (U((1 + h) ** (1 / 3)) - U((1 - h) ** (1 / 3))) / (2 * h * V)
    assert p_conf == pytest.approx(-dU, rel=1e-5, abs=1e-6)


def test_ideal_configuration_pressure():
    s = synth.make_bulk(100, seed_index=151, charged_frac=0.0, K=(8, 8, 8))
    s.A = 0.0
    V = float(np.prod(s.box))
    assert oracle.pressure(s, kT=1.5) == pytest.approx(100 * 1.5 / V, rel=1e-14)


def test_barostat_move_is_deterministic_and_reversible_in_law():
    s = synth.make_bulk(200, seed_index=152, charged_frac=0.1, K=(10, 10, 10))
    a = oracle.barostat_move(s, s.pos, s.box, 2.0, 1.0, 0.02, seed=5, move=3)
    b = oracle.barostat_move(s, s.pos, s.box, 2.0, 1.0, 0.02, seed=5, move=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    u0, u1 = oracle.barostat_uniforms(5, 3)
    assert 0.0 <= u0 < 1.0 and 0.0 <= u1 < 1.0
    assert oracle.barostat_uniforms(5, 4) != (u0, u1)
