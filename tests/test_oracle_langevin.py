"""Pins of the oracle's Langevin integrator and its noise generator.

The paper integrates the Langevin equations of motion (canonical ensemble)
without naming a splitting or a friction; the oracle takes BAOAB with
Philox4x64-10 noise.  Pinned here against things other than the oracle:

* the generator, word for word, against numpy's Philox (a library routine);
* the noise: mean, variance, normality (Kolmogorov-Smirnov), independence;
* for a harmonic oscillator BAOAB samples positions exactly, <x^2> = kT/k,
  and velocities with <v^2> = kT (1 - (omega dt)^2/4), at any stable step
  (Leimkuhler and Matthews 2013); the ABOBA and OBABO orderings each miss
  one of the two;
* free particles: <v(t) . v(0)> = 3 kT exp(-gamma t) and <v^2> stays 3 kT;
* gamma = 0 reduces BAOAB to velocity Verlet.
"""
import types

import numpy as np
import pytest
from scipy import stats

import oracle
import synth


@pytest.mark.parametrize("key,ctr", [
    ((0x0123456789ABCDEF, 0xFEDCBA9876543210), (5, 7, 11, 13)),
    ((0, 0), (0, 0, 0, 0)),
    ((2**64 - 1, 2**64 - 1), (2**64 - 2, 2**64 - 1, 2**64 - 1, 2**64 - 1)),
    ((2403081480, 0), (2**64 - 1, 3, 0, 0)),  # the next counter carries into word 1
])
def test_philox_matches_numpy(key, ctr):
    k = np.array(key, dtype=np.uint64)
    c = np.array(ctr, dtype=np.uint64)
    ref = np.random.Philox(key=k, counter=c).random_raw(12)
    # numpy advances the 256-bit counter before each block
    blocks, cc = [], [int(x) for x in ctr]
    for _ in range(3):
        v = sum(w << (64 * i) for i, w in enumerate(cc)) + 1
        cc = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
        blocks.append(oracle.philox4x64(np.array(cc, dtype=np.uint64)[None], k[None])[0])
    assert np.array_equal(np.concatenate(blocks), ref)


def test_noise_is_standard_normal_and_independent():
    z = np.concatenate([oracle.langevin_noise(7, n, 20000) for n in range(5)])
    assert z.shape == (100000, 3)
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / z.size)
    for a in range(3):
        assert stats.kstest(z[:, a], "norm").pvalue > 1e-3
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(3))) < 5.0 / np.sqrt(z.shape[0])
    # another step, bead or seed gives another stream
    a = oracle.langevin_noise(7, 3, 100)
    assert not np.allclose(a, oracle.langevin_noise(7, 4, 100))
    assert not np.allclose(a, oracle.langevin_noise(8, 3, 100))
    assert not np.allclose(a[1:], oracle.langevin_noise(7, 3, 101)[2:])
    assert np.array_equal(a, oracle.langevin_noise(7, 3, 100))


def _oscillators(n, dt, seed=3):
    rng = np.random.default_rng(seed)
    return types.SimpleNamespace(pos=rng.normal(size=(n, 3)), vel=rng.normal(size=(n, 3)), dt=dt)


def _harmonic(k):
    return lambda x: (-k * x, 0.5 * k * float(np.sum(x * x)))


def _moments(stepper, s, nsteps, burn):
    """<x^2> and <v^2> per component over steps burn..nsteps of a
    stepper(pos, vel, n) -> (pos, vel)."""
    pos, vel = s.pos.copy(), s.vel.copy()
    x2 = v2 = 0.0
    cnt = 0
    for n in range(nsteps):
        pos, vel = stepper(pos, vel, n)
        if n >= burn:
            x2 += float(np.mean(pos * pos))
            v2 += float(np.mean(vel * vel))
            cnt += 1
    return x2 / cnt, v2 / cnt


def test_baoab_harmonic_oscillator_closed_forms():
    """omega dt = 1 (half the stability limit).  For harmonic forces BAOAB
    samples positions exactly, <x^2> = kT/k, and velocities with
    <v^2> = kT (1 - (omega dt)^2 / 4).  The plausible wrong orderings miss
    one of the two: ABOBA gives <v^2> = kT / (1 - (omega dt)^2/4), OBABO
    gives <x^2> = kT / (k (1 - (omega dt)^2/4))."""
    k, kT, gamma, dt = 1.0, 1.0, 1.0, 1.0
    s = _oscillators(4000, dt)
    f = 1.0 - dt * dt * k / 4.0

    def baoab(pos, vel, n):
        t = types.SimpleNamespace(pos=pos, vel=vel, dt=dt)
        p, v, _ = oracle.langevin_baoab(t, 1, gamma, kT, seed=11, step0=n, force_fn=_harmonic(k))
        return p, v

    x2, v2 = _moments(baoab, s, 1500, 200)
    assert abs(x2 - kT / k) < 0.01, x2
    assert abs(v2 - kT * f) < 0.01, v2

    c1 = np.exp(-gamma * dt)
    c2 = np.sqrt((1 - c1 * c1) * kT)

    def aboba(pos, vel, n):
        pos = pos + 0.5 * dt * vel
        vel = vel - 0.5 * dt * k * pos
        vel = c1 * vel + c2 * oracle.langevin_noise(11, n, pos.shape[0])
        vel = vel - 0.5 * dt * k * pos
        pos = pos + 0.5 * dt * vel
        return pos, vel

    def obabo(pos, vel, n):
        vel = c1 * vel + c2 * oracle.langevin_noise(11, 2 * n, pos.shape[0])
        vel = vel - 0.5 * dt * k * pos
        pos = pos + dt * vel
        vel = vel - 0.5 * dt * k * pos
        vel = c1 * vel + c2 * oracle.langevin_noise(11, 2 * n + 1, pos.shape[0])
        return pos, vel

    _, v2_aboba = _moments(aboba, s, 1500, 200)
    x2_obabo, _ = _moments(obabo, s, 1500, 200)
    assert abs(v2_aboba - kT / f) < 0.02 and abs(v2_aboba - kT * f) > 0.3
    assert abs(x2_obabo - kT / (k * f)) < 0.02 and abs(x2_obabo - kT / k) > 0.2


def test_free_particle_velocity_autocorrelation():
    gamma, kT, dt, n = 2.0, 1.0, 0.05, 30000
    rng = np.random.default_rng(5)
    s = types.SimpleNamespace(pos=np.zeros((n, 3)), vel=rng.normal(size=(n, 3)) * np.sqrt(kT),
                              dt=dt)
    v0 = s.vel.copy()
    zero = lambda x: (np.zeros_like(x), 0.0)
    _, v, hist = oracle.langevin_baoab(s, 20, gamma, kT, seed=9, force_fn=zero)
    corr = float(np.mean(np.sum(v * v0, axis=1))) / (3 * kT)
    assert abs(corr - np.exp(-gamma * 20 * dt)) < 5.0 / np.sqrt(n)
    for h in hist:  # stationary: <v^2> = 3 kT per bead
        assert abs(2 * h["kinetic"] / n - 3 * kT) < 0.05


def test_gamma_zero_is_velocity_verlet():
    s = synth.make_bulk(300, seed_index=60, charged_frac=0.2, K=(8, 8, 8))
    p1, v1, h1 = oracle.velocity_verlet(s, 5)
    p2, v2, h2 = oracle.langevin_baoab(s, 5, gamma=0.0, kT=1.0, seed=1)
    assert np.max(np.abs(p1 - p2)) < 1e-12
    assert np.max(np.abs(v1 - v2)) < 1e-12
    assert abs(h1[-1]["potential"] - h2[-1]["potential"]) < 1e-9 * abs(h1[-1]["potential"])
