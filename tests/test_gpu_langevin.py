"""Langevin (BAOAB) dynamics through gcme_step against the oracle.

The noise is counter-based (Philox4x64-10 at counter (step, bead), key
(seed, 0)), so the GPU and the oracle draw the same numbers; the FP64 path
follows the oracle's trajectory to the FP64 bounds, the FP32 path to the
FP32 ones.  The step counter makes a trajectory independent of how its
steps are split into calls, and restartable from a checkpoint.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import ctx, lib

pytestmark = pytest.mark.gpu

GAMMA, KT, SEED = 1.0, 1.0, 2024


def _run(s, precision, nsteps, chunks=None, gamma=GAMMA, kT=KT, seed=SEED, step0=None):
    import torch
    g = lib()
    sysg = g.System(ctx(), g.params_from(s, precision, gamma=gamma, kT=kT, seed=seed), s.q,
                    s.bonds)
    if step0 is not None:
        sysg.set_step_count(step0)
    vdt = torch.float64 if precision == 1 else torch.float32
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    vel = torch.tensor(s.vel, dtype=vdt, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    for n in (chunks or [nsteps]):
        sysg.step(pos, vel, n, E)
    torch.cuda.synchronize()
    steps = sysg.info().steps
    out = pos.cpu().numpy(), vel.cpu().numpy().astype(np.float64), E.cpu().numpy(), steps
    sysg.close()
    return out


def test_fp64_langevin_follows_oracle():
    s = synth.make_polyelectrolyte(n_chains=5, chain_len=10, n_solvent=700, seed_index=120,
                                   K=(12, 12, 12))
    pos, vel, E, steps = _run(s, 1, 30)
    assert steps == 30
    p1, v1, hist = oracle.langevin_baoab(s, 30, GAMMA, KT, SEED)
    assert np.max(np.abs(pos - p1)) < 1e-7
    assert np.max(np.abs(vel - v1)) < 1e-6
    assert abs(E[8] - hist[-1]["potential"]) < 1e-8 * abs(hist[-1]["potential"])
    assert abs(E[9] - hist[-1]["kinetic"]) < 1e-7 * hist[-1]["kinetic"]


@pytest.mark.parametrize("geom", [synth.GEOM_BULK, synth.GEOM_SLAB_PC])
def test_fp32_langevin_follows_oracle(geom):
    if geom == synth.GEOM_BULK:
        s = synth.make_bulk(1500, seed_index=121, charged_frac=0.2, K=(12, 12, 12))
    else:
        s = synth.make_slab_fluid(synth.GEOM_SLAB_PC, 900, charged_frac=0.2, seed_index=122)
    pos, vel, E, _ = _run(s, 0, 20)
    p1, v1, hist = oracle.langevin_baoab(s, 20, GAMMA, KT, SEED)
    assert np.max(np.abs(pos - p1)) < 1e-4
    assert np.max(np.abs(vel - v1)) < 1e-3
    tot = E[8] + E[9]
    tot_o = hist[-1]["potential"] + hist[-1]["kinetic"]
    assert abs(tot - tot_o) / abs(tot_o) < 1e-5
    # the noise did act: the trajectory left the NVE one
    p0, _, _ = oracle.velocity_verlet(s, 20)
    assert np.max(np.abs(pos - p0)) > 1e-3


def test_steps_split_into_calls_and_restart_are_bit_identical():
    s = synth.make_bulk(1000, seed_index=123, charged_frac=0.2, K=(10, 10, 10))
    a = _run(s, 0, 20)
    b = _run(s, 0, 20, chunks=[7, 1, 12])
    assert a[3] == b[3] == 20
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # checkpoint after 8 steps, restart with the counter set to 8
    c8 = _run(s, 0, 8)
    t = synth.make_bulk(1000, seed_index=123, charged_frac=0.2, K=(10, 10, 10))
    t.pos, t.vel = c8[0], c8[1]
    c = _run(t, 0, 12, step0=8)
    assert c[3] == 20
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    # another seed, another trajectory
    d = _run(s, 0, 20, seed=SEED + 1)
    assert not np.array_equal(a[0], d[0])


def test_langevin_thermalises_cold_fluid():
    """From rest, a GCMe fluid reaches the bath temperature: the mean
    kinetic energy over the last 200 of 600 steps is 3/2 N kT within 3 %."""
    import torch
    g = lib()
    s = synth.make_bulk(3000, seed_index=124, charged_frac=0.1, K=(16, 16, 16))
    kT = 1.5
    sysg = g.System(ctx(), g.params_from(s, 0, gamma=2.0, kT=kT, seed=5), s.q)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    vel = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.step(pos, vel, 400, E)
    ke = []
    for _ in range(200):
        sysg.step(pos, vel, 1, E)
        ke.append(E[9].item())
    assert abs(np.mean(ke) / (1.5 * s.n * kT) - 1.0) < 0.03
