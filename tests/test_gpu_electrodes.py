"""Explicit electrodes (frozen close-packed layers of charged beads of size
d/2) through the C ABI against the oracle, in both slab geometries: forces
and energies, and trajectories in which the electrode beads stay put."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (ENERGY_RTOL_FP32, ENERGY_RTOL_FP64, FORCE_RTOL_FP32, FORCE_RTOL_FP64,
                      ctx, lib, rel_rms)

pytestmark = pytest.mark.gpu


def _slab(geometry):
    return synth.make_electrode_slab(geometry, nx=16, ny=18, H=12.0, n_chains=6, chain_len=10,
                                     sigma_q=0.3, seed_index=140 + geometry)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("geometry", [synth.GEOM_SLAB_NM, synth.GEOM_SLAB_PC])
def test_electrode_forces_match_oracle(geometry, precision):
    import torch
    g = lib()
    s = _slab(geometry)
    sysg = g.System(ctx(), g.params_from(s, precision), s.q, s.bonds, types=s.types)
    p = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    F = torch.zeros(3 * s.n, dtype=torch.int64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.forces(p, F, E)
    torch.cuda.synchronize()
    f = F.cpu().numpy().reshape(3, -1).T.astype(np.float64) / g.FORCE_SCALE
    e = E.cpu().numpy()
    ref = oracle.energy_forces(s)
    ftol, etol = (FORCE_RTOL_FP32, ENERGY_RTOL_FP32) if precision == 0 else \
        (FORCE_RTOL_FP64, ENERGY_RTOL_FP64)
    fluid = s.types == 0
    assert rel_rms(f[fluid], ref["forces"][fluid]) <= ftol
    assert rel_rms(f, ref["forces"]) <= ftol
    assert abs(e[8] - ref["potential"]) <= etol * abs(ref["potential"])
    assert e[6] == 0.0  # no continuum wall


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_electrodes_stay_put_and_trajectory_matches(gamma):
    import torch
    g = lib()
    s = _slab(synth.GEOM_SLAB_PC)
    sysg = g.System(ctx(), g.params_from(s, 1, gamma=gamma, seed=9), s.q, s.bonds,
                    types=s.types)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    vel = torch.tensor(s.vel, dtype=torch.float64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.step(pos, vel, 15, E)
    torch.cuda.synchronize()
    p = pos.cpu().numpy()
    frozen = s.types == 1
    assert np.array_equal(p[frozen], s.pos[frozen])
    assert np.array_equal(vel.cpu().numpy()[frozen], s.vel[frozen])
    if gamma == 0.0:
        p1, _, hist = oracle.velocity_verlet(s, 15)
    else:
        p1, _, hist = oracle.langevin_baoab(s, 15, gamma, 1.0, 9)
    assert np.max(np.abs(p - p1)) < 1e-7
    assert abs(E[9].item() - hist[-1]["kinetic"]) < 1e-7 * hist[-1]["kinetic"]
