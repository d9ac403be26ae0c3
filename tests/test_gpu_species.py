"""Several species (per-type A_ij, sigma_i, a_i) through the C ABI against
the oracle: forces and energies of charged mixtures in the three
geometries (FP32 and FP64 paths), the neighbour set, the equivalence of
identical species with one species, trajectories, and batches that mix
systems with and without species tables."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (ENERGY_RTOL_FP32, ENERGY_RTOL_FP64, FORCE_RTOL_FP32, FORCE_RTOL_FP64,
                      ctx, lib, rel_rms)

pytestmark = pytest.mark.gpu

A3 = np.array([[25.0, 27.0, 26.0], [27.0, 25.0, 30.0], [26.0, 30.0, 25.0]])
S3 = np.array([0.5, 0.6, 0.4])
a3 = np.array([0.5, 0.7, 0.35])


def _mixture(n, geometry=synth.GEOM_BULK, seed=130):
    return synth.make_mixture(n, (0.6, 0.2, 0.2), (0.0, 1.0, -1.0), A3, S3, a3,
                              seed_index=seed, geometry=geometry)


def _forces(s, precision=0, cell_factor=0, pair_path=0):
    import torch
    g = lib()
    sysg = g.System(ctx(), g.params_from(s, precision, cell_factor, pair_path), s.q, s.bonds,
                    types=s.types)
    p = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    F = torch.zeros(3 * s.n, dtype=torch.int64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.forces(p, F, E)
    torch.cuda.synchronize()
    f = F.cpu().numpy().reshape(3, -1).T.astype(np.float64) / g.FORCE_SCALE
    return f, dict(zip(oracle.TERMS + ("potential", "kinetic"), E.cpu().numpy().tolist())), \
        F.cpu().numpy()


CASES = {
    "bulk": lambda: _mixture(2500),
    "slab_nm": lambda: _mixture(1500, synth.GEOM_SLAB_NM, 131),
    "slab_pc": lambda: _mixture(1200, synth.GEOM_SLAB_PC, 132),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_species_forces_match_oracle(name, precision):
    s = CASES[name]()
    f, e, _ = _forces(s, precision)
    ref = oracle.energy_forces(s)
    ftol, etol = (FORCE_RTOL_FP32, ENERGY_RTOL_FP32) if precision == 0 else \
        (FORCE_RTOL_FP64, ENERGY_RTOL_FP64)
    assert rel_rms(f, ref["forces"]) <= ftol
    assert abs(e["potential"] - ref["potential"]) <= etol * abs(ref["potential"])
    scale = sum(abs(ref[t]) for t in oracle.TERMS)
    for t in oracle.TERMS:
        assert abs(e[t] - ref[t]) <= (1e-6 if precision == 0 else 1e-10) * scale, t


def test_species_pair_set_is_the_same_rule():
    import torch
    g = lib()
    s = CASES["slab_pc"]()
    sysg = g.System(ctx(), g.params_from(s), s.q, s.bonds, types=s.types)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    cap = 2_000_000
    trip = torch.zeros(3 * cap, dtype=torch.int32, device="cuda:0")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    sysg.debug_pairs(pos, trip, cap, cnt)
    torch.cuda.synchronize()
    got = trip[: 3 * int(cnt.item())].cpu().numpy().reshape(-1, 3)
    epos, _, _, n = oracle.electrostatic_beads(s)
    ref = oracle.pair_set(epos, s.box, s.rc)
    ref = ref[ref[:, 0] < n]
    assert np.array_equal(np.unique(got, axis=0), np.unique(ref, axis=0))


def test_identical_species_agree_with_one_species():
    s = synth.make_bulk(2000, seed_index=133, charged_frac=0.2, K=(12, 12, 12))
    t = s.copy()
    t.types = np.random.default_rng(4).integers(0, 3, size=s.n).astype(np.int32)
    t.A_tab = np.full((3, 3), s.A)
    t.sig_tab = np.full(3, s.sigma)
    t.a_tab = np.full(3, s.a)
    f0, e0, _ = _forces(s)
    f1, e1, _ = _forces(t)
    assert rel_rms(f1, f0) < 1e-6
    assert abs(e1["potential"] - e0["potential"]) < 1e-7 * abs(e0["potential"])


def test_species_paths_without_tables_support_are_rejected():
    g = lib()
    s = CASES["bulk"]()
    for factor, path in ((2, 0), (1, 1)):
        with pytest.raises(g.GcmeError):
            g.System(ctx(), g.params_from(s, 0, factor, path), s.q, types=s.types)


def test_species_trajectory_matches_oracle():
    import torch
    g = lib()
    s = _mixture(1500, seed=134)
    sysg = g.System(ctx(), g.params_from(s, 1), s.q, types=s.types)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    vel = torch.tensor(s.vel, dtype=torch.float64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.step(pos, vel, 20, E)
    torch.cuda.synchronize()
    p1, v1, hist = oracle.velocity_verlet(s, 20)
    assert np.max(np.abs(pos.cpu().numpy() - p1)) < 1e-7
    assert abs(E[8].item() - hist[-1]["potential"]) < 1e-9 * abs(hist[-1]["potential"])


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_with_and_without_species_matches_singles(mode):
    import torch
    g = lib()
    systems = [_mixture(900, seed=135), synth.make_bulk(800, seed_index=136, K=(10, 10, 10)),
               _mixture(700, synth.GEOM_SLAB_PC, 137)]
    b = g.Batch(ctx(), [g.params_from(s) for s in systems], [s.q for s in systems],
                [s.bonds for s in systems], types=[s.types for s in systems])
    b.set_state(np.concatenate([s.pos for s in systems]),
                np.concatenate([s.vel for s in systems]).astype(np.float32))
    b.step(10, mode)
    pos, vel, E = b.get_state()
    for k, s in enumerate(systems):
        sysg = g.System(ctx(), g.params_from(s), s.q, s.bonds, types=s.types)
        p = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
        v = torch.tensor(s.vel, dtype=torch.float32, device="cuda:0")
        e = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
        sysg.step(p, v, 10, e)
        torch.cuda.synchronize()
        lo, hi = b.offsets[k], b.offsets[k + 1]
        if s.types is None:
            # a one-species system in a species batch takes the table path:
            # the same physics, another FP32 rounding order
            assert np.max(np.abs(pos[lo:hi] - p.cpu().numpy())) < 1e-4
        else:
            assert np.array_equal(pos[lo:hi], p.cpu().numpy())
            assert np.array_equal(vel[lo:hi], v.cpu().numpy())
