"""The Verlet neighbour-list pair path.

The list holds every (j, image) within rc + skin (skin 0.4) of each real
bead and is reused until a bead has moved more than skin / 2 since the
build.  Checked here: the pair set and the forces at positions other than
the build's (beads that crossed the box included) equal those of a fresh
build bit for bit; the rebuild schedule follows the displacement rule; a
system whose lists overflow falls back to the 27-cell kernel and stays at
parity with the oracle; trajectories agree with the oracle's.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from gpu_util import ENERGY_RTOL_FP32, FORCE_RTOL_FP32, ctx, lib, rel_rms

pytestmark = pytest.mark.gpu

SKIN = 0.4


def _system(s, path=1):
    g = lib()
    return g.System(ctx(), g.params_from(s, 0, 1, path), s.q, s.bonds)


def _forces(sysg, s, pos):
    import torch
    g = lib()
    p = torch.tensor(pos, dtype=torch.float64, device="cuda:0")
    F = torch.zeros(3 * s.n, dtype=torch.int64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.forces(p, F, E)
    torch.cuda.synchronize()
    return F.cpu().numpy(), E.cpu().numpy()


def _pairs(sysg, s, pos):
    import torch
    p = torch.tensor(pos, dtype=torch.float64, device="cuda:0")
    cap = 2_000_000
    trip = torch.zeros(3 * cap, dtype=torch.int32, device="cuda:0")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    sysg.debug_pairs(p, trip, cap, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k <= cap
    return trip[: 3 * k].cpu().numpy().reshape(-1, 3)


def _oracle_pairs(s, pos):
    t = dataclasses.replace(s, pos=pos)
    epos, _, _, n = oracle.electrostatic_beads(t)
    ref = oracle.pair_set(epos, s.box, s.rc)
    return ref[ref[:, 0] < n]


def _displaced(s, amp, seed):
    rng = np.random.default_rng(seed)
    return s.pos + rng.uniform(-amp, amp, size=s.pos.shape)


@pytest.mark.parametrize("name", ["bulk", "slab_pc", "poly"])
def test_reused_list_is_bit_identical_to_fresh_build(name):
    """Build the list at X' (displaced by < skin/2 per bead, so that beads
    near the faces sit on the other side of the box), evaluate at X: no
    rebuild, and forces, energies and the pair set equal a fresh build at X."""
    s = {"bulk": synth.make_bulk(1500, seed_index=90, charged_frac=0.3, K=(12, 12, 12)),
         "slab_pc": synth.make_slab_fluid(synth.GEOM_SLAB_PC, 900, charged_frac=0.2,
                                          seed_index=91),
         "poly": synth.make_polyelectrolyte(n_chains=6, chain_len=10, n_solvent=1000,
                                            seed_index=92, K=(12, 12, 12))}[name]
    X = s.pos
    Xb = _displaced(s, 0.1, 1)  # |dx| <= 0.1 sqrt(3) < skin / 2
    crossed = np.floor(Xb / s.box) != np.floor(X / s.box)
    assert crossed.any()  # the image-shift correction is exercised
    reused = _system(s)
    _forces(reused, s, Xb)
    assert reused.info().list_builds == 1
    f1, e1 = _forces(reused, s, X)
    assert reused.info().list_builds == 1  # no rebuild: the list of X' serves X
    fresh = _system(s)
    f0, e0 = _forces(fresh, s, X)
    assert np.array_equal(f0, f1)
    assert np.array_equal(e0, e1)
    pr = _pairs(reused, s, X)
    assert reused.info().list_builds == 1
    ref = _oracle_pairs(s, X)
    a, b = np.unique(pr, axis=0), np.unique(ref, axis=0)
    assert a.shape[0] == pr.shape[0] and np.array_equal(a, b)


def test_rebuild_schedule_follows_displacement():
    s = synth.make_bulk(800, seed_index=93, charged_frac=0.1, K=(10, 10, 10))
    sysg = _system(s)
    _forces(sysg, s, s.pos)
    assert sysg.info().list_builds == 1
    p = s.pos.copy()
    p[17, 0] += 0.5 * SKIN - 0.01  # just inside the bound: list kept
    _forces(sysg, s, p)
    assert sysg.info().list_builds == 1
    p[17, 0] += 0.02  # now beyond skin / 2 from the build: rebuilt
    f, e = _forces(sysg, s, p)
    assert sysg.info().list_builds == 2
    f0, e0 = _forces(_system(s), s, p)
    assert np.array_equal(f, f0) and np.array_equal(e, e0)


def test_cell_path_keeps_no_list():
    s = synth.make_bulk(500, seed_index=94, charged_frac=0.1, K=(8, 8, 8))
    info = _system(s, 2).info()
    assert info.pair_path == 2 and info.list_stride == 0 and info.list_builds == 0
    info = _system(s, 0).info()
    assert info.pair_path == 2 and info.list_stride == 0  # the library's choice
    info = _system(s, 1).info()
    assert info.pair_path == 1 and info.list_stride > 0
    g = lib()
    with pytest.raises(g.GcmeError):
        g.System(ctx(), g.params_from(s, 1, 1, 1), s.q)  # FP64 has no list path


@pytest.mark.parametrize("side", [6.0, 8.0])
def test_overflowing_lists_fall_back_to_cell_kernel(side):
    """Beads packed into a side^3 corner of a 12^3 box: the list stride is
    sized from the mean density, so the lists overflow (side 8: a lane
    sublist exceeds the stride; side 6: the build buffer of 1024 candidates).
    The system is evaluated by the 27-cell kernel and stays at parity."""
    s = synth.make_bulk(2000, rho=2000 / 12.0 ** 3, seed_index=95, charged_frac=0.2,
                        K=(12, 12, 12))
    s.pos = s.pos * (side / 12.0)
    sysg = _system(s)
    f, e = _forces(sysg, s, s.pos)
    ref = oracle.energy_forces(s)
    got = f.reshape(3, -1).T.astype(np.float64) / lib().FORCE_SCALE
    assert rel_rms(got, ref["forces"]) <= FORCE_RTOL_FP32
    assert abs(e[8] - ref["potential"]) <= ENERGY_RTOL_FP32 * abs(ref["potential"])
    _forces(sysg, s, s.pos)
    assert sysg.info().list_builds == 2  # overflowed lists are rebuilt every evaluation
    pr = _pairs(sysg, s, s.pos)
    ref_p = _oracle_pairs(s, s.pos)
    a, b = np.unique(pr, axis=0), np.unique(ref_p, axis=0)
    assert a.shape[0] == pr.shape[0] and np.array_equal(a, b)


def test_list_trajectory_matches_oracle_and_rebuilds():
    """60 velocity-Verlet steps of a charged fluid on the list path: several
    rebuilds happen inside the captured step graph, and the trajectory stays
    with the oracle's (and with the 27-cell path's) to FP32 accuracy."""
    import torch
    g = lib()
    s = synth.make_bulk(1200, seed_index=96, charged_frac=0.2, K=(12, 12, 12))
    out = {}
    for path in (1, 2):
        sysg = _system(s, path)
        pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
        vel = torch.tensor(s.vel, dtype=torch.float32, device="cuda:0")
        E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
        sysg.step(pos, vel, 60, E)
        torch.cuda.synchronize()
        out[path] = (pos.cpu().numpy(), E.cpu().numpy(), sysg.info().list_builds)
    assert out[1][2] >= 3 and out[2][2] == 0
    p1, _, hist = oracle.velocity_verlet(s, 60)
    for path in (1, 2):
        assert np.max(np.abs(out[path][0] - p1)) < 1e-3
        tot = out[path][1][8] + out[path][1][9]
        tot_o = hist[-1]["potential"] + hist[-1]["kinetic"]
        assert abs(tot - tot_o) / abs(tot_o) < 1e-5
    assert np.max(np.abs(out[1][0] - out[2][0])) < 1e-3
