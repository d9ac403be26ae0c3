"""Batched multi-system stepping and the continuous-batching server.

Every kernel's arithmetic for a system depends only on that system and all
force accumulation is fixed point, so a system's trajectory is bit-identical
alone, in a batch and in a served mix; reported energies may differ in the
last bits because warps of bead-parallel reductions can span systems.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import ctx, lib

pytestmark = pytest.mark.gpu


def _mixed_systems():
    return [synth.make_bulk(700, seed_index=70, charged_frac=0.1, K=(10, 10, 10)),
            synth.make_polyelectrolyte(n_chains=5, chain_len=10, n_solvent=900, seed_index=71,
                                       K=(12, 12, 12)),
            synth.make_slab_fluid(synth.GEOM_SLAB_NM, 800, charged_frac=0.2, seed_index=72),
            synth.make_slab_fluid(synth.GEOM_SLAB_PC, 600, charged_frac=0.2, seed_index=73),
            synth.make_bulk(2100, seed_index=74, charged_frac=0.1, K=(15, 15, 15))]


def _params(g, s, path=0, gamma=0.0, seed=0):
    return g.params_from(s, pair_path=path, gamma=gamma, kT=1.0, seed=seed)


def _single_run(g, s, nsteps, path=0, gamma=0.0, seed=0, tuning=None):
    import torch
    sysg = g.System(ctx(), _params(g, s, path, gamma, seed), s.q, s.bonds)
    if tuning is not None:
        sysg.apply_tuning(tuning)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    vel = torch.tensor(s.vel, dtype=torch.float32, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.step(pos, vel, nsteps, E)
    torch.cuda.synchronize()
    out = pos.cpu().numpy(), vel.cpu().numpy(), E.cpu().numpy()
    sysg.close()
    return out


# the persistent launch (mode 1) evaluates pairs by the 27-cell kernel, so
# it is compared with single systems on that path; mode 0 on both paths
@pytest.mark.parametrize("mode,path,gamma", [(0, 1, 0.0), (0, 2, 0.0), (1, 2, 0.0),
                                             (0, 2, 1.0), (1, 2, 1.0)])
def test_batch_matches_single_systems(mode, path, gamma):
    """Also with Langevin noise: each system draws from its own seed and step
    counter, so its trajectory does not depend on the batch."""
    g = lib()
    systems = _mixed_systems()
    b = g.Batch(ctx(), [_params(g, s, path, gamma, 100 + k) for k, s in enumerate(systems)],
                [s.q for s in systems], [s.bonds for s in systems])
    b.set_state(np.concatenate([s.pos for s in systems]),
                np.concatenate([s.vel for s in systems]).astype(np.float32))
    b.step(12, mode)
    pos, vel, E = b.get_state()
    for k, s in enumerate(systems):
        lo, hi = b.offsets[k], b.offsets[k + 1]
        p1, v1, e1 = _single_run(g, s, 12, path, gamma, 100 + k)
        assert np.array_equal(pos[lo:hi], p1), f"system {k} positions differ"
        assert np.array_equal(vel[lo:hi], v1), f"system {k} velocities differ"
        assert np.allclose(E[k], e1, rtol=1e-9, atol=1e-9)


ITEM_TASKS = {"pair_split": 9, "pair_threads": 160, "pair_ctas_per_sm": 5, "pair_nelec": -2,
              "fft_lpb": [8, 8, 8], "fft_plane": True}


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_single_systems_item_tasks(mode):
    """Every warp taking the items' tasks (pair_nelec -2): a thread's sums
    depend only on its system's items and the two parts of the charged
    candidates, not on the warps of the CTA, so each trajectory is the same
    bit for bit alone and in the batch, per-phase graphs or the persistent
    launch (128-thread CTAs there, 160 here)."""
    g = lib()
    systems = _mixed_systems()
    b = g.Batch(ctx(), [_params(g, s, 2, 0.0, 100 + k) for k, s in enumerate(systems)],
                [s.q for s in systems], [s.bonds for s in systems])
    b.apply_tuning(ITEM_TASKS)
    b.set_state(np.concatenate([s.pos for s in systems]),
                np.concatenate([s.vel for s in systems]).astype(np.float32))
    b.step(12, mode)
    pos, vel, E = b.get_state()
    for k, s in enumerate(systems):
        lo, hi = b.offsets[k], b.offsets[k + 1]
        p1, v1, e1 = _single_run(g, s, 12, 2, 0.0, 100 + k, tuning=ITEM_TASKS)
        assert np.array_equal(pos[lo:hi], p1), f"system {k} positions differ"
        assert np.array_equal(vel[lo:hi], v1), f"system {k} velocities differ"
        assert np.allclose(E[k], e1, rtol=1e-9, atol=1e-9)


def test_persistent_launch_barrier_timeout_reports_error():
    """The persistent launch's grid barrier waits with a bound: a barrier
    that one CTA never reaches ends with GCME_ERR_TIMEOUT (the error word
    set by the kernel and read by the host), and the context stays usable."""
    g = lib()
    rc = ctx().barrier_timeout_probe(0.2)
    assert rc == -4
    s = synth.make_bulk(600, seed_index=75, K=(10, 10, 10))
    import oracle as _o
    from gpu_util import gpu_forces
    out = gpu_forces(s, 0)
    ref = _o.energy_forces(s)
    assert abs(out["energy"]["potential"] - ref["potential"]) <= 1e-6 * abs(ref["potential"])


def test_batch_energies_match_oracle():
    g = lib()
    systems = _mixed_systems()
    b = g.Batch(ctx(), [g.params_from(s) for s in systems], [s.q for s in systems],
                [s.bonds for s in systems])
    b.set_state(np.concatenate([s.pos for s in systems]),
                np.concatenate([s.vel for s in systems]).astype(np.float32))
    b.step(0)  # forces and energies of the initial state only
    _, _, E = b.get_state()
    for k, s in enumerate(systems):
        ref = oracle.energy_forces(s)
        assert abs(E[k, 8] - ref["potential"]) <= 1e-6 * abs(ref["potential"])


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_server_result_same_alone_and_in_mix(gamma):
    """Continuous batching: a request's result does not depend on what else
    is on the GPU (different sizes and geometries, admitted at different
    chunk boundaries), with or without Langevin noise."""
    g = lib()
    target = synth.make_polyelectrolyte(n_chains=6, chain_len=10, n_solvent=1500,
                                        seed_index=80, K=(12, 12, 12))
    others = [synth.make_bulk(900 + 300 * k, seed_index=81 + k, charged_frac=0.1)
              for k in range(4)]
    others.append(synth.make_slab_fluid(synth.GEOM_SLAB_PC, 700, seed_index=86))
    nsteps = 60

    def submit(srv, s, n):
        return srv.submit(_params(g, s, gamma=gamma, seed=s.n), s.pos, s.vel.astype(np.float32),
                          s.q, n, s.bonds)

    srv = g.Server(ctx(), 2 << 30, chunk_steps=7)
    t = submit(srv, target, nsteps)
    srv.drain(120)
    r, pos_alone, vel_alone = srv.poll(t, want_state=True)
    assert r.status == 0 and r.steps_done == nsteps
    e_alone = np.array(r.energy)
    srv.close()

    srv = g.Server(ctx(), 2 << 30, chunk_steps=7)
    tick = [submit(srv, others[0], 40), submit(srv, others[1], 25)]
    time.sleep(0.05)
    t = submit(srv, target, nsteps)
    for s in others[2:]:
        tick.append(submit(srv, s, 33))
        time.sleep(0.01)
    srv.drain(300)
    r, pos_mix, vel_mix = srv.poll(t, want_state=True)
    assert r.status == 0
    assert np.array_equal(pos_mix, pos_alone)
    assert np.array_equal(vel_mix, vel_alone)
    assert np.allclose(np.array(r.energy), e_alone, rtol=1e-9, atol=1e-9)
    for tk in tick:
        rr, _, _ = srv.poll(tk)
        assert rr.status == 0
    st = srv.stats()
    assert st["completed"] == 1 + len(tick) and st["peak_active"] >= 2
    # and the served result equals the single-system path
    p1, v1, _ = _single_run(g, target, nsteps, gamma=gamma, seed=target.n)
    assert np.array_equal(pos_mix, p1)
    srv.close()


def test_server_holds_each_member_at_its_own_step_count():
    """Requests of 7, 23 and 50 steps admitted together run as one chunk of 50
    steps: each member is held at its own count (forces cleared, state and
    step counter kept) while the others step on, so the chunk is not cut to
    the shortest segment, and each result is the same bit for bit as the
    request run alone (two chunks at most: the worker may start the first
    chunk before the later requests arrive; cut to the shortest remaining
    segment it would take three or more).
    """
    g = lib()
    systems = [synth.make_bulk(600 + 200 * k, seed_index=92 + k, charged_frac=0.2,
                               K=(10, 10, 10)) for k in range(3)]
    lengths = (7, 23, 50)

    def run(pairs):
        srv = g.Server(ctx(), 2 << 30, chunk_steps=50)
        ts = [srv.submit(_params(g, s, gamma=1.0, seed=s.n), s.pos, s.vel.astype(np.float32),
                         s.q, n, s.bonds) for s, n in pairs]
        srv.drain(120)
        out = []
        for t, (s, n) in zip(ts, pairs):
            r, p, v = srv.poll(t, want_state=True)
            assert r.status == 0 and r.steps_done == n
            out.append((p, v, np.array(r.energy)))
        st = srv.stats()
        srv.close()
        return out, st

    mix, st = run(list(zip(systems, lengths)))
    assert st["chunks"] <= 2
    for k, (s, n) in enumerate(zip(systems, lengths)):
        alone, _ = run([(s, n)])
        assert np.array_equal(mix[k][0], alone[0][0]), f"request {k} positions differ"
        assert np.array_equal(mix[k][1], alone[0][1]), f"request {k} velocities differ"
        assert np.allclose(mix[k][2], alone[0][2], rtol=1e-9, atol=1e-9)


def test_server_admission_and_rejection():
    """Host-side fault handling: malformed requests are rejected at submit,
    a request larger than the budget is refused, cancelled tickets never
    run, and the server keeps serving."""
    g = lib()
    s = synth.make_bulk(1200, seed_index=90)
    srv = g.Server(ctx(), 4 << 20, chunk_steps=5, max_active=2)
    bad_q = s.q.copy()
    bad_q[0] += 1.0
    with pytest.raises(g.GcmeError):
        srv.submit(g.params_from(s), s.pos, s.vel.astype(np.float32), bad_q, 10)
    big = synth.make_bulk(40000, seed_index=91, K=(48, 48, 48))
    with pytest.raises(g.GcmeError) as ei:
        srv.submit(g.params_from(big), big.pos, big.vel.astype(np.float32), big.q, 10)
    assert ei.value.code == -2
    t1 = srv.submit(g.params_from(s), s.pos, s.vel.astype(np.float32), s.q, 500)
    t2 = srv.submit(g.params_from(s), s.pos, s.vel.astype(np.float32), s.q, 500)
    t3 = srv.submit(g.params_from(s), s.pos, s.vel.astype(np.float32), s.q, 10)
    srv.cancel(t3)
    srv.drain(300)
    assert srv.poll(t1)[0].status == 0 and srv.poll(t2)[0].status == 0
    assert srv.poll(t3)[0].status < 0
    st = srv.stats()
    assert st["rejected"] == 2 and st["peak_active"] <= 2
    srv.close()
