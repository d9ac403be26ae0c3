"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Cell lists and neighbour sets must be bit-exact; forces and energies must
meet the FP32 bounds (relative RMS force <= 5e-4, relative potential energy
<= 1e-6) and the much tighter FP64-path bounds.  Inputs are the seeded
synthetic workloads of ``synth``.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (ENERGY_RTOL_FP32, ENERGY_RTOL_FP64, FORCE_RTOL_FP32, FORCE_RTOL_FP64,
                      PAIR_VARIANTS, ctx, gpu_forces, lib, record_error, rel_rms)

pytestmark = pytest.mark.gpu


def _small_cases():
    return {
        "bulk_n3000": synth.config1(),
        "poly_bonds": synth.make_polyelectrolyte(n_chains=8, chain_len=12, n_solvent=1200,
                                                 seed_index=50, K=(24, 24, 24)),
        "tiny_box_n120": synth.make_bulk(120, seed_index=51, charged_frac=0.3, K=(8, 8, 8)),
        "box_2cells_n700": synth.make_bulk(700, seed_index=52, charged_frac=0.2, K=(10, 10, 10)),
        "slab_nm": synth.make_slab_fluid(synth.GEOM_SLAB_NM, 900, charged_frac=0.2,
                                         seed_index=53),
        "slab_pc": synth.make_slab_fluid(synth.GEOM_SLAB_PC, 900, charged_frac=0.2,
                                         seed_index=54),
        "neutral_only": synth.make_bulk(500, seed_index=55, charged_frac=0.0, K=(8, 8, 8)),
        "ragged_odd_grid": synth.make_bulk(1000, seed_index=56, charged_frac=0.4,
                                           K=(15, 12, 10)),
        "odd_planes": synth.make_bulk(900, seed_index=57, charged_frac=0.4, K=(10, 9, 15)),
    }


CASES = _small_cases()


# --------------------------------------------------------------------------
# K1/K2: cell list, bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("factor", [1, 2])
@pytest.mark.parametrize("name", ["bulk_n3000", "tiny_box_n120", "slab_pc", "poly_bonds"])
def test_cell_list_bit_exact(name, factor):
    import torch
    g = lib()
    s = CASES[name]
    sysg = g.System(ctx(), g.params_from(s, cell_factor=factor), s.q, s.bonds)
    info = sysg.info()
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    cs = torch.zeros(info.ncell + 1, dtype=torch.int32, device=dev)
    si = torch.zeros(info.n_ext, dtype=torch.int32, device=dev)
    sysg.build_cells(pos, cs, si)
    torch.cuda.synchronize()
    epos, eq, etype, _ = oracle.electrostatic_beads(s)
    nc = oracle.cell_counts(s.box, s.rc, factor=info.cell_factor)
    assert list(nc) == list(info.nc)
    _, start, order = oracle.cell_list(epos, s.box, nc, oracle.bead_classes(s))
    assert np.array_equal(cs.cpu().numpy(), start)
    assert np.array_equal(si.cpu().numpy(), order)


def _edge_positions(s, rng):
    """Coordinates on and next to box and cell faces (one ulp, and the
    2^-40 L margin of the binning's shortcut), far images (|n| around 2^10)
    and ordinary ones."""
    pos = s.pos.copy()
    nc = oracle.cell_counts(s.box, s.rc)
    k = 0
    for a in range(3):
        L = s.box[a]
        faces = [m * L for m in range(-3, 4)] + [c * L / nc[a] for c in range(nc[a] + 1)]
        for f in faces:
            for v in (f, np.nextafter(f, np.inf), np.nextafter(f, -np.inf),
                      f + L * 2.0 ** -40, f - L * 2.0 ** -40,
                      np.nextafter(f + L * 2.0 ** -40, -np.inf), f + 3.7 * L * 2.0 ** -40):
                pos[k % s.n, a] = v
                k += 1
        for m in (1000, 1023, 1024, 1500, -1024, -1500):
            pos[k % s.n, a] = pos[k % s.n, a] % L + m * L
            k += 1
    return pos


def test_cell_list_bit_exact_at_faces_and_far_images():
    """The binning's exact shortcut (a coordinate's image index from the
    previous binning) against the rule, at the faces of the box and of the
    cells, with right and wrong previous indices."""
    import dataclasses
    import torch
    g = lib()
    s = synth.make_bulk(3000, seed_index=59, charged_frac=0.2, K=(12, 12, 12))  # 3^3 cells
    sysg = g.System(ctx(), g.params_from(s), s.q)
    info = sysg.info()
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(5)
    p0 = _edge_positions(s, rng)
    shifts = rng.integers(-2, 3, size=p0.shape) * s.box  # other images: the stored indices miss
    for pos in (p0, p0, p0 + shifts, p0):
        t = dataclasses.replace(s, pos=pos)
        cs = torch.zeros(info.ncell + 1, dtype=torch.int32, device=dev)
        si = torch.zeros(info.n_ext, dtype=torch.int32, device=dev)
        sysg.build_cells(torch.tensor(pos, dtype=torch.float64, device=dev), cs, si)
        torch.cuda.synchronize()
        epos, _, _, _ = oracle.electrostatic_beads(t)
        nc = oracle.cell_counts(s.box, s.rc)
        _, start, order = oracle.cell_list(epos, s.box, nc, oracle.bead_classes(t))
        assert np.array_equal(cs.cpu().numpy(), start)
        assert np.array_equal(si.cpu().numpy(), order)


# --------------------------------------------------------------------------
# K3 neighbour set, bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", list(PAIR_VARIANTS))
@pytest.mark.parametrize("name,prec", [("bulk_n3000", 0), ("tiny_box_n120", 0),
                                       ("box_2cells_n700", 0), ("slab_pc", 0),
                                       ("bulk_n3000", 1), ("slab_pc", 1)])
def test_pair_set_bit_exact(name, prec, variant):
    import torch
    g = lib()
    s = CASES[name]
    factor, path = PAIR_VARIANTS[variant]
    if prec == 1:
        path = 0  # the FP64 path scans cells
    sysg = g.System(ctx(), g.params_from(s, prec, factor, path), s.q, s.bonds)
    if prec == 0:
        assert sysg.info().pair_path == path
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    cap = 4_000_000
    trip = torch.zeros(3 * cap, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    sysg.debug_pairs(pos, trip, cap, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k <= cap
    got = trip[: 3 * k].cpu().numpy().reshape(-1, 3)
    epos, _, _, n = oracle.electrostatic_beads(s)
    ref = oracle.pair_set(epos, s.box, s.rc)
    ref = ref[ref[:, 0] < n]                    # the kernel's i runs over real beads
    a = np.unique(got, axis=0)
    assert a.shape[0] == got.shape[0], "duplicate triples"
    b = np.unique(ref, axis=0)
    assert a.shape == b.shape and np.array_equal(a, b)


# --------------------------------------------------------------------------
# Forces and energies
# --------------------------------------------------------------------------
def _check(s, out, ref, f_tol, e_tol, per_term_tol):
    ferr = rel_rms(out["forces"], ref["forces"])
    e = out["energy"]
    eerr = abs(e["potential"] - ref["potential"]) / abs(ref["potential"])
    scale = sum(abs(ref[t]) for t in oracle.TERMS)
    terms = {t: abs(e[t] - ref[t]) / scale for t in oracle.TERMS}
    assert ferr <= f_tol, f"force rel RMS {ferr:.3e}"
    assert eerr <= e_tol, f"energy rel {eerr:.3e} ({e['potential']} vs {ref['potential']})"
    for t, v in terms.items():
        assert v <= per_term_tol, f"term {t}: {e[t]} vs {ref[t]}"
    return ferr, eerr


@pytest.mark.parametrize("variant", list(PAIR_VARIANTS))
@pytest.mark.parametrize("name", list(CASES))
def test_forces_fp32(name, variant):
    s = CASES[name]
    factor, path = PAIR_VARIANTS[variant]
    out = gpu_forces(s, 0, cell_factor=factor, pair_path=path)
    ref = oracle.energy_forces(s)
    _check(s, out, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)


@pytest.mark.parametrize("name", ["bulk_n3000", "poly_bonds", "slab_nm", "slab_pc",
                                  "tiny_box_n120", "ragged_odd_grid"])
def test_forces_fp64(name):
    s = CASES[name]
    out = gpu_forces(s, 1)
    ref = oracle.energy_forces(s)
    _check(s, out, ref, FORCE_RTOL_FP64, ENERGY_RTOL_FP64, 1e-10)


def _shapes(plane, lpb):
    return {"pair_split": 3, "pair_threads": 160, "pair_ctas_per_sm": 0, "pair_nelec": 1,
            "fft_lpb": [lpb] * 3, "fft_plane": plane}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["odd_planes", "ragged_odd_grid", "slab_pc", "poly_bonds"])
def test_fft_paths(name, prec):
    """Both FFT schedules at parity with the oracle: x-y plane passes over
    pairs of real z-planes packed into one complex plane with the z pass on
    the Hermitian half spectrum (odd K0, K1 and K2 included: an unpaired
    last plane, no Nyquist column), and per-axis line passes on the full
    spectrum, at the smallest and largest tiles.  The reciprocal energies and
    virials of the schedules agree to the precision's rounding."""
    s = CASES[name]
    f_tol, e_tol, t_tol = ((FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6) if prec == 0 else
                           (FORCE_RTOL_FP64, ENERGY_RTOL_FP64, 1e-10))
    ref = oracle.energy_forces(s)
    w_tol = 1e-5 if prec == 0 else 1e-10
    outs = []
    for plane, lpb in ((True, 4), (True, 64), (False, 4), (False, 64)):
        out = gpu_forces(s, prec, virial=True, tuning=_shapes(plane, lpb))
        _check(s, out, ref, f_tol, e_tol, t_tol)
        # off-diagonal terms of the Nyquist planes (even K) cancel over the
        # full spectrum: the half spectrum must count each mirror as itself.
        # (The image-charge geometry's virial is not the oracle's sum of the
        # doubled system, see the header; its schedules are compared below.)
        if s.geometry != synth.GEOM_SLAB_PC:
            assert np.max(np.abs(out["virial"] - ref["virial"])) <= w_tol * np.max(
                np.abs(ref["virial"])), (plane, lpb)
        outs.append(out)
    # FP64: every mode's energy and virial term is rounded to 2^-32 before
    # the (exact) sums; the schedules round different but equal terms (the
    # half spectrum one term per mirror pair), about 1e-10 per mode
    rtol, atol = (1e-5, 0.0) if prec == 0 else (1e-12, 1e-6)
    for o in outs[1:]:
        assert o["energy"]["recip"] == pytest.approx(outs[0]["energy"]["recip"], rel=rtol,
                                                     abs=atol)
        wv = np.max(np.abs(outs[0]["virial"]))
        assert np.max(np.abs(o["virial"] - outs[0]["virial"])) <= rtol * wv + atol


@pytest.mark.parametrize("split,threads,nelec,ctas", [
    (9, 128, 1, 0), (9, 160, 1, 0), (9, 160, 2, 0), (9, 192, 2, 0), (9, 192, 3, 0),
    (3, 192, 3, 0), (9, 192, 3, 5), (3, 160, 2, 8),
    (9, 128, 0, 7), (3, 128, 0, 3), (9, 64, 0, 12), (9, 96, 0, 9),
    (9, 160, -2, 5), (9, 128, -1, 6), (9, 192, -3, 4), (3, 192, -2, 0)])
def test_pair_shapes_at_parity(split, threads, nelec, ctas):
    """Every launch shape of the 27-cell kernel (work items per cell, block
    size, electrostatics warps splitting each cell's charged candidates or
    every warp taking the item's tasks, static or dynamic CTAs, or one warp
    per work item) gives the oracle's forces and energies."""
    s = CASES["poly_bonds"]
    t = {"pair_split": split, "pair_threads": threads, "pair_ctas_per_sm": ctas,
         "pair_nelec": nelec, "fft_lpb": [8, 8, 8], "fft_plane": True}
    out = gpu_forces(s, 0, tuning=t)
    _check(s, out, oracle.energy_forces(s), FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)


@pytest.mark.parametrize("geom", [synth.GEOM_BULK, synth.GEOM_SLAB_PC])
@pytest.mark.parametrize("threads,nelec,ctas,group,snap", [
    (160, 2, 5, 2, False), (192, 3, 0, 3, False), (128, 1, 4, 3, True), (160, 1, 0, 2, True),
    (160, -2, 5, 2, True), (128, -1, 0, 3, False)])
def test_pair_group_items_at_parity(geom, threads, nelec, ctas, group, snap):
    """CTA work items of 2 or 3 consecutive home cells along x: 5 cells per
    axis (the last group of 3 is ragged: 3 + 2), the row's staged cells
    shared by the home cells, forces, energies and virial at parity with the
    oracle, and the neighbour set (debug triples, scalar path over the same
    items) bit-exact.  With a cell snapshot (snap) the items are ordered by
    cost and the cheapest end the list as single home cells (negative
    codes), two per resident CTA.  The conducting slab adds images to the
    charged candidates."""
    import torch
    g = lib()
    if geom not in _GROUP_CASES:
        if geom == synth.GEOM_BULK:
            s = synth.make_bulk(12000, seed_index=65, charged_frac=0.3, K=(20, 20, 20))
        else:
            s = synth.make_slab_fluid(synth.GEOM_SLAB_PC, 16000, charged_frac=0.2,
                                      seed_index=66, aspect=0.5)
        epos, _, _, n = oracle.electrostatic_beads(s)
        want = oracle.pair_set(epos, s.box, s.rc)
        _GROUP_CASES[geom] = (s, oracle.energy_forces(s), np.unique(want[want[:, 0] < n], axis=0))
    s, ref, want = _GROUP_CASES[geom]
    t = {"pair_split": 9, "pair_threads": threads, "pair_ctas_per_sm": ctas,
         "pair_nelec": nelec, "pair_group": group, "fft_lpb": [8, 8, 8], "fft_plane": True}
    out = gpu_forces(s, 0, virial=geom == synth.GEOM_BULK, tuning=t, snapshot=snap)
    _check(s, out, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)
    if geom == synth.GEOM_BULK:
        assert np.max(np.abs(out["virial"] - ref["virial"])) <= 1e-5 * np.max(
            np.abs(ref["virial"]))
    sysg = g.System(ctx(), g.params_from(s), s.q, s.bonds)
    assert sysg.info().pair_path == g.GCME_PAIR_CELLS
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    if snap:
        sysg.autotune(pos, flags=2)  # GCME_TUNE_NO_CACHE
    sysg.apply_tuning(t)
    cap = 12_000_000
    trip = torch.zeros(3 * cap, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    sysg.debug_pairs(pos, trip, cap, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    assert k <= cap
    got = np.unique(trip[: 3 * k].cpu().numpy().reshape(-1, 3), axis=0)
    assert got.shape[0] == k, "duplicate triples"
    assert np.array_equal(got, want)
    sysg.close()


_GROUP_CASES = {}  # geometry -> (system, oracle forces, oracle neighbour set)


@pytest.mark.parametrize("a", [0.12, 0.07])
def test_small_smearing_radius(a):
    """Small smearing radii: the real-space table grows with beta^2 rc^2
    (a = 0.12 d: about 9,000 intervals), and below a ~ 0.09 d the kernels
    evaluate g and h directly (Taylor series while beta r < 0.055)."""
    s = synth.make_bulk(1500, seed_index=60, charged_frac=0.3, K=(12, 12, 12))
    s.a = a
    for prec, f_tol, e_tol in ((0, FORCE_RTOL_FP32, ENERGY_RTOL_FP32),
                               (1, FORCE_RTOL_FP64, ENERGY_RTOL_FP64)):
        out = gpu_forces(s, prec)
        _check(s, out, oracle.energy_forces(s), f_tol, e_tol, 1e-6 if prec == 0 else 1e-10)


@pytest.mark.parametrize("sigma", [0.5, 0.8])
def test_gaussian_core_width(sigma):
    """The FP32 one-species kernel sums the core over every staged bead of the
    non-self cells only when the core term at rc is below 1e-10 of its
    contact value (sigma = 0.5 d: 1.9e-12); a wider core (sigma = 0.8 d:
    2.6e-5 at rc) keeps the per-candidate cutoff test.  Both match the
    oracle, whose sums stop at rc."""
    s = synth.make_bulk(1500, seed_index=61, charged_frac=0.3, K=(12, 12, 12))
    s.sigma = sigma
    for t in (None, WARP_ITEMS):
        out = gpu_forces(s, 0, tuning=t)
        _check(s, out, oracle.energy_forces(s), FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)


WARP_ITEMS = {"pair_split": 9, "pair_threads": 128, "pair_ctas_per_sm": 7, "pair_nelec": 0,
              "fft_lpb": [8, 8, 8], "fft_plane": True}


@pytest.mark.parametrize("geom", [synth.GEOM_BULK, synth.GEOM_SLAB_PC])
@pytest.mark.parametrize("sigma", [0.5, 0.8])
def test_warp_items_in_rounds(geom, sigma):
    """One warp per work item when an item's candidates exceed the warp's
    shared-memory capacity: a box of one cell per axis (every neighbour cell
    is the home cell or its periodic image), about 500 real and 150 charged
    beads per cell, so every item is staged and evaluated in rounds, the home
    cell itself split over rounds.  With sigma = 0.5 d the core runs without
    the cutoff test and takes off the home bead's own term; with 0.8 d it
    keeps the test and excludes the home bead by index.  The conducting slab
    adds image beads to the charged lists."""
    if geom == synth.GEOM_BULK:
        s = synth.make_bulk(520, seed_index=63, charged_frac=0.3, K=(10, 10, 10))
    else:
        s = synth.make_slab_fluid(synth.GEOM_SLAB_PC, 600, charged_frac=0.3, seed_index=64)
    s.sigma = sigma
    for t in (WARP_ITEMS, dict(WARP_ITEMS, pair_chunks=1), dict(WARP_ITEMS, pair_chunks=4),
              dict(WARP_ITEMS, pair_split=3, pair_ctas_per_sm=3)):
        out = gpu_forces(s, 0, virial=geom == synth.GEOM_BULK, tuning=t)
        ref = oracle.energy_forces(s)
        _check(s, out, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)
        if geom == synth.GEOM_BULK:
            assert np.max(np.abs(out["virial"] - ref["virial"])) <= 1e-5 * np.max(
                np.abs(ref["virial"]))


@pytest.mark.parametrize("name", ["poly_bonds", "slab_pc", "odd_planes", "tiny_box_n120",
                                  "neutral_only"])
def test_cell_spread_same_grid_as_direct_spread(name):
    """The charge spread cell by cell through shared memory rounds every
    contribution as the direct spread does and sums integers, so forces and
    energies are the same bit for bit; both match the oracle."""
    s = CASES[name]
    base = {"pair_split": 9, "pair_threads": 160, "pair_ctas_per_sm": 0, "pair_nelec": 2,
            "fft_lpb": [8, 8, 8], "fft_plane": True}
    a = gpu_forces(s, 0, virial=True, tuning=dict(base, spread_cells=False))
    b = gpu_forces(s, 0, virial=True, tuning=dict(base, spread_cells=True))
    assert np.array_equal(a["fixed"], b["fixed"])
    assert a["energy"] == b["energy"]
    assert np.array_equal(a["virial"], b["virial"])
    _check(s, b, oracle.energy_forces(s), FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)


@pytest.mark.parametrize("name", ["poly_bonds", "slab_nm", "slab_pc", "tiny_box_n120",
                                  "neutral_only", "dense_one_cell"])
def test_item_tasks_same_sums_as_role_warps(name):
    """Every warp taking the item's tasks (pair_nelec = -e: chunks of 32
    home beads for the core, chunks of 32 charged home beads in e parts)
    gives each thread the partial sums of the static role split with e
    electrostatics warps, so forces, energies and virial are the same bit for
    bit, whatever the CTA's warp count; both item splits, items of two home
    cells, and the dense one-cell box over the staged capacity (both take the
    scalar path there); at parity with the oracle."""
    if name == "dense_one_cell":
        s = synth.make_bulk(500, seed_index=69, charged_frac=0.6, K=(8, 8, 8))
    else:
        s = CASES[name]
    vir = s.geometry == synth.GEOM_BULK
    ref = oracle.energy_forces(s)
    base = {"fft_lpb": [8, 8, 8], "fft_plane": True}
    for split, group in ((9, 1), (3, 1), (9, 2)):
        for e, th_static, th_dyn, ctas in ((2, 160, 128, 5), (1, 128, 192, 0), (3, 192, 160, 4)):
            t = dict(base, pair_split=split, pair_group=group, pair_ctas_per_sm=ctas)
            a = gpu_forces(s, 0, virial=vir, tuning=dict(t, pair_threads=th_static, pair_nelec=e))
            b = gpu_forces(s, 0, virial=vir, tuning=dict(t, pair_threads=th_dyn, pair_nelec=-e))
            assert np.array_equal(a["fixed"], b["fixed"]), (split, group, e)
            assert a["energy"] == b["energy"]
            if vir:
                assert np.array_equal(a["virial"], b["virial"])
        _check(s, b, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)


def test_apply_tuning_rejects_bad_shapes():
    g = lib()
    s = synth.make_bulk(300, seed_index=58, charged_frac=0.2, K=(96, 96, 8))
    sysg = g.System(ctx(), g.params_from(s, 1), s.q)  # FP64 planes of 96 x 96 need 297 KB
    with pytest.raises(g.GcmeError):
        sysg.apply_tuning(_shapes(True, 8))
    for bad in (dict(fft_lpb=[3, 8, 8]), dict(fft_lpb=[8, 128, 8]), dict(pair_threads=96),
                dict(pair_split=4), dict(pair_ctas_per_sm=9), dict(pair_nelec=4),
                dict(pair_nelec=0, pair_ctas_per_sm=0), dict(pair_nelec=0, pair_threads=160,
                                                             pair_ctas_per_sm=4),
                dict(pair_nelec=0, pair_threads=128, pair_ctas_per_sm=8),
                dict(pair_nelec=0, pair_ctas_per_sm=4, pair_chunks=5),
                dict(pair_group=4), dict(pair_group=2, pair_split=3),
                dict(pair_group=2, pair_nelec=0, pair_threads=128, pair_ctas_per_sm=4),
                dict(pair_nelec=-4), dict(pair_nelec=-1, pair_threads=64),
                dict(pair_nelec=-2, pair_ctas_per_sm=9),
                dict(spread_cells=True)):  # FP64 system: no cell spread
        t = _shapes(False, 8)
        t.update(bad)
        with pytest.raises(g.GcmeError):
            sysg.apply_tuning(t)
    sysg.apply_tuning(_shapes(False, 8))
    sysg.close()


def test_virial_fp32_and_fp64():
    s = CASES["poly_bonds"]
    ref = oracle.energy_forces(s)["virial"]
    for prec, tol in ((0, 1e-5), (1, 1e-10)):
        W = gpu_forces(s, prec, virial=True)["virial"]
        assert np.max(np.abs(W - ref)) <= tol * np.max(np.abs(ref))


def test_forces_deterministic():
    s = CASES["poly_bonds"]
    a = gpu_forces(s, 0)
    b = gpu_forces(s, 0)
    assert np.array_equal(a["fixed"], b["fixed"])
    assert a["energy"] == b["energy"]


def test_pair_paths_agree_up_to_fp32_order():
    """The three pair-kernel decompositions compute the same pair set and the
    same FP32 pair terms; they sum them differently (the cell kernels in FP32
    per thread, where terms below half an ulp of the running sum are lost;
    the list kernel in integers of 2^-b), so forces agree to rounding and
    energies to the FP32 energy bound."""
    s = CASES["bulk_n3000"]
    outs = [gpu_forces(s, 0, cell_factor=f, pair_path=p) for f, p in PAIR_VARIANTS.values()]
    for b in outs[1:]:
        assert rel_rms(outs[0]["forces"], b["forces"]) < 1e-6
        for t in ("gc", "real"):
            assert abs(outs[0]["energy"][t] - b["energy"][t]) < ENERGY_RTOL_FP32 * abs(b["energy"][t])
    # the two cell decompositions share the FP32 summation: much closer
    assert abs(outs[1]["energy"]["gc"] - outs[2]["energy"]["gc"]) < 1e-7 * abs(outs[1]["energy"]["gc"])


def test_single_neutral_bead_and_kappa_beta_limit():
    """Degenerate cases: a single bead (no pairs, no charges), and the fully
    reciprocal choice kappa = beta (real term identically zero)."""
    s = synth.make_bulk(100, seed_index=57, charged_frac=0.0, K=(8, 8, 8))
    s.pos = s.pos[:1].copy()
    s.vel = s.vel[:1].copy()
    s.q = s.q[:1].copy()
    s.box = np.array([3.5, 3.5, 3.5])
    out = gpu_forces(s, 0)
    ref = oracle.energy_forces(s)
    assert abs(out["energy"]["potential"] - ref["potential"]) < 1e-9
    t = synth.make_bulk(800, seed_index=58, charged_frac=0.5, K=(24, 24, 24))
    t.kappa = float(np.sqrt(np.pi) / (2 * t.a))
    out = gpu_forces(t, 0)
    assert abs(out["energy"]["real"]) < 1e-6
    ref = oracle.energy_forces(t)
    assert rel_rms(out["forces"], ref["forces"]) < FORCE_RTOL_FP32


# --------------------------------------------------------------------------
# Full-size workloads: the bulk polyelectrolyte (N = 32,000, grid 64^3) and
# the slabs (N = 64,000, grid 64 x 64 x 192) against the full oracle.
# --------------------------------------------------------------------------
def test_config2_full_size():
    s = synth.config2()
    out = gpu_forces(s, 0)
    ref = oracle.energy_forces(s)
    ferr, eerr = _check(s, out, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)
    record_error("c2_bulk_polyelectrolyte_n32000", force_rel_rms=ferr, energy_rel=eerr)


@pytest.mark.parametrize("geom", [synth.GEOM_SLAB_NM, synth.GEOM_SLAB_PC])
def test_config3_full_size(geom):
    s = synth.config3(geom)
    out = gpu_forces(s, 0)
    ref = oracle.energy_forces(s)
    ferr, eerr = _check(s, out, ref, FORCE_RTOL_FP32, ENERGY_RTOL_FP32, 1e-6)
    record_error("c3_" + synth.GEOM_NAMES[geom] + "_n64000", force_rel_rms=ferr, energy_rel=eerr)


# --------------------------------------------------------------------------
# Velocity Verlet through gcme_step
# --------------------------------------------------------------------------
def test_step_fp64_config1_100_steps():
    """The plain FP64 workload: N = 3000, 100 steps of velocity Verlet."""
    import torch
    g = lib()
    s = synth.config1()
    sysg = g.System(ctx(), g.params_from(s, 1), s.q)
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    vel = torch.tensor(s.vel, dtype=torch.float64, device=dev)
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device=dev)
    sysg.step(pos, vel, 100, E)
    torch.cuda.synchronize()
    p1, v1, hist = oracle.velocity_verlet(s, 100)
    dx = np.max(np.abs(pos.cpu().numpy() - p1))
    dv = np.max(np.abs(vel.cpu().numpy() - v1))
    assert dx < 1e-7
    assert dv < 1e-6
    e = E.cpu().numpy()
    epot = abs(e[8] - hist[-1]["potential"]) / abs(hist[-1]["potential"])
    assert epot < ENERGY_RTOL_FP64 * 100
    assert abs(e[9] - hist[-1]["kinetic"]) / abs(hist[-1]["kinetic"]) < 1e-7
    record_error("c1_fp64_100_steps_n3000", max_position_dev=dx, max_velocity_dev=dv,
                 energy_rel=epot)


def test_step_fp32_polyelectrolyte():
    import torch
    g = lib()
    s = CASES["poly_bonds"]
    sysg = g.System(ctx(), g.params_from(s, 0), s.q, s.bonds)
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    vel = torch.tensor(s.vel, dtype=torch.float32, device=dev)
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device=dev)
    sysg.step(pos, vel, 20, E)
    torch.cuda.synchronize()
    p1, v1, hist = oracle.velocity_verlet(s, 20)
    assert np.max(np.abs(pos.cpu().numpy() - p1)) < 1e-4
    e = E.cpu().numpy()
    tot_g = e[8] + e[9]
    tot_o = hist[-1]["potential"] + hist[-1]["kinetic"]
    assert abs(tot_g - tot_o) / abs(tot_o) < 1e-5


def test_step_host_same_as_device_step():
    """The state held on the host (gcme_step_host: page-locked buffers
    copied in, stepped and copied back in one captured graph) follows the
    device-buffer path bit for bit: a first call with the force evaluation,
    then continued calls of one step and of several steps, against gcme_step
    and gcme_step_continue on device buffers; unpinned buffers and a
    continuation on other buffers are rejected."""
    import torch
    g = lib()
    s = CASES["poly_bonds"]
    dev = torch.device("cuda:0")
    a = g.System(ctx(), g.params_from(s), s.q, s.bonds)
    b = g.System(ctx(), g.params_from(s), s.q, s.bonds)
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    vel = torch.tensor(s.vel, dtype=torch.float32, device=dev)
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device=dev)
    hpos = torch.tensor(s.pos, dtype=torch.float64).pin_memory()
    hvel = torch.tensor(s.vel, dtype=torch.float32).pin_memory()
    hE = torch.zeros(g.NTERMS, dtype=torch.float64).pin_memory()
    a.step(pos, vel, 3, E)
    b.step_host(hpos, hvel, 3, hE)
    for k in range(4):
        a.step_continue(pos, vel, 1 if k % 2 == 0 else 2, E)
        b.step_host(hpos, hvel, 1 if k % 2 == 0 else 2, hE, cont=True)
    torch.cuda.synchronize()
    assert np.array_equal(hpos.numpy(), pos.cpu().numpy())
    assert np.array_equal(hvel.numpy(), vel.cpu().numpy())
    assert np.array_equal(hE.numpy(), E.cpu().numpy())
    with pytest.raises(g.GcmeError):
        b.step_host(np.zeros_like(s.pos), np.zeros(s.vel.shape, np.float32), 1)
    with pytest.raises(g.GcmeError):
        b.step_host(hpos.clone().pin_memory(), hvel, 1, cont=True)
    a.close()
    b.close()


def test_phase_timing_is_opt_in_and_changes_no_result():
    """Event nodes between the phases enter the step graph only with phase
    timing on; the trajectory is bit-identical with and without them."""
    import torch
    g = lib()
    s = CASES["poly_bonds"]
    dev = torch.device("cuda:0")
    res = []
    for on in (False, True):
        sysg = g.System(ctx(), g.params_from(s, 0), s.q, s.bonds)
        sysg.phase_timing(on)
        pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
        vel = torch.tensor(s.vel, dtype=torch.float32, device=dev)
        E = torch.zeros(g.NTERMS, dtype=torch.float64, device=dev)
        sysg.step(pos, vel, 5, E)
        torch.cuda.synchronize()
        nk = sysg.step_kernels()
        assert nk > 0
        if on:
            ms, nk2 = sysg.phase_ms()
            assert nk2 == nk and np.all(ms >= 0) and ms[2] > 0
            sysg.phase_timing(False)
            sysg.step_continue(pos, vel, 1, E)
            torch.cuda.synchronize()
            with pytest.raises(g.GcmeError):  # the last step ran without events
                sysg.phase_ms()
        else:
            with pytest.raises(g.GcmeError):
                sysg.phase_ms()
            sysg.step_continue(pos, vel, 1, E)
            torch.cuda.synchronize()
        res.append([t.cpu().numpy() for t in (pos, vel, E)])
        sysg.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_autotune_keeps_parity_and_caches(tmp_path, monkeypatch):
    """The autotuner times the candidate launch shapes, applies the fastest
    (results stay within tolerance of the oracle) and records it in the
    cache file, from which a second call applies it without timing."""
    import torch
    monkeypatch.setenv("GCME_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    g = lib()
    s = CASES["poly_bonds"]
    sysg = g.System(ctx(), g.params_from(s), s.q, s.bonds)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    t1 = sysg.autotune(pos)
    assert t1["pair_split"] in (3, 9) and t1["pair_threads"] in (64, 128, 160, 192)
    assert t1["pair_nelec"] in (-3, -2, -1, 0, 1, 2, 3)
    lst = g.System(ctx(), g.params_from(s, pair_path=g.GCME_PAIR_LIST), s.q, s.bonds)
    t3 = lst.autotune(pos)  # the list path has a cache entry of its own
    assert not t3["from_cache"]
    assert all(l in (4, 8, 16, 32, 64) for l in t1["fft_lpb"]) and not t1["from_cache"]
    F = torch.zeros(3 * s.n, dtype=torch.int64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.forces(pos, F, E)
    torch.cuda.synchronize()
    f = F.cpu().numpy().reshape(3, -1).T.astype(np.float64) / g.FORCE_SCALE
    ref = oracle.energy_forces(s)
    assert rel_rms(f, ref["forces"]) <= FORCE_RTOL_FP32
    assert abs(E[8].item() - ref["potential"]) <= ENERGY_RTOL_FP32 * abs(ref["potential"])
    sys2 = g.System(ctx(), g.params_from(s), s.q, s.bonds)
    t2 = sys2.autotune(pos)
    assert t2["from_cache"] and t2["pair_split"] == t1["pair_split"]
    assert t2["fft_lpb"] == t1["fft_lpb"]
    assert (tmp_path / "tune.jsonl").read_text().count("pair_split") == 2


# --------------------------------------------------------------------------
# The FFT passes alone, against cuFFT
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("plane", [True, False])
@pytest.mark.parametrize("name", ["poly_bonds", "odd_planes", "ragged_odd_grid", "slab_pc"])
def test_fft_passes_against_cufft(name, plane, prec):
    """The hand-written FFT passes checked on their own against cuFFT
    (torch.fft on the GPU): from the library's charge grid Q, the smooth-PME
    convolution theta * Q = F^-1[B C F(Q)] computed with torch.fft in FP64
    (B from the oracle's B-spline moduli, C(m) = lB exp(-pi^2 m^2 / kappa^2) /
    (pi V m^2), C(0) = 0; unnormalised transforms) equals the library's grid
    after its forward passes, influence function and backward passes, for the
    x-y plane schedule (half spectrum) and the per-axis line schedule, even
    and odd grid sizes."""
    import torch
    g = lib()
    s = CASES[name]
    sysg = g.System(ctx(), g.params_from(s, prec), s.q, s.bonds)
    sysg.apply_tuning({"pair_split": 9, "pair_threads": 128, "pair_ctas_per_sm": 0,
                       "pair_nelec": 1, "fft_lpb": [8, 8, 8], "fft_plane": plane})
    K0, K1, K2 = s.K
    G = K0 * K1 * K2
    dev = torch.device("cuda:0")
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    dq = torch.zeros(G, dtype=torch.float64, device=dev)
    dphi = torch.zeros(G, dtype=torch.float64, device=dev)
    sysg.debug_pme_grids(pos, dq, dphi)
    torch.cuda.synchronize()
    sysg.close()
    Q = dq.view(K2, K1, K0)
    assert abs(float(Q.sum())) < 1e-6 * float(Q.abs().sum())  # neutral: no m = 0 term
    F = torch.fft.fftn(Q)

    def mvec(K, L):
        i = np.arange(K)
        return np.where(i < (K + 1) // 2, i, i - K) / L

    mz, my, mx = np.meshgrid(mvec(K2, s.box[2]), mvec(K1, s.box[1]), mvec(K0, s.box[0]),
                             indexing="ij")
    m2 = mx * mx + my * my + mz * mz
    V = float(np.prod(s.box))
    with np.errstate(divide="ignore", invalid="ignore"):
        C = s.lB / (np.pi * V) * np.exp(-np.pi ** 2 * m2 / s.kappa ** 2) / m2
    C[0, 0, 0] = 0.0
    B = (oracle.bspline_moduli(s.order, K2)[:, None, None] *
         oracle.bspline_moduli(s.order, K1)[None, :, None] *
         oracle.bspline_moduli(s.order, K0)[None, None, :])
    BC = torch.tensor(B * C, dtype=torch.float64, device=dev)
    phi_ref = (torch.fft.ifftn(F * BC).real * G).view(-1)
    err = float((dphi - phi_ref).abs().max() / phi_ref.abs().max())
    assert err <= (2e-5 if prec == 0 else 1e-10), err
