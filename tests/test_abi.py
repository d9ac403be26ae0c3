"""The C ABI: library loads, exports every declared entry point, the
parameter struct layout matches, and host-side validation works (no device
calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08148_gb300 as pkg
    pkg.load()
    return pkg


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gcme_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(g):
    declared = _declared()
    assert len(declared) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", g.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gcme_[a-z0-9_]+)", out))
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    # and the binding resolves each of them
    lib = g.load()
    for name in declared:
        assert hasattr(lib, name)


def test_params_layout_matches_c(g):
    """gcme_params_default fills the C struct; reading it back through the
    ctypes mirror checks field order, offsets and size."""
    p = g.Params()
    g.load().gcme_params_default(ctypes.byref(p), 10.0, 32)
    assert list(p.box) == [10.0, 10.0, 10.0]
    assert (p.geometry, p.precision, p.order) == (0, 0, 5)
    assert (p.A, p.sigma, p.a, p.rc) == (25.0, 0.5, 0.5, 3.0)
    assert list(p.K) == [32, 32, 32]
    assert p.dt == 0.01 and p.bond_k == 100.0 and p.bond_r0 == 1.0
    assert p.H == 0.0 and p.wall_A == 0.0
    assert p.pair_path == 0 and p.gamma == 0.0 and p.kT == 1.0 and p.seed == 0


def _params(g, s):
    return g.params_from(s)


def test_validation_accepts_workloads(g):
    for s in (synth.config1(), synth.make_polyelectrolyte(10, 10, 500, K=(16, 16, 16)),
              synth.make_slab_fluid(synth.GEOM_SLAB_NM, 500),
              synth.make_slab_fluid(synth.GEOM_SLAB_PC, 500)):
        g.validate(_params(g, s), s.q, s.bonds)


@pytest.mark.parametrize("mutate,msg", [
    (lambda s, p, q: q.__setitem__(0, q[0] + 1.0), "neutral"),
    (lambda s, p, q: setattr(p, "order", 9), "order"),
    (lambda s, p, q: p.K.__setitem__(0, 7 * 11), "grid size"),
    (lambda s, p, q: p.box.__setitem__(1, 2.5), "shorter than the cutoff"),
    (lambda s, p, q: setattr(p, "A", 1.0), "non-collapse"),
    (lambda s, p, q: setattr(p, "geometry", 7), "geometry"),
    (lambda s, p, q: setattr(p, "pair_path", 3), "pair_path"),
    (lambda s, p, q: setattr(p, "gamma", -1.0), "gamma"),
])
def test_validation_rejects(g, mutate, msg):
    s = synth.make_bulk(400, seed_index=40)
    p = _params(g, s)
    q = s.q.copy()
    mutate(s, p, q)
    with pytest.raises(g.GcmeError) as ei:
        g.validate(p, q)
    assert ei.value.code == -1
    assert msg in str(ei.value)


def test_validation_rejects_bad_bonds_and_slab_box(g):
    s = synth.make_polyelectrolyte(4, 5, 100, K=(8, 8, 8))
    b = s.bonds.copy()
    b[0, 1] = s.n + 3
    with pytest.raises(g.GcmeError):
        g.validate(_params(g, s), s.q, b)
    t = synth.make_slab_fluid(synth.GEOM_SLAB_PC, 300)
    p = _params(g, t)
    p.box[2] = 2.5 * t.H
    with pytest.raises(g.GcmeError):
        g.validate(p, t.q)


def _mixture():
    A = np.array([[25.0, 27.0], [27.0, 25.0]])
    return synth.make_mixture(400, (0.8, 0.2), (0.0, 1.0), A, np.array([0.5, 0.6]),
                              np.array([0.5, 0.4]), seed_index=46)


def test_species_validation(g):
    t = _mixture()
    t.q = np.where(t.types == 1, 1.0, 0.0)
    t.q[np.nonzero(t.types == 0)[0][: int(t.q.sum())]] = -1.0  # neutral: species 0 takes -1
    g.validate(g.params_from(t), t.q, types=t.types)
    p = g.params_from(t)
    p.A_tab[1] = 26.0  # A_01 != A_10
    with pytest.raises(g.GcmeError, match="symmetric"):
        g.validate(p, t.q, types=t.types)
    bad = t.types.copy()
    bad[3] = 2
    with pytest.raises(g.GcmeError, match="out of range"):
        g.validate(g.params_from(t), t.q, types=bad)
    p = g.params_from(t)
    p.ntypes = 9
    with pytest.raises(g.GcmeError, match="ntypes"):
        g.validate(p, t.q, types=t.types)
    p = g.params_from(t)
    p.sigma_tab[1] = 0.0
    with pytest.raises(g.GcmeError, match="sigma"):
        g.validate(p, t.q, types=t.types)
    # the non-collapse condition is checked for the pair of charged species:
    # a tiny a_1 breaks it for (1, 1) even though (0, 0) is fine
    p = g.params_from(t)
    p.a_tab[1] = 0.02
    p.a_tab[0] = 0.02
    with pytest.raises(g.GcmeError, match="non-collapse"):
        g.validate(p, t.q, types=t.types)
    # species ids without tables
    with pytest.raises(g.GcmeError, match="out of range"):
        g.validate(g.params_from(synth.make_bulk(100, seed_index=47)),
                   synth.make_bulk(100, seed_index=47).q, types=np.ones(100, np.int32))


def test_no_device_reports_error_not_crash(g):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    with pytest.raises(g.GcmeError) as ei:
        g.Context(0)
    assert ei.value.code in (-1, -3)


def test_null_handles_are_rejected(g):
    """Entry points given a NULL system or batch return INVALID (-1) and set
    a message, with or without a device."""
    lib = g.load()
    assert lib.gcme_step_phase_timing(None, 1) == -1
    assert b"NULL" in lib.gcme_last_error()
    assert lib.gcme_batch_phase_timing(None, 0) == -1
    assert lib.gcme_step_phase_ms(None, None, 0, None) == -1
    assert lib.gcme_batch_phase_ms(None, None, 0, None) == -1
    assert lib.gcme_step_host(None, None, None, 1, None, 0, None) == -1
    assert b"gcme_step_host" in lib.gcme_last_error()


def test_noalloc_size_query_is_host_only(g):
    """gcme_cells_noalloc_size follows the cell rule of the header,
    ncell = prod_a max(1, floor(L_a / ((rc / f) (1 + 1e-4)))), for both cell
    factors, rejects what the allocation-free build rejects, and makes no
    CUDA call (it runs here without a device)."""
    import math
    for s in (synth.make_polyelectrolyte(20, 25, 4000, seed_index=60, K=(24, 24, 24)),
              synth.make_slab_fluid(synth.GEOM_SLAB_NM, 2500, charged_frac=0.2, seed_index=61)):
        for f in (0, 1, 2):
            p = g.params_from(s, cell_factor=f)
            want = 1
            for a in range(3):
                want *= max(1, math.floor(s.box[a] / ((s.rc / (f or 1)) * (1.0 + 1e-4))))
            assert g.cells_noalloc_size(p, s.n) == want
    s = synth.make_bulk(1000, seed_index=62)
    with pytest.raises(g.GcmeError, match="exceeds the maximum"):
        g.cells_noalloc_size(g.params_from(s), 70000)
    with pytest.raises(g.GcmeError, match="image-charge"):
        g.cells_noalloc_size(g.params_from(synth.make_slab_fluid(synth.GEOM_SLAB_PC, 900)), 900)
    p = g.params_from(s)
    p.cell_factor = 3
    with pytest.raises(g.GcmeError, match="cell_factor"):
        g.cells_noalloc_size(p, s.n)
    p = g.params_from(s)
    p.box[0] = 1e6
    with pytest.raises(g.GcmeError, match="cells"):
        g.cells_noalloc_size(p, s.n)
