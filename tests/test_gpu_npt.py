"""Pressure (Eq. pres_virial) and the Monte Carlo barostat through the C ABI
against the oracle: the virial pressure, forces after a box change (with and
without a change of the cell grid), and a sequence of volume moves whose
decisions, boxes and positions follow the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FORCE_RTOL_FP32, ctx, lib, rel_rms

pytestmark = pytest.mark.gpu


def _sys(s, precision):
    g = lib()
    return g.System(ctx(), g.params_from(s, precision), s.q, s.bonds)


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
def test_pressure_matches_oracle(precision, tol):
    import torch
    s = synth.make_polyelectrolyte(n_chains=6, chain_len=10, n_solvent=1200, seed_index=160,
                                   K=(16, 16, 16))
    sysg = _sys(s, precision)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    p = sysg.pressure(pos, kT=1.0)
    ref = oracle.pressure(s, kT=1.0)
    assert p == pytest.approx(ref, rel=tol, abs=tol)


@pytest.mark.parametrize("scale", [1.004, 0.93])  # same cell grid / another cell grid
def test_forces_after_box_change(scale):
    import torch
    g = lib()
    s = synth.make_bulk(700, seed_index=161, charged_frac=0.2, K=(10, 10, 10))
    sysg = _sys(s, 0)
    nc0 = list(sysg.info().nc)
    t = s.copy()
    t.box = s.box * scale
    t.pos = s.pos * scale
    sysg.set_box(t.box)
    info = sysg.info()
    assert np.allclose(list(info.box), t.box, rtol=0, atol=0)
    assert (list(info.nc) == nc0) == (scale > 1.0)
    pos = torch.tensor(t.pos, dtype=torch.float64, device="cuda:0")
    F = torch.zeros(3 * t.n, dtype=torch.int64, device="cuda:0")
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device="cuda:0")
    sysg.forces(pos, F, E)
    torch.cuda.synchronize()
    f = F.cpu().numpy().reshape(3, -1).T.astype(np.float64) / g.FORCE_SCALE
    ref = oracle.energy_forces(t)
    assert rel_rms(f, ref["forces"]) <= FORCE_RTOL_FP32
    assert abs(E[8].item() - ref["potential"]) <= 1e-6 * abs(ref["potential"])


def test_barostat_moves_follow_oracle():
    """FP64 path: the same uniforms, energies within 1e-10, so the same
    decisions; boxes and scaled positions agree to the last bits.  The box
    starts just below two cells per side and expands across the boundary,
    so the cell grid changes (an engine rebuild) within the sequence and
    rejected moves are restored across it."""
    import torch
    s = synth.make_bulk(700, seed_index=162, charged_frac=0.2, K=(10, 10, 10))
    f = 5.97 / s.box[0]  # just below two cells of side rc (1 + 1e-4) per axis
    s.box, s.pos = s.box * f, s.pos * f
    sysg = _sys(s, 1)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    p_ext, kT, dlnv, seed = 30.0, 1.0, 0.12, 77  # below the fluid's pressure: it expands
    opos, obox = s.pos.copy(), s.box.copy()
    decisions, grids = [], set()
    for m in range(16):
        acc = sysg.barostat_move(pos, p_ext, kT, dlnv, seed, m)
        opos, obox, oacc = oracle.barostat_move(s, opos, obox, p_ext, kT, dlnv, seed, m)
        decisions.append(acc)
        assert acc == oacc, m
        info = sysg.info()
        grids.add(tuple(info.nc))
        assert np.max(np.abs(np.array(info.box) - obox)) < 1e-12 * obox[0]
    torch.cuda.synchronize()
    assert np.max(np.abs(pos.cpu().numpy() - opos)) < 1e-12 * np.max(np.abs(opos))
    assert any(decisions) and not all(decisions)
    assert len(grids) >= 2


def test_barostat_rejects_slabs_and_bad_arguments():
    import torch
    g = lib()
    s = synth.make_slab_fluid(synth.GEOM_SLAB_NM, 500, seed_index=163)
    sysg = _sys(s, 0)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    with pytest.raises(g.GcmeError):
        sysg.barostat_move(pos, 1.0, 1.0, 0.1, 1, 0)
    b = _sys(synth.make_bulk(300, seed_index=164, K=(8, 8, 8)), 0)
    with pytest.raises(g.GcmeError):
        b.set_box([2.0, 9.0, 9.0])  # shorter than the cutoff
