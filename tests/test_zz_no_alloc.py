"""gcme_build_cells_noalloc: the cell-list build for callers that cannot
allocate device memory (their device memory belongs to another runtime's
pool, or cudaMalloc's implicit synchronisation is not acceptable on their
path).  Its output must equal gcme_build_cells' bit for bit, on calls in a
row that share the library's fixed scratch array, with the cell-start
buffer sized by the host-only query gcme_cells_noalloc_size (such a caller
cannot create a system to ask).  Collected last (file name) so that a run
stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _reference(g, ctx, s, pos, factor):
    import torch
    sysg = g.System(ctx, g.params_from(s, cell_factor=factor), s.q, s.bonds)
    info = sysg.info()
    cs = torch.zeros(info.ncell + 1, dtype=torch.int32, device="cuda:0")
    si = torch.zeros(info.n_ext, dtype=torch.int32, device="cuda:0")
    sysg.build_cells(pos, cs, si)
    torch.cuda.synchronize()
    out = cs.cpu().numpy(), si.cpu().numpy()
    sysg.close()
    return out


def test_noalloc_cells_match_existing_entry_point_twice():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08148_gb300 as g
    ctx = g.Context(0)
    cases = [synth.make_polyelectrolyte(n_chains=20, chain_len=25, n_solvent=4000,
                                        seed_index=60, K=(24, 24, 24)),
             synth.make_slab_fluid(synth.GEOM_SLAB_NM, 2500, charged_frac=0.2, seed_index=61)]
    # consecutive calls on the shared scratch: different sizes, both cell
    # factors (1: cells of side >= rc; 2: side >= rc / 2), the default (0)
    for s in cases:
        pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
        q = torch.tensor(s.q, dtype=torch.float64, device="cuda:0")
        for factor in (0, 1, 2):
            ref_start, ref_order = _reference(g, ctx, s, pos, factor)
            p = g.params_from(s, cell_factor=factor)
            ncell = g.cells_noalloc_size(p, s.n)
            assert ncell + 1 == ref_start.shape[0]
            cs = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda:0")
            si = torch.full((s.n,), -7, dtype=torch.int32, device="cuda:0")
            for _ in range(2):
                g.build_cells_noalloc(p, s.n, pos, q, cs, si)
                torch.cuda.synchronize()
                assert np.array_equal(cs.cpu().numpy(), ref_start)
                assert np.array_equal(si.cpu().numpy(), ref_order)


def test_noalloc_rejects_oversized_and_image_geometry():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08148_gb300 as g
    s = synth.make_bulk(1000, seed_index=62)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:0")
    q = torch.tensor(s.q, dtype=torch.float64, device="cuda:0")
    cs = torch.zeros(64, dtype=torch.int32, device="cuda:0")
    si = torch.zeros(s.n, dtype=torch.int32, device="cuda:0")
    with pytest.raises(g.GcmeError, match="exceeds the maximum"):
        g.build_cells_noalloc(g.params_from(s), 70000, pos, q, cs, si)
    p = g.params_from(synth.make_slab_fluid(synth.GEOM_SLAB_PC, 900))
    with pytest.raises(g.GcmeError, match="image-charge"):
        g.build_cells_noalloc(p, s.n, pos, q, cs, si)
