"""Helpers for the GPU parity tests: run the CUDA path through the C ABI."""
import json
import os

import numpy as np

import synth

TERMS = ("gc", "real", "recip", "corr", "self", "slab", "wall", "bond", "potential", "kinetic")

# Tolerances of the FP32 path against the FP64 oracle: relative RMS force
# error and relative error of the total potential energy.
FORCE_RTOL_FP32 = 5e-4
ENERGY_RTOL_FP32 = 1e-6
# FP64 path: limited by the 2^-32 fixed-point force quantum and the 2^-40
# charge-grid quantum, far below these bounds.
FORCE_RTOL_FP64 = 1e-8
ENERGY_RTOL_FP64 = 1e-10


def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_08148_gb300 as g
    g.load()
    return g


_CTX = None


def ctx():
    global _CTX
    g = lib()
    if _CTX is None:
        _CTX = g.Context(0)
    return _CTX


# FP32 pair-kernel variants: (cell_factor, pair_path) -- Verlet lists,
# 27-cell stencil, fine cells
PAIR_VARIANTS = {"list": (1, 1), "cells": (1, 2), "fine": (2, 2)}


def gpu_forces(s: synth.System, precision=0, virial=False, pos=None, cell_factor=0,
               pair_path=0, tuning=None, snapshot=False):
    """Forces, energies (and virial) of s through one System; snapshot: run
    the autotuner first (uncached), whose cell snapshot orders the work
    items by cost, before the given tuning is applied."""
    import torch
    g = lib()
    sysg = g.System(ctx(), g.params_from(s, precision, cell_factor, pair_path), s.q, s.bonds)
    dev = torch.device("cuda:0")
    p = torch.tensor(s.pos if pos is None else pos, dtype=torch.float64, device=dev)
    if snapshot:
        sysg.autotune(p, flags=2)  # GCME_TUNE_NO_CACHE
    if tuning is not None:
        sysg.apply_tuning(tuning)
    F = torch.zeros(3 * s.n, dtype=torch.int64, device=dev)
    E = torch.zeros(g.NTERMS, dtype=torch.float64, device=dev)
    W = torch.zeros(9, dtype=torch.float64, device=dev) if virial else None
    sysg.forces(p, F, E, W)
    torch.cuda.synchronize()
    f = F.cpu().numpy().reshape(3, -1).T.astype(np.float64) / g.FORCE_SCALE
    e = dict(zip(TERMS, E.cpu().numpy().tolist()))
    out = dict(forces=f, energy=e, fixed=F.cpu().numpy())
    if virial:
        out["virial"] = W.cpu().numpy().reshape(3, 3)
    sysg.close()
    return out


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


def record_error(name, **errors):
    """Append the measured errors of a parity case to the JSON-lines file
    named by GCME_PARITY_LOG (nothing when unset), tagged with the hash of the
    pair-kernel sources, so that a measurement summary can quote them."""
    path = os.environ.get("GCME_PARITY_LOG")
    if not path:
        return
    import bench
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "a") as f:
        f.write(json.dumps({"case": name, "kernel_sha": bench.kernel_sha(),
                            **{k: float(v) for k, v in errors.items()}}) + "\n")
