"""ctypes binding of libgcme (include/gcme.h).

Argument marshalling only: every step of the force/energy path runs in the
library's CUDA kernels.  Device buffers are torch tensors (their data
pointers are passed through), streams are torch.cuda streams.  If the
library is missing this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import builder as _build

GCME_BULK, GCME_SLAB_NONMETAL, GCME_SLAB_IMAGE = 0, 1, 2
GCME_FP32, GCME_FP64 = 0, 1
GCME_PAIR_AUTO, GCME_PAIR_LIST, GCME_PAIR_CELLS = 0, 1, 2
GCME_STEP_CONTINUE = 1
MAX_TYPES = 8
NTERMS = 10
TERM_NAMES = ("gc", "real", "recip", "corr", "self", "slab", "wall", "bond",
              "potential", "kinetic")
FORCE_SCALE = 2.0 ** 32

ERRORS = {-1: "INVALID", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "NONFINITE",
          -6: "FULL", -7: "NOTFOUND"}


class GcmeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gcme error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("geometry", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("A", ctypes.c_double),
                ("sigma", ctypes.c_double), ("a", ctypes.c_double), ("lB", ctypes.c_double),
                ("rc", ctypes.c_double), ("kappa", ctypes.c_double),
                ("K", ctypes.c_int32 * 3), ("order", ctypes.c_int32), ("dt", ctypes.c_double),
                ("H", ctypes.c_double), ("wall_A", ctypes.c_double),
                ("wall_sigma2", ctypes.c_double), ("bond_k", ctypes.c_double),
                ("bond_r0", ctypes.c_double), ("cell_factor", ctypes.c_int32),
                ("pair_path", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("kT", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("ntypes", ctypes.c_int32), ("frozen_mask", ctypes.c_int32),
                ("A_tab", ctypes.c_double * (MAX_TYPES * MAX_TYPES)),
                ("sigma_tab", ctypes.c_double * MAX_TYPES),
                ("a_tab", ctypes.c_double * MAX_TYPES)]


class SysInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_ext", ctypes.c_int64),
                ("n_charged_ext", ctypes.c_int64), ("ncell", ctypes.c_int64),
                ("nbonds", ctypes.c_int64), ("nc", ctypes.c_int32 * 3),
                ("cell_factor", ctypes.c_int32), ("scratch_bytes", ctypes.c_int64),
                ("pair_path", ctypes.c_int32), ("list_stride", ctypes.c_int32),
                ("list_builds", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("box", ctypes.c_double * 3)]


class Tuning(ctypes.Structure):
    _fields_ = [("pair_split", ctypes.c_int32), ("pair_threads", ctypes.c_int32),
                ("pair_ctas_per_sm", ctypes.c_int32), ("fft_lpb", ctypes.c_int32 * 3),
                ("fft_plane", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("cell_factor", ctypes.c_int32), ("pair_nelec", ctypes.c_int32),
                ("pair_chunks", ctypes.c_int32), ("spread_cells", ctypes.c_int32),
                ("pair_group", ctypes.c_int32),
                ("forces_ms", ctypes.c_double), ("pme_ms", ctypes.c_double)]

    @classmethod
    def from_dict(cls, d: dict) -> "Tuning":
        t = cls()
        for k in ("pair_split", "pair_threads", "pair_ctas_per_sm", "pair_nelec"):
            setattr(t, k, int(d[k]))
        t.pair_chunks = int(d.get("pair_chunks", 0))
        t.pair_group = int(d.get("pair_group", 1))
        t.spread_cells = int(bool(d.get("spread_cells", False)))
        for a in range(3):
            t.fft_lpb[a] = int(d["fft_lpb"][a])
        t.fft_plane = int(bool(d["fft_plane"]))
        return t

    def as_dict(self):
        return {"pair_split": self.pair_split, "pair_threads": self.pair_threads,
                "pair_ctas_per_sm": self.pair_ctas_per_sm, "fft_lpb": list(self.fft_lpb),
                "fft_plane": bool(self.fft_plane),
                "from_cache": bool(self.from_cache), "cell_factor": self.cell_factor,
                "pair_nelec": self.pair_nelec, "pair_chunks": self.pair_chunks,
                "pair_group": self.pair_group,
                "spread_cells": bool(self.spread_cells),
                "forces_ms": self.forces_ms,
                "pme_ms": self.pme_ms}


class Request(ctypes.Structure):
    _fields_ = [("params", Params), ("n", ctypes.c_int64),
                ("h_pos", ctypes.POINTER(ctypes.c_double)),
                ("h_vel", ctypes.POINTER(ctypes.c_float)),
                ("h_q", ctypes.POINTER(ctypes.c_double)),
                ("h_bonds", ctypes.POINTER(ctypes.c_int32)), ("nbonds", ctypes.c_int64),
                ("nsteps", ctypes.c_int64), ("h_types", ctypes.POINTER(ctypes.c_int32))]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps_done", ctypes.c_int64),
                ("energy", ctypes.c_double * NTERMS), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_SIGS = {
    "gcme_last_error": ([], ctypes.c_char_p),
    "gcme_version": ([], ctypes.c_char_p),
    "gcme_params_default": ([ctypes.POINTER(Params), ctypes.c_double, _i32], None),
    "gcme_validate": ([ctypes.POINTER(Params), _i64, _vp, _vp, _vp, _i64], ctypes.c_int),
    "gcme_ctx_create": ([ctypes.POINTER(_vp), ctypes.c_int], ctypes.c_int),
    "gcme_ctx_destroy": ([_vp], None),
    "gcme_system_create": ([_vp, ctypes.POINTER(Params), _i64, _vp, _vp, _vp, _i64,
                            ctypes.POINTER(_vp)], ctypes.c_int),
    "gcme_system_destroy": ([_vp], None),
    "gcme_system_info": ([_vp, ctypes.POINTER(SysInfo)], ctypes.c_int),
    "gcme_system_set_step_count": ([_vp, ctypes.c_int64, _vp], ctypes.c_int),
    "gcme_pressure": ([_vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp],
                      ctypes.c_int),
    "gcme_system_set_box": ([_vp, ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
    "gcme_barostat_move": ([_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                            _vp], ctypes.c_int),
    "gcme_build_cells": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_debug_pme_grids": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_forces": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_build_cells_noalloc": ([ctypes.POINTER(Params), _i64, _vp, _vp, _vp, _vp, _vp],
                                 ctypes.c_int),
    "gcme_cells_noalloc_size": ([ctypes.POINTER(Params), _i64, ctypes.POINTER(ctypes.c_int64)],
                                ctypes.c_int),
    "gcme_forces_to_f64": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_step": ([_vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "gcme_step_f64": ([_vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "gcme_step_continue": ([_vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "gcme_step_host": ([_vp, _vp, _vp, _i64, _vp, ctypes.c_int32, _vp], ctypes.c_int),
    "gcme_step_phase_ms": ([_vp, _vp, _i32, _vp], ctypes.c_int),
    "gcme_batch_phase_ms": ([_vp, _vp, _i32, _vp], ctypes.c_int),
    "gcme_step_phase_timing": ([_vp, _i32], ctypes.c_int),
    "gcme_batch_phase_timing": ([_vp, _i32], ctypes.c_int),
    "gcme_autotune": ([_vp, _vp, _i32, ctypes.POINTER(Tuning), _vp], ctypes.c_int),
    "gcme_batch_autotune": ([_vp, _i32, ctypes.POINTER(Tuning), _vp], ctypes.c_int),
    "gcme_apply_tuning": ([_vp, ctypes.POINTER(Tuning)], ctypes.c_int),
    "gcme_batch_apply_tuning": ([_vp, ctypes.POINTER(Tuning)], ctypes.c_int),
    "gcme_debug_barrier_timeout": ([_vp, ctypes.c_double, _vp], ctypes.c_int),
    "gcme_debug_pairs": ([_vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "gcme_batch_create": ([_vp, _i32, ctypes.POINTER(Params), _vp, _vp, _vp, _vp, _vp,
                           ctypes.POINTER(_vp)], ctypes.c_int),
    "gcme_batch_destroy": ([_vp], None),
    "gcme_batch_set_state": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_batch_get_state": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "gcme_batch_step": ([_vp, _i64, _i32, _vp], ctypes.c_int),
    "gcme_batch_pointers": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                             ctypes.POINTER(_vp), ctypes.POINTER(_vp)], ctypes.c_int),
    "gcme_server_create": ([_vp, ctypes.c_size_t, _i32, _i32, ctypes.POINTER(_vp)],
                           ctypes.c_int),
    "gcme_server_destroy": ([_vp], None),
    "gcme_submit": ([_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
                    ctypes.c_int),
    "gcme_poll": ([_vp, ctypes.c_uint64, ctypes.POINTER(Result), _vp, _vp], ctypes.c_int),
    "gcme_cancel": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "gcme_server_drain": ([_vp, ctypes.c_double], ctypes.c_int),
    "gcme_server_stats": ([_vp, _vp], ctypes.c_int),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libgcme.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libgcme.so not built ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise GcmeError(rc, load().gcme_last_error().decode())


def _ptr(t) -> Optional[int]:
    """Device/host pointer of a torch tensor or numpy array (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def params_from(s, precision: int = GCME_FP32, cell_factor: int = 0,
                pair_path: int = GCME_PAIR_AUTO, gamma: float = 0.0, kT: float = 1.0,
                seed: int = 0) -> Params:
    """gcme_params from a system description with the fields of synth.System;
    gamma > 0 selects Langevin dynamics at temperature kT with noise key seed."""
    p = Params()
    p.cell_factor = int(cell_factor)
    p.pair_path = int(pair_path)
    p.gamma, p.kT, p.seed = float(gamma), float(kT), int(seed)
    for a in range(3):
        p.box[a] = float(s.box[a])
        p.K[a] = int(s.K[a])
    p.geometry = int(s.geometry)
    p.precision = int(precision)
    p.A, p.sigma, p.a, p.lB = float(s.A), float(s.sigma), float(s.a), float(s.lB)
    p.rc, p.kappa, p.order, p.dt = float(s.rc), float(s.kappa), int(s.order), float(s.dt)
    p.H, p.wall_A, p.wall_sigma2 = float(s.H), float(s.wall_A), float(s.wall_sigma2)
    p.bond_k, p.bond_r0 = float(s.bond_k), float(s.bond_r0)
    if getattr(s, "types", None) is not None:  # several species
        nt = int(s.A_tab.shape[0])
        if nt > MAX_TYPES:
            raise ValueError(f"at most {MAX_TYPES} species")
        p.ntypes = nt
        p.frozen_mask = int(getattr(s, "frozen_mask", 0))
        for t in range(nt):
            p.sigma_tab[t] = float(s.sig_tab[t])
            p.a_tab[t] = float(s.a_tab[t])
            for u in range(nt):
                p.A_tab[t * MAX_TYPES + u] = float(s.A_tab[t, u])
    return p


def _types(types, n):
    if types is None:
        return None
    t = np.ascontiguousarray(types, np.int32)
    if t.shape != (n,):
        raise ValueError("one species per bead")
    return t


def validate(params: Params, q, bonds=None, types=None):
    """Host-only validation of a system description (no device needed)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    b = None if bonds is None or len(bonds) == 0 else np.ascontiguousarray(bonds, np.int32)
    t = _types(types, q.shape[0])
    _check(load().gcme_validate(ctypes.byref(params), int(q.shape[0]), q.ctypes.data,
                                None if t is None else t.ctypes.data,
                                None if b is None else b.ctypes.data,
                                0 if b is None else int(b.shape[0])))


def build_cells_noalloc(params: Params, n: int, d_pos, d_q, d_cell_start, d_sorted_idx,
                        stream=None):
    """Cell list without any device allocation (gcme_build_cells_noalloc)."""
    _check(load().gcme_build_cells_noalloc(ctypes.byref(params), int(n), _ptr(d_pos), _ptr(d_q),
                                           _ptr(d_cell_start), _ptr(d_sorted_idx),
                                           _stream(stream)))


def cells_noalloc_size(params: Params, n: int) -> int:
    """Cells gcme_build_cells_noalloc would use (host only, no GPU call):
    the cell-start buffer it writes holds this many + 1 entries."""
    out = ctypes.c_int64(0)
    _check(load().gcme_cells_noalloc_size(ctypes.byref(params), int(n), ctypes.byref(out)))
    return int(out.value)


class Context:
    def __init__(self, device: int = 0):
        L = load()
        h = _vp()
        _check(L.gcme_ctx_create(ctypes.byref(h), int(device)))
        self.h = h
        self.device = device

    def barrier_timeout_probe(self, timeout_s: float = 0.2, stream=None) -> int:
        """Run the bounded-wait barrier probe; returns the status code."""
        return int(load().gcme_debug_barrier_timeout(self.h, float(timeout_s), _stream(stream)))

    def close(self):
        if self.h:
            load().gcme_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """One GCMe system (gcme_system_create)."""

    def __init__(self, ctx: Context, params: Params, q: np.ndarray,
                 bonds: Optional[np.ndarray] = None, types: Optional[np.ndarray] = None):
        L = load()
        self.ctx = ctx
        self.params = params
        q = np.ascontiguousarray(q, dtype=np.float64)
        self.n = int(q.shape[0])
        b = None if bonds is None or len(bonds) == 0 else np.ascontiguousarray(bonds, np.int32)
        t = _types(types, self.n)
        h = _vp()
        _check(L.gcme_system_create(ctx.h, ctypes.byref(params), self.n, q.ctypes.data,
                                    None if t is None else t.ctypes.data,
                                    None if b is None else b.ctypes.data,
                                    0 if b is None else int(b.shape[0]), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().gcme_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> SysInfo:
        out = SysInfo()
        _check(load().gcme_system_info(self.h, ctypes.byref(out)))
        return out

    def pressure(self, d_pos, kT: float = 1.0, stream=None) -> float:
        p = ctypes.c_double(0.0)
        _check(load().gcme_pressure(self.h, _ptr(d_pos), float(kT), ctypes.byref(p),
                                    _stream(stream)))
        return p.value

    def set_box(self, box, stream=None):
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        _check(load().gcme_system_set_box(self.h, b, _stream(stream)))

    def barostat_move(self, d_pos, pressure: float, kT: float, dlnv: float, seed: int,
                      move: int, stream=None) -> bool:
        acc = ctypes.c_int32(0)
        _check(load().gcme_barostat_move(self.h, _ptr(d_pos), float(pressure), float(kT),
                                         float(dlnv), int(seed), int(move), ctypes.byref(acc),
                                         _stream(stream)))
        return bool(acc.value)

    def set_step_count(self, steps: int, stream=None):
        _check(load().gcme_system_set_step_count(self.h, int(steps), _stream(stream)))

    def build_cells(self, d_pos, d_cell_start=None, d_sorted_idx=None, stream=None):
        _check(load().gcme_build_cells(self.h, _ptr(d_pos), _ptr(d_cell_start),
                                       _ptr(d_sorted_idx), _stream(stream)))

    def forces(self, d_pos, d_force=None, d_energy=None, d_virial=None, stream=None):
        _check(load().gcme_forces(self.h, _ptr(d_pos), _ptr(d_force), _ptr(d_energy),
                                  _ptr(d_virial), _stream(stream)))

    def forces_to_f64(self, d_force, d_out, stream=None):
        _check(load().gcme_forces_to_f64(self.h, _ptr(d_force), _ptr(d_out), _stream(stream)))

    def step(self, d_pos, d_vel, nsteps: int, d_energy=None, stream=None):
        fn = load().gcme_step_f64 if self.params.precision == GCME_FP64 else load().gcme_step
        _check(fn(self.h, _ptr(d_pos), _ptr(d_vel), int(nsteps), _ptr(d_energy),
                  _stream(stream)))

    def autotune(self, d_pos, flags: int = 0, stream=None) -> dict:
        t = Tuning()
        _check(load().gcme_autotune(self.h, _ptr(d_pos), int(flags), ctypes.byref(t),
                                    _stream(stream)))
        return t.as_dict()

    def apply_tuning(self, tuning: dict):
        """Apply launch shapes (the keys of autotune()'s result) without timing."""
        _check(load().gcme_apply_tuning(self.h, ctypes.byref(Tuning.from_dict(tuning))))

    def step_host(self, h_pos, h_vel, nsteps: int, h_energy=None, cont: bool = False,
                  stream=None):
        """gcme_step_host: the state in page-locked host memory (pinned CPU
        tensors), copied in, stepped and copied back on `stream`; synchronise
        before reading it.  cont: reuse the previous call's forces."""
        _check(load().gcme_step_host(self.h, _ptr(h_pos), _ptr(h_vel), int(nsteps),
                                     _ptr(h_energy), GCME_STEP_CONTINUE if cont else 0,
                                     _stream(stream)))

    def step_continue(self, d_pos, d_vel, nsteps: int, d_energy=None, stream=None):
        _check(load().gcme_step_continue(self.h, _ptr(d_pos), _ptr(d_vel), int(nsteps),
                                         _ptr(d_energy), _stream(stream)))

    def phase_timing(self, on: bool):
        """Capture later step graphs with (or without) phase event nodes."""
        _check(load().gcme_step_phase_timing(self.h, int(bool(on))))

    def phase_ms(self):
        """Device ms of the phases of the last step (phase timing on), and
        kernels per step."""
        ms = np.zeros(8, np.float32)
        k = np.zeros(1, np.int32)
        _check(load().gcme_step_phase_ms(self.h, ms.ctypes.data, 8, k.ctypes.data))
        return ms, int(k[0])

    def step_kernels(self):
        """Kernel launches in one step graph."""
        k = np.zeros(1, np.int32)
        _check(load().gcme_step_phase_ms(self.h, None, 0, k.ctypes.data))
        return int(k[0])

    def debug_pme_grids(self, d_pos, d_q=None, d_phi=None, stream=None):
        """Charge grid Q and theta * Q (gcme_debug_pme_grids), FP64 device arrays."""
        _check(load().gcme_debug_pme_grids(self.h, _ptr(d_pos), _ptr(d_q), _ptr(d_phi),
                                           _stream(stream)))

    def debug_pairs(self, d_pos, d_triples, cap: int, d_count, stream=None):
        _check(load().gcme_debug_pairs(self.h, _ptr(d_pos), _ptr(d_triples), int(cap),
                                       _ptr(d_count), _stream(stream)))


class Batch:
    """Independent systems stepped together (gcme_batch_create)."""

    def __init__(self, ctx: Context, params: Sequence[Params], charges: Sequence[np.ndarray],
                 bonds: Optional[Sequence[np.ndarray]] = None,
                 types: Optional[Sequence[Optional[np.ndarray]]] = None):
        L = load()
        ns = len(params)
        parr = (Params * ns)(*params)
        n = np.array([len(q) for q in charges], dtype=np.int64)
        q = np.ascontiguousarray(np.concatenate(charges), dtype=np.float64)
        if bonds is None:
            bonds = [np.zeros((0, 2), np.int32)] * ns
        bc = np.array([len(b) for b in bonds], dtype=np.int64)
        ball = np.ascontiguousarray(np.concatenate([np.asarray(b, np.int32).reshape(-1, 2)
                                                    for b in bonds]), dtype=np.int32)
        tall = None
        if types is not None and any(t is not None for t in types):
            tall = np.ascontiguousarray(np.concatenate(
                [np.zeros(len(q_), np.int32) if t is None else np.asarray(t, np.int32)
                 for t, q_ in zip(types, charges)]), dtype=np.int32)
        h = _vp()
        _check(L.gcme_batch_create(ctx.h, ns, parr, n.ctypes.data, q.ctypes.data,
                                   None if tall is None else tall.ctypes.data,
                                   ball.ctypes.data if ball.size else None, bc.ctypes.data,
                                   ctypes.byref(h)))
        self.h = h
        self.ctx = ctx
        self.n = n
        self.nsys = ns
        self.offsets = np.concatenate([[0], np.cumsum(n)])

    def close(self):
        if getattr(self, "h", None):
            load().gcme_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, pos: np.ndarray, vel: np.ndarray, stream=None):
        pos = np.ascontiguousarray(pos, np.float64)
        vel = np.ascontiguousarray(vel, np.float32)
        _check(load().gcme_batch_set_state(self.h, pos.ctypes.data, vel.ctypes.data,
                                           _stream(stream)))
        import torch
        torch.cuda.current_stream().synchronize()

    def get_state(self, stream=None):
        N = int(self.offsets[-1])
        pos = np.empty((N, 3), np.float64)
        vel = np.empty((N, 3), np.float32)
        E = np.empty((self.nsys, NTERMS), np.float64)
        _check(load().gcme_batch_get_state(self.h, pos.ctypes.data, vel.ctypes.data,
                                           E.ctypes.data, _stream(stream)))
        return pos, vel, E

    def step(self, nsteps: int, mode: int = 0, stream=None):
        _check(load().gcme_batch_step(self.h, int(nsteps), int(mode), _stream(stream)))

    def autotune(self, flags: int = 0, stream=None) -> dict:
        t = Tuning()
        _check(load().gcme_batch_autotune(self.h, int(flags), ctypes.byref(t), _stream(stream)))
        return t.as_dict()

    def apply_tuning(self, tuning: dict):
        _check(load().gcme_batch_apply_tuning(self.h, ctypes.byref(Tuning.from_dict(tuning))))

    def phase_timing(self, on: bool):
        _check(load().gcme_batch_phase_timing(self.h, int(bool(on))))

    def phase_ms(self):
        ms = np.zeros(8, np.float32)
        k = np.zeros(1, np.int32)
        _check(load().gcme_batch_phase_ms(self.h, ms.ctypes.data, 8, k.ctypes.data))
        return ms, int(k[0])

    def step_kernels(self):
        k = np.zeros(1, np.int32)
        _check(load().gcme_batch_phase_ms(self.h, None, 0, k.ctypes.data))
        return int(k[0])

    def pointers(self):
        p, v, e, o = _vp(), _vp(), _vp(), _vp()
        _check(load().gcme_batch_pointers(self.h, ctypes.byref(p), ctypes.byref(v),
                                          ctypes.byref(e), ctypes.byref(o)))
        return p.value, v.value, e.value


class Server:
    """Continuous-batching request server (gcme_server_create)."""

    def __init__(self, ctx: Context, hbm_budget: int, chunk_steps: int = 50,
                 max_active: int = 256):
        h = _vp()
        _check(load().gcme_server_create(ctx.h, int(hbm_budget), int(chunk_steps),
                                         int(max_active), ctypes.byref(h)))
        self.h = h
        self.ctx = ctx
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            load().gcme_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, params: Params, pos, vel, q, nsteps: int, bonds=None, types=None) -> int:
        pos = np.ascontiguousarray(pos, np.float64)
        vel = np.ascontiguousarray(vel, np.float32)
        q = np.ascontiguousarray(q, np.float64)
        req = Request()
        req.params = params
        req.n = int(q.shape[0])
        req.h_pos = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        req.h_vel = vel.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        req.h_q = q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if bonds is not None and len(bonds):
            b = np.ascontiguousarray(bonds, np.int32)
            req.h_bonds = b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            req.nbonds = int(b.shape[0])
        req.nsteps = int(nsteps)
        ty = _types(types, req.n)
        if ty is not None:
            req.h_types = ty.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        t = ctypes.c_uint64(0)
        _check(load().gcme_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = int(q.shape[0])
        return t.value

    def poll(self, ticket: int, want_state: bool = False):
        r = Result()
        n = self._keep.get(ticket, 0)
        pos = np.empty((n, 3), np.float64) if want_state else None
        vel = np.empty((n, 3), np.float32) if want_state else None
        _check(load().gcme_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r),
                                pos.ctypes.data if want_state else None,
                                vel.ctypes.data if want_state else None))
        return r, pos, vel

    def cancel(self, ticket: int):
        _check(load().gcme_cancel(self.h, ctypes.c_uint64(ticket)))

    def drain(self, timeout_s: float = 600.0):
        _check(load().gcme_server_drain(self.h, float(timeout_s)))

    def stats(self):
        out = np.zeros(10, np.int64)
        _check(load().gcme_server_stats(self.h, out.ctypes.data))
        return dict(zip(("admitted", "completed", "rejected", "chunks", "bead_steps",
                         "peak_active", "peak_bytes", "engines_built", "build_us", "wait_us"),
                        out.tolist()))
