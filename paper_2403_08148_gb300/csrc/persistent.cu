// persistent.cu -- K13: every phase of nsteps velocity-Verlet steps of a
// whole batch in one cooperative launch.
//
// One CTA per resident slot (occupancy x SMs), all co-resident (cooperative
// launch).  Phases are separated by a grid barrier whose wait is bounded: a
// CTA that waits longer than the budget sets the batch's error word and
// every CTA leaves the kernel at its next barrier, so a broken phase ends
// the launch with GCME_ERR_TIMEOUT instead of hanging the GPU.  The phase
// bodies are the device functions of the per-phase kernels, so both modes
// compute bit-identical trajectories.
#include "cells.cuh"
#include "kernels.h"
#include "misc.cuh"
#include "pair.cuh"
#include "pair_warp.cuh"
#include "pme.cuh"

#include <algorithm>

namespace gcme {

struct Barrier {
  unsigned int *count;  // arrivals of the current barrier
  unsigned int *gen;    // generation, bumped by the last arrival
  int *err;             // 0 = fine, 1 = a wait ran out
  long long budget;     // clock64 cycles before giving up
};

// Grid-wide barrier with a bounded wait.  Returns false when any CTA timed
// out (then every CTA must leave the kernel).
__device__ __forceinline__ bool grid_barrier(const Barrier &B) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *vgen = B.gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(B.count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(B.count, 0u);
      __threadfence();
      atomicAdd(B.gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*(volatile int *)B.err) break;
        if (clock64() - t0 > B.budget) {
          atomicExch(B.err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)B.err == 0;
}

struct PersistArgs {
  const int2 *pair_work;
  int n_pair_work;
  int cell_factor;
  int warp_items;  // the pair work list holds warp items (pair_warp.cuh)
  int dyn;         // CTA items' tasks taken dynamically (SysDesc::pair_nelec < 0)
  PmePlan plan;
  long long nsteps;
  Barrier bar;
};

// Loop over [0, n) in steps of the whole grid, rounded up to full warps so
// warp-synchronous bodies see every lane.
#define GRID_LOOP(i, n)                                                              \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x,               \
                 _lim = ((n) + 31) / 32 * 32;                                        \
       i - threadIdx.x % 32 < _lim; i += (long long)gridDim.x * blockDim.x)

__global__ void __launch_bounds__(128) k_persistent(Pool P, PersistArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Barrier &B = A.bar;
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long step = 0; step < A.nsteps; ++step) {
    // ---- half kick + drift (which clears the forces it has read); clear
    // accumulators, cell counts, charge grid
    for (long long g = gtid; g < P.n_real; g += gthreads) dev_kick_drift<float>(P, g);
    for (long long k = gtid; k < (long long)P.nsys * kNacc; k += gthreads) P.acc[k] = 0;
    for (long long k = gtid; k < P.n_cells; k += gthreads) P.cell_cnt[k] = 0;
    for (long long k = gtid; k < P.n_grid; k += gthreads) P.qgrid[k] = 0;
    if (!grid_barrier(B)) return;
    // ---- K1 wrap + bin
    for (long long g = gtid; g < P.n_ext; g += gthreads) dev_bin(P, g);
    if (!grid_barrier(B)) return;
    // ---- K2 scan (one CTA), scatter, per-cell order
    if (blockIdx.x == 0) dev_scan_block(P.cell_cnt, P.cell_start, P.n_cells, (long long *)smem);
    if (!grid_barrier(B)) return;
    for (long long g = gtid; g < P.n_ext; g += gthreads) dev_scatter(P, g);
    if (!grid_barrier(B)) return;
    for (long long c = blockIdx.x; c < P.n_cells; c += gridDim.x)
      dev_cellsort_block(P, c, (long long *)smem, (int *)(smem + sizeof(long long) * kSortCap));
    if (!grid_barrier(B)) return;
    // ---- K3 pair kernel and K5 spread (independent outputs)
    if (A.cell_factor == 2) {
      for (int w = blockIdx.x; w < A.n_pair_work; w += gridDim.x)
        dev_pair_fine_item<false, false>(P, A.pair_work, w);
    } else {
      float4 *sj = reinterpret_cast<float4 *>(smem);
      PairSeg *seg = reinterpret_cast<PairSeg *>(smem + kPairSmemBytes);
      int *st =
          reinterpret_cast<int *>(smem + kPairSmemBytes + sizeof(PairSeg) * kItemSegs);
      // several species: the table (16-byte aligned) and the staged species
      int *stask = st + 2;  // three task counters
      const size_t toff = (kPairSmemBytes + sizeof(PairSeg) * kItemSegs + 32 + 15) / 16 * 16;
      PairTab *stab = reinterpret_cast<PairTab *>(smem + toff);
      unsigned char *stj = smem + toff + sizeof(PairTab) * kMaxTypes * kMaxTypes;
      if (A.warp_items) {  // one warp per work item (pair_warp.cuh)
        WarpSmem &W = reinterpret_cast<WarpSmem *>(smem)[threadIdx.x >> 5];
        const int nw = (int)gridDim.x * (int)(blockDim.x >> 5);
        for (int w = blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
             w < A.n_pair_work; w += nw)
          dev_pair_warp_item<false>(P, A.pair_work, w, W, (int)(threadIdx.x & 31));
      } else {
        for (int w = blockIdx.x; w < A.n_pair_work; w += gridDim.x) {
          if (P.ptab)
            dev_pair_f32_item<false, false, true>(P, A.pair_work, w, sj, seg, st, stj, stab);
          else if (A.dyn)
            dev_pair_f32_item_grp<false, true>(P, A.pair_work, w, smem, seg, st, stask);
          else
            dev_pair_f32_item_grp<false>(P, A.pair_work, w, smem, seg, st);
        }
      }
    }
    for (long long g = gtid; g < P.n_q * 8; g += gthreads) dev_spread<float, 0>(P, g);
    if (!grid_barrier(B)) return;
    // ---- K6/K7 FFT passes with the fused influence function
    if (A.plan.use_plane) {
      for (int w = blockIdx.x; w < A.plan.nplane; w += gridDim.x)
        dev_fft_plane<float, false>(P, A.plan.plane_work, w, smem);
      if (!grid_barrier(B)) return;
      for (int w = blockIdx.x; w < A.plan.nwork[2]; w += gridDim.x)
        dev_fft_item<float, false>(P, A.plan.work[2], w, 2, FFT_FWD_INFL_INV, A.plan.lpb[2], 1,
                                   smem);
      if (!grid_barrier(B)) return;
      for (int w = blockIdx.x; w < A.plan.nplane; w += gridDim.x)
        dev_fft_plane<float, true>(P, A.plan.plane_work, w, smem);
      if (!grid_barrier(B)) return;
    } else {
      const int axes[5] = {0, 1, 2, 1, 0};
      const int kinds[5] = {FFT_FWD_FROM_Q, FFT_FWD, FFT_FWD_INFL_INV, FFT_INV, FFT_INV};
      for (int ps = 0; ps < 5; ++ps) {
        const int ax = axes[ps];
        for (int w = blockIdx.x; w < A.plan.nwork[ax]; w += gridDim.x)
          dev_fft_item<float, false>(P, A.plan.work[ax], w, ax, kinds[ps], A.plan.lpb[ax], 0,
                                     smem);
        if (!grid_barrier(B)) return;
      }
    }
    // ---- K8 gather, K9 bonds, walls and dipole
    GRID_LOOP(g, P.n_q * 8) dev_gather<float, 0>(P, g);
    GRID_LOOP(b, P.n_bond) dev_bonds<false>(P, b);
    GRID_LOOP(g, P.n_real) dev_walls(P, g);
    if (!grid_barrier(B)) return;
    // ---- K10 Yeh-Berkowitz forces
    for (long long g = gtid; g < P.n_real; g += gthreads) dev_slab_apply(P, g);
    if (!grid_barrier(B)) return;
    // ---- K11 half kick, K12 energies
    GRID_LOOP(g, P.n_real) dev_kick<float>(P, g);
    if (!grid_barrier(B)) return;
    for (long long s = gtid; s < P.nsys; s += gthreads) dev_finalize<false>(P, (int)s);
    if (!grid_barrier(B)) return;
  }
}
#undef GRID_LOOP

size_t persistent_smem(const PmePlan &pl, bool species, bool warp_items) {
  size_t pair = kPairSmemBytes + sizeof(PairSeg) * kItemSegs + 32;
  if (warp_items) pair = std::max(pair, 4 * sizeof(WarpSmem));  // 128 threads = 4 warps
  if (species)
    pair = (pair + 15) / 16 * 16 + sizeof(PairTab) * kMaxTypes * kMaxTypes + kPairCap;
  size_t sort = sizeof(long long) * kSortCap + 16;
  size_t fft = 0;
  for (int a = 0; a < 3; ++a)
    fft = std::max(fft, (2 * (size_t)pl.lpb[a] + 1) * pl.kmax[a] * sizeof(float2));
  if (pl.use_plane)
    fft = std::max(fft, (2 * (size_t)pl.plane_elems + pl.kmax[0] + pl.kmax[1]) * sizeof(float2));
  return std::max(pair, std::max(sort, fft));
}

int launch_persistent(const Pool &P, const int2 *pair_work, int n_pair_work, int cell_factor,
                      const PmePlan &pl, long long nsteps, unsigned int *bar_words, double timeout_s,
                      cudaStream_t st, bool warp_items, bool dyn) {
  warp_items = warp_items && !P.ptab && cell_factor == 1;
  const size_t smem = persistent_smem(pl, P.ptab != nullptr, warp_items);
  cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0, per_sm = 0, clock_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, 128, smem);
  if (e != cudaSuccess || per_sm < 1) return -1;
  PersistArgs A;
  A.pair_work = pair_work;
  A.n_pair_work = n_pair_work;
  A.cell_factor = cell_factor;
  A.warp_items = warp_items ? 1 : 0;
  A.dyn = dyn && !P.ptab && cell_factor == 1 ? 1 : 0;
  A.plan = pl;
  A.nsteps = nsteps;
  A.bar.count = bar_words;
  A.bar.gen = bar_words + 1;
  A.bar.err = reinterpret_cast<int *>(bar_words + 2);
  A.bar.budget = (long long)(timeout_s * (double)clock_khz * 1e3);
  cudaMemsetAsync(bar_words, 0, 4 * sizeof(unsigned int), st);
  Pool Pc = P;
  void *args[] = {&Pc, &A};
  e = cudaLaunchCooperativeKernel((const void *)k_persistent, dim3(nsm * per_sm), dim3(128), args,
                                  smem, st);
  return e == cudaSuccess ? 0 : -2;
}

// A barrier that never completes: the last CTA leaves without arriving, so
// the generation word is never bumped and every waiting CTA's bounded wait
// must run out and set the error word.
__global__ void k_barrier_probe(Barrier B) {
  if (blockIdx.x == gridDim.x - 1) return;
  grid_barrier(B);
}

int launch_barrier_probe(unsigned int *bar_words, double timeout_s, cudaStream_t st) {
  int dev = 0, clock_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  Barrier B;
  B.count = bar_words;
  B.gen = bar_words + 1;
  B.err = reinterpret_cast<int *>(bar_words + 2);
  B.budget = (long long)(timeout_s * (double)clock_khz * 1e3);
  cudaMemsetAsync(bar_words, 0, 4 * sizeof(unsigned int), st);
  void *args[] = {&B};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(4), dim3(32),
                                              args, 0, st);
  return e == cudaSuccess ? 0 : -2;
}

}  // namespace gcme
