// pair.cu -- K3 per-phase kernels (FP32 body in pair.cuh) and the plain
// FP64 pair kernel.
#include "pair.cuh"
#include "pair_warp.cuh"
#include "kernels.h"
#include "misc.cuh"

#include <algorithm>

namespace gcme {

template <bool VIR, bool DBG>
__global__ void __launch_bounds__(kPairThreads) k_pair_fine(Pool P, const int2 *work, int nwork) {
  pdl_wait();
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) dev_pair_fine_item<VIR, DBG>(P, work, w);
}

// Work items are fetched dynamically from a counter (zero before the launch;
// the CTA that fetches the last index puts it back to zero, all other CTAs
// having fetched their final index before it): a CTA takes the next item when
// it finishes one, so heavy cells do not leave SMs idle at the end, and a grid
// smaller than the SMs' capacity leaves slots free for the concurrent PME
// branch.  Items nwork .. nwork + nbi - 1 are harmonic bonds (one per thread),
// taken last, by CTAs that would otherwise idle at the end of the launch.
// One species without the debug dump runs the packed item (pair_core2), of
// one home cell, or of several along x when GRP (SysDesc::pair_group); DYN
// (SysDesc::pair_nelec < 0): the warps of a CTA take each item's tasks
// dynamically (pk_compute).
template <bool VIR, bool DBG, bool MT, bool GRP = false, bool DYN = false>
__global__ void __launch_bounds__(192, 5) k_pair_f32(Pool P, const int2 *work, int nwork,
                                                     int nbi, int *counter) {
  __shared__ __align__(16) unsigned char raw[kPairSmemBytes];
  __shared__ PairSeg seg[kItemSegs];
  __shared__ int s_total[2];
  __shared__ int s_item;
  __shared__ int s_task[DYN ? 3 : 1];
  __shared__ unsigned char stj[MT ? kPairCap : 1];
  __shared__ __align__(16) PairTab stab[MT ? kMaxTypes * kMaxTypes : 1];
  float4 *sj = reinterpret_cast<float4 *>(raw);
  constexpr bool PK = !DBG && !MT;
  // no early trigger: the kernels after this one would wait on SM slots the
  // concurrent PME branch can use
  pdl_wait();
  const int ntot = nwork + nbi;
  if (!counter) {  // static: one item per CTA (grid = items)
    for (int w = blockIdx.x; w < ntot; w += gridDim.x) {
      if (!DBG && w >= nwork) {
        dev_bonds<VIR, true>(P, (long long)(w - nwork) * blockDim.x + threadIdx.x);
        continue;
      }
      if (PK && GRP) dev_pair_f32_item_grp<VIR, DYN>(P, work, w, raw, seg, s_total, s_task);
      else if (PK) dev_pair_f32_item_pk<VIR, DYN>(P, work, w, raw, seg, s_total, s_task);
      else dev_pair_f32_item<VIR, DBG, MT>(P, work, w, sj, seg, s_total, stj, stab);
    }
    return;
  }
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_item;
    if (w >= ntot) {
      if (threadIdx.x == 0 && w == ntot + (int)gridDim.x - 1) atomicExch(counter, 0);
      break;
    }
    if (!DBG && w >= nwork) {
      dev_bonds<VIR, true>(P, (long long)(w - nwork) * blockDim.x + threadIdx.x);
      __syncthreads();  // every thread has read s_item before the next fetch
      continue;
    }
    if (PK && GRP) dev_pair_f32_item_grp<VIR, DYN>(P, work, w, raw, seg, s_total, s_task);
    else if (PK) dev_pair_f32_item_pk<VIR, DYN>(P, work, w, raw, seg, s_total, s_task);
    else dev_pair_f32_item<VIR, DBG, MT>(P, work, w, sj, seg, s_total, stj, stab);
  }
}

// One warp per work item (pair_warp.cuh): each warp fetches items from the
// counter by itself (the warp that fetches the last index puts the counter
// back to zero, every other warp having made its final fetch before it);
// items nwork .. nwork + nbi - 1 are harmonic bonds, 32 per item.  Dynamic
// shared memory: one WarpSmem per warp.
template <bool VIR>
__global__ void __launch_bounds__(128, 7) k_pair_warp(Pool P, const int2 *work, int nwork,
                                                     int nbi, int *counter) {
  extern __shared__ __align__(16) unsigned char wsm[];
  const int lane = threadIdx.x & 31;
  WarpSmem &W = reinterpret_cast<WarpSmem *>(wsm)[threadIdx.x >> 5];
  pdl_wait();
  const int ntot = nwork + nbi;
  const int nwarps = (int)gridDim.x * (int)(blockDim.x >> 5);
  while (true) {
    // one item at a time: fetching the next one early would let the warps
    // that start first take items from the warps that start later
    int w = 0;
    if (lane == 0) w = atomicAdd(counter, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= ntot) {
      if (lane == 0 && w == ntot + nwarps - 1) atomicExch(counter, 0);
      break;
    }
    if (w >= nwork) dev_bonds<VIR, true>(P, (long long)(w - nwork) * 32 + lane);
    else dev_pair_warp_item<VIR>(P, work, w, W, lane);
  }
}

// ---------------------------------------------------------------------------
// Plain FP64 path: one thread per real bead, 27 neighbour cells read straight
// from global memory, FP64 physics on the FP64 wrapped positions.  The
// in-cutoff decision uses the same FP32 rule as the FP32 path.
// ---------------------------------------------------------------------------
template <bool VIR, bool DBG>
__global__ void __launch_bounds__(128) k_pair_f64(Pool P) {
  pdl_wait();
  const long long gs = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // sorted slot
  double eg = 0.0, er = 0.0;
  double W[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) W[k] = 0.0;
  int s = 0;
  bool active = gs < P.n_ext;
  if (active) {
    const int e = P.sorted_idx[gs];
    // system of this sorted slot: sorted ranges follow the ext ranges
    {
      int lo = 0, hi = P.nsys - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.sys[mid].ext_off <= gs) lo = mid;
        else hi = mid - 1;
      }
      s = lo;
    }
    const SysDesc &S = P.sys[s];
    if (e >= S.n) active = false;
    if (active) {
      const float4 xi = P.xyzq_s[gs];
      const dpos4 pi = P.xyzq_s64[gs];
      const int cell = P.cell_of[S.ext_off + e];
      const int cx = cell % S.nc[0], cy = (cell / S.nc[0]) % S.nc[1],
                cz = cell / (S.nc[0] * S.nc[1]);
      double f[3] = {0, 0, 0};
      const double two_sqrtpi = 1.1283791670955126;
      const int m = S.cell_factor;
      for (int dzo = -m; dzo <= m; ++dzo)
        for (int dyo = -m; dyo <= m; ++dyo)
          for (int dxo = -m; dxo <= m; ++dxo) {
            const int u[3] = {cx + dxo, cy + dyo, cz + dzo};
            int v[3], nn[3];
            for (int a = 0; a < 3; ++a) {
              nn[a] = floor_div(u[a], S.nc[a]);
              v[a] = u[a] - nn[a] * S.nc[a];
            }
            const long long cg = S.cell_off + v[0] + S.nc[0] * (v[1] + S.nc[1] * v[2]);
            const int jb = P.cell_start[cg], je = P.cell_start[cg + 1];
            const int ja = P.cell_nimg[cg];
            const float sh[3] = {(float)nn[0] * S.boxf[0], (float)nn[1] * S.boxf[1],
                                 (float)nn[2] * S.boxf[2]};
            const bool self = dxo == 0 && dyo == 0 && dzo == 0;
            const int code = (nn[0] + 1) + 3 * (nn[1] + 1) + 9 * (nn[2] + 1);
            for (int j = jb; j < je; ++j) {
              if (self && j == gs) continue;
              const float4 xj = P.xyzq_s[j];
              float d0 = __fadd_rn(__fsub_rn(xj.x, xi.x), sh[0]);
              float d1 = __fadd_rn(__fsub_rn(xj.y, xi.y), sh[1]);
              float d2 = __fadd_rn(__fsub_rn(xj.z, xi.z), sh[2]);
              float r2f = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)),
                                    __fmul_rn(d2, d2));
              if (!(r2f < S.rc2f)) continue;
              if (DBG) {
                unsigned long long k = atomicAdd(&P.acc[(long long)s * kNacc + ACC_NPAIR], 1ull);
                if ((long long)k < P.dbg_cap) {
                  P.dbg_triples[3 * k + 0] = e;
                  P.dbg_triples[3 * k + 1] = P.sorted_idx[j];
                  P.dbg_triples[3 * k + 2] = code;
                }
              }
              const dpos4 pj = P.xyzq_s64[j];
              const double d[3] = {pj.x + nn[0] * S.box[0] - pi.x, pj.y + nn[1] * S.box[1] - pi.y,
                                   pj.z + nn[2] * S.box[2] - pi.z};
              const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
              // pair constants: the system's, or the species pair's
              double pref = S.gc_pref, expc = S.gc_expc, fc = S.gc_fc, beta = S.beta;
              const double *ser_g = S.ser_g, *ser_h = S.ser_h;
              if (P.ptab64) {
                const PairTab64 &T =
                    P.ptab64[S.tab_off + S.ntypes * (int)P.type_s[gs] + (int)P.type_s[j]];
                pref = T.pref;
                expc = T.expc;
                fc = T.fc;
                beta = T.beta;
                ser_g = T.sg;
                ser_h = T.sh;
              }
              double fs = 0.0;
              if (j - jb >= ja) {  // real j: Gaussian core
                const double u = pref * exp(-expc * r2);
                eg += 0.5 * u;
                fs += fc * u;
              }
              const double qq = pi.w * pj.w;
              if (qq != 0.0) {
                double g, h;
                if (r2 < 1e-4) {
                  g = ser_g[0] + r2 * (ser_g[1] + r2 * (ser_g[2] + r2 * ser_g[3]));
                  h = ser_h[0] + r2 * (ser_h[1] + r2 * ser_h[2]);
                } else {
                  const double r = sqrt(r2);
                  g = (erfc(S.kappa * r) - erfc(beta * r)) / r;
                  const double dd = two_sqrtpi * (beta * exp(-beta * beta * r2) -
                                                  S.kappa * exp(-S.kappa * S.kappa * r2));
                  h = (g - dd) / r2;
                }
                er += 0.5 * S.lB * qq * g;
                fs += S.lB * qq * h;
              }
              for (int a = 0; a < 3; ++a) f[a] -= fs * d[a];
              if (VIR)
                for (int a = 0; a < 3; ++a)
                  for (int b = 0; b < 3; ++b) W[3 * a + b] += 0.5 * fs * d[a] * d[b];
            }
          }
      for (int a = 0; a < 3; ++a)
        atomic_add_fixed(force_ptr(P, S, e, a), f[a], kFScale);
    }
  }
  // per-thread atomics (plain path: simplicity over speed)
  if (active) {
    unsigned long long *acc = P.acc + (long long)s * kNacc;
    atomic_add_fixed(acc + ACC_GC, eg, kEScale);
    atomic_add_fixed(acc + ACC_REAL, er, kEScale);
    if (VIR)
      for (int k = 0; k < 9; ++k) atomic_add_fixed(P.vacc + (long long)s * 9 + k, W[k], kEScale);
  }
}

void launch_pair(const Pool &P, const int2 *work, int nwork, bool fp64, int cell_factor,
                 int threads, int ctas, int *counter, bool vir, bool dbg, bool bonds,
                 cudaStream_t st, bool warp_items, bool groups, bool dyn) {
  if (P.n_ext == 0) return;
  if (fp64) {
    int nb = (int)((P.n_ext + 127) / 128);
    if (dbg) launch_k(k_pair_f64<false, true>, nb, 128, 0, st, P);
    else if (vir) launch_k(k_pair_f64<true, false>, nb, 128, 0, st, P);
    else launch_k(k_pair_f64<false, false>, nb, 128, 0, st, P);
    return;
  }
  if (nwork == 0) return;
  if (cell_factor == 2) {
    if (dbg) launch_k(k_pair_fine<false, true>, nwork, kPairThreads, 0, st, P, work, nwork);
    else if (vir) launch_k(k_pair_fine<true, false>, nwork, kPairThreads, 0, st, P, work, nwork);
    else launch_k(k_pair_fine<false, false>, nwork, kPairThreads, 0, st, P, work, nwork);
    return;
  }
  if (warp_items && !dbg && !P.ptab && ctas > 0 && counter) {
    const int tb = (threads == 64 || threads == 96) ? threads : 128;
    const int nbi = bonds ? (int)((P.n_bond + 31) / 32) : 0;
    const int ntot = nwork + nbi;
    const int wpc = tb / 32;
    const int grid = std::max(1, std::min(ctas, (ntot + wpc - 1) / wpc));
    const size_t shm = sizeof(WarpSmem) * wpc;
    if (vir) launch_k(k_pair_warp<true>, grid, tb, shm, st, P, work, nwork, nbi, counter);
    else launch_k(k_pair_warp<false>, grid, tb, shm, st, P, work, nwork, nbi, counter);
    return;
  }
  const int tb = (threads == 160 || threads == 192) ? threads : 128;
  const int nbi = (bonds && !dbg) ? (int)((P.n_bond + tb - 1) / tb) : 0;
  const int ntot = nwork + nbi;
  // ctas <= 0: one CTA per item; else a grid of ctas fetching items
  const bool fetch = ctas > 0;
  const int grid = fetch ? std::max(1, std::min(ntot, ctas)) : ntot;
  if (!fetch) counter = nullptr;
  auto go = [&](auto kern) { launch_k(kern, grid, tb, 0, st, P, work, nwork, nbi, counter); };
  if (P.ptab) {  // several species
    if (dbg) go(k_pair_f32<false, true, true>);
    else if (vir) go(k_pair_f32<true, false, true>);
    else go(k_pair_f32<false, false, true>);
    return;
  }
  if (dbg) go(k_pair_f32<false, true, false>);
  else if (dyn && groups && vir) go(k_pair_f32<true, false, false, true, true>);
  else if (dyn && groups) go(k_pair_f32<false, false, false, true, true>);
  else if (dyn && vir) go(k_pair_f32<true, false, false, false, true>);
  else if (dyn) go(k_pair_f32<false, false, false, false, true>);
  else if (groups && vir) go(k_pair_f32<true, false, false, true>);
  else if (groups) go(k_pair_f32<false, false, false, true>);
  else if (vir) go(k_pair_f32<true, false, false>);
  else go(k_pair_f32<false, false, false>);
}

}  // namespace gcme
