// pair_warp.cuh -- K3 FP32 pair kernel of the 27-cell stencil with one warp per work item.
//
// Same terms and work items as the CTA kernel of pair.cuh (Eq. u_ex and the
// real part of Eq. ewald; a work item is a home cell and 3 of its neighbour
// cells along x), but one warp carries a whole item by itself: it stages the
// item's candidates into its own slice of shared memory (neighbour beads
// beyond rc of the home cell's box dropped), then takes the home cell's real
// beads 32 at a time, each lane one home bead, and evaluates both terms for
// them: the Gaussian core over the staged real beads, the real-space
// electrostatics of its charged home beads over the staged charged and image
// beads.  Warps never wait for each other: no CTA barrier, no roles that
// finish at different times, and the latency of one warp's setup and
// staging is covered by the other warps resident on the SM, each at its own
// point of its own item.
//
// Shared memory per warp: kWRCap real candidates (x, y, z arrays), kWQCap
// charged or image candidates (x, y, z, charge), the item's segments and the
// record of what is staged.  An item whose candidates exceed a capacity is
// staged and evaluated in rounds, each round's partial sums written with the
// same fixed-point atomics (integer sums: the result does not depend on the
// rounds).
//
// Gaussian core: on systems whose core term at rc is below 1e-10 of its
// contact value (SysDesc::gc_tail) every staged real bead contributes without
// the r < rc test, the home cell included: its term for the home bead itself
// is exactly 1 (the distance is exactly 0), which is taken off the energy sum
// and adds nothing to force or virial.  Otherwise the neighbour rule of
// pair.cuh decides each pair.  Electrostatics: always the neighbour rule.
//
// Items per (home cell, part): SysDesc::pair_nch, item h taking the home
// chunks h, h + pair_nch, ...: more, shorter items than warps resident, so
// that warps fetching items dynamically even out the heavy cells (a single
// warp cannot fill an SM's issue slots, so one long item sets the launch's
// end).  Each item stages its neighbour beads itself.
#pragma once
#include "pair.cuh"

namespace gcme {

constexpr int kWRCap = 352;   // staged real candidates per warp
constexpr int kWQCap = 160;   // staged charged and image candidates per warp
constexpr int kWPieces = 8;   // staged pieces per round (segments or parts of them)

// A staged piece: beads [t0, t1) of segment k's real (or charged and image)
// list, kept ones at soff .. soff + n (padded to even), the first at sorted
// index jsorted0 when the piece is staged whole (the home cell).
struct WPiece {
  int k, soff, n, t0, t1, jsorted0;
};

struct WarpSmem {
  float rx[kWRCap], ry[kWRCap], rz[kWRCap];
  float qx[kWQCap], qy[kWQCap], qz[kWQCap], qq[kWQCap];
  PairSeg seg[9];
  WPiece rp[kWPieces], qp[kWPieces];
};

// Real-space electrostatics of a charged home bead over n2 (even) staged
// charged or image candidates: the neighbour rule on two candidates per
// packed instruction sets one bit per pair in range, 32 candidates at a time;
// g and h are evaluated for the set bits only.
template <bool SHIFT, bool SELF, bool VIR, bool TAB>
__device__ __forceinline__ void welec(const float *__restrict__ X, const float *__restrict__ Y,
                                      const float *__restrict__ Z, const float *__restrict__ Q,
                                      int n2, int jsorted0, const float4 &xi, int isorted,
                                      const PairSeg &g, const SysDesc &S, float rc2, PairAcc &A,
                                      const float4 *__restrict__ tab, float tab_scale,
                                      int tab_nm1) {
  const float2 mx = make_float2(-xi.x, -xi.x), my = make_float2(-xi.y, -xi.y),
               mz = make_float2(-xi.z, -xi.z);
  const float2 hx = make_float2(g.sh[0], g.sh[0]), hy = make_float2(g.sh[1], g.sh[1]),
               hz = make_float2(g.sh[2], g.sh[2]);
  for (int c0 = 0; c0 < n2; c0 += 32) {
    const int cn = min(32, n2 - c0);
    unsigned m = 0u;
    for (int u = 0; u < cn; u += 2) {
      float2 dx = __fadd2_rn(*reinterpret_cast<const float2 *>(X + c0 + u), mx);
      float2 dy = __fadd2_rn(*reinterpret_cast<const float2 *>(Y + c0 + u), my);
      float2 dz = __fadd2_rn(*reinterpret_cast<const float2 *>(Z + c0 + u), mz);
      if (SHIFT) {
        dx = __fadd2_rn(dx, hx);
        dy = __fadd2_rn(dy, hy);
        dz = __fadd2_rn(dz, hz);
      }
      const float2 r2 =
          __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)), __fmul2_rn(dz, dz));
      bool in0 = r2.x < rc2, in1 = r2.y < rc2;
      if (SELF) {
        in0 = in0 && (jsorted0 + c0 + u != isorted);
        in1 = in1 && (jsorted0 + c0 + u + 1 != isorted);
      }
      m |= ((unsigned)in0 | ((unsigned)in1 << 1)) << u;
    }
    elec_hits<VIR, TAB>(m, c0, X, Y, Z, Q, SHIFT ? xi.x - g.sh[0] : xi.x,
                        SHIFT ? xi.y - g.sh[1] : xi.y, SHIFT ? xi.z - g.sh[2] : xi.z, S, A, tab,
                        tab_scale, tab_nm1);
  }
}

// Within rc (+1e-3) of the home cell's box [lo, hi], after the segment's
// periodic shift.
__device__ __forceinline__ bool wnear(const float4 &v, const PairSeg &g, const float lo[3],
                                      const float hi[3], float cut2) {
  const float e[3] = {v.x + g.sh[0], v.y + g.sh[1], v.z + g.sh[2]};
  float d2 = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float d = fmaxf(0.0f, fmaxf(lo[a] - e[a], e[a] - hi[a]));
    d2 = fmaf(d, d, d2);
  }
  return d2 <= cut2;
}

// Stage beads [t, nb) of a segment list starting at global sorted index gbeg
// into the arrays at `used` while a step of 64 (32 for the charged arrays)
// still fits with its pad; all = keep every bead (the home cell).  Returns
// the number kept and advances t.  Warp-synchronous.
template <bool CHARGED>
__device__ __forceinline__ int wstage(const Pool &P, long long gbeg, int &t, int nb, int used,
                                      bool all, const PairSeg &g, const float lo[3],
                                      const float hi[3], float cut2, WarpSmem &W, int lane) {
  constexpr int kStep = CHARGED ? 32 : 64;
  constexpr int kCap = CHARGED ? kWQCap : kWRCap;
  const unsigned lt = (1u << lane) - 1u;
  const float4 far = make_float4(1e30f, 1e30f, 1e30f, 0.0f);
  int kept = 0;
  while (t < nb && used + kept + kStep + 1 <= kCap) {
    float4 v[kStep / 32];
#pragma unroll
    for (int u = 0; u < kStep / 32; ++u) {
      const int tt = t + 32 * u + lane;
      v[u] = tt < nb ? P.xyzq_s[gbeg + tt] : far;
    }
#pragma unroll
    for (int u = 0; u < kStep / 32; ++u) {
      const int tt = t + 32 * u + lane;
      const bool keep = tt < nb && (all || wnear(v[u], g, lo, hi, cut2));
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int p = used + kept + __popc(m & lt);
        if (CHARGED) {
          W.qx[p] = v[u].x;
          W.qy[p] = v[u].y;
          W.qz[p] = v[u].z;
          W.qq[p] = v[u].w;
        } else {
          W.rx[p] = v[u].x;
          W.ry[p] = v[u].y;
          W.rz[p] = v[u].z;
        }
      }
      kept += __popc(m);
    }
    t = min(t + kStep, nb);
  }
  if ((kept & 1) && lane == 0) {  // pad to even: far away, no charge
    const int p = used + kept;
    if (CHARGED) {
      W.qx[p] = far.x;
      W.qy[p] = far.y;
      W.qz[p] = far.z;
      W.qq[p] = 0.0f;
    } else {
      W.rx[p] = far.x;
      W.ry[p] = far.y;
      W.rz[p] = far.z;
    }
  }
  return kept;
}

// Evaluate the item's chunks of 32 home real beads (chunks ch, ch + nch, ...)
// over the staged pieces and write the partial sums.  Warp-synchronous.
template <bool VIR>
__device__ __forceinline__ void wflush(const Pool &P, const SysDesc &S, int s, int rbeg, int hend,
                                       int nqr, int ch, int nch, int npr, int npq, WarpSmem &W,
                                       int lane) {
  __syncwarp();
  const float rc2 = S.rc2f, gcc = S.gc_c2f;
  const bool tail = S.gc_tail != 0;
  const float4 *tab = P.rtab + S.rtab_off;
  const float tab_scale = S.rtab_scale;
  const int tab_nm1 = S.rtab_n - 1;
  for (int c0 = 32 * ch; c0 < hend - rbeg; c0 += 32 * nch) {
    const int ih = c0 + lane;  // home index among the cell's real beads
    const int i = rbeg + ih;
    const bool valid = i < hend;
    const float4 xi = valid ? P.xyzq_s[i] : make_float4(1e30f, 1e30f, 1e30f, 0.0f);
    PairAcc A;
    A.eg = A.ere = A.gx = A.gy = A.gz = A.fx = A.fy = A.fz = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) A.wg[k] = A.we[k] = 0.0f;
    {
      PairAcc2 B;
      B.eg = B.gx = B.gy = B.gz = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 6; ++k) B.wg[k] = make_float2(0.0f, 0.0f);
      float self_term = 0.0f;
      for (int p = 0; p < npr; ++p) {
        const WPiece pc = W.rp[p];
        const PairSeg &g = W.seg[pc.k];
        const int n2 = (pc.n + 1) & ~1;
        const float *X = W.rx + pc.soff, *Y = W.ry + pc.soff, *Z = W.rz + pc.soff;
        if (tail) {
          pair_core2_tail<VIR>(X, Y, Z, n2, xi, g, gcc, B);
          // the home bead's own term (exactly 1) when it is staged here
          if (g.self && ih >= pc.t0 && ih < pc.t1) self_term += 1.0f;
        } else if (g.self) {
          pair_core2<false, true, VIR>(X, Y, Z, n2, pc.jsorted0, xi, i, g, rc2, gcc, B);
        } else if (g.shifted) {
          pair_core2<true, false, VIR>(X, Y, Z, n2, 0, xi, i, g, rc2, gcc, B);
        } else {
          pair_core2<false, false, VIR>(X, Y, Z, n2, 0, xi, i, g, rc2, gcc, B);
        }
      }
      A.eg = (B.eg.x + B.eg.y) - self_term;
      A.gx = B.gx.x + B.gx.y;
      A.gy = B.gy.x + B.gy.y;
      A.gz = B.gz.x + B.gz.y;
      if (VIR)
#pragma unroll
        for (int k = 0; k < 6; ++k) A.wg[k] = B.wg[k].x + B.wg[k].y;
    }
    // electrostatics for the charged home beads (the first nqr reals)
    const bool qi = valid && ih < nqr && xi.w != 0.0f;
    if (__any_sync(0xffffffffu, qi) && qi) {
      for (int p = 0; p < npq; ++p) {
        const WPiece pc = W.qp[p];
        const PairSeg &g = W.seg[pc.k];
        const int n2 = (pc.n + 1) & ~1;
        const float *X = W.qx + pc.soff, *Y = W.qy + pc.soff, *Z = W.qz + pc.soff,
                    *Q = W.qq + pc.soff;
        if (tab_nm1 >= 0) {
          if (g.self)
            welec<false, true, VIR, true>(X, Y, Z, Q, n2, pc.jsorted0, xi, i, g,
                                          S, rc2, A, tab, tab_scale, tab_nm1);
          else if (g.shifted)
            welec<true, false, VIR, true>(X, Y, Z, Q, n2, 0, xi, i, g,
                                          S, rc2, A, tab, tab_scale, tab_nm1);
          else
            welec<false, false, VIR, true>(X, Y, Z, Q, n2, 0, xi, i, g,
                                           S, rc2, A, tab, tab_scale, tab_nm1);
        } else {  // no table (very small smearing radius)
          if (g.self)
            welec<false, true, VIR, false>(X, Y, Z, Q, n2, pc.jsorted0, xi, i, g,
                                           S, rc2, A, tab, tab_scale, tab_nm1);
          else if (g.shifted)
            welec<true, false, VIR, false>(X, Y, Z, Q, n2, 0, xi, i, g,
                                           S, rc2, A, tab, tab_scale, tab_nm1);
          else
            welec<false, false, VIR, false>(X, Y, Z, Q, n2, 0, xi, i, g,
                                            S, rc2, A, tab, tab_scale, tab_nm1);
        }
      }
      elec_scale<VIR>(A, xi.w);
    }
    pair_write<VIR>(P, S, s, valid, i, A);
  }
  __syncwarp();
}

// One work item by one warp (see the file comment).  W is this warp's slice.
template <bool VIR>
__device__ __forceinline__ void dev_pair_warp_item(const Pool &P, const int2 *work, int w,
                                                   WarpSmem &W, int lane) {
  const int s = work[w].x, code = work[w].y;
  if (P.list_ovf && !P.list_ovf[s]) return;  // lists: only systems whose lists overflowed
  const SysDesc &S = P.sys[s];
  const int split = S.pair_split, nch = S.pair_nch;
  const int base = code / nch, ch = code - base * nch;  // chunk group
  const int cloc = base / split, part = base % split;
  const int nseg = 27 / split;
  const long long hg = S.cell_off + cloc;
  const int hbeg = P.cell_start[hg], hend = P.cell_start[hg + 1];
  const int himg = P.cell_nimg[hg], hq = P.cell_nq[hg];
  const int rbeg = hbeg + himg;
  if (hend - rbeg <= 32 * ch) return;  // no home chunk for this group
  const int nqr = hbeg + hq - rbeg;
  if (lane < nseg) W.seg[lane] = item_segment(P, S, cloc, part, lane);
  float lo[3], hi[3];
  {
    const int hc[3] = {cloc % S.nc[0], (cloc / S.nc[0]) % S.nc[1], cloc / (S.nc[0] * S.nc[1])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = (float)hc[a] * S.cside[a];
      hi[a] = lo[a] + S.cside[a];
    }
  }
  const float cut2 = S.cull2;
  __syncwarp();
  int usedr = 0, usedq = 0, npr = 0, npq = 0;
  for (int k = 0; k < nseg; ++k) {
    const PairSeg g = W.seg[k];
    const int nr = g.n - g.a, nb = g.b;
    int tr = 0, tq = 0;
    while (tr < nr || tq < nb) {
      if (tr < nr && npr < kWPieces) {
        const int t0 = tr;
        const int kept = wstage<false>(P, (long long)g.beg + g.a, tr, nr, usedr, g.self, g, lo, hi,
                                       cut2, W, lane);
        if (tr > t0 && lane == 0) {
          WPiece pc;
          pc.k = k;
          pc.soff = usedr;
          pc.n = kept;
          pc.t0 = t0;
          pc.t1 = tr;
          pc.jsorted0 = g.beg + g.a + t0;
          W.rp[npr] = pc;
        }
        if (tr > t0) {
          ++npr;
          usedr += (kept + 1) & ~1;
        }
      }
      if (tq < nb && npq < kWPieces) {
        const int t0 = tq;
        const int kept =
            wstage<true>(P, (long long)g.beg, tq, nb, usedq, g.self, g, lo, hi, cut2, W, lane);
        if (tq > t0 && lane == 0) {
          WPiece pc;
          pc.k = k;
          pc.soff = usedq;
          pc.n = kept;
          pc.t0 = t0;
          pc.t1 = tq;
          pc.jsorted0 = g.beg + t0;
          W.qp[npq] = pc;
        }
        if (tq > t0) {
          ++npq;
          usedq += (kept + 1) & ~1;
        }
      }
      if (tr < nr || tq < nb) {  // a capacity is reached: evaluate this round
        wflush<VIR>(P, S, s, rbeg, hend, nqr, ch, nch, npr, npq, W, lane);
        usedr = usedq = npr = npq = 0;
      }
    }
  }
  if (npr + npq > 0) wflush<VIR>(P, S, s, rbeg, hend, nqr, ch, nch, npr, npq, W, lane);
}

}  // namespace gcme
