// pair.cuh -- K3 device bodies: Gaussian core + real-space smeared Coulomb over cell pairs.
//
// For every ordered in-cutoff triple (i, j, image n) with i a real bead:
//   Gaussian core (Eq. u_ex), both beads real:
//     u = A (3/(2 pi s))^{3/2} exp(-3 r^2/(2 s)),  F_i = -(3/s) u d
//   real-space electrostatics (Eq. ewald, real part), both charged:
//     u = lB z_i z_j g(r),  g = [erfc(kappa r) - erfc(beta r)] / r
//     F_i = -lB z_i z_j h(r) d,  h = -g'(r)/r
// with d = r_j + n L - r_i.  Each bead i sums over all j (full shell), so
// every unordered pair is visited from both ends and energies are halved.
// Image beads (conducting-slab geometry) appear only as j; visiting the
// real-image pairs from the real side only yields exactly the physical
// energy E_rr + E_ri / 2.
//
// In-cutoff rule (bit-exact with the oracle): on the wrapped FP32 positions
//   d_a = fl(fl(x_j,a - x_i,a) + fl(n_a L_a)),
//   r2 = fl(fl(fl(d_x^2) + fl(d_y^2)) + fl(d_z^2)),  in iff r2 < fl(rc^2).
//
// FP32 path (27-cell stencil): one work item is a home cell and 3 (or 9) of
// its neighbour cells; a CTA of 128-192 threads stages the item's
// candidates in shared memory and splits into roles: Gaussian-core warps
// (one home bead per lane, two candidates per packed FP32x2 instruction over
// coordinate arrays) and 1-3 electrostatics warps (the charged home beads
// over the charged and image candidates, a 32-bit in-cutoff mask per 32
// candidates, then the real-space term from a per-system table for the
// hits only).  Within a cell the images, charged and neutral beads are
// contiguous, so no per-pair class test is needed.  Forces are summed in
// FP32 per lane and added to 64-bit fixed-point accumulators; each lane's
// energy and virial partials are rounded to 2^-32 fixed point and summed as
// integers (order-independent, no FP64 arithmetic).
#pragma once
#include "common.cuh"


namespace gcme {

constexpr int kPairThreads = 128;  // block of the fine-cell kernel
constexpr int kPairCap = 1536;  // staged j beads per work item (8 CTAs of 128 per SM)
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

struct PairAcc {
  float eg, ere;
  float gx, gy, gz;
  float fx, fy, fz;
  float wg[6], we[6];
};

struct PairSeg {
  int beg, n, a, b;  // global sorted begin, count, end of images, end of charged
  int soff;          // offset in shared memory
  int code;          // image code (nx+1) + 3 (ny+1) + 9 (nz+1)
  float sh[3];
  int self;
  int shifted;
  int qoff;          // packed items: offset of the charged/image beads' float4
  int nk, bk;        // packed items: real and charged/image beads staged (kept)
};

// Packed items: the real beads of the staged cells as three coordinate
// arrays of kPkCap floats, the charged and image beads as four arrays (x, y,
// z, charge) of kPkCapQ floats (each cell padded to an even count in both);
// this and the scalar items' float4 array share one shared-memory block of
// kPairSmemBytes.
constexpr int kPkCap = 1280;
// segments of a CTA work item in shared memory: up to 9 staged, then up to
// 3 home cells (packed items)
constexpr int kItemSegs = 12;
constexpr int kPkCapQ = 640;
constexpr int kPairSmemBytes =
    (16 * kPairCap > 12 * kPkCap + 16 * kPkCapQ) ? 16 * kPairCap : 12 * kPkCap + 16 * kPkCapQ;

// In-cutoff test of one candidate (the FP32 rule above).
template <bool SHIFT>
__device__ __forceinline__ float pair_r2(const float4 &xj, const float4 &xi, const PairSeg &sg,
                                         float &dx, float &dy, float &dz) {
  dx = __fsub_rn(xj.x, xi.x);
  dy = __fsub_rn(xj.y, xi.y);
  dz = __fsub_rn(xj.z, xi.z);
  if (SHIFT) {
    dx = __fadd_rn(dx, sg.sh[0]);
    dy = __fadd_rn(dy, sg.sh[1]);
    dz = __fadd_rn(dz, sg.sh[2]);
  }
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// g(r) and h(r) of the real-space term evaluated directly: the small-r
// Taylor series (sgf, shf) while beta r < 0.055 (its truncation error is
// then below 1e-9 relative), else erfc and exp.
__device__ __forceinline__ void real_gh_direct(float r2, float betaf, float kappaf,
                                               const float *sgf, const float *shf, float &g,
                                               float &h) {
  if (r2 * (betaf * betaf) < 3e-3f) {
    g = sgf[0] + r2 * (sgf[1] + r2 * (sgf[2] + r2 * sgf[3]));
    h = shf[0] + r2 * (shf[1] + r2 * shf[2]);
  } else {
    const float r = sqrtf(r2);
    const float rinv = 1.0f / r;
    const float xb = betaf * r, xk = kappaf * r;
    g = (erfcf(xk) - erfcf(xb)) * rinv;
    const float eb = ex2_approx(-xb * xb * kLog2e);
    const float ek = ex2_approx(-xk * xk * kLog2e);
    const float dd = kTwoOverSqrtPi * (betaf * eb - kappaf * ek);
    h = (g - dd) * (rinv * rinv);
  }
}

// Gaussian core over real j in [t0, t1): every lane evaluates every
// candidate (the exponential is cheap next to the test, so masking beats
// branching); out-of-cutoff candidates contribute exactly zero.
//
// MT (several species): the pair constants come from row[species of j] (the
// row of i's species in the system's table), e carries the prefactor and
// the force sums carry fc, so pair_write scales them by 1 instead.
template <bool SHIFT, bool SELF, bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void pair_core(const float4 *__restrict__ J, int t0, int t1,
                                          int jsorted0, const float4 &xi, int isorted,
                                          const PairSeg &sg, float rc2, float gcc, PairAcc &A,
                                          const Pool &P, int s, const PairTab *row = nullptr,
                                          const unsigned char *tj = nullptr) {
#pragma unroll 4
  for (int t = t0; t < t1; ++t) {
    float dx, dy, dz;
    const float r2 = pair_r2<SHIFT>(J[t], xi, sg, dx, dy, dz);
    bool in = r2 < rc2;
    if (SELF) in = in && (jsorted0 + t != isorted);
    float e, fs;
    if (MT) {
      const float4 T = *reinterpret_cast<const float4 *>(row + tj[t]);  // pref, c2, fc, beta
      e = in ? T.x * ex2_approx(r2 * T.y) : 0.0f;
      fs = T.z * e;
    } else {
      e = ex2_approx(r2 * gcc);
      e = in ? e : 0.0f;
      fs = e;
    }
    A.eg += e;
    A.gx = fmaf(fs, dx, A.gx);
    A.gy = fmaf(fs, dy, A.gy);
    A.gz = fmaf(fs, dz, A.gz);
    if (VIR) {
      float ex = fs * dx, ey = fs * dy;
      A.wg[0] = fmaf(ex, dx, A.wg[0]);
      A.wg[1] = fmaf(ey, dy, A.wg[1]);
      A.wg[2] = fmaf(fs * dz, dz, A.wg[2]);
      A.wg[3] = fmaf(ex, dy, A.wg[3]);
      A.wg[4] = fmaf(ex, dz, A.wg[4]);
      A.wg[5] = fmaf(ey, dz, A.wg[5]);
    }
    if (DBG && in) {
      unsigned long long k = atomicAdd(&P.acc[(long long)s * kNacc + ACC_NPAIR], 1ull);
      if ((long long)k < P.dbg_cap) {
        P.dbg_triples[3 * k + 0] = P.sorted_idx[isorted];
        P.dbg_triples[3 * k + 1] = P.sorted_idx[jsorted0 + t];
        P.dbg_triples[3 * k + 2] = sg.code;
      }
    }
  }
}

// Real-space electrostatics of a charged i over charged j in [t0, t1)
// (images and charged reals), 64 candidates at a time: a test pass sets
// one bit per in-cutoff pair, then the erfc/exp work runs over the set bits
// only, so a warp pays for it once per hit instead of once per candidate.
// tg marks the first real j (images below it carry no core and are dumped
// here in debug mode).
template <bool SHIFT, bool SELF, bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void pair_elec(const float4 *__restrict__ J, int t0, int t1, int tg,
                                          int jsorted0, const float4 &xi, int isorted,
                                          const PairSeg &sg, const SysDesc &S, float rc2,
                                          PairAcc &A, const Pool &P, int s,
                                          const PairTab *row = nullptr,
                                          const unsigned char *tj = nullptr) {
  const bool qi_nz = xi.w != 0.0f;
  for (int c0 = t0; c0 < t1; c0 += 64) {
    const int cn = min(64, t1 - c0);
    unsigned long long m = 0ull;
    if (qi_nz) {
      for (int u = 0; u < cn; ++u) {
        float dx, dy, dz;
        const float r2 = pair_r2<SHIFT>(J[c0 + u], xi, sg, dx, dy, dz);
        bool in = r2 < rc2;
        if (SELF) in = in && (jsorted0 + c0 + u != isorted);
        m |= (unsigned long long)in << u;
      }
    }
    while (m) {
      const int u = __ffsll((long long)m) - 1;
      m &= m - 1ull;
      const int t = c0 + u;
      const float4 xj = J[t];
      float dx, dy, dz;
      const float r2 = pair_r2<SHIFT>(xj, xi, sg, dx, dy, dz);
      const float qq = xi.w * xj.w;
      const float* sgf = S.ser_gf;
      const float* shf = S.ser_hf;
      float betaf = S.betaf;
      if (MT) {
        const PairTab &T = row[tj[t]];
        sgf = T.sg;
        shf = T.sh;
        betaf = T.beta;
      }
      float g, h;
      if (!MT && S.rtab_n > 0) real_gh_tab(P, S, r2, g, h);
      else real_gh_direct(r2, betaf, S.kappaf, sgf, shf, g, h);
      A.ere = fmaf(qq, g, A.ere);
      const float fq = qq * h;
      A.fx = fmaf(fq, dx, A.fx);
      A.fy = fmaf(fq, dy, A.fy);
      A.fz = fmaf(fq, dz, A.fz);
      if (VIR) {
        float ex = fq * dx, ey = fq * dy;
        A.we[0] = fmaf(ex, dx, A.we[0]);
        A.we[1] = fmaf(ey, dy, A.we[1]);
        A.we[2] = fmaf(fq * dz, dz, A.we[2]);
        A.we[3] = fmaf(ex, dy, A.we[3]);
        A.we[4] = fmaf(ex, dz, A.we[4]);
        A.we[5] = fmaf(ey, dz, A.we[5]);
      }
      if (DBG && t < tg) {
        unsigned long long k = atomicAdd(&P.acc[(long long)s * kNacc + ACC_NPAIR], 1ull);
        if ((long long)k < P.dbg_cap) {
          P.dbg_triples[3 * k + 0] = P.sorted_idx[isorted];
          P.dbg_triples[3 * k + 1] = P.sorted_idx[jsorted0 + t];
          P.dbg_triples[3 * k + 2] = sg.code;
        }
      }
    }
  }
}

// Gaussian core over the staged real beads of one cell, two candidates per
// instruction with the sm_100 packed FP32 operations (per component the
// same IEEE round-to-nearest operations as the scalar rule above, so the
// in-cutoff decisions are unchanged).  X, Y, Z: n2 (even) coordinates; a
// pad entry sits far away.  The two halves of each sum are kept apart.
struct PairAcc2 {
  float2 eg, gx, gy, gz;
  float2 wg[6];
};

template <bool SHIFT, bool SELF, bool VIR>
__device__ __forceinline__ void pair_core2(const float *__restrict__ X,
                                           const float *__restrict__ Y,
                                           const float *__restrict__ Z, int n2, int jsorted0,
                                           const float4 &xi, int isorted, const PairSeg &sg,
                                           float rc2, float gcc, PairAcc2 &A) {
  const float2 mx = make_float2(-xi.x, -xi.x), my = make_float2(-xi.y, -xi.y),
               mz = make_float2(-xi.z, -xi.z);
  const float2 hx = make_float2(sg.sh[0], sg.sh[0]), hy = make_float2(sg.sh[1], sg.sh[1]),
               hz = make_float2(sg.sh[2], sg.sh[2]);
  const float2 g2 = make_float2(gcc, gcc);
#pragma unroll 4
  for (int t = 0; t < n2; t += 2) {
    float2 dx = __fadd2_rn(*reinterpret_cast<const float2 *>(X + t), mx);
    float2 dy = __fadd2_rn(*reinterpret_cast<const float2 *>(Y + t), my);
    float2 dz = __fadd2_rn(*reinterpret_cast<const float2 *>(Z + t), mz);
    if (SHIFT) {
      dx = __fadd2_rn(dx, hx);
      dy = __fadd2_rn(dy, hy);
      dz = __fadd2_rn(dz, hz);
    }
    const float2 r2 =
        __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)), __fmul2_rn(dz, dz));
    bool in0 = r2.x < rc2, in1 = r2.y < rc2;
    if (SELF) {
      in0 = in0 && (jsorted0 + t != isorted);
      in1 = in1 && (jsorted0 + t + 1 != isorted);
    }
    const float2 arg = __fmul2_rn(r2, g2);
    float2 e;
    e.x = in0 ? ex2_approx(arg.x) : 0.0f;
    e.y = in1 ? ex2_approx(arg.y) : 0.0f;
    A.eg = __fadd2_rn(A.eg, e);
    A.gx = __ffma2_rn(e, dx, A.gx);
    A.gy = __ffma2_rn(e, dy, A.gy);
    A.gz = __ffma2_rn(e, dz, A.gz);
    if (VIR) {
      const float2 ex = __fmul2_rn(e, dx), ey = __fmul2_rn(e, dy);
      A.wg[0] = __ffma2_rn(ex, dx, A.wg[0]);
      A.wg[1] = __ffma2_rn(ey, dy, A.wg[1]);
      A.wg[2] = __ffma2_rn(__fmul2_rn(e, dz), dz, A.wg[2]);
      A.wg[3] = __ffma2_rn(ex, dy, A.wg[3]);
      A.wg[4] = __ffma2_rn(ex, dz, A.wg[4]);
      A.wg[5] = __ffma2_rn(ey, dz, A.wg[5]);
    }
  }
}

// Gaussian core of a non-self neighbour cell without the in-cutoff test
// (SysDesc::gc_tail): every staged bead contributes, those beyond rc with a
// term below 1e-10 of the contact value (the staging cull keeps beads within
// rc + 1e-3 of the home cell's box, and pads sit far away: their term is 0).
// The image shift is applied to xi once, and r^2 is two fused
// multiply-adds: with no cutoff decision here, no rounding rule has to be
// followed.
template <bool VIR>
__device__ __forceinline__ void pair_core2_tail(const float *__restrict__ X,
                                                const float *__restrict__ Y,
                                                const float *__restrict__ Z, int n2,
                                                const float4 &xi, const PairSeg &sg, float gcc,
                                                PairAcc2 &A) {
  const float ox = __fsub_rn(sg.sh[0], xi.x), oy = __fsub_rn(sg.sh[1], xi.y),
              oz = __fsub_rn(sg.sh[2], xi.z);
  const float2 mx = make_float2(ox, ox), my = make_float2(oy, oy), mz = make_float2(oz, oz);
  const float2 g2 = make_float2(gcc, gcc);
#pragma unroll 4
  for (int t = 0; t < n2; t += 2) {
    const float2 dx = __fadd2_rn(*reinterpret_cast<const float2 *>(X + t), mx);
    const float2 dy = __fadd2_rn(*reinterpret_cast<const float2 *>(Y + t), my);
    const float2 dz = __fadd2_rn(*reinterpret_cast<const float2 *>(Z + t), mz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float2 arg = __fmul2_rn(r2, g2);
    float2 e;
    e.x = ex2_approx(arg.x);
    e.y = ex2_approx(arg.y);
    A.eg = __fadd2_rn(A.eg, e);
    A.gx = __ffma2_rn(e, dx, A.gx);
    A.gy = __ffma2_rn(e, dy, A.gy);
    A.gz = __ffma2_rn(e, dz, A.gz);
    if (VIR) {
      const float2 ex = __fmul2_rn(e, dx), ey = __fmul2_rn(e, dy);
      A.wg[0] = __ffma2_rn(ex, dx, A.wg[0]);
      A.wg[1] = __ffma2_rn(ey, dy, A.wg[1]);
      A.wg[2] = __ffma2_rn(__fmul2_rn(e, dz), dz, A.wg[2]);
      A.wg[3] = __ffma2_rn(ex, dy, A.wg[3]);
      A.wg[4] = __ffma2_rn(ex, dz, A.wg[4]);
      A.wg[5] = __ffma2_rn(ey, dz, A.wg[5]);
    }
  }
}

// The real-space term of a charged home bead with the candidates c0 + u, u
// a set bit of m (each in range by the neighbour rule, decided before): g
// and h from the system's table (TAB; r^2 a rounding above rc^2 takes the
// last interval a hair beyond its end) or evaluated directly, the energy,
// force and virial summed WITHOUT the home bead's own charge (elec_scale
// applies it once per home bead).  xs is the home bead's position minus the
// segment's image shift, so that d = x_j - xs; d and r^2 are recomputed here
// with fused operations: they set the values of the terms, not the
// decision, which followed the exact rounding rule.
template <bool VIR, bool TAB>
__device__ __forceinline__ void elec_hits(unsigned m, int c0, const float *__restrict__ X,
                                          const float *__restrict__ Y,
                                          const float *__restrict__ Z,
                                          const float *__restrict__ Q, float xsx, float xsy,
                                          float xsz, const SysDesc &S, PairAcc &A,
                                          const float4 *__restrict__ tab, float tab_scale,
                                          int tab_nm1) {
  // two hits per pass: two independent load-table-force chains in flight
  // (an odd last hit pairs with itself at zero charge)
  while (m) {
    const int u0 = 31 - __clz(m);  // highest set bit first
    m ^= 1u << u0;
    const bool two = m != 0u;
    const int u1 = two ? 31 - __clz(m) : u0;
    if (two) m ^= 1u << u1;
    const int ta = c0 + u0, tb = c0 + u1;
    const float dxa = X[ta] - xsx, dya = Y[ta] - xsy, dza = Z[ta] - xsz;
    const float dxb = X[tb] - xsx, dyb = Y[tb] - xsy, dzb = Z[tb] - xsz;
    const float r2a = fmaf(dxa, dxa, fmaf(dya, dya, dza * dza));
    const float r2b = fmaf(dxb, dxb, fmaf(dyb, dyb, dzb * dzb));
    float ga, ha, gb, hb;
    if (TAB) {
      real_gh_tab(tab, tab_scale, tab_nm1, r2a, ga, ha);
      real_gh_tab(tab, tab_scale, tab_nm1, r2b, gb, hb);
    } else {
      real_gh_direct(r2a, S.betaf, S.kappaf, S.ser_gf, S.ser_hf, ga, ha);
      real_gh_direct(r2b, S.betaf, S.kappaf, S.ser_gf, S.ser_hf, gb, hb);
    }
    const float qa = Q[ta], qb = two ? Q[tb] : 0.0f;
    A.ere = fmaf(qb, gb, fmaf(qa, ga, A.ere));
    const float fa = qa * ha, fb = qb * hb;
    A.fx = fmaf(fb, dxb, fmaf(fa, dxa, A.fx));
    A.fy = fmaf(fb, dyb, fmaf(fa, dya, A.fy));
    A.fz = fmaf(fb, dzb, fmaf(fa, dza, A.fz));
    if (VIR) {
      const float exa = fa * dxa, eya = fa * dya, exb = fb * dxb, eyb = fb * dyb;
      A.we[0] = fmaf(exb, dxb, fmaf(exa, dxa, A.we[0]));
      A.we[1] = fmaf(eyb, dyb, fmaf(eya, dya, A.we[1]));
      A.we[2] = fmaf(fb * dzb, dzb, fmaf(fa * dza, dza, A.we[2]));
      A.we[3] = fmaf(exb, dyb, fmaf(exa, dya, A.we[3]));
      A.we[4] = fmaf(exb, dzb, fmaf(exa, dza, A.we[4]));
      A.we[5] = fmaf(eyb, dzb, fmaf(eya, dza, A.we[5]));
    }
  }
}

// The home bead's charge on its real-space sums (after its last elec_hits).
template <bool VIR>
__device__ __forceinline__ void elec_scale(PairAcc &A, float qi) {
  A.ere *= qi;
  A.fx *= qi;
  A.fy *= qi;
  A.fz *= qi;
  if (VIR)
#pragma unroll
    for (int k = 0; k < 6; ++k) A.we[k] *= qi;
}

// Real-space electrostatics of a charged i over the staged charged and image
// candidates [t0, t1) held as coordinate and charge arrays (t0, t1 even):
// the in-cutoff test runs on two candidates per packed FP32x2 instruction
// (the rounding of the neighbour rule, as in pair_core2) and sets one bit
// per hit, 32 candidates at a time (32-bit masks: no 64-bit shifts or bit
// scans); elec_hits evaluates the set bits.  jsorted0 + t is candidate t's
// sorted index (self segment, staged whole and in order).  TAB: g and h
// from the system's table (tab, its scale and last interval nm1), else
// evaluated directly.
template <bool SHIFT, bool SELF, bool VIR, bool TAB>
__device__ __forceinline__ void pair_elec2(const float *__restrict__ X, int t0, int t1,
                                           int jsorted0, const float4 &xi, int isorted,
                                           const PairSeg &sg, const SysDesc &S, float rc2,
                                           PairAcc &A, const float4 *__restrict__ tab,
                                           float tab_scale, int tab_nm1) {
  // y, z and charge arrays follow x at fixed strides (one base register)
  const float *__restrict__ Y = X + kPkCapQ;
  const float *__restrict__ Z = X + 2 * kPkCapQ;
  const float *__restrict__ Q = X + 3 * kPkCapQ;
  if (xi.w == 0.0f) return;
  const float2 mx = make_float2(-xi.x, -xi.x), my = make_float2(-xi.y, -xi.y),
               mz = make_float2(-xi.z, -xi.z);
  const float2 hx = make_float2(sg.sh[0], sg.sh[0]), hy = make_float2(sg.sh[1], sg.sh[1]),
               hz = make_float2(sg.sh[2], sg.sh[2]);
  for (int c0 = t0; c0 < t1; c0 += 32) {
    const int cn = min(32, t1 - c0);
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
    elec_hits<VIR, TAB>(m, c0, X, Y, Z, Q, SHIFT ? xi.x - sg.sh[0] : xi.x,
                        SHIFT ? xi.y - sg.sh[1] : xi.y, SHIFT ? xi.z - sg.sh[2] : xi.z, S, A, tab,
                        tab_scale, tab_nm1);
  }
}

// Debug only: in-cutoff images seen by a neutral i (or by every i when
// every_i is set) -- no interaction of their own here, but part of the
// neighbour set.
template <bool SHIFT>
__device__ __forceinline__ void pair_dump_images(const float4 *__restrict__ J, int t0, int t1,
                                                 int jsorted0, const float4 &xi, int isorted,
                                                 const PairSeg &sg, float rc2, const Pool &P,
                                                 int s, bool every_i = false) {
  if (!every_i && xi.w != 0.0f) return;
  for (int t = t0; t < t1; ++t) {
    float dx, dy, dz;
    if (!(pair_r2<SHIFT>(J[t], xi, sg, dx, dy, dz) < rc2)) continue;
    unsigned long long k = atomicAdd(&P.acc[(long long)s * kNacc + ACC_NPAIR], 1ull);
    if ((long long)k < P.dbg_cap) {
      P.dbg_triples[3 * k + 0] = P.sorted_idx[isorted];
      P.dbg_triples[3 * k + 1] = P.sorted_idx[jsorted0 + t];
      P.dbg_triples[3 * k + 2] = sg.code;
    }
  }
}

// Process one staged segment (the bead ranges of one neighbour cell),
// candidates clipped to [t0, t1): [0, a) images, [a, b) charged reals,
// [b, n) neutral reals.
template <bool VIR, bool DBG>
__device__ __forceinline__ void pair_segment(const float4 *J, int t0, int t1, int jsorted0,
                                             const PairSeg &sg, bool anyq, const float4 &xi,
                                             int isorted, const SysDesc &S, float rc2, float gcc,
                                             PairAcc &A, const Pool &P, int s) {
  const int a0 = max(t0, min(t1, sg.a)), b0 = max(t0, min(t1, sg.b));
#define GCME_SEG(SHIFT, SELF)                                                               \
  pair_core<SHIFT, SELF, VIR, DBG>(J, a0, t1, jsorted0, xi, isorted, sg, rc2, gcc, A, P, s);  \
  if (anyq)                                                                                   \
    pair_elec<SHIFT, SELF, VIR, DBG>(J, t0, b0, a0, jsorted0, xi, isorted, sg, S, rc2, A, P,  \
                                     s);                                                      \
  if (DBG) pair_dump_images<SHIFT>(J, t0, a0, jsorted0, xi, isorted, sg, rc2, P, s);
  if (sg.self) {
    GCME_SEG(false, true)
  } else if (sg.shifted) {
    GCME_SEG(true, false)
  } else {
    GCME_SEG(false, false)
  }
#undef GCME_SEG
}

// Write back one lane's partial sums: fixed-point forces, warp-reduced
// FP64 energies (core, electrostatics) and virial.
template <bool VIR, bool MT = false>
__device__ __forceinline__ void pair_write(const Pool &P, const SysDesc &S, int s, bool valid,
                                           int i, const PairAcc &A) {
  // FP32 throughout (the FP64 pipe is a small fraction of the FP32 rate):
  // per-warp sums of FP32 partials, then 64-bit fixed point
  const float cg = MT ? 1.0f : S.gc_forcef;
  const float lb = S.lbf;
  if (valid) {
    const int orig = P.sorted_idx[i];
    atomic_add_fixed_f(force_ptr(P, S, orig, 0), -(cg * A.gx + lb * A.fx), (float)kFScale);
    atomic_add_fixed_f(force_ptr(P, S, orig, 1), -(cg * A.gy + lb * A.fy), (float)kFScale);
    atomic_add_fixed_f(force_ptr(P, S, orig, 2), -(cg * A.gz + lb * A.fz), (float)kFScale);
  }
  // each lane's partial in fixed point first, then exact integer sums
  const long long eg = warp_sum(valid ? efix((MT ? 0.5f : S.gc_halfpref) * A.eg) : 0ll);
  const long long er = warp_sum(valid ? efix(S.lb_half * A.ere) : 0ll);
  unsigned long long *acc = P.acc + (long long)s * kNacc;
  if ((threadIdx.x & 31) == 0) {
    if (eg) atomicAdd(acc + ACC_GC, (unsigned long long)eg);
    if (er) atomicAdd(acc + ACC_REAL, (unsigned long long)er);
  }
  if (VIR) {
    // W_ab = 1/2 sum_visits fs d_a d_b  with fs = (3/s) u or lB qq h
    const float c1 = MT ? 0.5f : 0.5f * S.gc_forcef, c2 = S.lb_half;
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const long long v = warp_sum(valid ? efix(c1 * A.wg[map[k]] + c2 * A.we[map[k]]) : 0ll);
      if ((threadIdx.x & 31) == 0) atomicAdd(P.vacc + (long long)s * 9 + k, (unsigned long long)v);
    }
  }
}

// One staged range [t0, t1) of a segment, for one role: the core warps
// evaluate the Gaussian core over the real beads (and, in debug mode, list
// the in-cutoff images); the electrostatics warp evaluates the real-space
// term of its charged home beads over the charged and image beads.
template <bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void pair_role_range(bool core_role, const float4 *J, int t0, int t1,
                                                const PairSeg &sg, const float4 &xi, int i,
                                                const SysDesc &S, float rc2, float gcc,
                                                PairAcc &A, const Pool &P, int s,
                                                const PairTab *row = nullptr,
                                                const unsigned char *tj = nullptr) {
  const int a0 = max(t0, min(t1, sg.a)), b0 = max(t0, min(t1, sg.b));
#define GCME_ROLE(SHIFT, SELF)                                                                    \
  if (core_role) {                                                                                \
    pair_core<SHIFT, SELF, VIR, DBG, MT>(J, a0, t1, sg.beg, xi, i, sg, rc2, gcc, A, P, s, row,    \
                                         tj);                                                     \
    if (DBG) pair_dump_images<SHIFT>(J, t0, a0, sg.beg, xi, i, sg, rc2, P, s, true);              \
  } else {                                                                                        \
    pair_elec<SHIFT, SELF, VIR, false, MT>(J, t0, b0, 0, sg.beg, xi, i, sg, S, rc2, A, P, s, row, \
                                           tj);                                                   \
  }
  if (sg.self) {
    GCME_ROLE(false, true)
  } else if (sg.shifted) {
    GCME_ROLE(true, false)
  } else {
    GCME_ROLE(false, false)
  }
#undef GCME_ROLE
}

// Cell (x, y, z) of system S, each coordinate at most one period outside
// [0, nc), as a segment: its sorted range and class boundaries, image code
// and periodic shift; self = 0.
__device__ __forceinline__ PairSeg cell_segment(const Pool &P, const SysDesc &S, int x, int y,
                                                int z) {
  const int ncv[3] = {S.nc[0], S.nc[1], S.nc[2]};
  const int u[3] = {x, y, z};
  int v[3], nn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nn[a] = floor_div(u[a], ncv[a]);
    v[a] = u[a] - nn[a] * ncv[a];
  }
  const long long cg = S.cell_off + v[0] + ncv[0] * (v[1] + ncv[1] * v[2]);
  PairSeg g;
  g.beg = P.cell_start[cg];
  g.n = P.cell_start[cg + 1] - g.beg;
  g.a = P.cell_nimg[cg];
  g.b = P.cell_nq[cg];
  g.code = (nn[0] + 1) + 3 * (nn[1] + 1) + 9 * (nn[2] + 1);
#pragma unroll
  for (int a = 0; a < 3; ++a) g.sh[a] = (float)nn[a] * S.boxf[a];
  g.self = 0;
  g.shifted = (nn[0] != 0 || nn[1] != 0 || nn[2] != 0);
  g.soff = 0;
  g.qoff = 0;
  return g;
}

// Segment k of a work item of the 27-cell kernel with one home cell (split
// 3: the 9 cells at dz = part - 1; split 9: the 3 cells along x at dy, dz =
// part % 3 - 1, part / 3 - 1), with its periodic shift.
__device__ __forceinline__ PairSeg item_segment(const Pool &P, const SysDesc &S, int cloc,
                                                int part, int k) {
  const int split = S.pair_split;
  const int nc0 = S.nc[0], nc1 = S.nc[1];
  const int cx = cloc % nc0, cy = (cloc / nc0) % nc1, cz = cloc / (nc0 * nc1);
  const int dzo = (split == 3 ? part : part / 3) - 1;
  const int dxo = k % 3 - 1, dyo = split == 3 ? k / 3 - 1 : part % 3 - 1;
  PairSeg g = cell_segment(P, S, cx + dxo, cy + dyo, cz + dzo);
  g.self = (dxo == 0 && dyo == 0 && dzo == 0);
  return g;
}

// The home cells of a CTA work item: x0 .. x0 + nhome - 1 of the x-row
// (y, z), and its part.  SysDesc::pair_group = G > 1 (split 9 only): code =
// (row group) * 9 + part with ceil(nc_x / G) groups of G consecutive home
// cells per row, the last one shorter; its segments are the nhome + 2
// cells x0 - 1 .. x0 + nhome of the row (y + dy, z + dz), distinct because
// nc_x >= G + 2, and each home cell pairs with the three of them around
// it; code < 0: the single home cell -1 - code = cell * 9 + part (the
// items that end the list).  G = 1: code = cell * split + part.
struct ItemCells {
  int x0, y, z, nhome, part;
};
__device__ __forceinline__ ItemCells item_cells(const SysDesc &S, int code) {
  const int G = S.pair_group > 1 ? S.pair_group : 1;
  ItemCells c;
  if (G == 1 || code < 0) {
    const int split = S.pair_split;
    if (code < 0) code = -1 - code;
    const int cloc = code / split;
    c.part = code % split;
    c.x0 = cloc % S.nc[0];
    c.y = (cloc / S.nc[0]) % S.nc[1];
    c.z = cloc / (S.nc[0] * S.nc[1]);
    c.nhome = 1;
  } else {
    const int ngx = (S.nc[0] + G - 1) / G;
    const int gi = code / 9;
    c.part = code % 9;
    c.x0 = (gi % ngx) * G;
    c.y = (gi / ngx) % S.nc[1];
    c.z = gi / (ngx * S.nc[1]);
    c.nhome = min(G, S.nc[0] - c.x0);
  }
  return c;
}

// One home cell of a work item by the whole CTA (code = cell * split +
// part): the home cell and 9 (split 3) or 3 (split 9) of its 27 neighbour
// cells.  Shared memory: sj[kPairCap], seg[9], s_total[1].  Ends with a
// barrier.
//
// Warp roles: warps 0 .. W-2 take the home cell's real beads 32 per warp
// (Gaussian core over the staged real beads); warp W-1 takes its charged
// real beads (real-space electrostatics over the staged charged and image
// beads).  The two kinds of work run concurrently instead of one after the
// other in the warp that holds the charged beads.
//
// MT: stj[kPairCap] (species of the staged beads) and stab[nt * nt] (the
// system's pair table) in shared memory as well.
template <bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void dev_pair_f32_cell(const Pool &P, int s, int code, float4 *sj,
                                                  PairSeg *seg, int *s_total_p,
                                                  unsigned char *stj, PairTab *stab) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int ncore = (blockDim.x >> 5) - 1;  // core warps
  const bool core_role = warp < ncore;
  int &s_total = *s_total_p;
  // with neighbour lists, only the systems whose lists overflowed come here
  if (P.list_ovf && !P.list_ovf[s]) {
    __syncthreads();
    return;
  }
  const SysDesc &S = P.sys[s];
  const int nt = MT ? S.ntypes : 1;
  if (MT)
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) stab[k] = P.ptab[S.tab_off + k];
  // split 3: item = (cell, dz), 9 neighbour cells; split 9: item =
  // (cell, dy, dz), 3 neighbour cells along x
  const int split = S.pair_split;
  const int cloc = code / split;
  const int part = code % split;
  const int nseg = 27 / split;
  const int dzo = (split == 3 ? part : part / 3) - 1;
  const int dyf = split == 3 ? -2 : part % 3 - 1;  // fixed dy (split 9)
  const int nc0 = S.nc[0], nc1 = S.nc[1], nc2 = S.nc[2];
  const int cx = cloc % nc0, cy = (cloc / nc0) % nc1, cz = cloc / (nc0 * nc1);
  const long long hg = S.cell_off + cloc;
  const int hbeg = P.cell_start[hg], hend = P.cell_start[hg + 1];
  const int himg = P.cell_nimg[hg], hq = P.cell_nq[hg];
  const int rbeg = hbeg + himg;  // first real home bead; charged reals end at hbeg + hq
  if (tid < nseg) {
    const int dxo = tid % 3 - 1, dyo = split == 3 ? tid / 3 - 1 : dyf;
    const int u[3] = {cx + dxo, cy + dyo, cz + dzo};
    const int ncv[3] = {nc0, nc1, nc2};
    int v[3], nn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      nn[a] = floor_div(u[a], ncv[a]);
      v[a] = u[a] - nn[a] * ncv[a];
    }
    const long long cg = S.cell_off + v[0] + nc0 * (v[1] + nc1 * v[2]);
    PairSeg g;
    g.beg = P.cell_start[cg];
    g.n = P.cell_start[cg + 1] - g.beg;
    g.a = P.cell_nimg[cg];
    g.b = P.cell_nq[cg];
    g.code = (nn[0] + 1) + 3 * (nn[1] + 1) + 9 * (nn[2] + 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) g.sh[a] = (float)nn[a] * S.boxf[a];
    g.self = (dxo == 0 && dyo == 0 && dzo == 0);
    g.shifted = (nn[0] != 0 || nn[1] != 0 || nn[2] != 0);
    g.soff = 0;
    seg[tid] = g;
  }
  __syncthreads();
  if (tid == 0) {
    int off = 0;
    for (int k = 0; k < nseg; ++k) {
      seg[k].soff = off;
      off += seg[k].n;
    }
    s_total = off;
  }
  __syncthreads();
  const bool fits = s_total <= kPairCap;
  if (fits) {
    for (int k = 0; k < nseg; ++k) {
      const PairSeg &g = seg[k];
      for (int t = tid; t < g.n; t += blockDim.x) {
        sj[g.soff + t] = P.xyzq_s[g.beg + t];
        if (MT) stj[g.soff + t] = P.type_s[g.beg + t];
      }
    }
    __syncthreads();
  }
  const float rc2 = S.rc2f;
  const float gcc = S.gc_c2f;
  // home-bead chunks of each role; the chunk loop runs the same number of
  // times on every warp so that the staging barriers of large cells match
  const int nreal = hend - rbeg, nqr = hbeg + hq - rbeg;
  const int ncore_chunks = (nreal + 32 * ncore - 1) / (32 * ncore);
  const int nel_chunks = (nqr + 31) / 32;
  const int nchunk = max(ncore_chunks, nel_chunks);
  for (int c = 0; c < nchunk; ++c) {
    int i;
    bool valid;
    if (core_role) {
      i = rbeg + c * 32 * ncore + tid;
      valid = i < hend;
    } else {
      i = rbeg + c * 32 + lane;
      valid = i < hbeg + hq;
    }
    const float4 xi = valid ? P.xyzq_s[i] : make_float4(1e30f, 1e30f, 1e30f, 0.0f);
    const PairTab *row = MT ? stab + nt * (valid ? (int)P.type_s[i] : 0) : nullptr;
    const bool busy = __any_sync(0xffffffffu, valid);
    PairAcc A;
    A.eg = A.ere = A.gx = A.gy = A.gz = A.fx = A.fy = A.fz = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) A.wg[k] = A.we[k] = 0.0f;
    if (fits) {
      if (busy)
        for (int k = 0; k < nseg; ++k) {
          const PairSeg g = seg[k];
          pair_role_range<VIR, DBG, MT>(core_role, sj + g.soff, 0, g.n, g, xi, i, S, rc2, gcc, A,
                                        P, s, row, MT ? stj + g.soff : nullptr);
        }
    } else {
      for (int k = 0; k < nseg; ++k) {
        const PairSeg g = seg[k];
        for (int c0 = 0; c0 < g.n; c0 += kPairCap) {
          const int c1 = min(g.n, c0 + kPairCap);
          __syncthreads();
          for (int t = c0 + tid; t < c1; t += blockDim.x) {
            sj[t - c0] = P.xyzq_s[g.beg + t];
            if (MT) stj[t - c0] = P.type_s[g.beg + t];
          }
          __syncthreads();
          // ranges are in segment coordinates; shift the staged base
          if (busy)
            pair_role_range<VIR, DBG, MT>(core_role, sj - c0, c0, c1, g, xi, i, S, rc2, gcc, A, P,
                                          s, row, MT ? stj - c0 : nullptr);
        }
      }
    }
    if (busy) pair_write<VIR, MT>(P, S, s, valid, i, A);
  }
  __syncthreads();
}

// One work item (system wk.x, code wk.y) on the scalar path: each of its
// home cells in turn (one unless SysDesc::pair_group > 1).  Ends with a
// barrier.
template <bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void dev_pair_f32_item(const Pool &P, int2 wk, float4 *sj,
                                                  PairSeg *seg, int *s_total,
                                                  unsigned char *stj = nullptr,
                                                  PairTab *stab = nullptr) {
  const SysDesc &S = P.sys[wk.x];
  if (S.pair_group <= 1 || wk.y < 0) {  // one home cell (code -1 - code' ending a group list)
    dev_pair_f32_cell<VIR, DBG, MT>(P, wk.x, wk.y < 0 ? -1 - wk.y : wk.y, sj, seg, s_total, stj,
                                    stab);
    return;
  }
  const ItemCells c = item_cells(S, wk.y);
  for (int h = 0; h < c.nhome; ++h) {
    const int cloc = c.x0 + h + S.nc[0] * (c.y + S.nc[1] * c.z);
    dev_pair_f32_cell<VIR, DBG, MT>(P, wk.x, cloc * 9 + c.part, sj, seg, s_total, stj, stab);
  }
}
template <bool VIR, bool DBG, bool MT = false>
__device__ __forceinline__ void dev_pair_f32_item(const Pool &P, const int2 *work, int w,
                                                  float4 *sj, PairSeg *seg, int *s_total,
                                                  unsigned char *stj = nullptr,
                                                  PairTab *stab = nullptr) {
  dev_pair_f32_item<VIR, DBG, MT>(P, work[w], sj, seg, s_total, stj, stab);
}


// Packed items (one species, no debug dump), in three parts shared by the
// CTA kernel and the pipelined kernel: the staged-array layout and offsets,
// the culled staging of one segment by one warp, and the evaluation by the
// role warps.  The core warps run pair_core2 over coordinate arrays, the
// electrostatics warps (1 to 3, SysDesc::pair_nelec) pair_elec2 over the
// staged charged and image beads, each warp a contiguous part of every
// cell's candidates and each writing its partial sums (fixed-point atomics
// add them).

// Offsets of each segment in the packed arrays (real beads and charged /
// image beads, each segment even-padded); returns false when the item's
// beads exceed the capacities.  One thread.
__device__ __forceinline__ bool pk_offsets(PairSeg *seg, int nseg, int *s_tot) {
  int off = 0, qoff = 0;
  for (int k = 0; k < nseg; ++k) {
    seg[k].soff = off;
    seg[k].qoff = qoff;
    off += (seg[k].n - seg[k].a + 1) & ~1;
    qoff += (seg[k].b + 1) & ~1;
  }
  s_tot[0] = off;
  s_tot[1] = qoff;
  return off <= kPkCap && qoff <= kPkCapQ;
}

// Staging of segment g by one warp: only the candidates within rc (+1e-3) of
// the home cell's box [hlo, hhi] can be within rc of a home bead, so the
// others are dropped (about 30 % of the 27 cells' beads at cells of side
// ~rc), keeping order; the home cell itself is staged whole, in sorted order
// (its self-pair test uses the sorted index).  Sets g.nk and g.bk.
__device__ __forceinline__ void pk_stage_segment(const Pool &P, PairSeg &g, const float hlo[3],
                                                 const float hhi[3], float cut2,
                                                 unsigned char *smem, int lane) {
  float *sx = reinterpret_cast<float *>(smem);
  float *sy = sx + kPkCap;
  float *sz = sy + kPkCap;
  float *qx = sz + kPkCap, *qy = qx + kPkCapQ, *qz = qy + kPkCapQ, *qq = qz + kPkCapQ;
  const unsigned lt = (1u << lane) - 1u;
  const float4 far = make_float4(1e30f, 1e30f, 1e30f, 0.0f);  // pad: far away
  auto near_home = [&](const float4 &v) {
    const float e[3] = {v.x + g.sh[0], v.y + g.sh[1], v.z + g.sh[2]};
    float d2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float d = fmaxf(0.0f, fmaxf(hlo[a] - e[a], e[a] - hhi[a]));
      d2 = fmaf(d, d, d2);
    }
    return d2 <= cut2;
  };
  const bool all = g.self;
  const int nr = g.n - g.a;
  int kept = 0;
  for (int t0 = 0; t0 < nr; t0 += 128) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + 32 * u + lane;
      v[u] = t < nr ? P.xyzq_s[g.beg + g.a + t] : far;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + 32 * u + lane;
      const bool keep = t < nr && (all || near_home(v[u]));
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int p = g.soff + kept + __popc(m & lt);
        sx[p] = v[u].x;
        sy[p] = v[u].y;
        sz[p] = v[u].z;
      }
      kept += __popc(m);
    }
  }
  if ((kept & 1) && lane == 0) {
    sx[g.soff + kept] = far.x;
    sy[g.soff + kept] = far.y;
    sz[g.soff + kept] = far.z;
  }
  int keptq = 0;
  for (int t0 = 0; t0 < g.b; t0 += 32) {
    const int t = t0 + lane;
    const float4 v = t < g.b ? P.xyzq_s[g.beg + t] : far;
    const bool keep = t < g.b && (all || near_home(v));
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int p = g.qoff + keptq + __popc(m & lt);
      qx[p] = v.x;
      qy[p] = v.y;
      qz[p] = v.z;
      qq[p] = v.w;
    }
    keptq += __popc(m);
  }
  if ((keptq & 1) && lane == 0) {
    qx[g.qoff + keptq] = far.x;
    qy[g.qoff + keptq] = far.y;
    qz[g.qoff + keptq] = far.z;
    qq[g.qoff + keptq] = 0.0f;
  }
  if (lane == 0) {
    g.nk = kept;
    g.bk = keptq;
  }
}

// The box of the item's home cells x0 .. x0 + nhome - 1 of row (y, z), for
// the staging cull.
__device__ __forceinline__ void pk_home_box(const SysDesc &S, const ItemCells &c, float hlo[3],
                                            float hhi[3]) {
  const int lo[3] = {c.x0, c.y, c.z}, w[3] = {c.nhome, 1, 1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hlo[a] = (float)lo[a] * S.cside[a];
    hhi[a] = hlo[a] + (float)w[a] * S.cside[a];
  }
}

// Evaluation of one staged item by the role warps: rt is the thread's index
// among the nrole threads that take part (warps 0 .. ncore-1 of them core,
// the last nelec electrostatics).  Warp-synchronous per warp; no CTA barrier.
//
// GRP (items of several home cells): the self segment is seg[selfk] (each
// home cell's own among the staged cells around it); else the one flagged
// self.
//
// DYN (SysDesc::pair_nelec = -e): the item's work as tasks that every warp
// takes from the shared-memory counter *s_task (zero before the item):
// first the Gaussian-core chunks of 32 home beads (all real candidates),
// then each chunk of 32 charged home beads in e parts of the charged
// candidates.  A task computes what the role warp of the static split with
// e electrostatics warps computes for it, so the sums are the same; the
// warps stay busy when a cell needs more core chunks than there are core
// warps, or more than one electrostatics chunk.
template <bool VIR, bool GRP = false, bool DYN = false>
__device__ __forceinline__ void pk_compute(const Pool &P, const SysDesc &S, int s, int hbeg,
                                           int hend, int himg, int hq, const PairSeg *seg,
                                           int nseg, int selfk, const unsigned char *smem,
                                           int rt, int nrole, int *s_task = nullptr) {
  const float *sx = reinterpret_cast<const float *>(smem);
  const float *sy = sx + kPkCap;
  const float *sz = sy + kPkCap;
  const float *qx = sz + kPkCap;
  const int warp = rt >> 5, lane = rt & 31;
  const int nelec = min(max(S.pair_nelec, 1), 3);
  const int ncore = (nrole >> 5) - nelec;
  const bool core_role = warp < ncore;
  const int ew = warp - ncore;
  const int rbeg = hbeg + himg;
  const float rc2 = S.rc2f, gcc = S.gc_c2f;
  const int nreal = hend - rbeg, nqr = hbeg + hq - rbeg;
  // one chunk of home beads of one role (crole: the Gaussian core, else the
  // electrostatics, part ep of nep): this thread's home bead i
  auto task = [&](bool crole, int i, bool valid, int ep, int nep) {
    const float4 xi = valid ? P.xyzq_s[i] : make_float4(1e30f, 1e30f, 1e30f, 0.0f);
    const bool busy = __any_sync(0xffffffffu, valid);
    PairAcc A;
    A.eg = A.ere = A.gx = A.gy = A.gz = A.fx = A.fy = A.fz = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) A.wg[k] = A.we[k] = 0.0f;
    if (busy) {
      if (crole) {
        PairAcc2 B;
        B.eg = B.gx = B.gy = B.gz = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < 6; ++k) B.wg[k] = make_float2(0.0f, 0.0f);
        const bool tail = S.gc_tail != 0;
        for (int k = 0; k < nseg; ++k) {
          const PairSeg g = seg[k];
          const int n2 = (g.nk + 1) & ~1;
          const float *X = sx + g.soff, *Y = sy + g.soff, *Z = sz + g.soff;
          const int j0 = g.beg + g.a;
          if (GRP ? k == selfk : g.self != 0)
            pair_core2<false, true, VIR>(X, Y, Z, n2, j0, xi, i, g, rc2, gcc, B);
          else if (tail)
            pair_core2_tail<VIR>(X, Y, Z, n2, xi, g, gcc, B);
          else if (g.shifted)
            pair_core2<true, false, VIR>(X, Y, Z, n2, j0, xi, i, g, rc2, gcc, B);
          else
            pair_core2<false, false, VIR>(X, Y, Z, n2, j0, xi, i, g, rc2, gcc, B);
        }
        A.eg = B.eg.x + B.eg.y;
        A.gx = B.gx.x + B.gx.y;
        A.gy = B.gy.x + B.gy.y;
        A.gz = B.gz.x + B.gz.y;
        if (VIR)
#pragma unroll
          for (int k = 0; k < 6; ++k) A.wg[k] = B.wg[k].x + B.wg[k].y;
      } else {
        // the system's real-space table (tab_nm1 < 0: none)
        const float4 *tab = P.rtab + S.rtab_off;
        const float tab_scale = S.rtab_scale;
        const int tab_nm1 = S.rtab_n - 1;
        for (int k = 0; k < nseg; ++k) {
          const PairSeg g = seg[k];
          // this warp's part of the (even-padded) candidates, on even bounds
          const int np2 = (g.bk + 1) >> 1;
          const int lo = 2 * (np2 * ep / nep), hi = 2 * (np2 * (ep + 1) / nep);
          const float *X = qx + g.qoff;
          if (tab_nm1 < 0) {  // no table (very small smearing radius)
            if (GRP ? k == selfk : g.self != 0)
              pair_elec2<false, true, VIR, false>(X, lo, hi, g.beg, xi, i, g, S, rc2, A,
                                                  tab, tab_scale, tab_nm1);
            else if (g.shifted)
              pair_elec2<true, false, VIR, false>(X, lo, hi, g.beg, xi, i, g, S, rc2, A,
                                                  tab, tab_scale, tab_nm1);
            else
              pair_elec2<false, false, VIR, false>(X, lo, hi, g.beg, xi, i, g, S, rc2,
                                                   A, tab, tab_scale, tab_nm1);
          } else if (GRP ? k == selfk : g.self != 0) {
            pair_elec2<false, true, VIR, true>(X, lo, hi, g.beg, xi, i, g, S, rc2, A,
                                               tab, tab_scale, tab_nm1);
          } else if (g.shifted) {
            pair_elec2<true, false, VIR, true>(X, lo, hi, g.beg, xi, i, g, S, rc2, A,
                                               tab, tab_scale, tab_nm1);
          } else {
            pair_elec2<false, false, VIR, true>(X, lo, hi, g.beg, xi, i, g, S, rc2, A,
                                                tab, tab_scale, tab_nm1);
          }
        }
        elec_scale<VIR>(A, xi.w);
      }
      pair_write<VIR>(P, S, s, valid, i, A);
    }
  };
  if (DYN) {
    const int ne = min(max(-S.pair_nelec, 1), 3);  // electrostatics parts per chunk
    const int nc = (nreal + 31) >> 5, ntask = nc + ne * ((nqr + 31) >> 5);
    int t = lane == 0 ? atomicAdd(s_task, 1) : 0;
    t = __shfl_sync(0xffffffffu, t, 0);
    while (t < ntask) {
      const bool core_role = t < nc;
      const int c = core_role ? t : (t - nc) / ne;
      const int i = rbeg + 32 * c + lane;
      task(core_role, i, i < (core_role ? hend : hbeg + hq), core_role ? 0 : (t - nc) - c * ne,
           ne);
      t = lane == 0 ? atomicAdd(s_task, 1) : 0;
      t = __shfl_sync(0xffffffffu, t, 0);
    }
    return;
  }
  const int ncore_chunks = (nreal + 32 * ncore - 1) / (32 * ncore);
  const int nel_chunks = (nqr + 31) / 32;
  const int nchunk = max(ncore_chunks, nel_chunks);
  for (int c = 0; c < nchunk; ++c) {
    if (core_role) {
      const int i = rbeg + c * 32 * ncore + rt;
      task(true, i, i < hend, ew, nelec);
    } else {
      const int i = rbeg + c * 32 + lane;
      task(false, i, i < hbeg + hq, ew, nelec);
    }
  }
}

// Packed variant of dev_pair_f32_item, one CTA per item of one home cell
// (SysDesc::pair_group 1): items whose beads exceed the packed capacities
// take the scalar path.  smem: kPairSmemBytes; seg[kItemSegs]; s_tot[2].
// Ends with a barrier.
//
// DYN: the warps take the item's tasks from s_task[0] (pk_compute).
template <bool VIR, bool DYN = false>
__device__ __forceinline__ void dev_pair_f32_item_pk(const Pool &P, const int2 *work, int w,
                                                     unsigned char *smem, PairSeg *seg,
                                                     int *s_tot, int *s_task = nullptr) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int s = work[w].x;
  const int code = work[w].y;
  if (P.list_ovf && !P.list_ovf[s]) {
    __syncthreads();
    return;
  }
  if (DYN && tid == 0) s_task[0] = 0;
  const SysDesc &S = P.sys[s];
  const int split = S.pair_split;
  const int cloc = code / split, part = code % split;
  const int nseg = 27 / split;
  const long long hg = S.cell_off + cloc;
  const int hbeg = P.cell_start[hg], hend = P.cell_start[hg + 1];
  const int himg = P.cell_nimg[hg], hq = P.cell_nq[hg];
  if (tid < nseg) seg[tid] = item_segment(P, S, cloc, part, tid);
  __syncthreads();
  if (tid == 0) pk_offsets(seg, nseg, s_tot);
  __syncthreads();
  if (s_tot[0] > kPkCap || s_tot[1] > kPkCapQ) {
    dev_pair_f32_cell<VIR, false, false>(P, s, code, reinterpret_cast<float4 *>(smem), seg,
                                         s_tot, nullptr, nullptr);
    return;
  }
  {
    float hlo[3], hhi[3];
    ItemCells ic;
    ic.x0 = cloc % S.nc[0];
    ic.y = (cloc / S.nc[0]) % S.nc[1];
    ic.z = cloc / (S.nc[0] * S.nc[1]);
    ic.nhome = 1;
    pk_home_box(S, ic, hlo, hhi);
    const int nwarp = blockDim.x >> 5;
    for (int k = warp; k < nseg; k += nwarp)
      pk_stage_segment(P, seg[k], hlo, hhi, S.cull2, smem, lane);
  }
  __syncthreads();
  pk_compute<VIR, false, DYN>(P, S, s, hbeg, hend, himg, hq, seg, nseg, -1, smem, tid,
                              blockDim.x, s_task);
  __syncthreads();
}

// The scalar path for a packed item over capacity, out of line: its
// registers are its own, so that the rare fallback does not raise the
// packed path's register pressure.
template <bool VIR>
__device__ __noinline__ void pair_item_scalar(const Pool &P, int2 wk, float4 *sj, PairSeg *seg,
                                              int *s_tot) {
  dev_pair_f32_item<VIR, false, false>(P, wk, sj, seg, s_tot);
}

// The same for items of several home cells (SysDesc::pair_group > 1 in some
// system; systems with pair_group 1 take their single home cell here too):
// an item stages the nhome + 2 cells of its row once, culled against the
// box of all its home cells (the home cells themselves staged whole in the
// centre part), and evaluates each home cell over the three staged cells
// around it.  seg[kItemSegs]: staged segments from 0, the home cells from 9.
//
// DYN: the warps take the tasks of home cell h from s_task[h] (pk_compute).
template <bool VIR, bool DYN = false>
__device__ __forceinline__ void dev_pair_f32_item_grp(const Pool &P, const int2 *work, int w,
                                                      unsigned char *smem, PairSeg *seg,
                                                      int *s_tot, int *s_task = nullptr) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int s = work[w].x;
  const int code = work[w].y;
  if (P.list_ovf && !P.list_ovf[s]) {
    __syncthreads();
    return;
  }
  if (DYN && tid < 3) s_task[tid] = 0;
  const SysDesc &S = P.sys[s];
  const int split = S.pair_split;
  const ItemCells ic = item_cells(S, code);
  const int nseg = split == 3 ? 9 : ic.nhome + 2;
  const bool centre = ic.part == (split == 3 ? 1 : 4);
  if (tid < nseg) {
    if (ic.nhome == 1) {
      seg[tid] = item_segment(P, S, ic.x0 + S.nc[0] * (ic.y + S.nc[1] * ic.z), ic.part, tid);
    } else {
      PairSeg g = cell_segment(P, S, ic.x0 - 1 + tid, ic.y + ic.part % 3 - 1,
                               ic.z + ic.part / 3 - 1);
      g.self = centre && tid >= 1 && tid <= ic.nhome;  // a home cell: staged whole
      seg[tid] = g;
    }
  } else if (tid >= 32 && tid < 32 + ic.nhome) {
    seg[9 + tid - 32] = cell_segment(P, S, ic.x0 + tid - 32, ic.y, ic.z);
  }
  __syncthreads();
  if (tid == 0) pk_offsets(seg, nseg, s_tot);
  __syncthreads();
  if (s_tot[0] > kPkCap || s_tot[1] > kPkCapQ) {
    pair_item_scalar<VIR>(P, work[w], reinterpret_cast<float4 *>(smem), seg, s_tot);
    return;
  }
  {
    float hlo[3], hhi[3];
    pk_home_box(S, ic, hlo, hhi);
    const int nwarp = blockDim.x >> 5;
    for (int k = warp; k < nseg; k += nwarp)
      pk_stage_segment(P, seg[k], hlo, hhi, S.cull2, smem, lane);
  }
  __syncthreads();
  // one home cell: every staged segment, its own the self segment; several:
  // the three staged cells around home cell h
  const int selfk = centre ? (split == 3 ? 4 : 1) : -1;
  const int wseg = ic.nhome == 1 ? nseg : 3;
  for (int h = 0; h < ic.nhome; ++h) {
    const PairSeg &hc = seg[9 + h];
    pk_compute<VIR, true, DYN>(P, S, s, hc.beg, hc.beg + hc.n, hc.a, hc.b, seg + h, wseg, selfk,
                               smem, tid, blockDim.x, DYN ? s_task + h : nullptr);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Fine cells (side >= rc / 2), culled per warp.  A work item is one block of
// up to 2 x 2 x 2 cells and one third of its neighbour z-range.  Each warp
// takes 32 home beads in the block's Gray-code cell order (consecutive
// cells adjacent, so a warp's beads span a 2 x 2 x 1 cell box), computes
// their bounding box, and visits only the neighbour cells whose box lies
// within rc (+1e-3 margin, far above FP32 rounding) of it; candidates are
// read from the sorted positions in global memory (L1/L2 resident).  No
// shared memory and no CTA barriers: warps work independently.
// ---------------------------------------------------------------------------
template <bool VIR, bool DBG>
__device__ __forceinline__ void dev_pair_fine_item(const Pool &P, const int2 *work, int w) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int s = work[w].x, code = work[w].y;
  const SysDesc &S = P.sys[s];
  const int blk = code / 3, zpart = code % 3;
  const int nc0 = S.nc[0], nc1 = S.nc[1], nc2 = S.nc[2];
  const int bx = blk % S.nb[0], by = (blk / S.nb[0]) % S.nb[1], bz = blk / (S.nb[0] * S.nb[1]);
  const int lo[3] = {2 * bx, 2 * by, 2 * bz};
  const int wd[3] = {min(2, nc0 - lo[0]), min(2, nc1 - lo[1]), min(2, nc2 - lo[2])};
  // home cells in Gray-code order; non-image bead ranges and their prefix
  const int gray[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                          {0, 1, 1}, {1, 1, 1}, {1, 0, 1}, {0, 0, 1}};
  int hb[8], hp[9];
  hp[0] = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int b = 0, n = 0;
    if (gray[k][0] < wd[0] && gray[k][1] < wd[1] && gray[k][2] < wd[2]) {
      const long long cg = S.cell_off + (lo[0] + gray[k][0]) +
                           nc0 * ((lo[1] + gray[k][1]) + nc1 * (lo[2] + gray[k][2]));
      b = P.cell_start[cg] + P.cell_nimg[cg];
      n = P.cell_start[cg + 1] - b;
    }
    hb[k] = b;
    hp[k + 1] = hp[k] + n;
  }
  const int total = hp[8];
  // neighbour z-range [lo - 2, lo + wd + 1], this item's third of it
  const int zspan = wd[2] + 4;
  const int z0 = lo[2] - 2 + (zpart * zspan) / 3, z1 = lo[2] - 2 + ((zpart + 1) * zspan) / 3;
  const float rc2 = S.rc2f, gcc = S.gc_c2f;
  for (int c0 = warp * 32; c0 < total; c0 += nwarp * 32) {
    const int idx = c0 + lane;
    const bool valid = idx < total;
    int i = 0;
    if (valid) {
      int k = 0;
#pragma unroll
      for (int q = 1; q < 8; ++q) k += idx >= hp[q];
      i = hb[k] + (idx - hp[k]);
    }
    const float4 xi = valid ? P.xyzq_s[i] : make_float4(1e30f, 1e30f, 1e30f, 0.0f);
    // warp bounding box of the valid beads
    float bmin[3] = {valid ? xi.x : 3e38f, valid ? xi.y : 3e38f, valid ? xi.z : 3e38f};
    float bmax[3] = {valid ? xi.x : -3e38f, valid ? xi.y : -3e38f, valid ? xi.z : -3e38f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bmin[a] = fminf(bmin[a], __shfl_xor_sync(0xffffffffu, bmin[a], o));
        bmax[a] = fmaxf(bmax[a], __shfl_xor_sync(0xffffffffu, bmax[a], o));
      }
    const bool anyq = __any_sync(0xffffffffu, valid && xi.w != 0.0f);
    PairAcc A;
    A.eg = A.ere = A.gx = A.gy = A.gz = A.fx = A.fy = A.fz = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) A.wg[k] = A.we[k] = 0.0f;
    for (int uz = z0; uz < z1; ++uz) {
      const float gz_ =
          fmaxf(0.0f, fmaxf(uz * S.cside[2] - bmax[2], bmin[2] - (uz + 1) * S.cside[2]));
      const float dz2 = gz_ * gz_;
      if (dz2 > S.cull2) continue;
      for (int uy = lo[1] - 2; uy < lo[1] + wd[1] + 2; ++uy) {
        const float gy_ =
            fmaxf(0.0f, fmaxf(uy * S.cside[1] - bmax[1], bmin[1] - (uy + 1) * S.cside[1]));
        const float dyz2 = dz2 + gy_ * gy_;
        if (dyz2 > S.cull2) continue;
        for (int ux = lo[0] - 2; ux < lo[0] + wd[0] + 2; ++ux) {
          const float gx_ =
              fmaxf(0.0f, fmaxf(ux * S.cside[0] - bmax[0], bmin[0] - (ux + 1) * S.cside[0]));
          if (dyz2 + gx_ * gx_ > S.cull2) continue;
          const int u[3] = {ux, uy, uz};
          const int ncv[3] = {nc0, nc1, nc2};
          int v[3], nn[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            nn[a] = floor_div(u[a], ncv[a]);
            v[a] = u[a] - nn[a] * ncv[a];
          }
          const long long cg = S.cell_off + v[0] + nc0 * (v[1] + nc1 * v[2]);
          PairSeg sg;
          sg.beg = P.cell_start[cg];
          sg.n = P.cell_start[cg + 1] - sg.beg;
          sg.a = P.cell_nimg[cg];
          sg.b = P.cell_nq[cg];
          sg.code = (nn[0] + 1) + 3 * (nn[1] + 1) + 9 * (nn[2] + 1);
#pragma unroll
          for (int a = 0; a < 3; ++a) sg.sh[a] = (float)nn[a] * S.boxf[a];
          sg.shifted = (nn[0] != 0 || nn[1] != 0 || nn[2] != 0);
          // the cell can hold i itself only unshifted and inside the block
          sg.self = !sg.shifted && ux >= lo[0] && ux < lo[0] + wd[0] && uy >= lo[1] &&
                    uy < lo[1] + wd[1] && uz >= lo[2] && uz < lo[2] + wd[2];
          pair_segment<VIR, DBG>(P.xyzq_s + sg.beg, 0, sg.n, sg.beg, sg, anyq, xi, i, S, rc2, gcc,
                                 A, P, s);
        }
      }
    }
    const float cgf = S.gc_forcef;
    const float lb = S.lbf;
    if (valid) {
      const int orig = P.sorted_idx[i];
      atomic_add_fixed_f(force_ptr(P, S, orig, 0), -(cgf * A.gx + lb * A.fx), (float)kFScale);
      atomic_add_fixed_f(force_ptr(P, S, orig, 1), -(cgf * A.gy + lb * A.fy), (float)kFScale);
      atomic_add_fixed_f(force_ptr(P, S, orig, 2), -(cgf * A.gz + lb * A.fz), (float)kFScale);
    }
    const long long eg = warp_sum(valid ? efix(S.gc_halfpref * A.eg) : 0ll);
    const long long er = warp_sum(valid ? efix(S.lb_half * A.ere) : 0ll);
    unsigned long long *acc = P.acc + (long long)s * kNacc;
    if (lane == 0) {
      atomicAdd(acc + ACC_GC, (unsigned long long)eg);
      atomicAdd(acc + ACC_REAL, (unsigned long long)er);
    }
    if (VIR) {
      const float c1 = 0.5f * S.gc_forcef, c2 = S.lb_half;
      const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const long long vv =
            warp_sum(valid ? efix(c1 * A.wg[map[k]] + c2 * A.we[map[k]]) : 0ll);
        if (lane == 0) atomicAdd(P.vacc + (long long)s * 9 + k, (unsigned long long)vv);
      }
    }
  }
}

}  // namespace gcme
