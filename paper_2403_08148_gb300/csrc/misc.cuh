// misc.cuh -- K9-K12 device bodies: harmonic bonds, electrode walls, Yeh-Berkowitz slab
// term, velocity Verlet and the FP64 energy/virial finalisation.
#pragma once
#include "common.cuh"


namespace gcme {

// Add v to the accumulator `slot` of system s from every lane of a warp.
// Lanes of one warp may belong to different systems (bead-parallel kernels
// over a batch): the warp reduces when all lanes agree, else each lane adds.
// Add one fixed-point term per lane (efix units) to system s's accumulator:
// one integer warp sum when the warp's lanes share a system.
__device__ __forceinline__ void sys_acc_add(const Pool &P, int s, bool act, int slot,
                                            long long v) {
  const unsigned full = 0xffffffffu;
  const int s0 = __shfl_sync(full, s, 0);
  const bool same = __all_sync(full, s == s0);
  if (same) {
    const long long t = warp_sum(act ? v : 0ll);
    if ((threadIdx.x & 31) == 0 && s0 >= 0 && t)
      atomicAdd(P.acc + (long long)s0 * kNacc + slot, (unsigned long long)t);
  } else if (act && v) {
    atomicAdd(P.acc + (long long)s * kNacc + slot, (unsigned long long)v);
  }
}

__device__ __forceinline__ void sys_vir_add(const Pool &P, int s, bool act, const long long W[9]) {
  const unsigned full = 0xffffffffu;
  const int s0 = __shfl_sync(full, s, 0);
  const bool same = __all_sync(full, s == s0);
  for (int k = 0; k < 9; ++k) {
    if (same) {
      const long long t = warp_sum(act ? W[k] : 0ll);
      if ((threadIdx.x & 31) == 0 && s0 >= 0 && t)
        atomicAdd(P.vacc + (long long)s0 * 9 + k, (unsigned long long)t);
    } else if (act && W[k]) {
      atomicAdd(P.vacc + (long long)s * 9 + k, (unsigned long long)W[k]);
    }
  }
}

// Harmonic bond u = k/2 (r - r0)^2 on the minimum-image separation (periodic
// axes only: x, y, z in bulk, x, y in slabs).  FP32 arithmetic on the FP64
// difference (FP64 throughout for FP64 systems).
// F32: the caller runs FP32 systems only (the FP64 branch is not compiled)
template <bool VIR, bool F32 = false>
__device__ __forceinline__ void dev_bonds(const Pool &P, long long b) {
  const bool act = b < P.n_bond;
  int s = -1;
  long long E = 0;
  long long W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (act) {
    s = P.bond_sys[b];
    const SysDesc &S = P.sys[s];
    const int2 ij = P.bonds[b];
    const double *pi = P.pos + 3 * (S.bead_off + ij.x);
    const double *pj = P.pos + 3 * (S.bead_off + ij.y);
    const bool per[3] = {true, true, S.geometry == GCME_BULK};
    if (!F32 && S.precision == GCME_FP64) {
      double d[3];
      for (int a = 0; a < 3; ++a) {
        d[a] = pj[a] - pi[a];
        if (per[a]) d[a] -= S.box[a] * rint(d[a] / S.box[a]);
      }
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double fs = S.bond_k * (r - S.bond_r0) / r;
      E = efix(0.5 * S.bond_k * (r - S.bond_r0) * (r - S.bond_r0));
      for (int a = 0; a < 3; ++a) {
        atomic_add_fixed(force_ptr(P, S, ij.x, a), fs * d[a], kFScale);
        atomic_add_fixed(force_ptr(P, S, ij.y, a), -fs * d[a], kFScale);
      }
      if (VIR)
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) W[3 * a + c] = efix(-fs * d[a] * d[c]);
    } else {
      // FP32 arithmetic on the FP64 difference
      float d[3];
      for (int a = 0; a < 3; ++a) {
        d[a] = (float)(pj[a] - pi[a]);
        if (per[a]) d[a] -= S.boxf[a] * rintf(d[a] / S.boxf[a]);
      }
      const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const float kf = S.bond_kf, r0 = S.bond_r0f;
      const float fs = kf * (r - r0) / r;
      E = efix(0.5f * kf * (r - r0) * (r - r0));
      for (int a = 0; a < 3; ++a) {
        atomic_add_fixed_f(force_ptr(P, S, ij.x, a), fs * d[a], (float)kFScale);
        atomic_add_fixed_f(force_ptr(P, S, ij.y, a), -fs * d[a], (float)kFScale);
      }
      if (VIR)
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) W[3 * a + c] = efix(-fs * d[a] * d[c]);
    }
  }
  sys_acc_add(P, s, act, ACC_BOND, E);
  if (VIR) sys_vir_add(P, s, act, W);
}

// Electrode walls at z = 0 and z = H (continuum Gaussian-core layer)
//   u_w(h) = (A n_s) (3 / (2 pi s_w))^{1/2} exp(-3 h^2 / (2 s_w))
// and the slab dipole M_z = sum z_i z_pos,i for the Yeh-Berkowitz term.
__device__ __forceinline__ void dev_walls(const Pool &P, long long g) {
  bool act = g < P.n_real;
  int s = -1;
  long long Ew = 0, Mz = 0;
  bool slab = false, nm = false;
  if (act) {
    s = P.real_sys[g];
    const SysDesc &S = P.sys[s];
    slab = S.geometry != GCME_BULK;
    nm = S.geometry == GCME_SLAB_NONMETAL;
    if (slab) {
      const int i = (int)(g - S.bead_off);
      const double z = P.pos[3 * g + 2];
      if (S.wall_A != 0.0) {
        const double c = S.wall_A * sqrt(3.0 / (2.0 * 3.14159265358979323846 * S.wall_s2));
        const double h1 = S.H - z;
        if (S.precision == GCME_FP64) {
          const double u0 = c * exp(-1.5 * z * z / S.wall_s2);
          const double u1 = c * exp(-1.5 * h1 * h1 / S.wall_s2);
          Ew = efix(u0 + u1);
          const double fz = 3.0 * z / S.wall_s2 * u0 - 3.0 * h1 / S.wall_s2 * u1;
          atomic_add_fixed(force_ptr(P, S, i, 2), fz, kFScale);
        } else {
          const float zf = (float)z, h1f = (float)h1, s2 = (float)S.wall_s2, cf = (float)c;
          const float u0 = cf * expf(-1.5f * zf * zf / s2);
          const float u1 = cf * expf(-1.5f * h1f * h1f / s2);
          Ew = efix(u0 + u1);
          const float fz = 3.0f * zf / s2 * u0 - 3.0f * h1f / s2 * u1;
          atomic_add_fixed_f(force_ptr(P, S, i, 2), fz, (float)kFScale);
        }
      }
      if (nm) Mz = efix(P.q[g] * z);
    }
  }
  sys_acc_add(P, s, act && slab, ACC_WALL, Ew);
  sys_acc_add(P, s, act && nm, ACC_MZ, Mz);
}

// Yeh-Berkowitz force F_z,i = -4 pi lB z_i M_z / V (nonmetal slabs).
__device__ __forceinline__ void dev_slab_apply(const Pool &P, long long g) {
  if (g >= P.n_real) return;
  const int s = P.real_sys[g];
  const SysDesc &S = P.sys[s];
  if (S.geometry != GCME_SLAB_NONMETAL) return;
  const double Mz = (double)(long long)P.acc[(long long)s * kNacc + ACC_MZ] / kEScale;
  const double fz = -4.0 * 3.14159265358979323846 * S.lB * P.q[g] * Mz / S.V;
  unsigned long long *f = force_ptr(P, S, (int)(g - S.bead_off), 2);
  *f += (unsigned long long)__double2ll_rn(fz * kFScale);
}

// Per-system energies (FP64) from the fixed-point accumulators.
template <bool VIR>
__device__ __forceinline__ void dev_finalize(const Pool &P, int s) {
  if (s >= P.nsys) return;
  const SysDesc &S = P.sys[s];
  const unsigned long long *a = P.acc + (long long)s * kNacc;
  auto rd = [&](int k) { return (double)(long long)a[k] / kEScale; };
  double *E = P.energy + (long long)s * GCME_NTERMS;
  E[GCME_E_GC] = rd(ACC_GC);
  E[GCME_E_REAL] = rd(ACC_REAL);
  E[GCME_E_RECIP] = rd(ACC_RECIP);
  E[GCME_E_CORR] = S.e_corr;
  E[GCME_E_SELF] = S.e_self;
  double slab = 0.0;
  if (S.geometry == GCME_SLAB_NONMETAL) {
    const double Mz = rd(ACC_MZ);
    slab = 2.0 * 3.14159265358979323846 * S.lB * Mz * Mz / S.V;
  }
  E[GCME_E_SLAB] = slab;
  E[GCME_E_WALL] = rd(ACC_WALL);
  E[GCME_E_BOND] = rd(ACC_BOND);
  double pot = 0.0;
  for (int k = 0; k < 8; ++k) pot += E[k];
  E[GCME_E_POTENTIAL] = pot;
  E[GCME_E_KINETIC] = rd(ACC_KIN);
  if (VIR)
    for (int k = 0; k < 9; ++k)
      P.virial[(long long)s * 9 + k] = (double)(long long)P.vacc[(long long)s * 9 + k] / kEScale;
}

// Philox4x64-10 block function (Salmon, Moraes, Dror and Shaw, SC'11):
// ten rounds of two 64 x 64 -> 128-bit products with the round multipliers,
// the key bumped by the Weyl increments between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
  const unsigned long long m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
  const unsigned long long w0 = 0x9E3779B97F4A7C15ull, w1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += w0;
      k1 += w1;
    }
    const unsigned long long hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
    const unsigned long long hi1 = __umul64hi(m1, c[2]), lo1 = m1 * c[2];
    const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Langevin noise of bead i at step n: counter (n, i, 0, 0), key (seed, 0);
// uniforms u_k = (floor(w_k / 2^40) + 1/2) / 2^24; Box-Muller:
//   z_x = sqrt(-2 ln u0) cos(2 pi u1), z_y = sqrt(-2 ln u0) sin(2 pi u1),
//   z_z = sqrt(-2 ln u2) cos(2 pi u3).
// FP32 arithmetic for FP32 velocities, FP64 for FP64 velocities.
template <typename V>
__device__ __forceinline__ void langevin_noise(unsigned long long seed, unsigned long long n,
                                               unsigned long long i, V z[3]) {
  unsigned long long c[4] = {n, i, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
  V u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    u[k] = ((V)(c[k] >> 40) + V(0.5)) * V(1.0 / 16777216.0);
  if constexpr (sizeof(V) == 4) {
    const float r0 = sqrtf(-2.0f * logf(u[0])), r2 = sqrtf(-2.0f * logf(u[2]));
    float s1, c1;
    sincospif(2.0f * u[1], &s1, &c1);
    z[0] = r0 * c1;
    z[1] = r0 * s1;
    z[2] = r2 * cospif(2.0f * u[3]);
  } else {
    const double r0 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
    double s1, c1;
    sincospi(2.0 * u[1], &s1, &c1);
    z[0] = r0 * c1;
    z[1] = r0 * s1;
    z[2] = r2 * cospi(2.0 * u[3]);
  }
}

// Fixed-point force component as V (FP32: no 64-bit conversion).
template <typename V> __device__ __forceinline__ V force_value(long long fq);
template <> __device__ __forceinline__ float force_value<float>(long long fq) {
  return ll2f(fq) * (float)(1.0 / kFScale);
}
template <> __device__ __forceinline__ double force_value<double>(long long fq) {
  return (double)fq * (1.0 / kFScale);
}

// First half of a step, unit masses, FP64 positions.
//   velocity Verlet:  v += dt/2 F;  x += dt v.
//   Langevin (BAOAB): v += dt/2 F;  x += dt/2 v;  v = c1 v + c2 z;  x += dt/2 v
// with z the noise of this bead at the system's step counter.
// beads of a frozen species (explicit electrodes) keep x and v
__device__ __forceinline__ bool frozen_bead(const Pool &P, const SysDesc &S, int i) {
  return S.frozen_mask && ((S.frozen_mask >> P.type_u[S.ext_off + i]) & 1);
}

// Each bead's force is cleared once read (the step's force evaluation
// accumulates into it next).  ONE: the pool holds one system (s = 0, bead
// offset 0, n = n_real), so the force loads go out with the bead's state
// instead of after the system lookup.
template <typename V, bool ONE = false>
__device__ __forceinline__ void dev_kick_drift(const Pool &P, long long g) {
  if (g >= P.n_real) return;
  V *vel = reinterpret_cast<V *>(P.vel) + 3 * g;
  // the bead's state first: its loads do not wait for the system lookup
  V v0[3];
  double x0[3];
  long long f1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v0[a] = vel[a];
    x0[a] = P.pos[3 * g + a];
    if (ONE) f1[a] = P.force[(long long)a * P.n_real + g];
  }
  const int s = ONE ? 0 : P.real_sys[g];
  const SysDesc &S = P.sys[s];
  const int i = ONE ? (int)g : (int)(g - S.bead_off);
  auto fptr = [&](int a) {
    return ONE ? reinterpret_cast<unsigned long long *>(P.force + (long long)a * P.n_real + g)
               : force_ptr(P, S, i, a);
  };
  bool held = false;  // a system that has taken its steps (step limits)
  if (P.step_stop) {
    held = P.step_ctr[s] >= P.step_stop[s];
    if (i == 0) P.held[s] = held ? 1 : 0;
  }
  if (held || frozen_bead(P, S, i)) {
    for (int a = 0; a < 3; ++a) *fptr(a) = 0ull;
    return;
  }
  V h;
  if constexpr (sizeof(V) == 4) h = S.half_dtf;
  else h = 0.5 * S.dt;
  if (S.langevin) {
    V z[3];
    langevin_noise<V>(S.seed, P.step_ctr[s], (unsigned long long)i, z);
    const V c1 = V(S.lgv_c1), c2 = V(S.lgv_c2);
    const double hd = 0.5 * S.dt;
    for (int a = 0; a < 3; ++a) {
      unsigned long long *fp = fptr(a);
      const long long fq = ONE ? f1[a] : (long long)*fp;
      *fp = 0ull;
      V v = v0[a] + h * force_value<V>(fq);
      double x = x0[a] + hd * (double)v;
      v = c1 * v + c2 * z[a];
      vel[a] = v;
      P.pos[3 * g + a] = x + hd * (double)v;
    }
    return;
  }
  const double dt = S.dt;  // read before the stores below (no reload per axis)
  for (int a = 0; a < 3; ++a) {
    unsigned long long *fp = fptr(a);
    const long long fq = ONE ? f1[a] : (long long)*fp;
    *fp = 0ull;
    V v = v0[a] + h * force_value<V>(fq);
    vel[a] = v;
    P.pos[3 * g + a] = x0[a] + dt * (double)v;
  }
}

template <typename V, bool ONE = false>
__device__ __forceinline__ void dev_kick(const Pool &P, long long g) {
  const bool act = g < P.n_real;
  int s = -1;
  long long ke = 0;
  if (act) {
    V *vel = reinterpret_cast<V *>(P.vel) + 3 * g;
    V v0[3];
    long long f1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v0[a] = vel[a];
      if (ONE) f1[a] = P.force[(long long)a * P.n_real + g];
    }
    s = ONE ? 0 : P.real_sys[g];
    const SysDesc &S = P.sys[s];
    const int i = ONE ? (int)g : (int)(g - S.bead_off);
    V h;
    if constexpr (sizeof(V) == 4) h = S.half_dtf;
    else h = 0.5 * S.dt;
    const bool frozen = frozen_bead(P, S, i);
    // held (step limits): the state stays, its kinetic energy is reported
    const bool held = P.step_stop && P.held[s];
    V v2 = V(0);
    if (held)
      for (int a = 0; a < 3 && !frozen; ++a) v2 += v0[a] * v0[a];
    for (int a = 0; a < 3 && !frozen && !held; ++a) {
      const long long fq =
          ONE ? f1[a] : *reinterpret_cast<const long long *>(force_ptr(P, S, i, a));
      V v = v0[a] + h * force_value<V>(fq);
      vel[a] = v;
      v2 += v * v;
    }
    ke = efix(V(0.5) * v2);
    // the step is complete: advance the system's step counter (read by the
    // kick-drift kernel of the next step)
    if (i == 0 && P.step_ctr && !held) P.step_ctr[s] += 1;
  }
  sys_acc_add(P, s, act, ACC_KIN, ke);
}

}  // namespace gcme
