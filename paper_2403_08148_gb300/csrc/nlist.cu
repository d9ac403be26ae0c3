// nlist.cu -- Verlet neighbour list for the FP32 pair path.
//
// The 27-cell stencil tests ~6.5 candidates per in-cutoff pair.  A list of
// every (j, image) within rc + skin of each real bead, built from the cell
// list, holds ~1.45 candidates per in-cutoff pair and stays valid until
// some bead has moved more than skin / 2 since the build; the cell sort
// and the list build then run again.  The kernels of that chain read a
// device flag and return at once on the other steps, so a step stays one
// captured graph whatever the rebuild schedule.
//
// Exactness.  The in-cutoff decision is the FP32 rule of the cell kernels
// on the wrapped coordinates of this step:
//   d_a = fl(fl(x_j,a - x_i,a) + fl(n_a L_a)),  r2 = fl(...),  r2 < fl(rc^2).
// An entry keeps the image shift n of its build; since a bead that crosses
// the box is re-wrapped, the kernel corrects it by the image-index changes
// of both beads since the build, n' = n + dimg_j - dimg_i, the shift that
// joins the same two unwrapped positions.  Every (j, n') within rc now was
// within rc + skin at the build, so the pair set is the cell kernels'.
//
// Determinism.  Every pair term (force components, energies, virial) is
// rounded to a multiple of 2^-b (b per system, SysDesc::fix_bits, so that no
// term exceeds 2^30 units) and summed as 64-bit integers: the sums are the
// same in any order and any split over lanes, so forces and energies are
// bit-identical whenever and however the list was built (and between a
// system run alone, in a batch or in the server).  The rounding error,
// 2^-(b+1) per term (6e-8 for the paper's parameters), is below the FP32
// rounding of the terms themselves.
//
// A system whose lists overflow their stride runs the 27-cell kernel
// instead (per-system flag) and rebuilds every step until the list fits.
#include "kernels.h"
#include "pair.cuh"

namespace gcme {

constexpr int kListLanes = 4;     // lanes per bead in the list pair kernel
constexpr int kListWarps = 4;     // beads per CTA of the build kernel
constexpr int kDimgBias = 512;    // packed image change: 10 bits per axis
constexpr int kSlotBits = 25;     // sorted-slot bits of an entry

__device__ __forceinline__ int pack_dimg(int dx, int dy, int dz) {
  return (dx + kDimgBias) | ((dy + kDimgBias) << 10) | ((dz + kDimgBias) << 20);
}

__device__ __forceinline__ int slot_system(const Pool &P, long long g) {
  // sorted slots of system s fill [ext_off, ext_off + n_ext), like its ext beads
  int lo = 0, hi = P.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.sys[mid].ext_off <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Rebuild decision of this step: some real bead moved more than skin / 2
// since the last build (x_ref starts far away, so the first step builds),
// a system overflowed its list, or a rebuild was requested.
__global__ void k_list_check(Pool P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g == 0 && P.list_flags[1]) P.list_flags[0] = 1;
  if (g < P.nsys && P.list_ovf[g]) P.list_flags[0] = 1;
  if (g >= P.n_real) return;
  double d2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double d = P.pos[3 * g + a] - P.x_ref[3 * g + a];
    d2 += d * d;
  }
  if (!(d2 <= P.half_skin2)) P.list_flags[0] = 1;
}

// One CTA per cell; each warp takes 32 of the cell's real beads, one per
// lane.  The warp visits the cells within R cells of the home cell (R = 1
// when cells are at least rc + skin wide, else 2) whose box lies within
// rc + skin (+1e-3) of the warp's bounding box, reads their beads with
// warp-uniform loads (one transaction, L1-resident), and every lane appends
// the ones within rc + skin of its bead to its own list: first the image
// and charged beads of all visited cells, then the neutral ones.  The test
// here only has to keep a superset with margin (the displacement bound
// leaves 2e-4 of the skin), so it uses the cheaper d = x_j - (x_i - shift).
__global__ void __launch_bounds__(32 * kListWarps) k_list_build(Pool P) {
  if (!P.list_flags[0]) return;
  const long long cg = blockIdx.x;
  if (cg >= P.n_cells) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = P.cell_sys[cg];
  const SysDesc &S = P.sys[s];
  const int cloc = (int)(cg - S.cell_off);
  const int c[3] = {cloc % S.nc[0], (cloc / S.nc[0]) % S.nc[1], cloc / (S.nc[0] * S.nc[1])};
  const int hbeg = P.cell_start[cg], hend = P.cell_start[cg + 1];
  const int rbeg = hbeg + P.cell_nimg[cg];
  for (int t = hbeg + threadIdx.x; t < rbeg; t += blockDim.x) {  // images are never i
    P.nbr_cnt[t] = 0;
    P.nbr_nq[t] = 0;
  }
  const float rl2 = S.rl2f;
  const float rlm = sqrtf(rl2) + 1e-3f;
  const float cull = rlm * rlm;
  const int R = (S.cside[0] >= rlm && S.cside[1] >= rlm && S.cside[2] >= rlm) ? 1 : 2;
  const int cap = 4 * P.nbr_stride;
  const long long n4 = P.n_ext * kListLanes;
  bool over = false;
  for (int c0 = rbeg + warp * 32; c0 < hend; c0 += blockDim.x) {
    const int i = c0 + lane;
    const bool valid = i < hend;
    const float4 xi = valid ? P.xyzq_s[i] : P.xyzq_s[c0];
    float bmin[3] = {xi.x, xi.y, xi.z}, bmax[3] = {xi.x, xi.y, xi.z};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bmin[a] = fminf(bmin[a], __shfl_xor_sync(0xffffffffu, bmin[a], o));
        bmax[a] = fmaxf(bmax[a], __shfl_xor_sync(0xffffffffu, bmax[a], o));
      }
    int* const row = P.nbr + (long long)i * kListLanes;
    int cnt = 0, nq = 0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int oz = -R; oz <= R; ++oz) {
        const int uz = c[2] + oz;
        const float gz =
            fmaxf(0.0f, fmaxf(uz * S.cside[2] - bmax[2], bmin[2] - (uz + 1) * S.cside[2]));
        for (int oy = -R; oy <= R; ++oy) {
          const int uy = c[1] + oy;
          const float gy =
              fmaxf(0.0f, fmaxf(uy * S.cside[1] - bmax[1], bmin[1] - (uy + 1) * S.cside[1]));
          if (gz * gz + gy * gy > cull) continue;
          for (int ox = -R; ox <= R; ++ox) {
            const int ux = c[0] + ox;
            const float gx =
                fmaxf(0.0f, fmaxf(ux * S.cside[0] - bmax[0], bmin[0] - (ux + 1) * S.cside[0]));
            if (gz * gz + gy * gy + gx * gx > cull) continue;
            const int u[3] = {ux, uy, uz};
            int v[3], nn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              nn[a] = u[a] < 0 ? -1 - (-1 - u[a]) / S.nc[a] : u[a] / S.nc[a];
              v[a] = u[a] - nn[a] * S.nc[a];
            }
            const long long cj = S.cell_off + v[0] + S.nc[0] * (v[1] + S.nc[1] * v[2]);
            const int jb = P.cell_start[cj], je = P.cell_start[cj + 1];
            const int jq = jb + P.cell_nq[cj], ja = jb + P.cell_nimg[cj];
            const int t0 = pass == 0 ? jb : jq, t1 = pass == 0 ? jq : je;
            const float px = xi.x - (float)nn[0] * S.boxf[0];
            const float py = xi.y - (float)nn[1] * S.boxf[1];
            const float pz = xi.z - (float)nn[2] * S.boxf[2];
            const bool self = ox == 0 && oy == 0 && oz == 0;
            const unsigned code =
                (unsigned)((nn[0] + 1) | ((nn[1] + 1) << 2) | ((nn[2] + 1) << 4)) << kSlotBits;
            for (int j = t0; j < t1; ++j) {
              const float4 xj = P.xyzq_s[j];
              const float dx = xj.x - px, dy = xj.y - py, dz = xj.z - pz;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              if (valid && r2 < rl2 && !(self && j == i)) {
                if (cnt < cap)
                  row[(long long)(cnt >> 2) * n4 + (cnt & 3)] =
                      (int)((unsigned)j | code | (j < ja ? 0x80000000u : 0u));
                ++cnt;
              }
            }
          }
        }
      }
      if (pass == 0) nq = min(cnt, cap);
    }
    if (valid) {
      over = over || cnt > cap;
      P.nbr_cnt[i] = cnt > cap ? 0 : cnt;
      P.nbr_nq[i] = cnt > cap ? 0 : nq;
    }
  }
  if (over) P.list_ovf[P.nsys + s] = 1;  // this system takes the cell kernel
}

// After a build: reference positions and image indices of the list, the
// overflow flags of the new lists, the build counter.
__global__ void k_list_ref(Pool P) {
  if (!P.list_flags[0]) return;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < P.n_ext)
    for (int a = 0; a < 3; ++a) P.img_ref[3 * g + a] = P.img_now[3 * g + a];
  if (g < P.n_real)
    for (int a = 0; a < 3; ++a) P.x_ref[3 * g + a] = P.pos[3 * g + a];
  if (g < P.nsys) {
    P.list_ovf[g] = P.list_ovf[P.nsys + g];
    P.list_ovf[P.nsys + g] = 0;
  }
  if (g == 0) {
    P.list_flags[1] = 0;
    P.list_flags[2] += 1;
  }
}

// Every step: sorted positions of this step in the build's order, and the
// image change of each slot's bead since the build.
__global__ void k_list_refresh(Pool P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P.n_ext) return;
  const long long u = P.sys[slot_system(P, g)].ext_off + P.sorted_idx[g];
  P.xyzq_s[g] = P.xyzq_u[u];
  P.dimg_s[g] = pack_dimg(P.img_now[3 * u] - P.img_ref[3 * u],
                          P.img_now[3 * u + 1] - P.img_ref[3 * u + 1],
                          P.img_now[3 * u + 2] - P.img_ref[3 * u + 2]);
}

// Integer sum of a per-bead value over the warp's beads into a 64-bit
// fixed-point accumulator (acc points at system 0's slot, systems stride_s
// apart); one atomic per warp when its beads share a system.
__device__ __forceinline__ void warp_add_int(unsigned long long *acc, long long stride_s, int s,
                                             int s0, bool same, long long q) {
  if (same) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0 && s0 >= 0 && q != 0)
      atomicAdd(acc + (long long)s0 * stride_s, (unsigned long long)q);
  } else if (s >= 0 && q != 0) {
    atomicAdd(acc + (long long)s * stride_s, (unsigned long long)q);
  }
}

// exact float of a small integer without a conversion instruction
__device__ __forceinline__ float small_int_float(int m) {
  return __int_as_float(0x4B400000 + m) - 12582912.0f;
}

// per-lane integer sums of the pair terms, in units of 2^-fix_bits
struct ListAcc {
  long long f[3];   // sum fs d (the force on i is minus this)
  long long eg, ee; // sums of u_gc and u_elec
  long long w[6];   // sum fs d_a d_b: xx, yy, zz, xy, xz, yz
};

// Entries [k0, k1) of one lane.  ELEC: the real-space electrostatics too
// (charged i over the charged/image part of its list); IMG: the range may
// hold image beads (no Gaussian core with them).
template <bool ELEC, bool IMG, bool VIR, bool DBG>
__device__ __forceinline__ void list_range(const Pool &P, const SysDesc &S, const int *col,
                                           long long cstride, int k0, int k1, const float4 &xi,
                                           const int (&pib)[3], ListAcc &A, int s, int e) {
  const float rc2 = S.rc2f, gcc = S.gc_c2f, fsc = S.fix_scale;
  const float cgf = (float)(S.gc_fc * S.gc_pref) * fsc;  // force coefficient x 2^b
  const float ugf = (float)S.gc_pref * fsc;
  const float lbf = (float)S.lB * fsc;
  const float L0 = S.boxf[0], L1 = S.boxf[1], L2 = S.boxf[2];
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int ent = col[k * cstride];
    const int j = ent & ((1 << kSlotBits) - 1);
    const int pj = P.dimg_s[j];
    const float4 xj = P.xyzq_s[j];
    // n' = n + dimg_j - dimg_i (pib holds dimg_i + 1 with its packing bias)
    const int n0 = ((ent >> kSlotBits) & 3) + (pj & 1023) - pib[0];
    const int n1 = ((ent >> (kSlotBits + 2)) & 3) + ((pj >> 10) & 1023) - pib[1];
    const int n2 = ((ent >> (kSlotBits + 4)) & 3) + ((pj >> 20) & 1023) - pib[2];
    const float dx = __fadd_rn(__fsub_rn(xj.x, xi.x), small_int_float(n0) * L0);
    const float dy = __fadd_rn(__fsub_rn(xj.y, xi.y), small_int_float(n1) * L1);
    const float dz = __fadd_rn(__fsub_rn(xj.z, xi.z), small_int_float(n2) * L2);
    const float r2 =
        __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const bool in = r2 < rc2;
    float ex = ex2_approx(r2 * gcc);
    ex = (in && (!IMG || ent >= 0)) ? ex : 0.0f;
    float fs = cgf * ex;
    A.eg += __float2int_rn(ugf * ex);
    if (ELEC && in) {
      const float qq = xi.w * xj.w;
      float gg, hh;
      if (S.rtab_n > 0) real_gh_tab(P, S, r2, gg, hh);
      else real_gh_direct(r2, S.betaf, S.kappaf, S.ser_gf, S.ser_hf, gg, hh);
      const float lq = lbf * qq;
      A.ee += __float2int_rn(lq * gg);
      fs = fmaf(lq, hh, fs);
    }
    A.f[0] += __float2int_rn(fs * dx);
    A.f[1] += __float2int_rn(fs * dy);
    A.f[2] += __float2int_rn(fs * dz);
    if (VIR) {
      const float ax = fs * dx, ay = fs * dy;
      A.w[0] += __float2int_rn(ax * dx);
      A.w[1] += __float2int_rn(ay * dy);
      A.w[2] += __float2int_rn(fs * dz * dz);
      A.w[3] += __float2int_rn(ax * dy);
      A.w[4] += __float2int_rn(ax * dz);
      A.w[5] += __float2int_rn(ay * dz);
    }
    if (DBG && in) {
      const unsigned long long kk = atomicAdd(&P.acc[(long long)s * kNacc + ACC_NPAIR], 1ull);
      if ((long long)kk < P.dbg_cap) {
        P.dbg_triples[3 * kk + 0] = e;
        P.dbg_triples[3 * kk + 1] = P.sorted_idx[j];
        P.dbg_triples[3 * kk + 2] = (n0 + 1) + 3 * (n1 + 1) + 9 * (n2 + 1);
      }
    }
  }
}

// Pair kernel over the lists: lanes 4g .. 4g+3 take entries m = lane (mod
// 4) of sorted slot g; physics as in the cell kernels (pair.cuh).
template <bool VIR, bool DBG>
__global__ void __launch_bounds__(256) k_pair_list(Pool P) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long g = t / kListLanes;
  const int sub = (int)(t % kListLanes);
  bool act = g < P.n_ext;
  int s = -1, e = 0;
  if (act) {
    s = slot_system(P, g);
    e = P.sorted_idx[g];
    act = e < P.sys[s].n && !P.list_ovf[s];
  }
  const SysDesc &S = P.sys[s < 0 ? 0 : s];
  ListAcc A;
  A.f[0] = A.f[1] = A.f[2] = A.eg = A.ee = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) A.w[k] = 0;
  if (act) {
    const float4 xi = P.xyzq_s[g];
    const int pi = P.dimg_s[g];
    const int pib[3] = {(pi & 1023) + 1, ((pi >> 10) & 1023) + 1, ((pi >> 20) & 1023) + 1};
    const int C = P.nbr_cnt[g], Q = P.nbr_nq[g];
    const int cnt = (C + kListLanes - 1 - sub) / kListLanes;  // entries m = sub (mod 4)
    const int nq = (Q + kListLanes - 1 - sub) / kListLanes;
    const int *col = P.nbr + g * kListLanes + sub;
    const long long cstride = P.n_ext * kListLanes;
    if (xi.w != 0.0f)
      list_range<true, true, VIR, DBG>(P, S, col, cstride, 0, nq, xi, pib, A, s, e);
    else
      list_range<false, true, VIR, DBG>(P, S, col, cstride, 0, nq, xi, pib, A, s, e);
    list_range<false, false, VIR, DBG>(P, S, col, cstride, nq, cnt, xi, pib, A, s, e);
  }
  // combine the four lanes of a bead (integer sums: exact)
#pragma unroll
  for (int o = 1; o < kListLanes; o <<= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) A.f[a] += __shfl_xor_sync(0xffffffffu, A.f[a], o);
    A.eg += __shfl_xor_sync(0xffffffffu, A.eg, o);
    A.ee += __shfl_xor_sync(0xffffffffu, A.ee, o);
    if (VIR)
#pragma unroll
      for (int k = 0; k < 6; ++k) A.w[k] += __shfl_xor_sync(0xffffffffu, A.w[k], o);
  }
  const bool lead = act && sub == 0;
  // forces at the 2^32 scale: F_i = -sum fs d; energies and virial carry 1/2
  const long long up = 1LL << (32 - S.fix_bits), half = 1LL << (31 - S.fix_bits);
  if (lead)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      atomicAdd(force_ptr(P, S, e, a), (unsigned long long)(-A.f[a] * up));
  const int sl = lead ? s : -1;
  const int s0 = __reduce_max_sync(0xffffffffu, sl);
  const bool same = __all_sync(0xffffffffu, sl < 0 || sl == s0);
  warp_add_int(P.acc + ACC_GC, kNacc, sl, s0, same, lead ? A.eg * half : 0);
  warp_add_int(P.acc + ACC_REAL, kNacc, sl, s0, same, lead ? A.ee * half : 0);
  if (VIR) {
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
#pragma unroll
    for (int k = 0; k < 9; ++k)
      warp_add_int(P.vacc + k, 9, sl, s0, same, lead ? A.w[map[k]] * half : 0);
  }
}

void launch_list_check(const Pool &P, cudaStream_t st) {
  cudaMemsetAsync(P.list_flags, 0, sizeof(int), st);
  const long long n = P.n_real > P.nsys ? P.n_real : P.nsys;
  k_list_check<<<(int)((n + 255) / 256), 256, 0, st>>>(P);
}

void launch_list_build(const Pool &P, cudaStream_t st) {
  if (P.n_ext == 0) return;
  k_list_build<<<(unsigned)P.n_cells, 32 * kListWarps, 0, st>>>(P);
  const long long n = P.n_ext > P.nsys ? P.n_ext : P.nsys;
  k_list_ref<<<(int)((n + 255) / 256), 256, 0, st>>>(P);
}

void launch_list_refresh(const Pool &P, cudaStream_t st) {
  if (P.n_ext > 0) k_list_refresh<<<(int)((P.n_ext + 255) / 256), 256, 0, st>>>(P);
}

void launch_pair_list(const Pool &P, bool vir, bool dbg, cudaStream_t st) {
  if (P.n_ext == 0) return;
  const long long threads = P.n_ext * kListLanes;
  const int nb = (int)((threads + 255) / 256);
  if (dbg) k_pair_list<false, true><<<nb, 256, 0, st>>>(P);
  else if (vir) k_pair_list<true, false><<<nb, 256, 0, st>>>(P);
  else k_pair_list<false, false><<<nb, 256, 0, st>>>(P);
}

}  // namespace gcme
