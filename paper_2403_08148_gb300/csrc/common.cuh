// common.cuh -- descriptors and device helpers shared by the libgcme kernels.
//
// Every kernel works on a *batch* of independent systems held in pooled
// device arrays; a single system is a batch of one.  Per-system sizes,
// offsets and constants live in a device table of SysDesc; the pooled array
// base pointers travel by value in a Pool struct (a kernel argument), so the
// same kernels serve gcme_forces (caller's buffers), batches and the server.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gcme.h"

namespace gcme {

// FP64 position + charge (x, y, z, q), 32-byte aligned
struct __align__(32) dpos4 {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ dpos4 make_dpos4(double x, double y, double z, double w) {
  dpos4 r;
  r.x = x;
  r.y = y;
  r.z = z;
  r.w = w;
  return r;
}

constexpr int kNcls = 3;           // bead classes inside a cell: image, charged, neutral
constexpr int kMaxTypes = GCME_MAX_TYPES;  // species per system
constexpr int kMaxStages = 8;      // FFT stages per axis (K <= 1024)
constexpr int kNacc = 16;          // fixed-point accumulators per system
constexpr double kFScale = 4294967296.0;   // 2^32 force scale
constexpr double kEScale = 4294967296.0;   // 2^32 energy scale
constexpr double kQScale32 = 68719476736.0;    // 2^36 PME grid scale (FP32 path)
constexpr double kQScale64 = 1099511627776.0;  // 2^40 PME grid scale (FP64 path)

// accumulator slots (first 8 coincide with GCME_E_*)
enum {
  ACC_GC = 0, ACC_REAL = 1, ACC_RECIP = 2, ACC_WALL = 6, ACC_BOND = 7,
  ACC_MZ = 8,      // sum z_i z_pos,i (Yeh-Berkowitz dipole), scale 2^32
  ACC_KIN = 9,     // kinetic energy
  ACC_FLAGS = 10,  // error flags (bit 0: non-finite)
  ACC_NPAIR = 11   // debug pair count
};

// Pair constants of one species pair (i, j), several-species systems:
//   Gaussian core  u = pref exp(-3 r^2 / (2 s)) = pref 2^(c2 r^2),  F_i = -fc u d
//   real-space electrostatics with beta_ij, small-r series of g and h
struct PairTab {
  float pref, c2, fc, beta;
  float sg[4];
  float sh[3];
  float pad;
};
struct PairTab64 {
  double pref, expc, fc, beta;
  double sg[4];
  double sh[3];
  double pad;
};

struct SysDesc {
  // sizes
  int n, n_ext, nq_real, nq_ext;
  int geometry, precision, nbond, pad0;
  // offsets into pooled arrays
  long long bead_off;  // real-bead arrays (pos/vel: 3 per bead; force: SoA block of 3n)
  long long ext_off;   // extended-bead arrays (reals then images)
  long long q_off;     // charged-bead list
  long long img_off;   // image source list
  long long cell_off;  // cells
  long long grid_off;  // PME grid points
  long long bond_off;  // bonds
  int tw_off[3];       // twiddle tables per axis
  int bsp_off[3];      // B-spline moduli per axis
  int nstage[3];
  int radix[3][kMaxStages];
  int nc[3];
  int ncell;
  int K[3];
  int order;
  // geometry
  double box[3];
  double inv_cell[3];  // nc / L (FP64, the binning rule)
  float inv_cellf[3];  // FP32 copy (cell index away from cell faces)
  float boxf[3];
  float rc2f;          // fl(rc^2)
  float kfac[3];       // K / L
  float pad1;
  double V;
  // physics
  double A, sigma, a, lB, rc, kappa, beta;
  double gc_pref;      // A (3 / (2 pi s))^{3/2}
  double gc_expc;      // 3 / (2 s)
  double gc_fc;        // 3 / s
  double e_corr, e_self;
  double recip_scale;  // 1, or 1/2 for the image-charge geometry
  double H, wall_A, wall_s2;
  double bond_k, bond_r0;
  double dt;
  // Langevin (BAOAB) when langevin != 0: c1 = exp(-gamma dt),
  // c2 = sqrt((1 - c1^2) kT); noise keyed by seed
  double lgv_c1, lgv_c2;
  unsigned long long seed;
  int langevin;
  int ntypes;          // species of this system (several-species engines; else 0)
  int frozen_mask;     // bit t: beads of species t do not move
  int pair_nelec;      // electrostatics warps of a packed pair CTA (1 to 3)
  long long tab_off;   // its ntypes x ntypes block of the pooled pair tables
  // real-space table (FP32 one-species engines): 2 * rtab_n float4 from
  // rtab_off of Pool::rtab, interval k of u = r^2 at u * rtab_scale in [k, k+1)
  long long rtab_off;
  float rtab_scale;    // rtab_n / fl(rc^2)
  int rtab_n;
  // real-space kernel constants: small-r Taylor series of
  //   g(r) = [erf(beta r) - erf(kappa r)] / r        = sum_k ser_g[k] r^{2k}
  //   h(r) = -g'(r) / r                               = sum_k ser_h[k] r^{2k}
  double ser_g[4], ser_h[3];
  float ser_gf[4], ser_hf[3];
  float betaf, kappaf;
  float gc_c2f;        // -3/(2 s) log2(e): exponent of the core in base 2
  // 1 when the core term at rc is below 1e-10 of its contact value: the FP32
  // one-species kernel then sums the core over every staged neighbour bead
  // (the beads beyond rc add terms below the FP32 rounding of the sums)
  // instead of testing r < rc per candidate
  int gc_tail;
  // FP32 copies for the FP32 kernels (no FP64 arithmetic per thread)
  float gc_forcef;     // gc_fc gc_pref
  float gc_halfpref;   // gc_pref / 2
  float lbf, lb_half;  // lB, lB / 2
  float pme_cpref;     // lB / (pi V)
  float pme_pi2k2;     // pi^2 / kappa^2
  float inv_box[3];    // 1 / L
  float recip_scalef;
  float half_dtf;      // dt / 2
  float bond_kf, bond_r0f;
  // cell decomposition: cells of side >= rc / cell_factor; with factor 2 the
  // pair kernel works on blocks of 2 x 2 x 2 cells (nb blocks per axis)
  int cell_factor;
  int pair_split;      // work items per home cell: 3 (9 neighbour cells each) or 9 (3 each)
  int pair_group;      // CTA items of split 9: consecutive home cells along x per item (1-3)
  int pair_nch;        // warp items: items per (home cell, part), each taking every
                       // pair_nch-th chunk of 32 home beads (1 for CTA items)
  int nb[3];
  float cside[3];      // cell side L / nc (FP32, for bounding-box culling)
  float cull2;         // (rc + 1e-3)^2: cells farther than this are skipped
  float rl2f;          // (rc + skin)^2: neighbour-list cutoff
  // The list kernel rounds every pair term to a multiple of 2^-fix_bits and
  // sums integers, so the sums do not depend on the order of the terms;
  // fix_bits is the largest b with every pair force, energy and virial term
  // below 2^30 / 2^b (a bound from the potentials' maxima over r <= rc).
  float fix_scale;     // 2^fix_bits
  int fix_bits;
  int pad3;
};

// Pooled device arrays.  Passed by value to every kernel.
struct Pool {
  const SysDesc *sys;
  int nsys;
  int any_slab;         // some system is a slab (walls, dipole term, images)
  // state (real beads)
  double *pos;          // [3 * N] FP64
  const double *q;      // [N] charge numbers z_i of the real beads
  void *vel;            // [3 * N] FP32 or FP64
  long long *force;     // per system: SoA block [3 n]
  // extended beads
  float4 *xyzq_u;       // wrapped FP32 position + charge, ext order
  dpos4 *xyzq_u64;    // wrapped FP64 position + charge (FP64 path)
  int *cell_of;
  int *slot;
  int *sorted_idx;      // local ext index per sorted slot
  int *sort_tmp;        // scratch for oversized cells
  float4 *xyzq_s;       // sorted FP32
  dpos4 *xyzq_s64;    // sorted FP64 (FP64 path)
  int *ext_sys;         // system of each ext bead
  int *real_sys;        // system of each real bead
  int *qlist;           // local ext index of each charged bead (reals first, then images)
  int *q_sys;
  int *img_src;         // local real index of each image
  int *ext_src;         // pooled real bead giving each ext bead's position (images: -1 - it)
  // cells
  int *cell_cnt;
  int *cell_start;      // global (pooled) sorted offsets
  int *cell_nimg;
  int *cell_nq;
  int *cell_sys;
  // fused cell sort (small cell grids): bead e of cell c at bucket[c * bucket_cap
  // + slot] for slot < bucket_cap, as e | class << 30 (class 0 image, 1 charged
  // real, 2 neutral real), its wrapped FP32 position and charge at the same
  // place of bucket_pos; null: scan + scatter + sort kernels
  int *bucket;
  float4 *bucket_pos;
  int bucket_cap;
  int *wrap_n;          // [3 * n_ext] periodic image index of each coordinate at the last binning
  // PME
  unsigned long long *qgrid;  // fixed-point charge grid
  float2 *cgrid;              // complex grid (FP32 path)
  double2 *cgrid64;           // complex grid (FP64 path)
  const float4 *rtab;         // real-space g, h tables (FP32 one species), else null
  float2 *tw;                 // twiddles e^{-2 pi i t/K}
  double2 *tw64;
  float *bsp;                 // |b(m)|^2
  double *bsp64;
  // bonds
  int2 *bonds;
  int *bond_sys;
  // accumulators
  unsigned long long *acc;    // [nsys * kNacc]
  unsigned long long *vacc;   // [nsys * 9]
  double *energy;             // [nsys * GCME_NTERMS]
  double *virial;             // [nsys * 9]
  // totals
  long long n_real, n_ext, n_cells, n_q, n_bond;
  long long n_grid;
  // debug pair dump
  int *dbg_triples;
  long long dbg_cap;
  // Verlet neighbour list (FP32 path).  Entry m of sorted slot g sits at
  // nbr[((m / 4) * n_ext + g) * 4 + m % 4] (lane m % 4 of the bead's four
  // takes it): sorted slot j | (n_x+1 | (n_y+1) << 2 | (n_z+1) << 4) << 25 |
  // (j is an image) << 31, the charged and image j first.
  int *nbr;
  int *nbr_cnt;        // [n_ext] entries of each slot
  int *nbr_nq;         // [n_ext] of which charged or image (the first ones)
  int nbr_stride;      // entries per lane (a bead holds at most 4 x stride)
  int pad4;
  int *img_now;        // [3 n_ext] periodic image index of each bead this step
  int *img_ref;        // [3 n_ext] the same at the last list build
  int *dimg_s;         // per sorted slot: packed image change since the build
  double *x_ref;       // [3 n_real] unwrapped positions at the last build
  int *list_flags;     // [0] rebuild this step, [1] rebuild requested, [2] builds so far
  int *list_ovf;       // [2 nsys] per system: list overflowed (cell kernel), next build's
  const int *gate;     // if set, the cell-sort kernels run only when *gate != 0
  double half_skin2;   // (skin / 2)^2: displacement that forces a rebuild
  unsigned long long *step_ctr;  // [nsys] steps taken by each system (Langevin counter)
  // Per-system step limits (the server's pooled engines; null elsewhere): a
  // system whose step counter has reached step_stop[s] is held (the half
  // kick and drift clears its forces but moves nothing, the second half kick
  // leaves its velocities and its counter), while the others step on;
  // held[s] carries the decision of the step's first kernel to its last.
  const unsigned long long *step_stop;
  unsigned char *held;
  // several species: species of each ext bead (images: their source's),
  // the same in sorted order, and the pooled per-system pair tables
  unsigned char *type_u;
  unsigned char *type_s;
  const PairTab *ptab;
  const PairTab64 *ptab64;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_k (kernels.h)
// may start while its predecessor in the stream finishes.  pdl_wait() blocks
// until that predecessor grid has completed and its writes are visible (a
// no-op for a plain launch), so every kernel calls it before touching
// memory; pdl_trigger() lets the next kernel's launch begin now (else it
// begins when this grid's blocks have exited).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_begin() {
  pdl_wait();
  pdl_trigger();
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Real-space pair functions g(r) = [erf(beta r) - erf(kappa r)] / r and
// h(r) = -g'(r) / r at u = r^2 < rc^2 from the system's cubic table in u
// (Pool::rtab; 2 float4 per interval: g's then h's coefficients in t).
__device__ __forceinline__ void real_gh_tab(const float4 *__restrict__ tab, float scale,
                                            int nm1, float r2, float &g, float &h) {
  const float x = r2 * scale;
  const int k = min((int)x, nm1);
  const float t = x - (float)k;
  const float4 a = __ldg(tab + 2 * k), b = __ldg(tab + 2 * k + 1);
  g = fmaf(t, fmaf(t, fmaf(t, a.w, a.z), a.y), a.x);
  h = fmaf(t, fmaf(t, fmaf(t, b.w, b.z), b.y), b.x);
}
__device__ __forceinline__ void real_gh_tab(const Pool &P, const SysDesc &S, float r2, float &g,
                                            float &h) {
  real_gh_tab(P.rtab + S.rtab_off, S.rtab_scale, S.rtab_n - 1, r2, g, h);
}

__device__ __forceinline__ void atomic_add_fixed(unsigned long long *p, double v, double scale) {
  long long q = __double2ll_rn(v * scale);
  atomicAdd(p, (unsigned long long)q);
}

// Round-to-nearest-even of v as a 64-bit integer (|v| < 2^63), equal to
// __float2ll_rn(v) but from 32-bit conversions: the FP64 pipe, which the
// 64-bit conversions use, is a small fraction of the FP32 rate.  With
// a = |v| = h 2^32 + r, h = floor(a / 2^32) and r = a - h 2^32 are exact
// floats (r < 2^32 is a multiple of ulp(a)), so rounding r alone rounds a.
__device__ __forceinline__ long long f2ll_rn(float v) {
  const float a = fabsf(v);
  const float h = floorf(a * 2.3283064365386963e-10f);  // a / 2^32, exact
  const float r = fmaf(-h, 4294967296.0f, a);           // exact, in [0, 2^32)
  const long long q =
      (long long)(((unsigned long long)__float2uint_rn(h) << 32) + __float2uint_rn(r));
  return v < 0.0f ? -q : q;
}

// q as a float (within one rounding of the nearest float) from 32-bit
// conversions: |q| = h 2^32 + l, the high word converted exactly and the low
// word rounded once (error <= 128 <= 2^-25 |q| when h > 0; exact rounding
// when h = 0).
__device__ __forceinline__ float ll2f(long long q) {
  const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
  const float f = fmaf(__uint2float_rn((unsigned)(a >> 32)), 4294967296.0f,
                       __uint2float_rn((unsigned)(a & 0xffffffffull)));
  return q < 0 ? -f : f;
}

__device__ __forceinline__ void atomic_add_fixed_f(unsigned long long *p, float v, float scale) {
  atomicAdd(p, (unsigned long long)f2ll_rn(v * scale));
}

// Energy-scale fixed point of one term (2^32 units): terms are rounded
// before any sum, so sums of them are exact and independent of how the
// terms are grouped into threads, warps and tiles.
__device__ __forceinline__ long long efix(float v) { return f2ll_rn(v * 4294967296.0f); }
__device__ __forceinline__ long long efix(double v) { return __double2ll_rn(v * kEScale); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Wrap one coordinate into [0, L): x - L floor(x/L), each operation rounded
// once (no contraction); a result of L (or below 0) maps to 0.
__device__ __forceinline__ double wrap_coord(double x, double L) {
  double s = __ddiv_rn(x, L);
  double f = floor(s);
  double t = __dmul_rn(L, f);
  double w = __dsub_rn(x, t);
  if (w >= L) w = 0.0;
  if (w < 0.0) w = 0.0;
  return w;
}

// The same wrap with the image index f = floor(x / L) it used.
__device__ __forceinline__ double wrap_coord_n(double x, double L, double &f) {
  f = floor(__ddiv_rn(x, L));
  double w = __dsub_rn(x, __dmul_rn(L, f));
  if (w >= L) w = 0.0;
  if (w < 0.0) w = 0.0;
  return w;
}

__device__ __forceinline__ int floor_div(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// Load a bead position of the extended system: reals from the caller's
// array, images mirrored in z.
__device__ __forceinline__ void ext_position(const Pool &P, const SysDesc &S, int e,
                                             double &x, double &y, double &z) {
  if (e < S.n) {
    const double *p = P.pos + 3 * (S.bead_off + e);
    x = p[0];
    y = p[1];
    z = p[2];
  } else {
    int src = P.img_src[S.img_off + (e - S.n)];
    const double *p = P.pos + 3 * (S.bead_off + src);
    x = p[0];
    y = p[1];
    z = -p[2];
  }
}

__device__ __forceinline__ double ext_charge(const Pool &P, const SysDesc &S, int e) {
  if (e < S.n) return P.q[S.bead_off + e];
  return -P.q[S.bead_off + P.img_src[S.img_off + (e - S.n)]];
}

// fixed-point force array of a system: SoA block
__device__ __forceinline__ unsigned long long *force_ptr(const Pool &P, const SysDesc &S, int i,
                                                         int axis) {
  return reinterpret_cast<unsigned long long *>(P.force + 3 * S.bead_off + (long long)axis * S.n +
                                                i);
}

}  // namespace gcme
