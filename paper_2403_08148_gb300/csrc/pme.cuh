// pme.cuh -- K5-K8 device bodies: smooth particle-mesh Ewald for the reciprocal term of
// Eq. ewald (Essmann et al. 1995), orthorhombic boxes, order p B-splines.
//
//   u_a = K_a x_a / L_a
//   Q(k) = sum_i z_i prod_a M_p(u_ia - k_a)            (spread, periodic wrap)
//   E = 1/2 sum_{m != 0} B(m) C(m) |F(Q)(m)|^2,
//   B = prod_a |b_a(m_a)|^2,  C = lB / (pi V) exp(-pi^2 m^2 / kappa^2) / m^2
//   F_i = -sum_k dQ(k)/dr_i (theta * Q)(k),  theta * Q = F^{-1}[B C F(Q)]
// with unnormalised forward and backward transforms.
//
// GB300 layout: the charge grid is accumulated in 64-bit fixed point
// (order-independent, so the result is bit-reproducible), eight lanes per
// charge (one per z-plane of the stencil).  The 3D FFT is a batched
// mixed-radix (2, 3, 4, 5) Stockham transform along one axis per launch;
// each CTA moves a tile of lines through shared memory with coalesced loads
// (lines adjacent in x), the z pass fuses forward transform, influence
// function (energy, virial) and backward transform.
#pragma once
#include "common.cuh"


namespace gcme {

template <typename R> struct PmeT;
template <> struct PmeT<float> {
  using R2 = float2;
  static constexpr double qscale = kQScale32;
};
template <> struct PmeT<double> {
  using R2 = double2;
  static constexpr double qscale = kQScale64;
};

// fixed-point grid value -> R, and R -> nearest fixed-point integer; the
// FP32 forms use no 64-bit conversion (see f2ll_rn)
template <typename R> __device__ __forceinline__ R grid_value(long long q);
template <> __device__ __forceinline__ float grid_value<float>(long long q) {
  return ll2f(q) * (float)(1.0 / kQScale32);
}
template <> __device__ __forceinline__ double grid_value<double>(long long q) {
  return (double)q * (1.0 / kQScale64);
}
__device__ __forceinline__ long long to_fixed(float v) { return f2ll_rn(v); }
__device__ __forceinline__ long long to_fixed(double v) { return (long long)llrint(v); }

template <typename R>
__device__ __forceinline__ void load_pos(const Pool &P, long long g, R x[3], R &q);
template <>
__device__ __forceinline__ void load_pos<float>(const Pool &P, long long g, float x[3], float &q) {
  float4 p = P.xyzq_u[g];
  x[0] = p.x;
  x[1] = p.y;
  x[2] = p.z;
  q = p.w;
}
template <>
__device__ __forceinline__ void load_pos<double>(const Pool &P, long long g, double x[3], double &q) {
  dpos4 p = P.xyzq_u64[g];
  x[0] = p.x;
  x[1] = p.y;
  x[2] = p.z;
  q = p.w;
}

// Cardinal B-spline weights W[t] = M_p(fr + t), t = 0..p-1, by the recursion
// M_n(u) = [u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)] / (n - 1) from
// M_2(u) = 1 - |u - 1|; optionally dW[t] = M_{p-1}(fr+t) - M_{p-1}(fr+t-1).
template <typename R>
__device__ __forceinline__ void bspline_weights(int p, R fr, R *W, R *dW) {
  W[0] = fr;
  W[1] = R(1) - fr;
  for (int n = 3; n <= p; ++n) {
    if (n == p && dW) {
      dW[0] = W[0];
      for (int t = 1; t < n - 1; ++t) dW[t] = W[t] - W[t - 1];
      dW[n - 1] = -W[n - 2];
    }
    const R div = R(1) / R(n - 1);
    W[n - 1] = (R(1) - fr) * W[n - 2] * div;
    for (int t = n - 2; t >= 1; --t) W[t] = ((fr + R(t)) * W[t] + (R(n) - fr - R(t)) * W[t - 1]) * div;
    W[0] = fr * W[0] * div;
  }
  if (p == 2 && dW) {
    dW[0] = R(1);
    dW[1] = R(-1);
  }
}

// k mod K for -K <= k < 2K: the B-spline grid indices base - t, with base =
// floor(x K / L) in [0, K] for wrapped x and 0 <= t < p <= K.
__device__ __forceinline__ int wrap_index(int k, int K) {
  k = k < 0 ? k + K : k;
  return k >= K ? k - K : k;
}

template <typename R>
__device__ __forceinline__ R kfac_of(const SysDesc &S, int a);
template <>
__device__ __forceinline__ float kfac_of<float>(const SysDesc &S, int a) {
  return S.kfac[a];
}
template <>
__device__ __forceinline__ double kfac_of<double>(const SysDesc &S, int a) {
  return (double)S.K[a] / S.box[a];
}

// --------------------------------------------------------------------------
// spread: eight lanes per charge, lane tz handles the stencil plane tz
// --------------------------------------------------------------------------
// PO > 0: the spline order as a compile-time constant (every system of the
// launch has it), so the weight arrays and loops stay in registers.
template <typename R, int PO = 0>
__device__ __forceinline__ void dev_spread(const Pool &P, long long g) {
  const long long c = g >> 3;
  const int tz = (int)(g & 7);
  if (c >= P.n_q) return;
  const SysDesc &S = P.sys[P.q_sys[c]];
  const int p = PO > 0 ? PO : S.order;
  if (tz >= p) return;
  const int e = P.qlist[c];
  R x[3], q;
  load_pos<R>(P, S.ext_off + e, x, q);
  R W[3][8];
  int base[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R u = x[a] * kfac_of<R>(S, a);
    R fl = floor(u);
    base[a] = (int)fl;
    bspline_weights<R>(p, u - fl, W[a], (R *)nullptr);
  }
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  const int kz = wrap_index(base[2] - tz, K2);
  R w2 = W[2][0];  // W[2][tz] by a select, keeping the weights in registers
#pragma unroll
  for (int t = 1; t < 8; ++t)
    if (t < p && t == tz) w2 = W[2][t];
  const R wz = w2 * q * R(PmeT<R>::qscale);
  unsigned long long *grid = P.qgrid + S.grid_off;
#pragma unroll
  for (int ty = 0; ty < p; ++ty) {
    const int ky = wrap_index(base[1] - ty, K1);
    const R wyz = W[1][ty] * wz;
    unsigned long long *row = grid + (long long)K0 * (ky + (long long)K1 * kz);
#pragma unroll
    for (int tx = 0; tx < p; ++tx) {
      const int kx = wrap_index(base[0] - tx, K0);
      const long long v = to_fixed(W[0][tx] * wyz);
      atomicAdd(row + kx, (unsigned long long)v);
    }
  }
}

// --------------------------------------------------------------------------
// spread by cells through shared memory (FP32 path): one CTA per cell of the
// sorted cell list spreads the cell's charged and image beads into a brick
// of the grid held in shared memory with 64-bit integer atomics, then adds
// the brick's nonzero points to the global grid (one fixed-point atomic per
// point, consecutive along x).  Every contribution is rounded to fixed point
// exactly as in dev_spread and all sums are integer, so the grid is the same
// bit for bit as dev_spread's, whatever the order.  A cell with more than
// kSpreadQ charges, or whose charges span a brick larger than kSpreadBrick
// points, is spread straight to the global grid.
// --------------------------------------------------------------------------
constexpr int kSpreadQ = 128;
constexpr int kSpreadBrick = 4096;
constexpr int kSpreadMaxOrder = 8;

struct SpreadSmem {
  unsigned long long brick[kSpreadBrick];
  float w[kSpreadQ][3][kSpreadMaxOrder];
  float q[kSpreadQ];
  int base[kSpreadQ][3];
  int lo[3], hi[3];
};

template <int PO>
__device__ __forceinline__ void dev_spread_cell(const Pool &P, long long c, SpreadSmem &sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const SysDesc &S = P.sys[P.cell_sys[c]];
  const int p = PO > 0 ? PO : S.order;
  const int beg = P.cell_start[c], nq = P.cell_nq[c];  // images and charged reals
  if (nq == 0) return;
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  unsigned long long *grid = P.qgrid + S.grid_off;
  const float scale = (float)PmeT<float>::qscale;
  if (nq > kSpreadQ) {  // straight to the global grid, one thread per (charge, z-plane)
    for (int idx = tid; idx < nq * p; idx += nt) {
      const int k = idx / p, tz = idx - k * p;
      const float4 v = P.xyzq_s[beg + k];
      const float x[3] = {v.x, v.y, v.z};
      float W[3][kSpreadMaxOrder];
      int b[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float u = x[a] * S.kfac[a];
        const float fl = floorf(u);
        b[a] = (int)fl;
        bspline_weights<float>(p, u - fl, W[a], (float *)nullptr);
      }
      const float wz = W[2][tz] * v.w * scale;
      const int kz = wrap_index(b[2] - tz, K2);
      for (int ty = 0; ty < p; ++ty) {
        const float wyz = W[1][ty] * wz;
        unsigned long long *row = grid + (long long)K0 * (wrap_index(b[1] - ty, K1) + (long long)K1 * kz);
        for (int tx = 0; tx < p; ++tx)
          atomicAdd(row + wrap_index(b[0] - tx, K0), (unsigned long long)to_fixed(W[0][tx] * wyz));
      }
    }
    return;
  }
  if (tid < 3) {
    sm.lo[tid] = 1 << 30;
    sm.hi[tid] = -(1 << 30);
  }
  __syncthreads();
  for (int k = tid; k < nq; k += nt) {  // weights and bases of each charge
    const float4 v = P.xyzq_s[beg + k];
    const float x[3] = {v.x, v.y, v.z};
    sm.q[k] = v.w;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float u = x[a] * S.kfac[a];
      const float fl = floorf(u);
      const int b = (int)fl;
      sm.base[k][a] = b;
      bspline_weights<float>(p, u - fl, sm.w[k][a], (float *)nullptr);
      atomicMin(&sm.lo[a], b);
      atomicMax(&sm.hi[a], b);
    }
  }
  __syncthreads();
  // brick: grid points base - t (t < p) of every charge, from lo - (p - 1)
  const int E0 = sm.hi[0] - sm.lo[0] + p, E1 = sm.hi[1] - sm.lo[1] + p,
            E2 = sm.hi[2] - sm.lo[2] + p;
  const int o0 = sm.lo[0] - (p - 1), o1 = sm.lo[1] - (p - 1), o2 = sm.lo[2] - (p - 1);
  const int npts = E0 * E1 * E2;
  if (npts > kSpreadBrick) {  // charges spread over a wide brick: global atomics
    for (int idx = tid; idx < nq * p * p * p; idx += nt) {
      const int k = idx / (p * p * p), r = idx - k * p * p * p;
      const int tz = r / (p * p), ty = (r / p) % p, tx = r % p;
      const float wyz = sm.w[k][1][ty] * (sm.w[k][2][tz] * sm.q[k] * scale);
      const long long gi = wrap_index(sm.base[k][0] - tx, K0) +
                           (long long)K0 * (wrap_index(sm.base[k][1] - ty, K1) +
                                            (long long)K1 * wrap_index(sm.base[k][2] - tz, K2));
      atomicAdd(grid + gi, (unsigned long long)to_fixed(sm.w[k][0][tx] * wyz));
    }
    return;
  }
  for (int i = tid; i < npts; i += nt) sm.brick[i] = 0ull;
  __syncthreads();
  for (int idx = tid; idx < nq * p * p * p; idx += nt) {
    const int k = idx / (p * p * p), r = idx - k * p * p * p;
    const int tz = r / (p * p), ty = (r / p) % p, tx = r % p;
    // the same roundings as dev_spread: (W_x (W_y (W_z q scale)))
    const float wyz = sm.w[k][1][ty] * (sm.w[k][2][tz] * sm.q[k] * scale);
    const int li = (sm.base[k][0] - tx - o0) + E0 * ((sm.base[k][1] - ty - o1) +
                                                      E1 * (sm.base[k][2] - tz - o2));
    atomicAdd(&sm.brick[li], (unsigned long long)to_fixed(sm.w[k][0][tx] * wyz));
  }
  __syncthreads();
  for (int i = tid; i < npts; i += nt) {
    const unsigned long long v = sm.brick[i];
    if (v == 0ull) continue;
    const int ex = i % E0, ey = (i / E0) % E1, ez = i / (E0 * E1);
    const long long gi = wrap_index(o0 + ex, K0) +
                         (long long)K0 * (wrap_index(o1 + ey, K1) + (long long)K1 * wrap_index(o2 + ez, K2));
    atomicAdd(grid + gi, v);
  }
}

// --------------------------------------------------------------------------
// gather: eight lanes per charged real bead, reduced with shuffles
// --------------------------------------------------------------------------
// Warp-synchronous: every lane of the warp must call it (lanes past the end
// pass g beyond the last charge and contribute nothing).
template <typename R, int PO = 0>
__device__ __forceinline__ void dev_gather(const Pool &P, long long g) {
  using R2 = typename PmeT<R>::R2;
  const long long c = g >> 3;
  const int tz = (int)(g & 7);
  bool act = c < P.n_q;
  const SysDesc *Sp = act ? &P.sys[P.q_sys[c]] : &P.sys[0];
  const SysDesc &S = *Sp;
  const int p = PO > 0 ? PO : S.order;
  int e = 0;
  if (act) {
    const long long loc = c - S.q_off;
    act = loc < S.nq_real && tz < p;
    e = P.qlist[c];
  }
  R gx = 0, gy = 0, gz = 0, q = 0;
  if (act) {
    R x[3];
    load_pos<R>(P, S.ext_off + e, x, q);
    R W[3][8], dW[3][8];
    int base[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R u = x[a] * kfac_of<R>(S, a);
      R fl = floor(u);
      base[a] = (int)fl;
      bspline_weights<R>(p, u - fl, W[a], dW[a]);
    }
    const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
    const int kz = wrap_index(base[2] - tz, K2);
    const R2 *grid = (const R2 *)(sizeof(R) == 4 ? (const void *)P.cgrid : (const void *)P.cgrid64) +
                     S.grid_off;
    R wz = W[2][0], dwz = dW[2][0];  // W[2][tz], dW[2][tz] by a select
#pragma unroll
    for (int t = 1; t < 8; ++t)
      if (t < p && t == tz) {
        wz = W[2][t];
        dwz = dW[2][t];
      }
#pragma unroll
    for (int ty = 0; ty < p; ++ty) {
      const int ky = wrap_index(base[1] - ty, K1);
      const R2 *row = grid + (long long)K0 * (ky + (long long)K1 * kz);
      R sx = 0, sy = 0, sz = 0;
#pragma unroll
      for (int tx = 0; tx < p; ++tx) {
        const R v = row[wrap_index(base[0] - tx, K0)].x;
        sx += dW[0][tx] * v;
        sy += W[0][tx] * v;
      }
      sz = sy;
      gx += sx * W[1][ty] * wz;
      gy += sy * dW[1][ty] * wz;
      gz += sz * W[1][ty] * dwz;
    }
    gx *= kfac_of<R>(S, 0);
    gy *= kfac_of<R>(S, 1);
    gz *= kfac_of<R>(S, 2);
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
    gz += __shfl_xor_sync(0xffffffffu, gz, o);
  }
  if (act && tz == 0) {
    if (sizeof(R) == 4) {
      atomic_add_fixed_f(force_ptr(P, S, e, 0), (float)(-q * gx), (float)kFScale);
      atomic_add_fixed_f(force_ptr(P, S, e, 1), (float)(-q * gy), (float)kFScale);
      atomic_add_fixed_f(force_ptr(P, S, e, 2), (float)(-q * gz), (float)kFScale);
    } else {
      atomic_add_fixed(force_ptr(P, S, e, 0), (double)(-q * gx), kFScale);
      atomic_add_fixed(force_ptr(P, S, e, 1), (double)(-q * gy), kFScale);
      atomic_add_fixed(force_ptr(P, S, e, 2), (double)(-q * gz), kFScale);
    }
  }
}

// --------------------------------------------------------------------------
// batched mixed-radix Stockham FFT along one axis
// --------------------------------------------------------------------------
template <typename R2>
__device__ __forceinline__ R2 cmul(R2 a, R2 b) {
  R2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename R2>
__device__ __forceinline__ R2 cadd(R2 a, R2 b) {
  R2 r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename R2>
__device__ __forceinline__ R2 csub(R2 a, R2 b) {
  R2 r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
// multiply by -i (forward) or +i (inverse): sgn = -1 forward, +1 inverse
template <typename R2>
__device__ __forceinline__ R2 mul_i(R2 a, int sgn) {
  R2 r;
  if (sgn < 0) {
    r.x = a.y;
    r.y = -a.x;
  } else {
    r.x = -a.y;
    r.y = a.x;
  }
  return r;
}

// Small DFTs b_q = sum_r v_r exp(sgn 2 pi i r q / R).
template <typename R, typename R2>
__device__ __forceinline__ void dft_small(R2 *v, int Rd, int sgn) {
  if (Rd == 2) {
    R2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (Rd == 4) {
    R2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    R2 b0 = cadd(v[1], v[3]), b1 = mul_i(csub(v[1], v[3]), sgn);
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, b1);
    v[3] = csub(a1, b1);
  } else if (Rd == 3) {
    const R c = R(-0.5), sn = R(0.86602540378443864676);
    R2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    R2 m;
    m.x = v[0].x + c * t1.x;
    m.y = v[0].y + c * t1.y;
    R2 u = mul_i(t2, sgn);  // sgn i t2
    u.x *= sn;
    u.y *= sn;
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, u);
    v[2] = csub(m, u);
  } else if (Rd == 5) {
    const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
    const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
    R2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    R2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    R2 a1, a2, b1, b2;
    a1.x = v[0].x + c1 * t1.x + c2 * t2.x;
    a1.y = v[0].y + c1 * t1.y + c2 * t2.y;
    a2.x = v[0].x + c2 * t1.x + c1 * t2.x;
    a2.y = v[0].y + c2 * t1.y + c1 * t2.y;
    R2 s1v, s2v;
    s1v.x = s1 * t3.x + s2 * t4.x;
    s1v.y = s1 * t3.y + s2 * t4.y;
    s2v.x = s2 * t3.x - s1 * t4.x;
    s2v.y = s2 * t3.y - s1 * t4.y;
    b1 = mul_i(s1v, sgn);
    b2 = mul_i(s2v, sgn);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
}

// One radix-RD butterfly of a Stockham stage: inputs in[r * is], r < RD,
// times the twiddles w^(k r) (w = tw[twstep], conjugated for sgn > 0), a
// length-RD DFT, outputs out[q * os].  RD is a compile-time constant so the
// values stay in registers.
template <typename R, typename R2, int RD>
__device__ __forceinline__ void butterfly(const R2 *in, int is, R2 *out, int os, const R2 *tw,
                                          int k, int twstep, int sgn) {
  R2 v[RD];
#pragma unroll
  for (int r = 0; r < RD; ++r) {
    R2 x = in[r * is];
    if (r > 0 && k > 0) {
      R2 wv = tw[k * r * twstep];  // k r twstep < K: no wrap needed
      if (sgn > 0) wv.y = -wv.y;
      x = cmul(x, wv);
    }
    v[r] = x;
  }
  dft_small<R, R2>(v, RD, sgn);
#pragma unroll
  for (int q = 0; q < RD; ++q) out[q * os] = v[q];
}

template <typename R, typename R2>
__device__ __forceinline__ void butterfly_rd(int Rd, const R2 *in, int is, R2 *out, int os,
                                             const R2 *tw, int k, int twstep, int sgn) {
  switch (Rd) {
    case 4: butterfly<R, R2, 4>(in, is, out, os, tw, k, twstep, sgn); break;
    case 2: butterfly<R, R2, 2>(in, is, out, os, tw, k, twstep, sgn); break;
    case 3: butterfly<R, R2, 3>(in, is, out, os, tw, k, twstep, sgn); break;
    default: butterfly<R, R2, 5>(in, is, out, os, tw, k, twstep, sgn); break;
  }
}

// Quotient a / d for 0 <= a < 2^22 and 1 <= d <= 2^12, from the FP32
// product a * inv (inv = 1/d rounded): its error is below one unit for these
// ranges, so one correction step gives the exact quotient.  Replaces integer
// division by a runtime divisor in the FFT index arithmetic.
__device__ __forceinline__ int qdiv(int a, int d, float inv) {
  int q = (int)__fmul_rn((float)a, inv);
  const int r = a - q * d;
  q += (r >= d) - (r < 0);
  return q;
}

// index of element k of line l of a K0 x K1 x K2 grid along `axis`
// (lines along y: l = x + K0 z; inv0 = 1/K0)
__device__ __forceinline__ long long line_elem(int axis, int K0, int K1, int l, int k,
                                               float inv0) {
  if (axis == 0) return k + (long long)K0 * l;
  if (axis == 1) {
    const int z = qdiv(l, K0, inv0);
    return (l - z * K0) + (long long)K0 * (k + (long long)K1 * z);
  }
  return l + (long long)K0 * K1 * k;
}

enum { FFT_FWD_FROM_Q = 0, FFT_FWD = 1, FFT_FWD_INFL_INV = 2, FFT_INV = 3 };

// Stockham transform of nl lines of length K held in shared memory, element
// k of line l at A[l * ls + k * es] (the result uses the same layout).
// Threads run line-fastest when lines are adjacent (ls == 1) and
// element-fastest otherwise, so that a warp touches consecutive words.
// Ping-pongs between A and B; returns the buffer holding the result.  All
// threads of the CTA take part; every stage ends with a barrier.
template <typename R, typename R2>
__device__ __forceinline__ R2 *smem_fft(R2 *A, R2 *B, int nl, int K, int ls, int es,
                                        const int *radix, int nstage, const R2 *tw, int sgn) {
  const bool line_fast = ls == 1;
  const float inv_nl = 1.0f / (float)nl;
  int Ns = 1;
  for (int st = 0; st < nstage; ++st) {
    const int Rd = radix[st];
    const int T = K / Rd;
    const int twstep = K / (Ns * Rd);
    const float inv_T = 1.0f / (float)T, inv_Ns = 1.0f / (float)Ns;
    for (int t = threadIdx.x; t < nl * T; t += blockDim.x) {
      int li, j;
      if (line_fast) {
        j = qdiv(t, nl, inv_nl);
        li = t - j * nl;
      } else {
        li = qdiv(t, T, inv_T);
        j = t - li * T;
      }
      const int jq = qdiv(j, Ns, inv_Ns);
      const int k = j - jq * Ns;
      const int od = jq * Ns * Rd + k;
      butterfly_rd<R, R2>(Rd, A + li * ls + j * es, T * es, B + li * ls + od * es, Ns * es, tw, k,
                          twstep, sgn);
    }
    __syncthreads();
    R2 *tmp = A;
    A = B;
    B = tmp;
    Ns *= Rd;
  }
  return A;
}

// Two z-planes (x and y passes) of one system by the whole CTA, packed as
// the real and imaginary parts of one complex plane (both planes are real in
// position space).  Work item (s, p) covers planes 2p and 2p + 1 (the
// second absent when K2 is odd and 2p + 1 = K2).
//
// Forward (INV = false): Z = FFT2(q_2p + i q_2p+1) from the fixed-point
// charge grid, then X(k) = (Z(k) + conj Z(-k)) / 2 and
// Y(k) = (Z(k) - conj Z(-k)) / (2i) are the spectra of the two planes; only
// the half k0 < K0/2 + 1 is stored (Hermitian symmetry gives the rest), at
// the usual positions of each plane.
// Backward (INV = true): the half spectra X, Y of planes 2p, 2p + 1 (z
// pass done) are completed by X(k) = conj X(-k) for k0 >= K0/2 + 1, and
// the inverse FFT2 of X + i Y gives plane 2p in its real part and plane
// 2p + 1 in its imaginary part, written as real values (imaginary 0).
// smem: 2 * K0 * K1 + K0 + K1 complex values (two plane buffers, then the x
// and y twiddle tables).  Ends with a barrier.
template <typename R, bool INV>
__device__ __forceinline__ void dev_fft_plane(const Pool &P, const int2 *work, int w,
                                              unsigned char *smem_raw) {
  using R2 = typename PmeT<R>::R2;
  R2 *smem = reinterpret_cast<R2 *>(smem_raw);
  R2 *cg_all = (R2 *)(sizeof(R) == 4 ? (void *)P.cgrid : (void *)P.cgrid64);
  const R2 *tw_all = (const R2 *)(sizeof(R) == 4 ? (const void *)P.tw : (const void *)P.tw64);
  const int s = work[w].x, zp = work[w].y;
  const SysDesc &S = P.sys[s];
  const int K0 = S.K[0], K1 = S.K[1];
  const int G2 = K0 * K1, H0 = K0 / 2 + 1;
  const bool two = 2 * zp + 1 < S.K[2];
  const long long base0 = S.grid_off + (long long)(2 * zp) * G2;
  const long long base1 = base0 + G2;
  const float inv_K0 = 1.0f / (float)K0, inv_H0 = 1.0f / (float)H0;
  R2 *A = smem, *B = smem + G2;
  R2 *tw0 = smem + 2 * G2, *tw1 = tw0 + K0;
  for (int t = threadIdx.x; t < K0; t += blockDim.x) tw0[t] = tw_all[S.tw_off[0] + t];
  for (int t = threadIdx.x; t < K1; t += blockDim.x) tw1[t] = tw_all[S.tw_off[1] + t];
  // kPlaneLoads elements per thread in flight: their global loads are
  // issued together, then converted and stored to shared memory
  constexpr int kPlaneLoads = 4;
  for (int t0 = threadIdx.x; t0 < G2; t0 += kPlaneLoads * blockDim.x) {
    R2 X[kPlaneLoads], Y[kPlaneLoads];
    long long qa[kPlaneLoads], qb[kPlaneLoads];
#pragma unroll
    for (int u = 0; u < kPlaneLoads; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t >= G2) break;
      if (INV) {
        const int i1 = qdiv(t, K0, inv_K0), i0 = t - i1 * K0;
        // stored half, or the conjugate of its mirror
        const int m = i0 < H0 ? t : (K0 - i0) + K0 * (i1 == 0 ? 0 : K1 - i1);
        X[u] = cg_all[base0 + m];
        if (two) Y[u] = cg_all[base1 + m];
      } else {
        qa[u] = (long long)P.qgrid[base0 + t];
        qb[u] = two ? (long long)P.qgrid[base1 + t] : 0ll;
      }
    }
#pragma unroll
    for (int u = 0; u < kPlaneLoads; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t >= G2) break;
      R2 v;
      if (INV) {
        const int i0 = t - qdiv(t, K0, inv_K0) * K0;
        R2 x = X[u], y;
        if (two) y = Y[u];
        else y.x = y.y = R(0);
        if (i0 >= H0) {
          x.y = -x.y;
          y.y = -y.y;
        }
        v.x = x.x - y.y;  // X + i Y
        v.y = x.y + y.x;
      } else {  // and leave the grid zero for the next spread
        v.x = grid_value<R>(qa[u]);
        v.y = two ? grid_value<R>(qb[u]) : R(0);
        P.qgrid[base0 + t] = 0ull;
        if (two) P.qgrid[base1 + t] = 0ull;
      }
      A[t] = v;
    }
  }
  __syncthreads();
  const int sgn = INV ? +1 : -1;
  R2 *res;
  if (!INV) {
    res = smem_fft<R, R2>(A, B, K1, K0, K0, 1, S.radix[0], S.nstage[0], tw0, sgn);
    R2 *other = res == smem ? smem + G2 : smem;
    res = smem_fft<R, R2>(res, other, K0, K1, 1, K0, S.radix[1], S.nstage[1], tw1, sgn);
    for (int t = threadIdx.x; t < H0 * K1; t += blockDim.x) {
      const int i1 = qdiv(t, H0, inv_H0), i0 = t - i1 * H0;
      const R2 Z = res[i0 + K0 * i1];
      const R2 Zm = res[(i0 == 0 ? 0 : K0 - i0) + K0 * (i1 == 0 ? 0 : K1 - i1)];
      R2 X, Y;
      X.x = R(0.5) * (Z.x + Zm.x);
      X.y = R(0.5) * (Z.y - Zm.y);
      cg_all[base0 + i0 + K0 * i1] = X;
      if (two) {
        Y.x = R(0.5) * (Z.y + Zm.y);
        Y.y = R(0.5) * (Zm.x - Z.x);
        cg_all[base1 + i0 + K0 * i1] = Y;
      }
    }
  } else {
    res = smem_fft<R, R2>(A, B, K0, K1, 1, K0, S.radix[1], S.nstage[1], tw1, sgn);
    R2 *other = res == smem ? smem + G2 : smem;
    res = smem_fft<R, R2>(res, other, K1, K0, K0, 1, S.radix[0], S.nstage[0], tw0, sgn);
    for (int t = threadIdx.x; t < G2; t += blockDim.x) {
      const R2 z = res[t];
      R2 a, b;
      a.x = z.x;
      b.x = z.y;
      a.y = b.y = R(0);
      cg_all[base0 + t] = a;
      if (two) cg_all[base1 + t] = b;
    }
  }
  __syncthreads();
}

// One tile of lpb lines of one system along `axis` by the whole CTA (any
// block size).  half (z lines only): the grid holds the Hermitian half
// k0 < K0/2 + 1 of every z-plane's spectrum (the packed plane passes), so
// only those (K0/2 + 1) K1 lines exist; line l maps to k0 = l mod (K0/2 + 1),
// k1 = l div (K0/2 + 1), and the spectrum's energy and virial count each
// line with its mirror (weight 2 unless k0 = 0 or 2 k0 = K0).  smem: (2 * lpb + 1) * kmax complex values (two line buffers,
// then the axis' twiddle table).  Ends with a barrier.
template <typename R, bool VIR>
__device__ __forceinline__ void dev_fft_item(const Pool &P, const int2 *work, int w, int axis,
                                             int kind, int lpb, int half,
                                             unsigned char *smem_raw) {
  using R2 = typename PmeT<R>::R2;
  R2 *smem = reinterpret_cast<R2 *>(smem_raw);
  R2 *cg_all = (R2 *)(sizeof(R) == 4 ? (void *)P.cgrid : (void *)P.cgrid64);
  const R2 *tw_all = (const R2 *)(sizeof(R) == 4 ? (const void *)P.tw : (const void *)P.tw64);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int s = work[w].x, tile = work[w].y;
  const SysDesc &S = P.sys[s];
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  const int K = S.K[axis];
  half = half && axis == 2;
  const int H0 = half ? K0 / 2 + 1 : K0;  // stored k0 extent of a z-plane
  const int nlines = H0 * K1 * K2 / K;
  const int l0 = tile * lpb;
  const int nl = min(lpb, nlines - l0);
  const float inv_K = 1.0f / (float)K, inv_nl = 1.0f / (float)nl, inv_K0 = 1.0f / (float)K0;
  const float inv_H0 = 1.0f / (float)H0;
  // full-grid line index of tile line li (identity unless half)
  auto full_line = [&](int li) {
    const int l = l0 + li;
    if (!half) return l;
    const int i1 = qdiv(l, H0, inv_H0);
    return (l - i1 * H0) + K0 * i1;
  };
  R2 *grid = cg_all + S.grid_off;
  R2 *bufA = smem, *bufB = smem + lpb * K;
  R2 *tws = smem + 2 * lpb * K;
  for (int t = tid; t < K; t += nt) tws[t] = tw_all[S.tw_off[axis] + t];
  // ---- load (line index fastest for strided axes: coalesced along x);
  // kItemLoads elements per thread in flight, then stored to shared memory
  constexpr int kItemLoads = 4;
  for (int t0 = tid; t0 < nl * K; t0 += kItemLoads * nt) {
    R2 v[kItemLoads];
    int dst[kItemLoads];
    long long gq[kItemLoads], gidx[kItemLoads];
#pragma unroll
    for (int u = 0; u < kItemLoads; ++u) {
      const int t = t0 + u * nt;
      if (t >= nl * K) break;
      int li, k;
      if (axis == 0) {
        li = qdiv(t, K, inv_K);
        k = t - li * K;
      } else {
        k = qdiv(t, nl, inv_nl);
        li = t - k * nl;
      }
      dst[u] = li * K + k;
      const long long gi = line_elem(axis, K0, K1, full_line(li), k, inv_K0);
      gidx[u] = S.grid_off + gi;
      if (kind == FFT_FWD_FROM_Q) gq[u] = (long long)P.qgrid[gidx[u]];
      else v[u] = grid[gi];
    }
#pragma unroll
    for (int u = 0; u < kItemLoads; ++u) {
      if (t0 + u * nt >= nl * K) break;
      if (kind == FFT_FWD_FROM_Q) {  // and leave the grid zero for the next spread
        v[u].x = grid_value<R>(gq[u]);
        v[u].y = R(0);
        P.qgrid[gidx[u]] = 0ull;
      }
      bufA[dst[u]] = v[u];
    }
  }
  __syncthreads();
  const R2 *tw = tws;
  // one or two passes of stages (forward, then backward for the fused z pass)
  const int npass = (kind == FFT_FWD_INFL_INV) ? 2 : 1;
  // spectrum energy and virial: every mode's term in fixed point, summed as
  // integers (no FP64 arithmetic in FP32 kernels, and sums independent of
  // the tiling)
  R sc;
  if constexpr (sizeof(R) == 4) sc = S.recip_scalef;
  else sc = S.recip_scale;
  long long e_loc = 0;
  long long v_loc[6] = {0, 0, 0, 0, 0, 0};
  for (int pass = 0; pass < npass; ++pass) {
    const int sgn = (kind == FFT_INV || pass == 1) ? +1 : -1;
    int Ns = 1;
    for (int st = 0; st < S.nstage[axis]; ++st) {
      const int Rd = S.radix[axis][st];
      const int T = K / Rd;
      const int twstep = K / (Ns * Rd);
      const float inv_T = 1.0f / (float)T, inv_Ns = 1.0f / (float)Ns;
      for (int t = tid; t < nl * T; t += nt) {
        const int li = qdiv(t, T, inv_T), j = t - li * T;
        const int jq = qdiv(j, Ns, inv_Ns);
        const int k = j - jq * Ns;
        const int od = jq * Ns * Rd + k;
        butterfly_rd<R, R2>(Rd, bufA + li * K + j, T, bufB + li * K + od, Ns, tw, k, twstep, sgn);
      }
      __syncthreads();
      R2 *tmp = bufA;
      bufA = bufB;
      bufB = tmp;
      Ns *= Rd;
    }
    if (kind == FFT_FWD_INFL_INV && pass == 0) {
      // influence function B(m) C(m); energy and virial of the spectrum
      const R *b0 = (const R *)(sizeof(R) == 4 ? (const void *)P.bsp : (const void *)P.bsp64) +
                    S.bsp_off[0];
      const R *b1 = (const R *)(sizeof(R) == 4 ? (const void *)P.bsp : (const void *)P.bsp64) +
                    S.bsp_off[1];
      const R *b2 = (const R *)(sizeof(R) == 4 ? (const void *)P.bsp : (const void *)P.bsp64) +
                    S.bsp_off[2];
      R pi2k2, cpref, ib0, ib1, ib2;
      if constexpr (sizeof(R) == 4) {
        pi2k2 = S.pme_pi2k2;
        cpref = S.pme_cpref;
        ib0 = S.inv_box[0];
        ib1 = S.inv_box[1];
        ib2 = S.inv_box[2];
      } else {
        pi2k2 = R(9.8696044010893586188 / (S.kappa * S.kappa));
        cpref = R(S.lB / (3.14159265358979323846 * S.V));
        ib0 = R(1.0 / S.box[0]);
        ib1 = R(1.0 / S.box[1]);
        ib2 = R(1.0 / S.box[2]);
      }
      for (int t = tid; t < nl * K; t += nt) {
        const int li = qdiv(t, K, inv_K), k = t - li * K;
        const int l = full_line(li);
        const int i1 = qdiv(l, K0, inv_K0), i0 = l - i1 * K0, i2 = k;
        const int m0 = i0 < (K0 + 1) / 2 ? i0 : i0 - K0;
        const int m1 = i1 < (K1 + 1) / 2 ? i1 : i1 - K1;
        const int m2 = i2 < (K2 + 1) / 2 ? i2 : i2 - K2;
        R2 &F = bufA[li * K + k];
        if (m0 == 0 && m1 == 0 && m2 == 0) {
          F.x = F.y = R(0);
          continue;
        }
        const R mv0 = R(m0) * ib0, mv1 = R(m1) * ib1, mv2 = R(m2) * ib2;
        const R msq = mv0 * mv0 + mv1 * mv1 + mv2 * mv2;
        const R BC = b0[i0] * b1[i1] * b2[i2] * cpref * exp(-pi2k2 * msq) / msq;
        const bool pair = half && i0 != 0 && 2 * i0 != K0;  // stands for its mirror too
        const R Em = R(0.5) * sc * BC * (F.x * F.x + F.y * F.y);
        e_loc += efix(pair ? R(2) * Em : Em);
        if (VIR) {
          const R fac = R(2) * (R(1) + pi2k2 * msq) / msq;
          const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
          const R mv[3] = {mv0, mv1, mv2};
          // the mirror's wave vector: every component negated except a
          // Nyquist one (index K/2 of an even K is its own mirror, and keeps
          // the sign convention of m)
          const R mm[3] = {-mv0, 2 * i1 == K1 ? mv1 : -mv1, 2 * i2 == K2 ? mv2 : -mv2};
          for (int q = 0; q < 6; ++q) {
            const R d = ia[q] == ib[q] ? R(1) : R(0);
            R w = Em * (d - fac * mv[ia[q]] * mv[ib[q]]);
            if (pair) w += Em * (d - fac * mm[ia[q]] * mm[ib[q]]);
            v_loc[q] += efix(w);
          }
        }
        F.x *= BC;
        F.y *= BC;
      }
      __syncthreads();
    }
  }
  // ---- store
  for (int t = tid; t < nl * K; t += nt) {
    int li, k;
    if (axis == 0) {
      li = qdiv(t, K, inv_K);
      k = t - li * K;
    } else {
      k = qdiv(t, nl, inv_nl);
      li = t - k * nl;
    }
    grid[line_elem(axis, K0, K1, full_line(li), k, inv_K0)] = bufA[li * K + k];
  }
  if (kind == FFT_FWD_INFL_INV) {
    const long long ev = warp_sum(e_loc);
    if ((tid & 31) == 0 && ev)
      atomicAdd(P.acc + (long long)s * kNacc + ACC_RECIP, (unsigned long long)ev);
    if (VIR) {
      const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
      for (int q = 0; q < 9; ++q) {
        const long long vv = warp_sum(v_loc[map[q]]);
        if ((tid & 31) == 0 && vv) atomicAdd(P.vacc + (long long)s * 9 + q, (unsigned long long)vv);
      }
    }
  }
  __syncthreads();
}

}  // namespace gcme
