// cells.cuh -- device bodies of K1/K2 (wrap + bin, scan, scatter, per-cell
// stable order), shared by the per-phase kernels and the persistent kernel.
//
// Cell list of side >= rc (the 27-cell stencil of the pair kernel).  The
// binning is FP64 and bit-reproducible: wrapped x = x - L floor(x / L) with
// one rounding per operation, cell = floor(x nc / L) clamped to [0, nc-1]
// (dev_bin reaches the same results by exact shortcuts away from faces).
// Inside a cell, beads are ordered by (class, index) with class 0 = image,
// 1 = charged real, 2 = neutral real, so that the pair kernel finds the
// electrostatic beads (images + charged) and the Gaussian-core beads
// (charged + neutral reals) as two contiguous ranges.
#pragma once
#include "common.cuh"

namespace gcme {

constexpr int kSortCap = 1024;

// ONE: one system without image beads (ext index = bead index, s = 0).
template <bool ONE = false>
__device__ __forceinline__ void dev_bin(const Pool &P, long long g) {
  if (g >= P.n_ext) return;
  double x[3], q;
  if (ONE) {
    const double *p = P.pos + 3 * g;
    x[0] = p[0];
    x[1] = p[1];
    x[2] = p[2];
    q = P.q[g];
  } else if (P.ext_src) {  // position and charge from one index, beside the system lookup
    const int src = P.ext_src[g];
    const int r = src < 0 ? -1 - src : src;
    const double *p = P.pos + 3 * (long long)r;
    x[0] = p[0];
    x[1] = p[1];
    x[2] = src < 0 ? -p[2] : p[2];
    q = src < 0 ? -P.q[r] : P.q[r];
  }
  const int s = ONE ? 0 : P.ext_sys[g];
  const SysDesc &S = P.sys[s];
  const int e = ONE ? (int)g : (int)(g - S.ext_off);
  if (!ONE && !P.ext_src) {
    ext_position(P, S, e, x[0], x[1], x[2]);
    q = ext_charge(P, S, e);
  }
  // the system's constants into registers first: each is then one load in
  // flight with the positions, not a round trip behind the previous axis
  // (the rare store to wrap_n below would otherwise keep later loads behind it)
  double Lb[3], icell[3];
  float icellf[3];
  int ncs[3], np3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Lb[a] = S.box[a];
    icell[a] = S.inv_cell[a];
    icellf[a] = S.inv_cellf[a];
    ncs[a] = S.nc[a];
    np3[a] = P.wrap_n ? P.wrap_n[3 * g + a] : 0;
  }
  const long long cell_off = S.cell_off;
  const int sn = S.n;
  double w[3];
  float wf[3];
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // Wrap: with n the image index this coordinate had at the last binning,
    // w0 = x - L n (the rule's own two roundings).  If w0 lies in
    // [L 2^-40, L (1 - 2^-40)] and |n| < 2^10, the rule's floor(x / L) is n
    // (the roundings of x / L and L n are below L 2^-42 here), so w0 is the
    // rule's result and the FP64 division is skipped.
    const double L = Lb[a];
    const int np = np3[a];
    const double w0 = __dsub_rn(x[a], __dmul_rn(L, (double)np));
    const double d = L * 9.094947017729282e-13;  // L 2^-40
    if (np > -1024 && np < 1024 && w0 >= d && w0 <= L - d) {
      w[a] = w0;
    } else {
      double f;
      w[a] = wrap_coord_n(x[a], L, f);
      if (P.wrap_n) P.wrap_n[3 * g + a] = (int)fmax(-1073741824.0, fmin(1073741824.0, f));
    }
    wf[a] = __double2float_rn(w[a]);
    // cell: floor(w nc / L) in FP64 (the rule); the FP32 product decides when
    // it is at least 1e-4 from a cell face (its error is below 2e-5 for
    // nc <= 256)
    const float uf = wf[a] * icellf[a];
    int k = (int)floorf(uf);
    const float fr = uf - (float)k;
    if (ncs[a] > 256 || !(fr >= 1e-4f && fr <= 1.0f - 1e-4f))
      k = (int)floor(__dmul_rn(w[a], icell[a]));
    k = k > ncs[a] - 1 ? ncs[a] - 1 : k;
    k = k < 0 ? 0 : k;
    c[a] = k;
  }
  int cell = c[0] + ncs[0] * (c[1] + ncs[1] * c[2]);
  P.xyzq_u[g] = make_float4(wf[0], wf[1], wf[2], (float)q);
  if (P.xyzq_u64) P.xyzq_u64[g] = make_dpos4(w[0], w[1], w[2], q);
  if (P.img_now) {
    // periodic image index: x = w + img L exactly up to the wrap rule
#pragma unroll
    for (int a = 0; a < 3; ++a) P.img_now[3 * g + a] = (int)rint((x[a] - w[a]) / Lb[a]);
  }
  P.cell_of[g] = cell;
  const int slot = atomicAdd(&P.cell_cnt[cell_off + cell], 1);
  P.slot[g] = slot;
  if (P.bucket && slot < P.bucket_cap) {
    const long long b = (cell_off + cell) * (long long)P.bucket_cap + slot;
    const int cls = e >= sn ? 0 : ((float)q != 0.0f ? 1 : 2);
    P.bucket[b] = e | (cls << 30);
    P.bucket_pos[b] = make_float4(wf[0], wf[1], wf[2], (float)q);
  }
}

// Exclusive scan of the cell counts of all systems by one CTA (any size
// that is a multiple of 32); warp_tot is 32 entries of shared memory.
__device__ __forceinline__ void dev_scan_block(const int *cnt, int *start, long long n,
                                               long long *warp_tot) {
  const int T = blockDim.x;
  long long chunk = (n + T - 1) / T;
  long long b = threadIdx.x * chunk;
  long long e = b + chunk < n ? b + chunk : n;
  long long loc = 0;
  for (long long i = b; i < e; ++i) loc += cnt[i];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long v = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < (T >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  long long off = v - loc + (wid > 0 ? warp_tot[wid - 1] : 0);
  for (long long i = b; i < e; ++i) {
    start[i] = (int)off;
    off += cnt[i];
  }
  if (threadIdx.x == T - 1) start[n] = (int)off;
}

__device__ __forceinline__ void dev_scatter(const Pool &P, long long g) {
  if (g >= P.n_ext) return;
  if (P.gate && !*P.gate) return;
  const SysDesc &S = P.sys[P.ext_sys[g]];
  int e = (int)(g - S.ext_off);
  P.sorted_idx[P.cell_start[S.cell_off + P.cell_of[g]] + P.slot[g]] = e;
}

// One CTA per cell: stable (class, index) order of the cell's beads (sorted
// slots [beg, beg + cnt), filled in slot order) and the gather of their
// wrapped positions into sorted order.  key: kSortCap entries of shared
// memory, cnt2: two shared ints.  Ends with a barrier.
__device__ __forceinline__ void dev_cellsort_range(const Pool &P, const SysDesc &S, long long cg,
                                                   int beg, int cnt, long long *key, int *cnt2) {
  if (threadIdx.x == 0) {
    cnt2[0] = 0;
    cnt2[1] = 0;
  }
  __syncthreads();
  bool in_smem = cnt <= kSortCap;
  // keys: class in the high word, local ext index in the low word
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    int e = P.sorted_idx[beg + t];
    int cls;
    if (e >= S.n) cls = 0;
    else cls = P.xyzq_u[S.ext_off + e].w != 0.0f ? 1 : 2;
    long long k = ((long long)cls << 32) | (unsigned)e;
    if (in_smem) key[t] = k;
    if (cls == 0) atomicAdd(&cnt2[0], 1);
    if (cls <= 1) atomicAdd(&cnt2[1], 1);
  }
  __syncthreads();
  if (!in_smem) {
    // Oversized cell: rank against global memory, park the order in
    // sort_tmp, then move it into place after every rank is known.
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int e = P.sorted_idx[beg + t];
      int cls = e >= S.n ? 0 : (P.xyzq_u[S.ext_off + e].w != 0.0f ? 1 : 2);
      long long k = ((long long)cls << 32) | (unsigned)e;
      int rank = 0;
      for (int u = 0; u < cnt; ++u) {
        int f = P.sorted_idx[beg + u];
        int cf = f >= S.n ? 0 : (P.xyzq_u[S.ext_off + f].w != 0.0f ? 1 : 2);
        rank += (((long long)cf << 32) | (unsigned)f) < k;
      }
      P.sort_tmp[beg + rank] = e;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int e = P.sort_tmp[beg + t];
      P.sorted_idx[beg + t] = e;
      P.xyzq_s[beg + t] = P.xyzq_u[S.ext_off + e];
      if (P.xyzq_s64) P.xyzq_s64[beg + t] = P.xyzq_u64[S.ext_off + e];
      if (P.type_s) P.type_s[beg + t] = P.type_u[S.ext_off + e];
    }
  } else {
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      long long k = key[t];
      int rank = 0;
      for (int u = 0; u < cnt; ++u) rank += key[u] < k;
      int e = (int)(k & 0xffffffffLL);
      long long dst = beg + rank;
      P.sorted_idx[dst] = e;
      P.xyzq_s[dst] = P.xyzq_u[S.ext_off + e];
      if (P.xyzq_s64) P.xyzq_s64[dst] = P.xyzq_u64[S.ext_off + e];
      if (P.type_s) P.type_s[dst] = P.type_u[S.ext_off + e];
    }
  }
  if (threadIdx.x == 0) {
    P.cell_nimg[cg] = cnt2[0];
    P.cell_nq[cg] = cnt2[1];
  }
  __syncthreads();
}

__device__ __forceinline__ void dev_cellsort_block(const Pool &P, long long cg, long long *key,
                                                   int *cnt2) {
  const SysDesc &S = P.sys[P.cell_sys[cg]];
  const int beg = P.cell_start[cg];
  dev_cellsort_range(P, S, cg, beg, P.cell_start[cg + 1] - beg, key, cnt2);
}

// Scan, scatter and per-cell order in one pass, one CTA per cell (grids of
// at most kFusedSortCells cells per system): the cell's start is the
// system's first sorted slot plus the counts of the system's earlier cells
// (a block sum), its beads come from the bucket written by the binning
// (or, for a cell holding more than bucket_cap beads, from a search of the
// system's beads), and the stable (class, index) order follows as in
// dev_cellsort_range.  A cell within both the bucket and kSortCap is ranked
// straight from its bucket entries (class and index) and written from its
// bucket positions, with no round trip through the sorted index.  red: 32
// shared ints.  Ends with a barrier.
__device__ __forceinline__ void dev_cellsort_fused_block(const Pool &P, long long cg,
                                                         long long *key, int *cnt2, int *red) {
  const SysDesc &S = P.sys[P.cell_sys[cg]];
  const int cnt = P.cell_cnt[cg];
  const bool direct = cnt <= P.bucket_cap && cnt <= kSortCap;
  const int *b = P.bucket + cg * (long long)P.bucket_cap;
  if (threadIdx.x == 0) {
    cnt2[0] = 0;
    cnt2[1] = 0;
  }
  int part = 0;
  for (long long c = S.cell_off + threadIdx.x; c < cg; c += blockDim.x) part += P.cell_cnt[c];
  part = warp_sum(part);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = part;
  if (direct) {
    __syncthreads();  // counters cleared
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const unsigned be = (unsigned)b[t];
      const unsigned cls = be >> 30;
      key[t] = ((long long)cls << 32) | (be & 0x3fffffffu);
      if (cls == 0) atomicAdd(&cnt2[0], 1);
      if (cls <= 1) atomicAdd(&cnt2[1], 1);
    }
  }
  __syncthreads();
  int tot = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k];
  const int beg = (int)S.ext_off + tot;
  if (threadIdx.x == 0) {
    P.cell_start[cg] = beg;
    if (cg == P.n_cells - 1) P.cell_start[cg + 1] = beg + cnt;
  }
  if (direct) {
    const float4 *bp = P.bucket_pos + cg * (long long)P.bucket_cap;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const long long k = key[t];
      const float4 v = bp[t];
      int rank = 0;
      for (int u = 0; u < cnt; ++u) rank += key[u] < k;
      const int e = (int)(k & 0xffffffffLL);
      const long long dst = beg + rank;
      P.sorted_idx[dst] = e;
      P.xyzq_s[dst] = v;
      if (P.xyzq_s64) P.xyzq_s64[dst] = P.xyzq_u64[S.ext_off + e];
      if (P.type_s) P.type_s[dst] = P.type_u[S.ext_off + e];
    }
    if (threadIdx.x == 0) {
      P.cell_nimg[cg] = cnt2[0];
      P.cell_nq[cg] = cnt2[1];
    }
    __syncthreads();
    return;
  }
  if (cnt <= P.bucket_cap) {
    const int *b = P.bucket + cg * (long long)P.bucket_cap;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x)
      P.sorted_idx[beg + t] = (int)((unsigned)b[t] & 0x3fffffffu);
  } else {
    const int cl = (int)(cg - S.cell_off);
    for (long long g = S.ext_off + threadIdx.x; g < S.ext_off + S.n_ext; g += blockDim.x)
      if (P.cell_of[g] == cl) P.sorted_idx[beg + P.slot[g]] = (int)(g - S.ext_off);
  }
  __syncthreads();
  dev_cellsort_range(P, S, cg, beg, cnt, key, cnt2);
}

}  // namespace gcme
