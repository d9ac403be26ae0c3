// pme.cu -- K5-K8 per-phase kernels (bodies in pme.cuh).
#include "pme.cuh"
#include "kernels.h"

namespace gcme {

template <typename R, int PO>
__global__ void k_spread(Pool P) {
  pdl_begin();
  dev_spread<R, PO>(P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// one CTA per cell of the sorted cell list (FP32 path)
template <int PO>
__global__ void __launch_bounds__(128) k_spread_cells(Pool P) {
  __shared__ SpreadSmem sm;
  pdl_begin();
  dev_spread_cell<PO>(P, blockIdx.x, sm);
}

template <typename R, int PO>
__global__ void k_gather(Pool P) {
  pdl_begin();
  dev_gather<R, PO>(P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// spread/gather with the batch's common spline order as a constant (4, 5
// or 6), else the order read per system
template <typename R>
static void launch_spread_gather(const Pool &P, int order, bool gather, int nb, int tb,
                                 cudaStream_t st) {
#define GCME_SG(PO)                                          \
  do {                                                       \
    if (gather) launch_k(k_gather<R, PO>, nb, tb, 0, st, P); \
    else launch_k(k_spread<R, PO>, nb, tb, 0, st, P);        \
  } while (0)
  switch (order) {
    case 4: GCME_SG(4); break;
    case 5: GCME_SG(5); break;
    case 6: GCME_SG(6); break;
    default: GCME_SG(0); break;
  }
#undef GCME_SG
}

template <typename R, bool INV>
__global__ void __launch_bounds__(512) k_fft_plane(Pool P, const int2 *work, int nwork) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_begin();
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) dev_fft_plane<R, INV>(P, work, w, smem_raw);
}

template <typename R, bool VIR>
__global__ void __launch_bounds__(256) k_fft(Pool P, const int2 *work, int nwork, int axis, int kind,
                                             int lpb, int half) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_begin();
  for (int w = blockIdx.x; w < nwork; w += gridDim.x)
    dev_fft_item<R, VIR>(P, work, w, axis, kind, lpb, half, smem_raw);
}

void launch_pme_spread(const Pool &P, const PmePlan &pl, bool fp64, cudaStream_t st,
                       bool zero_grid) {
  if (P.n_q == 0 || P.n_grid == 0) return;
  if (zero_grid) cudaMemsetAsync(P.qgrid, 0, sizeof(unsigned long long) * P.n_grid, st);
  const int tb = 256;
  const int nb = (int)((P.n_q * 8 + tb - 1) / tb);
  if (fp64) {
    launch_spread_gather<double>(P, pl.order, false, nb, tb, st);
  } else if (pl.cell_spread && P.n_cells > 0) {
    const unsigned nc = (unsigned)P.n_cells;
    switch (pl.order) {
      case 4: launch_k(k_spread_cells<4>, nc, 128, 0, st, P); break;
      case 5: launch_k(k_spread_cells<5>, nc, 128, 0, st, P); break;
      case 6: launch_k(k_spread_cells<6>, nc, 128, 0, st, P); break;
      default: launch_k(k_spread_cells<0>, nc, 128, 0, st, P); break;
    }
  } else {
    launch_spread_gather<float>(P, pl.order, false, nb, tb, st);
  }
}

void launch_pme_fft(const Pool &P, const PmePlan &pl, bool fp64, bool vir, cudaStream_t st) {
  if (P.n_q == 0 || P.n_grid == 0) return;
  const size_t rsz = fp64 ? sizeof(double2) : sizeof(float2);
  // the z pass of the plane path works on the Hermitian half spectrum
  const int half = pl.use_plane;
  auto line_pass = [&](int ax, int kind) {
    const size_t shm = (2 * (size_t)pl.lpb[ax] + 1) * pl.kmax[ax] * rsz;
    const int nw = pl.nwork[ax], lpb = pl.lpb[ax];
    if (nw == 0) return;
    if (fp64) {
      if (vir) launch_k(k_fft<double, true>, nw, 256, shm, st, P, pl.work[ax], nw, ax, kind, lpb, half);
      else launch_k(k_fft<double, false>, nw, 256, shm, st, P, pl.work[ax], nw, ax, kind, lpb, half);
    } else {
      if (vir) launch_k(k_fft<float, true>, nw, 256, shm, st, P, pl.work[ax], nw, ax, kind, lpb, half);
      else launch_k(k_fft<float, false>, nw, 256, shm, st, P, pl.work[ax], nw, ax, kind, lpb, half);
    }
  };
  if (pl.use_plane) {
    const size_t shm = (2 * (size_t)pl.plane_elems + pl.kmax[0] + pl.kmax[1]) * rsz;
    if (fp64) launch_k(k_fft_plane<double, false>, pl.nplane, 512, shm, st, P, pl.plane_work, pl.nplane);
    else launch_k(k_fft_plane<float, false>, pl.nplane, 512, shm, st, P, pl.plane_work, pl.nplane);
    line_pass(2, FFT_FWD_INFL_INV);
    if (fp64) launch_k(k_fft_plane<double, true>, pl.nplane, 512, shm, st, P, pl.plane_work, pl.nplane);
    else launch_k(k_fft_plane<float, true>, pl.nplane, 512, shm, st, P, pl.plane_work, pl.nplane);
  } else {
    const int axes[5] = {0, 1, 2, 1, 0};
    const int kinds[5] = {FFT_FWD_FROM_Q, FFT_FWD, FFT_FWD_INFL_INV, FFT_INV, FFT_INV};
    for (int ps = 0; ps < 5; ++ps) line_pass(axes[ps], kinds[ps]);
  }
}

void launch_pme_gather(const Pool &P, const PmePlan &pl, bool fp64, cudaStream_t st) {
  if (P.n_q == 0 || P.n_grid == 0) return;
  const int tb = 256;
  const int nb = (int)((P.n_q * 8 + tb - 1) / tb);
  if (fp64) launch_spread_gather<double>(P, pl.order, true, nb, tb, st);
  else launch_spread_gather<float>(P, pl.order, true, nb, tb, st);
}

void launch_pme(const Pool &P, const PmePlan &pl, bool fp64, bool vir, cudaStream_t st,
                bool zero_grid) {
  launch_pme_spread(P, pl, fp64, st, zero_grid);
  launch_pme_fft(P, pl, fp64, vir, st);
  launch_pme_gather(P, pl, fp64, st);
}

// Grids as FP64 for inspection: the fixed-point charge grid times
// 1 / qscale, and the real parts of the complex grid.
__global__ void k_qgrid_to_f64(const unsigned long long *q, double *out, long long n, double inv) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < n) out[g] = (double)(long long)q[g] * inv;
}
template <typename R2>
__global__ void k_cgrid_real(const R2 *c, double *out, long long n) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < n) out[g] = (double)c[g].x;
}

void launch_grids_to_f64(const Pool &P, bool fp64, double *d_q, double *d_phi, cudaStream_t st) {
  const long long n = P.n_grid;
  const int nb = (int)((n + 255) / 256);
  if (d_q) k_qgrid_to_f64<<<nb, 256, 0, st>>>(P.qgrid, d_q, n, fp64 ? 1.0 / kQScale64 : 1.0 / kQScale32);
  if (d_phi) {
    if (fp64) k_cgrid_real<double2><<<nb, 256, 0, st>>>(P.cgrid64, d_phi, n);
    else k_cgrid_real<float2><<<nb, 256, 0, st>>>(P.cgrid, d_phi, n);
  }
}

void pme_set_smem_limits() {
  const int lim = 200 * 1024;
  cudaFuncSetAttribute(k_fft<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft_plane<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft_plane<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft_plane<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_fft_plane<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

}  // namespace gcme
