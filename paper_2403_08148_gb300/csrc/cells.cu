// cells.cu -- K1/K2 per-phase kernels: wrap + bin, then either the fused
// scan + scatter + per-cell stable order (grids of at most kFusedSortCells
// cells per system) or the three separate passes (bodies in cells.cuh).
#include "cells.cuh"
#include "kernels.h"

namespace gcme {

__global__ void k_bin(Pool P) {
  pdl_begin();
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (P.nsys == 1 && P.n_ext == P.n_real) dev_bin<true>(P, g);
  else dev_bin<false>(P, g);
}

__global__ void __launch_bounds__(1024) k_scan(const int *cnt, int *start, long long n,
                                              const int *gate) {
  __shared__ long long warp_tot[32];
  pdl_begin();
  if (gate && !*gate) return;
  dev_scan_block(cnt, start, n, warp_tot);
}

__global__ void k_scatter(Pool P) {
  pdl_begin();
  dev_scatter(P, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_cellsort(Pool P) {
  __shared__ long long key[kSortCap];
  __shared__ int cnt2[2];
  pdl_begin();
  if (blockIdx.x >= P.n_cells) return;
  if (P.gate && !*P.gate) return;
  dev_cellsort_block(P, blockIdx.x, key, cnt2);
}

__global__ void __launch_bounds__(256) k_cellsort_fused(Pool P) {
  __shared__ long long key[kSortCap];
  __shared__ int cnt2[2];
  __shared__ int red[32];
  pdl_begin();
  if (blockIdx.x >= P.n_cells) return;
  if (P.gate && !*P.gate) return;
  dev_cellsort_fused_block(P, blockIdx.x, key, cnt2, red);
}

void launch_bin(const Pool &P, cudaStream_t st, bool zero_counts) {
  if (P.n_ext == 0) return;
  const int tb = 256;
  const int nb = (int)((P.n_ext + tb - 1) / tb);
  if (zero_counts) cudaMemsetAsync(P.cell_cnt, 0, sizeof(int) * P.n_cells, st);
  launch_k(k_bin, nb, tb, 0, st, P);
}

void launch_sort(const Pool &P, cudaStream_t st) {
  if (P.n_ext == 0) return;
  const int tb = 256;
  const int nb = (int)((P.n_ext + tb - 1) / tb);
  if (P.bucket) {
    launch_k(k_cellsort_fused, (unsigned)P.n_cells, 256, 0, st, P);
    return;
  }
  launch_k(k_scan, 1, 1024, 0, st, (const int *)P.cell_cnt, P.cell_start, (long long)P.n_cells,
           (const int *)P.gate);
  launch_k(k_scatter, nb, tb, 0, st, P);
  launch_k(k_cellsort, (unsigned)P.n_cells, 256, 0, st, P);
}

void launch_cells(const Pool &P, cudaStream_t st) {
  launch_bin(P, st);
  launch_sort(P, st);
}

}  // namespace gcme
