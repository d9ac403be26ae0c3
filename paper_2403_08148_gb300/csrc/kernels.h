// kernels.h -- host-side launchers of the libgcme kernels.
#pragma once
#include "common.cuh"

namespace gcme {

// Launch with programmatic stream serialization (captured into graphs as
// programmatic edges): the kernel may be launched before its predecessor in
// the stream has finished, hiding the launch latency; it must call
// pdl_wait() (common.cuh) before it reads or writes memory.
template <typename... K, typename... A>
inline cudaError_t launch_k(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<K>(args)...);
}


// FFT work per axis: int2 (system, tile of lpb lines), lines per tile and
// the largest grid extent along that axis over the batch.
struct PmePlan {
  const int2 *work[3];
  int nwork[3];
  int lpb[3];
  int kmax[3];
  // x-y plane passes (one CTA per z-plane of every system) when every
  // plane fits in shared memory: 3 FFT launches instead of 5
  const int2 *plane_work;
  int nplane;
  int use_plane;
  int plane_elems;  // largest K0 * K1 of the batch
  int order;        // B-spline order shared by every system, else 0
  // FP32 spread by cells of the sorted cell list through shared memory
  // (k_spread_cells): the PME branch then starts after the cell sort
  int cell_spread;
};

void launch_cells(const Pool &P, cudaStream_t st);  // launch_bin + launch_sort
// K1: wrap, cell ids, wrapped float4; zero_counts = false when the cell
// counts were cleared earlier on another stream
void launch_bin(const Pool &P, cudaStream_t st, bool zero_counts = true);
// largest per-system cell grid of the fused cell sort (each of its CTAs sums
// the counts of the system's earlier cells)
constexpr int kFusedSortCells = 4096;
// K2: scan, scatter, per-cell order (one fused kernel when P.bucket is set)
void launch_sort(const Pool &P, cudaStream_t st);
// ctas: grid of the 27-cell kernel (CTAs loop over items fetched from
// *counter, a device int that is zero before the launch and that the launch
// leaves zero).  bonds: the FP32 27-cell kernel also evaluates the harmonic
// bonds, one bond per thread in work items after the cell items.
// warp_items: the FP32 one-species kernel with one warp per work item
// (pair_warp.cuh; ctas > 0 required), else one CTA per work item; groups:
// CTA items of several home cells (SysDesc::pair_group > 1 in some system);
// dyn: the warps of a CTA take each item's tasks dynamically
// (SysDesc::pair_nelec < 0).
void launch_pair(const Pool &P, const int2 *work, int nwork, bool fp64, int cell_factor,
                 int threads, int ctas, int *counter, bool vir, bool dbg, bool bonds,
                 cudaStream_t st, bool warp_items = false, bool groups = false,
                 bool dyn = false);
// Verlet neighbour list (nlist.cu): rebuild decision (clears the flag,
// then sets it when a bead moved more than skin/2 since the last build or a
// rebuild is pending), the gated build, the per-step refresh of the sorted
// positions and image changes, and the pair kernel over the lists.
void launch_list_check(const Pool &P, cudaStream_t st);
void launch_list_build(const Pool &P, cudaStream_t st);
void launch_list_refresh(const Pool &P, cudaStream_t st);
void launch_pair_list(const Pool &P, bool vir, bool dbg, cudaStream_t st);
// zero_grid = false when the charge grid is known to be zero (the forward FFT
// pass clears every grid point it reads)
void launch_pme(const Pool &P, const PmePlan &pl, bool fp64, bool vir, cudaStream_t st,
                bool zero_grid = true);
// its three stages: spread into the charge grid, the FFT passes with the
// influence function (the forward pass leaves the charge grid zero, the
// last pass leaves theta * Q in the real parts of the complex grid), gather
void launch_pme_spread(const Pool &P, const PmePlan &pl, bool fp64, cudaStream_t st,
                       bool zero_grid);
void launch_pme_fft(const Pool &P, const PmePlan &pl, bool fp64, bool vir, cudaStream_t st);
void launch_pme_gather(const Pool &P, const PmePlan &pl, bool fp64, cudaStream_t st);
// the charge grid (times 1 / qscale) and the real parts of the complex grid
// as FP64 arrays of P.n_grid values (either may be NULL)
void launch_grids_to_f64(const Pool &P, bool fp64, double *d_q, double *d_phi, cudaStream_t st);
void pme_set_smem_limits();
// bonds (unless the pair kernel took them), walls, dipole
void launch_bonded(const Pool &P, bool vir, bool bonds, cudaStream_t st);
void launch_slab_apply(const Pool &P, cudaStream_t st);         // Yeh-Berkowitz forces
void launch_finalize(const Pool &P, bool vir, cudaStream_t st); // energies -> FP64
void launch_kick_drift(const Pool &P, bool vel64, cudaStream_t st);
void launch_kick(const Pool &P, bool vel64, cudaStream_t st);
// one cooperative launch of nsteps steps of the whole batch (FP32); the
// four words at bar_words hold the barrier state and the error word;
// warp_items: the pair phase runs one warp per work item (pair_warp.cuh;
// one-species 27-cell batches), as the per-phase launches do under the same
// launch shapes (the same kernel path gives the same roundings); dyn: the
// CTA items' tasks taken dynamically (SysDesc::pair_nelec < 0)
int launch_persistent(const Pool &P, const int2 *pair_work, int n_pair_work, int cell_factor,
                      const PmePlan &pl,
                      long long nsteps, unsigned int *bar_words, double timeout_s,
                      cudaStream_t st, bool warp_items = false, bool dyn = false);
int launch_barrier_probe(unsigned int *bar_words, double timeout_s, cudaStream_t st);
void launch_force_to_f64(const long long *f, double *out, long long n3, cudaStream_t st);
// copy of the state (and the energies when se is set) by the SMs, either
// side in page-locked host memory (read or written directly by the GPU)
void launch_state_copy(const double *sp, const float *sv, double *dp, float *dv, long long n3,
                       const double *se, double *de, cudaStream_t st);
void launch_scale(double *x, long long n3, double s, cudaStream_t st);  // x *= s

}  // namespace gcme
