// misc.cu -- K9-K12 per-phase kernels (bodies in misc.cuh).
#include "kernels.h"

#include <algorithm>
#include <cstdint>
#include "misc.cuh"

namespace gcme {

#define GCME_TID (blockIdx.x * (long long)blockDim.x + threadIdx.x)
template <bool VIR>
__global__ void k_bonds(Pool P) {
  pdl_begin();
  dev_bonds<VIR>(P, GCME_TID);
}
__global__ void k_walls(Pool P) {
  pdl_begin();
  dev_walls(P, GCME_TID);
}
__global__ void k_slab_apply(Pool P) {
  pdl_begin();
  dev_slab_apply(P, GCME_TID);
}
template <bool VIR>
__global__ void k_finalize(Pool P) {
  pdl_begin();
  dev_finalize<VIR>(P, (int)GCME_TID);
}
template <typename V>
__global__ void k_kick_drift(Pool P) {
  pdl_begin();
  if (P.nsys == 1) dev_kick_drift<V, true>(P, GCME_TID);
  else dev_kick_drift<V, false>(P, GCME_TID);
  // the step's accumulators and cell counts start from zero (the previous
  // step has read them)
  const long long nt = (long long)gridDim.x * blockDim.x;
  for (long long k = GCME_TID; k < (long long)P.nsys * kNacc; k += nt) P.acc[k] = 0ull;
  for (long long k = GCME_TID; k < P.n_cells; k += nt) P.cell_cnt[k] = 0;
}
template <typename V>
__global__ void k_kick(Pool P) {
  pdl_begin();
  if (P.nsys == 1) dev_kick<V, true>(P, GCME_TID);
  else dev_kick<V, false>(P, GCME_TID);
}
#undef GCME_TID

void launch_bonded(const Pool &P, bool vir, bool bonds, cudaStream_t st) {
  if (bonds && P.n_bond > 0) {
    int nb = (int)((P.n_bond + 255) / 256);
    if (vir) launch_k(k_bonds<true>, nb, 256, 0, st, P);
    else launch_k(k_bonds<false>, nb, 256, 0, st, P);
  }
  // walls and the slab dipole exist only in slab geometries
  if (P.n_real > 0 && P.any_slab) launch_k(k_walls, (int)((P.n_real + 255) / 256), 256, 0, st, P);
}

void launch_slab_apply(const Pool &P, cudaStream_t st) {
  if (P.n_real > 0 && P.any_slab)
    launch_k(k_slab_apply, (int)((P.n_real + 255) / 256), 256, 0, st, P);
}

void launch_finalize(const Pool &P, bool vir, cudaStream_t st) {
  int nb = (P.nsys + 127) / 128;
  if (vir) launch_k(k_finalize<true>, nb, 128, 0, st, P);
  else launch_k(k_finalize<false>, nb, 128, 0, st, P);
}

void launch_kick_drift(const Pool &P, bool vel64, cudaStream_t st) {
  if (P.n_real == 0) return;
  int nb = (int)((P.n_real + 255) / 256);
  if (vel64) launch_k(k_kick_drift<double>, nb, 256, 0, st, P);
  else launch_k(k_kick_drift<float>, nb, 256, 0, st, P);
}

void launch_kick(const Pool &P, bool vel64, cudaStream_t st) {
  if (P.n_real == 0) return;
  int nb = (int)((P.n_real + 255) / 256);
  if (vel64) launch_k(k_kick<double>, nb, 256, 0, st, P);
  else launch_k(k_kick<float>, nb, 256, 0, st, P);
}

__global__ void k_force_to_f64(const long long *f, double *out, long long n3) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < n3) out[g] = (double)f[g] * (1.0 / kFScale);
}

void launch_force_to_f64(const long long *f, double *out, long long n3, cudaStream_t st) {
  if (n3 > 0) k_force_to_f64<<<(int)((n3 + 255) / 256), 256, 0, st>>>(f, out, n3);
}

// The state (positions FP64, velocities FP32, n3 values each) and the
// energies copied by the SMs, one side of them page-locked host memory
// (gcme_step_host; the GPU reads and writes it directly, over the coherent
// CPU-GPU link of a Grace system): 16-byte vectors where both addresses
// allow, else single values.
__global__ void k_state_copy(const double *__restrict__ sp, const float *__restrict__ sv,
                             double *__restrict__ dp, float *__restrict__ dv, long long n3,
                             const double *__restrict__ se, double *__restrict__ de) {
  pdl_wait();
  const long long g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const bool vp = ((reinterpret_cast<uintptr_t>(sp) | reinterpret_cast<uintptr_t>(dp)) & 15) == 0;
  const bool vv = ((reinterpret_cast<uintptr_t>(sv) | reinterpret_cast<uintptr_t>(dv)) & 15) == 0;
  const long long np2 = vp ? n3 / 2 : 0, nv4 = vv ? n3 / 4 : 0;
  for (long long k = g0; k < np2; k += gs)
    reinterpret_cast<double2 *>(dp)[k] = reinterpret_cast<const double2 *>(sp)[k];
  for (long long k = 2 * np2 + g0; k < n3; k += gs) dp[k] = sp[k];
  for (long long k = g0; k < nv4; k += gs)
    reinterpret_cast<float4 *>(dv)[k] = reinterpret_cast<const float4 *>(sv)[k];
  for (long long k = 4 * nv4 + g0; k < n3; k += gs) dv[k] = sv[k];
  if (se && g0 < GCME_NTERMS) de[g0] = se[g0];
}

void launch_state_copy(const double *sp, const float *sv, double *dp, float *dv, long long n3,
                       const double *se, double *de, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n3 / 2 + 255) / 256;  // about one 16-byte vector per thread
  const int nb = (int)std::max(1LL, std::min(want, 4LL * nsm));
  launch_k(k_state_copy, nb, 256, 0, st, sp, sv, dp, dv, n3, se, de);
}

// isotropic scaling of positions with the box (barostat volume moves)
__global__ void k_scale(double *x, long long n3, double s) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < n3) x[g] *= s;
}

void launch_scale(double *x, long long n3, double s, cudaStream_t st) {
  if (n3 > 0) k_scale<<<(int)((n3 + 255) / 256), 256, 0, st>>>(x, n3, s);
}

}  // namespace gcme
