// noalloc.cu -- cell-list build that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host program whose device memory
// is handed out by another runtime's pool (an MD engine that owns the GPU's
// memory and lends this library only its own buffers), or a latency-bound
// loop where cudaMalloc's implicit device synchronisation is not
// acceptable.  gcme_build_cells_noalloc serves them: it runs the same K1/K2
// kernels as gcme_build_cells, with every scratch array carved from one
// file-scope device array of fixed size (kNoAllocBytes, held by every GPU
// that loads the library until the process exits).  The caller still owns
// the inputs (positions, charges) and the outputs (cell starts, order).
// gcme_cells_noalloc_size tells such a caller, without touching the GPU,
// how long its cell-start buffer must be.
#include <mutex>
#include <string>

#include "engine.h"

namespace gcme {
namespace {

constexpr long long kNoAllocMaxBeads = 65536;
constexpr long long kNoAllocMaxCells = 32768;

// byte offsets of the scratch arrays (each 256-byte aligned)
constexpr long long al(long long b) { return (b + 255) / 256 * 256; }
constexpr long long kOffDesc = 0;
constexpr long long kOffXyzq = kOffDesc + al(sizeof(SysDesc));
constexpr long long kOffCellOf = kOffXyzq + al(16 * kNoAllocMaxBeads);
constexpr long long kOffSlot = kOffCellOf + al(4 * kNoAllocMaxBeads);
constexpr long long kOffSortTmp = kOffSlot + al(4 * kNoAllocMaxBeads);
constexpr long long kOffXyzqS = kOffSortTmp + al(4 * kNoAllocMaxBeads);
constexpr long long kOffExtSys = kOffXyzqS + al(16 * kNoAllocMaxBeads);
constexpr long long kOffCellCnt = kOffExtSys + al(4 * kNoAllocMaxBeads);
constexpr long long kOffCellNimg = kOffCellCnt + al(4 * kNoAllocMaxCells);
constexpr long long kOffCellNq = kOffCellNimg + al(4 * kNoAllocMaxCells);
constexpr long long kOffCellSys = kOffCellNq + al(4 * kNoAllocMaxCells);
constexpr long long kNoAllocBytes = kOffCellSys + al(4 * kNoAllocMaxCells);  // ~3.9 MB

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the host-side symbol is not a device address).
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128] = {};

int noalloc_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 128) {
    set_error("device index out of range");
    return GCME_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
      return GCME_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  return GCME_OK;
}

// Checks shared by the size query and the build: the parameters, the bead
// count and the cell grid against the fixed maxima; fills the descriptor's
// cell grid and box fields (the same helpers as the allocating path).
int noalloc_geometry(const gcme_params *p, int64_t n, SysDesc &S, long long &ncell) {
  if (!p || n < 1) {
    set_error("gcme_build_cells_noalloc: NULL parameters or n < 1");
    return GCME_ERR_INVALID;
  }
  if (n > kNoAllocMaxBeads) {
    set_error("gcme_build_cells_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
              std::to_string(kNoAllocMaxBeads) + " beads");
    return GCME_ERR_INVALID;
  }
  if (p->geometry == GCME_SLAB_IMAGE) {
    set_error("gcme_build_cells_noalloc: the image-charge geometry is not supported");
    return GCME_ERR_INVALID;
  }
  if (p->geometry != GCME_BULK && p->geometry != GCME_SLAB_NONMETAL) {
    set_error("gcme_build_cells_noalloc: unknown geometry");
    return GCME_ERR_INVALID;
  }
  if (!(p->rc > 0)) {
    set_error("gcme_build_cells_noalloc: rc must be > 0");
    return GCME_ERR_INVALID;
  }
  if (p->cell_factor != 0 && p->cell_factor != 1 && p->cell_factor != 2) {
    set_error("gcme_build_cells_noalloc: cell_factor must be 0, 1 or 2");
    return GCME_ERR_INVALID;
  }
  const int factor = p->cell_factor ? p->cell_factor : kDefaultCellFactor;
  ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(p->box[a] >= p->rc * (1.0 + 1e-4))) {
      set_error("gcme_build_cells_noalloc: box side shorter than the cutoff");
      return GCME_ERR_INVALID;
    }
    if (p->box[a] / ((p->rc / factor) * (1.0 + 1e-4)) > (double)kNoAllocMaxCells) {
      set_error("gcme_build_cells_noalloc: too many cells");
      return GCME_ERR_INVALID;
    }
    S.nc[a] = cells_per_axis(p->box[a], p->rc, factor);
    ncell *= S.nc[a];
    set_cell_box_axis(S, a, p->box[a]);
  }
  if (ncell > kNoAllocMaxCells) {
    set_error("gcme_build_cells_noalloc: " + std::to_string(ncell) +
              " cells exceed the maximum of " + std::to_string(kNoAllocMaxCells));
    return GCME_ERR_INVALID;
  }
  S.n = (int)n;
  S.n_ext = (int)n;
  S.ncell = (int)ncell;
  S.cell_factor = factor;
  S.geometry = p->geometry;
  return GCME_OK;
}

// Writes the call's descriptor (a kernel argument, copied at launch) into
// the scratch and clears the per-bead and per-cell system tables (all zero
// for one system): nothing is copied from host memory.
__global__ void k_noalloc_init(SysDesc S, SysDesc *dst, int *ext_sys, int n, int *cell_sys,
                               int ncell) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) *dst = S;
  for (int k = g; k < n; k += gridDim.x * blockDim.x) ext_sys[k] = 0;
  for (int k = g; k < ncell; k += gridDim.x * blockDim.x) cell_sys[k] = 0;
}

}  // namespace
}  // namespace gcme

using namespace gcme;

extern "C" int gcme_cells_noalloc_size(const gcme_params *p, int64_t n, int64_t *ncell) {
  if (!ncell) {
    set_error("gcme_cells_noalloc_size: NULL output");
    return GCME_ERR_INVALID;
  }
  SysDesc S{};
  long long nc = 0;
  const int rc = noalloc_geometry(p, n, S, nc);
  if (rc) return rc;
  *ncell = nc;
  return GCME_OK;
}

extern "C" int gcme_build_cells_noalloc(const gcme_params *p, int64_t n, const double *d_pos,
                                        const double *d_q, int32_t *d_cell_start,
                                        int32_t *d_sorted_idx, gcme_stream_t stream) {
  if (!d_pos || !d_q || !d_cell_start || !d_sorted_idx) {
    set_error("invalid argument to gcme_build_cells_noalloc");
    return GCME_ERR_INVALID;
  }
  SysDesc S{};
  long long ncell = 0;
  int rc = noalloc_geometry(p, n, S, ncell);
  if (rc) return rc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  unsigned char *base = nullptr;
  rc = noalloc_scratch(dev, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Pool Q{};
  Q.sys = reinterpret_cast<const SysDesc *>(base + kOffDesc);
  Q.nsys = 1;
  Q.pos = const_cast<double *>(d_pos);
  Q.q = d_q;
  Q.xyzq_u = reinterpret_cast<float4 *>(base + kOffXyzq);
  Q.cell_of = reinterpret_cast<int *>(base + kOffCellOf);
  Q.slot = reinterpret_cast<int *>(base + kOffSlot);
  Q.sort_tmp = reinterpret_cast<int *>(base + kOffSortTmp);
  Q.xyzq_s = reinterpret_cast<float4 *>(base + kOffXyzqS);
  Q.ext_sys = reinterpret_cast<int *>(base + kOffExtSys);
  Q.sorted_idx = d_sorted_idx;
  Q.cell_cnt = reinterpret_cast<int *>(base + kOffCellCnt);
  Q.cell_start = d_cell_start;
  Q.cell_nimg = reinterpret_cast<int *>(base + kOffCellNimg);
  Q.cell_nq = reinterpret_cast<int *>(base + kOffCellNq);
  Q.cell_sys = reinterpret_cast<int *>(base + kOffCellSys);
  Q.n_real = n;
  Q.n_ext = n;
  Q.n_cells = ncell;
  // every call shares the scratch: the descriptor and the system tables are
  // rewritten here, the cell counts are cleared by launch_cells
  const long long span = std::max<long long>(n, ncell);
  const int nb = (int)std::min<long long>(1024, (span + 255) / 256);
  k_noalloc_init<<<nb, 256, 0, st>>>(S, reinterpret_cast<SysDesc *>(base + kOffDesc), Q.ext_sys,
                                      (int)n, Q.cell_sys, (int)ncell);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("k_noalloc_init: ") + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  launch_cells(Q, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("gcme_build_cells_noalloc: ") + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  return GCME_OK;
}
