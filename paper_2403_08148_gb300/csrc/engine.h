// engine.h -- host-side batch engine behind the C ABI.
#pragma once
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.h"

namespace gcme {

// cell factor used when the parameters leave the choice to the library
constexpr int kDefaultCellFactor = 1;
// work items per home cell of the 27-cell pair kernel (3 or 9)
constexpr int kDefaultPairSplit = 9;
constexpr int kDefaultPairThreads = 128;
constexpr int kTailCtasPerSm = 5;  // resident pair CTAs per SM assumed for the single-cell
                                   // tail of one-CTA-per-item launches
constexpr int kMaxPairChunks = 4;  // warp items per (home cell, part), at most
// real-space table intervals in r^2: N = 18.25 beta^2 rc^2 keeps the cubic
// interpolation error near 1e-7 of g(0) (the error scales as (beta^2 du)^4);
// at least kRealTabMin, and direct evaluation above kRealTabMax (a < ~0.09 d)
constexpr int kRealTabMin = 512;
constexpr int kRealTabMax = 16384;
constexpr int kMinLpb = 4;                       // fewest FFT lines per tile
constexpr size_t kFftSmemLimit = 200 * 1024;     // dynamic smem of k_fft
// Verlet-list skin (bead diameters): the list holds every pair within
// rc + skin and is rebuilt once a bead has moved more than skin / 2
constexpr double kListSkin = 0.4;

void set_error(const std::string &msg);

// Cells along a box side L: the most cells of side >= rc / factor (with a
// 1e-4 margin), so that the 27-cell stencil (factor 1) or the 125-cell
// stencil (factor 2) holds every pair within rc.
inline int cells_per_axis(double L, double rc, int factor) {
  return std::max(1, (int)std::floor(L / ((rc / factor) * (1.0 + 1e-4))));
}

// Box-derived cell fields of axis a for the cell count S.nc[a]: box side
// (FP64 and FP32), nc / L for the binning rule (FP64 and its FP32 copy for
// the shortcut away from cell faces) and the cell side.  Every path that
// fills a SysDesc for binning goes through here.
inline void set_cell_box_axis(SysDesc &S, int a, double L) {
  S.box[a] = L;
  S.boxf[a] = (float)L;
  S.inv_cell[a] = (double)S.nc[a] / L;
  S.inv_cellf[a] = (float)S.inv_cell[a];
  S.cside[a] = (float)(L / S.nc[a]);
}

struct SysSpec {
  gcme_params p;
  int64_t n = 0;
  std::vector<double> q;
  std::vector<int32_t> types;  // species per bead (empty: all species 0)
  std::vector<int32_t> bonds;  // 2 * nbond, local indices
};

// Validate one system's parameters and charges; returns "" when valid.
std::string validate_spec(const SysSpec &sp);

// A batch of independent systems in pooled device memory.  A single system
// is a batch of one whose state pointers may be the caller's buffers.
class Engine {
 public:
  ~Engine();
  void release();  // free everything build() made (build() may then run again)
  // own_state: allocate pos/vel/force/q pools (batch and server); else the
  // caller passes pos/force per call and only q is stored.
  int build(int device, const std::vector<SysSpec> &specs, bool own_state);

  // enqueue one force evaluation of every system at P.pos into P.force
  void enqueue_forces(const Pool &P, cudaStream_t st, bool vir, bool dbg);
  // enqueue one velocity-Verlet step (forces at P.pos must be current)
  void enqueue_step(const Pool &P, cudaStream_t st);
  // cell sort (gated by the rebuild flag with lists) and the pair kernels;
  // fork > 0: fork the PME branch after the sort (1: grid known to be zero,
  // 2: clear it first)
  void enqueue_sort_pairs(const Pool &P, cudaStream_t st, bool vir, bool dbg, bool timed,
                          int fork = 0);
  // make the next force evaluation rebuild the neighbour lists (after the
  // cell order was changed outside the list path)
  void request_rebuild(cudaStream_t st);
  // the pooled arrays as the cell-only kernels see them (no list fields)
  Pool cell_only(const Pool &Q) const;
  long long list_builds();  // synchronises the device
  void fork_pme(const Pool &P, cudaStream_t st, bool vir, bool timed, bool zero_grid = true);
  cudaStream_t side_stream = nullptr;  // PME branch
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

  // graph of one step for the given state pointers (cached)
  int step_graph(const Pool &P, cudaGraphExec_t *out);
  int forces_graph(const Pool &P, cudaGraphExec_t *out);
  // state on the host (page-locked h_pos[3n], h_vel[3n], h_energy or NULL),
  // P.pos / P.vel the device copies: part 1 copies the state in (and, unless
  // cont, evaluates the starting forces), part 2 copies the state and the
  // energies out, part 3 is both around one step (cached per host buffers)
  int host_graph(const Pool &P, const double *h_pos, const float *h_vel, double *h_energy,
                 bool cont, int part, cudaGraphExec_t *out);

  int nsys() const { return (int)hsys.size(); }
  // (system, code) pair work items: code = cell * split + part, times
  // S.pair_nch plus the chunk group when chunked (warp items); group > 1
  // (CTA items of split 9): code = row group * 9 + part, row groups of
  // `group` consecutive home cells along x
  std::vector<int2> make_pair_work(int split, bool chunked = false, int group = 1) const;
  // chunk groups per (home cell, part) of warp items for system s:
  // pair_chunks when set, else the median real-bead count of its non-empty
  // cells in chunks of 32 (from the last cell snapshot, else n / ncell),
  // 1..kMaxPairChunks
  int chunks_of(int s) const;
  std::vector<int2> make_fft_work(int axis, int lpb) const;
  int set_pair_config(int split, int threads, int ctas_per_sm, int nelec = 1, int chunks = 0,
                      int group = 1);
  bool pair_group_ok(int split, int nelec, int group) const;
  int group_of(int s, int group) const;  // system s's home cells per item
  // cell occupancy of the last cell sort (host copy) and the work-item
  // order it implies (heaviest first)
  int snapshot_cells(cudaStream_t st);
  // (group > 1: then `tail` single-cell items at the end of the list)
  void order_by_cost(std::vector<int2> &pw, int split, bool chunked = false, int group = 1,
                     int tail = 0) const;
  std::vector<int> snap_cnt, snap_nimg, snap_nq;
  int set_fft_lpb(int axis, int lpb);
  bool plane_fits() const;
  int set_fft_plane(bool on);
  // launch shapes given by the caller (checked before any is changed)
  int apply_tuning(int split, int threads, int ctas_per_sm, int nelec, const int lpb[3],
                   bool plane, int chunks = 0, bool spread_cells = false, int group = 1);
  // charges spread cell by cell through shared memory (FP32 27-cell path
  // without lists), else straight to the global grid
  bool cell_spread_ok() const { return !fp64 && cell_factor == 1 && !use_list; }
  int set_spread_cells(bool on);
  void clear_graphs();
  // time candidate configurations on the current state and keep the
  // fastest (tune.cu); from_cache reports a hit of the tuning cache
  int autotune(const Pool &Q, cudaStream_t st, int flags, double *pair_ms, double *pme_ms,
               bool *from_cache);
  // Phase marks recorded inside the captured step graph: 0 start, 1 after
  // the first half kick + drift, 9 after binning (the PME branch forks
  // here), 2 after the cell list, 3 after the pair kernel, 4 after
  // bonds/walls, 5/6 around the PME branch on the side stream, 7 after the
  // join, 10/11 around the second half kick, 8 after the energies.
  static constexpr int kNPhaseEv = 12;
  cudaEvent_t phase_ev[kNPhaseEv] = {};
  int step_kernels = 0;  // kernel nodes in the step graph
  // phase timing: step graphs captured with event nodes between the phases
  // (off by default: the event nodes lengthen the step); last_step_timed
  // tells whether the most recent step graph carried them
  bool phase_timing = false;
  bool last_step_timed = false;
  unsigned int *bar_words = nullptr;  // persistent-launch barrier state (4 words)
  // per-system step limits (Pool::step_stop; the server's engines): a device
  // array of nsys counters the caller fills; enable_step_limits() makes the
  // step kernels hold each system at its limit
  unsigned long long *step_stop_buf = nullptr;
  void enable_step_limits();
  bool fp64 = false;
  int cell_factor = 1;  // 1: 27-cell stencil; 2: fine cells with culling
  bool use_list = false;  // FP32 pair terms over Verlet neighbour lists
  bool species = false;   // several species: per-pair constants from tables
  int pair_split = 0;   // 3 or 9 work items per home cell (0: default)
  int pair_threads = kDefaultPairThreads;  // 128, 160 or 192 threads per pair CTA
  int pair_nelec = 1;  // of which electrostatics warps (1 to 3; 0: one warp per item)
  int pair_chunks = 0;  // warp items per (home cell, part): 1..4, 0 automatic
  int pair_group = 1;   // CTA items of split 9: home cells along x per item (1..3), for
                        // systems with at least pair_group + 2 cells along x
  bool pair_groups_on = false;  // some system takes items of several home cells
  int pair_ctas_per_sm = 0;  // 0: one CTA per work item; else resident CTAs per SM fetching items
  int n_sm = 152;
  int *pair_counter = nullptr;  // dynamic work-item counter of the pair kernel
  int pair_ctas() const { return pair_ctas_per_sm > 0 ? n_sm * pair_ctas_per_sm : 0; }
  // the FP32 27-cell kernel (one cell per stencil step, no pair dump) also
  // runs the harmonic bonds, as work items after the cell items
  bool bonds_in_pair(bool dbg) const {
    return !fp64 && !dbg && cell_factor == 1 && n_pair_work > 0 && P.n_bond > 0;
  }
  int device = 0;
  std::vector<SysDesc> hsys;
  Pool P{};  // device pointers of the pooled arrays
  std::vector<long long> bead_off;
  long long n_real = 0, n_ext = 0;
  size_t scratch_bytes = 0;
  int2 *pair_work = nullptr;
  int n_pair_work = 0;
  PmePlan plan{};
  cudaStream_t capture_stream = nullptr;

 private:
  void *arena_ = nullptr;
  std::map<std::tuple<void *, void *, void *, int>, cudaGraphExec_t> graphs_;
  std::vector<cudaGraph_t> graph_objs_;
};

// radix factorisation of a 5-smooth grid size (4s first)
std::vector<int> fft_radices(int K);
bool is_smooth(int K);

}  // namespace gcme

struct gcme_ctx {
  int device;
};
