// tune.cu -- autotuner of the pair-kernel work shape and the PME FFT tiling.
//
// Candidates are timed with CUDA events on the caller's stream on the
// actual system (or batch) at its current positions:
//   pair kernel (27-cell path): 3 or 9 work items per home cell (9 or 3 neighbour cells
//                each) x {128 threads with 1 electrostatics warp, 160 with 1
//                or 2, 192 with 2 or 3; the other warps Gaussian core} x {one CTA
//                per work item, or 3, 4, 5, 6 or 8 resident CTAs per SM fetching
//                items dynamically so that the remaining slots host the
//                concurrent PME branch}, the same CTAs with every warp
//                taking the items' tasks (core chunks, parts of charged
//                chunks) dynamically, and one warp per work item
//                (CTAs of 4 warps, 3-7 per SM, or of 2 warps, 8-14 per SM);
//                then, for the fastest CTA-item shape of split 9, items of 2
//                or 3 consecutive home cells along x;
//   PME:         lines per FFT tile along each axis in {4, 8, 16, 32, 64}
//                (shared memory permitting), one axis at a time, x-y
//                plane passes (one CTA per z-plane) vs per-axis passes, and
//                the charge spread by cells through shared memory vs
//                straight to the global grid;
// each candidate timed on replays of the captured step graph (scratch state).
// The fastest configuration is kept and recorded in a JSON-lines cache
// (GCME_TUNE_CACHE, else $HOME/.cache/gcme_tune.jsonl) keyed by the GPU
// name and the workload shape, so later runs apply it without timing.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "engine.h"

namespace gcme {
namespace {

#define TUNE_CK(call)                                                           \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) {                                                    \
      set_error(std::string("autotune: ") + #call + ": " + cudaGetErrorString(_e)); \
      return GCME_ERR_CUDA;                                                     \
    }                                                                           \
  } while (0)

std::mutex g_cache_mu;

std::string cache_path() {
  const char *p = std::getenv("GCME_TUNE_CACHE");
  if (p && *p) return p;
  const char *h = std::getenv("HOME");
  std::string dir = std::string(h && *h ? h : "/tmp") + "/.cache";
  mkdir(dir.c_str(), 0755);  // may exist already
  return dir + "/gcme_tune.jsonl";
}

struct Tuned {
  int split = 0, threads = 0, ctas = 0, lpb[3] = {0, 0, 0}, plane = 0, nelec = 1, chunks = 0,
      spread = 0, group = 1;
  double pair_ms = 0, pme_ms = 0;
};

bool cache_lookup(const std::string &key, Tuned *t) {
  std::lock_guard<std::mutex> g(g_cache_mu);
  std::ifstream f(cache_path());
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    const std::string kk = "\"key\": \"" + key + "\"";
    if (line.find(kk) == std::string::npos) continue;
    Tuned x;
    const char *c = std::strstr(line.c_str(), "\"pair_split\":");
    if (!c) continue;
    if (std::sscanf(c,
                    "\"pair_split\": %d, \"pair_threads\": %d, \"pair_ctas_per_sm\": %d, "
                    "\"fft_lpb\": [%d, %d, %d], \"fft_plane\": %d, \"forces_ms\": %lf, "
                    "\"pme_ms\": %lf",
                    &x.split, &x.threads, &x.ctas, &x.lpb[0], &x.lpb[1], &x.lpb[2], &x.plane,
                    &x.pair_ms, &x.pme_ms) == 9) {
      const char *e = std::strstr(line.c_str(), "\"pair_nelec\":");
      if (e && std::sscanf(e, "\"pair_nelec\": %d", &x.nelec) != 1) x.nelec = 1;
      const char *h = std::strstr(line.c_str(), "\"pair_chunks\":");
      if (!h || std::sscanf(h, "\"pair_chunks\": %d", &x.chunks) != 1) x.chunks = 0;
      const char *sc = std::strstr(line.c_str(), "\"spread_cells\":");
      if (!sc || std::sscanf(sc, "\"spread_cells\": %d", &x.spread) != 1) x.spread = 0;
      const char *gr = std::strstr(line.c_str(), "\"pair_group\":");
      if (!gr || std::sscanf(gr, "\"pair_group\": %d", &x.group) != 1) x.group = 1;
      *t = x;  // the last entry for a key wins
      found = true;
    }
  }
  return found;
}

void cache_store(const std::string &key, const Tuned &t) {
  std::lock_guard<std::mutex> g(g_cache_mu);
  std::ofstream f(cache_path(), std::ios::app);
  if (!f) return;
  char buf[512];
  std::snprintf(buf, sizeof buf,
                "{\"key\": \"%s\", \"pair_split\": %d, \"pair_threads\": %d, "
                "\"pair_ctas_per_sm\": %d, \"fft_lpb\": [%d, %d, %d], \"fft_plane\": %d, "
                "\"forces_ms\": %.6f, \"pme_ms\": %.6f, \"pair_nelec\": %d, "
                "\"pair_chunks\": %d, \"spread_cells\": %d, \"pair_group\": %d}\n",
                key.c_str(), t.split, t.threads, t.ctas, t.lpb[0], t.lpb[1], t.lpb[2], t.plane,
                t.pair_ms, t.pme_ms, t.nelec, t.chunks, t.spread, t.group);
  f << buf;
}

// median device time (ms) of `reps` runs of fn after one warm-up
template <typename F>
double time_ms(cudaStream_t st, int reps, F fn) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();
  std::vector<float> v;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    fn();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    v.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(v.begin(), v.end());
  return v[v.size() / 2];
}

}  // namespace

int Engine::autotune(const Pool &Q, cudaStream_t st, int flags, double *pair_ms, double *pme_ms,
                     bool *from_cache) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    set_error("cudaGetDeviceProperties failed");
    return GCME_ERR_CUDA;
  }
  long long ngrid = 0, nq = 0, ncell = 0;
  int geom = 0;
  for (auto &S : hsys) {
    ngrid += (long long)S.K[0] * S.K[1] * S.K[2];
    nq += S.nq_ext;
    ncell += S.ncell;
    geom |= 1 << S.geometry;
  }
  std::ostringstream key;
  key << prop.name << "|nsys=" << hsys.size() << "|n=" << n_real << "|ext=" << n_ext
      << "|q=" << nq << "|cells=" << ncell << "|grid=" << ngrid << "|fp64=" << (int)fp64
      << "|cf=" << cell_factor << "|geom=" << geom << "|list=" << (int)use_list
      << "|species=" << (int)species;
  const bool remeasure = flags & 1, no_cache = flags & 2;
  Tuned t;
  *from_cache = false;
  // one force evaluation for the cell occupancy that orders the pair work
  // items (heaviest first) under every configuration below
  {
    cudaGraphExec_t g0 = nullptr;
    int rc0 = forces_graph(Q, &g0);
    if (rc0) return rc0;
    if (cudaGraphLaunch(g0, st) != cudaSuccess) {
      set_error("autotune: force evaluation failed");
      return GCME_ERR_CUDA;
    }
    rc0 = snapshot_cells(st);
    if (rc0) return rc0;
  }
  if (!remeasure && !no_cache && cache_lookup(key.str(), &t)) {
    int rc = set_pair_config(t.split, t.threads, t.ctas, t.nelec, t.chunks, t.group);
    for (int a = 0; !rc && a < 3; ++a) rc = set_fft_lpb(a, t.lpb[a]);
    if (!rc) rc = set_fft_plane(t.plane != 0);
    if (!rc) rc = set_spread_cells(t.spread != 0 && cell_spread_ok());
    if (!rc) {
      *pair_ms = t.pair_ms;
      *pme_ms = t.pme_ms;
      *from_cache = true;
      return GCME_OK;
    }
  }
  // Every candidate is timed on whole steps (kick and drift, cell list,
  // pair kernel and bonds concurrent with the PME branch, kick and
  // energies), replays of the captured step graph as production runs it:
  // the concurrency is what the launch shapes trade against each other, and
  // the force evaluation alone ranks them differently.  The steps run on a
  // scratch copy of the positions, from rest, after one force evaluation
  // there; the systems' step counters are put back afterwards.
  const int reps = 15;  // median of 15: candidates lie within a few per cent
  const size_t vbytes = (fp64 ? sizeof(double) : sizeof(float)) * 3 * n_real;
  double *spos = nullptr;
  void *svel = nullptr;
  std::vector<unsigned long long> ctr(nsys());
  if (cudaMalloc(&spos, sizeof(double) * 3 * n_real) != cudaSuccess ||
      cudaMalloc(&svel, vbytes) != cudaSuccess) {
    cudaFree(spos);
    set_error("autotune: scratch state allocation failed");
    return GCME_ERR_OOM;
  }
  struct Scratch {  // freed on every return path
    double *p;
    void *v;
    ~Scratch() {
      cudaFree(p);
      cudaFree(v);
    }
  } scratch{spos, svel};
  TUNE_CK(cudaMemcpyAsync(spos, Q.pos, sizeof(double) * 3 * n_real, cudaMemcpyDeviceToDevice, st));
  TUNE_CK(cudaMemsetAsync(svel, 0, vbytes, st));
  TUNE_CK(cudaMemcpyAsync(ctr.data(), P.step_ctr, sizeof(unsigned long long) * ctr.size(),
                          cudaMemcpyDeviceToHost, st));
  TUNE_CK(cudaStreamSynchronize(st));
  Pool T = Q;
  T.pos = spos;
  T.vel = svel;
  cudaGraphExec_t fg = nullptr, sg = nullptr;
  auto timed_n = [&](int n) -> double {
    if (forces_graph(T, &fg) != GCME_OK || step_graph(T, &sg) != GCME_OK) return 1e30;
    cudaGraphLaunch(fg, st);  // forces at the scratch positions
    return time_ms(st, n, [&] { cudaGraphLaunch(sg, st); });
  };
  auto timed = [&]() -> double { return timed_n(reps); };
  double best = 1e30;
  int bs = pair_split, bt = pair_threads, bc = pair_ctas_per_sm, be = pair_nelec,
      bh = pair_chunks, bg = pair_group;
  struct Cand {
    double ms;
    int split, threads, ctas, nelec, chunks;
  };
  std::vector<Cand> cands;
  if (cell_factor == 1 && !use_list) {  // with lists the cell kernel only serves overflows
    // threads, electrostatics warps (0: one warp per work item; negative:
    // every warp takes tasks, the charged candidates in that many parts)
    const int shapes[12][2] = {{128, 1},  {160, 1},  {160, 2},  {192, 2},  {192, 3},  {128, 0},
                               {64, 0},   {128, -1}, {128, -2}, {160, -2}, {192, -2}, {192, -3}};
    for (int split : {3, 9})
      for (const auto &sh : shapes)
        for (int ctas : {0, 3, 4, 5, 6, 7, 8, 10, 12, 14}) {
          const int threads = sh[0], nelec = sh[1];
          if (nelec != 0 && (ctas > 8 || ctas == 7 || ctas > 40 / (threads / 32)))
            continue;  // register-limited residency (64 regs)
          if (nelec == 0 && (split == 3 || ctas < 3 || ctas * (threads / 32) > 28 ||
                             (threads == 64 && ctas < 8)))
            continue;  // shared-memory-limited residency; 9-cell items exceed a warp's slice
          for (int chunks : {1, 0}) {  // warp items: whole home cells, or split by chunks
            if (nelec > 0 && chunks == 1) continue;
            int rc = set_pair_config(split, threads, ctas, nelec, chunks);
            if (rc) return rc;
            cands.push_back({timed(), split, threads, ctas, nelec, chunks});
          }
        }
    // the closest few again, with three times the replays: candidates lie
    // within a few per cent of each other
    std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
    for (size_t k = 0; k < cands.size() && k < 4; ++k) {
      const Cand &c = cands[k];
      int rc = set_pair_config(c.split, c.threads, c.ctas, c.nelec, c.chunks);
      if (rc) return rc;
      const double ms = timed_n(3 * reps);
      if (ms < best) {
        best = ms;
        bs = c.split;
        bt = c.threads;
        bc = c.ctas;
        be = c.nelec;
        bh = c.chunks;
        bg = 1;
      }
    }
    // items of 2 or 3 home cells along x for the fastest CTA-item shape of
    // split 9, around its resident CTAs per SM (larger items, fewer of them)
    for (const Cand &c : cands) {
      if (c.split != 9 || c.nelec == 0) continue;
      for (int group : {2, 3}) {
        bool any = false;  // some system takes the group
        for (int s = 0; s < nsys(); ++s) any = any || group_of(s, group) > 1;
        if (!any) continue;
        const int opts[4] = {0, c.ctas - 1, c.ctas, c.ctas + 1};
        for (int q = 0; q < 4; ++q) {
          const int ctas = opts[q];
          bool seen = false;
          for (int r = 0; r < q; ++r) seen = seen || opts[r] == ctas;
          if (seen || ctas < 0 || ctas == 1 || ctas == 2 || ctas == 7 || ctas > 8 ||
              ctas > 40 / (c.threads / 32))
            continue;  // as in the search above
          int rc = set_pair_config(9, c.threads, ctas, c.nelec, 0, group);
          if (rc) return rc;
          const double ms = timed_n(3 * reps);
          if (ms < best) {
            best = ms;
            bs = 9;
            bt = c.threads;
            bc = ctas;
            be = c.nelec;
            bh = 0;
            bg = group;
          }
        }
      }
      break;  // the fastest such shape only (candidates are sorted)
    }
    int rc = set_pair_config(bs, bt, bc, be, bh, bg);
    if (rc) return rc;
  } else {
    best = timed();
  }
  const size_t rsz = fp64 ? sizeof(double2) : sizeof(float2);
  for (int a = 0; a < 3; ++a) {
    int bl = plan.lpb[a];
    for (int lpb : {4, 8, 16, 32, 64}) {
      if ((2 * (size_t)lpb + 1) * plan.kmax[a] * rsz > kFftSmemLimit) continue;
      int rc = set_fft_lpb(a, lpb);
      if (rc) return rc;
      const double ms = timed();
      if (ms < best) {
        best = ms;
        bl = lpb;
      }
    }
    int rc = set_fft_lpb(a, bl);
    if (rc) return rc;
  }
  if (plane_fits()) {  // x-y plane passes vs per-axis line passes
    const int cur = plan.use_plane;
    int rc = set_fft_plane(!cur);
    if (rc) return rc;
    const double ms = timed();
    if (ms < best) best = ms;
    else if ((rc = set_fft_plane(cur)) != GCME_OK) return rc;
  }
  if (cell_spread_ok()) {  // spread through shared memory by cells vs straight to the grid
    const bool cur = plan.cell_spread != 0;
    int rc = set_spread_cells(!cur);
    if (rc) return rc;
    const double ms = timed();
    if (ms < best) best = ms;
    else if ((rc = set_spread_cells(cur)) != GCME_OK) return rc;
  }
  const double pme_best = time_ms(st, reps, [&] { launch_pme(Q, plan, fp64, false, st); });
  TUNE_CK(cudaMemcpyAsync(P.step_ctr, ctr.data(), sizeof(unsigned long long) * ctr.size(),
                          cudaMemcpyHostToDevice, st));
  TUNE_CK(cudaStreamSynchronize(st));
  clear_graphs();  // the step graphs of the scratch buffers
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("autotune: ") + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  t.split = pair_split;
  t.threads = pair_threads;
  t.ctas = pair_ctas_per_sm;
  t.nelec = pair_nelec;
  t.chunks = pair_chunks;
  t.group = pair_group;
  t.spread = plan.cell_spread;
  t.plane = plan.use_plane;
  for (int a = 0; a < 3; ++a) t.lpb[a] = plan.lpb[a];
  t.pair_ms = best;
  t.pme_ms = pme_best;
  if (!no_cache) cache_store(key.str(), t);
  *pair_ms = best;
  *pme_ms = pme_best;
  return GCME_OK;
}

}  // namespace gcme
