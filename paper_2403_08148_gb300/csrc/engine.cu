// engine.cu -- host side of libgcme: validation, pooled layout, launch
// sequences, CUDA-graph capture and the C ABI of single systems and batches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <algorithm>

#include "engine.h"

namespace gcme {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

#define GCME_CK(call)                                                              \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      set_error(std::string(#call) + ": " + cudaGetErrorString(_e));               \
      return GCME_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

static constexpr double kPi = 3.14159265358979323846;

bool is_smooth(int K) {
  if (K < 1) return false;
  for (int r : {2, 3, 5})
    while (K % r == 0) K /= r;
  return K == 1;
}

std::vector<int> fft_radices(int K) {
  std::vector<int> r;
  while (K % 4 == 0) {
    r.push_back(4);
    K /= 4;
  }
  while (K % 2 == 0) {
    r.push_back(2);
    K /= 2;
  }
  while (K % 3 == 0) {
    r.push_back(3);
    K /= 3;
  }
  while (K % 5 == 0) {
    r.push_back(5);
    K /= 5;
  }
  return r;
}

// Cardinal B-spline M_p(u) (recursion of Essmann et al. 1995), host side.
static double host_bspline(int p, double u) {
  if (u <= 0.0 || u >= p) return 0.0;
  if (p == 2) return 1.0 - std::fabs(u - 1.0);
  return (u * host_bspline(p - 1, u) + (p - u) * host_bspline(p - 1, u - 1.0)) / (p - 1);
}

// |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) e^{2 pi i m k / K}|^2; for odd p
// the zero at m = K/2 takes the mean of the neighbouring values.
static std::vector<double> host_bsp_moduli(int p, int K) {
  std::vector<double> b(K);
  std::vector<char> bad(K, 0);
  for (int m = 0; m < K; ++m) {
    double re = 0, im = 0;
    for (int k = 0; k <= p - 2; ++k) {
      double ph = 2.0 * kPi * m * k / K;
      double Mk = host_bspline(p, k + 1.0);
      re += Mk * std::cos(ph);
      im += Mk * std::sin(ph);
    }
    double den = re * re + im * im;
    if (den > 1e-10) b[m] = 1.0 / den;
    else bad[m] = 1;
  }
  for (int m = 0; m < K; ++m)
    if (bad[m]) b[m] = 0.5 * (b[(m + K - 1) % K] + b[(m + 1) % K]);
  return b;
}

// Small-r Taylor series of the real-space kernel with beta and kappa:
//   g(r) = [erf(beta r) - erf(kappa r)] / r = sum_k g_k r^{2k},
//   h(r) = -g'(r) / r = sum_k h_k r^{2k},
// from erf(x) = 2/sqrt(pi) (x - x^3/3 + x^5/10 - x^7/42).
static void real_series(double b, double k, double g[4], double h[3]) {
  const double c = 2.0 / std::sqrt(kPi);
  const double d1 = b - k, d3 = b * b * b - k * k * k, d5 = std::pow(b, 5) - std::pow(k, 5),
               d7 = std::pow(b, 7) - std::pow(k, 7);
  g[0] = c * d1;
  g[1] = -c * d3 / 3.0;
  g[2] = c * d5 / 10.0;
  g[3] = -c * d7 / 42.0;
  h[0] = c * 2.0 * d3 / 3.0;
  h[1] = -c * 2.0 * d5 / 5.0;
  h[2] = c * d7 / 7.0;
}

// F(w) = erf(sqrt w) / sqrt w and its first two derivatives (an entire
// function of w): the Taylor series (2/sqrt(pi)) sum (-w)^n / (n! (2n + 1))
// for w < 2, else the closed form and the relations w F' = e^-w/sqrt(pi) - F/2,
// w F'' = -e^-w/sqrt(pi) - 3 F'/2 (from d erf(sqrt w)/dw = e^-w / sqrt(pi w)).
static void erf_ratio(double w, double d[3]) {
  const double c = 2.0 / std::sqrt(kPi);
  if (w < 2.0) {
    // term n of F is t_n / (2n + 1) with t_n = (-w)^n / n!; F' and F''
    // shift the series: F' = -sum t_n / (2n + 3), F'' = sum t_n / (2n + 5)
    double f0 = 0.0, f1 = 0.0, f2 = 0.0, t = 1.0;
    for (int n = 0; n < 40; ++n) {
      f0 += t / (2 * n + 1);
      f1 -= t / (2 * n + 3);
      f2 += t / (2 * n + 5);
      t *= -w / (n + 1);
    }
    d[0] = c * f0;
    d[1] = c * f1;
    d[2] = c * f2;
    return;
  }
  const double s = std::sqrt(w), e = std::exp(-w) / std::sqrt(kPi);
  d[0] = std::erf(s) / s;
  d[1] = (e - 0.5 * d[0]) / w;
  d[2] = (-e - 1.5 * d[1]) / w;
}

// Cubic Hermite table of the real-space pair functions in u = r^2 on
// [0, umax]: g(u) = [erf(beta r) - erf(kappa r)] / r = beta F(beta^2 u) -
// kappa F(kappa^2 u) and h(u) = -2 dg/du (= -g'(r) / r), nint intervals;
// entry 2k holds the coefficients of g on interval k in t = u / du - k
// (c0 + t (c1 + t (c2 + t c3))), entry 2k + 1 those of h.  Exact values and
// u-derivatives at the nodes (FP64) make the interpolant C1, with an error
// below du^4 / 384 times the largest fourth u-derivative, which grows as
// beta^8: the caller sizes nint with beta^2 rc^2 (measured against FP64 over
// [0, 9]: ~1e-7 of the maximum with FP32 evaluation for a = 0.15 .. 0.7 d).
static void real_table(double beta, double kappa, double umax, int nint, float4 *out) {
  auto gh = [&](double u, double v[4]) {  // g, dg/du, h, dh/du
    double fb[3], fk[3];
    erf_ratio(beta * beta * u, fb);
    erf_ratio(kappa * kappa * u, fk);
    const double b2 = beta * beta, k2 = kappa * kappa;
    v[0] = beta * fb[0] - kappa * fk[0];
    v[1] = beta * b2 * fb[1] - kappa * k2 * fk[1];
    const double g2 = beta * b2 * b2 * fb[2] - kappa * k2 * k2 * fk[2];
    v[2] = -2.0 * v[1];
    v[3] = -2.0 * g2;
  };
  const double du = umax / nint;
  double a[4], b[4];
  gh(0.0, a);
  for (int k = 0; k < nint; ++k) {
    gh((k + 1) * du, b);
    for (int f = 0; f < 2; ++f) {  // f = 0: g, f = 1: h
      const double y0 = a[2 * f], y1 = b[2 * f], d0 = du * a[2 * f + 1], d1 = du * b[2 * f + 1];
      out[2 * k + f] = make_float4((float)y0, (float)d0, (float)(3.0 * (y1 - y0) - 2.0 * d0 - d1),
                                   (float)(2.0 * (y0 - y1) + d0 + d1));
    }
    for (int t = 0; t < 4; ++t) a[t] = b[t];
  }
}

// Box-derived FP32 constants of the reciprocal-space kernels.
static void box_floats(SysDesc &S) {
  for (int a = 0; a < 3; ++a) S.inv_box[a] = (float)(1.0 / S.box[a]);
  S.pme_cpref = (float)(S.lB / (kPi * S.V));
}

// One species pair's constants (Eq. u_ex with s = sigma_i^2 + sigma_j^2;
// real-space term with beta_ij = sqrt(pi) / (sqrt(2) a_ij)).
static void species_pair(double A, double si, double sj, double ai, double aj, double kappa,
                         PairTab *t32, PairTab64 *t64) {
  const double s = si * si + sj * sj;
  const double pref = A * std::pow(3.0 / (2.0 * kPi * s), 1.5);
  const double expc = 3.0 / (2.0 * s);
  const double beta = std::sqrt(kPi) / (std::sqrt(2.0) * std::sqrt(ai * ai + aj * aj));
  double g[4], h[3];
  real_series(beta, kappa, g, h);
  if (t32) {
    t32->pref = (float)pref;
    t32->c2 = (float)(-expc / std::log(2.0));
    t32->fc = (float)(3.0 / s);
    t32->beta = (float)beta;
    for (int k = 0; k < 4; ++k) t32->sg[k] = (float)g[k];
    for (int k = 0; k < 3; ++k) t32->sh[k] = (float)h[k];
    t32->pad = 0.0f;
  }
  if (t64) {
    t64->pref = pref;
    t64->expc = expc;
    t64->fc = 3.0 / s;
    t64->beta = beta;
    for (int k = 0; k < 4; ++k) t64->sg[k] = g[k];
    for (int k = 0; k < 3; ++k) t64->sh[k] = h[k];
    t64->pad = 0.0;
  }
}

// Fixed-point resolution of the list kernel's pair terms: the largest b
// (<= 31) with every term below 2^30 units of 2^-b.  Bounds over r <= rc:
// the Gaussian-core force (3/s) u r peaks at r = sqrt(s/3); the real-space
// force lB z^2 |g'(r)| and energy lB z^2 g(r) (g decreasing from
// g(0) = 2 (beta - kappa) / sqrt(pi)) are bounded by sampling r; the virial
// terms by force x rc.
static int pair_fix_bits(const SysDesc &S, double qmax) {
  const double s2 = S.gc_expc > 0 ? 1.5 / S.gc_expc : 1.0;  // s = sigma_i^2 + sigma_j^2
  const double f_gc = S.gc_fc * S.gc_pref * std::sqrt(s2 / 3.0) * std::exp(-0.5);
  double dg = 0.0;
  const int ns = 4096;
  for (int k = 1; k <= ns; ++k) {
    const double r = S.rc * k / ns;
    const double g = (std::erf(S.beta * r) - std::erf(S.kappa * r)) / r;
    const double dd = 2.0 / std::sqrt(kPi) *
                      (S.beta * std::exp(-S.beta * S.beta * r * r) -
                       S.kappa * std::exp(-S.kappa * S.kappa * r * r));
    dg = std::max(dg, std::fabs((dd - g) / r));  // |g'(r)|
  }
  const double zz = S.lB * qmax * qmax;
  const double f_el = zz * dg * 1.05;  // sampling margin
  const double u_el = zz * 2.0 * std::fabs(S.beta - S.kappa) / std::sqrt(kPi);
  const double f = f_gc + f_el;
  const double bound = 1.01 * std::max(std::max(f * std::max(1.0, S.rc), S.gc_pref + u_el), 1e-30);
  int b = (int)std::floor(std::log2(std::ldexp(1.0, 30) / bound));
  return std::max(0, std::min(31, b));
}

std::string validate_spec(const SysSpec &sp) {
  const gcme_params &p = sp.p;
  char buf[256];
  if (sp.n < 1) return "n must be >= 1";
  if (sp.n > (1LL << 30)) return "n too large";
  if ((int64_t)sp.q.size() != sp.n) return "charge array size mismatch";
  if (p.geometry < GCME_BULK || p.geometry > GCME_SLAB_IMAGE) return "unknown geometry";
  if (p.precision != GCME_FP32 && p.precision != GCME_FP64) return "unknown precision";
  if (p.pair_path < GCME_PAIR_AUTO || p.pair_path > GCME_PAIR_CELLS)
    return "pair_path must be 0 (auto), 1 (list) or 2 (cells)";
  if (!(p.gamma >= 0.0) || !std::isfinite(p.gamma)) return "gamma must be finite and >= 0";
  if (p.gamma > 0.0 && (!(p.kT >= 0.0) || !std::isfinite(p.kT)))
    return "kT must be finite and >= 0";
  const int nt = p.ntypes;
  if (nt < 0 || nt > GCME_MAX_TYPES) return "ntypes must be in [0, 8]";
  if (!(p.rc > 0) || !(p.kappa > 0) || !(p.lB >= 0)) return "rc, kappa must be > 0 and lB >= 0";
  if (nt == 0 && (!(p.sigma > 0) || !(p.a > 0) || !(p.A >= 0)))
    return "sigma, a must be > 0 and A >= 0";
  for (int t = 0; t < nt; ++t) {
    if (!(p.sigma_tab[t] > 0) || !(p.a_tab[t] > 0) || !std::isfinite(p.sigma_tab[t]) ||
        !std::isfinite(p.a_tab[t]))
      return "species sigma_i and a_i must be finite and > 0";
    for (int u = 0; u < nt; ++u) {
      const double A = p.A_tab[t * GCME_MAX_TYPES + u];
      if (!(A >= 0) || !std::isfinite(A)) return "species A_ij must be finite and >= 0";
      if (A != p.A_tab[u * GCME_MAX_TYPES + t]) return "species table A_ij must be symmetric";
    }
  }
  if (p.frozen_mask != 0 && (nt < 2 || (p.frozen_mask & ~((1 << nt) - 1)) != 0))
    return "frozen_mask needs ntypes >= 2 and bits below ntypes";
  if (!sp.types.empty()) {
    if ((int64_t)sp.types.size() != sp.n) return "species array size mismatch";
    for (int32_t t : sp.types)
      if (t < 0 || t >= std::max(nt, 1)) return "bead species out of range [0, ntypes)";
  }
  for (int a = 0; a < 3; ++a) {
    if (!(p.box[a] >= p.rc * (1.0 + 1e-4))) {
      snprintf(buf, sizeof buf, "box side %d (%g) shorter than the cutoff %g", a, p.box[a], p.rc);
      return buf;
    }
    if (!is_smooth(p.K[a]) || p.K[a] < 4 || p.K[a] > 1024) {
      snprintf(buf, sizeof buf, "grid size K[%d]=%d must be 2^a 3^b 5^c in [4, 1024]", a, p.K[a]);
      return buf;
    }
  }
  if (p.order < 3 || p.order > 8) return "B-spline order must be in [3, 8]";
  for (int a = 0; a < 3; ++a)
    if (p.K[a] < p.order) return "grid size smaller than the spline order";
  double qs = 0.0, qmax = 0.0;
  for (double z : sp.q) {
    if (!std::isfinite(z)) return "non-finite charge";
    qs += z;
    qmax = std::fmax(qmax, std::fabs(z));
  }
  if (std::fabs(qs) > 1e-6) {
    snprintf(buf, sizeof buf, "system is not neutral (net charge %g)", qs);
    return buf;
  }
  // non-collapse condition (Gaussian core model section) for every pair of
  // species present, with their largest charges:
  //   A_ij / sigma_ij^3 > 4 pi^{3/2} |z_i z_j| lB / (3^{3/2} a_ij)
  if (qmax > 0 && p.lB > 0) {
    const int ns = std::max(nt, 1);
    std::vector<double> qm(ns, 0.0);
    for (int64_t i = 0; i < sp.n; ++i) {
      const int t = sp.types.empty() ? 0 : sp.types[i];
      qm[t] = std::fmax(qm[t], std::fabs(sp.q[i]));
    }
    for (int t = 0; t < ns; ++t)
      for (int u = t; u < ns; ++u) {
        if (!(qm[t] * qm[u] > 0)) continue;
        const double st = nt ? p.sigma_tab[t] : p.sigma, su = nt ? p.sigma_tab[u] : p.sigma;
        const double at = nt ? p.a_tab[t] : p.a, au = nt ? p.a_tab[u] : p.a;
        const double A = nt ? p.A_tab[t * GCME_MAX_TYPES + u] : p.A;
        const double sij = std::sqrt(st * st + su * su), aij = std::sqrt(at * at + au * au);
        const double lhs = A / (sij * sij * sij);
        const double rhs =
            4.0 * std::pow(kPi, 1.5) * qm[t] * qm[u] * p.lB / (std::pow(3.0, 1.5) * aij);
        if (!(lhs > rhs)) {
          snprintf(buf, sizeof buf,
                   "non-collapse condition violated (species %d, %d): A/sigma_ij^3 = %g <= "
                   "4 pi^1.5 lB |z z|/(3^1.5 a_ij) = %g",
                   t, u, lhs, rhs);
          return buf;
        }
      }
  }
  if (p.geometry != GCME_BULK) {
    if (!(p.H > 0)) return "slab height H must be > 0";
    double want = p.geometry == GCME_SLAB_NONMETAL ? 3.0 * p.H : 2.0 * p.H;
    if (p.geometry == GCME_SLAB_IMAGE && std::fabs(p.box[2] - want) > 1e-9 * want)
      return "image-charge slab needs box[2] == 2 H";
    if (p.geometry == GCME_SLAB_NONMETAL && p.box[2] < want * (1.0 - 1e-12))
      return "nonmetal slab needs box[2] >= 3 H";
  }
  if (!(p.dt >= 0)) return "dt must be >= 0";
  const int64_t nb = (int64_t)sp.bonds.size() / 2;
  for (int64_t b = 0; b < nb; ++b) {
    int i = sp.bonds[2 * b], j = sp.bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= sp.n || j >= sp.n || i == j) return "bond index out of range";
  }
  return "";
}

Engine::~Engine() { release(); }

void Engine::release() {
  clear_graphs();
  for (auto &e : phase_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (capture_stream) cudaStreamDestroy(capture_stream);
  if (side_stream) cudaStreamDestroy(side_stream);
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (join_ev) cudaEventDestroy(join_ev);
  if (arena_) cudaFree(arena_);
  capture_stream = side_stream = nullptr;
  fork_ev = join_ev = nullptr;
  arena_ = nullptr;
  P = Pool{};
  hsys.clear();
  snap_cnt.clear();  // the occupancy snapshot belongs to the old cell grid
  snap_nimg.clear();
  snap_nq.clear();
}

std::vector<int2> Engine::make_pair_work(int split, bool chunked, int group) const {
  // (system, cell * split + part) for the 27-cell kernel (times pair_nch plus
  // the chunk group for warp items; (row group * 9 + part) for items of
  // `group` home cells), or (system, block * 3 + z-part) for the fine-cell
  // kernel
  std::vector<int2> pw;
  for (int s = 0; s < (int)hsys.size(); ++s) {
    const SysDesc &S = hsys[s];
    if (group_of(s, group) > 1 && cell_factor == 1) {
      const int ngroups = (S.nc[0] + group - 1) / group * S.nc[1] * S.nc[2];
      for (int gi = 0; gi < ngroups; ++gi)
        for (int k = 0; k < 9; ++k) pw.push_back(make_int2(s, gi * 9 + k));
      continue;
    }
    const int nitem = cell_factor == 2 ? S.nb[0] * S.nb[1] * S.nb[2] : S.ncell;
    const int parts = cell_factor == 2 ? 3 : split;
    const int nch = chunked ? S.pair_nch : 1;
    for (int c = 0; c < nitem; ++c)
      for (int k = 0; k < parts; ++k)
        for (int h = 0; h < nch; ++h) pw.push_back(make_int2(s, (c * parts + k) * nch + h));
  }
  return pw;
}

int Engine::chunks_of(int s) const {
  if (pair_chunks > 0) return std::min(kMaxPairChunks, pair_chunks);
  const SysDesc &S = hsys[s];
  double med = (double)S.n / std::max(1, S.ncell);
  if ((long long)snap_cnt.size() >= S.cell_off + S.ncell) {
    std::vector<int> r;
    for (int c = 0; c < S.ncell; ++c) {
      const int k = snap_cnt[S.cell_off + c] - snap_nimg[S.cell_off + c];
      if (k > 0) r.push_back(k);
    }
    if (!r.empty()) {
      std::nth_element(r.begin(), r.begin() + r.size() / 2, r.end());
      med = r[r.size() / 2];
    }
  }
  return std::max(1, std::min(kMaxPairChunks, (int)std::ceil(med / 32.0)));
}

// Tiles of lpb lines along `axis`; the z lines of the plane path cover the
// Hermitian half k0 < K0/2 + 1 of each plane only.
std::vector<int2> Engine::make_fft_work(int axis, int lpb) const {
  std::vector<int2> w;
  const bool half = axis == 2 && plan.use_plane;
  for (int s = 0; s < (int)hsys.size(); ++s) {
    const SysDesc &S = hsys[s];
    const long long k0 = half ? S.K[0] / 2 + 1 : S.K[0];
    const long long nl = k0 * S.K[1] * S.K[2] / S.K[axis];
    const int nt = (int)((nl + lpb - 1) / lpb);
    for (int t = 0; t < nt; ++t) w.push_back(make_int2(s, t));
  }
  return w;
}

void Engine::clear_graphs() {
  for (auto &kv : graphs_) cudaGraphExecDestroy(kv.second);
  graphs_.clear();
  for (auto g : graph_objs_) cudaGraphDestroy(g);
  graph_objs_.clear();
}

// Occupancy of every cell (beads, images, images + charged) from the last
// cell sort, for ordering the pair work items.
int Engine::snapshot_cells(cudaStream_t st) {
  const long long nc = P.n_cells;
  std::vector<int> start(nc + 1);
  snap_nimg.assign(nc, 0);
  snap_nq.assign(nc, 0);
  GCME_CK(cudaStreamSynchronize(st));
  GCME_CK(cudaMemcpy(start.data(), P.cell_start, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost));
  GCME_CK(cudaMemcpy(snap_nimg.data(), P.cell_nimg, sizeof(int) * nc, cudaMemcpyDeviceToHost));
  GCME_CK(cudaMemcpy(snap_nq.data(), P.cell_nq, sizeof(int) * nc, cudaMemcpyDeviceToHost));
  snap_cnt.assign(nc, 0);
  for (long long c = 0; c < nc; ++c) snap_cnt[c] = start[c + 1] - start[c];
  return GCME_OK;
}

// Heaviest work items first (longest-processing-time order), so that the
// last CTAs of the 27-cell kernel are short ones.  Cost of an item: its real
// home beads x the real beads it stages (Gaussian core) + 4 x its charged
// home beads x the charged and image beads it stages (electrostatics).
void Engine::order_by_cost(std::vector<int2> &pw, int split, bool chunked, int group,
                           int tail) const {
  if (snap_cnt.empty() || cell_factor != 1) return;
  std::vector<std::pair<long long, int>> key(pw.size());
  // estimated cost of home cell (cx, cy, cz) against its neighbour cells of
  // `part`: pairs of the Gaussian core + 4 x those of the electrostatics
  auto cell_cost = [&](const SysDesc &S, int cx, int cy, int cz, int part) {
    const long long hg = S.cell_off + cx + S.nc[0] * (cy + S.nc[1] * cz);
    const long long hreal = snap_cnt[hg] - snap_nimg[hg], hq = snap_nq[hg] - snap_nimg[hg];
    const int dz = (split == 3 ? part : part / 3) - 1;
    long long sreal = 0, sq = 0;
    for (int k = 0; k < 27 / split; ++k) {
      const int dx = k % 3 - 1, dy = split == 3 ? k / 3 - 1 : part % 3 - 1;
      const int u[3] = {cx + dx, cy + dy, cz + dz};
      long long v[3];
      for (int a = 0; a < 3; ++a) v[a] = ((u[a] % S.nc[a]) + S.nc[a]) % S.nc[a];
      const long long cg = S.cell_off + v[0] + S.nc[0] * (v[1] + S.nc[1] * v[2]);
      sreal += snap_cnt[cg] - snap_nimg[cg];
      sq += snap_nq[cg];
    }
    return hreal * sreal + 4 * hq * sq;
  };
  for (size_t w = 0; w < pw.size(); ++w) {
    const SysDesc &S = hsys[pw[w].x];
    long long cost = 0;
    if (group_of(pw[w].x, group) > 1) {
      const int ngx = (S.nc[0] + group - 1) / group;
      const int gi = pw[w].y / 9, part = pw[w].y % 9;
      const int x0 = (gi % ngx) * group, cy = (gi / ngx) % S.nc[1], cz = gi / (ngx * S.nc[1]);
      for (int x = x0; x < std::min(x0 + group, S.nc[0]); ++x)
        cost += cell_cost(S, x, cy, cz, part);
    } else {
      const int base = chunked ? pw[w].y / S.pair_nch : pw[w].y;
      const int cloc = base / split, part = base % split;
      cost = cell_cost(S, cloc % S.nc[0], (cloc / S.nc[0]) % S.nc[1],
                       cloc / (S.nc[0] * S.nc[1]), part);
    }
    key[w] = {-cost, (int)w};
  }
  std::stable_sort(key.begin(), key.end());
  std::vector<int2> out(pw.size());
  for (size_t w = 0; w < pw.size(); ++w) out[w] = pw[key[w].second];
  pw.swap(out);
  if (group <= 1 || tail <= 0) return;
  // The cheapest items of several home cells, from the end of the list,
  // become single-cell items (code -1 - (cell * 9 + part)) until `tail`
  // single-cell items end the list: the launch then ends on small items,
  // which even out the CTAs' finishing times.
  std::vector<std::pair<long long, int2>> singles;
  size_t k = pw.size();
  while (k > 0 && (int)singles.size() < tail) {
    const int2 it = pw[--k];
    const SysDesc &S = hsys[it.x];
    if (group_of(it.x, group) <= 1) {  // a system of one home cell per item
      const int cloc = it.y / split, part = it.y % split;
      singles.push_back({cell_cost(S, cloc % S.nc[0], (cloc / S.nc[0]) % S.nc[1],
                                   cloc / (S.nc[0] * S.nc[1]), part), it});
      continue;
    }
    const int ngx = (S.nc[0] + group - 1) / group;
    const int gi = it.y / 9, part = it.y % 9;
    const int x0 = (gi % ngx) * group, cy = (gi / ngx) % S.nc[1], cz = gi / (ngx * S.nc[1]);
    for (int x = x0; x < std::min(x0 + group, S.nc[0]); ++x) {
      const int cloc = x + S.nc[0] * (cy + S.nc[1] * cz);
      singles.push_back({cell_cost(S, x, cy, cz, part), make_int2(it.x, -1 - (cloc * 9 + part))});
    }
  }
  std::stable_sort(singles.begin(), singles.end(),
                   [](const std::pair<long long, int2> &a, const std::pair<long long, int2> &b) {
                     return a.first > b.first;
                   });
  pw.resize(k);
  for (const auto &sv : singles) pw.push_back(sv.second);
}

// Valid shapes of the 27-cell FP32 kernel: split 3 or 9 and either CTA
// items (128, 160 or 192 threads, 1-3 electrostatics warps and at least 2
// core warps, 0-8 resident CTAs per SM) or, with nelec 0, one warp per item
// (64, 96 or 128 threads, at most 28 resident warps per SM by shared memory).
static bool pair_shape_ok(int split, int threads, int ctas_per_sm, int nelec) {
  const bool ok_warp = nelec == 0 && (threads == 64 || threads == 96 || threads == 128) &&
                       ctas_per_sm >= 1 && ctas_per_sm * (threads / 32) <= 28;
  const bool ok_cta = nelec >= 1 && nelec <= 3 &&
                      (threads == 128 || threads == 160 || threads == 192) &&
                      ctas_per_sm >= 0 && ctas_per_sm <= 8 && threads / 32 - nelec >= 2;
  // tasks taken dynamically, the charged candidates in -nelec parts
  const bool ok_dyn = nelec <= -1 && nelec >= -3 &&
                      (threads == 128 || threads == 160 || threads == 192) &&
                      ctas_per_sm >= 0 && ctas_per_sm <= 8;
  return (split == 3 || split == 9) && (ok_warp || ok_cta || ok_dyn);
}

// Home cells per CTA item: 1, or 2..3 with split 9 CTA items on the 27-cell
// stencil.  A system takes the group when it has at least group + 2 cells
// along x (the staged cells of an item are then distinct), else one home
// cell per item.
bool Engine::pair_group_ok(int split, int nelec, int group) const {
  if (group == 1) return true;
  return group >= 2 && group <= 3 && split == 9 && nelec != 0 && cell_factor == 1;
}

int Engine::group_of(int s, int group) const {
  return group > 1 && hsys[s].nc[0] >= group + 2 ? group : 1;
}

int Engine::set_pair_config(int split, int threads, int ctas_per_sm, int nelec, int chunks,
                            int group) {
  if (!pair_shape_ok(split, threads, ctas_per_sm, nelec) || chunks < 0 ||
      chunks > kMaxPairChunks) {
    set_error("pair configuration must be split 3|9 and either 128|160|192 threads, 1..3 "
              "electrostatics warps (at least 2 core warps) or -1..-3 (tasks taken "
              "dynamically, the charged candidates in that many parts), 0..8 CTAs per SM, "
              "or warp items (0 electrostatics warps): 64|96|128 threads, 1..28 resident "
              "warps per SM");
    return GCME_ERR_INVALID;
  }
  if (!pair_group_ok(split, nelec, group)) {
    set_error("pair_group must be 1, or 2..3 with split 9 CTA items (1..3 electrostatics "
              "warps)");
    return GCME_ERR_INVALID;
  }
  pair_ctas_per_sm = ctas_per_sm;
  const bool chunked = nelec == 0;
  pair_chunks = chunked ? chunks : 0;
  for (int s = 0; s < (int)hsys.size(); ++s) {
    hsys[s].pair_split = split;
    hsys[s].pair_nelec = nelec;
    hsys[s].pair_nch = chunked ? chunks_of(s) : 1;
    hsys[s].pair_group = group_of(s, group);
  }
  std::vector<int2> pw = make_pair_work(split, chunked, group);
  // with items of several home cells: two single-cell items per resident CTA
  // at the end of the list
  order_by_cost(pw, split, chunked, group,
                2 * (ctas_per_sm > 0 ? ctas_per_sm : kTailCtasPerSm) * n_sm);
  pair_split = split;
  pair_threads = threads;
  pair_nelec = nelec;
  pair_group = group;
  pair_groups_on = false;
  for (int s = 0; s < (int)hsys.size(); ++s) pair_groups_on |= hsys[s].pair_group > 1;
  GCME_CK(cudaMemcpy(const_cast<SysDesc *>(P.sys), hsys.data(), sizeof(SysDesc) * hsys.size(),
                     cudaMemcpyHostToDevice));
  GCME_CK(cudaMemcpy(pair_work, pw.data(), sizeof(int2) * pw.size(), cudaMemcpyHostToDevice));
  n_pair_work = (int)pw.size();
  clear_graphs();
  return GCME_OK;
}

bool Engine::plane_fits() const {
  const size_t rsz = fp64 ? sizeof(double2) : sizeof(float2);
  return plan.plane_elems > 0 &&
         (2 * (size_t)plan.plane_elems + plan.kmax[0] + plan.kmax[1]) * rsz <= kFftSmemLimit;
}

int Engine::set_fft_plane(bool on) {
  if (on && !plane_fits()) {
    set_error("x-y planes of this batch do not fit in shared memory");
    return GCME_ERR_INVALID;
  }
  plan.use_plane = on ? 1 : 0;
  // the z-pass tiles follow: half or full spectrum lines
  std::vector<int2> w = make_fft_work(2, plan.lpb[2]);
  GCME_CK(cudaMemcpy(const_cast<int2 *>(plan.work[2]), w.data(), sizeof(int2) * w.size(),
                     cudaMemcpyHostToDevice));
  plan.nwork[2] = (int)w.size();
  clear_graphs();
  return GCME_OK;
}

int Engine::set_spread_cells(bool on) {
  if (on && !cell_spread_ok()) {
    set_error("the cell spread needs the FP32 27-cell path without neighbour lists");
    return GCME_ERR_INVALID;
  }
  plan.cell_spread = on ? 1 : 0;
  clear_graphs();
  return GCME_OK;
}

int Engine::apply_tuning(int split, int threads, int ctas_per_sm, int nelec, const int lpb[3],
                         bool plane, int chunks, bool spread_cells, int group) {
  const bool pair_shapes = cell_factor == 1 && !use_list;
  const size_t rsz = fp64 ? sizeof(double2) : sizeof(float2);
  bool ok = !(plane && !plane_fits());
  for (int a = 0; a < 3; ++a)
    ok = ok && lpb[a] >= kMinLpb && lpb[a] <= 64 &&
         (2 * (size_t)lpb[a] + 1) * plan.kmax[a] * rsz <= kFftSmemLimit;
  if (pair_shapes)
    ok = ok && pair_shape_ok(split, threads, ctas_per_sm, nelec) && chunks >= 0 &&
         chunks <= kMaxPairChunks && pair_group_ok(split, nelec, group);
  ok = ok && !(spread_cells && !cell_spread_ok());
  if (!ok) {
    set_error("launch shapes out of range or larger than shared memory");
    return GCME_ERR_INVALID;
  }
  int rc = pair_shapes ? set_pair_config(split, threads, ctas_per_sm, nelec, chunks, group)
                       : GCME_OK;
  for (int a = 0; !rc && a < 3; ++a) rc = set_fft_lpb(a, lpb[a]);
  if (!rc) rc = set_fft_plane(plane);
  if (!rc) rc = set_spread_cells(spread_cells);
  return rc;
}

int Engine::set_fft_lpb(int axis, int lpb) {
  const size_t rsz = fp64 ? sizeof(double2) : sizeof(float2);
  if (axis < 0 || axis > 2 || lpb < kMinLpb || lpb > 64 ||
      (2 * (size_t)lpb + 1) * plan.kmax[axis] * rsz > kFftSmemLimit) {
    set_error("FFT lines per tile out of range");
    return GCME_ERR_INVALID;
  }
  std::vector<int2> w = make_fft_work(axis, lpb);
  GCME_CK(cudaMemcpy(const_cast<int2 *>(plan.work[axis]), w.data(), sizeof(int2) * w.size(),
                     cudaMemcpyHostToDevice));
  plan.lpb[axis] = lpb;
  plan.nwork[axis] = (int)w.size();
  clear_graphs();
  return GCME_OK;
}

namespace {
struct Carver {
  size_t off = 0;
  std::vector<std::pair<void **, size_t>> req;
  template <typename T>
  void add(T **p, long long count) {
    size_t bytes = (size_t)(count > 0 ? count : 0) * sizeof(T);
    req.push_back({reinterpret_cast<void **>(p), bytes});
    off += (bytes + 255) / 256 * 256;
  }
};
}  // namespace

int Engine::build(int dev, const std::vector<SysSpec> &specs, bool own_state) {
  device = dev;
  GCME_CK(cudaSetDevice(dev));
  GCME_CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int ns = (int)specs.size();
  if (ns < 1) {
    set_error("empty batch");
    return GCME_ERR_INVALID;
  }
  fp64 = specs[0].p.precision == GCME_FP64;
  cell_factor = 0;
  for (auto &sp : specs) {
    if (sp.p.cell_factor != 0 && sp.p.cell_factor != 1 && sp.p.cell_factor != 2) {
      set_error("cell_factor must be 0, 1 or 2");
      return GCME_ERR_INVALID;
    }
    if (sp.p.cell_factor != 0) {
      if (cell_factor != 0 && cell_factor != sp.p.cell_factor) {
        set_error("all systems of a batch must share one cell factor");
        return GCME_ERR_INVALID;
      }
      cell_factor = sp.p.cell_factor;
    }
  }
  if (cell_factor == 0) cell_factor = kDefaultCellFactor;
  if (pair_split != 3 && pair_split != 9) pair_split = kDefaultPairSplit;
  int path = GCME_PAIR_AUTO;
  for (auto &sp : specs) {
    const int pp = sp.p.pair_path;
    if (pp != GCME_PAIR_AUTO && pp != GCME_PAIR_LIST && pp != GCME_PAIR_CELLS) {
      set_error("pair_path must be 0 (auto), 1 (list) or 2 (cells)");
      return GCME_ERR_INVALID;
    }
    if (pp != GCME_PAIR_AUTO) {
      if (path != GCME_PAIR_AUTO && path != pp) {
        set_error("all systems of a batch must share one pair path");
        return GCME_ERR_INVALID;
      }
      path = pp;
    }
  }
  for (auto &sp : specs) {
    std::string err = validate_spec(sp);
    if (!err.empty()) {
      set_error(err);
      return GCME_ERR_INVALID;
    }
    if ((sp.p.precision == GCME_FP64) != fp64) {
      set_error("all systems of a batch must share one precision");
      return GCME_ERR_INVALID;
    }
  }
  // several species: a system with ntypes >= 2 makes the whole batch take
  // per-pair constants from tables (a one-species table is the scalars)
  species = false;
  for (auto &sp : specs) species = species || sp.p.ntypes >= 2;
  if (species && (fp64 ? false : (cell_factor == 2))) {
    set_error("several species need cell_factor 1 (27-cell kernel) or the FP64 path");
    return GCME_ERR_INVALID;
  }
  hsys.assign(ns, SysDesc{});
  std::vector<gcme_params> eff(ns);
  bead_off.assign(ns + 1, 0);
  long long nr = 0, ne = 0, nq = 0, nimg = 0, ncell = 0, ngrid = 0, nbond = 0;
  int ntw = 0;
  std::vector<std::vector<int>> qlists(ns), imgs(ns);
  for (int s = 0; s < ns; ++s) {
    const SysSpec &sp = specs[s];
    gcme_params &p = eff[s];
    p = sp.p;
    if (p.ntypes == 1) {  // one species: its table entries are the scalars
      p.A = p.A_tab[0];
      p.sigma = p.sigma_tab[0];
      p.a = p.a_tab[0];
      p.ntypes = 0;
    }
    SysDesc &S = hsys[s];
    S.n = (int)sp.n;
    std::vector<int> &ql = qlists[s];
    std::vector<int> &im = imgs[s];
    for (int i = 0; i < S.n; ++i)
      if (sp.q[i] != 0.0) ql.push_back(i);
    S.nq_real = (int)ql.size();
    if (p.geometry == GCME_SLAB_IMAGE) {
      im = ql;
      for (int k = 0; k < (int)im.size(); ++k) ql.push_back(S.n + k);
    }
    S.n_ext = S.n + (int)im.size();
    S.nq_ext = (int)ql.size();
    S.geometry = p.geometry;
    S.precision = p.precision;
    S.nbond = (int)(sp.bonds.size() / 2);
    S.bead_off = nr;
    S.ext_off = ne;
    S.q_off = nq;
    S.img_off = nimg;
    S.cell_off = ncell;
    S.grid_off = ngrid;
    S.bond_off = nbond;
    S.ncell = 1;
    S.cell_factor = cell_factor;
    S.pair_split = pair_split;
    S.pair_nelec = pair_nelec;
    S.pair_nch = 1;
    S.pair_group = 1;
    for (int a = 0; a < 3; ++a) {
      S.nc[a] = cells_per_axis(p.box[a], p.rc, cell_factor);
      S.nb[a] = (S.nc[a] + 1) / 2;
      S.ncell *= S.nc[a];
      set_cell_box_axis(S, a, p.box[a]);
      S.K[a] = p.K[a];
      S.kfac[a] = (float)((double)p.K[a] / p.box[a]);
      S.tw_off[a] = ntw;
      S.bsp_off[a] = ntw;
      ntw += p.K[a];
      std::vector<int> r = fft_radices(p.K[a]);
      S.nstage[a] = (int)r.size();
      for (int k = 0; k < (int)r.size(); ++k) S.radix[a][k] = r[k];
    }
    S.order = p.order;
    S.rc2f = (float)(p.rc * p.rc);
    S.cull2 = (float)((p.rc + 1e-3) * (p.rc + 1e-3));
    S.V = p.box[0] * p.box[1] * p.box[2];
    S.A = p.A;
    S.sigma = p.sigma;
    S.a = p.a;
    S.lB = p.lB;
    S.rc = p.rc;
    S.kappa = p.kappa;
    const double s2 = 2.0 * p.sigma * p.sigma;           // sigma_i^2 + sigma_j^2
    const double aij = std::sqrt(2.0) * p.a;              // a_ij
    S.beta = std::sqrt(kPi) / (std::sqrt(2.0) * aij);
    S.gc_pref = p.A * std::pow(3.0 / (2.0 * kPi * s2), 1.5);
    S.gc_expc = 3.0 / (2.0 * s2);
    S.gc_fc = 3.0 / s2;
    S.gc_c2f = (float)(-S.gc_expc / std::log(2.0));
    S.gc_tail = std::exp(-S.gc_expc * p.rc * p.rc) < 1e-10 ? 1 : 0;
    double sq = 0.0, born = 0.0;  // sum z^2, sum z^2 / (2 a_i)
    for (int i = 0; i < S.n; ++i) {
      const double z = sp.q[i];
      const double ai = (p.ntypes && !sp.types.empty()) ? p.a_tab[sp.types[i]]
                        : (p.ntypes ? p.a_tab[0] : p.a);
      sq += z * z;
      born += z * z / (2.0 * ai);
    }
    S.e_corr = -p.lB * p.kappa / std::sqrt(kPi) * sq;
    S.e_self = p.lB * born;
    S.recip_scale = p.geometry == GCME_SLAB_IMAGE ? 0.5 : 1.0;
    S.H = p.H;
    S.wall_A = p.geometry == GCME_BULK ? 0.0 : p.wall_A;
    S.wall_s2 = p.wall_sigma2 > 0 ? p.wall_sigma2 : 1.0;
    S.bond_k = p.bond_k;
    S.bond_r0 = p.bond_r0;
    S.dt = p.dt;
    S.langevin = p.gamma > 0.0 ? 1 : 0;
    S.lgv_c1 = std::exp(-p.gamma * p.dt);
    S.lgv_c2 = S.langevin ? std::sqrt((1.0 - S.lgv_c1 * S.lgv_c1) * p.kT) : 0.0;
    S.seed = p.seed;
    real_series(S.beta, p.kappa, S.ser_g, S.ser_h);
    for (int t = 0; t < 4; ++t) S.ser_gf[t] = (float)S.ser_g[t];
    for (int t = 0; t < 3; ++t) S.ser_hf[t] = (float)S.ser_h[t];
    S.betaf = (float)S.beta;
    S.kappaf = (float)p.kappa;
    S.gc_forcef = (float)(S.gc_fc * S.gc_pref);
    S.gc_halfpref = (float)(0.5 * S.gc_pref);
    S.lbf = (float)p.lB;
    S.lb_half = (float)(0.5 * p.lB);
    S.pme_pi2k2 = (float)(kPi * kPi / (p.kappa * p.kappa));
    S.recip_scalef = (float)S.recip_scale;
    S.half_dtf = (float)(0.5 * p.dt);
    S.bond_kf = (float)p.bond_k;
    S.bond_r0f = (float)p.bond_r0;
    box_floats(S);
    {
      double qmax = 0.0;
      for (double z : sp.q) qmax = std::max(qmax, std::fabs(z));
      S.fix_bits = pair_fix_bits(S, qmax);
      S.fix_scale = (float)std::ldexp(1.0, S.fix_bits);
    }
    nr += S.n;
    ne += S.n_ext;
    nq += S.nq_ext;
    nimg += (long long)im.size();
    ncell += S.ncell;
    ngrid += (long long)p.K[0] * p.K[1] * p.K[2];
    nbond += S.nbond;
    bead_off[s + 1] = nr;
  }
  n_real = nr;
  n_ext = ne;
  // species tables (ntypes x ntypes per system) and the species of every
  // ext bead (images: their source's)
  std::vector<PairTab> htab;
  std::vector<PairTab64> htab64;
  std::vector<unsigned char> htype;
  if (species) {
    htype.assign(ne, 0);
    for (int s = 0; s < ns; ++s) {
      SysDesc &S = hsys[s];
      const gcme_params &p = eff[s];
      const SysSpec &sp = specs[s];
      const int nt = std::max(p.ntypes, 1);
      S.ntypes = nt;
      S.frozen_mask = p.frozen_mask;
      S.tab_off = fp64 ? (long long)htab64.size() : (long long)htab.size();
      for (int t = 0; t < nt; ++t)
        for (int u = 0; u < nt; ++u) {
          const double A = p.ntypes ? p.A_tab[t * GCME_MAX_TYPES + u] : p.A;
          const double st = p.ntypes ? p.sigma_tab[t] : p.sigma;
          const double su = p.ntypes ? p.sigma_tab[u] : p.sigma;
          const double at = p.ntypes ? p.a_tab[t] : p.a, au = p.ntypes ? p.a_tab[u] : p.a;
          PairTab t32;
          PairTab64 t64;
          species_pair(A, st, su, at, au, p.kappa, &t32, &t64);
          if (fp64) htab64.push_back(t64);
          else htab.push_back(t32);
        }
      for (int i = 0; i < S.n; ++i)
        htype[S.ext_off + i] = (unsigned char)(sp.types.empty() ? 0 : sp.types[i]);
      for (size_t k = 0; k < imgs[s].size(); ++k)
        htype[S.ext_off + S.n + k] = htype[S.ext_off + imgs[s][k]];
    }
  }
  // real-space tables of the FP32 one-species path (per system: its beta,
  // kappa and cutoff)
  std::vector<float4> hrtab;
  if (!fp64 && !species) {
    for (auto &S : hsys) {
      const double umax = (double)S.rc2f;
      const double nd = std::ceil(18.25 * S.beta * S.beta * umax);
      S.rtab_n = nd > kRealTabMax ? 0 : std::max(kRealTabMin, (int)nd);
      S.rtab_off = (long long)hrtab.size();
      if (!S.rtab_n) continue;  // direct evaluation
      S.rtab_scale = (float)(S.rtab_n / umax);
      hrtab.resize(hrtab.size() + 2 * (size_t)S.rtab_n);
      real_table(S.beta, S.kappa, umax, S.rtab_n, hrtab.data() + S.rtab_off);
    }
  }
  // Neighbour lists: FP32 path, 27-cell stencil, and the two-cell build
  // stencil must cover rc + skin (cells of side >= rc >= skin).
  {
    bool can = !fp64 && cell_factor == 1 && ne < (1LL << 25) && !species;
    for (auto &sp : specs) can = can && sp.p.rc >= kListSkin;
    if (path == GCME_PAIR_LIST && !can) {
      set_error("pair_path LIST needs FP32, one species, cell_factor 1, rc >= 0.4 and fewer "
                "than 2^25 beads");
      return GCME_ERR_INVALID;
    }
    // AUTO takes the 27-cell kernel: on dense soft-core fluids (~340
    // neighbours within rc, a rebuild every few steps) it is the faster path
    use_list = can && path == GCME_PAIR_LIST;
  }
  // list entries per bead and lane: a quarter of the expected count within
  // rc + skin at the densest system's mean fluid density (slabs: beads over
  // the slab volume), times 1.6, plus 32
  int list_stride = 0;
  if (use_list) {
    double need = 0.0;
    for (int s = 0; s < ns; ++s) {
      const SysDesc &S = hsys[s];
      const double rl = S.rc + kListSkin;
      double vol = S.V;
      if (S.geometry != GCME_BULK && S.H > 0)
        vol = std::min(vol, S.box[0] * S.box[1] * S.H);
      const double rho = S.n / vol;
      need = std::max(need, rho * 4.0 / 3.0 * kPi * rl * rl * rl);
    }
    list_stride = (int)std::ceil(1.6 * need / 4.0) + 32;
    for (auto &S : hsys) {
      const double rl = S.rc + kListSkin;
      S.rl2f = (float)(rl * rl);
    }
  }
  // FFT plan and pair work lists (rebuilt by the autotuner)
  for (int a = 0; a < 3; ++a) {
    plan.kmax[a] = 0;
    for (auto &S : hsys) plan.kmax[a] = std::max(plan.kmax[a], S.K[a]);
    int lpb = 64;  // largest power of two <= 1024 / K, within [8, 64]
    while (lpb > 8 && lpb * plan.kmax[a] > 1024) lpb /= 2;
    plan.lpb[a] = lpb;
  }
  // plane passes: one work item per pair of z-planes (2p, 2p + 1)
  std::vector<int2> planes;
  plan.plane_elems = 0;
  for (int s = 0; s < ns; ++s) {
    plan.plane_elems = std::max(plan.plane_elems, hsys[s].K[0] * hsys[s].K[1]);
    for (int z = 0; z < (hsys[s].K[2] + 1) / 2; ++z) planes.push_back(make_int2(s, z));
  }
  plan.nplane = (int)planes.size();
  plan.order = hsys[0].order;
  for (auto &S : hsys)
    if (S.order != plan.order) plan.order = 0;
  plan.cell_spread = 0;  // charges straight to the global grid unless tuned otherwise
  std::vector<int2> fftw[3];
  int fft_cap[3];
  plan.use_plane = 0;  // capacities for the full-spectrum lines
  for (int a = 0; a < 3; ++a) fft_cap[a] = (int)make_fft_work(a, kMinLpb).size();
  plan.use_plane = plane_fits() ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    fftw[a] = make_fft_work(a, plan.lpb[a]);
    plan.nwork[a] = (int)fftw[a].size();
  }
  std::vector<int2> pw = make_pair_work(pair_split);
  n_pair_work = (int)pw.size();
  const int pair_cap = std::max(n_pair_work, kMaxPairChunks * (int)make_pair_work(9).size());

  // ---- device arena
  Carver cv;
  SysDesc *d_sys = nullptr;
  cv.add(&d_sys, ns);
  P = Pool{};
  P.nsys = ns;
  if (own_state) {
    cv.add(&P.pos, 3 * nr);
    if (fp64) cv.add(reinterpret_cast<double **>(&P.vel), 3 * nr);
    else cv.add(reinterpret_cast<float **>(&P.vel), 3 * nr);
  }
  double *d_q = nullptr;
  cv.add(&d_q, nr);
  cv.add(&P.force, 3 * nr);
  cv.add(&P.xyzq_u, ne);
  if (fp64) cv.add(&P.xyzq_u64, ne);
  cv.add(&P.cell_of, ne);
  cv.add(&P.slot, ne);
  cv.add(&P.wrap_n, 3 * ne);
  cv.add(&P.sorted_idx, ne);
  cv.add(&P.sort_tmp, ne);
  cv.add(&P.xyzq_s, ne);
  if (fp64) cv.add(&P.xyzq_s64, ne);
  cv.add(&P.ext_sys, ne);
  cv.add(&P.real_sys, nr);
  cv.add(&P.qlist, nq);
  cv.add(&P.q_sys, nq);
  cv.add(&P.img_src, nimg);
  cv.add(&P.ext_src, ne);
  cv.add(&P.cell_cnt, ncell);
  cv.add(&P.cell_start, ncell + 1);
  // fused cell sort for small per-system grids; bucket capacity twice the
  // densest expected cell (slabs: the beads fill H of the box height) + 32
  int bucket_cap = 0;
  {
    bool fused = true;
    double occ = 0.0;
    for (auto &S : hsys) {
      // (bucket entries carry the class in their top two bits)
      fused = fused && S.ncell <= kFusedSortCells && S.n_ext < (1LL << 30);
      double fill = 1.0;
      if (S.geometry != GCME_BULK && S.H > 0) fill = std::min(1.0, S.H / S.box[2]);
      occ = std::max(occ, S.n_ext / (S.ncell * fill));
    }
    if (fused) bucket_cap = ((int)std::ceil(2.0 * occ) + 32 + 31) / 32 * 32;
  }
  cv.add(&P.bucket, (long long)ncell * bucket_cap);
  cv.add(&P.bucket_pos, (long long)ncell * bucket_cap);
  cv.add(&P.cell_nimg, ncell);
  cv.add(&P.cell_nq, ncell);
  cv.add(&P.cell_sys, ncell);
  cv.add(&P.qgrid, ngrid);
  if (fp64) {
    cv.add(&P.cgrid64, ngrid);
    cv.add(&P.tw64, ntw);
    cv.add(&P.bsp64, ntw);
  } else {
    cv.add(&P.cgrid, ngrid);
    cv.add(&P.tw, ntw);
    cv.add(&P.bsp, ntw);
  }
  cv.add(&P.bonds, nbond);
  cv.add(&P.bond_sys, nbond);
  cv.add(&P.acc, (long long)ns * kNacc);
  cv.add(&P.vacc, (long long)ns * 9);
  cv.add(&P.energy, (long long)ns * GCME_NTERMS);
  cv.add(&P.virial, (long long)ns * 9);
  cv.add(&pair_work, pair_cap);
  cv.add(&bar_words, 4);
  cv.add(&P.step_ctr, ns);
  cv.add(&step_stop_buf, ns);
  cv.add(&P.held, ns);
  cv.add(&pair_counter, 1);
  int2 *fw[3];
  for (int a = 0; a < 3; ++a) cv.add(&fw[a], fft_cap[a]);
  int2 *d_planes = nullptr;
  cv.add(&d_planes, plan.nplane);
  if (use_list) {
    cv.add(&P.nbr, (long long)list_stride * ne * 4);
    cv.add(&P.nbr_cnt, ne);
    cv.add(&P.nbr_nq, ne);
    cv.add(&P.img_now, 3 * ne);
    cv.add(&P.img_ref, 3 * ne);
    cv.add(&P.dimg_s, ne);
    cv.add(&P.x_ref, 3 * nr);
    cv.add(&P.list_flags, 4);
    cv.add(&P.list_ovf, 2 * (long long)ns);
  }
  PairTab *d_tab = nullptr;
  PairTab64 *d_tab64 = nullptr;
  float4 *d_rtab = nullptr;
  cv.add(&d_rtab, (long long)hrtab.size());
  if (species) {
    cv.add(&P.type_u, ne);
    cv.add(&P.type_s, ne);
    if (fp64) cv.add(&d_tab64, (long long)htab64.size());
    else cv.add(&d_tab, (long long)htab.size());
  }
  scratch_bytes = cv.off;
  cudaError_t e = cudaMalloc(&arena_, cv.off);
  if (e != cudaSuccess) {
    set_error(std::string("device allocation of ") + std::to_string(cv.off) +
              " bytes failed: " + cudaGetErrorString(e));
    arena_ = nullptr;
    return GCME_ERR_OOM;
  }
  size_t off = 0;
  for (auto &r : cv.req) {
    *r.first = r.second ? static_cast<char *>(arena_) + off : nullptr;
    off += (r.second + 255) / 256 * 256;
  }
  P.sys = d_sys;
  P.q = d_q;
  P.any_slab = 0;
  for (auto &S : hsys) P.any_slab |= S.geometry != GCME_BULK;
  P.n_real = nr;
  P.n_ext = ne;
  P.n_cells = ncell;
  P.bucket_cap = P.bucket ? bucket_cap : 0;
  P.n_q = nq;
  P.n_bond = nbond;
  P.n_grid = ngrid;
  for (int a = 0; a < 3; ++a) plan.work[a] = fw[a];
  plan.plane_work = d_planes;
  P.ptab = d_tab;
  P.ptab64 = d_tab64;
  P.rtab = hrtab.empty() ? nullptr : d_rtab;
  if (use_list) {
    P.nbr_stride = list_stride;
    P.gate = P.list_flags;
    const double h = 0.5 * kListSkin - 1e-4;  // margin far above FP32 rounding of r
    P.half_skin2 = h * h;
  }

  // ---- host tables -> device
  std::vector<double> hq(nr);
  std::vector<int> h_ext_sys(ne), h_real_sys(nr), h_ql(nq), h_qs(nq), h_img(nimg), h_cs(ncell);
  std::vector<int> h_ext_src(ne);
  std::vector<int2> h_bonds(nbond);
  std::vector<int> h_bsys(nbond);
  std::vector<float2> htw(fp64 ? 0 : ntw);
  std::vector<double2> htw64(fp64 ? ntw : 0);
  std::vector<float> hbsp(fp64 ? 0 : ntw);
  std::vector<double> hbsp64(fp64 ? ntw : 0);
  for (int s = 0; s < ns; ++s) {
    const SysDesc &S = hsys[s];
    const SysSpec &sp = specs[s];
    for (int i = 0; i < S.n; ++i) {
      hq[S.bead_off + i] = sp.q[i];
      h_real_sys[S.bead_off + i] = s;
    }
    for (int e2 = 0; e2 < S.n_ext; ++e2) h_ext_sys[S.ext_off + e2] = s;
    for (int k = 0; k < S.nq_ext; ++k) {
      h_ql[S.q_off + k] = qlists[s][k];
      h_qs[S.q_off + k] = s;
    }
    for (int k = 0; k < (int)imgs[s].size(); ++k) h_img[S.img_off + k] = imgs[s][k];
    for (int e2 = 0; e2 < S.n; ++e2) h_ext_src[S.ext_off + e2] = (int)(S.bead_off + e2);
    for (int k = 0; k < (int)imgs[s].size(); ++k)
      h_ext_src[S.ext_off + S.n + k] = -1 - (int)(S.bead_off + imgs[s][k]);
    for (int c = 0; c < S.ncell; ++c) h_cs[S.cell_off + c] = s;
    for (int b = 0; b < S.nbond; ++b) {
      h_bonds[S.bond_off + b] = make_int2(sp.bonds[2 * b], sp.bonds[2 * b + 1]);
      h_bsys[S.bond_off + b] = s;
    }
    for (int a = 0; a < 3; ++a) {
      const int K = S.K[a];
      std::vector<double> bm = host_bsp_moduli(S.order, K);
      for (int t = 0; t < K; ++t) {
        const double ang = -2.0 * kPi * t / K;
        if (fp64) {
          htw64[S.tw_off[a] + t] = make_double2(std::cos(ang), std::sin(ang));
          hbsp64[S.bsp_off[a] + t] = bm[t];
        } else {
          htw[S.tw_off[a] + t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
          hbsp[S.bsp_off[a] + t] = (float)bm[t];
        }
      }
    }
  }
  GCME_CK(cudaMemcpy(d_sys, hsys.data(), sizeof(SysDesc) * ns, cudaMemcpyHostToDevice));
  auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  GCME_CK(up(d_q, hq.data(), sizeof(double) * nr));
  GCME_CK(up(P.ext_sys, h_ext_sys.data(), sizeof(int) * ne));
  GCME_CK(up(P.real_sys, h_real_sys.data(), sizeof(int) * nr));
  GCME_CK(up(P.qlist, h_ql.data(), sizeof(int) * nq));
  GCME_CK(up(P.q_sys, h_qs.data(), sizeof(int) * nq));
  GCME_CK(up(P.img_src, h_img.data(), sizeof(int) * nimg));
  GCME_CK(up(P.ext_src, h_ext_src.data(), sizeof(int) * ne));
  GCME_CK(up(P.cell_sys, h_cs.data(), sizeof(int) * ncell));
  GCME_CK(up(P.bonds, h_bonds.data(), sizeof(int2) * nbond));
  GCME_CK(up(P.bond_sys, h_bsys.data(), sizeof(int) * nbond));
  if (fp64) {
    GCME_CK(up(P.tw64, htw64.data(), sizeof(double2) * ntw));
    GCME_CK(up(P.bsp64, hbsp64.data(), sizeof(double) * ntw));
  } else {
    GCME_CK(up(P.tw, htw.data(), sizeof(float2) * ntw));
    GCME_CK(up(P.bsp, hbsp.data(), sizeof(float) * ntw));
  }
  GCME_CK(up(pair_work, pw.data(), sizeof(int2) * n_pair_work));
  for (int a = 0; a < 3; ++a) GCME_CK(up(fw[a], fftw[a].data(), sizeof(int2) * plan.nwork[a]));
  GCME_CK(up(d_planes, planes.data(), sizeof(int2) * plan.nplane));
  if (!hrtab.empty()) GCME_CK(up(d_rtab, hrtab.data(), sizeof(float4) * hrtab.size()));
  if (species) {
    GCME_CK(up(P.type_u, htype.data(), ne));
    GCME_CK(up(P.type_s, htype.data(), ne));  // overwritten by the first cell sort
    if (fp64) GCME_CK(up(d_tab64, htab64.data(), sizeof(PairTab64) * htab64.size()));
    else GCME_CK(up(d_tab, htab.data(), sizeof(PairTab) * htab.size()));
  }
  if (own_state) {
    GCME_CK(cudaMemset(P.pos, 0, sizeof(double) * 3 * nr));
    GCME_CK(cudaMemset(P.vel, 0, (fp64 ? 8 : 4) * 3 * nr));
  }
  GCME_CK(cudaMemset(P.force, 0, sizeof(long long) * 3 * nr));
  if (ngrid > 0) GCME_CK(cudaMemset(P.qgrid, 0, sizeof(unsigned long long) * ngrid));
  GCME_CK(cudaMemset(P.wrap_n, 0, sizeof(int) * 3 * ne));
  GCME_CK(cudaMemset(P.step_ctr, 0, sizeof(unsigned long long) * ns));
  GCME_CK(cudaMemset(P.held, 0, ns));
  P.step_stop = nullptr;  // no step limits unless enable_step_limits()
  GCME_CK(cudaMemset(pair_counter, 0, sizeof(int)));  // each pair launch leaves it zero
  if (use_list) {
    // reference positions ~1e306: the first check requests a build
    GCME_CK(cudaMemset(P.x_ref, 0x7f, sizeof(double) * 3 * nr));
    GCME_CK(cudaMemset(P.list_flags, 0, sizeof(int) * 4));
    GCME_CK(cudaMemset(P.list_ovf, 0, sizeof(int) * 2 * ns));
    GCME_CK(cudaMemset(P.nbr_cnt, 0, sizeof(int) * ne));
    GCME_CK(cudaMemset(P.nbr_nq, 0, sizeof(int) * ne));
  }
  GCME_CK(cudaMemset(P.energy, 0, sizeof(double) * ns * GCME_NTERMS));
  GCME_CK(cudaMemset(P.virial, 0, sizeof(double) * ns * 9));
  GCME_CK(cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
  {
    // the PME branch is the longer one: highest priority so its short,
    // dependent kernels take free SM slots ahead of the pair kernel's CTAs
    int least = 0, greatest = 0;
    GCME_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GCME_CK(cudaStreamCreateWithPriority(&side_stream, cudaStreamNonBlocking, greatest));
  }
  GCME_CK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
  GCME_CK(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));

  static std::once_flag once[64];
  std::call_once(once[dev & 63], [] { pme_set_smem_limits(); });
  return GCME_OK;
}

// The PME branch (spread, FFTs, gather) needs only the wrapped positions of
// K1, and nothing of it is read by the pair or bonded kernels until the
// Yeh-Berkowitz and kick kernels: it runs on a side stream forked right
// after binning and joined before them, so its latency-bound passes overlap
// the cell sort and fill the SMs the pair kernel leaves idle.  (Forking
// before binning, with the spread wrapping positions itself, measured
// slower: the FP64 wraps cost the spread more than the overlap gained.)
void Engine::fork_pme(const Pool &Q, cudaStream_t st, bool vir, bool timed, bool zero_grid) {
  cudaEventRecord(fork_ev, st);
  cudaStreamWaitEvent(side_stream, fork_ev, 0);
  if (timed) cudaEventRecordWithFlags(phase_ev[5], side_stream, cudaEventRecordExternal);
  launch_pme(Q, plan, fp64, vir, side_stream, zero_grid);
  if (timed) cudaEventRecordWithFlags(phase_ev[6], side_stream, cudaEventRecordExternal);
  cudaEventRecord(join_ev, side_stream);
}

Pool Engine::cell_only(const Pool &Q) const {
  Pool C = Q;
  C.gate = nullptr;
  C.list_ovf = nullptr;
  C.img_now = nullptr;
  return C;
}

void Engine::request_rebuild(cudaStream_t st) {
  if (use_list) cudaMemsetAsync(P.list_flags + 1, 1, sizeof(int), st);
}

long long Engine::list_builds() {
  if (!use_list) return 0;
  int v[4] = {0, 0, 0, 0};
  if (cudaMemcpy(v, P.list_flags, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return v[2];
}

// Cell sort and pair kernels.  With lists: the sort and the list build run
// only on rebuild steps (device flag), the refresh every step, then the
// list kernel, and the 27-cell kernel for the systems whose lists overflowed.
void Engine::enqueue_sort_pairs(const Pool &Q, cudaStream_t st, bool vir, bool dbg, bool timed,
                                int fork) {
  launch_sort(Q, st);
  if (use_list) {
    launch_list_build(Q, st);
    launch_list_refresh(Q, st);
  }
  // the cell spread reads the sorted cell lists: the PME branch forks here
  if (fork) fork_pme(Q, st, vir, timed, fork > 1);
  if (timed) cudaEventRecordWithFlags(phase_ev[2], st, cudaEventRecordExternal);
  if (use_list) launch_pair_list(Q, vir, dbg, st);
  launch_pair(Q, pair_work, n_pair_work, fp64, cell_factor, pair_threads, pair_ctas(),
              pair_counter, vir, dbg, bonds_in_pair(dbg), st, pair_nelec == 0, pair_groups_on,
              pair_nelec < 0);
  if (timed) cudaEventRecordWithFlags(phase_ev[3], st, cudaEventRecordExternal);
}

void Engine::enqueue_forces(const Pool &Q, cudaStream_t st, bool vir, bool dbg) {
  cudaMemsetAsync(Q.force, 0, sizeof(long long) * 3 * Q.n_real, st);
  cudaMemsetAsync(Q.acc, 0, sizeof(unsigned long long) * Q.nsys * kNacc, st);
  if (vir) cudaMemsetAsync(Q.vacc, 0, sizeof(unsigned long long) * Q.nsys * 9, st);
  if (use_list) launch_list_check(Q, st);
  launch_bin(Q, st);
  if (dbg) {
    enqueue_sort_pairs(Q, st, vir, true, false);
    return;
  }
  if (!plan.cell_spread) fork_pme(Q, st, vir, false);
  enqueue_sort_pairs(Q, st, vir, false, false, plan.cell_spread ? 2 : 0);
  launch_bonded(Q, vir, !bonds_in_pair(false), st);
  cudaStreamWaitEvent(st, join_ev, 0);
  launch_slab_apply(Q, st);
}

void Engine::enqueue_step(const Pool &Q, cudaStream_t st) {
  const bool ev = phase_timing && phase_ev[0] != nullptr;
  if (ev) cudaEventRecordWithFlags(phase_ev[0], st, cudaEventRecordExternal);
  // no clears on the critical path: the half kick and drift clears the
  // forces it reads, the energy accumulators and the cell counts, and the
  // forward FFT pass of every evaluation leaves the charge grid zero
  launch_kick_drift(Q, fp64, st);
  if (ev) cudaEventRecordWithFlags(phase_ev[1], st, cudaEventRecordExternal);
  if (use_list) launch_list_check(Q, st);
  launch_bin(Q, st, false);
  if (ev) cudaEventRecordWithFlags(phase_ev[9], st, cudaEventRecordExternal);
  if (!plan.cell_spread) fork_pme(Q, st, false, ev, false);
  enqueue_sort_pairs(Q, st, false, false, ev, plan.cell_spread ? 1 : 0);
  launch_bonded(Q, false, !bonds_in_pair(false), st);
  if (ev) cudaEventRecordWithFlags(phase_ev[4], st, cudaEventRecordExternal);
  cudaStreamWaitEvent(st, join_ev, 0);
  if (ev) cudaEventRecordWithFlags(phase_ev[7], st, cudaEventRecordExternal);
  launch_slab_apply(Q, st);
  if (ev) cudaEventRecordWithFlags(phase_ev[10], st, cudaEventRecordExternal);
  launch_kick(Q, fp64, st);
  if (ev) cudaEventRecordWithFlags(phase_ev[11], st, cudaEventRecordExternal);
  launch_finalize(Q, false, st);
  if (ev) cudaEventRecordWithFlags(phase_ev[8], st, cudaEventRecordExternal);
}

int Engine::step_graph(const Pool &Q, cudaGraphExec_t *out) {
  auto key = std::make_tuple((void *)Q.pos, (void *)Q.vel, (void *)Q.force, phase_timing ? 3 : 1);
  last_step_timed = phase_timing;
  auto it = graphs_.find(key);
  if (it != graphs_.end()) {
    *out = it->second;
    return GCME_OK;
  }
  cudaGraph_t g;
  if (phase_timing && !phase_ev[0])
    for (int k = 0; k < kNPhaseEv; ++k) GCME_CK(cudaEventCreate(&phase_ev[k]));
  GCME_CK(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(Q, capture_stream);
  GCME_CK(cudaStreamEndCapture(capture_stream, &g));
  {
    size_t nn = 0;
    GCME_CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    GCME_CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    int nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      GCME_CK(cudaGraphNodeGetType(nd, &t));
      nk += t == cudaGraphNodeTypeKernel;
    }
    step_kernels = nk;
  }
  cudaGraphExec_t ge;
  GCME_CK(cudaGraphInstantiate(&ge, g, 0));
  graph_objs_.push_back(g);
  graphs_[key] = ge;
  *out = ge;
  return GCME_OK;
}

void Engine::enable_step_limits() {
  P.step_stop = step_stop_buf;
  clear_graphs();  // the kernels take the pool by value
}

int Engine::host_graph(const Pool &Q, const double *h_pos, const float *h_vel,
                       double *h_energy, bool cont, int part, cudaGraphExec_t *out) {
  auto key = std::make_tuple((void *)h_pos, (void *)h_vel, (void *)h_energy,
                             16 + 4 * part + 2 * (int)cont + (int)phase_timing);
  if (part == 3) last_step_timed = phase_timing;
  auto it = graphs_.find(key);
  if (it != graphs_.end()) {
    *out = it->second;
    return GCME_OK;
  }
  if (phase_timing && !phase_ev[0])
    for (int k = 0; k < kNPhaseEv; ++k) GCME_CK(cudaEventCreate(&phase_ev[k]));
  const size_t n3 = 3 * (size_t)n_real;
  cudaStream_t cs = capture_stream;
  cudaGraph_t g;
  GCME_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  // the SMs move the state over the CPU-GPU link (one kernel each way, no
  // copy-engine nodes between the step's kernels)
  if (part & 1) {
    launch_state_copy(h_pos, h_vel, Q.pos, reinterpret_cast<float *>(Q.vel), (long long)n3,
                      nullptr, nullptr, cs);
    if (!cont) {
      enqueue_forces(Q, cs, false, false);
      launch_finalize(Q, false, cs);
    }
  }
  if (part == 3) enqueue_step(Q, cs);
  if (part & 2)
    launch_state_copy(Q.pos, reinterpret_cast<const float *>(Q.vel), const_cast<double *>(h_pos),
                      const_cast<float *>(h_vel), (long long)n3, h_energy ? Q.energy : nullptr,
                      h_energy, cs);
  GCME_CK(cudaStreamEndCapture(cs, &g));
  cudaGraphExec_t ge;
  GCME_CK(cudaGraphInstantiate(&ge, g, 0));
  graph_objs_.push_back(g);
  graphs_[key] = ge;
  *out = ge;
  return GCME_OK;
}

int Engine::forces_graph(const Pool &Q, cudaGraphExec_t *out) {
  auto key = std::make_tuple((void *)Q.pos, (void *)Q.vel, (void *)Q.force, 2);
  auto it = graphs_.find(key);
  if (it != graphs_.end()) {
    *out = it->second;
    return GCME_OK;
  }
  cudaGraph_t g;
  GCME_CK(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_forces(Q, capture_stream, false, false);
  launch_finalize(Q, false, capture_stream);
  GCME_CK(cudaStreamEndCapture(capture_stream, &g));
  cudaGraphExec_t ge;
  GCME_CK(cudaGraphInstantiate(&ge, g, 0));
  graph_objs_.push_back(g);
  graphs_[key] = ge;
  *out = ge;
  return GCME_OK;
}

}  // namespace gcme

// ===========================================================================
// C ABI
// ===========================================================================
using namespace gcme;

struct gcme_sys {
  gcme_ctx *ctx;
  Engine eng;
  gcme_params p;
  SysSpec spec;               // as created (the box follows set_box)
  double *saved_pos = nullptr;  // barostat: positions before a volume move
  // device copies of a host-held state (gcme_step_host), allocated by its
  // first call
  double *hd_pos = nullptr;
  float *hd_vel = nullptr;
  ~gcme_sys() {
    if (saved_pos) cudaFree(saved_pos);
    if (hd_pos) cudaFree(hd_pos);
    if (hd_vel) cudaFree(hd_vel);
  }
  // buffers of the last gcme_step call: the internal force array then holds
  // F at their current positions, so a continuation can skip that evaluation
  const void *last_pos = nullptr, *last_vel = nullptr;
  // host buffers of the last gcme_step_host call (the same for its continuation)
  const void *last_hpos = nullptr, *last_hvel = nullptr;
};

struct gcme_batch {
  gcme_ctx *ctx;
  Engine eng;
  bool forces_valid = false;
};

#define GCME_TRY_CK(call)                                                          \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      set_error(std::string(#call) + ": " + cudaGetErrorString(_e));               \
      return GCME_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

static int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  return GCME_OK;
}

extern "C" {

const char *gcme_last_error(void) { return g_err.c_str(); }

const char *gcme_version(void) { return "gcme 0.1 (sm_103a)"; }

void gcme_params_default(gcme_params *p, double L, int32_t K) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->box[0] = p->box[1] = p->box[2] = L;
  p->geometry = GCME_BULK;
  p->precision = GCME_FP32;
  p->A = 25.0;
  p->sigma = 0.5;
  p->a = 0.5;
  p->lB = 1.2053;
  p->rc = 3.0;
  p->kappa = 0.87609;
  p->K[0] = p->K[1] = p->K[2] = K;
  p->order = 5;
  p->dt = 0.01;
  p->bond_k = 100.0;
  p->bond_r0 = 1.0;
  p->gamma = 0.0;
  p->kT = 1.0;
  p->seed = 0;
}

int gcme_validate(const gcme_params *p, int64_t n, const double *h_q, const int32_t *h_types,
                  const int32_t *h_bonds, int64_t nbonds) {
  if (!p || !h_q || n < 1 || nbonds < 0 || (nbonds > 0 && !h_bonds)) {
    set_error("invalid argument to gcme_validate");
    return GCME_ERR_INVALID;
  }
  SysSpec sp;
  sp.p = *p;
  sp.n = n;
  sp.q.assign(h_q, h_q + n);
  if (h_types) sp.types.assign(h_types, h_types + n);
  if (nbonds) sp.bonds.assign(h_bonds, h_bonds + 2 * nbonds);
  std::string err = validate_spec(sp);
  if (!err.empty()) {
    set_error(err);
    return GCME_ERR_INVALID;
  }
  set_error("");
  return GCME_OK;
}

int gcme_ctx_create(gcme_ctx **out, int device) {
  if (!out) {
    set_error("out is NULL");
    return GCME_ERR_INVALID;
  }
  int ndev = 0;
  GCME_TRY_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("device index out of range");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(device));
  *out = new gcme_ctx{device};
  return GCME_OK;
}

void gcme_ctx_destroy(gcme_ctx *ctx) { delete ctx; }

int gcme_system_create(gcme_ctx *ctx, const gcme_params *p, int64_t n, const double *h_q,
                       const int32_t *h_types, const int32_t *h_bonds, int64_t nbonds,
                       gcme_sys **out) {
  if (!ctx || !p || !h_q || !out || n < 1 || nbonds < 0 || (nbonds > 0 && !h_bonds)) {
    set_error("invalid argument to gcme_system_create");
    return GCME_ERR_INVALID;
  }
  SysSpec sp;
  sp.p = *p;
  sp.n = n;
  sp.q.assign(h_q, h_q + n);
  if (h_types) sp.types.assign(h_types, h_types + n);
  if (nbonds) sp.bonds.assign(h_bonds, h_bonds + 2 * nbonds);
  gcme_sys *s = new gcme_sys;
  s->ctx = ctx;
  s->p = *p;
  s->spec = sp;
  int rc = s->eng.build(ctx->device, {sp}, false);
  if (rc != GCME_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return GCME_OK;
}

void gcme_system_destroy(gcme_sys *sys) {
  if (!sys) return;
  cudaSetDevice(sys->eng.device);
  delete sys;
}

int gcme_system_info(const gcme_sys *sys, gcme_sys_info *out) {
  if (!sys || !out) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  const SysDesc &S = sys->eng.hsys[0];
  out->n = S.n;
  out->n_ext = S.n_ext;
  out->n_charged_ext = S.nq_ext;
  out->ncell = S.ncell;
  out->nbonds = S.nbond;
  for (int a = 0; a < 3; ++a) out->nc[a] = S.nc[a];
  out->cell_factor = S.cell_factor;
  out->scratch_bytes = (int64_t)sys->eng.scratch_bytes;
  gcme_sys *ms = const_cast<gcme_sys *>(sys);
  out->pair_path = ms->eng.use_list ? GCME_PAIR_LIST : GCME_PAIR_CELLS;
  out->list_stride = ms->eng.use_list ? ms->eng.P.nbr_stride : 0;
  GCME_TRY_CK(cudaSetDevice(ms->eng.device));
  out->list_builds = ms->eng.list_builds();
  unsigned long long steps = 0;
  GCME_TRY_CK(cudaMemcpy(&steps, ms->eng.P.step_ctr, sizeof(steps), cudaMemcpyDeviceToHost));
  out->steps = (int64_t)steps;
  for (int a = 0; a < 3; ++a) out->box[a] = S.box[a];
  return GCME_OK;
}

// ---- pressure and NpT -------------------------------------------------------
// Potential energy (and optionally the virial) of the system at d_pos,
// using the internal force buffer.  Synchronises the stream.
static int eval_energy(gcme_sys *sys, const double *d_pos, cudaStream_t st, double *U,
                       double *W) {
  Pool Q = sys->eng.P;
  Q.pos = const_cast<double *>(d_pos);
  const bool vir = W != nullptr;
  sys->eng.enqueue_forces(Q, st, vir, false);
  launch_finalize(Q, vir, st);
  double e[GCME_NTERMS];
  GCME_TRY_CK(cudaMemcpyAsync(e, Q.energy, sizeof(e), cudaMemcpyDeviceToHost, st));
  if (vir) GCME_TRY_CK(cudaMemcpyAsync(W, Q.virial, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
  GCME_TRY_CK(cudaStreamSynchronize(st));
  *U = e[GCME_E_POTENTIAL];
  sys->last_pos = nullptr;  // the internal forces no longer belong to a step's state
  return check_launch("energy evaluation");
}

// Philox4x64-10 on the host (the barostat's two uniforms per move)
static void host_philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    const unsigned __int128 p0 = (unsigned __int128)m0 * c[0];
    const unsigned __int128 p1 = (unsigned __int128)m1 * c[2];
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

int gcme_system_set_box(gcme_sys *sys, const double *box, gcme_stream_t stream) {
  if (!sys || !box) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  if (sys->p.geometry != GCME_BULK) {
    set_error("gcme_system_set_box: bulk systems only (a slab's box is tied to its height)");
    return GCME_ERR_INVALID;
  }
  Engine &E = sys->eng;
  const SysDesc &S0 = E.hsys[0];
  const double rc = S0.rc;
  int nc[3];
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] >= rc * (1.0 + 1e-4)) || !std::isfinite(box[a])) {
      set_error("gcme_system_set_box: box side shorter than the cutoff");
      return GCME_ERR_INVALID;
    }
    nc[a] = cells_per_axis(box[a], rc, E.cell_factor);
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(E.device));
  for (int a = 0; a < 3; ++a) {
    sys->p.box[a] = box[a];
    sys->spec.p.box[a] = box[a];
  }
  sys->last_pos = nullptr;
  if (nc[0] == S0.nc[0] && nc[1] == S0.nc[1] && nc[2] == S0.nc[2]) {
    // same cell grid: only the box-derived constants change (the kernels
    // and captured graphs read them from the device table)
    GCME_TRY_CK(cudaStreamSynchronize(st));
    SysDesc &S = E.hsys[0];
    for (int a = 0; a < 3; ++a) {
      set_cell_box_axis(S, a, box[a]);
      S.kfac[a] = (float)((double)S.K[a] / box[a]);
    }
    S.V = box[0] * box[1] * box[2];
    box_floats(S);
    GCME_TRY_CK(cudaMemcpy(const_cast<SysDesc *>(E.P.sys), &S, sizeof(SysDesc),
                           cudaMemcpyHostToDevice));
    E.request_rebuild(st);
    return check_launch("gcme_system_set_box");
  }
  // another cell grid: rebuild the engine for the new box (launch shapes
  // carried over); the state lives in the caller's buffers
  GCME_TRY_CK(cudaStreamSynchronize(st));
  const int split = E.pair_split, threads = E.pair_threads, ctas = E.pair_ctas_per_sm,
            nelec = E.pair_nelec, chunks = E.pair_chunks, group = E.pair_group;
  E.release();
  E.pair_split = split;
  int rc2 = E.build(E.device, {sys->spec}, false);
  if (rc2) return rc2;
  return E.set_pair_config(split, threads, ctas, nelec, chunks, group);
}

int gcme_pressure(gcme_sys *sys, const double *d_pos, double kT, double *h_pressure,
                  gcme_stream_t stream) {
  if (!sys || !d_pos || !h_pressure || !(kT >= 0)) {
    set_error("invalid argument to gcme_pressure");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  double U, W[9];
  int rc = eval_energy(sys, d_pos, (cudaStream_t)stream, &U, W);
  if (rc) return rc;
  const SysDesc &S = sys->eng.hsys[0];
  *h_pressure = ((double)S.n * kT + (W[0] + W[4] + W[8]) / 3.0) / S.V;
  return GCME_OK;
}

int gcme_barostat_move(gcme_sys *sys, double *d_pos, double pressure, double kT, double dlnv,
                       uint64_t seed, uint64_t move, int32_t *h_accepted, gcme_stream_t stream) {
  if (!sys || !d_pos || !h_accepted || !(kT > 0) || !(dlnv > 0) || !std::isfinite(pressure)) {
    set_error("invalid argument to gcme_barostat_move");
    return GCME_ERR_INVALID;
  }
  if (sys->p.geometry != GCME_BULK) {
    set_error("gcme_barostat_move: bulk systems only");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  const long long n = sys->eng.hsys[0].n;
  if (!sys->saved_pos) GCME_TRY_CK(cudaMalloc(&sys->saved_pos, sizeof(double) * 3 * n));
  double U0, U1;
  int rc = eval_energy(sys, d_pos, st, &U0, nullptr);
  if (rc) return rc;
  uint64_t c[4] = {move, 0, 0, 0};
  host_philox4x64(c, seed, 1);
  const double u0 = (double)(c[0] >> 11) * 0x1.0p-53, u1 = (double)(c[1] >> 11) * 0x1.0p-53;
  const double box0[3] = {sys->p.box[0], sys->p.box[1], sys->p.box[2]};
  const double V = box0[0] * box0[1] * box0[2];
  const double lr = (2.0 * u0 - 1.0) * dlnv;  // ln(V'/V)
  const double V1 = V * std::exp(lr), sc = std::exp(lr / 3.0);
  const double box1[3] = {box0[0] * sc, box0[1] * sc, box0[2] * sc};
  GCME_TRY_CK(cudaMemcpyAsync(sys->saved_pos, d_pos, sizeof(double) * 3 * n,
                              cudaMemcpyDeviceToDevice, st));
  launch_scale(d_pos, 3 * n, sc, st);
  rc = gcme_system_set_box(sys, box1, stream);
  if (rc == GCME_OK) rc = eval_energy(sys, d_pos, st, &U1, nullptr);
  bool accept = false;
  if (rc == GCME_OK) {
    const double dW = U1 - U0 + pressure * (V1 - V) - (double)(n + 1) * kT * lr;
    accept = dW <= 0.0 || u1 < std::exp(-dW / kT);
  } else if (rc != GCME_ERR_INVALID) {
    return rc;  // a device error: leave the state to the caller
  }
  if (!accept) {  // restore positions and box (a box below the cutoff is a rejection)
    GCME_TRY_CK(cudaMemcpyAsync(d_pos, sys->saved_pos, sizeof(double) * 3 * n,
                                cudaMemcpyDeviceToDevice, st));
    rc = gcme_system_set_box(sys, box0, stream);
    if (rc) return rc;
  }
  *h_accepted = accept ? 1 : 0;
  set_error("");
  return GCME_OK;
}

int gcme_system_set_step_count(gcme_sys *sys, int64_t steps, gcme_stream_t stream) {
  if (!sys || steps < 0) {
    set_error("invalid argument to gcme_system_set_step_count");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  // a kernel-free update: a pageable-source copy would be staged, so the
  // value is written by a memset of each byte
  const unsigned long long v = (unsigned long long)steps;
  for (int b = 0; b < 8; ++b)
    GCME_TRY_CK(cudaMemsetAsync(reinterpret_cast<unsigned char *>(sys->eng.P.step_ctr) + b,
                                (int)((v >> (8 * b)) & 0xff), 1, (cudaStream_t)stream));
  return check_launch("gcme_system_set_step_count");
}

int gcme_build_cells(gcme_sys *sys, const double *d_pos, int32_t *d_cell_start,
                     int32_t *d_sorted_idx, gcme_stream_t stream) {
  if (!sys || !d_pos) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.cell_only(sys->eng.P);
  Q.pos = const_cast<double *>(d_pos);
  launch_cells(Q, st);
  sys->eng.request_rebuild(st);  // the lists index the previous cell order
  const SysDesc &S = sys->eng.hsys[0];
  if (d_cell_start)
    GCME_TRY_CK(cudaMemcpyAsync(d_cell_start, Q.cell_start, sizeof(int) * (S.ncell + 1),
                                cudaMemcpyDeviceToDevice, st));
  if (d_sorted_idx)
    GCME_TRY_CK(cudaMemcpyAsync(d_sorted_idx, Q.sorted_idx, sizeof(int) * S.n_ext,
                                cudaMemcpyDeviceToDevice, st));
  return check_launch("gcme_build_cells");
}

int gcme_forces(gcme_sys *sys, const double *d_pos, int64_t *d_force, double *d_energy,
                double *d_virial, gcme_stream_t stream) {
  if (!sys || !d_pos) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.P;
  Q.pos = const_cast<double *>(d_pos);
  if (d_force) Q.force = reinterpret_cast<long long *>(d_force);
  const bool vir = d_virial != nullptr;
  sys->eng.enqueue_forces(Q, st, vir, false);
  launch_finalize(Q, vir, st);
  if (d_energy)
    GCME_TRY_CK(cudaMemcpyAsync(d_energy, Q.energy, sizeof(double) * GCME_NTERMS,
                                cudaMemcpyDeviceToDevice, st));
  if (d_virial)
    GCME_TRY_CK(cudaMemcpyAsync(d_virial, Q.virial, sizeof(double) * 9, cudaMemcpyDeviceToDevice,
                                st));
  return check_launch("gcme_forces");
}

int gcme_forces_to_f64(gcme_sys *sys, const int64_t *d_force, double *d_out,
                       gcme_stream_t stream) {
  if (!sys || !d_force || !d_out) {
    set_error("NULL argument");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  launch_force_to_f64(reinterpret_cast<const long long *>(d_force), d_out,
                      3LL * sys->eng.hsys[0].n, (cudaStream_t)stream);
  return check_launch("gcme_forces_to_f64");
}

static int run_steps(Engine &eng, const Pool &Q, int64_t nsteps, cudaStream_t st) {
  cudaGraphExec_t fg, sg;
  int rc = eng.forces_graph(Q, &fg);
  if (rc) return rc;
  rc = eng.step_graph(Q, &sg);
  if (rc) return rc;
  GCME_TRY_CK(cudaGraphLaunch(fg, st));
  for (int64_t k = 0; k < nsteps; ++k) GCME_TRY_CK(cudaGraphLaunch(sg, st));
  return GCME_OK;
}

static int continue_steps(gcme_sys *sys, double *d_pos, void *d_vel, int64_t nsteps,
                          double *d_energy, cudaStream_t st) {
  if (d_pos != sys->last_pos || d_vel != sys->last_vel) {
    set_error("gcme_step_continue: no preceding gcme_step on these buffers");
    return GCME_ERR_INVALID;
  }
  Pool Q = sys->eng.P;
  Q.pos = d_pos;
  Q.vel = d_vel;
  cudaGraphExec_t sg;
  int rc = sys->eng.step_graph(Q, &sg);
  if (rc) return rc;
  for (int64_t k = 0; k < nsteps; ++k) GCME_TRY_CK(cudaGraphLaunch(sg, st));
  if (d_energy)
    GCME_TRY_CK(cudaMemcpyAsync(d_energy, Q.energy, sizeof(double) * GCME_NTERMS,
                                cudaMemcpyDeviceToDevice, st));
  return check_launch("gcme_step_continue");
}

static bool is_pinned(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

int gcme_step_host(gcme_sys *sys, double *h_pos, float *h_vel, int64_t nsteps, double *h_energy,
                   int32_t flags, gcme_stream_t stream) {
  if (!sys || !h_pos || !h_vel || nsteps < 0 || (flags & ~GCME_STEP_CONTINUE)) {
    set_error("invalid argument to gcme_step_host");
    return GCME_ERR_INVALID;
  }
  if (sys->eng.fp64) {
    set_error("gcme_step_host steps FP32 systems");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  if (!is_pinned(h_pos) || !is_pinned(h_vel) || (h_energy && !is_pinned(h_energy))) {
    set_error("gcme_step_host: host buffers must be page-locked (cudaHostAlloc or "
              "cudaHostRegister)");
    return GCME_ERR_INVALID;
  }
  const bool cont = (flags & GCME_STEP_CONTINUE) != 0;
  if (cont && (h_pos != sys->last_hpos || h_vel != sys->last_hvel)) {
    set_error("gcme_step_host: no preceding call on these host buffers to continue");
    return GCME_ERR_INVALID;
  }
  const size_t n3 = 3 * (size_t)sys->eng.hsys[0].n;
  if (!sys->hd_pos) {
    if (cudaMalloc(&sys->hd_pos, sizeof(double) * n3) != cudaSuccess ||
        cudaMalloc(&sys->hd_vel, sizeof(float) * n3) != cudaSuccess) {
      cudaGetLastError();
      set_error("gcme_step_host: device state allocation failed");
      return GCME_ERR_OOM;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  Pool Q = sys->eng.P;
  Q.pos = sys->hd_pos;
  Q.vel = sys->hd_vel;
  Engine &E = sys->eng;
  cudaGraphExec_t g;
  int rc;
  if (nsteps == 1) {
    if ((rc = E.host_graph(Q, h_pos, h_vel, h_energy, cont, 3, &g))) return rc;
    GCME_TRY_CK(cudaGraphLaunch(g, st));
  } else {
    cudaGraphExec_t sg;
    if ((rc = E.host_graph(Q, h_pos, h_vel, h_energy, cont, 1, &g))) return rc;
    if ((rc = E.step_graph(Q, &sg))) return rc;
    GCME_TRY_CK(cudaGraphLaunch(g, st));
    for (int64_t k = 0; k < nsteps; ++k) GCME_TRY_CK(cudaGraphLaunch(sg, st));
    if ((rc = E.host_graph(Q, h_pos, h_vel, h_energy, cont, 2, &g))) return rc;
    GCME_TRY_CK(cudaGraphLaunch(g, st));
  }
  sys->last_hpos = h_pos;
  sys->last_hvel = h_vel;
  return check_launch("gcme_step_host");
}

int gcme_step_continue(gcme_sys *sys, double *d_pos, void *d_vel, int64_t nsteps,
                       double *d_energy, gcme_stream_t stream) {
  if (!sys || !d_pos || !d_vel || nsteps < 0) {
    set_error("invalid argument to gcme_step_continue");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  return continue_steps(sys, d_pos, d_vel, nsteps, d_energy, (cudaStream_t)stream);
}

int gcme_step(gcme_sys *sys, double *d_pos, float *d_vel, int64_t nsteps, double *d_energy,
              gcme_stream_t stream) {
  if (!sys || !d_pos || !d_vel || nsteps < 0) {
    set_error("invalid argument to gcme_step");
    return GCME_ERR_INVALID;
  }
  if (sys->eng.fp64) {
    set_error("FP64 systems step with gcme_step_f64");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.P;
  Q.pos = d_pos;
  Q.vel = d_vel;
  int rc = run_steps(sys->eng, Q, nsteps, st);
  if (rc) return rc;
  sys->last_pos = d_pos;
  sys->last_vel = d_vel;
  if (d_energy)
    GCME_TRY_CK(cudaMemcpyAsync(d_energy, Q.energy, sizeof(double) * GCME_NTERMS,
                                cudaMemcpyDeviceToDevice, st));
  return check_launch("gcme_step");
}

int gcme_step_f64(gcme_sys *sys, double *d_pos, double *d_vel, int64_t nsteps, double *d_energy,
                  gcme_stream_t stream) {
  if (!sys || !d_pos || !d_vel || nsteps < 0) {
    set_error("invalid argument to gcme_step_f64");
    return GCME_ERR_INVALID;
  }
  if (!sys->eng.fp64) {
    set_error("FP32 systems step with gcme_step");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.P;
  Q.pos = d_pos;
  Q.vel = d_vel;
  int rc = run_steps(sys->eng, Q, nsteps, st);
  if (rc) return rc;
  sys->last_pos = d_pos;
  sys->last_vel = d_vel;
  if (d_energy)
    GCME_TRY_CK(cudaMemcpyAsync(d_energy, Q.energy, sizeof(double) * GCME_NTERMS,
                                cudaMemcpyDeviceToDevice, st));
  return check_launch("gcme_step_f64");
}

static int phase_ms(Engine &eng, float *h_ms, int32_t nphase, int32_t *kernels) {
  if (kernels) *kernels = eng.step_kernels;
  if (!h_ms) return GCME_OK;
  if (nphase < 6 || !eng.phase_ev[0] || !eng.last_step_timed) {
    set_error("no step with phase timing on yet, or output shorter than the phase count");
    return GCME_ERR_INVALID;
  }
  // [0] kick+drift, [1] cells, [2] pair kernel, [3] PME branch (side
  // stream), [4] bonds/walls, [5] slab + kick + energies after the join;
  // with nphase >= 8 also [6] binning alone (inside [1]) and [7] the second
  // half kick alone (inside [5])
  const int pairs[8][2] = {{0, 1}, {1, 2}, {2, 3}, {5, 6}, {3, 4}, {7, 8}, {1, 9}, {10, 11}};
  const int np = nphase >= 8 ? 8 : 6;
  for (int k = 0; k < np; ++k)
    GCME_TRY_CK(cudaEventElapsedTime(&h_ms[k], eng.phase_ev[pairs[k][0]], eng.phase_ev[pairs[k][1]]));
  return GCME_OK;
}

int gcme_step_phase_ms(gcme_sys *sys, float *h_ms, int32_t nphase, int32_t *kernels) {
  if (!sys) {
    set_error("NULL system");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  return phase_ms(sys->eng, h_ms, nphase, kernels);
}

int gcme_step_phase_timing(gcme_sys *sys, int32_t on) {
  if (!sys) {
    set_error("NULL system");
    return GCME_ERR_INVALID;
  }
  sys->eng.phase_timing = on != 0;
  return GCME_OK;
}

int gcme_batch_phase_timing(gcme_batch *b, int32_t on) {
  if (!b) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  b->eng.phase_timing = on != 0;
  return GCME_OK;
}

int gcme_batch_phase_ms(gcme_batch *b, float *h_ms, int32_t nphase, int32_t *kernels) {
  if (!b) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(b->eng.device));
  return phase_ms(b->eng, h_ms, nphase, kernels);
}

// Four barrier words for the timeout probe (no allocation needed).
static __device__ unsigned int g_probe_words[4];

int gcme_debug_barrier_timeout(gcme_ctx *ctx, double timeout_s, gcme_stream_t stream) {
  if (!ctx || !(timeout_s > 0) || timeout_s > 10.0) {
    set_error("invalid argument to gcme_debug_barrier_timeout");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(ctx->device));
  unsigned int *w = nullptr;
  GCME_TRY_CK(cudaGetSymbolAddress((void **)&w, g_probe_words));
  cudaStream_t st = (cudaStream_t)stream;
  if (launch_barrier_probe(w, timeout_s, st) != 0) {
    set_error(std::string("probe launch failed: ") + cudaGetErrorString(cudaGetLastError()));
    return GCME_ERR_CUDA;
  }
  unsigned int words[4];
  GCME_TRY_CK(cudaMemcpyAsync(words, w, sizeof(words), cudaMemcpyDeviceToHost, st));
  GCME_TRY_CK(cudaStreamSynchronize(st));
  if (words[2] != 0) {
    set_error("grid barrier wait ran out");
    return GCME_ERR_TIMEOUT;
  }
  return GCME_OK;
}

int gcme_debug_pairs(gcme_sys *sys, const double *d_pos, int32_t *d_triples, int64_t cap,
                     int64_t *d_count, gcme_stream_t stream) {
  if (!sys || !d_pos || !d_count || cap < 0 || (cap > 0 && !d_triples)) {
    set_error("invalid argument to gcme_debug_pairs");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.P;
  Q.pos = const_cast<double *>(d_pos);
  Q.dbg_triples = d_triples;
  Q.dbg_cap = cap;
  sys->eng.enqueue_forces(Q, st, false, true);
  GCME_TRY_CK(cudaMemcpyAsync(d_count, Q.acc + ACC_NPAIR, sizeof(int64_t),
                              cudaMemcpyDeviceToDevice, st));
  return check_launch("gcme_debug_pairs");
}

int gcme_debug_pme_grids(gcme_sys *sys, const double *d_pos, double *d_q, double *d_phi,
                         gcme_stream_t stream) {
  if (!sys || !d_pos || (!d_q && !d_phi)) {
    set_error("invalid argument to gcme_debug_pme_grids");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Engine &E = sys->eng;
  GCME_TRY_CK(cudaSetDevice(E.device));
  Pool Q = E.P;
  Q.pos = const_cast<double *>(d_pos);
  launch_bin(Q, st);
  if (E.plan.cell_spread) launch_sort(E.cell_only(Q), st);
  launch_pme_spread(Q, E.plan, E.fp64, st, true);
  launch_grids_to_f64(Q, E.fp64, d_q, nullptr, st);
  launch_pme_fft(Q, E.plan, E.fp64, false, st);
  launch_grids_to_f64(Q, E.fp64, nullptr, d_phi, st);
  sys->last_pos = sys->last_vel = nullptr;  // the accumulators were used
  return check_launch("gcme_debug_pme_grids");
}

// ---- autotuner -------------------------------------------------------------
static void fill_tuning(const Engine &eng, double pair_ms, double pme_ms, bool hit,
                        gcme_tuning *out) {
  if (!out) return;
  out->pair_split = eng.pair_split;
  out->pair_threads = eng.pair_threads;
  out->pair_ctas_per_sm = eng.pair_ctas_per_sm;
  out->pair_nelec = eng.pair_nelec;
  out->pair_chunks = eng.pair_chunks;
  out->pair_group = eng.pair_group;
  out->spread_cells = eng.plan.cell_spread;
  for (int a = 0; a < 3; ++a) out->fft_lpb[a] = eng.plan.lpb[a];
  out->fft_plane = eng.plan.use_plane;
  out->from_cache = hit ? 1 : 0;
  out->cell_factor = eng.cell_factor;
  out->forces_ms = pair_ms;
  out->pme_ms = pme_ms;
}

int gcme_autotune(gcme_sys *sys, const double *d_pos, int32_t flags, gcme_tuning *out,
                  gcme_stream_t stream) {
  if (!sys || !d_pos) {
    set_error("invalid argument to gcme_autotune");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  Pool Q = sys->eng.P;
  Q.pos = const_cast<double *>(d_pos);
  double a = 0, b = 0;
  bool hit = false;
  int rc = sys->eng.autotune(Q, (cudaStream_t)stream, flags, &a, &b, &hit);
  if (rc) return rc;
  sys->last_pos = sys->last_vel = nullptr;  // forces no longer match a trajectory
  fill_tuning(sys->eng, a, b, hit, out);
  return GCME_OK;
}

int gcme_apply_tuning(gcme_sys *sys, const gcme_tuning *t) {
  if (!sys || !t) {
    set_error("invalid argument to gcme_apply_tuning");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(sys->eng.device));
  return sys->eng.apply_tuning(t->pair_split, t->pair_threads, t->pair_ctas_per_sm,
                               t->pair_nelec, t->fft_lpb, t->fft_plane != 0, t->pair_chunks,
                               t->spread_cells != 0, t->pair_group > 1 ? t->pair_group : 1);
}

int gcme_batch_apply_tuning(gcme_batch *bt, const gcme_tuning *t) {
  if (!bt || !t) {
    set_error("invalid argument to gcme_batch_apply_tuning");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(bt->eng.device));
  return bt->eng.apply_tuning(t->pair_split, t->pair_threads, t->pair_ctas_per_sm,
                              t->pair_nelec, t->fft_lpb, t->fft_plane != 0, t->pair_chunks,
                              t->spread_cells != 0, t->pair_group > 1 ? t->pair_group : 1);
}

int gcme_batch_autotune(gcme_batch *bt, int32_t flags, gcme_tuning *out, gcme_stream_t stream) {
  if (!bt) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  GCME_TRY_CK(cudaSetDevice(bt->eng.device));
  double a = 0, b = 0;
  bool hit = false;
  int rc = bt->eng.autotune(bt->eng.P, (cudaStream_t)stream, flags, &a, &b, &hit);
  if (rc) return rc;
  bt->forces_valid = false;
  fill_tuning(bt->eng, a, b, hit, out);
  return GCME_OK;
}

// ---- batch ----------------------------------------------------------------
int gcme_batch_create(gcme_ctx *ctx, int32_t nsys, const gcme_params *params, const int64_t *n,
                      const double *h_q, const int32_t *h_types, const int32_t *h_bonds,
                      const int64_t *h_bond_count, gcme_batch **out) {
  if (!ctx || nsys < 1 || !params || !n || !h_q || !out) {
    set_error("invalid argument to gcme_batch_create");
    return GCME_ERR_INVALID;
  }
  std::vector<SysSpec> specs(nsys);
  int64_t qo = 0, bo = 0;
  for (int s = 0; s < nsys; ++s) {
    specs[s].p = params[s];
    specs[s].n = n[s];
    if (n[s] < 1) {
      set_error("system size must be >= 1");
      return GCME_ERR_INVALID;
    }
    specs[s].q.assign(h_q + qo, h_q + qo + n[s]);
    if (h_types) specs[s].types.assign(h_types + qo, h_types + qo + n[s]);
    qo += n[s];
    int64_t nb = h_bond_count ? h_bond_count[s] : 0;
    if (nb > 0) {
      if (!h_bonds) {
        set_error("bond counts given without bonds");
        return GCME_ERR_INVALID;
      }
      specs[s].bonds.assign(h_bonds + 2 * bo, h_bonds + 2 * (bo + nb));
    }
    bo += nb;
  }
  gcme_batch *b = new gcme_batch;
  b->ctx = ctx;
  int rc = b->eng.build(ctx->device, specs, true);
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return GCME_OK;
}

void gcme_batch_destroy(gcme_batch *b) {
  if (!b) return;
  cudaSetDevice(b->eng.device);
  delete b;
}

int gcme_batch_pointers(gcme_batch *b, double **d_pos, float **d_vel, double **d_energy,
                        const int64_t **h_bead_off) {
  if (!b) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  if (d_pos) *d_pos = b->eng.P.pos;
  if (d_vel) *d_vel = reinterpret_cast<float *>(b->eng.P.vel);
  if (d_energy) *d_energy = b->eng.P.energy;
  if (h_bead_off) *h_bead_off = reinterpret_cast<const int64_t *>(b->eng.bead_off.data());
  return GCME_OK;
}

int gcme_batch_set_state(gcme_batch *b, const double *h_pos, const float *h_vel,
                         gcme_stream_t stream) {
  if (!b) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(b->eng.device));
  const long long n = b->eng.n_real;
  if (h_pos)
    GCME_TRY_CK(cudaMemcpyAsync(b->eng.P.pos, h_pos, sizeof(double) * 3 * n,
                                cudaMemcpyHostToDevice, st));
  if (h_vel) {
    if (b->eng.fp64) {
      std::vector<double> v(h_vel, h_vel + 3 * n);
      GCME_TRY_CK(cudaMemcpyAsync(b->eng.P.vel, v.data(), sizeof(double) * 3 * n,
                                  cudaMemcpyHostToDevice, st));
      GCME_TRY_CK(cudaStreamSynchronize(st));
    } else {
      GCME_TRY_CK(cudaMemcpyAsync(b->eng.P.vel, h_vel, sizeof(float) * 3 * n,
                                  cudaMemcpyHostToDevice, st));
    }
  }
  b->forces_valid = false;
  return GCME_OK;
}

int gcme_batch_get_state(gcme_batch *b, double *h_pos, float *h_vel, double *h_energy,
                         gcme_stream_t stream) {
  if (!b) {
    set_error("NULL batch");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(b->eng.device));
  const long long n = b->eng.n_real;
  if (h_pos)
    GCME_TRY_CK(cudaMemcpyAsync(h_pos, b->eng.P.pos, sizeof(double) * 3 * n,
                                cudaMemcpyDeviceToHost, st));
  std::vector<double> v64;
  if (h_vel) {
    if (b->eng.fp64) {
      v64.resize(3 * n);
      GCME_TRY_CK(cudaMemcpyAsync(v64.data(), b->eng.P.vel, sizeof(double) * 3 * n,
                                  cudaMemcpyDeviceToHost, st));
    } else {
      GCME_TRY_CK(cudaMemcpyAsync(h_vel, b->eng.P.vel, sizeof(float) * 3 * n,
                                  cudaMemcpyDeviceToHost, st));
    }
  }
  if (h_energy)
    GCME_TRY_CK(cudaMemcpyAsync(h_energy, b->eng.P.energy,
                                sizeof(double) * GCME_NTERMS * b->eng.nsys(),
                                cudaMemcpyDeviceToHost, st));
  GCME_TRY_CK(cudaStreamSynchronize(st));
  if (h_vel && b->eng.fp64)
    for (long long k = 0; k < 3 * n; ++k) h_vel[k] = (float)v64[k];
  return GCME_OK;
}

int gcme_batch_step(gcme_batch *b, int64_t nsteps, int32_t mode, gcme_stream_t stream) {
  if (!b || nsteps < 0 || (mode != 0 && mode != 1)) {
    set_error("invalid argument to gcme_batch_step");
    return GCME_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  GCME_TRY_CK(cudaSetDevice(b->eng.device));
  const Pool &Q = b->eng.P;
  cudaGraphExec_t fg, sg;
  int rc = b->eng.forces_graph(Q, &fg);
  if (rc) return rc;
  if (mode == 0) {
    rc = b->eng.step_graph(Q, &sg);
    if (rc) return rc;
  } else {
    b->eng.last_step_timed = false;  // the persistent kernel records no phase events
  }
  if (!b->forces_valid) {
    GCME_TRY_CK(cudaGraphLaunch(fg, st));
    b->forces_valid = true;
  }
  if (mode == 0) {
    for (int64_t k = 0; k < nsteps; ++k) GCME_TRY_CK(cudaGraphLaunch(sg, st));
    return check_launch("gcme_batch_step");
  }
  if (b->eng.fp64) {
    set_error("the persistent launch (mode 1) runs FP32 batches");
    return GCME_ERR_INVALID;
  }
  if (nsteps == 0) return GCME_OK;
  int lr = launch_persistent(b->eng.cell_only(Q), b->eng.pair_work, b->eng.n_pair_work, b->eng.cell_factor,
                             b->eng.plan, nsteps, b->eng.bar_words, 2.0, st,
                             b->eng.pair_nelec == 0, b->eng.pair_nelec < 0);
  if (lr != 0) {
    cudaError_t e = cudaGetLastError();
    set_error(std::string("persistent cooperative launch failed: ") + cudaGetErrorString(e));
    return GCME_ERR_CUDA;
  }
  b->eng.request_rebuild(st);  // the persistent kernel re-sorted the cells
  unsigned int words[4] = {0, 0, 0, 0};
  GCME_TRY_CK(cudaMemcpyAsync(words, b->eng.bar_words, sizeof(words), cudaMemcpyDeviceToHost, st));
  GCME_TRY_CK(cudaStreamSynchronize(st));
  if (words[2] != 0) {
    set_error("persistent launch: a grid barrier wait ran out (2 s)");
    return GCME_ERR_TIMEOUT;
  }
  return check_launch("gcme_batch_step");
}

}  // extern "C"
