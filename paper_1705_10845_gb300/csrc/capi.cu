// C ABI of the XL-BOMD hot path and its host-side orchestration.
//
// Per system the library keeps: positions, velocities, forces, the n history
// n(t - k dt) (Eq. VRL_Damp), H0 and H[n], gamma, the expansion matrices
// T_0..T_n and Y_0..Y_{n-1} of the recursive Fermi-operator expansion (kept
// for the response chains), the response work matrices and the rank-m probes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/xlbomd.h"
#include "internal.h"
#include "precision.h"

using namespace xl;

std::atomic<long long> xl::g_launch_count{0};
thread_local long long xl::t_launch_count = 0;

namespace {

constexpr double kKB = 8.617333262e-5;
constexpr double kAcc = 9.648533e-3;   // 1 eV/(amu A) in A/fs^2

struct Sys {
  int nat = 0, N = 0, np = 0, natp = 0, ng = 0, kp = 0;
  double L = 0, mass = 0, nocc = 0, eta = 0;
  // device, FP64
  double *R = nullptr, *V = nullptr, *F = nullptr, *Z = nullptr, *nh = nullptr, *q = nullptr, *r = nullptr;
  double *Kr = nullptr, *pot = nullptr, *potv = nullptr, *gam = nullptr, *SF = nullptr, *G4 = nullptr;
  double *H0 = nullptr, *H = nullptr, *Dm = nullptr;
  double *ddiag = nullptr, *dmu_diag = nullptr, *d1 = nullptr, *dvec = nullptr, *dvec_mu = nullptr;
  double *pV = nullptr, *pW = nullptr, *scal = nullptr, *work = nullptr, *energy = nullptr;
  double *Kfull = nullptr, *Jm = nullptr;   // exact kernel (natoms x natoms) and its work matrix
  // exact kernel, split precisions: chain slots for probes run side by side, and per slot the
  // probe v, response w, potential, diagonal perturbation, chain diagonal and scratch
  std::vector<MatSet> slots;
  double* slot_vec = nullptr;
  MatSet mats;   // expansion matrices in the working precision
  // host
  double mu = 0.0;
  bool mu_valid = false;
  double mu_hist[3] = {0, 0, 0};
  int n_mu_hist = 0;
  double dmu_last = 0.0;
  double kc = 0.0;          // c of J_0 = c I for this system
  bool have_density = false;
  bool have_K = false;      // Kfull holds an exact kernel
  long long md_steps = 0;   // MD steps taken by this system
  int probes_used = 0;
  double stats[5] = {0, 0, 0, 0, 0};
  double eh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<double> G4h;
  // captured work (params.graphs): one graph per Newton-Schulz plan of a chemical-potential pass,
  // one per probe slot of the kernel update; dpar holds mu and the start scales c_k
  struct Captured {
    std::vector<int> key;
    int seen = 0;                      // eager runs before the capture
    cudaGraphExec_t exec = nullptr;
    double stats[5] = {0, 0, 0, 0, 0};  // host counters one run adds
    long long launches = 0;            // kernels one run launches
  };
  std::vector<Captured> graphs;
  double* dpar = nullptr;
};

}  // namespace

struct xlbomd_ctx {
  xlbomd_params p{};
  cudaStream_t stream = nullptr;
  std::vector<Sys> sys;
  double* pinned = nullptr;
  double* pinned_group = nullptr;   // lockstep: 2 doubles per system
  double* ppar = nullptr;   // pinned staging of the device parameters of a captured pass
  double* cdev = nullptr;
  int status = XLBOMD_OK;
  std::string msg;
  xl::Engine* eng = nullptr;
};

namespace {

bool debug_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("XLBOMD_DEBUG");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

xlbomd_status fail(xlbomd_ctx* c, xlbomd_status st, const std::string& m) {
  if (c) {
    if (c->status == XLBOMD_OK) {
      c->status = st;
      c->msg = m;
    }
  }
  return st;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, XLBOMD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKS(call)                          \
  do {                                     \
    xlbomd_status s_ = (call);             \
    if (s_ != XLBOMD_OK) return s_;        \
  } while (0)

xlbomd_status dalloc(xlbomd_ctx* ctx, double** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(double) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(ctx, XLBOMD_ERR_OOM, "cudaMalloc failed");
  }
  e = cudaMemsetAsync(*p, 0, sizeof(double) * std::max<size_t>(count, 1), ctx->stream);
  if (e != cudaSuccess) return fail(ctx, XLBOMD_ERR_CUDA, cudaGetErrorString(e));
  return XLBOMD_OK;
}

ModelConst model_of(const xlbomd_params& p) {
  ModelConst m;
  m.eps_s = p.eps_s;
  m.eps_p = p.eps_p;
  for (int k = 0; k < 4; ++k) m.t0[k] = p.t0[k];
  m.r_decay = p.r_decay;
  m.r_cut = p.r_cut;
  m.r_taper = p.r_taper;
  m.U = p.hubbard_U;
  m.k = p.coulomb_k;
  m.rep_A = p.rep_A;
  m.rep_rho = p.rep_rho;
  return m;
}

double beta_of(const xlbomd_params& p) { return 1.0 / (kKB * p.Te); }

// Reciprocal vectors of the Ewald sum: eta = 4/L, G = 2 pi h / L with h in a
// half space, 0 < |G| <= 2 eta 6.07; weight w = 2 * 4 pi / V exp(-G^2/4eta^2)/G^2.
void ewald_vectors(double L, double& eta, std::vector<double>& G4) {
  eta = 4.0 / L;
  const double gmax = 2.0 * eta * 6.07;
  const int hmax = (int)std::ceil(gmax * L / (2.0 * kPi));
  G4.clear();
  for (int hx = -hmax; hx <= hmax; ++hx)
    for (int hy = -hmax; hy <= hmax; ++hy)
      for (int hz = -hmax; hz <= hmax; ++hz) {
        const bool pos = hx > 0 || (hx == 0 && (hy > 0 || (hy == 0 && hz > 0)));
        if (!pos) continue;
        const double gx = 2 * kPi * hx / L, gy = 2 * kPi * hy / L, gz = 2 * kPi * hz / L;
        const double g2 = gx * gx + gy * gy + gz * gz;
        if (g2 > gmax * gmax) continue;
        const double w = 2.0 * 4.0 * kPi / (L * L * L) * std::exp(-g2 / (4.0 * eta * eta)) / g2;
        G4.push_back(gx);
        G4.push_back(gy);
        G4.push_back(gz);
        G4.push_back(w);
      }
}

xlbomd_status check(xlbomd_ctx* ctx, int sys) {
  if (!ctx) return XLBOMD_ERR_ARG;
  if (ctx->status != XLBOMD_OK) return (xlbomd_status)ctx->status;
  if (sys < 0 || sys >= (int)ctx->sys.size()) return fail(ctx, XLBOMD_ERR_ARG, "system index out of range");
  return XLBOMD_OK;
}

// Work that params.graphs may capture: split precisions, up to 2048 padded orbitals (where
// launch overhead matters), no per-product event timing, and a caller stream (the legacy
// default stream cannot be captured).
bool use_graphs(const xlbomd_ctx* ctx, const Sys& S) {
  return ctx->p.graphs == 1 && ctx->p.prec != XLBOMD_FP64 && S.np <= 2048 && !ctx->eng->prof &&
         ctx->stream != nullptr && ctx->stream != cudaStreamLegacy && ctx->stream != cudaStreamPerThread;
}

// Enqueue fn's work on the context stream: eagerly the first time `key` is seen (this also
// makes every lazy set-up happen outside a capture), captured into a CUDA graph the second
// time, replayed from the graph afterwards.  fn must enqueue the same work for the same key;
// what may differ between runs lives in device memory (for the chemical-potential pass, mu
// and the Newton-Schulz start scales in S.dpar).
xlbomd_status run_captured(xlbomd_ctx* ctx, Sys& S, const std::vector<int>& key,
                           const std::function<xlbomd_status()>& fn) {
  cudaStream_t st = ctx->stream;
  Sys::Captured* g = nullptr;
  for (auto& x : S.graphs)
    if (x.key == key) g = &x;
  if (!g) {
    S.graphs.emplace_back();
    g = &S.graphs.back();
    g->key = key;
  }
  if (g->exec) {
    CK(cudaGraphLaunch(g->exec, st));
    for (int k = 0; k < 5; ++k) S.stats[k] += g->stats[k];
    g_launch_count.fetch_add(g->launches, std::memory_order_relaxed);
    return XLBOMD_OK;
  }
  if (g->seen == 0) {
    g->seen = 1;
    return fn();
  }
  double before[5];
  std::memcpy(before, S.stats, sizeof(before));
  const long long l0 = t_launch_count;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const xlbomd_status rs = fn();
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (rs != XLBOMD_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rs != XLBOMD_OK ? rs : fail(ctx, XLBOMD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    g->exec = nullptr;
    return fail(ctx, XLBOMD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  }
  for (int k = 0; k < 5; ++k) g->stats[k] = S.stats[k] - before[k];
  g->launches = t_launch_count - l0;
  CK(cudaGraphLaunch(g->exec, st));   // the captured work has not run yet
  return XLBOMD_OK;
}

xlbomd_status sync_read(xlbomd_ctx* ctx, const double* dev, int count) {
  CK(cudaMemcpyAsync(ctx->pinned, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return XLBOMD_OK;
}

// y = gamma x (real-space matrix plus the reciprocal part through the structure factors)
cudaError_t gamma_apply(xlbomd_ctx* ctx, Sys& S, const double* x, double* y, double* tmp) {
  return launch_gamma_apply(ctx->stream, S.nat, S.gam, S.natp, S.SF, S.kp, ctx->p.coulomb_k, x, y, tmp);
}

// a1-a2
xlbomd_status build_H(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  const ModelConst m = model_of(ctx->p);
  CK(launch_build_H0(st, m, S.nat, S.L, S.R, S.H0, S.np));
  const bool fp32_pairs = ctx->p.prec != XLBOMD_FP64;
  if (ctx->p.coulomb_k != 0.0) {
    CK(launch_gamma_real(st, m, S.nat, S.L, S.eta, S.R, S.gam, S.natp, fp32_pairs));
    CK(launch_structure_factors(st, S.nat, S.ng, S.G4, S.R, S.SF, S.kp));
  }
  CK(gamma_apply(ctx, S, S.nh, S.pot, S.work));
  CK(launch_apply_potential(st, S.nat, S.np, S.H0, S.pot, S.H));
  S.have_density = false;
  return XLBOMD_OK;
}

// Newton-Schulz plan per level from the scalar map over t in [0, t_max(k)]:
// level 0 starts from Y = I - S (error t^4), level k > 0 from c_k Y_{k-1}
// with c_k minimising max |1 - c b_k / b_{k-1}|, b = 1 + t^2.
void ns_plan(double t0max, int n, double tol, std::vector<int>& s, std::vector<double>& c) {
  const int G = 2001;
  std::vector<double> t(G), prev(G);
  for (int i = 0; i < G; ++i) t[i] = t0max * i / (G - 1);
  s.assign(n, 0);
  c.assign(n, 1.0);
  for (int k = 0; k < n; ++k) {
    double e;
    if (k == 0) {
      e = 0.0;
      for (int i = 0; i < G; ++i) e = std::max(e, std::fabs(1.0 - (1.0 + t[i] * t[i]) * (1.0 - t[i] * t[i])));
    } else {
      double rmin = 1e300, rmax = -1e300;
      for (int i = 0; i < G; ++i) {
        const double rho = (1.0 + t[i] * t[i]) / (1.0 + prev[i] * prev[i]);
        rmin = std::min(rmin, rho);
        rmax = std::max(rmax, rho);
      }
      c[k] = 2.0 / (rmin + rmax);
      e = (rmax - rmin) / (rmax + rmin);
    }
    int it = 0;
    double err = e;
    while (err > tol && it < 10) {
      err = err * err;
      ++it;
    }
    s[k] = it;
    prev = t;
    for (int i = 0; i < G; ++i) t[i] = 2.0 * t[i] / (1.0 + t[i] * t[i]);
  }
}

// Safeguarded Newton search for the chemical potential of one system (Tr D(mu) = N_occ): the
// host side of the mu passes, shared by the one-system and the lockstep paths.
struct MuSearch {
  double glo = 0, ghi = 0, mu = 0, blo = 0, bhi = 0, dmu = 0, t0max = 0;
  int pass = 0;
  bool done = false;
  std::vector<int> plan_s;
  std::vector<double> plan_c;

  // start from the Gershgorin interval [glo, ghi] and the system's mu history
  xlbomd_status start(xlbomd_ctx* ctx, const Sys& S, double lo, double hi) {
    glo = lo;
    ghi = hi;
    if (!std::isfinite(glo) || !std::isfinite(ghi))
      return fail(ctx, XLBOMD_ERR_SPECTRUM, "non-finite Hamiltonian (Gershgorin bounds)");
    if (S.mu_valid) {
      mu = S.mu;
      if (S.n_mu_hist >= 3)
        mu = 3.0 * S.mu_hist[0] - 3.0 * S.mu_hist[1] + S.mu_hist[2];
      else if (S.n_mu_hist == 2)
        mu = 2.0 * S.mu_hist[0] - S.mu_hist[1];
    } else {
      mu = 0.5 * (glo + ghi);
    }
    blo = glo - 1.0;   // bracket of the root of Tr D(mu) = N_occ
    bhi = ghi + 1.0;
    dmu = 0.0;
    pass = 0;
    done = false;
    return XLBOMD_OK;
  }

  // spectral bound and Newton-Schulz plan of the next pass
  xlbomd_status prepare(xlbomd_ctx* ctx, Sys& S) {
    const xlbomd_params& p = ctx->p;
    if (pass >= p.mu_max_iter) return fail(ctx, XLBOMD_ERR_NOT_CONVERGED, "chemical potential did not converge");
    const double sc = beta_of(p) / std::ldexp(1.0, p.n_sq + 1);
    t0max = sc * std::max(std::fabs(ghi - mu), std::fabs(mu - glo));
    if (!(t0max < 1.0)) return fail(ctx, XLBOMD_ERR_SPECTRUM, "|beta (e - mu)| / 2^(n+1) >= 1");
    ns_plan(t0max, p.n_sq, (p.prec == XLBOMD_FP64) ? 1e-16 : 1e-8, plan_s, plan_c);
    S.mats.t0max = t0max;
    return XLBOMD_OK;
  }

  // the pass's traces: Tr T_n (tn) and Tr dT_n/dmu (tmu)
  xlbomd_status update(xlbomd_ctx* ctx, Sys& S, double tn, double tmu) {
    const xlbomd_params& p = ctx->p;
    const double beta = beta_of(p);
    const double occ_floor = ((p.prec == XLBOMD_FP64) ? 1e-12 : 1e-6) * S.N;
    const double trD = 0.5 * (S.N + tn);
    const double trDmu = 0.5 * tmu;
    if (!std::isfinite(trD) || !std::isfinite(trDmu))
      return fail(ctx, XLBOMD_ERR_NOT_CONVERGED, "non-finite trace in the expansion");
    if (trD < S.nocc)
      blo = std::max(blo, mu);
    else
      bhi = std::min(bhi, mu);
    const double dmu_prev = dmu;
    const double err = S.nocc - trD;
    // Newton step; none where Tr D is flat in mu (mu in a gap or outside the spectrum)
    dmu = (trDmu > 0.0) ? err / trDmu : HUGE_VAL;
    S.stats[0] += 1;
    if (debug_enabled())
      std::fprintf(stderr, "[xlbomd] mu pass %d: mu %.12f trD %.10f (nocc %.1f) trDmu %.6e dmu %.3e bracket [%.6f, %.6f] t0max %.4e\n",
                   pass, mu, trD, S.nocc, trDmu, dmu, blo, bhi, t0max);
    ++pass;
    if (std::fabs(dmu) * beta < p.mu_tol) {
      done = true;
      return XLBOMD_OK;
    }
    // flat region with the occupation already met to the trace's rounding floor: keep mu
    if (std::fabs(err) < occ_floor) {
      dmu = 0.0;
      done = true;
      return XLBOMD_OK;
    }
    // Newton converges quadratically; once a step is not much smaller than
    // the previous one (and already small), the rounding noise of the
    // product arithmetic has been reached: keep the first-order correction.
    if (pass >= 2 && std::fabs(dmu) * beta < 0.05 && std::fabs(dmu) > 0.25 * std::fabs(dmu_prev)) {
      done = true;
      return XLBOMD_OK;
    }
    double next = mu + dmu;
    if (!(trDmu > 0.0) || !(next > blo && next < bhi)) next = 0.5 * (blo + bhi);
    mu = next;
    return XLBOMD_OK;
  }

  // first-order correction D(mu + dmu) = D(mu) + dmu dD/dmu and the mu history
  void finish(Sys& S) const {
    S.dmu_last = dmu;
    S.mu = mu + dmu;
    S.mu_valid = true;
    S.mu_hist[2] = S.mu_hist[1];
    S.mu_hist[1] = S.mu_hist[0];
    S.mu_hist[0] = S.mu;
    S.n_mu_hist = std::min(S.n_mu_hist + 1, 3);
  }
};

// density matrix, charges (and forces) from the final mu pass
xlbomd_status density_finish(xlbomd_ctx* ctx, Sys& S, const MuSearch& ms, bool with_forces) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  ms.finish(S);
  CK(ctx->eng->density_out(st, S.mats, S.N, ms.dmu, S.dmu_diag, S.ddiag, S.Dm));
  CK(launch_charges(st, S.nat, S.ddiag, S.Z, S.nh, S.q, S.r));
  if (with_forces) {
    CK(launch_forces(st, model_of(p), S.nat, S.L, S.eta, S.ng, S.G4, S.R, S.Dm, S.np, S.q, S.nh, S.F, S.work,
                     p.prec != XLBOMD_FP64));
  }
  S.have_density = true;
  return XLBOMD_OK;
}

// a3-a6
xlbomd_status density(xlbomd_ctx* ctx, Sys& S, bool with_forces) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  const int n = p.n_sq;
  const double sc = beta_of(p) / std::ldexp(1.0, n + 1);
  Engine& E = *ctx->eng;

  CK(launch_gershgorin(st, S.N, S.np, S.H, S.work));
  CKS(sync_read(ctx, S.work, 2));
  MuSearch ms;
  CKS(ms.start(ctx, S, ctx->pinned[0], ctx->pinned[1]));
  while (!ms.done) {
    CKS(ms.prepare(ctx, S));
    const double mu = ms.mu;
    auto mu_pass = [&](const double* dp) -> xlbomd_status {
      CK(E.foe(st, S.mats, S.H, S.N, mu, sc, ms.plan_s, ms.plan_c, S.stats, dp));
      // mu chain: T1_0 = +sc I, full last level
      CK(E.chain(st, S.mats, S.dvec_mu, S.N, true, S.dmu_diag, S.stats));
      CK(E.trace_tn(st, S.mats, S.N, S.scal));          // scal[0] = sum_i T_n,ii
      CK(launch_sum(st, S.N, S.dmu_diag, S.scal + 1));    // scal[1] = sum_i dT_n,ii/dmu
      return XLBOMD_OK;
    };
    if (use_graphs(ctx, S)) {
      if (!S.dpar) CKS(dalloc(ctx, &S.dpar, 64));
      ctx->ppar[0] = mu;
      for (int k = 0; k < n && k < 63; ++k) ctx->ppar[1 + k] = ms.plan_c[k];
      CK(cudaMemcpyAsync(S.dpar, ctx->ppar, sizeof(double) * 64, cudaMemcpyHostToDevice, st));
      std::vector<int> key{0};
      key.insert(key.end(), ms.plan_s.begin(), ms.plan_s.end());
      CKS(run_captured(ctx, S, key, [&] { return mu_pass(S.dpar); }));
    } else {
      CKS(mu_pass(nullptr));
    }
    int* herr = reinterpret_cast<int*>(ctx->pinned + 63);
    *herr = 0;
    if (const int* derr = E.device_error())
      CK(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKS(sync_read(ctx, S.scal, 2));
    if (*herr != 0) return fail(ctx, XLBOMD_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up or a tile was out of range");
    CKS(ms.update(ctx, S, ctx->pinned[0], ctx->pinned[1]));
  }
  return density_finish(ctx, S, ms, with_forces);
}

// a3-a6 for several systems of one padded size in lockstep: every mu pass runs the expansion
// and the mu chain of all systems still searching as grouped launches, with one host
// synchronisation per pass for all of them.  Each system takes exactly the steps of density().
xlbomd_status density_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G, bool with_forces) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  const double sc = beta_of(p) / std::ldexp(1.0, p.n_sq + 1);
  Engine& E = *ctx->eng;
  const size_t B = G.size();
  double* h = ctx->pinned_group;
  for (size_t i = 0; i < B; ++i) {
    CK(launch_gershgorin(st, G[i]->N, G[i]->np, G[i]->H, G[i]->work));
    CK(cudaMemcpyAsync(h + 2 * i, G[i]->work, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  std::vector<MuSearch> ms(B);
  for (size_t i = 0; i < B; ++i) CKS(ms[i].start(ctx, *G[i], h[2 * i], h[2 * i + 1]));
  std::vector<size_t> active(B);
  for (size_t i = 0; i < B; ++i) active[i] = i;
  while (!active.empty()) {
    std::vector<FoeJob> fj;
    std::vector<ChainJob> cj;
    for (size_t i : active) {
      Sys& S = *G[i];
      CKS(ms[i].prepare(ctx, S));
      FoeJob f;
      f.m = &S.mats;
      f.H = S.H;
      f.N = S.N;
      f.mu = ms[i].mu;
      f.ns = &ms[i].plan_s;
      f.nc = &ms[i].plan_c;
      f.stats = S.stats;
      fj.push_back(f);
      ChainJob c;
      c.m = &S.mats;
      c.dvec = S.dvec_mu;   // mu chain: T1_0 = +sc I, full last level
      c.N = S.N;
      c.out_diag = S.dmu_diag;
      c.stats = S.stats;
      cj.push_back(c);
    }
    CK(E.foe_group(st, fj, sc));
    CK(E.chain_group(st, cj, true));
    for (size_t k = 0; k < active.size(); ++k) {
      Sys& S = *G[active[k]];
      CK(E.trace_tn(st, S.mats, S.N, S.scal));
      CK(launch_sum(st, S.N, S.dmu_diag, S.scal + 1));
      CK(cudaMemcpyAsync(h + 2 * k, S.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    int* herr = reinterpret_cast<int*>(ctx->pinned + 63);
    *herr = 0;
    if (const int* derr = E.device_error())
      CK(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*herr != 0) return fail(ctx, XLBOMD_ERR_TIMEOUT, "tensor-core product: a bounded wait gave up or a tile was out of range");
    std::vector<size_t> next;
    for (size_t k = 0; k < active.size(); ++k) {
      const size_t i = active[k];
      CKS(ms[i].update(ctx, *G[i], h[2 * k], h[2 * k + 1]));
      if (ms[i].done)
        CKS(density_finish(ctx, *G[i], ms[i], with_forces));
      else
        next.push_back(i);
    }
    active.swap(next);
  }
  return XLBOMD_OK;
}

// a7: one probe.  H1 = diag(gamma v) on orbitals, T1_0 = -sc H1.
xlbomd_status response(xlbomd_ctx* ctx, Sys& S, const double* v, double* w) {
  cudaStream_t st = ctx->stream;
  const double sc = beta_of(ctx->p) / std::ldexp(1.0, ctx->p.n_sq + 1);
  CK(gamma_apply(ctx, S, v, S.potv, S.work));
  CK(launch_expand_potential(st, S.nat, S.np, -sc, S.potv, S.dvec));
  CK(ctx->eng->chain(st, S.mats, S.dvec, S.N, false, S.d1, S.stats));
  CK(launch_response_finish(st, S.nat, S.N, S.d1, S.dmu_diag, S.scal + 4, w));
  return XLBOMD_OK;
}

// Columns of J - I for the exact kernel with the unit-probe responses run side by side: up
// to 64 probes at a time, each in its own chain slot, every chain product one grouped launch
// over the probes.  The number of slots is bounded by a quarter of the free device memory.
xlbomd_status exact_columns_grouped(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  const double sc = beta_of(ctx->p) / std::ldexp(1.0, ctx->p.n_sq + 1);
  const size_t per_vec = 2 * (size_t)S.nat + 3 * (size_t)S.np + (size_t)S.kp + 64;   // v, w, potv?, ...
  if (S.slots.empty()) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t per_slot = chain_slot_bytes(S.np, ctx->p.prec) + per_vec * sizeof(double);
    int G = (int)std::min<size_t>(64, std::max<size_t>(1, free_b / 4 / per_slot));
    G = std::min(G, S.nat);
    S.slots.resize(G);
    for (int j = 0; j < G; ++j)
      if (alloc_chain_slot(S.slots[j], S.mats, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, XLBOMD_ERR_OOM, "exact kernel: chain slot allocation failed");
      }
    CKS(dalloc(ctx, &S.slot_vec, per_vec * G));
  }
  const int G = (int)S.slots.size();
  auto vec = [&](int j, int what) -> double* {   // 0 v, 1 w, 2 potv, 3 dvec, 4 d1, 5 scal, 6 tmp
    double* b = S.slot_vec + per_vec * (size_t)j;
    const size_t off[7] = {0, (size_t)S.nat, 2 * (size_t)S.nat, 2 * (size_t)S.nat + S.np,
                           2 * (size_t)S.nat + 2 * (size_t)S.np, 2 * (size_t)S.nat + 3 * (size_t)S.np,
                           2 * (size_t)S.nat + 3 * (size_t)S.np + 32};
    return b + off[what];
  };
  for (int I0 = 0; I0 < S.nat; I0 += G) {
    const int g = std::min(G, S.nat - I0);
    std::vector<ChainJob> cj(g);
    for (int j = 0; j < g; ++j) {
      CK(launch_unit_vector(st, S.nat, I0 + j, vec(j, 0)));
      CK(launch_gamma_apply(st, S.nat, S.gam, S.natp, S.SF, S.kp, ctx->p.coulomb_k, vec(j, 0), vec(j, 2),
                            vec(j, 6)));
      CK(launch_expand_potential(st, S.nat, S.np, -sc, vec(j, 2), vec(j, 3)));
      cj[j].m = &S.slots[j];
      cj[j].dvec = vec(j, 3);
      cj[j].N = S.N;
      cj[j].out_diag = vec(j, 4);
      cj[j].stats = S.stats;
    }
    CK(ctx->eng->chain_group(st, cj, false));
    for (int j = 0; j < g; ++j) {
      CK(launch_response_finish(st, S.nat, S.N, vec(j, 4), S.dmu_diag, vec(j, 5), vec(j, 1)));
      CK(launch_jacobian_column(st, S.nat, I0 + j, vec(j, 1), S.Jm, S.Kfull));
    }
  }
  return XLBOMD_OK;
}

// a7-a8
// Exact kernel K = (J - I)^-1 (Eq. KK): J column by column from the responses to the
// unit directions e_I, then Gauss-Jordan with partial pivoting in FP64.
xlbomd_status kernel_exact(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  if (!S.have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  const size_t nn = (size_t)S.nat * S.nat;
  if (!S.Kfull) CKS(dalloc(ctx, &S.Kfull, nn));
  if (!S.Jm) CKS(dalloc(ctx, &S.Jm, nn));
  if (ctx->p.prec != XLBOMD_FP64 && S.nat > 1) {
    CKS(exact_columns_grouped(ctx, S));
  } else {
    double* v = S.pV + (size_t)kMaxRank * S.nat;   // spare probe rows
    double* w = S.pW + (size_t)kMaxRank * S.nat;
    for (int I = 0; I < S.nat; ++I) {
      CK(launch_unit_vector(st, S.nat, I, v));
      CKS(response(ctx, S, v, w));
      CK(launch_jacobian_column(st, S.nat, I, w, S.Jm, S.Kfull));
    }
  }
  CK(cudaMemsetAsync(S.scal + 10, 0, sizeof(double), st));
  CK(launch_gauss_jordan(st, S.nat, S.Jm, S.Kfull, S.work, S.scal + 10));
  CKS(sync_read(ctx, S.scal + 10, 1));
  if (ctx->pinned[0] != 0.0) return fail(ctx, XLBOMD_ERR_NOT_CONVERGED, "J - I is numerically singular");
  S.have_K = true;
  return XLBOMD_OK;
}

// Accumulated kernel: the carried K (= (J - I)^-1) gets one rank-1 update at the current
// state (end of Section V.F): v = K r/|K r|, u = w - J v, J += u v^T,
// K -= K u v^T K / (1 + v^T K u) (Eq. K_up).  A (re)started kernel is K_0 = (c-1)^-1 I,
// J_0 = c I with no update: at the t0 ground state r is rounding noise, and a probe along it
// would keep that noise in K.
xlbomd_status kernel_accumulate(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  if (!S.have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  const int n = S.nat;
  if (!S.Kfull) CKS(dalloc(ctx, &S.Kfull, (size_t)n * n));
  if (!S.Jm) CKS(dalloc(ctx, &S.Jm, (size_t)n * n));
  if (!S.have_K) {
    CK(launch_scaled_identity(st, n, 1.0 / (S.kc - 1.0), S.Kfull));
    CK(launch_scaled_identity(st, n, S.kc, S.Jm));
    S.have_K = true;
    return XLBOMD_OK;
  }
  double* v = S.pV + (size_t)kMaxRank * n;   // spare probe rows
  double* w = S.pW + (size_t)kMaxRank * n;
  double *t = S.work, *u = S.work + n, *Ku = S.work + 2 * n, *vK = S.work + 3 * n;
  CK(launch_gemv(st, n, S.Kfull, n, S.r, v));
  CK(launch_normalize(st, n, v, S.scal + 11));
  CKS(sync_read(ctx, S.scal + 11, 1));
  if (ctx->pinned[0] == 1.0) {
    CKS(response(ctx, S, v, w));
    CK(launch_gemv(st, n, S.Jm, n, v, t));
    CK(launch_sub(st, n, w, t, u));
    CK(launch_gemv(st, n, S.Kfull, n, u, Ku));
    CK(launch_gemv_t(st, n, S.Kfull, v, vK));
    CK(launch_dot1p(st, n, v, Ku, S.scal + 12));
    CK(launch_rank1_update(st, n, u, v, Ku, vK, S.scal + 12, S.Jm, S.Kfull));
  }
  return XLBOMD_OK;
}

xlbomd_status kernel_update(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  if (p.kernel_mode == 2) {
    CKS(kernel_accumulate(ctx, S));
    CK(launch_gemv(st, S.nat, S.Kfull, S.nat, S.r, S.Kr));
    S.probes_used = 1;
    S.stats[2] = 1;
    return XLBOMD_OK;
  }
  if (p.kernel_mode == 1) {
    if (!S.have_K) CKS(kernel_exact(ctx, S));
    CK(launch_gemv(st, S.nat, S.Kfull, S.nat, S.r, S.Kr));
    S.probes_used = S.nat;
    S.stats[2] = S.nat;
    return XLBOMD_OK;
  }
  int m = 0;
  for (int i = 0; i < p.rank_m; ++i) {
    CK(launch_kernel_vec(st, 0, S.nat, i, S.kc, S.r, S.pV, S.pW, nullptr, S.scal + 8));
    CKS(sync_read(ctx, S.scal + 8, 1));
    if (ctx->pinned[0] != 1.0) break;
    double* vi = S.pV + (size_t)i * S.nat;
    double* wi = S.pW + (size_t)i * S.nat;
    if (use_graphs(ctx, S))
      CKS(run_captured(ctx, S, {1, i}, [&] { return response(ctx, S, vi, wi); }));
    else
      CKS(response(ctx, S, vi, wi));
    m = i + 1;
  }
  CK(launch_kernel_vec(st, 1, S.nat, m, S.kc, S.r, S.pV, S.pW, S.Kr, S.scal + 8));
  S.probes_used = m;
  S.stats[2] = m;
  return XLBOMD_OK;
}

// a10
xlbomd_status energy(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(S.energy + 4, 0, sizeof(double), st));
  if (ctx->p.rep_A != 0.0) {
    CK(launch_repulsion(st, model_of(ctx->p), S.nat, S.L, S.R, nullptr, S.work));
    CK(launch_sum(st, S.nat, S.work, S.energy + 4));
  }
  CK(launch_frob_dot(st, S.N, S.np, S.Dm, S.H0, S.work, S.energy + 0));
  CK(launch_energy_vec(st, S.nat, S.q, S.nh, S.pot, S.V, S.mass, S.energy + 1));
  CK(ctx->eng->entropy(st, S.mats, S.N, beta_of(ctx->p), ctx->p.n_sq, S.mu, S.dmu_last, S.Dm, S.H, S.work,
                       S.energy + 3));
  CKS(sync_read(ctx, S.energy, 5));
  const double band = 2.0 * ctx->pinned[0], coul = ctx->pinned[1], ke = ctx->pinned[2];
  const double ent = -2.0 * kKB * ctx->p.Te * ctx->pinned[3], rep = ctx->pinned[4];
  const double om = band + coul + ent + rep;
  const double out[7] = {om, band, coul, ent, ke, om + ke, rep};
  std::memcpy(S.eh, out, sizeof(out));
  return XLBOMD_OK;
}

// Most negative eigenvalue of J = dq/dn by power iteration on the response
// (J has real non-positive spectrum: it is similar to -g^(1/2) chi g^(1/2)).
xlbomd_status stiffest_mode(xlbomd_ctx* ctx, Sys& S, double* lambda) {
  cudaStream_t st = ctx->stream;
  std::vector<double> v(S.nat);
  for (int I = 0; I < S.nat; ++I) v[I] = ((I * 7919) % 17) - 8.0;
  double mean = 0.0;
  for (double x : v) mean += x;
  mean /= S.nat;
  double nv = 0.0;
  for (double& x : v) {
    x -= mean;
    nv += x * x;
  }
  nv = std::sqrt(nv);
  if (nv == 0.0) {
    *lambda = 0.0;
    return XLBOMD_OK;
  }
  for (double& x : v) x /= nv;
  double* dv = S.pV + (size_t)kMaxRank * S.nat;   // spare probe rows
  double* dw = S.pW + (size_t)kMaxRank * S.nat;
  double lam = 0.0;
  std::vector<double> w(S.nat);
  for (int it = 0; it < 12; ++it) {
    CK(cudaMemcpyAsync(dv, v.data(), sizeof(double) * S.nat, cudaMemcpyHostToDevice, st));
    CKS(response(ctx, S, dv, dw));
    CK(cudaMemcpyAsync(w.data(), dw, sizeof(double) * S.nat, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double dot = 0.0, nw = 0.0;
    for (int I = 0; I < S.nat; ++I) {
      dot += v[I] * w[I];
      nw += w[I] * w[I];
    }
    nw = std::sqrt(nw);
    lam = dot;
    if (!(nw > 0.0) || !std::isfinite(nw)) break;
    for (int I = 0; I < S.nat; ++I) v[I] = w[I] / nw;
  }
  *lambda = lam;
  return XLBOMD_OK;
}

xlbomd_status scf(xlbomd_ctx* ctx, Sys& S) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  double best = HUGE_VAL;
  int since_best = 0;
  for (int it = 0; it < p.scf_max_iter; ++it) {
    CK(gamma_apply(ctx, S, S.nh, S.pot, S.work));
    CK(launch_apply_potential(st, S.nat, S.np, S.H0, S.pot, S.H));
    CKS(density(ctx, S, false));
    if (it == 0 && p.kernel_auto) {
      double lam = 0.0;
      CKS(stiffest_mode(ctx, S, &lam));
      if (lam < 0.0) S.kc = 1.2 * lam;
      if (debug_enabled()) std::fprintf(stderr, "[xlbomd] stiffest mode %.4f -> c = %.4f\n", lam, S.kc);
    }
    CK(launch_absmax(st, S.nat, S.r, S.scal + 9));
    CKS(sync_read(ctx, S.scal + 9, 1));
    const double res = ctx->pinned[0];
    if (debug_enabled()) std::fprintf(stderr, "[xlbomd] scf it %d max|q - n| %.3e mu %.8f\n", it, res, S.mu);
    if (!std::isfinite(res) || res > 1e3) return fail(ctx, XLBOMD_ERR_DIVERGED, "t0 SCF diverged");
    // split precisions: the residual stops falling at the rounding floor of the products
    if (res < 0.9 * best) {
      best = res;
      since_best = 0;
    } else {
      ++since_best;
    }
    const bool floor = p.prec != XLBOMD_FP64 && since_best >= 4 && res < 100.0 * p.scf_tol;
    if (floor && debug_enabled()) std::fprintf(stderr, "[xlbomd] scf stops at the rounding floor %.3e\n", res);
    if (res < p.scf_tol || floor) {
      CK(launch_fill_history(st, S.nat, p.kmax, S.nh));
      CK(launch_forces(st, model_of(p), S.nat, S.L, S.eta, S.ng, S.G4, S.R, S.Dm, S.np, S.q, S.nh, S.F, S.work,
                       p.prec != XLBOMD_FP64));
      S.have_K = false;   // exact or accumulated kernel: start again at the t0 state
      return kernel_update(ctx, S);
    }
    if (p.scf_mode == 1 && p.rank_m > 0) {
      CKS(kernel_update(ctx, S));                      // n <- n - K_m r (Eq. SCF_K)
      CK(launch_axpy(st, S.nat, -1.0, S.Kr, S.nh));
    } else {
      CK(launch_axpy(st, S.nat, p.mix_alpha, S.r, S.nh));
    }
  }
  return fail(ctx, XLBOMD_ERR_NOT_CONVERGED, "t0 SCF did not converge");
}

xlbomd_status md_step(xlbomd_ctx* ctx, Sys& S, bool do_energy) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  const double minv = kAcc / S.mass;
  CK(launch_verlet_first(st, S.nat, S.L, p.dt, minv, S.R, S.V, S.F, S.nh, p.kmax, S.Kr, p.kappa, p.alpha,
                         ctx->cdev));
  CKS(build_H(ctx, S));
  CKS(density(ctx, S, true));
  ++S.md_steps;
  if (p.kernel_mode == 1 && p.kernel_every > 0 && S.md_steps % p.kernel_every == 0) S.have_K = false;
  CKS(kernel_update(ctx, S));
  CK(launch_verlet_second(st, S.nat, p.dt, minv, S.V, S.F));
  CK(launch_absmax(st, S.nat, S.r, S.scal + 9));
  if (do_energy) CKS(energy(ctx, S));
  CKS(sync_read(ctx, S.scal + 9, 1));
  if (!(ctx->pinned[0] <= p.diverge_tol)) return fail(ctx, XLBOMD_ERR_DIVERGED, "residual |q - n| too large");
  S.stats[4] += 1;
  return XLBOMD_OK;
}

// The responses w_j = d q/d lambda along v_j of several systems of one padded size, their
// chains as one grouped launch per product (v, w: one device vector per system).
xlbomd_status response_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G, const std::vector<const double*>& v,
                             const std::vector<double*>& w) {
  cudaStream_t st = ctx->stream;
  const double sc = beta_of(ctx->p) / std::ldexp(1.0, ctx->p.n_sq + 1);
  std::vector<ChainJob> cj;
  for (size_t k = 0; k < G.size(); ++k) {
    Sys& S = *G[k];
    CK(gamma_apply(ctx, S, v[k], S.potv, S.work));
    CK(launch_expand_potential(st, S.nat, S.np, -sc, S.potv, S.dvec));
    ChainJob c;
    c.m = &S.mats;
    c.dvec = S.dvec;
    c.N = S.N;
    c.out_diag = S.d1;
    c.stats = S.stats;
    cj.push_back(c);
  }
  CK(ctx->eng->chain_group(st, cj, false));
  for (size_t k = 0; k < G.size(); ++k) {
    Sys& S = *G[k];
    CK(launch_response_finish(st, S.nat, S.N, S.d1, S.dmu_diag, S.scal + 4, w[k]));
  }
  return XLBOMD_OK;
}

// Rank-m kernel update (kernel_mode 0) of several systems of one padded size in lockstep: probe
// i of every system still probing runs as one grouped response chain, with one host
// synchronisation per probe index for all of them.  Each system takes exactly the probes of
// kernel_update().  Other kernel modes update one system after another.
xlbomd_status kernel_update_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  if (p.kernel_mode != 0) {
    for (Sys* S : G) CKS(kernel_update(ctx, *S));
    return XLBOMD_OK;
  }
  const size_t B = G.size();
  double* h = ctx->pinned_group;
  std::vector<int> m(B, 0);
  std::vector<size_t> active(B);
  for (size_t i = 0; i < B; ++i) active[i] = i;
  for (int i = 0; i < p.rank_m && !active.empty(); ++i) {
    for (size_t k = 0; k < active.size(); ++k) {
      Sys& S = *G[active[k]];
      CK(launch_kernel_vec(st, 0, S.nat, i, S.kc, S.r, S.pV, S.pW, nullptr, S.scal + 8));
      CK(cudaMemcpyAsync(h + k, S.scal + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    std::vector<size_t> probing;
    for (size_t k = 0; k < active.size(); ++k)
      if (h[k] == 1.0) probing.push_back(active[k]);
    std::vector<Sys*> g;
    std::vector<const double*> dv;
    std::vector<double*> dw;
    for (size_t j : probing) {
      Sys& S = *G[j];
      g.push_back(&S);
      dv.push_back(S.pV + (size_t)i * S.nat);
      dw.push_back(S.pW + (size_t)i * S.nat);
      m[j] = i + 1;
    }
    if (!g.empty()) CKS(response_group(ctx, g, dv, dw));
    active.swap(probing);
  }
  for (size_t j = 0; j < B; ++j) {
    Sys& S = *G[j];
    CK(launch_kernel_vec(st, 1, S.nat, m[j], S.kc, S.r, S.pV, S.pW, S.Kr, S.scal + 8));
    S.probes_used = m[j];
    S.stats[2] = m[j];
  }
  return XLBOMD_OK;
}

// stiffest_mode() of several systems in lockstep (one grouped response per power iteration)
xlbomd_status stiffest_mode_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G) {
  cudaStream_t st = ctx->stream;
  const size_t B = G.size();
  std::vector<std::vector<double>> v(B), w(B);
  std::vector<double> lam(B, 0.0);
  std::vector<size_t> active;
  for (size_t k = 0; k < B; ++k) {
    Sys& S = *G[k];
    v[k].resize(S.nat);
    w[k].resize(S.nat);
    for (int I = 0; I < S.nat; ++I) v[k][I] = ((I * 7919) % 17) - 8.0;
    double mean = 0.0;
    for (double x : v[k]) mean += x;
    mean /= S.nat;
    double nv = 0.0;
    for (double& x : v[k]) {
      x -= mean;
      nv += x * x;
    }
    nv = std::sqrt(nv);
    if (nv == 0.0) continue;
    for (double& x : v[k]) x /= nv;
    active.push_back(k);
  }
  for (int it = 0; it < 12 && !active.empty(); ++it) {
    std::vector<Sys*> g;
    std::vector<const double*> dv;
    std::vector<double*> dw;
    for (size_t k : active) {
      Sys& S = *G[k];
      double* pv = S.pV + (size_t)kMaxRank * S.nat;   // spare probe rows
      double* pw = S.pW + (size_t)kMaxRank * S.nat;
      CK(cudaMemcpyAsync(pv, v[k].data(), sizeof(double) * S.nat, cudaMemcpyHostToDevice, st));
      g.push_back(&S);
      dv.push_back(pv);
      dw.push_back(pw);
    }
    CKS(response_group(ctx, g, dv, dw));
    for (size_t j = 0; j < active.size(); ++j)
      CK(cudaMemcpyAsync(w[active[j]].data(), dw[j], sizeof(double) * g[j]->nat, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<size_t> next;
    for (size_t k : active) {
      const int nat = G[k]->nat;
      double dot = 0.0, nw = 0.0;
      for (int I = 0; I < nat; ++I) {
        dot += v[k][I] * w[k][I];
        nw += w[k][I] * w[k][I];
      }
      nw = std::sqrt(nw);
      lam[k] = dot;
      if (!(nw > 0.0) || !std::isfinite(nw)) continue;
      for (int I = 0; I < nat; ++I) v[k][I] = w[k][I] / nw;
      next.push_back(k);
    }
    active.swap(next);
  }
  for (size_t k = 0; k < B; ++k) {
    if (lam[k] < 0.0) G[k]->kc = 1.2 * lam[k];
    if (debug_enabled()) std::fprintf(stderr, "[xlbomd] stiffest mode %.4f -> c = %.4f\n", lam[k], G[k]->kc);
  }
  return XLBOMD_OK;
}

// t0 SCF of several systems of one padded size in lockstep: each takes exactly the iterations
// of scf(), with the densities, the stiffest-mode search and the kernel updates grouped.
xlbomd_status scf_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  const size_t B = G.size();
  std::vector<double> best(B, HUGE_VAL);
  std::vector<int> since_best(B, 0);
  std::vector<size_t> active(B);
  for (size_t k = 0; k < B; ++k) active[k] = k;
  double* h = ctx->pinned_group;
  for (int it = 0; it < p.scf_max_iter && !active.empty(); ++it) {
    std::vector<Sys*> g;
    for (size_t k : active) {
      Sys& S = *G[k];
      CK(gamma_apply(ctx, S, S.nh, S.pot, S.work));
      CK(launch_apply_potential(st, S.nat, S.np, S.H0, S.pot, S.H));
      g.push_back(&S);
    }
    CKS(density_group(ctx, g, false));
    if (it == 0 && p.kernel_auto) CKS(stiffest_mode_group(ctx, g));
    for (size_t j = 0; j < g.size(); ++j) {
      CK(launch_absmax(st, g[j]->nat, g[j]->r, g[j]->scal + 9));
      CK(cudaMemcpyAsync(h + j, g[j]->scal + 9, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    std::vector<size_t> next;
    std::vector<Sys*> converged, going;
    for (size_t j = 0; j < g.size(); ++j) {
      const size_t k = active[j];
      Sys& S = *G[k];
      const double res = h[j];
      if (debug_enabled()) std::fprintf(stderr, "[xlbomd] scf it %d system %zu max|q - n| %.3e mu %.8f\n", it, k, res, S.mu);
      if (!std::isfinite(res) || res > 1e3) return fail(ctx, XLBOMD_ERR_DIVERGED, "t0 SCF diverged");
      if (res < 0.9 * best[k]) {
        best[k] = res;
        since_best[k] = 0;
      } else {
        ++since_best[k];
      }
      const bool floor = p.prec != XLBOMD_FP64 && since_best[k] >= 4 && res < 100.0 * p.scf_tol;
      if (res < p.scf_tol || floor) {
        CK(launch_fill_history(st, S.nat, p.kmax, S.nh));
        CK(launch_forces(st, model_of(p), S.nat, S.L, S.eta, S.ng, S.G4, S.R, S.Dm, S.np, S.q, S.nh, S.F, S.work,
                         p.prec != XLBOMD_FP64));
        S.have_K = false;   // exact or accumulated kernel: start again at the t0 state
        converged.push_back(&S);
      } else {
        going.push_back(&S);
        next.push_back(k);
      }
    }
    if (!converged.empty()) CKS(kernel_update_group(ctx, converged));
    if (!going.empty()) {
      if (p.scf_mode == 1 && p.rank_m > 0) {
        CKS(kernel_update_group(ctx, going));            // n <- n - K_m r (Eq. SCF_K)
        for (Sys* S : going) CK(launch_axpy(st, S->nat, -1.0, S->Kr, S->nh));
      } else {
        for (Sys* S : going) CK(launch_axpy(st, S->nat, p.mix_alpha, S->r, S->nh));
      }
    }
    active.swap(next);
  }
  if (!active.empty()) return fail(ctx, XLBOMD_ERR_NOT_CONVERGED, "t0 SCF did not converge");
  return XLBOMD_OK;
}

// One MD step of several systems of one padded size in lockstep (md_step of each, with the
// expansion, mu passes and probe chains grouped).
xlbomd_status md_step_group(xlbomd_ctx* ctx, const std::vector<Sys*>& G) {
  cudaStream_t st = ctx->stream;
  const xlbomd_params& p = ctx->p;
  for (Sys* S : G) {
    CK(launch_verlet_first(st, S->nat, S->L, p.dt, kAcc / S->mass, S->R, S->V, S->F, S->nh, p.kmax, S->Kr, p.kappa,
                           p.alpha, ctx->cdev));
    CKS(build_H(ctx, *S));
  }
  CKS(density_group(ctx, G, true));
  for (Sys* S : G) {
    ++S->md_steps;
    if (p.kernel_mode == 1 && p.kernel_every > 0 && S->md_steps % p.kernel_every == 0) S->have_K = false;
  }
  CKS(kernel_update_group(ctx, G));
  double* h = ctx->pinned_group;
  for (size_t k = 0; k < G.size(); ++k) {
    Sys& S = *G[k];
    CK(launch_verlet_second(st, S.nat, p.dt, kAcc / S.mass, S.V, S.F));
    CK(launch_absmax(st, S.nat, S.r, S.scal + 9));
    const bool e = p.energy_every > 0 && ((int)S.stats[4] + 1) % p.energy_every == 0;
    if (e) CKS(energy(ctx, S));
    CK(cudaMemcpyAsync(h + k, S.scal + 9, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  for (size_t k = 0; k < G.size(); ++k) {
    if (!(h[k] <= p.diverge_tol)) return fail(ctx, XLBOMD_ERR_DIVERGED, "residual |q - n| too large");
    G[k]->stats[4] += 1;
  }
  return XLBOMD_OK;
}

void free_sys(Sys& S) {
  double** ptrs[] = {&S.R,  &S.V,        &S.F,    &S.Z,  &S.nh,  &S.q,    &S.r,     &S.Kr,    &S.pot,
                     &S.potv, &S.gam,    &S.SF,   &S.G4, &S.H0,  &S.H,    &S.Dm,    &S.ddiag, &S.dmu_diag,
                     &S.d1, &S.dvec,     &S.dvec_mu, &S.pV, &S.pW, &S.scal, &S.work, &S.energy,
                     &S.Kfull, &S.Jm, &S.dpar};
  for (double** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  for (auto& g : S.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  S.graphs.clear();
  for (MatSet& m : S.slots) free_chain_slot(m);
  S.slots.clear();
  if (S.slot_vec) cudaFree(S.slot_vec);
  S.slot_vec = nullptr;
  free_matset(S.mats);
}

}  // namespace

// ---- one-probe response whose work memory is a static device array ----
//
// For callers that may not allocate device memory at run time.  The chain's
// work matrices and vectors live in this file-scope array, which every GPU
// that loads the library holds until the process exits.  Its size bounds the
// system: padded orbital count <= kStaticMaxNp.
namespace {
constexpr int kStaticMaxNp = 256;
constexpr size_t kStaticMat = (size_t)kStaticMaxNp * kStaticMaxNp;
constexpr int kStaticSf = 4096;   // structure-factor work vector (reciprocal vectors x 2)
constexpr size_t kStaticDoubles = 5 * kStaticMat + 3 * kStaticMaxNp + 64 + kStaticSf;
}  // namespace

static __device__ __align__(256) double g_response_scratch[kStaticDoubles];

namespace {

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_response_scratch on the current device (looked up once
// per device; in host code the symbol itself is only a host-side stand-in).
xlbomd_status static_scratch(xlbomd_ctx* ctx, double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, XLBOMD_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_response_scratch);
    if (e != cudaSuccess || !p)
      return fail(ctx, XLBOMD_ERR_CUDA, std::string("cudaGetSymbolAddress(g_response_scratch): ") +
                                            cudaGetErrorString(e));
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return XLBOMD_OK;
}

}  // namespace

extern "C" {

xlbomd_status xlbomd_response_noalloc(xlbomd_ctx* ctx, int sys, const double* v_dev, double* w_dev) {
  CKS(check(ctx, sys));
  if (!v_dev || !w_dev) return fail(ctx, XLBOMD_ERR_ARG, "null probe pointer");
  if (ctx->p.prec != XLBOMD_FP64)
    return fail(ctx, XLBOMD_ERR_UNSUPPORTED, "xlbomd_response_noalloc serves FP64 contexts only");
  Sys& S = ctx->sys[sys];
  if (S.np > kStaticMaxNp)
    return fail(ctx, XLBOMD_ERR_ARG,
                "xlbomd_response_noalloc: padded orbital count " + std::to_string(S.np) +
                    " exceeds the static work-array limit of " + std::to_string(kStaticMaxNp) +
                    " (64 atoms); use xlbomd_response");
  if (!S.have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  if (S.kp > kStaticSf) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_response_noalloc: too many reciprocal vectors");
  // every argument check is above: nothing is enqueued on the shared array before the call is accepted
  double* base = nullptr;
  CKS(static_scratch(ctx, &base));
  cudaStream_t st = ctx->stream;
  const double sc = beta_of(ctx->p) / std::ldexp(1.0, ctx->p.n_sq + 1);
  const size_t mat = (size_t)S.np * S.np;
  MatSet m = S.mats;   // shallow view: expansion matrices of the context, work matrices in the array
  m.G = base;
  m.A1 = base + mat;
  m.Mt = base + 2 * mat;
  m.T1a = base + 3 * mat;
  m.T1b = base + 4 * mat;
  m.Tmu = nullptr;
  double* potv = base + 5 * kStaticMat;
  double* dvec = potv + kStaticMaxNp;
  double* d1 = dvec + kStaticMaxNp;
  double* scal = d1 + kStaticMaxNp;
  // the array keeps the previous call's contents: the diagonal accumulator starts at zero
  CK(cudaMemsetAsync(d1, 0, sizeof(double) * kStaticMaxNp, st));
  CK(gamma_apply(ctx, S, v_dev, potv, scal + 64));
  CK(launch_expand_potential(st, S.nat, S.np, -sc, potv, dvec));
  const bool prof = ctx->eng->prof;
  ctx->eng->prof = false;   // event timing would create CUDA events
  const cudaError_t ce = ctx->eng->chain(st, m, dvec, S.N, false, d1, S.stats);   // counted in XLBOMD_STATS
  ctx->eng->prof = prof;
  CK(ce);
  CK(launch_response_finish(st, S.nat, S.N, d1, S.dmu_diag, scal, w_dev));
  return XLBOMD_OK;
}

void xlbomd_default_params(xlbomd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps_s = -8.0;
  p->eps_p = -3.0;
  p->t0[0] = -2.5;
  p->t0[1] = -1.8;
  p->t0[2] = 1.2;
  p->t0[3] = -0.6;
  p->r_decay = 1.2;
  p->r_cut = 5.0;
  p->r_taper = 4.5;
  p->hubbard_U = 6.0;
  p->coulomb_k = 14.399645;
  p->Te = 1000.0;
  p->n_sq = 10;
  p->dt = 0.25;
  p->kappa = 1.82;
  p->alpha = 0.018;
  const double c5[6] = {-6, 14, -8, -3, 4, -1};
  for (int k = 0; k < 6; ++k) p->c[k] = c5[k];
  p->kmax = 5;
  p->rank_m = 2;
  p->mix_alpha = 0.06;
  p->kernel_c = 1.0 - 1.0 / 0.06;
  p->scf_tol = 1e-10;
  p->scf_max_iter = 2000;
  p->mu_tol = 1e-9;
  p->mu_max_iter = 60;
  p->diverge_tol = 1.0;
  p->prec = XLBOMD_FP64;
  p->energy_every = 0;
  p->scf_mode = 0;
  p->kernel_auto = 0;
  p->kernel_mode = 0;
  p->kernel_every = 0;
  p->rep_A = 0.0;
  p->rep_rho = 0.3;
  p->kernel_prec = 0;
  p->graphs = 0;
  p->mu_prec = 0;
}

xlbomd_status xlbomd_table_i(xlbomd_params* p, int kmax) {
  // Table I: kappa, alpha, c_0..c_kmax
  static const double kappa[3] = {1.82, 1.84, 1.86}, alpha[3] = {0.018, 0.0055, 0.0016};
  static const double c[3][8] = {{-6, 14, -8, -3, 4, -1, 0, 0},
                                 {-14, 36, -27, -2, 12, -6, 1, 0},
                                 {-36, 99, -88, 11, 32, -25, 8, -1}};
  if (!p || kmax < 5 || kmax > 7) return XLBOMD_ERR_ARG;
  const int r = kmax - 5;
  p->kmax = kmax;
  p->kappa = kappa[r];
  p->alpha = alpha[r];
  for (int k = 0; k < 8; ++k) p->c[k] = c[r][k];
  return XLBOMD_OK;
}

xlbomd_status xlbomd_init(const xlbomd_params* params, const xlbomd_system* systems, int nsys, void* cuda_stream,
                          xlbomd_ctx** out) {
  if (!params || !systems || !out || nsys < 1) return XLBOMD_ERR_ARG;
  *out = nullptr;
  const xlbomd_params& p = *params;
  if (p.n_sq < 1 || p.n_sq > 40 || p.kmax < 1 || p.kmax > 7 || p.rank_m < 0 || p.rank_m > kMaxRank ||
      p.kernel_c == 1.0 || !(p.Te > 0) || !(p.dt > 0) || p.mu_max_iter < 1 || p.scf_mode < 0 || p.scf_mode > 1 ||
      p.kernel_mode < 0 || p.kernel_mode > 2 || p.kernel_every < 0 || p.rep_A < 0.0 || !(p.rep_rho > 0.0) ||
      p.kernel_prec < 0 || p.kernel_prec > 1 || p.graphs < 0 || p.graphs > 1 || p.mu_prec < 0 || p.mu_prec > 1)
    return XLBOMD_ERR_ARG;
  if (p.prec != XLBOMD_FP64 && p.prec != XLBOMD_FP16x3 && p.prec != XLBOMD_BF16x3 &&
      p.prec != XLBOMD_TF32x3)
    return XLBOMD_ERR_ARG;
  for (int i = 0; i < nsys; ++i) {
    const xlbomd_system& s = systems[i];
    if (s.natoms < 1 || !(s.box_L > p.r_cut) || !s.R || !s.V || !s.Z || !(s.mass > 0)) return XLBOMD_ERR_ARG;
  }
  xlbomd_ctx* ctx = new xlbomd_ctx();
  ctx->p = p;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->eng = make_engine(p.prec);
  if (!ctx->eng) {
    delete ctx;
    return XLBOMD_ERR_UNSUPPORTED;
  }
  ctx->eng->set_chain_segments(p.kernel_prec == 1 ? 1 : 3, p.mu_prec == 1 ? 1 : 3);
  auto bail = [&](xlbomd_status st) {
    xlbomd_free(ctx);
    return st;
  };
  if (cudaMallocHost((void**)&ctx->pinned, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->ppar, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->pinned_group, 2 * (size_t)nsys * sizeof(double)) != cudaSuccess)
    return bail(XLBOMD_ERR_OOM);
  if (dalloc(ctx, &ctx->cdev, 8) != XLBOMD_OK) return bail(XLBOMD_ERR_OOM);
  // every upload and memset below runs on the context's stream, which may be non-blocking
  if (cudaMemcpyAsync(ctx->cdev, p.c, sizeof(double) * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return bail(XLBOMD_ERR_CUDA);
  ctx->sys.resize(nsys);
  const double sc = beta_of(p) / std::ldexp(1.0, p.n_sq + 1);
  for (int i = 0; i < nsys; ++i) {
    const xlbomd_system& s = systems[i];
    Sys& S = ctx->sys[i];
    S.nat = s.natoms;
    S.N = 4 * s.natoms;
    S.np = (S.N + 127) / 128 * 128;
    S.natp = (S.nat + 63) / 64 * 64;
    S.L = s.box_L;
    S.mass = s.mass;
    S.kc = p.kernel_c;
    double zs = 0;
    for (int a = 0; a < S.nat; ++a) zs += s.Z[a];
    S.nocc = 0.5 * zs;
    ewald_vectors(S.L, S.eta, S.G4h);
    S.ng = (int)(S.G4h.size() / 4);
    S.kp = (2 * S.ng + 15) / 16 * 16;
    const size_t nat = S.nat, np2 = (size_t)S.np * S.np;
    xlbomd_status st = XLBOMD_OK;
    auto A = [&](double** ptr, size_t cnt) {
      if (st == XLBOMD_OK) st = dalloc(ctx, ptr, cnt);
    };
    A(&S.R, 3 * nat);
    A(&S.V, 3 * nat);
    A(&S.F, 3 * nat);
    A(&S.Z, nat);
    A(&S.nh, (size_t)(p.kmax + 1) * nat);
    A(&S.q, nat);
    A(&S.r, nat);
    A(&S.Kr, nat);
    A(&S.pot, nat);
    A(&S.potv, nat);
    A(&S.gam, (size_t)S.natp * S.natp);
    A(&S.SF, (size_t)S.natp * S.kp);
    A(&S.G4, std::max<size_t>(S.G4h.size(), 4));
    A(&S.H0, np2);
    A(&S.H, np2);
    A(&S.Dm, np2);
    A(&S.ddiag, S.np);
    A(&S.dmu_diag, S.np);
    A(&S.d1, S.np);
    A(&S.dvec, S.np);
    A(&S.dvec_mu, S.np);
    A(&S.pV, (size_t)(kMaxRank + 1) * nat);
    A(&S.pW, (size_t)(kMaxRank + 1) * nat);
    A(&S.scal, 64);
    A(&S.work, std::max<size_t>({(size_t)4 * S.ng + 16, (size_t)2 * S.N + 16, (size_t)4096}));
    A(&S.energy, 8);
    if (st != XLBOMD_OK) return bail(st);
    if (alloc_matset(S.mats, p.prec, S.np, p.n_sq, ctx->stream) != cudaSuccess) return bail(XLBOMD_ERR_OOM);
    // R wrapped into [0, L)
    std::vector<double> Rw(3 * nat);
    for (size_t a = 0; a < 3 * nat; ++a) Rw[a] = s.R[a] - S.L * std::floor(s.R[a] / S.L);
    std::vector<double> dmu(S.np, 0.0);
    for (int a = 0; a < S.N; ++a) dmu[a] = sc;
    const cudaStream_t cs = ctx->stream;
    if (cudaMemcpyAsync(S.R, Rw.data(), sizeof(double) * 3 * nat, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(S.V, s.V, sizeof(double) * 3 * nat, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(S.Z, s.Z, sizeof(double) * nat, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        (S.ng && cudaMemcpyAsync(S.G4, S.G4h.data(), sizeof(double) * S.G4h.size(), cudaMemcpyHostToDevice, cs) !=
                     cudaSuccess) ||
        cudaMemcpyAsync(S.dvec_mu, dmu.data(), sizeof(double) * S.np, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)   // Rw and dmu are host temporaries
      return bail(XLBOMD_ERR_CUDA);
    if (build_H(ctx, S) != XLBOMD_OK) return bail((xlbomd_status)ctx->status);
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bail(XLBOMD_ERR_CUDA);
  *out = ctx;
  return XLBOMD_OK;
}

xlbomd_status xlbomd_scf(xlbomd_ctx* ctx, int sys) {
  if (!ctx) return XLBOMD_ERR_ARG;
  const int lo = sys < 0 ? 0 : sys, hi = sys < 0 ? (int)ctx->sys.size() : sys + 1;
  for (int i = lo; i < hi; ++i) CKS(check(ctx, i));
  if (hi - lo == 1) return scf(ctx, ctx->sys[lo]);
  // every system: those of one padded size in lockstep
  std::vector<int> sizes;
  for (const Sys& S : ctx->sys)
    if (std::find(sizes.begin(), sizes.end(), S.np) == sizes.end()) sizes.push_back(S.np);
  for (int np : sizes) {
    std::vector<Sys*> G;
    for (Sys& S : ctx->sys)
      if (S.np == np) G.push_back(&S);
    if (G.size() == 1)
      CKS(scf(ctx, *G[0]));
    else
      CKS(scf_group(ctx, G));
  }
  return XLBOMD_OK;
}

xlbomd_status xlbomd_build_H(xlbomd_ctx* ctx, int sys) {
  CKS(check(ctx, sys));
  return build_H(ctx, ctx->sys[sys]);
}

xlbomd_status xlbomd_density(xlbomd_ctx* ctx, int sys) {
  CKS(check(ctx, sys));
  return density(ctx, ctx->sys[sys], true);
}

xlbomd_status xlbomd_kernel_exact(xlbomd_ctx* ctx, int sys) {
  CKS(check(ctx, sys));
  return kernel_exact(ctx, ctx->sys[sys]);
}

xlbomd_status xlbomd_response(xlbomd_ctx* ctx, int sys, const double* v_dev, double* w_dev) {
  CKS(check(ctx, sys));
  if (!v_dev || !w_dev) return fail(ctx, XLBOMD_ERR_ARG, "null probe pointer");
  if (!ctx->sys[sys].have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  return response(ctx, ctx->sys[sys], v_dev, w_dev);
}

xlbomd_status xlbomd_kernel_update(xlbomd_ctx* ctx, int sys) {
  CKS(check(ctx, sys));
  if (!ctx->sys[sys].have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  return kernel_update(ctx, ctx->sys[sys]);
}

xlbomd_status xlbomd_energy(xlbomd_ctx* ctx, int sys) {
  CKS(check(ctx, sys));
  if (!ctx->sys[sys].have_density) return fail(ctx, XLBOMD_ERR_ARG, "xlbomd_density must run first");
  return energy(ctx, ctx->sys[sys]);
}

xlbomd_status xlbomd_step(xlbomd_ctx* ctx, int nsteps) {
  if (!ctx || nsteps < 0) return XLBOMD_ERR_ARG;
  for (int i = 0; i < (int)ctx->sys.size(); ++i) CKS(check(ctx, i));
  // systems of one padded size advance in lockstep (grouped launches); a size held by one
  // system takes the one-system step
  std::vector<int> sizes;
  for (const Sys& S : ctx->sys)
    if (std::find(sizes.begin(), sizes.end(), S.np) == sizes.end()) sizes.push_back(S.np);
  for (int t = 0; t < nsteps; ++t)
    for (int np : sizes) {
      std::vector<Sys*> G;
      for (Sys& S : ctx->sys)
        if (S.np == np) G.push_back(&S);
      if (G.size() == 1) {
        Sys& S = *G[0];
        const bool e = ctx->p.energy_every > 0 && ((int)S.stats[4] + 1) % ctx->p.energy_every == 0;
        CKS(md_step(ctx, S, e));
      } else {
        CKS(md_step_group(ctx, G));
      }
    }
  return XLBOMD_OK;
}

xlbomd_status xlbomd_get(xlbomd_ctx* ctx, int sys, int what, double* host_out) {
  CKS(check(ctx, sys));
  if (!host_out) return fail(ctx, XLBOMD_ERR_ARG, "null output");
  Sys& S = ctx->sys[sys];
  const size_t nat = S.nat;
  auto cp = [&](const double* d, size_t cnt) -> xlbomd_status {
    CK(cudaMemcpyAsync(host_out, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return XLBOMD_OK;
  };
  auto cp2d = [&](const double* d, int rows, int ld) -> xlbomd_status {
    CK(cudaMemcpy2DAsync(host_out, sizeof(double) * rows, d, sizeof(double) * ld, sizeof(double) * rows, rows,
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return XLBOMD_OK;
  };
  switch (what) {
    case XLBOMD_Q: return cp(S.q, nat);
    case XLBOMD_N: return cp(S.nh, nat);
    case XLBOMD_NHIST: return cp(S.nh, (size_t)(ctx->p.kmax + 1) * nat);
    case XLBOMD_F: return cp(S.F, 3 * nat);
    case XLBOMD_R: return cp(S.R, 3 * nat);
    case XLBOMD_V: return cp(S.V, 3 * nat);
    case XLBOMD_KR: return cp(S.Kr, nat);
    case XLBOMD_RES: return cp(S.r, nat);
    case XLBOMD_ENERGY: std::memcpy(host_out, S.eh, 7 * sizeof(double)); return XLBOMD_OK;
    case XLBOMD_MU: host_out[0] = S.mu; return XLBOMD_OK;
    case XLBOMD_D: return cp2d(S.Dm, S.N, S.np);
    case XLBOMD_H: return cp2d(S.H, S.N, S.np);
    case XLBOMD_GAMMA: {
      // gamma_real + k SF SF^T, formed on demand
      double* full = nullptr;
      if (cudaMalloc((void**)&full, sizeof(double) * (size_t)S.natp * S.natp) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, XLBOMD_ERR_OOM, "cudaMalloc failed");
      }
      EpiF64 e;
      e.alpha = ctx->p.coulomb_k;
      e.E = S.gam;
      e.lde = S.natp;
      e.beta = 1.0;
      cudaError_t ce = gemm_f64_nt(ctx->stream, S.natp, S.natp, S.kp, S.SF, S.kp, S.SF, S.kp, full, S.natp, e, false);
      xlbomd_status rs = ce == cudaSuccess ? cp2d(full, S.nat, S.natp) : fail(ctx, XLBOMD_ERR_CUDA, "gamma product");
      cudaFree(full);
      return rs;
    }
    case XLBOMD_STATS: std::memcpy(host_out, S.stats, 5 * sizeof(double)); return XLBOMD_OK;
    case XLBOMD_KMAT:
      if (!S.have_K) return fail(ctx, XLBOMD_ERR_ARG, "no exact kernel held (xlbomd_kernel_exact)");
      return cp(S.Kfull, nat * nat);
    case XLBOMD_PROBES: {
      CK(cudaMemcpyAsync(host_out, S.pV, sizeof(double) * ctx->p.rank_m * nat, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(host_out + ctx->p.rank_m * nat, S.pW, sizeof(double) * ctx->p.rank_m * nat,
                         cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      return XLBOMD_OK;
    }
    default: return fail(ctx, XLBOMD_ERR_ARG, "unknown quantity");
  }
}

xlbomd_status xlbomd_set(xlbomd_ctx* ctx, int sys, int what, const double* host_in) {
  CKS(check(ctx, sys));
  if (!host_in) return fail(ctx, XLBOMD_ERR_ARG, "null input");
  Sys& S = ctx->sys[sys];
  const size_t nat = S.nat;
  switch (what) {
    case XLBOMD_R: {
      std::vector<double> Rw(3 * nat);
      for (size_t a = 0; a < 3 * nat; ++a) Rw[a] = host_in[a] - S.L * std::floor(host_in[a] / S.L);
      CK(cudaMemcpyAsync(S.R, Rw.data(), sizeof(double) * 3 * nat, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      S.have_density = false;
      return XLBOMD_OK;
    }
    case XLBOMD_V:
      CK(cudaMemcpyAsync(S.V, host_in, sizeof(double) * 3 * nat, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      return XLBOMD_OK;
    case XLBOMD_N:
      for (int k = 0; k <= ctx->p.kmax; ++k)
        CK(cudaMemcpyAsync(S.nh + k * nat, host_in, sizeof(double) * nat, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      S.have_density = false;
      return XLBOMD_OK;
    case XLBOMD_NHIST:
      CK(cudaMemcpyAsync(S.nh, host_in, sizeof(double) * (ctx->p.kmax + 1) * nat, cudaMemcpyHostToDevice,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      S.have_density = false;
      return XLBOMD_OK;
    case XLBOMD_MU:
      S.mu = host_in[0];
      S.mu_valid = true;
      S.n_mu_hist = 0;
      return XLBOMD_OK;
    default: return fail(ctx, XLBOMD_ERR_ARG, "quantity cannot be set");
  }
}

xlbomd_status xlbomd_sizes(xlbomd_ctx* ctx, int sys, int* natoms, int* n_orb, int* n_pad) {
  if (!ctx || sys < 0 || sys >= (int)ctx->sys.size()) return XLBOMD_ERR_ARG;
  if (natoms) *natoms = ctx->sys[sys].nat;
  if (n_orb) *n_orb = ctx->sys[sys].N;
  if (n_pad) *n_pad = ctx->sys[sys].np;
  return XLBOMD_OK;
}

xlbomd_status xlbomd_clear_error(xlbomd_ctx* ctx) {
  if (!ctx) return XLBOMD_ERR_ARG;
  ctx->status = XLBOMD_OK;
  ctx->msg.clear();
  cudaGetLastError();
  return XLBOMD_OK;
}

const char* xlbomd_last_error(xlbomd_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->msg.c_str();
}

long long xlbomd_launch_count(void) { return g_launch_count.load(); }

xlbomd_status xlbomd_gemm_profile(xlbomd_ctx* ctx, int mode, double* out) {
  if (!ctx) return XLBOMD_ERR_ARG;
  Engine& E = *ctx->eng;
  if (mode == 0) {
    E.prof = false;
  } else if (mode == 1) {
    E.prof = true;
    E.prof_reset();
  } else if (mode == 2) {
    if (!out) return fail(ctx, XLBOMD_ERR_ARG, "null output");
    CK(E.prof_collect(out));
  } else {
    return fail(ctx, XLBOMD_ERR_ARG, "unknown profile mode");
  }
  return XLBOMD_OK;
}

xlbomd_status xlbomd_selftest_gemm(int n, int prec, int sym, double* result) {
  if (!result || n <= 0 || n % 128 || sym < 0 || sym > 6 || sym == 3) return XLBOMD_ERR_ARG;
  const int rc = selftest_gemm(n, prec, sym, result);
  if (rc == -1) return XLBOMD_ERR_ARG;
  return rc == 0 ? XLBOMD_OK : XLBOMD_ERR_CUDA;
}

xlbomd_status xlbomd_selftest_gemm_group(int n, int prec, int sym, int nprob, double* result) {
  if (!result || n <= 0 || n % 128 || sym < 0 || sym > 6 || sym == 3 || nprob < 2 || nprob > 64)
    return XLBOMD_ERR_ARG;
  const int rc = selftest_gemm_group(n, prec, sym, nprob, result);
  if (rc == -1) return XLBOMD_ERR_ARG;
  return rc == 0 ? XLBOMD_OK : XLBOMD_ERR_CUDA;
}

xlbomd_status xlbomd_free(xlbomd_ctx* ctx) {
  if (!ctx) return XLBOMD_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);   // no work of this context may still use its memory
  for (Sys& S : ctx->sys) free_sys(S);
  if (ctx->cdev) cudaFree(ctx->cdev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->ppar) cudaFreeHost(ctx->ppar);
  if (ctx->pinned_group) cudaFreeHost(ctx->pinned_group);
  delete ctx->eng;
  delete ctx;
  return XLBOMD_OK;
}

}  // extern "C"
