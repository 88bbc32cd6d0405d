// Plain-FP64 engine of the recursive Fermi-operator expansion (tanh-doubling
// form) and of its canonical density-matrix perturbation chains.
//
// Products whose result is symmetric (T^2, the Newton-Schulz update
// (2I - Y B) Y, 2 T Y, Y M for the response) run in symmetric-output mode:
// only upper tiles are computed and mirrored, which halves their cost and
// keeps them exactly symmetric.  Exact symmetry matters: with the A B^T
// product form, an antisymmetric rounding component of Y would be doubled by
// every Newton-Schulz step.
#include <cstdio>

#include "precision.h"

namespace xl {
namespace {

#define RET(x)                            \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

class EngineF64 : public Engine {
 public:
  cudaError_t gemm(cudaStream_t s, int np, const double* A, const double* B, double* C, const EpiF64& e, bool sym,
                   double* stats) {
    if (stats) stats[3] += sym ? 0.5 : 1.0;
    RET(prof_begin(s));
    RET(gemm_f64_nt(s, np, np, np, A, np, B, np, C, np, e, sym));
    return prof_end(s, 2.0 * (double)np * np * np * (sym ? 0.5 : 1.0));
  }

  cudaError_t foe(cudaStream_t s, MatSet& m, const double* H, int N, double mu, double sc,
                  const std::vector<int>& ns, const std::vector<double>& nc, double* stats, const double*) override {
    const int np = m.np, n = m.n;
    RET(launch_t0_init(s, N, np, H, mu, sc, m.T[0]));
    for (int k = 0; k < n; ++k) {
      EpiF64 e1;
      RET(gemm(s, np, m.T[k], m.T[k], m.S, e1, true, stats));              // S = T^2
      if (k == 0)
        RET(launch_ident_minus(s, np, m.S, m.Y[0]));                       // Y = I - S
      else
        RET(launch_scale(s, (size_t)np * np, nc[k], m.Y[k - 1], m.Y[k]));  // Y = c_k Y_{k-1}
      for (int it = 0; it < ns[k]; ++it) {
        EpiF64 eq;                                                         // Q = 2I - Y - Y S = 2I - Y B
        eq.alpha = -1.0;
        eq.E = m.Y[k];
        eq.lde = np;
        eq.beta = -1.0;
        eq.diag = 2.0;
        RET(gemm(s, np, m.Y[k], m.S, m.Q, eq, false, stats));
        EpiF64 ey;
        RET(gemm(s, np, m.Q, m.Y[k], m.Yw, ey, true, stats));              // Y <- Q Y
        std::swap(m.Y[k], m.Yw);
        if (stats) stats[1] += 1;
      }
      EpiF64 et;
      et.alpha = 2.0;
      RET(gemm(s, np, m.T[k], m.Y[k], m.T[k + 1], et, true, stats));       // T_{k+1} = 2 T Y
    }
    return cudaSuccess;
  }

  cudaError_t chain(cudaStream_t s, MatSet& m, const double* dvec, int N, bool full_last, double* out_diag,
                    double* stats) override {
    const int np = m.np, n = m.n;
    double* T1 = m.T1a;
    double* T1n = m.T1b;
    for (int k = 0; k < n; ++k) {
      const bool last = (k == n - 1);
      EpiF64 em;
      em.alpha = -1.0;
      if (k == 0) {
        RET(launch_level0_A1(s, np, m.T[0], dvec, m.A1));      // A1 = T0 D + D T0
        em.dvec = dvec;                                         // Mt = 2 D - T_1 A1
        em.ndvec = np;
        em.dvec_scale = 2.0;
      } else {
        EpiF64 eg;
        RET(gemm(s, np, m.T[k], T1, m.G, eg, false, stats));   // G = T T1
        RET(launch_transpose_add(s, np, m.G, m.A1));           // A1 = G + G^T
        em.E = T1;                                              // Mt = 2 T1 - T_{k+1} A1
        em.lde = np;
        em.beta = 2.0;
      }
      RET(gemm(s, np, m.T[k + 1], m.A1, m.Mt, em, false, stats));
      if (last && !full_last) return launch_row_dot(s, N, np, m.Y[k], m.Mt, out_diag);   // diag(Y M)
      double* dst = (last && full_last) ? m.Tmu : T1n;
      EpiF64 ey;
      RET(gemm(s, np, m.Y[k], m.Mt, dst, ey, true, stats));    // T1' = Y M  (= Y Mt^T)
      if (last) return launch_get_diag(s, N, np, dst, out_diag);
      T1n = T1;
      T1 = dst;
    }
    return cudaSuccess;
  }

  cudaError_t trace_tn(cudaStream_t s, MatSet& m, int N, double* out) override {
    return launch_diag_sum(s, N, m.np, m.T[m.n], out);
  }

  cudaError_t density_out(cudaStream_t s, MatSet& m, int N, double dmu, const double*, double* ddiag,
                          double* D) override {
    return launch_density_out_f64(s, N, m.np, m.T[m.n], m.Tmu, dmu, ddiag, D);
  }

  cudaError_t entropy(cudaStream_t s, MatSet& m, int N, double beta, int n_sq, double mu, double dmu,
                      const double* D, const double* H, double* work, double* out) override {
    return launch_entropy_f64(s, m, N, beta, n_sq, mu, dmu, D, H, work, out);
  }
};

}  // namespace

cudaError_t alloc_matset(MatSet& m, int prec, int np, int n, cudaStream_t s) {
  m.prec = prec;
  m.np = np;
  m.n = n;
  const size_t bytes = sizeof(double) * (size_t)np * np;
  if (prec != 0) return alloc_matset_split(m, s);
  auto A = [&](double** p) -> cudaError_t {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
      *p = nullptr;
      return e;
    }
    return cudaMemsetAsync(*p, 0, bytes, s);
  };
  m.T.assign(n + 1, nullptr);
  m.Y.assign(n, nullptr);
  for (auto& p : m.T) RET(A(&p));
  for (auto& p : m.Y) RET(A(&p));
  double** w[] = {&m.S, &m.Q, &m.Yw, &m.G, &m.A1, &m.Mt, &m.T1a, &m.T1b, &m.Tmu};
  for (double** p : w) RET(A(p));
  return cudaSuccess;
}

void free_matset(MatSet& m) {
  for (auto& p : m.T)
    if (p) cudaFree(p);
  for (auto& p : m.Y)
    if (p) cudaFree(p);
  m.T.clear();
  m.Y.clear();
  double** w[] = {&m.S, &m.Q, &m.Yw, &m.G, &m.A1, &m.Mt, &m.T1a, &m.T1b, &m.Tmu};
  for (double** p : w) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  free_matset_split(m);
}

// Default grouped operations: one system after another.
cudaError_t Engine::foe_group(cudaStream_t s, std::vector<FoeJob>& jobs, double sc) {
  for (auto& j : jobs) RET(foe(s, *j.m, j.H, j.N, j.mu, sc, *j.ns, *j.nc, j.stats, j.dpar));
  return cudaSuccess;
}

cudaError_t Engine::chain_group(cudaStream_t s, std::vector<ChainJob>& jobs, bool full_last) {
  for (auto& j : jobs) RET(chain(s, *j.m, j.dvec, j.N, full_last, j.out_diag, j.stats));
  return cudaSuccess;
}

Engine* make_engine(int prec) {
  if (prec == 0) return new EngineF64();
  return make_split_engine(prec);
}

}  // namespace xl
