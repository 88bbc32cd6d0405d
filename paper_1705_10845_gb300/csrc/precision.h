// Precision engines of the expansion and response chains.
//
// The orchestration (capi.cu) is written once; an Engine runs the matrix
// recursions in one arithmetic: plain FP64 products, or split-precision
// tensor-core products (hi/lo FP16, BF16 or TF32 operands, FP32 accumulation).
#pragma once
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <vector>

#include "internal.h"

namespace xl {

constexpr int XLBOMD_FP16x3_ID = 1;
constexpr int XLBOMD_BF16x3_ID = 2;
constexpr int XLBOMD_TF32x3_ID = 3;

inline bool is_split_prec(int prec) {
  return prec == XLBOMD_FP16x3_ID || prec == XLBOMD_BF16x3_ID || prec == XLBOMD_TF32x3_ID;
}
// product operand format of a split precision (0 FP16, 1 BF16, 2 TF32) and its bytes per element
inline int operand_fmt(int prec) { return prec == XLBOMD_TF32x3_ID ? 2 : prec == XLBOMD_BF16x3_ID ? 1 : 0; }
inline int operand_bytes(int prec) { return prec == XLBOMD_TF32x3_ID ? 4 : 2; }

// Matrices of one system in the working precision.  In the FP64 engine each
// logical matrix is a double array; the split engines keep an FP32 value
// array plus hi/lo operand arrays (16-bit FP16/BF16, or TF32 in FP32 words)
// with a power-of-two scale.
struct SplitMat {
  float2* d = nullptr;       // double-float value hi + lo (matrices carried with an exact leading term)
  float* f = nullptr;        // FP32 value (np x np)
  void* hi = nullptr;        // operand hi part of value * scale
  void* lo = nullptr;        // operand lo part
  float* scale = nullptr;    // device scalar
  unsigned* amax = nullptr;  // device scalar: float bits of max |value|
};

struct MatSet {
  int prec = 0, np = 0, n = 0;
  // FP64 engine
  std::vector<double*> T, Y;
  double *S = nullptr, *Q = nullptr, *Yw = nullptr, *G = nullptr, *A1 = nullptr, *Mt = nullptr;
  double *T1a = nullptr, *T1b = nullptr, *Tmu = nullptr;
  // split engines
  std::vector<SplitMat> sT, sY;
  SplitMat sS, sQ, sYw, sA1, sMt, sT1a, sT1b, sTmu;
  void* tc_plan = nullptr;   // device scalars (scales, max |x|) of the split engine
  double t0max = 0.0;        // spectral bound |T_0| of the last expansion
  // FP64 work matrices of the split engine's entropy (allocated on first use)
  double* e64[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

cudaError_t alloc_matset(MatSet& m, int prec, int np, int n, cudaStream_t s);
void free_matset(MatSet& m);

// One system's part of a grouped expansion or response chain (systems of one size np advanced
// in lockstep; see Engine::foe_group, Engine::chain_group).
struct FoeJob {
  MatSet* m = nullptr;
  const double* H = nullptr;
  int N = 0;
  double mu = 0.0;
  const std::vector<int>* ns = nullptr;
  const std::vector<double>* nc = nullptr;
  double* stats = nullptr;
  const double* dpar = nullptr;
};
struct ChainJob {
  MatSet* m = nullptr;
  const double* dvec = nullptr;
  int N = 0;
  double* out_diag = nullptr;
  double* stats = nullptr;
};

class Engine {
 public:
  virtual ~Engine() {
    for (auto e : ev_) cudaEventDestroy(e);
  }
  // Timing of the matrix products with CUDA events on their stream.
  bool prof = false;
  std::vector<cudaEvent_t> ev_;
  std::vector<double> prof_flops_;
  size_t nprof_ = 0;
  void prof_reset() { nprof_ = 0; }
  cudaError_t prof_begin(cudaStream_t s) {
    if (!prof) return cudaSuccess;
    while (ev_.size() < 2 * (nprof_ + 1)) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev_.push_back(e);
    }
    return cudaEventRecord(ev_[2 * nprof_], s);
  }
  std::vector<int> prof_kind_;
  cudaError_t prof_end(cudaStream_t s, double flops, int kind = 0) {
    if (!prof) return cudaSuccess;
    cudaError_t r = cudaEventRecord(ev_[2 * nprof_ + 1], s);
    if (prof_flops_.size() <= nprof_) prof_flops_.resize(nprof_ + 1);
    if (prof_kind_.size() <= nprof_) prof_kind_.resize(nprof_ + 1);
    prof_kind_[nprof_] = kind;
    prof_flops_[nprof_++] = flops;
    return r;
  }
  // out = [launches, total ms, algorithmic flops]
  cudaError_t prof_collect(double* out) {
    out[0] = (double)nprof_;
    out[1] = 0.0;
    out[2] = 0.0;
    for (size_t i = 0; i < nprof_; ++i) {
      cudaError_t r = cudaEventSynchronize(ev_[2 * i + 1]);
      if (r != cudaSuccess) return r;
      float ms = 0.f;
      r = cudaEventElapsedTime(&ms, ev_[2 * i], ev_[2 * i + 1]);
      if (r != cudaSuccess) return r;
      out[1] += ms;
      out[2] += prof_flops_[i];
      if (i < prof_kind_.size()) {
        const int k = prof_kind_[i] & 63;
        kind_ms_[k] += ms;
        kind_n_[k] += 1;
      }
    }
    const char* e = std::getenv("XLBOMD_DEBUG");
    if (e && e[0] && e[0] != '0')
      for (int k = 0; k < 64; ++k)
        if (kind_n_[k] > 0)
          std::fprintf(stderr, "[xlbomd] product kind %2d: %6d launches, %8.3f ms avg\n", k, kind_n_[k],
                       kind_ms_[k] / kind_n_[k]);
    return cudaSuccess;
  }
  double kind_ms_[64] = {0};
  int kind_n_[64] = {0};
  // T_0 = -sc (H - mu I); n levels T_{k+1} = 2 T_k Y_k, Y_k = (I + T_k^2)^-1 by
  // plan.s[k] Newton-Schulz steps (2I - Y B) Y from Y = I - S (k = 0) or c_k Y_{k-1}.
  // dpar (device, may be null): when set, mu = dpar[0] and the Newton-Schulz start scales
  // c_k = dpar[1 + k] are read on the device instead of the host values mu, nc (so that a
  // captured graph of the expansion can be replayed with new values; split engines only).
  virtual cudaError_t foe(cudaStream_t s, MatSet& m, const double* H, int N, double mu, double sc,
                          const std::vector<int>& ns, const std::vector<double>& nc, double* stats,
                          const double* dpar) = 0;
  // Response chain with diagonal T1_0 = diag(dvec): T1_{k+1} = Y_k (2 T1_k - A1 T_{k+1}),
  // A1 = T_k T1_k + T1_k T_k.  out_diag = diag(T1_n); full_last keeps T1_n in Tmu.
  virtual cudaError_t chain(cudaStream_t s, MatSet& m, const double* dvec, int N, bool full_last,
                            double* out_diag, double* stats) = 0;
  // The same for several systems of one padded size (lockstep: the split engine runs each
  // product over all of them in one grouped launch; the FP64 engine one after another).
  virtual cudaError_t foe_group(cudaStream_t s, std::vector<FoeJob>& jobs, double sc);
  virtual cudaError_t chain_group(cudaStream_t s, std::vector<ChainJob>& jobs, bool full_last);
  // out[0] = sum_{i<N} (T_n)_ii
  // Device flag that the tensor-core product sets when a bounded wait gives up or a
  // tile falls outside the matrix (null: this engine has none).
  virtual const int* device_error() const { return nullptr; }
  // Split engines: tensor products per level of the probe chains and of the mu chain
  // (3, or 1 = hi operands only)
  virtual void set_chain_segments(int, int) {}
  virtual cudaError_t trace_tn(cudaStream_t s, MatSet& m, int N, double* out) = 0;
  // ddiag = 1 + diag(T_n) + dmu dmu_diag (= 2 D_aa);  D = (I + T_n)/2 + dmu Tmu / 2 (FP64)
  virtual cudaError_t density_out(cudaStream_t s, MatSet& m, int N, double dmu, const double* dmu_diag,
                                  double* ddiag, double* D) = 0;
  // out[0] = sum_i s(f_i) (electronic entropy / kB of the occupations of D)
  virtual cudaError_t entropy(cudaStream_t s, MatSet& m, int N, double beta, int n_sq, double mu, double dmu,
                              const double* D, const double* H, double* work, double* out) = 0;
};

Engine* make_engine(int prec);



// split-precision engines (engine_split.cu)
Engine* make_split_engine(int prec);
cudaError_t alloc_matset_split(MatSet& m, cudaStream_t s);
// response-chain slots of a split-precision system (grouped probes of one system)
cudaError_t alloc_chain_slot(MatSet& slot, const MatSet& base, cudaStream_t s);
void free_chain_slot(MatSet& slot);
size_t chain_slot_bytes(int np, int prec);
void free_matset_split(MatSet& m);

// tensor-core product self-test (engine_split.cu)
int selftest_gemm(int n, int prec, int sym, double* result);
int selftest_gemm_group(int n, int prec, int mode, int nprob, double* result);

// FP64 eigenvalue-free entropy (entropy.cu)
cudaError_t entropy_fp64(cudaStream_t s, int N, int np, int n, int n_sq, const double* T0,
                         const std::function<cudaError_t(int, double*)>& load_Y, double* G, double* S, double* Q,
                         double* Yw, double* A1, double* Mt, int nterms, const double* D, double* work,
                         double* out);
cudaError_t launch_entropy_f64(cudaStream_t s, MatSet& m, int N, double beta, int n_sq, double mu, double dmu,
                               const double* D, const double* H, double* work, double* out);

// misc FP64 launchers (foe_kernels.cu)
cudaError_t launch_expand_potential(cudaStream_t s, int nat, int np, double scale, const double* pot, double* dvec);
cudaError_t launch_response_finish(cudaStream_t s, int nat, int N, const double* d1, const double* dmu_diag,
                                   double* scal, double* w);
cudaError_t launch_absmax(cudaStream_t s, int n, const double* x, double* out);
cudaError_t launch_fill_history(cudaStream_t s, int nat, int kmax, double* nh);
cudaError_t launch_axpy(cudaStream_t s, int n, double a, const double* x, double* y);
cudaError_t launch_diag_sum(cudaStream_t s, int n, int np, const double* X, double* out);
// exact kernel (foe_kernels.cu): v = e_i; column col of J - I from w (and of B = I);
// B <- (A)^-1 B by Gauss-Jordan with partial pivoting (A row-major n x n, destroyed;
// f: n doubles of work; *flag set to 1 on a zero or non-finite pivot)
cudaError_t launch_unit_vector(cudaStream_t s, int n, int i, double* v);
cudaError_t launch_jacobian_column(cudaStream_t s, int n, int col, const double* w, double* A, double* B);
cudaError_t launch_gauss_jordan(cudaStream_t s, int n, double* A, double* B, double* f, double* flag);
// accumulated rank-1 kernel (foe_kernels.cu), row-major n x n FP64 matrices:
// M = a I; y = M^T x; v <- v/|v| (flag 1 if |v| > 0); u = w - t; out = 1 + a.b;
// J += u v^T and K -= Ku vK^T / denom
cudaError_t launch_scaled_identity(cudaStream_t s, int n, double a, double* M);
cudaError_t launch_gemv_t(cudaStream_t s, int n, const double* M, const double* x, double* y);
cudaError_t launch_normalize(cudaStream_t s, int n, double* v, double* flag);
cudaError_t launch_sub(cudaStream_t s, int n, const double* w, const double* t, double* u);
cudaError_t launch_dot1p(cudaStream_t s, int n, const double* a, const double* b, double* out);
cudaError_t launch_rank1_update(cudaStream_t s, int n, const double* u, const double* v, const double* Ku,
                                const double* vK, const double* denom, double* J, double* K);
cudaError_t launch_density_out_f64(cudaStream_t s, int N, int np, const double* Tn, const double* Tmu, double dmu,
                                   double* ddiag, double* D);

}  // namespace xl
