// Electronic entropy of the occupations of D without eigenvalues (energy
// monitor, Eq. S_entropy).
//
// With f = (1 + t_n)/2 and the tanh-doubling map, ln(f/(1-f)) = 2^(n+1)
// artanh(t_0), and 1 - f satisfies ln(1 - x_{k+1}) = 2 ln(1 - x_k) - ln b_k
// with b_k = (1 + t_k^2)/2.  Summed over eigenstates:
//   sum_i s(f_i) = -sum ln(1 - f_i) - Tr[D 2^(n+1) artanh(T_0)]
//   sum ln(1 - f_i) = 2^n logdet(I - T_0) + sum_k 2^(n-1-k) logdet(Y_k) - N ln 2
// where Y_k = (I + T_k^2)^-1.  Every logdet is of a well-conditioned SPD
// matrix (spectra in [1 - |t_0|max, 1 + |t_0|max] and [1/2, 1]) and is taken
// by a blocked FP64 Cholesky factorisation; artanh(T_0) is its odd power
// series (|t_0| << 1), whose traces against D come from Frobenius products.
#include <cmath>
#include <functional>

#include "precision.h"

namespace xl {
namespace {

#define RET(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

constexpr int CB = 64;

// Factor the CB x CB diagonal block at (kb, kb) in place (lower Cholesky);
// part[kb / CB] = sum 2 ln L_ii; a non-positive pivot writes NaN.
__global__ void chol_panel_kernel(double* A, int np, int kb, double* part) {
  __shared__ double a[CB][CB + 1];
  __shared__ double lsum;
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) a[e / CB][e % CB] = A[(size_t)(kb + e / CB) * np + kb + e % CB];
  if (tid == 0) lsum = 0.0;
  __syncthreads();
  for (int j = 0; j < CB; ++j) {
    if (tid == 0) {
      const double d = a[j][j];
      const double l = d > 0.0 ? sqrt(d) : nan("");
      a[j][j] = l;
      lsum += 2.0 * log(l);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < CB; i += blockDim.x) a[i][j] /= a[j][j];
    __syncthreads();
    const int rem = CB - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= i) a[i][c] -= a[i][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, c = e % CB;
    A[(size_t)(kb + i) * np + kb + c] = (c <= i) ? a[i][c] : 0.0;
  }
  if (tid == 0) part[kb / CB] = lsum;
}

// Rows below the panel: X L^T = A_row  ->  X = A_row L^-T (one thread per row).
__global__ void chol_trsm_kernel(double* A, int np, int kb) {
  __shared__ double L[CB][CB + 1];
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) L[e / CB][e % CB] = A[(size_t)(kb + e / CB) * np + kb + e % CB];
  __syncthreads();
  const int row = kb + CB + blockIdx.x * CB + threadIdx.x;
  if (threadIdx.x >= CB || row >= np) return;
  double x[CB];
  double* ar = A + (size_t)row * np + kb;
#pragma unroll 4
  for (int j = 0; j < CB; ++j) {
    double t = ar[j];
    for (int c = 0; c < j; ++c) t -= x[c] * L[j][c];
    x[j] = t / L[j][j];
  }
#pragma unroll 4
  for (int j = 0; j < CB; ++j) ar[j] = x[j];
}

// W = I - T (np x np)
__global__ void ident_minus_f64_kernel(size_t count, int np, const double* __restrict__ T, double* __restrict__ W) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  W[idx] = (i == j ? 1.0 : 0.0) - T[idx];
}

struct EntW {
  double w_ld[42];   // weights of the logdet slots
  double w_tr[8];    // weights of the trace slots
  int nld, ntr;
  double cst;        // N ln 2
};

// out = cst - sum_k w_ld[k] ld[k] - sum_j w_tr[j] tr[j]
__global__ void entropy_combine_kernel(EntW w, const double* __restrict__ ld, const double* __restrict__ tr,
                                       double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = w.cst;
  for (int k = 0; k < w.nld; ++k) s -= w.w_ld[k] * ld[k];
  for (int j = 0; j < w.ntr; ++j) s -= w.w_tr[j] * tr[j];
  *out = s;
}

// logdet of the SPD matrix in W (destroyed); result in *out.  part >= np/CB doubles.
cudaError_t logdet_spd(cudaStream_t s, double* W, int np, double* part, double* out) {
  for (int kb = 0; kb < np; kb += CB) {
    chol_panel_kernel<<<1, 256, 0, s>>>(W, np, kb, part);
    note_launch();
    RET(cudaGetLastError());
    const int rest = np - kb - CB;
    if (rest > 0) {
      chol_trsm_kernel<<<rest / CB, CB, 0, s>>>(W, np, kb);
      note_launch();
      RET(cudaGetLastError());
      EpiF64 e;
      e.alpha = -1.0;
      e.E = W + (size_t)(kb + CB) * np + kb + CB;
      e.lde = np;
      e.beta = 1.0;
      const double* Lp = W + (size_t)(kb + CB) * np + kb;
      RET(gemm_f64_nt(s, rest, rest, CB, Lp, np, Lp, np, W + (size_t)(kb + CB) * np + kb + CB, np, e, true));
    }
  }
  return launch_sum(s, np / CB, part, out);
}

}  // namespace

// Entropy from FP64 inputs.  T0: FP64 T_0; load_Y(k, dst) writes Y_k as an
// FP64 matrix into dst; G, S, Q, Yw, A1, Mt: FP64 work matrices (np x np);
// nterms: terms j = 0..nterms-1 of the artanh series.
cudaError_t entropy_fp64(cudaStream_t s, int N, int np, int n, int n_sq, const double* T0,
                         const std::function<cudaError_t(int, double*)>& load_Y, double* G, double* S, double* Q,
                         double* Yw, double* A1, double* Mt, int nterms, const double* D, double* work,
                         double* out) {
  if (n + 1 > 42 || nterms < 1 || nterms > 6) return cudaErrorInvalidValue;
  // work layout: [0, 64): logdet slots, [64, 72): trace slots, [128, 128 + np/CB): Cholesky partials,
  // [1024, 2048): Frobenius partials
  double* ld = work;
  double* tr = work + 64;
  double* part = work + 128;
  double* fwork = work + 1024;
  const size_t count = (size_t)np * np;
  // logdet(I - T_0)
  ident_minus_f64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, np, T0, G);
  note_launch();
  RET(cudaGetLastError());
  RET(logdet_spd(s, G, np, part, ld + 0));
  // logdet(Y_k)
  for (int k = 0; k < n; ++k) {
    RET(load_Y(k, G));
    RET(logdet_spd(s, G, np, part, ld + 1 + k));
  }
  // Tr[D T0^(2j+1)] from S0 = T0^2, S2 = S0^2, S4 = S2^2, P1 = D T0, P3 = P1 S0
  EpiF64 e;
  RET(cudaMemsetAsync(tr, 0, 8 * sizeof(double), s));
  RET(launch_frob_dot(s, N, np, D, T0, fwork, tr + 0));                                    // Tr D T0
  if (nterms > 1) {
    RET(gemm_f64_nt(s, np, np, np, T0, np, T0, np, S, np, e, true));                        // S0
    RET(gemm_f64_nt(s, np, np, np, D, np, T0, np, A1, np, e, false));                       // P1 = D T0
    RET(launch_frob_dot(s, N, np, A1, S, fwork, tr + 1));                                   // Tr D T0^3
  }
  if (nterms > 2) {
    RET(gemm_f64_nt(s, np, np, np, S, np, S, np, Q, np, e, true));                          // S2 = S0^2
    RET(launch_frob_dot(s, N, np, A1, Q, fwork, tr + 2));                                   // Tr D T0^5
  }
  if (nterms > 3) {
    RET(gemm_f64_nt(s, np, np, np, A1, np, S, np, Mt, np, e, false));                       // P3 = P1 S0
    RET(launch_frob_dot(s, N, np, Mt, Q, fwork, tr + 3));                                   // Tr D T0^7
  }
  if (nterms > 4) {
    RET(gemm_f64_nt(s, np, np, np, Q, np, Q, np, Yw, np, e, true));                         // S4
    RET(launch_frob_dot(s, N, np, A1, Yw, fwork, tr + 4));                                  // Tr D T0^9
  }
  if (nterms > 5) RET(launch_frob_dot(s, N, np, Mt, Yw, fwork, tr + 5));                    // Tr D T0^11
  EntW w{};
  w.nld = n + 1;
  w.w_ld[0] = std::ldexp(1.0, n_sq);
  for (int k = 0; k < n; ++k) w.w_ld[1 + k] = std::ldexp(1.0, n_sq - 1 - k);
  w.ntr = nterms;
  for (int j = 0; j < nterms; ++j) w.w_tr[j] = std::ldexp(1.0, n_sq + 1) / (2.0 * j + 1.0);
  w.cst = N * std::log(2.0);
  entropy_combine_kernel<<<1, 32, 0, s>>>(w, ld, tr, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_entropy_f64(cudaStream_t s, MatSet& m, int N, double beta, int n_sq, double mu, double dmu,
                               const double* D, const double* H, double* work, double* out) {
  (void)beta;
  (void)mu;
  (void)dmu;
  (void)H;
  const size_t count = (size_t)m.np * m.np;
  auto load_Y = [&](int k, double* dst) {
    return cudaMemcpyAsync(dst, m.Y[k], sizeof(double) * count, cudaMemcpyDeviceToDevice, s);
  };
  return entropy_fp64(s, N, m.np, m.n, n_sq, m.T[0], load_Y, m.G, m.S, m.Q, m.Yw, m.A1, m.Mt, 6, D, work, out);
}

}  // namespace xl
