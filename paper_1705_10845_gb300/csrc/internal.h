// Internal declarations of the XL-BOMD library (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace xl {

// Epilogue of C = alpha * A B^T + beta * E + diag * I + diag(dvec):
// E is a matrix with leading dimension lde (may be null), dvec a device
// vector added on the diagonal for i < ndvec (may be null).
struct EpiF64 {
  double alpha = 1.0;
  const double* E = nullptr;
  int lde = 0;
  double beta = 0.0;
  double diag = 0.0;
  const double* dvec = nullptr;
  int ndvec = 0;
  double dvec_scale = 1.0;
};

// FP64 C[M x N] = epi(A[M x K] * B[N x K]^T), row-major.  M, N multiples of
// 64, K a multiple of 16.  sym: M == N and only tiles on or above the
// diagonal are computed; each is written to (i, j) and mirrored to (j, i), so
// the result is exactly symmetric (E must then be null or symmetric).
cudaError_t gemm_f64_nt(cudaStream_t s, int M, int N, int K, const double* A, int lda,
                        const double* B, int ldb, double* C, int ldc, const EpiF64& e, bool sym);

// ---- model (model_kernels.cu) ----
struct ModelConst {
  double eps_s, eps_p, t0[4], r_decay, r_cut, r_taper, U, k;
  double rep_A, rep_rho;   // pair repulsion rep_A exp(-r/rep_rho) S(r); rep_A = 0: off
};

// H0 (np x np, zeroed padding) from positions R (natoms x 3) in a box L.
cudaError_t launch_build_H0(cudaStream_t s, const ModelConst& m, int nat, double L, const double* R,
                            double* H0, int np);
// Real-space part of gamma over 27 images of the minimum image (natp x natp, ld natp);
// fp32: pair terms in FP32 (sums in FP64), for the split-precision path.
cudaError_t launch_gamma_real(cudaStream_t s, const ModelConst& m, int nat, double L, double eta,
                              const double* R, double* gam, int natp, bool fp32);
// y = gamma x with gamma = gamma_real + k SF SF^T applied through the structure
// factors (tmp: kp doubles; SF may be null when k = 0).
cudaError_t launch_gamma_apply(cudaStream_t s, int nat, const double* gam, int natp, const double* SF, int kp,
                               double k, const double* x, double* y, double* tmp);
// Structure-factor matrix SF (natp x kp): row I = sqrt(A_g) [cos(G_g.R_I), sin(G_g.R_I)].
cudaError_t launch_structure_factors(cudaStream_t s, int nat, int ng, const double* G4, const double* R,
                                     double* SF, int kp);
// pot[I] = sum_J gamma_IJ x_J  (natoms)
cudaError_t launch_gemv(cudaStream_t s, int nat, const double* gam, int natp, const double* x, double* y);
// H = H0 + diag(pot per orbital)
cudaError_t launch_apply_potential(cudaStream_t s, int nat, int np, const double* H0, const double* pot,
                                   double* H);
// Gershgorin interval of H: out[0] = min(H_ii - r_i), out[1] = max(H_ii + r_i)
cudaError_t launch_gershgorin(cudaStream_t s, int n, int np, const double* H, double* out);
// Forces: band part from D (np x np) and Coulomb real-space + reciprocal parts.
cudaError_t launch_forces(cudaStream_t s, const ModelConst& m, int nat, double L, double eta, int ng,
                          const double* G4, const double* R, const double* D, int np, const double* q,
                          const double* n, double* F, double* work /* >= 4*ng */, bool fp32);
// Pair repulsion: F_I += -dE_rep/dR_I when F is not null; e_I = half the pair energy of atom I
// when e is not null (E_rep = sum_I e_I).  No launch when rep_A = 0.
cudaError_t launch_repulsion(cudaStream_t s, const ModelConst& m, int nat, double L, const double* R, double* F,
                             double* e);
// q_I = sum_{a in I} (1 + Tn_aa) + 2 dmu dmu_diag_a - Z_I, r = q - n
cudaError_t launch_charges(cudaStream_t s, int nat, const double* ddiag, const double* Z,
                           const double* n, double* q, double* r);
// Verlet (Eqs. Integration, VRL_Damp): first half kick + drift + n update.
cudaError_t launch_verlet_first(cudaStream_t s, int nat, double L, double dt, double mass_inv_acc,
                                double* R, double* V, const double* F, double* nh, int kmax,
                                const double* Kr, double kappa, double alpha, const double* c);
cudaError_t launch_verlet_second(cudaStream_t s, int nat, double dt, double mass_inv_acc, double* V,
                                 const double* F);

// ---- expansion helpers (foe_kernels.cu), FP64 ----
cudaError_t launch_t0_init(cudaStream_t s, int n, int np, const double* H, double mu, double scale,
                           double* T0);
cudaError_t launch_ident_minus(cudaStream_t s, int np, const double* S, double* Y);
cudaError_t launch_scale(cudaStream_t s, size_t count, double c, const double* X, double* Y);
cudaError_t launch_level0_A1(cudaStream_t s, int np, const double* T0, const double* d, double* A1);
cudaError_t launch_transpose_add(cudaStream_t s, int np, const double* G, double* A1);
cudaError_t launch_row_dot(cudaStream_t s, int n, int np, const double* Y, const double* M, double* out);
cudaError_t launch_get_diag(cudaStream_t s, int n, int np, const double* X, double* out);
// out[slot] = sum_{i<n} x[i] (deterministic, one block)
cudaError_t launch_sum(cudaStream_t s, int n, const double* x, double* out);
// out = sum_{i,j<n} A_ij B_ij (deterministic two-level reduction; work >= 1024 doubles)
cudaError_t launch_frob_dot(cudaStream_t s, int n, int np, const double* A, const double* B, double* work,
                            double* out);
// Small vector algebra of the kernel update (one CTA, FP64).
cudaError_t launch_kernel_vec(cudaStream_t s, int mode, int nat, int m, double c, const double* r,
                              double* V, const double* W, double* out, double* flag);
// Energy parts: out[0..] from vectors (Coulomb, kinetic).
cudaError_t launch_energy_vec(cudaStream_t s, int nat, const double* q, const double* n,
                              const double* pot, const double* V, double mass, double* out);

}  // namespace xl
