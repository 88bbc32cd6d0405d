// Model kernels of the XL-BOMD path: the Slater-Koster Hamiltonian H0, the
// periodic Ohno-Klopman Coulomb matrix gamma, H[n] = H0 + diag(gamma n), the
// Hellmann-Feynman forces (Eq. EqMotFT), Mulliken charges, and the
// velocity-Verlet / dissipative-Verlet updates (Eqs. Integration, VRL_Damp).
//
// All of this is O(natoms^2) or O(N^2) FP64 work; the pair kernels are
// organised one warp per atom I with the lanes striding over J, so every
// 4x4 block row written to H0 is a coalesced 32-byte-per-lane store.
#include "internal.h"

namespace xl {
namespace {

struct Bond {
  double V[4], dV[4];
};

// V_k(r) = t0_k exp(-r/r_decay) S(r), S the quintic switch on [r_taper, r_cut].
__device__ __forceinline__ Bond bond(const ModelConst& m, double r) {
  const double w = m.r_cut - m.r_taper;
  double s = (r - m.r_taper) / w;
  s = fmin(fmax(s, 0.0), 1.0);
  const double s2 = s * s, s3 = s2 * s;
  const double S = 1.0 - 10.0 * s3 + 15.0 * s3 * s - 6.0 * s3 * s2;
  const double dS = (-30.0 * s2 + 60.0 * s3 - 30.0 * s3 * s) / w;
  const double e = exp(-r / m.r_decay);
  Bond b;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b.V[k] = m.t0[k] * e * S;
    b.dV[k] = m.t0[k] * e * (dS - S / m.r_decay);
  }
  return b;
}

// Adds the s/p block E_ab(d) (Slater-Koster direction-cosine rules).
__device__ __forceinline__ void add_block(const ModelConst& m, double dx, double dy, double dz, double r,
                                          double E[4][4]) {
  const Bond b = bond(m, r);
  const double c[3] = {dx / r, dy / r, dz / r};
  E[0][0] += b.V[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E[0][1 + a] += c[a] * b.V[1];
    E[1 + a][0] -= c[a] * b.V[1];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      E[1 + a][1 + q] += c[a] * c[q] * (b.V[2] - b.V[3]) + (a == q ? b.V[3] : 0.0);
  }
}

// sum_ab D_ab dE_ab/dd_g for one bond vector d (adds to f[3]).
__device__ __forceinline__ void add_block_grad(const ModelConst& m, double dx, double dy, double dz, double r,
                                               const double D[4][4], double f[3]) {
  const Bond b = bond(m, r);
  const double c[3] = {dx / r, dy / r, dz / r};
  const double dVpp = b.V[2] - b.V[3], ddVpp = b.dV[2] - b.dV[3];
  double spsum[3] = {0, 0, 0};   // sum_a (D_0a - D_a0) over p orbitals, per gradient component
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    double acc = D[0][0] * b.dV[0] * c[g];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double dca = ((a == g ? 1.0 : 0.0) - c[a] * c[g]) / r;
      const double gsp = dca * b.V[1] + c[a] * b.dV[1] * c[g];
      acc += (D[0][1 + a] - D[1 + a][0]) * gsp;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double dcq = ((q == g ? 1.0 : 0.0) - c[q] * c[g]) / r;
        const double gpp = (dca * c[q] + c[a] * dcq) * dVpp + c[a] * c[q] * ddVpp * c[g] +
                           (a == q ? b.dV[3] * c[g] : 0.0);
        acc += D[1 + a][1 + q] * gpp;
      }
    }
    spsum[g] = acc;
  }
  f[0] += spsum[0];
  f[1] += spsum[1];
  f[2] += spsum[2];
}

__global__ void build_H0_kernel(ModelConst m, int nat, double L, const double* __restrict__ R,
                                double* __restrict__ H0, int np) {
  const int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= nat) return;
  const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2];
  const double rc2 = m.r_cut * m.r_cut;
  for (int J = lane; J < nat; J += 32) {
    double E[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) E[a][b] = 0.0;
    const double x0 = R[3 * J] - xi, y0 = R[3 * J + 1] - yi, z0 = R[3 * J + 2] - zi;
    for (int tx = -1; tx <= 1; ++tx)
      for (int ty = -1; ty <= 1; ++ty)
        for (int tz = -1; tz <= 1; ++tz) {
          if (J == I && tx == 0 && ty == 0 && tz == 0) continue;
          const double dx = x0 + tx * L, dy = y0 + ty * L, dz = z0 + tz * L;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 >= rc2) continue;
          add_block(m, dx, dy, dz, sqrt(r2), E);
        }
    if (J == I) {
      E[0][0] += m.eps_s;
      E[1][1] += m.eps_p;
      E[2][2] += m.eps_p;
      E[3][3] += m.eps_p;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double* row = H0 + (size_t)(4 * I + a) * np + 4 * J;
#pragma unroll
      for (int b = 0; b < 4; ++b) row[b] = E[a][b];
    }
  }
}

// F_I += 4 sum_J sum_T sum_ab D_{Ia,Jb} dE_ab/dd, d = R_J + T L - R_I
__global__ void forces_band_kernel(ModelConst m, int nat, double L, const double* __restrict__ R,
                                   const double* __restrict__ D, int np, double* __restrict__ F) {
  const int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= nat) return;
  const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2];
  const double rc2 = m.r_cut * m.r_cut;
  double f[3] = {0, 0, 0};
  for (int J = lane; J < nat; J += 32) {
    if (J == I) continue;   // self images do not depend on R_I
    const double x0 = R[3 * J] - xi, y0 = R[3 * J + 1] - yi, z0 = R[3 * J + 2] - zi;
    bool loaded = false;
    double Db[4][4];
    for (int tx = -1; tx <= 1; ++tx)
      for (int ty = -1; ty <= 1; ++ty)
        for (int tz = -1; tz <= 1; ++tz) {
          const double dx = x0 + tx * L, dy = y0 + ty * L, dz = z0 + tz * L;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 >= rc2) continue;
          if (!loaded) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) Db[a][b] = D[(size_t)(4 * I + a) * np + 4 * J + b];
            loaded = true;
          }
          add_block_grad(m, dx, dy, dz, sqrt(r2), Db, f);
        }
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const double v = warp_sum(f[g]);
    if (lane == 0) F[3 * I + g] = 4.0 * v;
  }
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

template <typename R>
__device__ __forceinline__ R ok_real_t(R r, R a, R eta) {
  const R s = sqrt(r * r + a * a);
  return erfc(eta * r) / r - a * a / (r * s * (s + r));
}

template <typename R>
__device__ __forceinline__ R ok_real_dr_t(R r, R a, R eta) {
  const R s2 = r * r + a * a;
  return erf(eta * r) / (r * r) - R(2) * eta / sqrt(R(kPi)) * exp(-eta * eta * r * r) / r - r / (s2 * sqrt(s2));
}

template <typename R>
__global__ void gamma_real_kernel(ModelConst m, int nat, double L, double eta, const double* __restrict__ R_,
                                  double* __restrict__ gam, int natp) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = blockIdx.y;
  if (J >= natp) return;
  if (J >= nat) {
    gam[(size_t)I * natp + J] = 0.0;
    return;
  }
  const double a = m.k / m.U;
  const double dx0 = min_image(R_[3 * J] - R_[3 * I], L);
  const double dy0 = min_image(R_[3 * J + 1] - R_[3 * I + 1], L);
  const double dz0 = min_image(R_[3 * J + 2] - R_[3 * I + 2], L);
  double acc = 0.0;
  for (int tx = -1; tx <= 1; ++tx)
    for (int ty = -1; ty <= 1; ++ty)
      for (int tz = -1; tz <= 1; ++tz) {
        if (I == J && tx == 0 && ty == 0 && tz == 0) {
          acc += 1.0 / a - 2.0 * eta / sqrt(kPi);
          continue;
        }
        const double dx = dx0 + tx * L, dy = dy0 + ty * L, dz = dz0 + tz * L;
        acc += (double)ok_real_t<R>((R)sqrt(dx * dx + dy * dy + dz * dz), (R)a, (R)eta);
      }
  gam[(size_t)I * natp + J] = m.k * acc;
}

// SF[I][g] = sqrt(w_g) cos(G_g.R_I), SF[I][ng+g] = sqrt(w_g) sin(G_g.R_I); zero padding.
__global__ void structure_factor_kernel(int nat, int ng, const double* __restrict__ G4,
                                        const double* __restrict__ R, double* __restrict__ SF, int kp,
                                        int natp) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = blockIdx.y;
  if (g >= kp || I >= natp) return;
  double v = 0.0;
  if (I < nat) {
    const int gg = g < ng ? g : g - ng;
    if (gg < ng && g < 2 * ng) {
      const double ph = G4[4 * gg] * R[3 * I] + G4[4 * gg + 1] * R[3 * I + 1] + G4[4 * gg + 2] * R[3 * I + 2];
      const double sw = sqrt(G4[4 * gg + 3]);
      v = (g < ng) ? sw * cos(ph) : sw * sin(ph);
    }
  }
  SF[(size_t)I * kp + g] = v;
}

__global__ void gemv_kernel(int nat, const double* __restrict__ gam, int natp, const double* __restrict__ x,
                            double* __restrict__ y) {
  const int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= nat) return;
  double acc = 0.0;
  for (int J = lane; J < nat; J += 32) acc += gam[(size_t)I * natp + J] * x[J];
  acc = warp_sum(acc);
  if (lane == 0) y[I] = acc;
}

// t[g] = sum_I SF[I][g] x[I]
__global__ void sf_dot_kernel(int nat, int kp, const double* __restrict__ SF, const double* __restrict__ x,
                              double* __restrict__ t) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= kp) return;
  double acc = 0.0;
  for (int I = 0; I < nat; ++I) acc += SF[(size_t)I * kp + g] * x[I];
  t[g] = acc;
}

// y_I = sum_J gamma_real_IJ x_J + k sum_g SF[I][g] t[g]
__global__ void gamma_apply_kernel(int nat, const double* __restrict__ gam, int natp, const double* __restrict__ SF,
                                   int kp, double k, const double* __restrict__ t, const double* __restrict__ x,
                                   double* __restrict__ y) {
  const int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= nat) return;
  double acc = 0.0, rec = 0.0;
  for (int J = lane; J < nat; J += 32) acc += gam[(size_t)I * natp + J] * x[J];
  if (SF)
    for (int g = lane; g < kp; g += 32) rec += SF[(size_t)I * kp + g] * t[g];
  acc = warp_sum(acc + k * rec);
  if (lane == 0) y[I] = acc;
}

__global__ void add_potential_kernel(int nat, int np, const double* __restrict__ pot, double* __restrict__ H) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= 4 * nat) return;
  H[(size_t)a * np + a] += pot[a >> 2];
}

__global__ void gershgorin_rows_kernel(int n, int np, const double* __restrict__ H, double* __restrict__ lohi) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (j != i) acc += fabs(H[(size_t)i * np + j]);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double d = H[(size_t)i * np + i];
    lohi[i] = d - acc;
    lohi[n + i] = d + acc;
  }
}

__global__ void minmax_kernel(int n, const double* __restrict__ lohi, double* __restrict__ out) {
  __shared__ double sl[32], sh[32];
  double lo = 1e300, hi = -1e300;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    bad |= !isfinite(lohi[i]) || !isfinite(lohi[n + i]);
    lo = fmin(lo, lohi[i]);
    hi = fmax(hi, lohi[n + i]);
  }
  // fmin/fmax drop NaN: a non-finite row poisons both bounds so that the host sees it
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) out[0] = out[1] = nan("");
    return;
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sl[wid] = lo;
    sh[wid] = hi;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    lo = lane < nw ? sl[lane] : 1e300;
    hi = lane < nw ? sh[lane] : -1e300;
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
      out[0] = lo;
      out[1] = hi;
    }
  }
}

// Coulomb real-space force: F_K -= k sum_{I != K} w_IK sum_T phi'(r) d/r,
// d = mi(R_K - R_I) + T L, w_IK = (a_I b_K + a_K b_I)/2, a = 2q - n, b = n.
template <typename R>
__global__ void forces_coul_real_kernel(ModelConst m, int nat, double L, double eta, const double* __restrict__ R_,
                                        const double* __restrict__ q, const double* __restrict__ n,
                                        double* __restrict__ F) {
  const int K = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (K >= nat) return;
  const double a = m.k / m.U;
  const double aK = 2.0 * q[K] - n[K], bK = n[K];
  double f[3] = {0, 0, 0};
  for (int I = lane; I < nat; I += 32) {
    if (I == K) continue;
    const double w = 0.5 * ((2.0 * q[I] - n[I]) * bK + aK * n[I]);
    const double dx0 = min_image(R_[3 * K] - R_[3 * I], L);
    const double dy0 = min_image(R_[3 * K + 1] - R_[3 * I + 1], L);
    const double dz0 = min_image(R_[3 * K + 2] - R_[3 * I + 2], L);
    for (int tx = -1; tx <= 1; ++tx)
      for (int ty = -1; ty <= 1; ++ty)
        for (int tz = -1; tz <= 1; ++tz) {
          const double dx = dx0 + tx * L, dy = dy0 + ty * L, dz = dz0 + tz * L;
          const R r = (R)sqrt(dx * dx + dy * dy + dz * dz);
          const double g = w * (double)(ok_real_dr_t<R>(r, (R)a, (R)eta) / r);
          f[0] += g * dx;
          f[1] += g * dy;
          f[2] += g * dz;
        }
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const double v = warp_sum(f[g]);
    if (lane == 0) F[3 * K + g] -= m.k * v;
  }
}

// Per reciprocal vector: C_a, S_a, C_b, S_b (a = 2q - n, b = n).
__global__ void coul_sums_kernel(int nat, int ng, const double* __restrict__ G4, const double* __restrict__ R,
                                 const double* __restrict__ q, const double* __restrict__ n,
                                 double* __restrict__ sums) {
  __shared__ double sh[32];
  const int g = blockIdx.x;
  double ca = 0, sa = 0, cb = 0, sb = 0;
  for (int I = threadIdx.x; I < nat; I += blockDim.x) {
    const double ph = G4[4 * g] * R[3 * I] + G4[4 * g + 1] * R[3 * I + 1] + G4[4 * g + 2] * R[3 * I + 2];
    double sv, cv;
    sincos(ph, &sv, &cv);
    const double a = 2.0 * q[I] - n[I], b = n[I];
    ca += a * cv;
    sa += a * sv;
    cb += b * cv;
    sb += b * sv;
  }
  ca = block_sum(ca, sh);
  sa = block_sum(sa, sh);
  cb = block_sum(cb, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    sums[4 * g] = ca;
    sums[4 * g + 1] = sa;
    sums[4 * g + 2] = cb;
    sums[4 * g + 3] = sb;
  }
}

// F_K -= (k/2) sum_g w_g G [cos(G.R_K)(a_K S_b + b_K S_a) - sin(G.R_K)(a_K C_b + b_K C_a)]
__global__ void forces_coul_recip_kernel(double kcoul, int nat, int ng, const double* __restrict__ G4,
                                         const double* __restrict__ R, const double* __restrict__ q,
                                         const double* __restrict__ n, const double* __restrict__ sums,
                                         double* __restrict__ F) {
  const int K = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (K >= nat) return;
  const double aK = 2.0 * q[K] - n[K], bK = n[K];
  double f[3] = {0, 0, 0};
  for (int g = lane; g < ng; g += 32) {
    const double gx = G4[4 * g], gy = G4[4 * g + 1], gz = G4[4 * g + 2], w = G4[4 * g + 3];
    double sv, cv;
    sincos(gx * R[3 * K] + gy * R[3 * K + 1] + gz * R[3 * K + 2], &sv, &cv);
    const double ca = sums[4 * g], sa = sums[4 * g + 1], cb = sums[4 * g + 2], sb = sums[4 * g + 3];
    const double t = w * (cv * (aK * sb + bK * sa) - sv * (aK * cb + bK * ca));
    f[0] += t * gx;
    f[1] += t * gy;
    f[2] += t * gz;
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const double v = warp_sum(f[g]);
    if (lane == 0) F[3 * K + g] -= 0.5 * kcoul * v;
  }
}

__global__ void charges_kernel(int nat, const double* __restrict__ ddiag, const double* __restrict__ Z,
                               const double* __restrict__ n, double* __restrict__ q, double* __restrict__ r) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nat) return;
  const double qi = ddiag[4 * I] + ddiag[4 * I + 1] + ddiag[4 * I + 2] + ddiag[4 * I + 3] - Z[I];
  q[I] = qi;
  r[I] = qi - n[I];
}

__global__ void verlet_first_kernel(int nat, double L, double dt, double minv, double* __restrict__ R,
                                    double* __restrict__ V, const double* __restrict__ F, double* __restrict__ nh,
                                    int kmax, const double* __restrict__ Kr, double kappa, double alpha,
                                    const double* __restrict__ c) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nat) return;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    double v = V[3 * I + g] + 0.5 * dt * F[3 * I + g] * minv;
    double x = R[3 * I + g] + dt * v;
    x -= L * floor(x / L);
    if (x >= L) x -= L;
    V[3 * I + g] = v;
    R[3 * I + g] = x;
  }
  double diss = 0.0;
  for (int k = 0; k <= kmax; ++k) diss += c[k] * nh[(size_t)k * nat + I];
  const double nn = 2.0 * nh[I] - nh[(size_t)nat + I] - kappa * Kr[I] + alpha * diss;
  for (int k = kmax; k >= 1; --k) nh[(size_t)k * nat + I] = nh[(size_t)(k - 1) * nat + I];
  nh[I] = nn;
}

__global__ void verlet_second_kernel(int nat, double dt, double minv, double* __restrict__ V,
                                     const double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nat) return;
  V[i] += 0.5 * dt * F[i] * minv;
}

// out[0] = 1/2 sum (2q - n) pot (Coulomb), out[1] = kinetic energy (eV)
// Pair repulsion A exp(-r/rho) S(r) over the 27 images of the minimum image (one warp per
// atom I, lanes over J): F_I += sum_{J,T} d(e S)/dr (R_J + T L - R_I)/r, e_I = 1/2 sum e S.
__global__ void repulsion_kernel(ModelConst m, int nat, double L, const double* __restrict__ R,
                                 double* __restrict__ F, double* __restrict__ e) {
  const int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (I >= nat) return;
  const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2];
  const double rc2 = m.r_cut * m.r_cut, w = m.r_cut - m.r_taper;
  double fx = 0.0, fy = 0.0, fz = 0.0, en = 0.0;
  for (int J = lane; J < nat; J += 32) {
    const double x0 = R[3 * J] - xi, y0 = R[3 * J + 1] - yi, z0 = R[3 * J + 2] - zi;
    for (int tx = -1; tx <= 1; ++tx)
      for (int ty = -1; ty <= 1; ++ty)
        for (int tz = -1; tz <= 1; ++tz) {
          if (J == I && tx == 0 && ty == 0 && tz == 0) continue;
          const double dx = x0 + tx * L, dy = y0 + ty * L, dz = z0 + tz * L;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 >= rc2) continue;
          const double r = sqrt(r2);
          const double u = fmin(fmax((r - m.r_taper) / w, 0.0), 1.0);
          const double S = 1.0 - u * u * u * (10.0 - u * (15.0 - 6.0 * u));
          const double dS = -30.0 * u * u * (1.0 - u) * (1.0 - u) / w;
          const double ex = m.rep_A * exp(-r / m.rep_rho);
          const double de = ex * (dS - S / m.rep_rho);
          fx += de * dx / r;
          fy += de * dy / r;
          fz += de * dz / r;
          en += 0.5 * ex * S;
        }
  }
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  fz = warp_sum(fz);
  en = warp_sum(en);
  if (lane == 0) {
    if (F) {
      F[3 * I] += fx;
      F[3 * I + 1] += fy;
      F[3 * I + 2] += fz;
    }
    if (e) e[I] = en;
  }
}

__global__ void energy_vec_kernel(int nat, const double* __restrict__ q, const double* __restrict__ n,
                                  const double* __restrict__ pot, const double* __restrict__ V, double mass,
                                  double* __restrict__ out) {
  __shared__ double sh[32];
  double ec = 0.0, ke = 0.0;
  for (int I = threadIdx.x; I < nat; I += blockDim.x) {
    ec += (2.0 * q[I] - n[I]) * pot[I];
    ke += V[3 * I] * V[3 * I] + V[3 * I + 1] * V[3 * I + 1] + V[3 * I + 2] * V[3 * I + 2];
  }
  ec = block_sum(ec, sh);
  ke = block_sum(ke, sh);
  if (threadIdx.x == 0) {
    out[0] = 0.5 * ec;
    out[1] = 0.5 * mass * ke / 9.648533e-3;
  }
}

}  // namespace

cudaError_t launch_build_H0(cudaStream_t s, const ModelConst& m, int nat, double L, const double* R, double* H0,
                            int np) {
  const int wpb = 8;
  build_H0_kernel<<<(nat + wpb - 1) / wpb, 32 * wpb, 0, s>>>(m, nat, L, R, H0, np);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gamma_real(cudaStream_t s, const ModelConst& m, int nat, double L, double eta, const double* R,
                              double* gam, int natp, bool fp32) {
  dim3 grid((natp + 127) / 128, nat);
  if (fp32)
    gamma_real_kernel<float><<<grid, 128, 0, s>>>(m, nat, L, eta, R, gam, natp);
  else
    gamma_real_kernel<double><<<grid, 128, 0, s>>>(m, nat, L, eta, R, gam, natp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gamma_apply(cudaStream_t s, int nat, const double* gam, int natp, const double* SF, int kp,
                               double k, const double* x, double* y, double* tmp) {
  if (SF && k != 0.0) {
    sf_dot_kernel<<<(kp + 255) / 256, 256, 0, s>>>(nat, kp, SF, x, tmp);
    note_launch();
  } else {
    SF = nullptr;
  }
  const int wpb = 8;
  gamma_apply_kernel<<<(nat + wpb - 1) / wpb, 32 * wpb, 0, s>>>(nat, gam, natp, SF, kp, k, tmp, x, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_structure_factors(cudaStream_t s, int nat, int ng, const double* G4, const double* R, double* SF,
                                     int kp) {
  const int natp = (nat + 63) / 64 * 64;
  dim3 grid((kp + 127) / 128, natp);
  structure_factor_kernel<<<grid, 128, 0, s>>>(nat, ng, G4, R, SF, kp, natp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemv(cudaStream_t s, int nat, const double* gam, int natp, const double* x, double* y) {
  const int wpb = 8;
  gemv_kernel<<<(nat + wpb - 1) / wpb, 32 * wpb, 0, s>>>(nat, gam, natp, x, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply_potential(cudaStream_t s, int nat, int np, const double* H0, const double* pot,
                                   double* H) {
  cudaError_t e = cudaMemcpyAsync(H, H0, sizeof(double) * (size_t)np * np, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  add_potential_kernel<<<(4 * nat + 255) / 256, 256, 0, s>>>(nat, np, pot, H);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gershgorin(cudaStream_t s, int n, int np, const double* H, double* out) {
  // out[0..1] result; out[2 .. 2+2n) scratch
  gershgorin_rows_kernel<<<n, 256, 0, s>>>(n, np, H, out + 2);
  note_launch();
  minmax_kernel<<<1, 1024, 0, s>>>(n, out + 2, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_repulsion(cudaStream_t s, const ModelConst& m, int nat, double L, const double* R, double* F,
                             double* e) {
  if (m.rep_A == 0.0) return cudaSuccess;
  const int wpb = 8;
  repulsion_kernel<<<(nat + wpb - 1) / wpb, 32 * wpb, 0, s>>>(m, nat, L, R, F, e);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_forces(cudaStream_t s, const ModelConst& m, int nat, double L, double eta, int ng,
                          const double* G4, const double* R, const double* D, int np, const double* q,
                          const double* n, double* F, double* work, bool fp32) {
  const int wpb = 8;
  const int nb = (nat + wpb - 1) / wpb;
  forces_band_kernel<<<nb, 32 * wpb, 0, s>>>(m, nat, L, R, D, np, F);
  note_launch();
  if (m.k != 0.0) {
    if (fp32)
      forces_coul_real_kernel<float><<<nb, 32 * wpb, 0, s>>>(m, nat, L, eta, R, q, n, F);
    else
      forces_coul_real_kernel<double><<<nb, 32 * wpb, 0, s>>>(m, nat, L, eta, R, q, n, F);
    note_launch();
    coul_sums_kernel<<<ng, 256, 0, s>>>(nat, ng, G4, R, q, n, work);
    note_launch();
    forces_coul_recip_kernel<<<nb, 32 * wpb, 0, s>>>(m.k, nat, ng, G4, R, q, n, work, F);
    note_launch();
  }
  if (cudaError_t e = launch_repulsion(s, m, nat, L, R, F, nullptr)) return e;
  return cudaGetLastError();
}

cudaError_t launch_charges(cudaStream_t s, int nat, const double* ddiag, const double* Z, const double* n,
                           double* q, double* r) {
  charges_kernel<<<(nat + 127) / 128, 128, 0, s>>>(nat, ddiag, Z, n, q, r);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_verlet_first(cudaStream_t s, int nat, double L, double dt, double minv, double* R, double* V,
                                const double* F, double* nh, int kmax, const double* Kr, double kappa,
                                double alpha, const double* c) {
  verlet_first_kernel<<<(nat + 127) / 128, 128, 0, s>>>(nat, L, dt, minv, R, V, F, nh, kmax, Kr, kappa, alpha, c);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_verlet_second(cudaStream_t s, int nat, double dt, double minv, double* V, const double* F) {
  verlet_second_kernel<<<(3 * nat + 127) / 128, 128, 0, s>>>(nat, dt, minv, V, F);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_energy_vec(cudaStream_t s, int nat, const double* q, const double* n, const double* pot,
                              const double* V, double mass, double* out) {
  energy_vec_kernel<<<1, 1024, 0, s>>>(nat, q, n, pot, V, mass, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace xl
