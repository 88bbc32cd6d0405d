// Element-wise and reduction kernels of the recursive Fermi-operator expansion
// and of its response chains (FP64 storage), plus the small FP64 vector
// algebra of the rank-m kernel update (Eqs. K_up, v_1; Woodbury form).
//
// The expansion is run in its tanh-doubling form: with
// T_0 = -beta (H - mu I) / 2^(n+1), the recursion
// X_{k+1} = X_k^2 [X_k^2 + (I - X_k)^2]^-1 on X = (I + T)/2 becomes
// T_{k+1} = 2 T_k (I + T_k^2)^-1 and D = (I + T_n)/2.
#include "precision.h"

namespace xl {
namespace {

__global__ void t0_init_kernel(int n, int np, const double* __restrict__ H, double mu, double scale,
                               double* __restrict__ T0) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * np) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  double v = 0.0;
  if (i < n && j < n) v = -scale * (H[idx] - (i == j ? mu : 0.0));
  T0[idx] = v;
}

__global__ void ident_minus_kernel(int np, const double* __restrict__ S, double* __restrict__ Y) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * np) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  Y[idx] = (i == j ? 1.0 : 0.0) - S[idx];
}

__global__ void scale_kernel(size_t count, double c, const double* __restrict__ X, double* __restrict__ Y) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) Y[idx] = c * X[idx];
}

// A1 = T0 diag(d) + diag(d) T0  (first level of a chain with diagonal T1_0)
__global__ void level0_A1_kernel(int np, const double* __restrict__ T0, const double* __restrict__ d,
                                 double* __restrict__ A1) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * np) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  A1[idx] = T0[idx] * (d[i] + d[j]);
}

// A1 = G + G^T through 32x32 shared-memory tiles (coalesced both ways).
__global__ void transpose_add_kernel(int np, const double* __restrict__ G, double* __restrict__ A1) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < 32; r += 8) tile[r][tx] = G[(size_t)(bx + r) * np + by + tx];   // rows of block (bx, by)^T
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const size_t o = (size_t)(by + r) * np + bx + tx;
    A1[o] = G[o] + tile[tx][r];
  }
}

// out[i] = sum_j Y_ij M_ij (i < n): the diagonal of Y M^T, one warp per row.
__global__ void row_dot_kernel(int n, int np, const double* __restrict__ Y, const double* __restrict__ M,
                               double* __restrict__ out) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* y = Y + (size_t)i * np;
  const double* m = M + (size_t)i * np;
  double acc = 0.0;
  for (int j = lane; j < np; j += 32) acc += y[j] * m[j];
  acc = warp_sum(acc);
  if (lane == 0) out[i] = acc;
}

__global__ void get_diag_kernel(int n, int np, const double* __restrict__ X, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = X[(size_t)i * np + i];
}

__global__ void sum_kernel(int n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

// partial[b] = sum over rows b, b + gridDim.x, ... of sum_{j<n} A_ij B_ij
__global__ void frob_partial_kernel(int n, int np, const double* __restrict__ A, const double* __restrict__ B,
                                    double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < n; j += blockDim.x) acc += A[(size_t)i * np + j] * B[(size_t)i * np + j];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// ---- rank-m kernel update (one CTA) ----
//
// With orthonormal probes V (rows), responses W, U = W - c V and
// S = (c - 1) I_m + V U^T, the Sherman-Morrison sequence of Eq. K_up equals
// K_m x = [x - U^T S^-1 V x] / (c - 1).
// mode 0: v_i = K_{i} r orthonormalised (two Gram-Schmidt passes) against the
//         first i probes; flag = 1 and V[i] = v_i, or flag = 0 when less than
//         1e-12 of it is left (K_i r already in the span).
// mode 1: out = K_m r.
__device__ void kernel_apply(int nat, int m, double c, const double* r, const double* V, const double* W,
                             double* x, double* sh, double* Smat, double* y) {
  // x = K_m r
  const int tid = threadIdx.x;
  if (m == 0) {
    for (int I = tid; I < nat; I += blockDim.x) x[I] = r[I] / (c - 1.0);
    __syncthreads();
    return;
  }
  for (int a = 0; a < m; ++a) {
    for (int b = 0; b < m; ++b) {
      double acc = 0.0;
      for (int I = tid; I < nat; I += blockDim.x)
        acc += V[(size_t)a * nat + I] * (W[(size_t)b * nat + I] - c * V[(size_t)b * nat + I]);
      acc = block_sum(acc, sh);
      if (tid == 0) Smat[a * kMaxRank + b] = acc + (a == b ? c - 1.0 : 0.0);
    }
    double acc = 0.0;
    for (int I = tid; I < nat; I += blockDim.x) acc += V[(size_t)a * nat + I] * r[I];
    acc = block_sum(acc, sh);
    if (tid == 0) y[a] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    // Gaussian elimination with partial pivoting on the m x m system S y = V r
    double A[kMaxRank][kMaxRank + 1];
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) A[a][b] = Smat[a * kMaxRank + b];
      A[a][m] = y[a];
    }
    for (int col = 0; col < m; ++col) {
      int piv = col;
      for (int a = col + 1; a < m; ++a)
        if (fabs(A[a][col]) > fabs(A[piv][col])) piv = a;
      if (piv != col)
        for (int b = 0; b <= m; ++b) {
          const double t = A[col][b];
          A[col][b] = A[piv][b];
          A[piv][b] = t;
        }
      for (int a = col + 1; a < m; ++a) {
        const double f = A[a][col] / A[col][col];
        for (int b = col; b <= m; ++b) A[a][b] -= f * A[col][b];
      }
    }
    for (int a = m - 1; a >= 0; --a) {
      double t = A[a][m];
      for (int b = a + 1; b < m; ++b) t -= A[a][b] * y[b];
      y[a] = t / A[a][a];
    }
  }
  __syncthreads();
  for (int I = tid; I < nat; I += blockDim.x) {
    double t = r[I];
    for (int a = 0; a < m; ++a) t -= (W[(size_t)a * nat + I] - c * V[(size_t)a * nat + I]) * y[a];
    x[I] = t / (c - 1.0);
  }
  __syncthreads();
}

__global__ void kernel_vec_kernel(int mode, int nat, int m, double c, const double* __restrict__ r,
                                  double* __restrict__ V, const double* __restrict__ W, double* __restrict__ out,
                                  double* __restrict__ flag) {
  __shared__ double sh[32];
  __shared__ double Smat[kMaxRank * kMaxRank];
  __shared__ double y[kMaxRank];
  const int tid = threadIdx.x;
  if (mode == 1) {
    kernel_apply(nat, m, c, r, V, W, out, sh, Smat, y);
    return;
  }
  // mode 0: candidate into V[m]
  double* v = V + (size_t)m * nat;
  kernel_apply(nat, m, c, r, V, W, v, sh, Smat, y);
  double n0 = 0.0;
  for (int I = tid; I < nat; I += blockDim.x) n0 += v[I] * v[I];
  n0 = sqrt(block_sum(n0, sh));
  for (int pass = 0; pass < 2; ++pass)
    for (int a = 0; a < m; ++a) {
      double d = 0.0;
      for (int I = tid; I < nat; I += blockDim.x) d += V[(size_t)a * nat + I] * v[I];
      d = block_sum(d, sh);
      for (int I = tid; I < nat; I += blockDim.x) v[I] -= d * V[(size_t)a * nat + I];
      __syncthreads();
    }
  double nv = 0.0;
  for (int I = tid; I < nat; I += blockDim.x) nv += v[I] * v[I];
  nv = sqrt(block_sum(nv, sh));
  const bool ok = (n0 > 0.0) && isfinite(nv) && (nv > 1e-12 * n0);
  if (ok)
    for (int I = tid; I < nat; I += blockDim.x) v[I] /= nv;
  if (tid == 0) *flag = ok ? 1.0 : 0.0;
}

__global__ void expand_potential_kernel(int nat, int np, double scale, const double* __restrict__ pot,
                                        double* __restrict__ dvec) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= np) return;
  dvec[a] = (a < 4 * nat) ? scale * pot[a >> 2] : 0.0;
}

// mu1 = -sum d1 / sum dmu;  w_I = sum_{a in I} (d1_a + mu1 dmu_a)  (one block)
__global__ void response_finish_kernel(int nat, int N, const double* __restrict__ d1,
                                       const double* __restrict__ dmu, double* __restrict__ scal,
                                       double* __restrict__ w) {
  __shared__ double sh[32];
  double s1 = 0.0, s2 = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    s1 += d1[a];
    s2 += dmu[a];
  }
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  const double mu1 = (s2 != 0.0) ? -s1 / s2 : 0.0;
  if (threadIdx.x == 0) {
    scal[0] = s1;
    scal[1] = s2;
    scal[2] = mu1;
  }
  for (int I = threadIdx.x; I < nat; I += blockDim.x) {
    double t = 0.0;
    for (int a = 4 * I; a < 4 * I + 4; ++a) t += d1[a] + mu1 * dmu[a];
    w[I] = t;
  }
}

__global__ void absmax_kernel(int n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) {
      // NaN anywhere poisons the result so that the host sees it
      bool bad = false;
      for (int i = 0; i < n; ++i)
        if (!isfinite(x[i])) {
          bad = true;
          break;
        }
      *out = bad ? nan("") : m;
    }
  }
}

__global__ void fill_history_kernel(int nat, int kmax, double* __restrict__ nh) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nat) return;
  for (int k = 1; k <= kmax; ++k) nh[(size_t)k * nat + I] = nh[I];
}

__global__ void axpy_kernel(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void diag_sum_kernel(int n, int np, const double* __restrict__ X, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += X[(size_t)i * np + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

// ddiag_a = 1 + Tn_aa + dmu Tmu_aa (a < N);  D = (I + Tn + dmu Tmu) / 2 on the N x N block, 0 elsewhere
__global__ void density_out_kernel(int N, int np, const double* __restrict__ Tn, const double* __restrict__ Tmu,
                                   double dmu, double* __restrict__ ddiag, double* __restrict__ D) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * np) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  double v = 0.0;
  if (i < N && j < N) {
    v = 0.5 * (Tn[idx] + dmu * Tmu[idx] + (i == j ? 1.0 : 0.0));
    if (i == j) ddiag[i] = 2.0 * v;
  }
  D[idx] = v;
}

inline unsigned blocks_for(size_t count, int tpb) { return (unsigned)((count + tpb - 1) / tpb); }

}  // namespace

cudaError_t launch_expand_potential(cudaStream_t s, int nat, int np, double scale, const double* pot, double* dvec) {
  expand_potential_kernel<<<blocks_for(np, 256), 256, 0, s>>>(nat, np, scale, pot, dvec);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_response_finish(cudaStream_t s, int nat, int N, const double* d1, const double* dmu,
                                   double* scal, double* w) {
  response_finish_kernel<<<1, 1024, 0, s>>>(nat, N, d1, dmu, scal, w);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_absmax(cudaStream_t s, int n, const double* x, double* out) {
  absmax_kernel<<<1, 1024, 0, s>>>(n, x, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_history(cudaStream_t s, int nat, int kmax, double* nh) {
  fill_history_kernel<<<blocks_for(nat, 128), 128, 0, s>>>(nat, kmax, nh);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_axpy(cudaStream_t s, int n, double a, const double* x, double* y) {
  axpy_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, a, x, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_diag_sum(cudaStream_t s, int n, int np, const double* X, double* out) {
  diag_sum_kernel<<<1, 1024, 0, s>>>(n, np, X, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_density_out_f64(cudaStream_t s, int N, int np, const double* Tn, const double* Tmu, double dmu,
                                   double* ddiag, double* D) {
  density_out_kernel<<<blocks_for((size_t)np * np, 256), 256, 0, s>>>(N, np, Tn, Tmu, dmu, ddiag, D);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_t0_init(cudaStream_t s, int n, int np, const double* H, double mu, double scale, double* T0) {
  t0_init_kernel<<<blocks_for((size_t)np * np, 256), 256, 0, s>>>(n, np, H, mu, scale, T0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ident_minus(cudaStream_t s, int np, const double* S, double* Y) {
  ident_minus_kernel<<<blocks_for((size_t)np * np, 256), 256, 0, s>>>(np, S, Y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(cudaStream_t s, size_t count, double c, const double* X, double* Y) {
  scale_kernel<<<blocks_for(count, 256), 256, 0, s>>>(count, c, X, Y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_level0_A1(cudaStream_t s, int np, const double* T0, const double* d, double* A1) {
  level0_A1_kernel<<<blocks_for((size_t)np * np, 256), 256, 0, s>>>(np, T0, d, A1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_transpose_add(cudaStream_t s, int np, const double* G, double* A1) {
  if (np % 32) return cudaErrorInvalidValue;
  dim3 grid(np / 32, np / 32), block(32, 8);
  transpose_add_kernel<<<grid, block, 0, s>>>(np, G, A1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_row_dot(cudaStream_t s, int n, int np, const double* Y, const double* M, double* out) {
  row_dot_kernel<<<(n + 7) / 8, 256, 0, s>>>(n, np, Y, M, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_get_diag(cudaStream_t s, int n, int np, const double* X, double* out) {
  get_diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, np, X, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sum(cudaStream_t s, int n, const double* x, double* out) {
  sum_kernel<<<1, 1024, 0, s>>>(n, x, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_frob_dot(cudaStream_t s, int n, int np, const double* A, const double* B, double* work,
                            double* out) {
  const int nb = n < 1024 ? n : 1024;
  frob_partial_kernel<<<nb, 256, 0, s>>>(n, np, A, B, work);
  note_launch();
  sum_kernel<<<1, 1024, 0, s>>>(nb, work, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_kernel_vec(cudaStream_t s, int mode, int nat, int m, double c, const double* r, double* V,
                              const double* W, double* out, double* flag) {
  kernel_vec_kernel<<<1, 1024, 0, s>>>(mode, nat, m, c, r, V, W, out, flag);
  note_launch();
  return cudaGetLastError();
}


// ---- exact kernel K = (J - I)^-1 (Eq. KK) ----

namespace {

__global__ void unit_vector_kernel(int n, int i, double* __restrict__ v) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) v[a] = (a == i) ? 1.0 : 0.0;
}

// A[a][col] = w[a] - delta(a, col): column col of J - I (row-major n x n); B = I alongside
__global__ void jacobian_column_kernel(int n, int col, const double* __restrict__ w, double* __restrict__ A,
                                       double* __restrict__ B) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  A[(size_t)a * n + col] = w[a] - (a == col ? 1.0 : 0.0);
  B[(size_t)a * n + col] = (a == col) ? 1.0 : 0.0;
}

// Gauss-Jordan step k, part 1 (one CTA): partial pivot of column k over rows k..n-1,
// swap of rows k and p in A and B, scaling of row k by 1 / A_kk, and the elimination
// factors f_i = A_ik (f_k = 0) copied out so that part 2 reads no column it writes.
__global__ void gj_pivot_kernel(int n, int k, double* __restrict__ A, double* __restrict__ B,
                                double* __restrict__ f, double* __restrict__ flag) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  double best = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[(size_t)i * n + k]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sv[wid] = best;
    si[wid] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int p = k;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < p)) {
        b = sv[w];
        p = si[w];
      }
    s_p = p;
  }
  __syncthreads();
  const int p = s_p;
  if (p != k)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double ta = A[(size_t)k * n + j], tb = B[(size_t)k * n + j];
      A[(size_t)k * n + j] = A[(size_t)p * n + j];
      B[(size_t)k * n + j] = B[(size_t)p * n + j];
      A[(size_t)p * n + j] = ta;
      B[(size_t)p * n + j] = tb;
    }
  __syncthreads();
  const double piv = A[(size_t)k * n + k];
  const bool bad = !(fabs(piv) > 0.0) || !isfinite(piv);
  __syncthreads();   // every thread has read the pivot before row k is scaled
  if (bad) {
    if (threadIdx.x == 0) *flag = 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = 0.0;
    return;
  }
  const double inv = 1.0 / piv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    A[(size_t)k * n + j] *= inv;
    B[(size_t)k * n + j] *= inv;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = (i == k) ? 0.0 : A[(size_t)i * n + k];
}

// Gauss-Jordan step k, part 2: row_i -= f_i row_k for every i != k, over A's columns >= k
// (the columns left of k are already those of the identity) and all of B's.
__global__ void gj_eliminate_kernel(int n, int k, double* __restrict__ A, double* __restrict__ B,
                                    const double* __restrict__ f) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == k || j >= 2 * n) return;
  const double fi = f[i];
  if (fi == 0.0) return;
  if (j < n) {
    if (j >= k) A[(size_t)i * n + j] -= fi * A[(size_t)k * n + j];
  } else {
    const int c = j - n;
    B[(size_t)i * n + c] -= fi * B[(size_t)k * n + c];
  }
}

}  // namespace

cudaError_t launch_unit_vector(cudaStream_t s, int n, int i, double* v) {
  unit_vector_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, i, v);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_jacobian_column(cudaStream_t s, int n, int col, const double* w, double* A, double* B) {
  jacobian_column_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, col, w, A, B);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(cudaStream_t s, int n, double* A, double* B, double* f, double* flag) {
  if (n < 1 || n > 65535) return cudaErrorInvalidValue;
  const dim3 grid((2 * n + 255) / 256, n);
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, s>>>(n, k, A, B, f, flag);
    note_launch();
    gj_eliminate_kernel<<<grid, 256, 0, s>>>(n, k, A, B, f);
    note_launch();
  }
  return cudaGetLastError();
}


// ---- accumulated rank-1 kernel (one Sherman-Morrison update per step) ----

namespace {

__global__ void scaled_identity_kernel(int n, double a, double* __restrict__ M) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  M[idx] = (idx / n == idx % n) ? a : 0.0;
}

// y_j = sum_i M_ij x_i (row-major n x n; one thread per column, coalesced over j)
__global__ void gemv_t_kernel(int n, const double* __restrict__ M, const double* __restrict__ x,
                              double* __restrict__ y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += M[(size_t)i * n + j] * x[i];
  y[j] = acc;
}

// v <- v / |v|; flag = 1 when |v| is positive and finite, else 0 (v untouched)
__global__ void normalize_kernel(int n, double* __restrict__ v, double* __restrict__ flag) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += v[i] * v[i];
  a = sqrt(block_sum(a, sh));
  const bool ok = a > 0.0 && isfinite(a);
  if (ok)
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] /= a;
  if (threadIdx.x == 0) *flag = ok ? 1.0 : 0.0;
}

// u = w - t;  out = 1 + v . Ku is formed later by dot1p_kernel
__global__ void sub_kernel(int n, const double* __restrict__ w, const double* __restrict__ t, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] = w[i] - t[i];
}

__global__ void dot1p_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                             double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += a[i] * b[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = 1.0 + acc;
}

// J += u v^T;  K -= (K u)(v^T K) / (1 + v^T K u)
__global__ void rank1_update_kernel(int n, const double* __restrict__ u, const double* __restrict__ v,
                                    const double* __restrict__ Ku, const double* __restrict__ vK,
                                    const double* __restrict__ denom, double* __restrict__ J, double* __restrict__ K) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  J[idx] += u[i] * v[j];
  K[idx] -= Ku[i] * vK[j] / *denom;
}

inline unsigned blocks_for(size_t count) { return (unsigned)((count + 255) / 256); }

}  // namespace

cudaError_t launch_scaled_identity(cudaStream_t s, int n, double a, double* M) {
  scaled_identity_kernel<<<blocks_for((size_t)n * n), 256, 0, s>>>(n, a, M);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemv_t(cudaStream_t s, int n, const double* M, const double* x, double* y) {
  gemv_t_kernel<<<blocks_for(n), 256, 0, s>>>(n, M, x, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_normalize(cudaStream_t s, int n, double* v, double* flag) {
  normalize_kernel<<<1, 1024, 0, s>>>(n, v, flag);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sub(cudaStream_t s, int n, const double* w, const double* t, double* u) {
  sub_kernel<<<blocks_for(n), 256, 0, s>>>(n, w, t, u);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dot1p(cudaStream_t s, int n, const double* a, const double* b, double* out) {
  dot1p_kernel<<<1, 1024, 0, s>>>(n, a, b, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rank1_update(cudaStream_t s, int n, const double* u, const double* v, const double* Ku,
                                const double* vK, const double* denom, double* J, double* K) {
  rank1_update_kernel<<<blocks_for((size_t)n * n), 256, 0, s>>>(n, u, v, Ku, vK, denom, J, K);
  note_launch();
  return cudaGetLastError();
}

}  // namespace xl
