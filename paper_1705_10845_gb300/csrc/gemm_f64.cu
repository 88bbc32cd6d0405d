// FP64 matrix products of the plain-FP64 path: C = epi(A * B^T).
//
// GB300 runs FP64 on its CUDA cores only (no FP64 tensor path), so this is a
// plain shared-memory tiled SIMT kernel: 64x64 output tiles, 256 threads, a
// 4x4 register tile per thread with strided rows/columns (conflict-free
// shared-memory reads, coalesced stores), K staged 16 at a time.
#include "internal.h"

namespace xl {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool SYM>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int M, int N, int K, const double* __restrict__ A,
                                                       int lda, const double* __restrict__ B, int ldb,
                                                       double* __restrict__ C, int ldc, EpiF64 e) {
  int bi, bj;
  if (SYM) {
    // upper-triangular tile index -> (bi, bj), bj >= bi
    const int nt = N / BN;
    int t = blockIdx.x, r = 0;
    while (t >= nt - r) {
      t -= nt - r;
      ++r;
    }
    bi = r;
    bj = r + t;
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
  }
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double* Ab = A + (size_t)bi * BM * lda;
  const double* Bb = B + (size_t)bj * BN * ldb;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int el = tid + 256 * r, row = el >> 4, col = el & 15;
      As[col][row] = Ab[(size_t)row * lda + k0 + col];
      Bs[col][row] = Bb[(size_t)row * ldb + k0 + col];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = bi * BM + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = bj * BN + tx + 16 * j;
      if (SYM && bi == bj && row > col) continue;
      double v = e.alpha * acc[i][j];
      if (e.E) v += e.beta * e.E[(size_t)row * e.lde + col];
      if (row == col) {
        v += e.diag;
        if (e.dvec && row < e.ndvec) v += e.dvec_scale * e.dvec[row];
      }
      C[(size_t)row * ldc + col] = v;
      if (SYM && row != col) C[(size_t)col * ldc + row] = v;
    }
  }
}

}  // namespace

cudaError_t gemm_f64_nt(cudaStream_t s, int M, int N, int K, const double* A, int lda, const double* B,
                        int ldb, double* C, int ldc, const EpiF64& e, bool sym) {
  if (M % BM || N % BN || K % BK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if (sym) {
    if (M != N) return cudaErrorInvalidValue;
    const int nt = N / BN;
    gemm_f64_kernel<true><<<nt * (nt + 1) / 2, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    note_launch();
  } else {
    dim3 grid(N / BN, M / BM);
    gemm_f64_kernel<false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, e);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace xl
