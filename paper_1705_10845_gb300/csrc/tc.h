// Tensor-core split-precision product (gemm_tc.cu) interface.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

namespace xl {

struct TcArgs {
  int K = 0;                      // inner dimension (set by gemm_tc)
  int n = 0;                      // matrix size (set by gemm_tc)
  int split_acc = 0;              // one-CTA-per-tile kernel: 1 = the hi*hi K blocks split over both
                                  // accumulators (below)
  int bn = 0;                     // grouped products: tile width 128 or 256 (0: 256 where n is a
                                  // multiple of 256, else 128)
  int chunk_kb = 0;               // persistent kernel, split products: the hi*hi sum is accumulated in
                                  // chunks of this many K blocks, folded in FP32 (0: one chunk)
  int nseg = 3;                   // 1: hi only; 3: hi*hi + hi*lo + lo*hi
  int pairs = 1;                  // 2: C = A B^T + B A^T (the swapped pair as a second K range)
  int sym = 0;                    // symmetric output (upper tiles, mirrored)
  int fmt = 0;                    // operand type: 0 FP16, 1 BF16 (kind::f16), 2 TF32 (kind::tf32,
                                  // FP32 words; persistent kernel only)
  int tiles_n = 0;                // set by gemm_tc
  const int* tile_list = nullptr; // set by gemm_tc
  float alpha = 1.0f;             // C = alpha acc / (sa sb) + beta E^T + beta2 E2^T + beta64 E64(^T)
  const float* E = nullptr;       //     + diag I + dvec_scale diag(dvec); E and E2 are read
                                  //     transposed (callers pass symmetric side inputs)
  float beta = 0.0f;
  const float* E2 = nullptr;
  float beta2 = 0.0f;
  const float2* E64 = nullptr;    // double-float side input, read transposed when e64_trans
  float beta64 = 0.0f;            // a power of two, so that beta64 E64 is exact
  int e64_trans = 0;
  float2* C64 = nullptr;          // double-float output (written instead of C when set)
  float diag = 0.0f;
  const double* dvec = nullptr;
  int ndvec = 0;
  float dvec_scale = 1.0f;
  float* C = nullptr;
  int ldc = 0;
  unsigned* amax = nullptr;       // max |C| (float bits), atomically raised
  const float* sa = nullptr;      // operand scales (device scalars)
  const float* sb = nullptr;
  int* err = nullptr;             // set non-zero when a bounded wait gives up
};

// One problem of a grouped product launch, in device memory: its tensor maps (A hi, A lo, B hi,
// B lo, and the swapped pair's A2 hi, A2 lo, B2 hi, B2 lo) and its epilogue arguments.  The
// problems of a group share n, the segment and pair counts, the symmetric mode and the operand
// type; they differ in their matrices and scalars.
struct TcEntry {   // CUtensorMap's own alignment (64 bytes) aligns every entry
  CUtensorMap map[8];
  TcArgs args;
};

// One problem of a grouped product: operands and its epilogue arguments (n, K, nseg, pairs,
// sym, fmt, chunk_kb and err come from the launch's shared arguments).
struct TcProblem {
  const void *Ahi = nullptr, *Alo = nullptr, *Bhi = nullptr, *Blo = nullptr;   // operand arrays (n x n, row-major)
  TcArgs epi;
};

// Device tile lists of the symmetric-output products of one size n (pairs of ints (tm, tn)):
// 128 x 128 tiles, 128 x 256 tiles (n a multiple of 256) and 256 x 256 tiles of the two-SM
// products (n a multiple of 256; null: two-SM products are not used for this size).
struct TcTiles {
  const int* sym128 = nullptr;
  int n128 = 0;
  const int* sym256 = nullptr;
  int n256 = 0;
  const int* pair = nullptr;
  int npair = 0;
};

// n x n product (n a multiple of 128); the symmetric tile lists come from tc_sym_tiles and
// tc_sym_tiles_pair.
cudaError_t gemm_tc(cudaStream_t s, int n, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo,
                    TcArgs args, const TcTiles& tiles);
// Grouped product: the problems' tiles in one persistent launch (one-SM kernel).  The device
// table of each distinct problem list is built once and kept in `cache` (key: the table's
// bytes), so repeated groups upload nothing.
struct TcGroupCache;
TcGroupCache* tc_group_cache_new();
void tc_group_cache_free(TcGroupCache* c);
cudaError_t gemm_tc_group(cudaStream_t s, int n, const TcProblem* probs, int nprob, TcArgs shared,
                          const TcTiles& tiles, TcGroupCache* cache);
std::vector<int> tc_sym_tiles(int n, int bn);
std::vector<int> tc_sym_tiles_pair(int n);
void tc_forget_maps(const void* base);

}  // namespace xl
