// Split-precision engine: the expansion and response chains with tensor-core
// products on hi/lo operand pairs (FP16x3, BF16x3 or TF32x3).
//
// Every matrix keeps a value array -- FP32, or double-float (an FP32 hi + lo
// pair) for T_k, M and T1, whose leading terms the correction form keeps out of
// the products -- and a split operand pair hi = rn(x s), lo = rn(x s - hi)
// (rn: rounding to FP16, BF16 or TF32) with a power-of-two scale s chosen from
// max |x| so that max |x s| lies in [2^10, 2^11) (FP16 keeps full precision in
// both parts); producers raise max |x| atomically and a conversion pass writes
// hi/lo.  A product takes three tensor-core products (hi*hi, hi*lo, lo*hi), or
// one (hi*hi) in the probe chains and the mu chain when the context asks for
// it.  Traces, charges and the density matrix handed to the forces are
// accumulated in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <unordered_map>

#include "precision.h"
#include "tc.h"

namespace xl {
namespace {

#define RET(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

inline unsigned nblk(size_t count, int tpb = 256) { return (unsigned)((count + tpb - 1) / tpb); }

// element-wise kernels that raise a matrix's max |x| walk their elements grid-stride with at
// most this many blocks, so that each launch issues few atomics on the one max
constexpr unsigned kEwBlocks = 152 * 16;

// One-CTA-per-tile product kernel: products of at least this size split their hi*hi sums over
// both accumulators.
constexpr int kSplitAccMin = 8192;
// Persistent product kernel, split products: the hi*hi sum is accumulated in chunks of this many
// 64-wide K blocks of 16-bit operands (K = 1024; the same K with TF32's 32-wide blocks), each folded
// into the running sum with round-to-nearest FP32 adds.
// The tensor core truncates as it accumulates, so a sum's error grows with its length: at 2048
// atoms (N = 8192) the charge error fell from 4.7e-5 e (one 8192-long sum) to 2.5e-5 e (two
// halves), and it keeps halving with the chunk length.
constexpr int kChunkKb = 16;

// Raise *amax to the block's max |v| with one atomic per block (all threads
// of the block must call it).
__device__ __forceinline__ void raise_amax(unsigned* amax, float v) {
  __shared__ float wmax[32];
  v = fabsf(v);
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) wmax[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    float m = 0.0f;
    for (int w = 0; w < (nthr + 31) / 32; ++w) m = fmaxf(m, wmax[w]);
    atomicMax(amax, __float_as_uint(m));
  }
}

// Operand words: FP16 or BF16 in 16 bits, TF32 in an FP32 word whose low 13 mantissa bits are
// zero (fmt 0, 1, 2).
template <int FMT>
struct OpWord {
  using T = unsigned short;
  using V4 = ushort4;
};
template <>
struct OpWord<2> {
  using T = unsigned;
  using V4 = uint4;
};

// Round x to the operand format; v receives the rounded value.  TF32 rounding (to 10 explicit
// mantissa bits, nearest, ties away from zero) is the cvt.rna.tf32.f32 instruction.
template <int FMT>
__device__ __forceinline__ typename OpWord<FMT>::T op_round(float x, float& v) {
  if constexpr (FMT == 2) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    v = __uint_as_float(r);
    return r;
  } else if constexpr (FMT == 1) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    v = __bfloat162float(b);
    return __bfloat16_as_ushort(b);
  } else {
    const __half h = __float2half_rn(x);
    v = __half2float(h);
    return __half_as_ushort(h);
  }
}

// Four operand words at index i (16-byte groups for TF32, 8-byte for 16-bit words).
template <int FMT>
__device__ __forceinline__ void store4(void* base, size_t i, const typename OpWord<FMT>::T (&w)[4]) {
  using V4 = typename OpWord<FMT>::V4;
  V4 v;
  v.x = w[0];
  v.y = w[1];
  v.z = w[2];
  v.w = w[3];
  reinterpret_cast<V4*>(base)[i] = v;
}

// Conversion of four values to the split operand pair: hi = rn(x s), lo = rn((x s - hi) + xl s)
// (xl: the low word of a double-float value, else 0; s is a power of two, so x s is exact).
// MODE 0: FP32 value -> hi, lo; 1: double-float value -> hi, lo; 2: FP32 value -> hi.
template <int FMT, int MODE>
__device__ __forceinline__ void convert4(size_t i, float s, const float* __restrict__ f, const float2* __restrict__ d,
                                         void* hi, void* lo) {
  float xs[4], xl[4] = {0.f, 0.f, 0.f, 0.f};
  if (MODE == 1) {
    const float4* d4 = reinterpret_cast<const float4*>(d);   // two double-float values per float4
    const float4 a = d4[2 * i], b = d4[2 * i + 1];
    xs[0] = a.x * s; xs[1] = a.z * s; xs[2] = b.x * s; xs[3] = b.z * s;
    xl[0] = a.y * s; xl[1] = a.w * s; xl[2] = b.y * s; xl[3] = b.w * s;
  } else {
    const float4 x = reinterpret_cast<const float4*>(f)[i];
    xs[0] = x.x * s; xs[1] = x.y * s; xs[2] = x.z * s; xs[3] = x.w * s;
  }
  typename OpWord<FMT>::T h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float hv, lv;
    h[k] = op_round<FMT>(xs[k], hv);
    if (MODE == 1) l[k] = op_round<FMT>((xs[k] - hv) + xl[k], lv);
    if (MODE == 0) l[k] = op_round<FMT>(xs[k] - hv, lv);
  }
  store4<FMT>(hi, i, h);
  if (MODE != 2) store4<FMT>(lo, i, l);
}

// The operand scale from max |x|: a power of two that puts max |x s| in [2^10, 2^11) (FP16
// keeps full precision in both parts; BF16 and TF32 have FP32's range and lose nothing by it).
__device__ __forceinline__ float operand_scale(const unsigned* amax) {
  const float m = __uint_as_float(*amax);
  return (m > 0.0f && isfinite(m)) ? ldexpf(1.0f, 10 - ilogbf(m)) : 1.0f;
}

// One matrix: all threads derive the same scale from amax; thread 0 of block 0 publishes it.
// Four elements per thread and step (count is a multiple of 4).
template <int FMT, int MODE>
__global__ void convert_kernel(size_t count, const float* __restrict__ f, const float2* __restrict__ d,
                               const unsigned* __restrict__ amax, void* hi, void* lo, float* __restrict__ scale) {
  const float s = operand_scale(amax);
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = s;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += (size_t)gridDim.x * blockDim.x)
    convert4<FMT, MODE>(i, s, f, d, hi, lo);
}

__global__ void df_to_f64_kernel(size_t count, const float2* __restrict__ x, double* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = (double)x[i].x + (double)x[i].y;
}

// dst = I - W (W an FP32 value, dst FP64)
__global__ void ident_minus_f32_to_f64_kernel(size_t count, int np, const float* __restrict__ W,
                                              double* __restrict__ dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int r = (int)(i / np), c = (int)(i % np);
  dst[i] = (r == c ? 1.0 : 0.0) - (double)W[i];
}

__device__ __forceinline__ double df_val(float2 v) { return (double)v.x + (double)v.y; }

__global__ void diag_sum_d_kernel(int n, int np, const float2* __restrict__ X, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += df_val(X[(size_t)i * np + i]);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void density_out_d_kernel(int N, int np, const float2* __restrict__ Tn, const float2* __restrict__ Tmu,
                                     double dmu, double* __restrict__ ddiag, double* __restrict__ D) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)np * np) return;
  const int i = (int)(idx / np), j = (int)(idx % np);
  double v = 0.0;
  if (i < N && j < N) {
    v = 0.5 * (df_val(Tn[idx]) + dmu * df_val(Tmu[idx]) + (i == j ? 1.0 : 0.0));
    if (i == j) ddiag[i] = 2.0 * v;
  }
  D[idx] = v;
}

// ---- grouped element-wise kernels ----
//
// Batched trajectories step in lockstep: the same element-wise operation runs on the matrices
// of every system of a group in one launch, blockIdx.y selecting the system.  The per-system
// pointers travel by value in the kernel parameters (at most kMaxGroup systems per launch).
constexpr int kMaxGroup = 64;

struct MatList {
  int n = 0;
  float* f[kMaxGroup];
  float2* d[kMaxGroup];
  void* hi[kMaxGroup];
  void* lo[kMaxGroup];
  float* scale[kMaxGroup];
  unsigned* amax[kMaxGroup];
};

__global__ void zero_amax_kernel(MatList L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.n) *L.amax[i] = 0u;
}

// convert_kernel per system (blockIdx.y)
template <int FMT, int MODE>
__global__ void convert_group_kernel(size_t count, MatList L) {
  const int j = blockIdx.y;
  const float s = operand_scale(L.amax[j]);
  if (blockIdx.x == 0 && threadIdx.x == 0) *L.scale[j] = s;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += (size_t)gridDim.x * blockDim.x)
    convert4<FMT, MODE>(i, s, L.f[j], L.d[j], L.hi[j], L.lo[j]);
}

// Y = a I + b X per system (W_k start of the Newton-Schulz iteration)
struct AxpiList {
  int n = 0;
  const float* X[kMaxGroup];
  float* Y[kMaxGroup];
  unsigned* amax[kMaxGroup];
  float a[kMaxGroup], b[kMaxGroup];
  const double* dc[kMaxGroup];   // device c (a = 1 - c, b = c) when not null
};

__global__ void axpi_group_kernel(int np, AxpiList L) {
  const int j = blockIdx.y;
  float a = L.a[j], b = L.b[j];
  if (L.dc[j]) {
    a = (float)(1.0 - L.dc[j][0]);
    b = (float)L.dc[j][0];
  }
  const size_t count = (size_t)np * np;
  const float* X = L.X[j];
  float* Y = L.Y[j];
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / np), c = (int)(idx % np);
    const float v = b * X[idx] + (r == c ? a : 0.0f);
    Y[idx] = v;
    m = fmaxf(m, fabsf(v));
  }
  raise_amax(L.amax[j], m);
}

// T0 = -sc (H - mu I) as a double-float, per system
struct T0List {
  int n = 0;
  int N[kMaxGroup];
  const double* H[kMaxGroup];
  double mu[kMaxGroup];
  const double* dmu[kMaxGroup];
  float2* T0[kMaxGroup];
  unsigned* amax[kMaxGroup];
};

__global__ void t0_init_group_kernel(int np, double sc, T0List L) {
  const int j = blockIdx.y;
  const double mu = L.dmu[j] ? L.dmu[j][0] : L.mu[j];
  const int n = L.N[j];
  const double* H = L.H[j];
  float2* T0 = L.T0[j];
  const size_t count = (size_t)np * np;
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / np), c = (int)(idx % np);
    double v = 0.0;
    if (r < n && c < n) v = -sc * (H[idx] - (r == c ? mu : 0.0));
    const float vh = (float)v;
    T0[idx] = make_float2(vh, (float)(v - (double)vh));
    m = fmaxf(m, fabsf(vh));
  }
  raise_amax(L.amax[j], m);
}

// A1 of chain level 0 per system: (T0 hi + lo)(d_i + d_j)
struct A1List {
  int n = 0;
  const float2* T0[kMaxGroup];
  const double* d[kMaxGroup];
  float* A1[kMaxGroup];
  unsigned* amax[kMaxGroup];
};

__global__ void level0_A1_group_kernel(int np, A1List L) {
  const int j = blockIdx.y;
  const float2* T0 = L.T0[j];
  const double* d = L.d[j];
  float* A1 = L.A1[j];
  const size_t count = (size_t)np * np;
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / np), c = (int)(idx % np);
    const float2 t = T0[idx];
    const float v = (t.x + t.y) * (float)(d[r] + d[c]);
    A1[idx] = v;
    m = fmaxf(m, fabsf(v));
  }
  raise_amax(L.amax[j], m);
}

// Diagonal reductions of the chains' last level, per system
struct DiagList {
  int n = 0;
  int N[kMaxGroup];
  const float* W[kMaxGroup];    // row_dot: W_k (FP32)
  const float2* X[kMaxGroup];   // row_dot: M^T; get_diag: T1_n (double-float)
  double* out[kMaxGroup];
};

// out_i = (Y M)_ii = Mt_ii - sum_j W_ij Mt_ij  (Y = I - W, Mt = M^T), one warp per row
__global__ void row_dot_last_group_kernel(int np, DiagList L) {
  const int j = blockIdx.y;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= L.N[j]) return;
  const float* W = L.W[j];
  const float2* Mt = L.X[j];
  float accf = 0.0f;
  double acc = 0.0;
  for (int c = lane, t = 0; c < np; c += 32, ++t) {
    const float2 mm = Mt[(size_t)i * np + c];
    accf += W[(size_t)i * np + c] * (mm.x + mm.y);
    if ((t & 15) == 15) {
      acc += (double)accf;
      accf = 0.0f;
    }
  }
  acc += (double)accf;
  acc = warp_sum(acc);
  if (lane == 0) L.out[j][i] = df_val(Mt[(size_t)i * np + i]) - acc;
}

__global__ void get_diag_group_kernel(int np, DiagList L) {
  const int j = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.N[j]) L.out[j][i] = df_val(L.X[j][(size_t)i * np + i]);
}

// Epilogue options of one split product.  The FP32 side inputs E, E2 are
// read transposed by the product kernel, so they must be symmetric (S, W and
// the Newton-Schulz residual Q, whose rounding asymmetry the iteration
// removes).
struct Epi {
  float alpha = 1.0f;
  const SplitMat* E = nullptr;
  float beta = 0.0f;
  const SplitMat* E2 = nullptr;
  float beta2 = 0.0f;
  const float2* E64 = nullptr;
  float beta64 = 0.0f;
  int e64_trans = 0;
  float diag = 0.0f;
  const double* dvec = nullptr;
  float dvec_scale = 1.0f;
  bool out64 = false;       // write C.d (and convert from it) instead of C.f
  bool convert = true;      // produce the split operand pair of C
  bool hi_only = false;     // produce only the hi operand (C enters single products only)
  int nseg = 3;             // 3: hi*hi + hi*lo + lo*hi; 1: hi*hi only
  int pairs = 1;            // 2: C = A B^T + B A^T
};

// The recursion is carried in correction form so that its exact leading
// terms never pass through the rounded operands:
//   T_{k+1} = 2 T_k - 2 T_k W_k,  W_k = I - Y_k = I - (I + T_k^2)^-1,
// W_k from the Newton-Schulz step written for W (Q = S - W - W S,
// W <- W + Q - Q W), and the response chains as
//   M = 2 T1_k - A1 T_{k+1},  T1_{k+1} = M - W_k M.
// T_k, M and T1_k are FP64 values; W, S, Q, A1 FP32 values; every product
// operand is the hi/lo split of a value.
class EngineSplit : public Engine {
 public:
  explicit EngineSplit(int prec) : fmt_(operand_fmt(prec)) {}
  ~EngineSplit() override {
    for (auto& kv : tiles_) cudaFree(kv.second.first);
    if (err_) cudaFree(err_);
    tc_group_cache_free(group_cache_);
  }

  // operand split of one matrix: mode 0 FP32 -> hi, lo; 1 double-float -> hi, lo; 2 FP32 -> hi
  template <int FMT>
  void launch_convert(cudaStream_t s, SplitMat& m, size_t count, unsigned g, int mode) {
    if (mode == 0) convert_kernel<FMT, 0><<<g, 256, 0, s>>>(count, m.f, m.d, m.amax, m.hi, m.lo, m.scale);
    else if (mode == 1) convert_kernel<FMT, 1><<<g, 256, 0, s>>>(count, m.f, m.d, m.amax, m.hi, m.lo, m.scale);
    else convert_kernel<FMT, 2><<<g, 256, 0, s>>>(count, m.f, m.d, m.amax, m.hi, m.lo, m.scale);
  }

  cudaError_t convert_mode(cudaStream_t s, SplitMat& m, int np, int mode) {
    const size_t count = (size_t)np * np;
    const unsigned g = std::min<size_t>(nblk(count), 152 * 16);
    if (fmt_ == 2)
      launch_convert<2>(s, m, count, g, mode);
    else if (fmt_ == 1)
      launch_convert<1>(s, m, count, g, mode);
    else
      launch_convert<0>(s, m, count, g, mode);
    note_launch();
    return cudaGetLastError();
  }
  cudaError_t convert(cudaStream_t s, SplitMat& m, int np) { return convert_mode(s, m, np, 0); }
  cudaError_t convert_d(cudaStream_t s, SplitMat& m, int np) { return convert_mode(s, m, np, 1); }
  cudaError_t convert_hi(cudaStream_t s, SplitMat& m, int np) { return convert_mode(s, m, np, 2); }

  // Symmetric-product tile lists for size np, uploaded on the stream that uses them (the
  // context's stream may be non-blocking, so a legacy-stream copy would not be ordered
  // before the first product).
  cudaError_t prep_tiles(int np, cudaStream_t s) {
    if (tiles_.count(np)) return cudaSuccess;
    const bool wide = (np % 256 == 0);
    std::vector<int> t128 = tc_sym_tiles(np, 128), t256 = wide ? tc_sym_tiles(np, 256) : std::vector<int>();
    std::vector<int> tp = wide ? tc_sym_tiles_pair(np) : std::vector<int>();
    std::vector<int> all(t128);
    all.insert(all.end(), t256.begin(), t256.end());
    all.insert(all.end(), tp.begin(), tp.end());
    int* d = nullptr;
    RET(cudaMalloc((void**)&d, sizeof(int) * std::max<size_t>(all.size(), 2)));
    RET(cudaMemcpyAsync(d, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, s));
    TcTiles t;
    t.sym128 = d;
    t.n128 = (int)t128.size() / 2;
    t.sym256 = d + t128.size();
    t.n256 = (int)t256.size() / 2;
    t.pair = wide ? d + t128.size() + t256.size() : nullptr;
    t.npair = (int)tp.size() / 2;
    tiles_[np] = {d, t};
    if (!err_) {
      RET(cudaMalloc((void**)&err_, sizeof(int)));
      RET(cudaMemsetAsync(err_, 0, sizeof(int), s));
    }
    return cudaStreamSynchronize(s);   // `all` is a host temporary
  }

  cudaError_t gemm(cudaStream_t s, int np, const SplitMat& A, const SplitMat& B, SplitMat& C, const Epi& e,
                   bool sym, double* stats) {
    RET(prep_tiles(np, s));
    const TcTiles& tl = tiles_[np].second;
    RET(cudaMemsetAsync(C.amax, 0, sizeof(unsigned), s));
    TcArgs a;
    a.nseg = e.nseg;
    a.pairs = e.pairs;
    a.sym = sym ? 1 : 0;
    a.fmt = fmt_;
    a.alpha = e.alpha;
    a.E = e.E ? e.E->f : nullptr;
    a.beta = e.beta;
    a.E2 = e.E2 ? e.E2->f : nullptr;
    a.beta2 = e.beta2;
    a.E64 = e.E64;
    a.beta64 = e.beta64;
    a.e64_trans = e.e64_trans;
    a.diag = e.diag;
    a.dvec = e.dvec;
    a.ndvec = e.dvec ? np : 0;
    a.dvec_scale = e.dvec_scale;
    a.C = e.out64 ? nullptr : C.f;
    a.C64 = e.out64 ? C.d : nullptr;
    a.ldc = np;
    a.amax = C.amax;
    a.sa = A.scale;
    a.sb = B.scale;
    a.err = err_;
    RET(prof_begin(s));
    // large products: split the hi*hi sums over both accumulators (the tensor core truncates as it
    // accumulates, so a K-long sum's error grows with K)
    a.split_acc = (np >= kSplitAccMin) ? 1 : 0;
    a.chunk_kb = chunk_kb();
    RET(gemm_tc(s, np, A.hi, A.lo, B.hi, B.lo, a, tl));
    // kind bits: 1 sym, 2 E, 4 E2, 8 E64, 16 E64 transposed, 32 FP64 output
    const int kind = (sym ? 1 : 0) | (e.E ? 2 : 0) | (e.E2 ? 4 : 0) | (e.E64 ? 8 : 0) | (e.e64_trans ? 16 : 0) |
                     (e.out64 ? 32 : 0);
    RET(prof_end(s, 2.0 * (double)np * np * np * (sym ? 0.5 : 1.0) * e.pairs, kind));
    if (stats) stats[3] += (sym ? 0.5 : 1.0) * e.pairs;
    if (!e.convert) return cudaSuccess;
    if (e.hi_only && !e.out64) return convert_hi(s, C, np);
    return e.out64 ? convert_d(s, C, np) : convert(s, C, np);
  }

  // ---- grouped operations (one launch over the systems of a lockstep group) ----

  struct GemmOp {
    const SplitMat* A;
    const SplitMat* B;
    SplitMat* C;
    Epi e;
    double* stats;
  };

  static MatList mat_list(const std::vector<SplitMat*>& ms) {
    MatList L;
    L.n = (int)ms.size();
    for (int i = 0; i < L.n; ++i) {
      L.f[i] = ms[i]->f;
      L.d[i] = ms[i]->d;
      L.hi[i] = ms[i]->hi;
      L.lo[i] = ms[i]->lo;
      L.scale[i] = ms[i]->scale;
      L.amax[i] = ms[i]->amax;
    }
    return L;
  }

  cudaError_t zero_amax_group(cudaStream_t s, const std::vector<SplitMat*>& ms) {
    if (ms.size() == 1) return cudaMemsetAsync(ms[0]->amax, 0, sizeof(unsigned), s);
    zero_amax_kernel<<<1, kMaxGroup, 0, s>>>(mat_list(ms));
    note_launch();
    return cudaGetLastError();
  }

  // operand split of each matrix: mode 0 FP32 -> hi, lo; 1 double-float -> hi, lo; 2 FP32 -> hi
  cudaError_t convert_group(cudaStream_t s, const std::vector<SplitMat*>& ms, int np, int mode) {
    if (ms.size() == 1) {
      if (mode == 0) return convert(s, *ms[0], np);
      if (mode == 1) return convert_d(s, *ms[0], np);
      return convert_hi(s, *ms[0], np);
    }
    const size_t count = (size_t)np * np;
    const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>(nblk(count), (152 * 16) / ms.size()));
    const dim3 grid(gx, (unsigned)ms.size());
    const MatList L = mat_list(ms);
    if (fmt_ == 2) {
      if (mode == 0) convert_group_kernel<2, 0><<<grid, 256, 0, s>>>(count, L);
      else if (mode == 1) convert_group_kernel<2, 1><<<grid, 256, 0, s>>>(count, L);
      else convert_group_kernel<2, 2><<<grid, 256, 0, s>>>(count, L);
    } else if (fmt_ == 1) {
      if (mode == 0) convert_group_kernel<1, 0><<<grid, 256, 0, s>>>(count, L);
      else if (mode == 1) convert_group_kernel<1, 1><<<grid, 256, 0, s>>>(count, L);
      else convert_group_kernel<1, 2><<<grid, 256, 0, s>>>(count, L);
    } else {
      if (mode == 0) convert_group_kernel<0, 0><<<grid, 256, 0, s>>>(count, L);
      else if (mode == 1) convert_group_kernel<0, 1><<<grid, 256, 0, s>>>(count, L);
      else convert_group_kernel<0, 2><<<grid, 256, 0, s>>>(count, L);
    }
    note_launch();
    return cudaGetLastError();
  }

  static dim3 ew_grid(size_t count, int nsys) {
    return dim3((unsigned)std::max<size_t>(1, std::min<size_t>(nblk(count), kEwBlocks / nsys)), (unsigned)nsys);
  }

  // One product per op, all in one grouped launch (ops share sym, nseg, pairs), then each C's
  // max |x| and operand split.
  cudaError_t gemm_group(cudaStream_t s, int np, std::vector<GemmOp>& ops, bool sym) {
    if (ops.empty()) return cudaSuccess;
    if (ops.size() == 1) {
      GemmOp& o = ops[0];
      return gemm(s, np, *o.A, *o.B, *o.C, o.e, sym, o.stats);
    }
    RET(prep_tiles(np, s));
    const TcTiles& tl = tiles_[np].second;
    const Epi& e0 = ops[0].e;
    std::vector<SplitMat*> outs;
    for (auto& o : ops) outs.push_back(o.C);
    RET(zero_amax_group(s, outs));
    TcArgs shared;
    shared.nseg = e0.nseg;
    shared.pairs = e0.pairs;
    shared.sym = sym ? 1 : 0;
    shared.fmt = fmt_;
    shared.split_acc = (np >= kSplitAccMin) ? 1 : 0;
    shared.chunk_kb = chunk_kb();
    shared.err = err_;
    std::vector<TcProblem> probs(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
      const GemmOp& o = ops[i];
      const Epi& e = o.e;
      TcArgs& a = probs[i].epi;
      probs[i].Ahi = o.A->hi;
      probs[i].Alo = o.A->lo;
      probs[i].Bhi = o.B->hi;
      probs[i].Blo = o.B->lo;
      a.alpha = e.alpha;
      a.E = e.E ? e.E->f : nullptr;
      a.beta = e.beta;
      a.E2 = e.E2 ? e.E2->f : nullptr;
      a.beta2 = e.beta2;
      a.E64 = e.E64;
      a.beta64 = e.beta64;
      a.e64_trans = e.e64_trans;
      a.diag = e.diag;
      a.dvec = e.dvec;
      a.ndvec = e.dvec ? np : 0;
      a.dvec_scale = e.dvec_scale;
      a.C = e.out64 ? nullptr : o.C->f;
      a.C64 = e.out64 ? o.C->d : nullptr;
      a.ldc = np;
      a.amax = o.C->amax;
      a.sa = o.A->scale;
      a.sb = o.B->scale;
      if (o.stats) o.stats[3] += (sym ? 0.5 : 1.0) * e0.pairs;
    }
    if (!group_cache_) group_cache_ = tc_group_cache_new();
    RET(tune_group(s, np, probs, shared, tl));
    shared.bn = tuned_bn_[np];
    RET(prof_begin(s));
    RET(gemm_tc_group(s, np, probs.data(), (int)probs.size(), shared, tl, group_cache_));
    const int kind = 64 | (sym ? 1 : 0) | (e0.E ? 2 : 0) | (e0.E2 ? 4 : 0) | (e0.E64 ? 8 : 0) |
                     (e0.e64_trans ? 16 : 0) | (e0.out64 ? 32 : 0);
    RET(prof_end(s, (double)ops.size() * 2.0 * (double)np * np * np * (sym ? 0.5 : 1.0) * e0.pairs, kind));
    if (!e0.convert) return cudaSuccess;
    const int mode = (e0.hi_only && !e0.out64) ? 2 : (e0.out64 ? 1 : 0);
    return convert_group(s, outs, np, mode);
  }

  // Tile-width autotuner of grouped products: the first grouped product of a size that both
  // widths can tile (n a multiple of 256) runs twice with 128-wide and twice with 256-wide
  // tiles, timed with CUDA events on the stream, and the faster width serves every later
  // grouped product of that size.  (Few large tiles leave SMs idle on small matrices; narrow
  // tiles stage more operand bytes per flop on large ones.)  The product is recomputed from the
  // same operands each time, so the tuning runs change nothing.
  cudaError_t tune_group(cudaStream_t s, int np, std::vector<TcProblem>& probs, TcArgs shared, const TcTiles& tl) {
    if (tuned_bn_.count(np)) return cudaSuccess;
    if (np % 256 != 0) {
      tuned_bn_[np] = 128;
      return cudaSuccess;
    }
    cudaEvent_t ev[3];
    for (auto& e : ev) RET(cudaEventCreate(&e));
    float ms[2] = {0.f, 0.f};
    const int widths[2] = {128, 256};
    cudaError_t rc = cudaSuccess;
    for (int w = 0; w < 2 && rc == cudaSuccess; ++w) {
      shared.bn = widths[w];
      rc = gemm_tc_group(s, np, probs.data(), (int)probs.size(), shared, tl, group_cache_);   // warm-up
      if (rc == cudaSuccess) rc = cudaEventRecord(ev[0], s);
      if (rc == cudaSuccess) rc = gemm_tc_group(s, np, probs.data(), (int)probs.size(), shared, tl, group_cache_);
      if (rc == cudaSuccess) rc = cudaEventRecord(ev[1], s);
      if (rc == cudaSuccess) rc = cudaEventSynchronize(ev[1]);
      if (rc == cudaSuccess) rc = cudaEventElapsedTime(&ms[w], ev[0], ev[1]);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    RET(rc);
    tuned_bn_[np] = (ms[0] < ms[1]) ? 128 : 256;
    if (const char* d = std::getenv("XLBOMD_DEBUG"))
      if (d[0] && d[0] != '0')
        std::fprintf(stderr, "[xlbomd] tile autotuner n %d, %zu problems: 128-wide %.3f ms, 256-wide %.3f ms -> %d\n",
                     np, probs.size(), ms[0], ms[1], tuned_bn_[np]);
    return cudaSuccess;
  }

  cudaError_t foe(cudaStream_t s, MatSet& m, const double* H, int N, double mu, double sc,
                  const std::vector<int>& ns, const std::vector<double>& nc, double* stats,
                  const double* dpar) override {
    std::vector<FoeJob> jobs(1);
    jobs[0].m = &m;
    jobs[0].H = H;
    jobs[0].N = N;
    jobs[0].mu = mu;
    jobs[0].ns = &ns;
    jobs[0].nc = &nc;
    jobs[0].stats = stats;
    jobs[0].dpar = dpar;
    return foe_group(s, jobs, sc);
  }

  // The recursion of every job's system in lockstep: each product of a level is one grouped
  // launch over the jobs that need it (a job runs its own Newton-Schulz iteration count).
  cudaError_t foe_group(cudaStream_t s, std::vector<FoeJob>& jobs, double sc) override {
    const int B = (int)jobs.size();
    if (B == 0) return cudaSuccess;
    if (B > kMaxGroup) {
      for (int i = 0; i < B; i += kMaxGroup) {
        std::vector<FoeJob> part(jobs.begin() + i, jobs.begin() + std::min(B, i + kMaxGroup));
        RET(foe_group(s, part, sc));
      }
      return cudaSuccess;
    }
    const int np = jobs[0].m->np, n = jobs[0].m->n;
    for (auto& j : jobs)
      if (j.m->np != np || j.m->n != n) return cudaErrorInvalidValue;
    const size_t cnt = (size_t)np * np;
    std::vector<SplitMat*> T0s;
    T0List tl;
    tl.n = B;
    for (int i = 0; i < B; ++i) {
      FoeJob& j = jobs[i];
      T0s.push_back(&j.m->sT[0]);
      tl.N[i] = j.N;
      tl.H[i] = j.H;
      tl.mu[i] = j.mu;
      tl.dmu[i] = j.dpar;
      tl.T0[i] = j.m->sT[0].d;
      tl.amax[i] = j.m->sT[0].amax;
    }
    RET(zero_amax_group(s, T0s));
    t0_init_group_kernel<<<ew_grid(cnt, B), 256, 0, s>>>(np, sc, tl);
    note_launch();
    RET(cudaGetLastError());
    RET(convert_group(s, T0s, np, 1));
    std::vector<SplitMat*> W(B), Wn(B);
    for (int k = 0; k < n; ++k) {
      std::vector<GemmOp> ops;
      for (auto& j : jobs) ops.push_back({&j.m->sT[k], &j.m->sT[k], &j.m->sS, Epi(), j.stats});   // S = T^2
      RET(gemm_group(s, np, ops, true));
      // the Newton-Schulz iterates alternate between sY[k] and the work matrix; the start is
      // chosen by the parity of the iteration count so that W_k always ends in sY[k] (the
      // buffers every later use, and a captured graph of this pass, refer to)
      AxpiList al;
      al.n = B;
      int maxit = 0;
      for (int i = 0; i < B; ++i) {
        FoeJob& j = jobs[i];
        MatSet& m = *j.m;
        const int nsk = (*j.ns)[k];
        maxit = std::max(maxit, nsk);
        W[i] = (nsk % 2 == 1) ? &m.sYw : &m.sY[k];
        Wn[i] = (W[i] == &m.sY[k]) ? &m.sYw : &m.sY[k];
        al.Y[i] = W[i]->f;
        al.amax[i] = W[i]->amax;
        if (k == 0) {                                                             // W = S
          al.X[i] = m.sS.f;
          al.a[i] = 0.f;
          al.b[i] = 1.f;
          al.dc[i] = nullptr;
        } else {                                                                  // W = (1-c) I + c W_{k-1}
          al.X[i] = m.sY[k - 1].f;
          al.a[i] = (float)(1.0 - (*j.nc)[k]);
          al.b[i] = (float)(*j.nc)[k];
          al.dc[i] = j.dpar ? j.dpar + 1 + k : nullptr;
        }
      }
      RET(zero_amax_group(s, W));
      axpi_group_kernel<<<ew_grid(cnt, B), 256, 0, s>>>(np, al);
      note_launch();
      RET(cudaGetLastError());
      RET(convert_group(s, W, np, 0));
      for (int it = 0; it < maxit; ++it) {
        std::vector<GemmOp> oq, ow;
        std::vector<int> who;
        for (int i = 0; i < B; ++i) {
          FoeJob& j = jobs[i];
          if ((*j.ns)[k] <= it) continue;
          MatSet& m = *j.m;
          Epi eq;                                                                 // Q = S - W - W S
          eq.alpha = -1.f;
          eq.E = &m.sS;
          eq.beta = 1.f;
          eq.E2 = W[i];
          eq.beta2 = -1.f;
          oq.push_back({W[i], &m.sS, &m.sQ, eq, j.stats});
          Epi ew;                                                                 // W <- W + Q - Q W
          ew.alpha = -1.f;
          ew.E = W[i];
          ew.beta = 1.f;
          ew.E2 = &m.sQ;
          ew.beta2 = 1.f;
          ow.push_back({&m.sQ, W[i], Wn[i], ew, j.stats});
          who.push_back(i);
        }
        RET(gemm_group(s, np, oq, false));
        RET(gemm_group(s, np, ow, true));
        for (int i : who) {
          std::swap(W[i], Wn[i]);
          if (jobs[i].stats) jobs[i].stats[1] += 1;
        }
      }
      std::vector<GemmOp> ot;
      for (auto& j : jobs) {
        MatSet& m = *j.m;
        Epi et;                                                                   // T' = 2T - 2 T W
        et.alpha = -2.f;
        et.E64 = m.sT[k].d;                                                       // symmetric: read transposed
        et.e64_trans = 1;
        et.beta64 = 2.0f;
        et.out64 = true;
        ot.push_back({&m.sT[k], &m.sY[k], &m.sT[k + 1], et, j.stats});
      }
      RET(gemm_group(s, np, ot, true));
    }
    return cudaSuccess;
  }

  cudaError_t chain(cudaStream_t s, MatSet& m, const double* dvec, int N, bool full_last, double* out_diag,
                    double* stats) override {
    std::vector<ChainJob> jobs(1);
    jobs[0].m = &m;
    jobs[0].dvec = dvec;
    jobs[0].N = N;
    jobs[0].out_diag = out_diag;
    jobs[0].stats = stats;
    return chain_group(s, jobs, full_last);
  }

  // Response chains of several systems (or several probes of one system, each with its own
  // chain matrices) in lockstep, every product a grouped launch.
  cudaError_t chain_group(cudaStream_t s, std::vector<ChainJob>& jobs, bool full_last) override {
    const int B = (int)jobs.size();
    if (B == 0) return cudaSuccess;
    if (B > kMaxGroup) {
      for (int i = 0; i < B; i += kMaxGroup) {
        std::vector<ChainJob> part(jobs.begin() + i, jobs.begin() + std::min(B, i + kMaxGroup));
        RET(chain_group(s, part, full_last));
      }
      return cudaSuccess;
    }
    const int np = jobs[0].m->np, n = jobs[0].m->n;
    for (auto& j : jobs)
      if (j.m->np != np || j.m->n != n) return cudaErrorInvalidValue;
    const size_t cnt = (size_t)np * np;
    // either chain may run on the hi operands alone (the mu chain is the one with a full last level)
    const int nseg = full_last ? mu_nseg_ : probe_nseg_;
    // A single-product chain keeps M and T1 as FP32 values with hi operands only: its products
    // carry ~2^-11 relative error, so the double-float values and lo operands of the three-product
    // chain would add traffic and no accuracy.  The last level still writes the double-float array
    // the reductions read (with a zero low word).
    const bool single = (nseg == 1);
    std::vector<SplitMat*> T1(B), T1n(B), A1s(B), Mts(B);
    for (int i = 0; i < B; ++i) {
      T1[i] = &jobs[i].m->sT1a;
      T1n[i] = &jobs[i].m->sT1b;
      A1s[i] = &jobs[i].m->sA1;
      Mts[i] = &jobs[i].m->sMt;
    }
    for (int k = 0; k < n; ++k) {
      const bool last = (k == n - 1);
      RET(zero_amax_group(s, A1s));
      Epi em;                                                                    // Mt = 2 T1 - T_{k+1} A1
      em.alpha = -1.f;
      em.out64 = !single || (last && !full_last);
      em.hi_only = single;
      em.convert = !(last && !full_last);                                        // the last M of a probe
      em.nseg = nseg;                                                            // chain is only reduced
      std::vector<GemmOp> om;
      if (k == 0) {
        A1List al;
        al.n = B;
        for (int i = 0; i < B; ++i) {
          al.T0[i] = jobs[i].m->sT[0].d;
          al.d[i] = jobs[i].dvec;
          al.A1[i] = A1s[i]->f;
          al.amax[i] = A1s[i]->amax;
        }
        level0_A1_group_kernel<<<ew_grid(cnt, B), 256, 0, s>>>(np, al);
        note_launch();
        RET(cudaGetLastError());
        for (int i = 0; i < B; ++i) {
          Epi e = em;
          e.dvec = jobs[i].dvec;
          e.dvec_scale = 2.f;
          om.push_back({&jobs[i].m->sT[k + 1], A1s[i], Mts[i], e, jobs[i].stats});
        }
      } else {
        // A1 = T T1 + T1 T (T, T1 symmetric): one symmetric-output product over the two K pairs
        std::vector<GemmOp> oa;
        for (int i = 0; i < B; ++i) {
          Epi ea;
          ea.convert = false;
          ea.nseg = nseg;
          ea.pairs = 2;
          oa.push_back({&jobs[i].m->sT[k], T1[i], A1s[i], ea, jobs[i].stats});
        }
        RET(gemm_group(s, np, oa, true));
        for (int i = 0; i < B; ++i) {
          Epi e = em;
          if (single) {
            e.E = T1[i];                                                          // FP32, symmetric
            e.beta = 2.0f;
          } else {
            e.E64 = T1[i]->d;                                                     // symmetric: read transposed
            e.e64_trans = 1;
            e.beta64 = 2.0f;
          }
          om.push_back({&jobs[i].m->sT[k + 1], A1s[i], Mts[i], e, jobs[i].stats});
        }
      }
      RET(convert_group(s, A1s, np, single ? 2 : 0));
      RET(gemm_group(s, np, om, false));
      if (last && !full_last) {
        DiagList dl;
        dl.n = B;
        int maxN = 0;
        for (int i = 0; i < B; ++i) {
          dl.N[i] = jobs[i].N;
          dl.W[i] = jobs[i].m->sY[k].f;
          dl.X[i] = Mts[i]->d;
          dl.out[i] = jobs[i].out_diag;
          maxN = std::max(maxN, jobs[i].N);
        }
        row_dot_last_group_kernel<<<dim3((maxN + 7) / 8, B), 256, 0, s>>>(np, dl);
        note_launch();
        return cudaGetLastError();
      }
      std::vector<SplitMat*> dst(B);
      std::vector<GemmOp> oy;
      for (int i = 0; i < B; ++i) {
        dst[i] = (last && full_last) ? &jobs[i].m->sTmu : T1n[i];
        Epi ey;                                                                  // T1' = M - W M
        ey.alpha = -1.f;
        if (single) {
          ey.E = Mts[i];                                                          // read transposed: M
          ey.beta = 1.0f;
          ey.out64 = last;                                                        // T_mu (double-float)
          ey.hi_only = true;
        } else {
          ey.E64 = Mts[i]->d;
          ey.beta64 = 1.0f;
          ey.e64_trans = 1;
          ey.out64 = true;
        }
        ey.convert = !last;
        ey.nseg = nseg;
        oy.push_back({&jobs[i].m->sY[k], Mts[i], dst[i], ey, jobs[i].stats});
      }
      RET(gemm_group(s, np, oy, true));
      if (last) {
        DiagList dl;
        dl.n = B;
        int maxN = 0;
        for (int i = 0; i < B; ++i) {
          dl.N[i] = jobs[i].N;
          dl.X[i] = dst[i]->d;
          dl.out[i] = jobs[i].out_diag;
          maxN = std::max(maxN, jobs[i].N);
        }
        get_diag_group_kernel<<<dim3((maxN + 255) / 256, B), 256, 0, s>>>(np, dl);
        note_launch();
        return cudaGetLastError();
      }
      for (int i = 0; i < B; ++i) {
        T1n[i] = T1[i];
        T1[i] = dst[i];
      }
    }
    return cudaSuccess;
  }

  const int* device_error() const override { return err_; }
  void set_chain_segments(int probe_nseg, int mu_nseg) override {
    probe_nseg_ = (probe_nseg == 1) ? 1 : 3;
    mu_nseg_ = (mu_nseg == 1) ? 1 : 3;
  }

  cudaError_t trace_tn(cudaStream_t s, MatSet& m, int N, double* out) override {
    diag_sum_d_kernel<<<1, 1024, 0, s>>>(N, m.np, m.sT[m.n].d, out);
    note_launch();
    return cudaGetLastError();
  }

  cudaError_t density_out(cudaStream_t s, MatSet& m, int N, double dmu, const double*, double* ddiag,
                          double* D) override {
    density_out_d_kernel<<<nblk((size_t)m.np * m.np), 256, 0, s>>>(N, m.np, m.sT[m.n].d, m.sTmu.d, dmu, ddiag, D);
    note_launch();
    return cudaGetLastError();
  }

  cudaError_t entropy(cudaStream_t s, MatSet& m, int N, double, int n_sq, double, double, const double* D,
                      const double*, double* work, double* out) override {
    // FP64 route from the split values: T_0 from its double-float value, Y_k = I - W_k
    const size_t cnt = (size_t)m.np * m.np;
    for (double*& p : m.e64)
      if (!p) RET(cudaMalloc((void**)&p, cnt * sizeof(double)));
    double* T0 = m.e64[6];
    df_to_f64_kernel<<<nblk(cnt), 256, 0, s>>>(cnt, m.sT[0].d, T0);
    note_launch();
    RET(cudaGetLastError());
    auto load_Y = [&](int k, double* dst) -> cudaError_t {
      ident_minus_f32_to_f64_kernel<<<nblk(cnt), 256, 0, s>>>(cnt, m.np, m.sY[k].f, dst);
      note_launch();
      return cudaGetLastError();
    };
    // artanh series: terms until 2^(n+1) t0max^(2j+1) / (2j+1) N < 1e-10
    int nterms = 1;
    const double t = m.t0max;
    while (nterms < 6 && std::ldexp(1.0, n_sq + 1) * std::pow(t, 2 * nterms + 1) / (2 * nterms + 1) * N > 1e-10)
      ++nterms;
    return entropy_fp64(s, N, m.np, m.n, n_sq, T0, load_Y, m.e64[0], m.e64[1], m.e64[2], m.e64[3], m.e64[4],
                        m.e64[5], nterms, D, work, out);
  }

  int* err_ = nullptr;

 private:
  int chunk_kb() const { return fmt_ == 2 ? 2 * kChunkKb : kChunkKb; }   // K blocks per 1024-long chunk

  int fmt_;   // operand format: 0 FP16, 1 BF16, 2 TF32
  int probe_nseg_ = 3;
  int mu_nseg_ = 3;
  std::unordered_map<int, std::pair<int*, TcTiles>> tiles_;
  TcGroupCache* group_cache_ = nullptr;
  std::unordered_map<int, int> tuned_bn_;   // grouped products: tile width per size
};

// which value arrays a matrix keeps
enum { kF = 1, kD = 2 };

// Zeroing runs on the stream `s` that later uses the matrix.
// esz: bytes of one operand element (2: FP16/BF16, 4: TF32)
cudaError_t alloc_split(SplitMat& m, int np, int esz, float* scal_f, unsigned* scal_u, int what, cudaStream_t s) {
  const size_t cnt = (size_t)np * np;
  if (what & kF) {
    RET(cudaMalloc((void**)&m.f, cnt * sizeof(float)));
    RET(cudaMemsetAsync(m.f, 0, cnt * sizeof(float), s));
  }
  if (what & kD) {
    RET(cudaMalloc((void**)&m.d, cnt * sizeof(float2)));
    RET(cudaMemsetAsync(m.d, 0, cnt * sizeof(float2), s));
  }
  RET(cudaMalloc((void**)&m.hi, cnt * esz));
  RET(cudaMalloc((void**)&m.lo, cnt * esz));
  RET(cudaMemsetAsync(m.hi, 0, cnt * esz, s));
  RET(cudaMemsetAsync(m.lo, 0, cnt * esz, s));
  m.scale = scal_f;
  m.amax = scal_u;
  return cudaSuccess;
}

void free_split(SplitMat& m) {
  if (m.f) cudaFree(m.f);
  if (m.d) cudaFree(m.d);
  if (m.hi) {
    tc_forget_maps(m.hi);
    cudaFree(m.hi);
  }
  if (m.lo) {
    tc_forget_maps(m.lo);
    cudaFree(m.lo);
  }
  m.f = nullptr;
  m.d = nullptr;
  m.hi = m.lo = nullptr;
}

}  // namespace

Engine* make_split_engine(int prec) {
  if (!is_split_prec(prec)) return nullptr;
  return new EngineSplit(prec);
}

cudaError_t alloc_matset_split(MatSet& m, cudaStream_t s) {
  const int np = m.np, n = m.n, esz = operand_bytes(m.prec);
  const int nmat = (n + 1) + n + 9;
  float* scal = nullptr;
  RET(cudaMalloc((void**)&scal, sizeof(float) * 2 * nmat));
  RET(cudaMemsetAsync(scal, 0, sizeof(float) * 2 * nmat, s));
  m.tc_plan = scal;
  float* sf = scal;
  unsigned* su = reinterpret_cast<unsigned*>(scal + nmat);
  int idx = 0;
  m.sT.assign(n + 1, SplitMat());
  m.sY.assign(n, SplitMat());
  for (auto& x : m.sT) {
    RET(alloc_split(x, np, esz, sf + idx, su + idx, kD, s));
    ++idx;
  }
  for (auto& x : m.sY) {
    RET(alloc_split(x, np, esz, sf + idx, su + idx, kF, s));
    ++idx;
  }
  struct W {
    SplitMat* m;
    int what;
  } w[] = {{&m.sS, kF},  {&m.sQ, kF},  {&m.sYw, kF},  {&m.sA1, kF},
           {&m.sMt, kD | kF}, {&m.sT1a, kD | kF}, {&m.sT1b, kD | kF}, {&m.sTmu, kD}};
  for (auto& x : w) {
    RET(alloc_split(*x.m, np, esz, sf + idx, su + idx, x.what, s));
    ++idx;
  }
  return cudaSuccess;
}

// A chain slot: a view of a system's expansion matrices (T_k, W_k shared) with its own
// response-chain matrices (A1, M, T1 twice, T_mu) and their scalars, so that several probes of
// one system can run their chains side by side (grouped launches).
cudaError_t alloc_chain_slot(MatSet& slot, const MatSet& base, cudaStream_t s) {
  slot = base;
  slot.e64[0] = slot.e64[1] = slot.e64[2] = slot.e64[3] = slot.e64[4] = slot.e64[5] = slot.e64[6] = nullptr;
  const int np = base.np, esz = operand_bytes(base.prec);
  float* scal = nullptr;
  RET(cudaMalloc((void**)&scal, sizeof(float) * 2 * 5));
  RET(cudaMemsetAsync(scal, 0, sizeof(float) * 2 * 5, s));
  slot.tc_plan = scal;
  slot.sA1 = SplitMat();
  slot.sMt = SplitMat();
  slot.sT1a = SplitMat();
  slot.sT1b = SplitMat();
  slot.sTmu = SplitMat();
  unsigned* su = reinterpret_cast<unsigned*>(scal + 5);
  RET(alloc_split(slot.sA1, np, esz, scal + 0, su + 0, kF, s));
  RET(alloc_split(slot.sMt, np, esz, scal + 1, su + 1, kD | kF, s));
  RET(alloc_split(slot.sT1a, np, esz, scal + 2, su + 2, kD | kF, s));
  RET(alloc_split(slot.sT1b, np, esz, scal + 3, su + 3, kD | kF, s));
  RET(alloc_split(slot.sTmu, np, esz, scal + 4, su + 4, kD, s));
  return cudaSuccess;
}

void free_chain_slot(MatSet& slot) {
  SplitMat* w[] = {&slot.sA1, &slot.sMt, &slot.sT1a, &slot.sT1b, &slot.sTmu};
  for (SplitMat* x : w) free_split(*x);
  if (slot.tc_plan) cudaFree(slot.tc_plan);
  slot.tc_plan = nullptr;
  slot.sT.clear();
  slot.sY.clear();
}

// bytes of one chain slot of size np
size_t chain_slot_bytes(int np, int prec) {
  return (size_t)np * np * (8 + 3 * 16 + 12 + 5 * 2 * (operand_bytes(prec) - 2));
}

void free_matset_split(MatSet& m) {
  for (auto& x : m.sT) free_split(x);
  for (auto& x : m.sY) free_split(x);
  m.sT.clear();
  m.sY.clear();
  SplitMat* w[] = {&m.sS, &m.sQ, &m.sYw, &m.sA1, &m.sMt, &m.sT1a, &m.sT1b, &m.sTmu};
  for (SplitMat* x : w) free_split(*x);
  if (m.tc_plan) cudaFree(m.tc_plan);
  m.tc_plan = nullptr;
  for (double*& p : m.e64) {
    if (p) cudaFree(p);
    p = nullptr;
  }
}

// ---- self-test of the tensor-core product against the FP64 product ----

namespace {

__global__ void fill_random_kernel(size_t count, int np, uint64_t seed, int sym, double* out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  size_t i = idx / np, j = idx % np;
  if (sym && j < i) {
    const size_t t = i;
    i = j;
    j = t;
  }
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i * (uint64_t)np + j + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  out[idx] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

__global__ void to_f32_kernel(size_t count, const double* __restrict__ x, float* __restrict__ f, unsigned* amax) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.0f;
  if (idx < count) {
    v = (float)x[idx];
    f[idx] = v;
  }
  raise_amax(amax, v);
}

__global__ void diff_f32_kernel(size_t count, const float* __restrict__ a, const float* __restrict__ b,
                                double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)a[i] - (double)b[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(t));
  }
}

__global__ void max_abs_diff_kernel(size_t count, const float* __restrict__ a, const double* __restrict__ b,
                                    double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)a[i] - b[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
    unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
    atomicMax(o, (unsigned long long)__double_as_longlong(t));
  }
}

}  // namespace

// Timing of the plain-FP64 product (the product of the FP64 path) at size n: one warm-up
// product at 128, then one timed product at n (sym: symmetric-output mode, half the tiles).
// Writes [0, 0, 0, ms per product].
int selftest_gemm_f64(int n, int sym, double* result) {
  const size_t cnt = (size_t)n * n;
  double *A = nullptr, *B = nullptr, *C = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  int rc = -2;
  EpiF64 e;
  if (cudaMalloc((void**)&A, cnt * 8) || cudaMalloc((void**)&B, cnt * 8) || cudaMalloc((void**)&C, cnt * 8))
    goto done;
  fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 11, 0, A);
  note_launch();
  fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 23, sym, B);
  note_launch();
  if (gemm_f64_nt(nullptr, 128, 128, 128, A, n, B, n, C, n, e, sym != 0)) goto done;
  if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) goto done;
  cudaEventRecord(e0, nullptr);
  if (gemm_f64_nt(nullptr, n, n, n, A, n, B, n, C, n, e, sym != 0)) goto done;
  cudaEventRecord(e1, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  cudaEventElapsedTime(&ms, e0, e1);
  result[0] = result[1] = result[2] = 0.0;
  result[3] = ms;
  rc = 0;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (A) cudaFree(A);
  if (B) cudaFree(B);
  if (C) cudaFree(C);
  return rc;
}

// Grouped products against single products: nprob seeded operand pairs, each product computed
// alone and then all of them in one grouped launch (with 128- and 256-wide tiles where n allows
// both); result = [max |C_group - C_single| over the problems and widths, error flag].
int selftest_gemm_group(int n, int prec, int mode, int nprob, double* result) {
  if (n % 128 || n <= 0 || nprob < 2 || nprob > kMaxGroup || !is_split_prec(prec)) return -1;
  const int esz = operand_bytes(prec);
  const bool single = mode >= 4;
  const int sym = single ? mode - 4 : mode;
  if (sym < 0 || sym > 2) return -1;
  EngineSplit eng(prec);
  const size_t cnt = (size_t)n * n;
  std::vector<SplitMat> A(nprob), B(nprob), C(nprob), R(nprob);
  double *tmp = nullptr, *out = nullptr;
  float* scal = nullptr;
  int rc = -2;
  std::vector<double> worst(1, 0.0);
  if (cudaMalloc((void**)&tmp, cnt * 8) || cudaMalloc((void**)&out, 8) ||
      cudaMalloc((void**)&scal, 8 * nprob * sizeof(float)))
    goto done;
  cudaMemset(scal, 0, 8 * nprob * sizeof(float));
  for (int i = 0; i < nprob; ++i) {
    float* sf = scal + 4 * i;
    unsigned* su = reinterpret_cast<unsigned*>(scal + 4 * nprob + 4 * i);
    if (alloc_split(A[i], n, esz, sf, su, kF, nullptr) || alloc_split(B[i], n, esz, sf + 1, su + 1, kF, nullptr) ||
        alloc_split(C[i], n, esz, sf + 2, su + 2, kF, nullptr) || alloc_split(R[i], n, esz, sf + 3, su + 3, kF, nullptr))
      goto done;
    fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 101 + 7 * i, 0, tmp);
    note_launch();
    to_f32_kernel<<<nblk(cnt), 256>>>(cnt, tmp, A[i].f, A[i].amax);
    note_launch();
    fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 203 + 11 * i, sym, tmp);
    note_launch();
    to_f32_kernel<<<nblk(cnt), 256>>>(cnt, tmp, B[i].f, B[i].amax);
    note_launch();
    if (eng.convert(nullptr, A[i], n) || eng.convert(nullptr, B[i], n)) goto done;
  }
  {
    Epi ep;
    ep.pairs = (sym == 2) ? 2 : 1;
    ep.nseg = single ? 1 : 3;
    ep.alpha = 0.75f;
    for (int i = 0; i < nprob; ++i)
      if (eng.gemm(nullptr, n, A[i], B[i], R[i], ep, sym != 0, nullptr)) goto done;
    std::vector<EngineSplit::GemmOp> ops;
    for (int i = 0; i < nprob; ++i) ops.push_back({&A[i], &B[i], &C[i], ep, nullptr});
    // the autotuner runs both widths on the first grouped product of this size; then the
    // chosen width; compare after each
    for (int rep = 0; rep < 2; ++rep) {
      if (eng.gemm_group(nullptr, n, ops, sym != 0)) goto done;
      for (int i = 0; i < nprob; ++i) {
        if (cudaMemset(out, 0, 8)) goto done;
        diff_f32_kernel<<<304, 256>>>(cnt, C[i].f, R[i].f, out);
        note_launch();
        double h = 0.0;
        if (cudaMemcpy(&h, out, 8, cudaMemcpyDeviceToHost)) goto done;
        worst[0] = std::max(worst[0], h);
      }
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  {
    int herr = 0;
    cudaMemcpy(&herr, eng.err_, sizeof(int), cudaMemcpyDeviceToHost);
    result[0] = worst[0];
    result[1] = herr;
    rc = 0;
  }
done:
  for (int i = 0; i < nprob; ++i) {
    free_split(A[i]);
    free_split(B[i]);
    free_split(C[i]);
    free_split(R[i]);
  }
  if (tmp) cudaFree(tmp);
  if (out) cudaFree(out);
  if (scal) cudaFree(scal);
  return rc;
}

// Returns 0 on success and writes [max |C_tc - C_ref|, max |C_ref|, error flag, ms per product].
int selftest_gemm(int n, int prec, int sym, double* result) {
  if (prec == 0 && n % 128 == 0 && n > 0 && sym >= 0 && sym <= 1) return selftest_gemm_f64(n, sym, result);
  if (n % 128 || n <= 0 || !is_split_prec(prec)) return -1;
  const int esz = operand_bytes(prec);
  const bool single = sym >= 4;   // one product of the hi operands only, as in the single-product chains
  if (single) sym -= 4;
  if (sym < 0 || sym > 2) return -1;
  EngineSplit eng(prec);
  const size_t cnt = (size_t)n * n;
  double *A = nullptr, *B = nullptr, *Cref = nullptr, *Cref2 = nullptr, *out = nullptr;
  const bool pair = (sym == 2);   // C = A B^T + B A^T
  float* scal = nullptr;
  SplitMat sa, sb, sc;
  cudaStream_t s = nullptr;
  int rc = -2;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  if (cudaMalloc((void**)&A, cnt * 8) || cudaMalloc((void**)&B, cnt * 8) || cudaMalloc((void**)&Cref, cnt * 8) ||
      cudaMalloc((void**)&out, 8) || cudaMalloc((void**)&scal, 6 * sizeof(float)) ||
      (pair && cudaMalloc((void**)&Cref2, cnt * 8)))
    goto done;
  cudaMemset(scal, 0, 6 * sizeof(float));
  if (alloc_split(sa, n, esz, scal, (unsigned*)scal + 3, kF, s) || alloc_split(sb, n, esz, scal + 1, (unsigned*)scal + 4, kF, s) ||
      alloc_split(sc, n, esz, scal + 2, (unsigned*)scal + 5, kF, s))
    goto done;
  fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 11, 0, A);
  note_launch();
  fill_random_kernel<<<nblk(cnt), 256>>>(cnt, n, 23, sym, B);
  note_launch();
  to_f32_kernel<<<nblk(cnt), 256>>>(cnt, A, sa.f, sa.amax);
  note_launch();
  to_f32_kernel<<<nblk(cnt), 256>>>(cnt, B, sb.f, sb.amax);
  note_launch();
  if (eng.convert(s, sa, n) || eng.convert(s, sb, n)) goto done;
  {
    EpiF64 e;
    if (gemm_f64_nt(s, n, n, n, A, n, B, n, Cref, n, e, sym == 1)) goto done;
    if (pair) {   // Cref2 = B A^T + A B^T
      EpiF64 e2;
      e2.E = Cref;
      e2.lde = n;
      e2.beta = 1.0;
      if (gemm_f64_nt(s, n, n, n, B, n, A, n, Cref2, n, e2, false)) goto done;
    }
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  {
    Epi ep;
    ep.pairs = pair ? 2 : 1;
    ep.nseg = single ? 1 : 3;
    if (eng.gemm(s, n, sa, sb, sc, ep, sym != 0, nullptr)) goto done;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 5; ++r)
      if (eng.gemm(s, n, sa, sb, sc, ep, sym != 0, nullptr)) goto done;
  }
  cudaEventRecord(e1, s);
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaMemset(out, 0, 8);
  max_abs_diff_kernel<<<304, 256>>>(cnt, sc.f, pair ? Cref2 : Cref, out);
  note_launch();
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  {
    double h[1];
    int herr = 0;
    cudaMemcpy(h, out, 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, eng.err_, sizeof(int), cudaMemcpyDeviceToHost);
    result[0] = h[0];
    result[1] = 0.0;
    result[2] = herr;
    result[3] = ms / 5.0;
    rc = 0;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_split(sa);
  free_split(sb);
  free_split(sc);
  if (A) cudaFree(A);
  if (B) cudaFree(B);
  if (Cref) cudaFree(Cref);
  if (Cref2) cudaFree(Cref2);
  if (out) cudaFree(out);
  if (scal) cudaFree(scal);
  return rc;
}

}  // namespace xl
