// Split-precision engine: the expansion and response chains with tensor-core
// products on hi/lo 16-bit operands (FP16x3 or BF16x3).
//
// Every matrix keeps a value array -- FP32, or double-float (an FP32 hi + lo
// pair) for T_k, M and T1, whose leading terms the correction form keeps out of
// the products -- and a split operand pair hi = rn16(x s), lo = rn16(x s - hi)
// with a power-of-two scale s chosen from max |x| so that max |x s| lies in
// [2^10, 2^11) (FP16 keeps full precision in both parts); producers raise
// max |x| atomically and a conversion pass writes hi/lo.  A product takes three
// 16-bit products (hi*hi, hi*lo, lo*hi), or one (hi*hi) in the probe chains
// and the mu chain when the context asks for it.  Traces, charges and the
// density matrix handed to the forces are accumulated in FP64.
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
inline unsigned ew_blocks(size_t count) { return (unsigned)std::min<size_t>(nblk(count), kEwBlocks); }

// One-CTA-per-tile product kernel: products of at least this size split their hi*hi sums over
// both accumulators.
constexpr int kSplitAccMin = 8192;
// Persistent product kernel, split products: the hi*hi sum is accumulated in chunks of this many
// 64-wide K blocks (K = 1024), each folded into the running sum with round-to-nearest FP32 adds.
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

// Conversion to the split operand pair: hi = rn16(x s), lo = rn16(x s - hi).
template <bool BF16>
__device__ __forceinline__ void split16(float x, unsigned short& h, unsigned short& l) {
  if (BF16) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(x);
    h = __bfloat16_as_ushort(hb);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hb)));
  } else {
    const __half hh = __float2half_rn(x);
    h = __half_as_ushort(hh);
    l = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
  }
}

// All threads derive the same scale from amax; thread 0 of block 0 publishes it.  Four
// elements per thread and step (16-byte loads, 8-byte stores; count is a multiple of 4).
template <bool BF16>
__global__ void convert_split_kernel(size_t count, const float* __restrict__ f, const unsigned* __restrict__ amax,
                                     uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, float* __restrict__ scale) {
  const float m = __uint_as_float(*amax);
  float s = 1.0f;
  if (m > 0.0f && isfinite(m)) s = ldexpf(1.0f, 10 - ilogbf(m));
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = s;
  const float4* f4 = reinterpret_cast<const float4*>(f);
  ushort4* h4 = reinterpret_cast<ushort4*>(hi);
  ushort4* l4 = reinterpret_cast<ushort4*>(lo);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 x = f4[i];
    ushort4 h, l;
    split16<BF16>(x.x * s, h.x, l.x);
    split16<BF16>(x.y * s, h.y, l.y);
    split16<BF16>(x.z * s, h.z, l.z);
    split16<BF16>(x.w * s, h.w, l.w);
    h4[i] = h;
    l4[i] = l;
  }
}

// The hi part alone, for matrices that only enter single products (hi*hi).
template <bool BF16>
__global__ void convert_hi_kernel(size_t count, const float* __restrict__ f, const unsigned* __restrict__ amax,
                                  uint16_t* __restrict__ hi, float* __restrict__ scale) {
  const float m = __uint_as_float(*amax);
  float s = 1.0f;
  if (m > 0.0f && isfinite(m)) s = ldexpf(1.0f, 10 - ilogbf(m));
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = s;
  const float4* f4 = reinterpret_cast<const float4*>(f);
  ushort4* h4 = reinterpret_cast<ushort4*>(hi);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 x = f4[i];
    ushort4 h;
    if (BF16) {
      h.x = __bfloat16_as_ushort(__float2bfloat16_rn(x.x * s));
      h.y = __bfloat16_as_ushort(__float2bfloat16_rn(x.y * s));
      h.z = __bfloat16_as_ushort(__float2bfloat16_rn(x.z * s));
      h.w = __bfloat16_as_ushort(__float2bfloat16_rn(x.w * s));
    } else {
      h.x = __half_as_ushort(__float2half_rn(x.x * s));
      h.y = __half_as_ushort(__float2half_rn(x.y * s));
      h.z = __half_as_ushort(__float2half_rn(x.z * s));
      h.w = __half_as_ushort(__float2half_rn(x.w * s));
    }
    h4[i] = h;
  }
}

// Y = a I + b X (grid-stride, one max-|Y| atomic per block)
__global__ void axpi_f32_kernel(int np, float a, float b, const float* __restrict__ X, float* __restrict__ Y,
                                unsigned* amax, const double* __restrict__ dc = nullptr) {
  if (dc) {   // a = 1 - c, b = c from the device copy of c
    a = (float)(1.0 - dc[0]);
    b = (float)dc[0];
  }
  const size_t count = (size_t)np * np;
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / np), j = (int)(idx % np);
    const float v = b * X[idx] + (i == j ? a : 0.0f);
    Y[idx] = v;
    m = fmaxf(m, fabsf(v));
  }
  raise_amax(amax, m);
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

// The same from a double-float value hi + lo: the 16-bit pair splits (xh - hi16) + xl, so the
// low FP32 word is not lost (s is a power of two, so x s is exact).
template <bool BF16>
__global__ void convert_split_d_kernel(size_t count, const float2* __restrict__ d, const unsigned* __restrict__ amax,
                                       uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                       float* __restrict__ scale) {
  const float m = __uint_as_float(*amax);
  float s = 1.0f;
  if (m > 0.0f && isfinite(m)) s = ldexpf(1.0f, 10 - ilogbf(m));
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = s;
  const float4* d4 = reinterpret_cast<const float4*>(d);   // two double-float values per float4
  ushort4* h4 = reinterpret_cast<ushort4*>(hi);
  ushort4* l4 = reinterpret_cast<ushort4*>(lo);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 a = d4[2 * i], b = d4[2 * i + 1];
    const float xs[4] = {a.x * s, a.z * s, b.x * s, b.z * s};
    const float xl[4] = {a.y * s, a.w * s, b.y * s, b.w * s};
    unsigned short h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (BF16) {
        const __nv_bfloat16 hb = __float2bfloat16_rn(xs[k]);
        h[k] = __bfloat16_as_ushort(hb);
        l[k] = __bfloat16_as_ushort(__float2bfloat16_rn((xs[k] - __bfloat162float(hb)) + xl[k]));
      } else {
        const __half hh = __float2half_rn(xs[k]);
        h[k] = __half_as_ushort(hh);
        l[k] = __half_as_ushort(__float2half_rn((xs[k] - __half2float(hh)) + xl[k]));
      }
    }
    h4[i] = make_ushort4(h[0], h[1], h[2], h[3]);
    l4[i] = make_ushort4(l[0], l[1], l[2], l[3]);
  }
}

// T0 = -sc (H - mu I) as a double-float (hi = rn32(v), lo = rn32(v - hi))
__global__ void t0_init_d_kernel(int n, int np, const double* __restrict__ H, double mu, double sc,
                                 float2* __restrict__ T0, unsigned* amax, const double* __restrict__ dmu = nullptr) {
  if (dmu) mu = dmu[0];
  const size_t count = (size_t)np * np;
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / np), j = (int)(idx % np);
    double v = 0.0;
    if (i < n && j < n) v = -sc * (H[idx] - (i == j ? mu : 0.0));
    const float vh = (float)v;
    T0[idx] = make_float2(vh, (float)(v - (double)vh));
    m = fmaxf(m, fabsf(vh));
  }
  raise_amax(amax, m);
}

__global__ void level0_A1_d_kernel(int np, const float2* __restrict__ T0, const double* __restrict__ d,
                                   float* __restrict__ A1, unsigned* amax) {
  const size_t count = (size_t)np * np;
  float m = 0.0f;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / np), j = (int)(idx % np);
    const float2 t = T0[idx];
    const float v = (t.x + t.y) * (float)(d[i] + d[j]);
    A1[idx] = v;
    m = fmaxf(m, fabsf(v));
  }
  raise_amax(amax, m);
}

__device__ __forceinline__ double df_val(float2 v) { return (double)v.x + (double)v.y; }

// out_i = (Y M)_ii = Mt_ii - sum_j W_ij Mt_ij  (Y = I - W, Mt = M^T), one warp per row
__global__ void row_dot_last_kernel(int n, int np, const float* __restrict__ W, const float2* __restrict__ Mt,
                                    double* __restrict__ out) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  float accf = 0.0f;
  double acc = 0.0;
  for (int j = lane, c = 0; j < np; j += 32, ++c) {
    const float2 m = Mt[(size_t)i * np + j];
    accf += W[(size_t)i * np + j] * (m.x + m.y);
    if ((c & 15) == 15) {
      acc += (double)accf;
      accf = 0.0f;
    }
  }
  acc += (double)accf;
  acc = warp_sum(acc);
  if (lane == 0) out[i] = df_val(Mt[(size_t)i * np + i]) - acc;
}

__global__ void get_diag_d_kernel(int n, int np, const float2* __restrict__ X, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = df_val(X[(size_t)i * np + i]);
}

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
// terms never pass through 16-bit operands:
//   T_{k+1} = 2 T_k - 2 T_k W_k,  W_k = I - Y_k = I - (I + T_k^2)^-1,
// W_k from the Newton-Schulz step written for W (Q = S - W - W S,
// W <- W + Q - Q W), and the response chains as
//   M = 2 T1_k - A1 T_{k+1},  T1_{k+1} = M - W_k M.
// T_k, M and T1_k are FP64 values; W, S, Q, A1 FP32 values; every product
// operand is the hi/lo split of a value.
class EngineSplit : public Engine {
 public:
  explicit EngineSplit(int prec) : bf16_(prec == XLBOMD_BF16x3_ID ? 1 : 0) {}
  ~EngineSplit() override {
    for (auto& kv : tiles_) cudaFree(kv.second.first);
    if (err_) cudaFree(err_);
  }

  cudaError_t convert(cudaStream_t s, SplitMat& m, int np) {
    const size_t count = (size_t)np * np;
    const unsigned g = std::min<size_t>(nblk(count), 152 * 16);
    if (bf16_)
      convert_split_kernel<true><<<g, 256, 0, s>>>(count, m.f, m.amax, m.hi, m.lo, m.scale);
    else
      convert_split_kernel<false><<<g, 256, 0, s>>>(count, m.f, m.amax, m.hi, m.lo, m.scale);
    note_launch();
    return cudaGetLastError();
  }

  cudaError_t convert_hi(cudaStream_t s, SplitMat& m, int np) {
    const size_t count = (size_t)np * np;
    const unsigned g = std::min<size_t>(nblk(count), 152 * 16);
    if (bf16_)
      convert_hi_kernel<true><<<g, 256, 0, s>>>(count, m.f, m.amax, m.hi, m.scale);
    else
      convert_hi_kernel<false><<<g, 256, 0, s>>>(count, m.f, m.amax, m.hi, m.scale);
    note_launch();
    return cudaGetLastError();
  }

  cudaError_t convert_d(cudaStream_t s, SplitMat& m, int np) {
    const size_t count = (size_t)np * np;
    const unsigned g = std::min<size_t>(nblk(count), 152 * 16);
    if (bf16_)
      convert_split_d_kernel<true><<<g, 256, 0, s>>>(count, m.d, m.amax, m.hi, m.lo, m.scale);
    else
      convert_split_d_kernel<false><<<g, 256, 0, s>>>(count, m.d, m.amax, m.hi, m.lo, m.scale);
    note_launch();
    return cudaGetLastError();
  }

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
    a.bf16 = bf16_;
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
    a.chunk_kb = kChunkKb;
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

  cudaError_t foe(cudaStream_t s, MatSet& m, const double* H, int N, double mu, double sc,
                  const std::vector<int>& ns, const std::vector<double>& nc, double* stats,
                  const double* dpar) override {
    const int np = m.np, n = m.n;
    const size_t cnt = (size_t)np * np;
    RET(cudaMemsetAsync(m.sT[0].amax, 0, sizeof(unsigned), s));
    t0_init_d_kernel<<<ew_blocks(cnt), 256, 0, s>>>(N, np, H, mu, sc, m.sT[0].d, m.sT[0].amax, dpar);
    note_launch();
    RET(cudaGetLastError());
    RET(convert_d(s, m.sT[0], np));
    for (int k = 0; k < n; ++k) {
      Epi es;
      RET(gemm(s, np, m.sT[k], m.sT[k], m.sS, es, true, stats));                 // S = T^2
      // the Newton-Schulz iterates alternate between sY[k] and the work matrix; the start is
      // chosen by the parity of the iteration count so that W_k always ends in sY[k] (the
      // buffers every later use, and a captured graph of this pass, refer to)
      SplitMat* W = (ns[k] % 2 == 1) ? &m.sYw : &m.sY[k];
      SplitMat* Wn = (W == &m.sY[k]) ? &m.sYw : &m.sY[k];
      RET(cudaMemsetAsync(W->amax, 0, sizeof(unsigned), s));
      if (k == 0)
        axpi_f32_kernel<<<ew_blocks(cnt), 256, 0, s>>>(np, 0.f, 1.f, m.sS.f, W->f, W->amax);        // W = S
      else
        axpi_f32_kernel<<<ew_blocks(cnt), 256, 0, s>>>(np, (float)(1.0 - nc[k]), (float)nc[k], m.sY[k - 1].f, W->f,
                                                 W->amax, dpar ? dpar + 1 + k : nullptr);  // W = (1-c) I + c W_{k-1}
      note_launch();
      RET(cudaGetLastError());
      RET(convert(s, *W, np));
      for (int it = 0; it < ns[k]; ++it) {
        Epi eq;                                                                   // Q = S - W - W S
        eq.alpha = -1.f;
        eq.E = &m.sS;
        eq.beta = 1.f;
        eq.E2 = W;
        eq.beta2 = -1.f;
        RET(gemm(s, np, *W, m.sS, m.sQ, eq, false, stats));
        Epi ew;                                                                   // W <- W + Q - Q W
        ew.alpha = -1.f;
        ew.E = W;
        ew.beta = 1.f;
        ew.E2 = &m.sQ;
        ew.beta2 = 1.f;
        RET(gemm(s, np, m.sQ, *W, *Wn, ew, true, stats));
        std::swap(W, Wn);
        if (stats) stats[1] += 1;
      }
      Epi et;                                                                     // T' = 2T - 2 T W
      et.alpha = -2.f;
      et.E64 = m.sT[k].d;                                                         // symmetric: read transposed
      et.e64_trans = 1;
      et.beta64 = 2.0f;
      et.out64 = true;
      RET(gemm(s, np, m.sT[k], m.sY[k], m.sT[k + 1], et, true, stats));
    }
    return cudaSuccess;
  }

  cudaError_t chain(cudaStream_t s, MatSet& m, const double* dvec, int N, bool full_last, double* out_diag,
                    double* stats) override {
    const int np = m.np, n = m.n;
    const size_t cnt = (size_t)np * np;
    // either chain may run on the hi operands alone (the mu chain is the one with a full last level)
    const int nseg = full_last ? mu_nseg_ : probe_nseg_;
    // A single-product chain keeps M and T1 as FP32 values with hi operands only: its products
    // carry ~2^-11 relative error, so the double-float values and lo operands of the three-product
    // chain would add traffic and no accuracy.  The last level still writes the double-float array
    // the reductions read (with a zero low word).
    const bool single = (nseg == 1);
    SplitMat* T1 = &m.sT1a;
    SplitMat* T1n = &m.sT1b;
    for (int k = 0; k < n; ++k) {
      const bool last = (k == n - 1);
      RET(cudaMemsetAsync(m.sA1.amax, 0, sizeof(unsigned), s));
      Epi em;                                                                    // Mt = 2 T1 - T_{k+1} A1
      em.alpha = -1.f;
      em.out64 = !single || (last && !full_last);
      em.hi_only = single;
      em.convert = !(last && !full_last);                                        // the last M of a probe
      em.nseg = nseg;                                                            // chain is only reduced
      if (k == 0) {
        level0_A1_d_kernel<<<ew_blocks(cnt), 256, 0, s>>>(np, m.sT[0].d, dvec, m.sA1.f, m.sA1.amax);
        note_launch();
        RET(cudaGetLastError());
        em.dvec = dvec;
        em.dvec_scale = 2.f;
      } else {
        // A1 = T T1 + T1 T (T, T1 symmetric): one symmetric-output product over the two K pairs
        Epi ea;
        ea.convert = false;
        ea.nseg = nseg;
        ea.pairs = 2;
        RET(gemm(s, np, m.sT[k], *T1, m.sA1, ea, true, stats));
        if (single) {
          em.E = T1;                                                              // FP32, symmetric
          em.beta = 2.0f;
        } else {
          em.E64 = T1->d;                                                         // symmetric: read transposed
          em.e64_trans = 1;
          em.beta64 = 2.0f;
        }
      }
      RET(single ? convert_hi(s, m.sA1, np) : convert(s, m.sA1, np));
      RET(gemm(s, np, m.sT[k + 1], m.sA1, m.sMt, em, false, stats));
      if (last && !full_last) {
        row_dot_last_kernel<<<(N + 7) / 8, 256, 0, s>>>(N, np, m.sY[k].f, m.sMt.d, out_diag);
        note_launch();
        return cudaGetLastError();
      }
      SplitMat* dst = (last && full_last) ? &m.sTmu : T1n;
      Epi ey;                                                                    // T1' = M - W M
      ey.alpha = -1.f;
      if (single) {
        ey.E = &m.sMt;                                                            // read transposed: M
        ey.beta = 1.0f;
        ey.out64 = last;                                                          // T_mu (double-float)
        ey.hi_only = true;
      } else {
        ey.E64 = m.sMt.d;
        ey.beta64 = 1.0f;
        ey.e64_trans = 1;
        ey.out64 = true;
      }
      ey.convert = !last;
      ey.nseg = nseg;
      RET(gemm(s, np, m.sY[k], m.sMt, *dst, ey, true, stats));
      if (last) {
        get_diag_d_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, np, dst->d, out_diag);
        note_launch();
        return cudaGetLastError();
      }
      T1n = T1;
      T1 = dst;
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
  int bf16_;
  int probe_nseg_ = 3;
  int mu_nseg_ = 3;
  std::unordered_map<int, std::pair<int*, TcTiles>> tiles_;
};

// which value arrays a matrix keeps
enum { kF = 1, kD = 2 };

// Zeroing runs on the stream `s` that later uses the matrix.
cudaError_t alloc_split(SplitMat& m, int np, float* scal_f, unsigned* scal_u, int what, cudaStream_t s) {
  const size_t cnt = (size_t)np * np;
  if (what & kF) {
    RET(cudaMalloc((void**)&m.f, cnt * sizeof(float)));
    RET(cudaMemsetAsync(m.f, 0, cnt * sizeof(float), s));
  }
  if (what & kD) {
    RET(cudaMalloc((void**)&m.d, cnt * sizeof(float2)));
    RET(cudaMemsetAsync(m.d, 0, cnt * sizeof(float2), s));
  }
  RET(cudaMalloc((void**)&m.hi, cnt * sizeof(uint16_t)));
  RET(cudaMalloc((void**)&m.lo, cnt * sizeof(uint16_t)));
  RET(cudaMemsetAsync(m.hi, 0, cnt * sizeof(uint16_t), s));
  RET(cudaMemsetAsync(m.lo, 0, cnt * sizeof(uint16_t), s));
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
  if (prec != XLBOMD_FP16x3_ID && prec != XLBOMD_BF16x3_ID) return nullptr;
  return new EngineSplit(prec);
}

cudaError_t alloc_matset_split(MatSet& m, cudaStream_t s) {
  const int np = m.np, n = m.n;
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
    RET(alloc_split(x, np, sf + idx, su + idx, kD, s));
    ++idx;
  }
  for (auto& x : m.sY) {
    RET(alloc_split(x, np, sf + idx, su + idx, kF, s));
    ++idx;
  }
  struct W {
    SplitMat* m;
    int what;
  } w[] = {{&m.sS, kF},  {&m.sQ, kF},  {&m.sYw, kF},  {&m.sA1, kF},
           {&m.sMt, kD | kF}, {&m.sT1a, kD | kF}, {&m.sT1b, kD | kF}, {&m.sTmu, kD}};
  for (auto& x : w) {
    RET(alloc_split(*x.m, np, sf + idx, su + idx, x.what, s));
    ++idx;
  }
  return cudaSuccess;
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

// Returns 0 on success and writes [max |C_tc - C_ref|, max |C_ref|, error flag, ms per product].
int selftest_gemm(int n, int prec, int sym, double* result) {
  if (prec == 0 && n % 128 == 0 && n > 0 && sym >= 0 && sym <= 1) return selftest_gemm_f64(n, sym, result);
  if (n % 128 || n <= 0 || (prec != XLBOMD_FP16x3_ID && prec != XLBOMD_BF16x3_ID)) return -1;
  const bool single = sym >= 4;   // one 16-bit product (hi operands only), as in the single-product chains
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
  if (alloc_split(sa, n, scal, (unsigned*)scal + 3, kF, s) || alloc_split(sb, n, scal + 1, (unsigned*)scal + 4, kF, s) ||
      alloc_split(sc, n, scal + 2, (unsigned*)scal + 5, kF, s))
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
