// Split-precision tensor-core products for sm_103a (tcgen05 + TMEM + TMA).
//
// C = epi( sum_seg A_seg B_seg^T ) with 16-bit operands (FP16 or BF16) and an
// FP32 accumulation in tensor memory.  A split product uses three K segments,
// A_hi B_hi + A_hi B_lo + A_lo B_hi (one, A_hi B_hi, for single-product
// chains); the operands carry power-of-two scales that the epilogue removes.
//
// Two kernels share the pipeline.  The default is persistent: one CTA per SM
// walks the 128 x BN output tiles.  The other (XLBOMD_GEMM=classic) gives
// each CTA one tile.  Warp 0 issues TMA loads (128-byte swizzle, K-major) into
// a STAGES-deep ring guarded by mbarriers; warp 1 allocates TMEM and one
// elected thread issues tcgen05.mma (M = 128, N = BN, K = 16) per 32-byte K
// step; warps 2-5 wait for the accumulators, read them with tcgen05.ld (32
// lanes x 32 columns per load), apply the epilogue and store FP32 or
// double-float rows (and the mirrored columns of a symmetric product).  In the
// persistent kernel the epilogue folds accumulator 0 into accumulator 1 and
// releases it at once, so the next tile's first K blocks overlap the rest of
// the epilogue.
//
// The tensor core adds each K = 16 step into its FP32 accumulator with
// truncation, so a small term added to a large accumulator loses bits.  The
// hi*hi segment and the two correction segments (hi*lo, lo*hi, about 2^-11
// smaller) therefore go to two separate TMEM accumulators (2 x BN columns)
// that the epilogue adds in FP32.  Products of large n also split the hi*hi
// sum over the two accumulators (split_acc), since the truncation error of a
// sum grows with its length.  A pair product (pairs = 2) adds the swapped
// operands as a second K range, C = A B^T + B A^T.  Every mbarrier wait is
// bounded: on timeout the kernel records an error code and leaves its loops,
// and TMEM is always released.
//
// TF32 operands (fmt = 2, persistent kernel only) are FP32 words whose low 13
// mantissa bits are zero.  A 128-byte swizzle row then holds 32 elements, and
// each tcgen05.mma of kind::tf32 (K = 8) takes the same 32-byte step.  So the
// ring's stage bytes, the shared-memory descriptors and the per-stage MMA
// count stay as they are.  Only the K-block width (32 elements), the tensor
// map's element type and the instruction kind change.
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_map>

#include "precision.h"
#include "tc.h"

namespace xl {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;           // 64 x 16-bit = 128 bytes: one swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int kWaitLimit = 1 << 24;
constexpr int kGroupM = 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the completion of the phase with the given parity (the epilogue warps'
// waits: each try may suspend the thread for a hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// The same without suspending (mbarrier.test_wait in a bounded spin): the waits of the producer
// and MMA threads, which hand the operand ring's stages to each other (MMA completion -> empty
// -> producer -> full -> MMA thread).  With the default suspension those hand-offs cost about
// 20 % of a product (n = 8192 split product: 2.46 ms with the hand-off and no operand loads at
// all, 2.01 ms with neither), and the spin closes that gap (no loads: 1.92 ms; with loads 2.21
// against 2.26 ms with a 20 ns suspend hint).  The epilogue warps keep the suspending wait:
// polling from them would take issue slots from the two single-thread loops on the
// sub-partitions they share.
__device__ __forceinline__ bool mbar_wait_fast(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < (kWaitLimit << 4); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

// A tensor map written to global memory by the host (grouped launches) reaches the TMA unit
// through the tensormap proxy: acquire it before its first use in the kernel.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16 / kind::tf32: D = F32, A/B = F16 (0) or BF16 (1) under
// kind::f16, TF32 (2) under kind::tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc_m(int m, int bn, int ab_fmt) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
__host__ __device__ constexpr uint32_t instr_desc(int bn, int ab_fmt) { return instr_desc_m(BM, bn, ab_fmt); }

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  // r tied to the wait: no use of the loaded registers is scheduled before it
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])),
      "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
      "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])),
      "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])),
      "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])),
      "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}

// 64 columns of this warp's 32 lanes, without waiting (tcgen05.wait::ld before use)
__device__ __forceinline__ void tmem_ld64_nowait(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
}

// Wait for this thread's tcgen05.ld results; r is tied to the wait so that no use of the loaded
// registers is scheduled before it.
__device__ __forceinline__ void tmem_wait_ld64(uint32_t (&r)[64]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]), "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]), "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])::"memory");
}

// Orders the uses of r after the preceding tcgen05.wait::ld (volatile asm statements keep their order).
__device__ __forceinline__ void tmem_after_wait64(uint32_t (&r)[64]) { asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]), "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]), "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])); }

__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t (&v)[64]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64};" ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]), "r"(v[32]), "r"(v[33]), "r"(v[34]), "r"(v[35]), "r"(v[36]), "r"(v[37]), "r"(v[38]), "r"(v[39]), "r"(v[40]), "r"(v[41]), "r"(v[42]), "r"(v[43]), "r"(v[44]), "r"(v[45]), "r"(v[46]), "r"(v[47]), "r"(v[48]), "r"(v[49]), "r"(v[50]), "r"(v[51]), "r"(v[52]), "r"(v[53]), "r"(v[54]), "r"(v[55]), "r"(v[56]), "r"(v[57]), "r"(v[58]), "r"(v[59]), "r"(v[60]), "r"(v[61]), "r"(v[62]), "r"(v[63]) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Output tile of tile id: from the symmetric tile list, or the grouped raster (GROUP_M row
// panels at a time, so that the CTAs in flight share their A and B panels in L2).  False for
// a tile outside the matrix (a bad tile list), which is reported and never stored.
__device__ __forceinline__ bool tile_coords(const TcArgs& a, int id, int& tm, int& tn) {
  if (a.tile_list) {
    tm = a.tile_list[2 * id];
    tn = a.tile_list[2 * id + 1];
  } else {
    const int tiles_m = a.n / BM;
    const int per_group = kGroupM * a.tiles_n;
    const int g = id / per_group, r = id % per_group;
    const int first = g * kGroupM;
    const int gm = min(tiles_m - first, kGroupM);
    tm = first + r % gm;
    tn = r / gm;
  }
  return tm >= 0 && tm < a.n / BM && tn >= 0 && tn < a.tiles_n;
}

// The K blocks of a tile run as a few segments, each one operand pair pr (0: A B^T, 1: the
// swapped pair B A^T) and split part kind (0 = hi*hi, 1 = hi*lo, 2 = lo*hi) over K blocks
// [k0, k1).  Default order: the hi*hi segments of every pair (accumulator 0), then the
// corrections (accumulator 1).  split_acc (large n): the first half of the hi*hi K blocks
// (accumulator 0), the corrections into accumulator 1 while it is still small, then the second
// half of the hi*hi K blocks on top of accumulator 1 -- the tensor core truncates as it
// accumulates, so each large sum is half as long.  Accumulator 1 starts at K block acc1_start.
struct KSeg {
  int seg, kidx, k1, pr, kind;
};

__device__ __forceinline__ void kseg_decode(const TcArgs& a, int nk, KSeg& q) {
  const int P = a.pairs, NC = (a.nseg - 1) * a.pairs;   // hi*hi pairs, correction segments
  int k0 = 0;
  q.k1 = nk;
  if (!a.split_acc) {
    if (q.seg < P) {
      q.pr = q.seg;
      q.kind = 0;
    } else {
      const int r = q.seg - P;
      q.pr = r >> 1;
      q.kind = 1 + (r & 1);
    }
  } else if (q.seg == 0 || q.seg > NC) {
    const bool second = q.seg > NC;
    q.kind = 0;
    if (P == 2) {
      q.pr = second ? 1 : 0;
    } else {
      q.pr = 0;
      k0 = second ? nk / 2 : 0;
      q.k1 = second ? nk : nk / 2;
    }
  } else {
    const int r = q.seg - 1;
    q.pr = r >> 1;
    q.kind = 1 + (r & 1);
  }
  q.kidx = k0;
}

__device__ __forceinline__ void kseg_begin(const TcArgs& a, int nk, KSeg& q) {
  q.seg = 0;
  kseg_decode(a, nk, q);
}

__device__ __forceinline__ void kseg_next(const TcArgs& a, int nk, KSeg& q) {
  if (++q.kidx == q.k1) {
    ++q.seg;
    kseg_decode(a, nk, q);
  }
}

__device__ __forceinline__ int acc1_start(const TcArgs& a, int nk) {
  return a.split_acc ? a.pairs * nk / 2 : a.pairs * nk;
}

// L2 prefetch of the side inputs of tile (tm, tn) by the 128 epilogue threads (t = 0..127)
template <int BN>
__device__ __forceinline__ void prefetch_sides(const TcArgs& a, int tm, int tn, int t) {
  const int r = tm * BM + t;
  const float* fsides[2] = {a.E, a.E2};
  for (int k = 0; k < 2; ++k)
    if (fsides[k])
      for (int rr = t; rr < BN; rr += 128)
        for (int c = 0; c < BM; c += 32) prefetch_l2(fsides[k] + (size_t)(tn * BN + rr) * a.ldc + tm * BM + c);
  if (a.E64) {
    if (a.e64_trans) {
      for (int rr = t; rr < BN; rr += 128)
        for (int c = 0; c < BM; c += 16) prefetch_l2(a.E64 + (size_t)(tn * BN + rr) * a.ldc + tm * BM + c);
    } else {
      for (int c = 0; c < BN; c += 16) prefetch_l2(a.E64 + (size_t)r * a.ldc + tn * BN + c);
    }
  }
}

// a + b for a double-float a and a float b (Knuth two-sum, then renormalise)
__device__ __forceinline__ float2 df_add(float2 a, float b) {
  const float s = a.x + b;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (b - bb) + a.y;
  const float hi = s + err;
  return make_float2(hi, err - (hi - s));
}

// Epilogue of one 32-column chunk: v holds this lane's row `row`, columns
// col0 .. col0 + 31 of the raw accumulator sum; scales, adds the side inputs
// and the diagonal, stores through the per-warp staging tiles tx, ty (32 x 33),
// and raises vmax.
__device__ __forceinline__ void epilogue_chunk(const TcArgs& a, float (&v)[32], int row, int row0, int col0,
                                               int lane, float (*tx)[33], float (*ty)[33], float inv,
                                               float& vmax) {
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] *= inv;
  // FP32 side inputs of symmetric value, read transposed: for a fixed
  // column the 32 lanes read 32 consecutive rows (coalesced)
  if (a.E) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] += a.beta * a.E[(size_t)(col0 + i) * a.ldc + row];
  }
  if (a.E2) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] += a.beta2 * a.E2[(size_t)(col0 + i) * a.ldc + row];
  }
  const int dc = row - col0;   // diagonal column of this lane, if in the chunk
  if (dc >= 0 && dc < 32) {
    float dd = a.diag;
    if (a.dvec && row < a.ndvec) dd += a.dvec_scale * (float)a.dvec[row];
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i == dc) v[i] += dd;
  }
  if (a.C64) {
    // double-float value: exact leading term beta64 E64 plus the FP32 part
    float hi[32], lo[32];
    if (a.E64 && a.e64_trans) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float2 e = a.E64[(size_t)(col0 + i) * a.ldc + row];
        const float2 x = df_add(make_float2(a.beta64 * e.x, a.beta64 * e.y), v[i]);
        hi[i] = x.x;
        lo[i] = x.y;
      }
    } else if (a.E64) {
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const float2 e = a.E64[(size_t)(row0 + i) * a.ldc + col0 + lane];
        tx[i][lane] = e.x;
        ty[i][lane] = e.y;
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float2 x = df_add(make_float2(a.beta64 * tx[lane][i], a.beta64 * ty[lane][i]), v[i]);
        hi[i] = x.x;
        lo[i] = x.y;
      }
      __syncwarp();
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        hi[i] = v[i];
        lo[i] = 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int col = col0 + i;
      if (!a.sym || col >= row) vmax = fmaxf(vmax, fabsf(hi[i]));
      if (a.sym && col > row) a.C64[(size_t)col * a.ldc + row] = make_float2(hi[i], lo[i]);
      tx[lane][i] = hi[i];
      ty[lane][i] = lo[i];
    }
    __syncwarp();
    for (int i = 0; i < 32; ++i) {
      const int r = row0 + i, c = col0 + lane;
      if (!a.sym || c >= r) a.C64[(size_t)r * a.ldc + c] = make_float2(tx[i][lane], ty[i][lane]);
    }
    __syncwarp();
    return;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int col = col0 + i;
    if (!a.sym || col >= row) vmax = fmaxf(vmax, fabsf(v[i]));
    if (a.sym && col > row) a.C[(size_t)col * a.ldc + row] = v[i];
    tx[lane][i] = v[i];
  }
  __syncwarp();
  for (int i = 0; i < 32; ++i) {
    const int r = row0 + i, c = col0 + lane;
    if (!a.sym || c >= r) a.C[(size_t)r * a.ldc + c] = tx[i][lane];
  }
  __syncwarp();
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                   const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                   const __grid_constant__ CUtensorMap mA2hi, const __grid_constant__ CUtensorMap mA2lo,
                   const __grid_constant__ CUtensorMap mB2hi, const __grid_constant__ CUtensorMap mB2lo, TcArgs a) {
  constexpr int B_BYTES = BN * BK * 2;
  constexpr uint32_t TMEM_COLS = 2 * BN;   // two accumulators: 256 or 512 columns
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm, tn;
  if (a.tile_list) {
    tm = a.tile_list[2 * blockIdx.x];
    tn = a.tile_list[2 * blockIdx.x + 1];
  } else {
    // grouped raster: GROUP_M row panels at a time, so that the CTAs in flight
    // share their A and B panels in L2
    const int tiles_m = a.n / BM;
    const int per_group = kGroupM * a.tiles_n;
    const int g = blockIdx.x / per_group, r = blockIdx.x % per_group;
    const int first = g * kGroupM;
    const int gm = min(tiles_m - first, kGroupM);
    tm = first + r % gm;
    tn = r / gm;
  }
  // a tile outside the matrix (a bad tile list) is reported, never stored
  if (tm < 0 || tm >= a.n / BM || tn < 0 || tn >= a.tiles_n) {
    if (threadIdx.x == 0 && a.err) atomicExch(a.err, 4);
    return;
  }

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nk = a.K / BK;
  const int total = a.nseg * a.pairs * nk;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      KSeg q;
      kseg_begin(a, nk, q);
      for (int kb = 0; kb < total; ++kb, kseg_next(a, nk, q)) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (kb >= STAGES && !mbar_wait_fast(&empty[s], ph ^ 1)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        const int kk = q.kidx * BK;
        const CUtensorMap* ma = (q.kind == 2) ? (q.pr ? &mA2lo : &mAlo) : (q.pr ? &mA2hi : &mAhi);
        const CUtensorMap* mb = (q.kind == 1) ? (q.pr ? &mB2lo : &mBlo) : (q.pr ? &mB2hi : &mBhi);
        tma_load_2d(sA + s * A_BYTES, ma, kk, tm * BM, &full[s]);
        tma_load_2d(sB + s * B_BYTES, mb, kk, tn * BN, &full[s]);
      }
      if (!ok) atomicExch(a.err, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc_f16 = instr_desc(BN, 0);
      constexpr uint32_t idesc_bf16 = instr_desc(BN, 1);
      const uint32_t idesc = a.fmt ? idesc_bf16 : idesc_f16;
      for (int kb = 0; kb < total; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait_fast(&full[s], ph)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nk0 = acc1_start(a, nk);                // first K block of accumulator 1
        const uint32_t dcol = kb >= nk0 ? (uint32_t)BN : 0u;
        const bool first = (kb == 0) || (kb == nk0);
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {
          const uint64_t ad = smem_desc(sA + s * A_BYTES + j * 32);
          const uint64_t bd = smem_desc(sB + s * B_BYTES + j * 32);
          mma_f16(tmem + dcol, ad, bd, idesc, (first && j == 0) ? 0u : 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
      if (!ok) atomicExch(a.err, 2);
    }
  } else {
    // epilogue warps 2..5: TMEM lanes 32 * (warp % 4) ..
    const int q = warp & 3;
    {
      // while the tensor cores run, pull this tile's side inputs into L2
      const int t = (warp - 2) * 32 + lane;            // 0..127
      const int r = tm * BM + t;
      const float* fsides[2] = {a.E, a.E2};
      for (int k = 0; k < 2; ++k)
        if (fsides[k])
          for (int rr = t; rr < BN; rr += 128)
            for (int c = 0; c < BM; c += 32) prefetch_l2(fsides[k] + (size_t)(tn * BN + rr) * a.ldc + tm * BM + c);
      if (a.E64) {
        if (a.e64_trans) {
          for (int rr = t; rr < BN; rr += 128)
            for (int c = 0; c < BM; c += 16) prefetch_l2(a.E64 + (size_t)(tn * BN + rr) * a.ldc + tm * BM + c);
        } else {
          for (int c = 0; c < BN; c += 16) prefetch_l2(a.E64 + (size_t)r * a.ldc + tn * BN + c);
        }
      }
    }
    if (!mbar_wait(accf, 0)) {
      if (lane == 0) atomicExch(a.err, 3);
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row0 = tm * BM + q * 32;
      const int row = row0 + lane;
      const float inv = a.alpha / (__ldg(a.sa) * __ldg(a.sb));
      // per-warp 32 x 33 staging tiles in the (now idle) operand ring, so that
      // side inputs are loaded and outputs stored as whole 128-byte rows
      float(*tx)[33] = reinterpret_cast<float(*)[33]>(sA + q * (2 * 32 * 33 * 4));
      float(*ty)[33] = reinterpret_cast<float(*)[33]>(sA + q * (2 * 32 * 33 * 4) + 32 * 33 * 4);
      float vmax = 0.0f;
      for (int ch = 0; ch < BN / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32), v);
        if (a.nseg > 1 || a.split_acc) {
          float w[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(BN + ch * 32), w);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] += w[i];
        }
        const int col0 = tn * BN + ch * 32;
        // this lane holds row `row`, columns col0 .. col0 + 31
        epilogue_chunk(a, v, row, row0, col0, lane, tx, ty, inv, vmax);
      }
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0 && a.amax) atomicMax(a.amax, __float_as_uint(vmax));
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Persistent variant: one CTA per SM walks the tiles id = blockIdx.x, blockIdx.x + gridDim.x, ...
// The producer and MMA threads run ahead into the next tile while the epilogue drains the
// previous one.  Two accumulator modes:
//  - single products (one segment, hi*hi only): tiles alternate between the two accumulators
//    (tile it uses accumulator it % 2), so the whole MMA of the next tile overlaps the epilogue
//    of the previous one.  acc_full[b] and acc_free[b] carry one phase per use of accumulator b;
//    with one barrier pair per accumulator no barrier can run two phases ahead of its waiter.
//  - split products (three segments): the tensor core truncates as it accumulates, so the error
//    of a K-long sum grows with K.  The hi*hi sum is therefore accumulated in chunks of
//    chunk_kb K blocks, and the epilogue warps fold each finished chunk into the tile's sum with
//    round-to-nearest FP32 adds (tcgen05.ld + st).  A tile with parity p first accumulates the
//    two correction segments into accumulator p (while it is small), then each hi*hi chunk into
//    accumulator p ^ 1; after each chunk the epilogue folds accumulator p ^ 1 into accumulator p
//    and releases it for the next chunk, and after the last fold writes out accumulator p and
//    releases it.  Tiles alternate p, so a tile's long correction segments run while the
//    previous tile is written out from the other accumulator.  acc_full[0] carries one phase per
//    fold; acc_free[b] one phase per release of accumulator b, and the MMA thread waits for
//    release u - 1 of b before its u-th fresh write to b.  Each phase needs the previous one
//    consumed, so no barrier runs two phases ahead.
// Barriers: full/empty (operand ring), acc_full[2] (MMA -> epilogue), acc_free[2] (epilogue ->
// MMA, four warp arrivals per phase).  Every wait is bounded; a role that gives up records an
// error and raises a shared abort flag that ends the other roles' loops.

// Grouped launch (tab != null): tile id -> problem p of the group and its tile lid; tiles_per
// tiles per problem.  Otherwise one problem.
__device__ __forceinline__ void group_tile(const TcEntry* tab, int tiles_per, int id, int& p, int& lid) {
  if (tab) {
    p = id / tiles_per;
    lid = id - p * tiles_per;
  } else {
    p = 0;
    lid = id;
  }
}

// K-block order of one tile (the producer and the MMA thread walk it alike): the Cn correction
// K blocks first (hi*lo, lo*hi of pair 0, then of pair 1), then the hi*hi sequence (pair 0's K
// blocks, then pair 1's).  Counters only, no divisions.
struct KWalk {
  int phase;           // 0: corrections, 1: hi*hi
  int pr, kind, kidx;  // current K block: operand pair, split part (0 hi*hi, 1 hi*lo, 2 lo*hi), index
  int h, c;            // hi*hi and correction K blocks issued before the current one
};

__device__ __forceinline__ void kwalk_begin(KWalk& w, int Cn) {
  w.phase = Cn > 0 ? 0 : 1;
  w.pr = w.kidx = 0;
  w.kind = Cn > 0 ? 1 : 0;
  w.h = w.c = 0;
}

__device__ __forceinline__ void kwalk_next(KWalk& w, int nk, int Cn) {
  if (w.phase == 0) {
    ++w.c;
    if (++w.kidx == nk) {
      w.kidx = 0;
      if (w.kind == 1) {
        w.kind = 2;
      } else {
        w.kind = 1;
        ++w.pr;
      }
    }
    if (w.c == Cn) {
      w.phase = 1;
      w.pr = w.kind = w.kidx = 0;
    }
    return;
  }
  ++w.h;
  if (++w.kidx == nk) {
    w.kidx = 0;
    ++w.pr;
  }
}

// TF32: operands are TF32 words (kind::tf32, 32-element K blocks); else FP16 or BF16 by a.fmt.
template <int BN, bool TF32>
__global__ void __launch_bounds__(192, 1)
    gemm_tc_persistent_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                              const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                              const __grid_constant__ CUtensorMap mA2hi, const __grid_constant__ CUtensorMap mA2lo,
                              const __grid_constant__ CUtensorMap mB2hi, const __grid_constant__ CUtensorMap mB2lo,
                              TcArgs a, int ntiles, const TcEntry* __restrict__ tab, int tiles_per) {
  constexpr int B_BYTES = BN * BK * 2;
  constexpr uint32_t TMEM_COLS = 2 * BN;
  constexpr int STAGE_TILE = 32 * 33 * 4;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint8_t* stage = sB + STAGES * B_BYTES;   // 4 warps x 2 staging tiles of the epilogue
  uint64_t* full = reinterpret_cast<uint64_t*>(stage + 4 * 2 * STAGE_TILE);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;     // [2]
  uint64_t* acc_free = acc_full + 2;       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    mbar_init(&acc_free[0], 4);
    mbar_init(&acc_free[1], 4);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  constexpr int bk = TF32 ? BK / 2 : BK;           // elements per K block (one 128-byte row)
  const int nk = a.K / bk;
  const int total = a.nseg * a.pairs * nk;
  const bool chunked = a.nseg > 1;                 // split products; else single products alternate
  const int H = a.pairs * nk;                      // hi*hi K blocks
  const int Cn = total - H;                        // correction K blocks
  const int Lc = (chunked && a.chunk_kb > 0 && a.chunk_kb < H) ? a.chunk_kb : H;   // chunk length
  const int nchunks = (H + Lc - 1) / Lc;
  const int nfold = chunked ? nchunks : 0;   // folds per tile

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int last_p = -1;
      for (int id = blockIdx.x; id < ntiles && ok && !*abort_flag; id += gridDim.x) {
        int tm, tn, p, lid;
        group_tile(tab, tiles_per, id, p, lid);
        if (!tile_coords(a, lid, tm, tn)) {
          atomicExch(a.err, 4);
          *abort_flag = 1;
          break;
        }
        const CUtensorMap* maps = tab ? tab[p].map : nullptr;   // grouped: this problem's maps
        if (maps && p != last_p) {
          for (int i = 0; i < 8; ++i) tensormap_acquire(&maps[i]);
          last_p = p;
        }
        KWalk w;
        kwalk_begin(w, Cn);
        for (int kb = 0; kb < total; ++kb, ++g, kwalk_next(w, nk, Cn)) {
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (g >= STAGES && !mbar_wait_fast(&empty[s], ph ^ 1)) {
            atomicExch(a.err, 1);
            *abort_flag = 1;
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
          const int kk = w.kidx * bk;
          const int ia = (w.kind == 2) ? (w.pr ? 5 : 1) : (w.pr ? 4 : 0);
          const int ib = (w.kind == 1) ? (w.pr ? 7 : 3) : (w.pr ? 6 : 2);
          const CUtensorMap* ma = maps ? &maps[ia] : (w.kind == 2) ? (w.pr ? &mA2lo : &mAlo) : (w.pr ? &mA2hi : &mAhi);
          const CUtensorMap* mb = maps ? &maps[ib] : (w.kind == 1) ? (w.pr ? &mB2lo : &mBlo) : (w.pr ? &mB2hi : &mBhi);
          tma_load_2d(sA + s * A_BYTES, ma, kk, tm * BM, &full[s]);
          tma_load_2d(sB + s * B_BYTES, mb, kk, tn * BN, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc_f16 = instr_desc(BN, 0);
      constexpr uint32_t idesc_bf16 = instr_desc(BN, 1);
      constexpr uint32_t idesc_tf32 = instr_desc(BN, 2);
      const uint32_t idesc = TF32 ? idesc_tf32 : a.fmt ? idesc_bf16 : idesc_f16;
      uint32_t g = 0;
      int it = 0;
      int uses0 = 0, uses1 = 0;      // fresh writes of each accumulator so far (split products)
      int par = 0;                   // split products: accumulator parity p of this tile
      for (int id = blockIdx.x; id < ntiles && !*abort_flag; id += gridDim.x, ++it, par ^= 1) {
        int tm, tn;
        int p_, lid;
        group_tile(tab, tiles_per, id, p_, lid);
        if (!tile_coords(a, lid, tm, tn)) break;
        bool ok = true;
        const int buf = it & 1;      // single products: accumulator of this tile
        int cur = 0;                 // accumulator of the current step
        int bnd = 0;                 // first hi*hi K block of the next chunk
        KWalk w;
        kwalk_begin(w, Cn);
        for (int kb = 0; kb < total; ++kb, ++g, kwalk_next(w, nk, Cn)) {
          // does this K block start a step, and into which accumulator?
          int fresh = -1;            // accumulator written fresh from this K block, or -1
          if (!chunked) {
            if (kb == 0) fresh = buf;
          } else if (w.phase == 0) {
            if (w.c == 0) fresh = par;                     // corrections: the tile's sum accumulator
          } else if (w.h == bnd) {
            if (bnd > 0) mma_commit(&acc_full[0]);                    // the previous chunk is complete: fold it
            fresh = par ^ 1;                               // next hi*hi chunk
            bnd += Lc;
          }
          if (fresh >= 0) {
            // wait until the epilogue has released the accumulator's previous contents
            const int u = chunked ? (fresh ? uses1 : uses0) : (it >> 1);
            if (u > 0) {
              if (!mbar_wait_fast(&acc_free[fresh], (uint32_t)((u - 1) & 1)) || *abort_flag) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            if (chunked) {
              if (fresh)
                ++uses1;
              else
                ++uses0;
            }
            cur = fresh;
          }
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (!mbar_wait_fast(&full[s], ph)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dcol = cur ? (uint32_t)BN : 0u;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint64_t ad = smem_desc(sA + s * A_BYTES + j * 32);
            const uint64_t bd = smem_desc(sB + s * B_BYTES + j * 32);
            if constexpr (TF32)
              mma_tf32(tmem + dcol, ad, bd, idesc, (fresh >= 0 && j == 0) ? 0u : 1u);
            else
              mma_f16(tmem + dcol, ad, bd, idesc, (fresh >= 0 && j == 0) ? 0u : 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) {
          atomicExch(a.err, 2);
          *abort_flag = 1;
          break;
        }
        mma_commit(&acc_full[chunked ? 0 : buf]);         // last step of the tile
      }
    }
  } else {
    // epilogue warps 2..5: TMEM lanes 32 * (warp % 4) ..
    const int q = warp & 3;
    float(*tx)[33] = reinterpret_cast<float(*)[33]>(stage + q * 2 * STAGE_TILE);
    float(*ty)[33] = reinterpret_cast<float(*)[33]>(stage + q * 2 * STAGE_TILE + STAGE_TILE);
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int it = 0;
    uint32_t ev = 0;                 // acc_full[0] phases consumed (split products)
    int par = 0;                     // split products: accumulator parity p of this tile
    for (int id = blockIdx.x; id < ntiles && !*abort_flag; id += gridDim.x, ++it, par ^= 1) {
      int tm, tn, p, lid;
      group_tile(tab, tiles_per, id, p, lid);
      if (!tile_coords(a, lid, tm, tn)) break;
      const TcArgs& ea = tab ? tab[p].args : a;     // this problem's epilogue
      const float inv = ea.alpha / (__ldg(ea.sa) * __ldg(ea.sb));
      prefetch_sides<BN>(ea, tm, tn, (warp - 2) * 32 + lane);
      int src;                       // accumulator holding the tile's sum
      bool ok = true;
      if (!chunked) {
        src = it & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[src], (uint32_t)((it >> 1) & 1)));
        if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      } else {
        // fold f: accumulator (f % 2) ^ p += the other one, which is then released
        src = par;
        for (int f = 1; f <= nfold && ok; ++f, ++ev) {
          ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[0], ev & 1));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int dst = par, from = par ^ 1;
          // 64 columns at a time: both loads in flight before one wait
          for (int ch = 0; ch < BN / 64; ++ch) {
            uint32_t v[64], u[64];
            tmem_ld64_nowait(tmem + lane_base + (uint32_t)(from * BN + ch * 64), v);
            tmem_ld64_nowait(tmem + lane_base + (uint32_t)(dst * BN + ch * 64), u);
            tmem_wait_ld64(v);
            tmem_after_wait64(u);
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) + __uint_as_float(u[i]));
            tmem_st64(tmem + lane_base + (uint32_t)(dst * BN + ch * 64), v);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_free[from]);
          src = dst;
        }
      }
      if (!ok || *abort_flag) {
        if (lane == 0) atomicExch(a.err, 3);
        *abort_flag = 1;
        break;
      }
      // the epilogue proper from the accumulator that holds the sum
      const int row0 = tm * BM + q * 32;
      const int row = row0 + lane;
      float vmax = 0.0f;
      for (int ch = 0; ch < BN / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(src * BN + ch * 32), v);
        epilogue_chunk(ea, v, row, row0, tn * BN + ch * 32, lane, tx, ty, inv, vmax);
      }
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0 && ea.amax) atomicMax(ea.amax, __float_as_uint(vmax));
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_free[src]);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- two-SM products (cta_group::2) ----
//
// A cluster of two CTAs on two SMs computes a 256 x 256 output tile with tcgen05.mma.cta_group::2
// (M = 256, N = 256, K = 16): CTA r of the pair holds rows 128 r .. 128 r + 127 of the A tile and
// of the B tile in its own shared memory and rows 128 r .. of the accumulator in its own TMEM.
// The tensor cores of both SMs read both CTAs' operands, so each SM stages half as many B bytes
// per flop as the one-SM product: 32 KB per 64-wide K block instead of 48 KB, six ring stages
// instead of four, a third less shared-memory traffic per flop.  The accumulator modes (single
// products alternating accumulators, split products with chunked FP32 folds) are those of the
// one-SM persistent kernel, run by both CTAs' epilogue warps on their own TMEM lanes.
//
// Roles.  Both CTAs: warp 0 lane 0 loads the CTA's A and B halves of each K block by TMA,
// signalling the leader CTA's (rank 0) full barrier; warps 2-5 run the epilogue.  Leader only:
// warp 1 lane 0 waits for both halves (full), issues the MMAs and commits to the empty, acc_full
// barriers of both CTAs (multicast).  The epilogue warps of both CTAs release accumulators on the
// leader's acc_free barriers (eight warp arrivals per phase, four of them remote).  TMEM is
// allocated and freed collectively by warp 1 of both CTAs.  Cluster barriers after the barrier
// set-up and before the TMEM release are reached by every thread of both CTAs; every other wait
// is bounded.
constexpr int PSTAGES = 6;
constexpr int PB_BYTES = 128 * BK * 2;           // a CTA's half of the 256-row B tile
constexpr int kPairGroupM = 8;                   // 256-row panels per raster group

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// the shared::cluster address of the same shared-memory word in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(const void* p, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// TMA load into this CTA's shared memory that signals an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}

__device__ __forceinline__ void mma_f16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on the same barrier in both CTAs of the pair once the MMAs issued so far complete
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((unsigned short)3)
      : "memory");
}

// arrive on this CTA's barrier once the pair MMAs issued so far complete
__device__ __forceinline__ void mma_commit_pair_local(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool pair_tile_coords(const TcArgs& a, int id, int& tm, int& tn) {
  const int tiles = a.n / 256;
  if (a.tile_list) {
    tm = a.tile_list[2 * id];
    tn = a.tile_list[2 * id + 1];
  } else {
    const int per_group = kPairGroupM * tiles;
    const int g = id / per_group, r = id % per_group;
    const int first = g * kPairGroupM;
    const int gm = min(tiles - first, kPairGroupM);
    tm = first + r % gm;
    tn = r / gm;
  }
  return tm >= 0 && tm < tiles && tn >= 0 && tn < tiles;
}

__global__ void __launch_bounds__(192, 1)
    gemm_tc_pair_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                        const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                        const __grid_constant__ CUtensorMap mA2hi, const __grid_constant__ CUtensorMap mA2lo,
                        const __grid_constant__ CUtensorMap mB2hi, const __grid_constant__ CUtensorMap mB2lo,
                        TcArgs a, int ntiles) {
  constexpr int BN = 256;
  constexpr uint32_t TMEM_COLS = 2 * BN;
  constexpr int STAGE_TILE = 32 * 33 * 4;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + PSTAGES * A_BYTES;
  uint8_t* stage = sB + PSTAGES * PB_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(stage + 4 * 2 * STAGE_TILE);
  uint64_t* empty = full + PSTAGES;
  uint64_t* acc_full = empty + PSTAGES;    // [2]
  uint64_t* acc_free = acc_full + 2;       // [2], used in the leader
  uint64_t* drain = acc_full + 4;          // leader: completion of the last MMAs before teardown
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = (rank == 0);
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < PSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    mbar_init(&acc_free[0], 8);
    mbar_init(&acc_free[1], 8);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();   // both CTAs' barriers exist before any remote signal
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nk = a.K / BK;
  const int total = a.nseg * a.pairs * nk;
  const bool chunked = a.nseg > 1;
  const int H = a.pairs * nk;
  const int Cn = total - H;
  const int Lc = (chunked && a.chunk_kb > 0 && a.chunk_kb < H) ? a.chunk_kb : H;
  const int nchunks = (H + Lc - 1) / Lc;
  const int nfold = chunked ? nchunks : 0;

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t full_leader0 = map_to_rank(&full[0], 0);   // leader's full[0]; stages 8 bytes apart
      uint32_t g = 0;
      bool ok = true;
      for (int id = pair; id < ntiles && ok && !*abort_flag; id += npairs) {
        int tm, tn;
        if (!pair_tile_coords(a, id, tm, tn)) {
          atomicExch(a.err, 4);
          *abort_flag = 1;
          break;
        }
        const int arow = tm * 256 + (int)rank * 128, brow = tn * 256 + (int)rank * 128;
        KWalk w;
        kwalk_begin(w, Cn);
        for (int kb = 0; kb < total; ++kb, ++g, kwalk_next(w, nk, Cn)) {
          const int s = g % PSTAGES;
          const uint32_t ph = (g / PSTAGES) & 1;
          if (g >= PSTAGES && !mbar_wait_fast(&empty[s], ph ^ 1)) {
            atomicExch(a.err, 1);
            *abort_flag = 1;
            ok = false;
            break;
          }
          if (leader) mbar_expect_tx(&full[s], 2 * (A_BYTES + PB_BYTES));   // both CTAs' halves
          const int kk = w.kidx * BK;
          const CUtensorMap* ma = (w.kind == 2) ? (w.pr ? &mA2lo : &mAlo) : (w.pr ? &mA2hi : &mAhi);
          const CUtensorMap* mb = (w.kind == 1) ? (w.pr ? &mB2lo : &mBlo) : (w.pr ? &mB2hi : &mBhi);
          const uint32_t bar = full_leader0 + 8u * (uint32_t)s;
          tma_load_2d_pair(sA + s * A_BYTES, ma, kk, arow, bar);
          tma_load_2d_pair(sB + s * PB_BYTES, mb, kk, brow, bar);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      constexpr uint32_t idesc_f16 = instr_desc_m(256, BN, 0);
      constexpr uint32_t idesc_bf16 = instr_desc_m(256, BN, 1);
      const uint32_t idesc = a.fmt ? idesc_bf16 : idesc_f16;
      uint32_t g = 0;
      int it = 0;
      int uses0 = 0, uses1 = 0;
      int par = 0;
      bool issued = false;
      for (int id = pair; id < ntiles && !*abort_flag; id += npairs, ++it, par ^= 1) {
        int tm, tn;
        if (!pair_tile_coords(a, id, tm, tn)) break;
        bool ok = true;
        const int buf = it & 1;
        int cur = 0;
        int bnd = 0;
        KWalk w;
        kwalk_begin(w, Cn);
        for (int kb = 0; kb < total; ++kb, ++g, kwalk_next(w, nk, Cn)) {
          int fresh = -1;
          if (!chunked) {
            if (kb == 0) fresh = buf;
          } else if (w.phase == 0) {
            if (w.c == 0) fresh = par;                     // corrections: the tile's sum accumulator
          } else if (w.h == bnd) {
            if (bnd > 0) mma_commit_pair(&acc_full[0]);
            fresh = par ^ 1;                               // next hi*hi chunk
            bnd += Lc;
          }
          if (fresh >= 0) {
            const int u = chunked ? (fresh ? uses1 : uses0) : (it >> 1);
            if (u > 0) {
              if (!mbar_wait_fast(&acc_free[fresh], (uint32_t)((u - 1) & 1)) || *abort_flag) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            if (chunked) {
              if (fresh)
                ++uses1;
              else
                ++uses0;
            }
            cur = fresh;
          }
          const int s = g % PSTAGES;
          const uint32_t ph = (g / PSTAGES) & 1;
          if (!mbar_wait_fast(&full[s], ph)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dcol = cur ? (uint32_t)BN : 0u;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint64_t ad = smem_desc(sA + s * A_BYTES + j * 32);
            const uint64_t bd = smem_desc(sB + s * PB_BYTES + j * 32);
            mma_f16_pair(tmem + dcol, ad, bd, idesc, (fresh >= 0 && j == 0) ? 0u : 1u);
          }
          issued = true;
          mma_commit_pair(&empty[s]);
        }
        if (!ok) {
          atomicExch(a.err, 2);
          *abort_flag = 1;
          break;
        }
        mma_commit_pair(&acc_full[chunked ? 0 : buf]);
      }
      // no MMA may still write either CTA's TMEM when the pair frees it
      if (issued) {
        mma_commit_pair_local(drain);
        if (!mbar_wait(drain, 0)) atomicExch(a.err, 5);
      }
    }
  } else {
    const int q = warp & 3;
    float(*tx)[33] = reinterpret_cast<float(*)[33]>(stage + q * 2 * STAGE_TILE);
    float(*ty)[33] = reinterpret_cast<float(*)[33]>(stage + q * 2 * STAGE_TILE + STAGE_TILE);
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const float inv = a.alpha / (__ldg(a.sa) * __ldg(a.sb));
    const uint32_t free_leader0 = map_to_rank(&acc_free[0], 0), free_leader1 = map_to_rank(&acc_free[1], 0);
    int it = 0;
    uint32_t ev = 0;
    int par = 0;
    for (int id = pair; id < ntiles && !*abort_flag; id += npairs, ++it, par ^= 1) {
      int tm, tn;
      if (!pair_tile_coords(a, id, tm, tn)) break;
      const int tm128 = 2 * tm + (int)rank;          // this CTA's 128-row panel
      prefetch_sides<BN>(a, tm128, tn, (warp - 2) * 32 + lane);
      int src;
      bool ok = true;
      if (!chunked) {
        src = it & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[src], (uint32_t)((it >> 1) & 1)));
        if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      } else {
        src = par;
        for (int f = 1; f <= nfold && ok; ++f, ++ev) {
          ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[0], ev & 1));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int dst = par, from = par ^ 1;
          for (int ch = 0; ch < BN / 64; ++ch) {
            uint32_t v[64], u[64];
            tmem_ld64_nowait(tmem + lane_base + (uint32_t)(from * BN + ch * 64), v);
            tmem_ld64_nowait(tmem + lane_base + (uint32_t)(dst * BN + ch * 64), u);
            tmem_wait_ld64(v);
            tmem_after_wait64(u);
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) + __uint_as_float(u[i]));
            tmem_st64(tmem + lane_base + (uint32_t)(dst * BN + ch * 64), v);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(from ? free_leader1 : free_leader0);
          src = dst;
        }
      }
      if (!ok || *abort_flag) {
        if (lane == 0) atomicExch(a.err, 3);
        *abort_flag = 1;
        break;
      }
      const int row0 = tm128 * BM + q * 32;
      const int row = row0 + lane;
      float vmax = 0.0f;
      for (int ch = 0; ch < BN / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(src * BN + ch * 32), v);
        epilogue_chunk(a, v, row, row0, tn * BN + ch * 32, lane, tx, ty, inv, vmax);
      }
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0 && a.amax) atomicMax(a.amax, __float_as_uint(vmax));
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(src ? free_leader1 : free_leader0);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();   // the peer is done with this CTA's shared memory and TMEM
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- host side: tensor maps ----

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

struct MapKey {
  const void* p;
  int rows, box, fmt;
  bool operator==(const MapKey& o) const { return p == o.p && rows == o.rows && box == o.box && fmt == o.fmt; }
};
struct MapHash {
  size_t operator()(const MapKey& k) const {
    return std::hash<const void*>()(k.p) ^ (size_t)k.rows * 1315423911u ^ (size_t)k.box * 2654435761u ^ k.fmt;
  }
};

std::mutex g_map_mu;
std::unordered_map<MapKey, CUtensorMap, MapHash> g_maps;

// n x n row-major operand, boxes of one 128-byte swizzle row (64 16-bit or 32 TF32 elements) by
// box_rows rows; fmt 0 FP16, 1 BF16, 2 TF32 (FP32 words)
bool make_map(CUtensorMap* out, const void* base, int n, int box_rows, int fmt) {
  std::lock_guard<std::mutex> lk(g_map_mu);
  MapKey k{base, n, box_rows, fmt};
  auto it = g_maps.find(k);
  if (it != g_maps.end()) {
    *out = it->second;
    return true;
  }
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const int esz = fmt == 2 ? 4 : 2;
  cuuint64_t strides[1] = {(cuuint64_t)n * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  const CUtensorMapDataType dt = fmt == 2   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = enc(&m, dt, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  g_maps[k] = m;
  *out = m;
  return true;
}

template <int BN>
int smem_bytes() {
  return STAGES * (A_BYTES + BN * BK * 2) + (2 * STAGES + 1) * 8 + 16 + 1024;
}

template <int BN>
int smem_bytes_persistent() {
  return STAGES * (A_BYTES + BN * BK * 2) + 4 * 2 * 32 * 33 * 4 + (2 * STAGES + 4) * 8 + 16 + 1024;
}

int smem_bytes_pair() {
  return PSTAGES * (A_BYTES + PB_BYTES) + 4 * 2 * 32 * 33 * 4 + (2 * PSTAGES + 5) * 8 + 16 + 1024;
}

// 1: one-SM persistent CTAs (default); 2: two-SM products where n is a multiple of 256
// (XLBOMD_GEMM=pair), else one-SM persistent CTAs; 0: one CTA per output tile
// (XLBOMD_GEMM=classic).
int tc_variant() {
  static int v = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* e = std::getenv("XLBOMD_GEMM");
    const std::string x = e ? std::string(e) : std::string();
    v = (x == "classic") ? 0 : (x == "pair") ? 2 : 1;
  });
  return v;
}

// Per-device launch state: the SM count and whether each kernel's dynamic shared-memory limit
// has been raised on that device (a process may drive several devices).
constexpr int kMaxDevices = 64;
struct DeviceState {
  int sms = 0;
  int pair_clusters = 0;   // co-resident clusters of the two-SM product kernel
  bool smem_set[7] = {false, false, false, false, false, false, false};
};
std::mutex g_dev_mu;
DeviceState g_dev[kMaxDevices];

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  return dev;
}

int sm_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceState& d = g_dev[dev];
  if (d.sms <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return 148;
    }
    d.sms = n;
  }
  return d.sms;
}

// How many two-SM clusters of the pair kernel fit on the current device at once (its shared
// memory allows one CTA per SM; pairs must sit on SM pairs of one GPC).
int pair_clusters(int smem) {
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_dev[dev].pair_clusters > 0) return g_dev[dev].pair_clusters;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(192, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, gemm_tc_pair_kernel, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = sm_count() / 2;
  }
  std::lock_guard<std::mutex> lk(g_dev_mu);
  g_dev[dev].pair_clusters = n;
  return n;
}

// Raise kernel `slot`'s dynamic shared-memory limit to `bytes` on the current device (once per
// device; a failed attempt is retried on the next launch).
template <typename Kern>
cudaError_t ensure_smem(int slot, Kern kern, int bytes) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_dev[dev].smem_set[slot]) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_dev[dev].smem_set[slot] = true;
  return e;
}

// Persistent launch with tiles of width BN (grid CTAs, one per SM); TF32 operands (a.fmt = 2)
// take their own instantiation, so the FP16/BF16 kernel keeps compile-time K blocks.
template <int BN>
cudaError_t launch_persistent(cudaStream_t s, int grid, const CUtensorMap (&m)[8], const TcArgs& a, int ntiles,
                              const TcEntry* tab, int tiles_per) {
  const int sb = smem_bytes_persistent<BN>();
  const bool tf32 = a.fmt == 2;
  auto kern = tf32 ? gemm_tc_persistent_kernel<BN, true> : gemm_tc_persistent_kernel<BN, false>;
  const cudaError_t attr = ensure_smem((BN == 256 ? 0 : 1) + (tf32 ? 5 : 0), kern, sb);
  if (attr != cudaSuccess) return attr;
  kern<<<grid, 192, sb, s>>>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], a, ntiles, tab, tiles_per);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

void tc_forget_maps(const void* base) {
  std::lock_guard<std::mutex> lk(g_map_mu);
  for (auto it = g_maps.begin(); it != g_maps.end();) {
    if (it->first.p == base)
      it = g_maps.erase(it);
    else
      ++it;
  }
}

cudaError_t gemm_tc(cudaStream_t s, int n, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo,
                    TcArgs args, const TcTiles& tiles) {
  if (n % 128 != 0 || n <= 0) return cudaErrorInvalidValue;
  if (args.pairs != 1 && args.pairs != 2) return cudaErrorInvalidValue;
  const bool wide = (n % 256 == 0);
  if (args.fmt < 0 || args.fmt > 2) return cudaErrorInvalidValue;
  // TF32 operands run on the persistent kernel only
  const int variant = args.fmt == 2 ? 1 : tc_variant();
  const bool two_sm = (variant == 2) && wide && tiles.pair != nullptr;
  // B boxes: a CTA's 128-row half of the 256-row tile (two-SM), else the tile's bn rows
  const int bn = wide ? 256 : 128;
  const int bbox = two_sm ? 128 : bn;
  CUtensorMap mAhi, mAlo, mBhi, mBlo, mA2hi, mA2lo, mB2hi, mB2lo;
  if (!make_map(&mAhi, Ahi, n, BM, args.fmt) || !make_map(&mAlo, Alo ? Alo : Ahi, n, BM, args.fmt) ||
      !make_map(&mBhi, Bhi, n, bbox, args.fmt) || !make_map(&mBlo, Blo ? Blo : Bhi, n, bbox, args.fmt))
    return cudaErrorInvalidValue;
  if (args.pairs == 2) {
    // the swapped pair: B in the A role (BM-row boxes), A in the B role
    if (!make_map(&mA2hi, Bhi, n, BM, args.fmt) || !make_map(&mA2lo, Blo ? Blo : Bhi, n, BM, args.fmt) ||
        !make_map(&mB2hi, Ahi, n, bbox, args.fmt) || !make_map(&mB2lo, Alo ? Alo : Ahi, n, bbox, args.fmt))
      return cudaErrorInvalidValue;
  } else {
    mA2hi = mAhi;
    mA2lo = mAlo;
    mB2hi = mBhi;
    mB2lo = mBlo;
  }
  args.n = n;
  args.K = n;
  if (args.split_acc && n / BK < 2) return cudaErrorInvalidValue;   // both accumulators get K blocks
  args.tiles_n = n / bn;
  if (two_sm) {
    int ntiles;
    if (args.sym) {
      args.tile_list = tiles.pair;
      ntiles = tiles.npair;
    } else {
      args.tile_list = nullptr;
      ntiles = (n / 256) * (n / 256);
    }
    const int sb = smem_bytes_pair();
    const cudaError_t attr = ensure_smem(4, gemm_tc_pair_kernel, sb);
    if (attr != cudaSuccess) return attr;
    const int npairs = std::min(ntiles, pair_clusters(sb));
    if (const char* dbg = std::getenv("XLBOMD_DEBUG"))
      if (dbg[0] && dbg[0] != '0')
        std::fprintf(stderr, "[xlbomd] two-SM product n %d: %d tiles on %d CTA pairs (%d co-resident)\n", n, ntiles,
                     npairs, pair_clusters(sb));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = sb;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, gemm_tc_pair_kernel, mAhi, mAlo, mBhi, mBlo, mA2hi, mA2lo, mB2hi,
                                             mB2lo, args, ntiles);
    note_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  int nblocks;
  if (args.sym) {
    args.tile_list = wide ? tiles.sym256 : tiles.sym128;
    nblocks = wide ? tiles.n256 : tiles.n128;
  } else {
    args.tile_list = nullptr;
    nblocks = (n / BM) * (n / bn);
  }
  if (variant >= 1) {
    const int grid = std::min(nblocks, sm_count());
    const CUtensorMap maps[8] = {mAhi, mAlo, mBhi, mBlo, mA2hi, mA2lo, mB2hi, mB2lo};
    return wide ? launch_persistent<256>(s, grid, maps, args, nblocks, nullptr, 0)
                : launch_persistent<128>(s, grid, maps, args, nblocks, nullptr, 0);
  }
  if (wide) {
    const int sb = smem_bytes<256>();
    const cudaError_t attr = ensure_smem(2, gemm_tc_kernel<256>, sb);
    if (attr != cudaSuccess) return attr;
    gemm_tc_kernel<256><<<nblocks, 192, sb, s>>>(mAhi, mAlo, mBhi, mBlo, mA2hi, mA2lo, mB2hi, mB2lo, args);
    note_launch();
  } else {
    const int sb = smem_bytes<128>();
    const cudaError_t attr = ensure_smem(3, gemm_tc_kernel<128>, sb);
    if (attr != cudaSuccess) return attr;
    gemm_tc_kernel<128><<<nblocks, 192, sb, s>>>(mAhi, mAlo, mBhi, mBlo, mA2hi, mA2lo, mB2hi, mB2lo, args);
    note_launch();
  }
  return cudaGetLastError();
}

struct TcGroupCache {
  std::unordered_map<uint64_t, TcEntry*> tables;
};

TcGroupCache* tc_group_cache_new() { return new TcGroupCache(); }

void tc_group_cache_free(TcGroupCache* c) {
  if (!c) return;
  for (auto& kv : c->tables) cudaFree(kv.second);
  delete c;
}

namespace {
inline uint64_t fnv_mix(uint64_t h, uint64_t x) {
  for (int i = 0; i < 8; ++i) {
    h ^= (x >> (8 * i)) & 0xff;
    h *= 1099511628211ull;
  }
  return h;
}
template <typename T>
inline uint64_t bits_of(T v) {
  uint64_t x = 0;
  std::memcpy(&x, &v, sizeof(T) < 8 ? sizeof(T) : 8);
  return x;
}
}  // namespace

cudaError_t gemm_tc_group(cudaStream_t s, int n, const TcProblem* probs, int nprob, TcArgs shared,
                          const TcTiles& tiles, TcGroupCache* cache) {
  if (nprob < 1 || !cache || shared.fmt < 0 || shared.fmt > 2) return cudaErrorInvalidValue;
  if (n % 128 != 0 || n <= 0 || (shared.pairs != 1 && shared.pairs != 2)) return cudaErrorInvalidValue;
  if (nprob == 1) {
    TcArgs a = probs[0].epi;
    a.nseg = shared.nseg;
    a.pairs = shared.pairs;
    a.sym = shared.sym;
    a.fmt = shared.fmt;
    a.split_acc = shared.split_acc;
    a.chunk_kb = shared.chunk_kb;
    a.err = shared.err;
    return gemm_tc(s, n, probs[0].Ahi, probs[0].Alo, probs[0].Bhi, probs[0].Blo, a, tiles);
  }
  const bool wide = (n % 256 == 0) && shared.bn != 128;
  const int bn = wide ? 256 : 128;
  // table key: the problems' operands and epilogue arguments (a table is rebuilt only when
  // one of them changes)
  uint64_t key = 1469598103934665603ull;
  key = fnv_mix(key, (uint64_t)n * 1000003u + shared.nseg * 7 + shared.pairs * 31 + shared.sym * 131 +
                         shared.fmt * 521 + (uint64_t)bn * 7919);
  key = fnv_mix(key, (uint64_t)(shared.sym ? (wide ? tiles.sym256 : tiles.sym128) : nullptr));
  key = fnv_mix(key, (uint64_t)shared.err + (uint64_t)shared.chunk_kb);
  for (int i = 0; i < nprob; ++i) {
    const TcProblem& q = probs[i];
    const TcArgs& e = q.epi;
    const uint64_t w[] = {(uint64_t)q.Ahi, (uint64_t)q.Alo, (uint64_t)q.Bhi, (uint64_t)q.Blo, (uint64_t)e.E,
                          (uint64_t)e.E2, (uint64_t)e.E64, (uint64_t)e.C64, (uint64_t)e.dvec, (uint64_t)e.C,
                          (uint64_t)e.amax, (uint64_t)e.sa, (uint64_t)e.sb, bits_of(e.alpha), bits_of(e.beta),
                          bits_of(e.beta2), bits_of(e.beta64), bits_of(e.diag), bits_of(e.dvec_scale),
                          (uint64_t)e.e64_trans * 3 + (uint64_t)e.ndvec * 17 + (uint64_t)e.ldc * 65537};
    for (uint64_t x : w) key = fnv_mix(key, x);
  }
  TcArgs a = shared;
  a.n = n;
  a.K = n;
  a.tiles_n = n / bn;
  int tiles_per;
  if (a.sym) {
    a.tile_list = wide ? tiles.sym256 : tiles.sym128;
    tiles_per = wide ? tiles.n256 : tiles.n128;
  } else {
    a.tile_list = nullptr;
    tiles_per = (n / BM) * (n / bn);
  }
  TcEntry* table = nullptr;
  auto it = cache->tables.find(key);
  if (it != cache->tables.end()) {
    table = it->second;
  } else {
    std::vector<TcEntry> host(nprob);
    for (int i = 0; i < nprob; ++i) {
      const TcProblem& q = probs[i];
      TcEntry& t = host[i];
      const void* Alo = q.Alo ? q.Alo : q.Ahi;
      const void* Blo = q.Blo ? q.Blo : q.Bhi;
      if (!make_map(&t.map[0], q.Ahi, n, BM, shared.fmt) || !make_map(&t.map[1], Alo, n, BM, shared.fmt) ||
          !make_map(&t.map[2], q.Bhi, n, bn, shared.fmt) || !make_map(&t.map[3], Blo, n, bn, shared.fmt))
        return cudaErrorInvalidValue;
      if (shared.pairs == 2) {
        if (!make_map(&t.map[4], q.Bhi, n, BM, shared.fmt) || !make_map(&t.map[5], Blo, n, BM, shared.fmt) ||
            !make_map(&t.map[6], q.Ahi, n, bn, shared.fmt) || !make_map(&t.map[7], Alo, n, bn, shared.fmt))
          return cudaErrorInvalidValue;
      } else {
        t.map[4] = t.map[0];
        t.map[5] = t.map[1];
        t.map[6] = t.map[2];
        t.map[7] = t.map[3];
      }
      // the problem's epilogue arguments, with the launch's shared fields (the epilogue reads
      // sym, the kernel's walk n, K, nseg, pairs, ...)
      t.args = q.epi;
      t.args.n = a.n;
      t.args.K = a.K;
      t.args.nseg = a.nseg;
      t.args.pairs = a.pairs;
      t.args.sym = a.sym;
      t.args.fmt = a.fmt;
      t.args.split_acc = a.split_acc;
      t.args.chunk_kb = a.chunk_kb;
      t.args.bn = a.bn;
      t.args.tiles_n = a.tiles_n;
      t.args.tile_list = a.tile_list;
      t.args.err = a.err;
    }
    cudaError_t e = cudaMalloc((void**)&table, sizeof(TcEntry) * nprob);
    if (e != cudaSuccess) return e;
    // pageable source: the call returns once the bytes are staged, ordered on the stream
    e = cudaMemcpyAsync(table, host.data(), sizeof(TcEntry) * nprob, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(table);
      return e;
    }
    cache->tables[key] = table;
  }
  const int ntiles = nprob * tiles_per;
  const int grid = std::min(ntiles, sm_count());
  // the launch's own maps are unused (every problem's maps come from the table)
  CUtensorMap dummy[8];
  std::memset(dummy, 0, sizeof(dummy));
  return wide ? launch_persistent<256>(s, grid, dummy, a, ntiles, table, tiles_per)
              : launch_persistent<128>(s, grid, dummy, a, ntiles, table, tiles_per);
}

// Tile list of symmetric two-SM products: the 256 x 256 tiles (tm, tn) with tn >= tm, in the
// grouped raster of the dense products.
std::vector<int> tc_sym_tiles_pair(int n) {
  std::vector<int> t;
  const int tiles = n / 256;
  for (int first = 0; first < tiles; first += kPairGroupM) {
    const int gm = std::min(tiles - first, kPairGroupM);
    for (int tn = 0; tn < tiles; ++tn)
      for (int tm = first; tm < first + gm; ++tm)
        if (tn >= tm) {
          t.push_back(tm);
          t.push_back(tn);
        }
  }
  return t;
}

// Tile lists of symmetric products: tiles (tm, tn) of BM x bn that reach the
// upper triangle (bn tn + bn > BM tm), row-major order.
std::vector<int> tc_sym_tiles(int n, int bn) {
  std::vector<int> t;
  const int tiles_m = n / BM, tiles_n = n / bn;
  for (int first = 0; first < tiles_m; first += kGroupM) {
    const int gm = std::min(tiles_m - first, kGroupM);
    for (int tn = 0; tn < tiles_n; ++tn)
      for (int tm = first; tm < first + gm; ++tm)
        if (bn * tn + bn > BM * tm) {
          t.push_back(tm);
          t.push_back(tn);
        }
  }
  return t;
}

}  // namespace xl
