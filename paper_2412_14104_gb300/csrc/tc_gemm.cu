// Split-precision contractions on the 5th-generation tensor cores (sm_103a).
//
// A float64 operand x is split into two tensor-core numbers, x = hi + lo + O(2^-22 |x|)
// for TF32 (f = float(x), hi = tf32(f), lo = tf32(f - hi)) or O(2^-16 |x|) for BF16, and
// A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in tensor memory
// ("3xTF32" / "BF16x3").  Flow per contraction:
//   pack   : gather the multi-mode operand into a K-major, zero-padded [rows][K] panel of
//            hi and lo values (one pass over HBM, coalesced writes);
//   gemm   : persistent kernel, one CTA per SM walking 128 x 128 output tiles; warp 0
//            issues TMA loads of 128-byte K slices (SWIZZLE_128B) into a ring of
//            shared-memory stages, one thread of warp 1 issues tcgen05.mma (M = N = 128)
//            into one of two TMEM chunk buffers and frees a stage with tcgen05.commit,
//            sixteen epilogue warps fold every finished chunk (64 K elements) into
//            double-float sums kept in TMEM and write float64 results through the
//            multi-mode C strides (atomic adds when K is split across CTAs);
//   every mbarrier wait is bounded in time; a wait that runs out raises an error flag,
//   the CTA stops issuing work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>
#include <tuple>

#include "kernels.cuh"
#include "philox.cuh"

namespace tatrg {
namespace {

// bytes of K per shared-memory stage row: one SWIZZLE_64B or SWIZZLE_128B atom row
#ifndef TATRG_KSLICE
#define TATRG_KSLICE 128
#endif
// K elements accumulated in one FP32 chain before a drain into the double-float sums: 128
// halves the drains of 64 (the χ = 48 step 8 % faster) for ~1.7 times the per-step error of
// the float-grade forms (measured on the χ = 24 run)
#ifndef TATRG_CHAIN_K
#define TATRG_CHAIN_K 128
#endif

constexpr int TC_BM = 128;
constexpr int TC_BN = 128;
constexpr int KSLICE = TATRG_KSLICE;
static_assert(KSLICE == 64 || KSLICE == 128, "stage rows are one 64- or 128-byte swizzle atom");
constexpr int SMEM_BUDGET = 192 * 1024;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s: the bound of every mbarrier wait

__device__ int g_tc_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// the same with acquire at cluster scope: for barriers that CTAs of a pair arrive on remotely
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and the error flag) when the deadline passes
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  while (!(CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))) {
    if (now_ns() > deadline) {
      atomicExch(&g_tc_error, 1);
      return false;
    }
  }
  return true;
}
// CTA pairs (a cluster of two CTAs on two SMs sharing one MMA)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
// every thread of both CTAs of the pair
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// hint: bring a box into L2 ahead of its load (no shared memory, no barrier)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}
// the same box written to the same shared-memory offset of every CTA in `mask` (a cluster of
// this GPU's own CTAs), each of whose barriers at `bar`'s offset receives the bytes it got
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], "
      "[%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major operand tile in shared memory, KSLICE-byte rows, swizzled in 8-row atoms of
// 8 * KSLICE bytes (SWIZZLE_64B or SWIZZLE_128B).
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFF) >> 4);          // start address, 16-byte units
  d |= uint64_t(1) << 16;                         // leading byte offset (unused for this layout)
  d |= uint64_t((8 * KSLICE) >> 4) << 32;         // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                         // descriptor version
  d |= uint64_t(KSLICE == 128 ? 2 : 4) << 61;     // SWIZZLE_128B : SWIZZLE_64B
  return d;
}
// CG = 1: the MMA of one CTA; CG = 2: issued by the pair's first CTA for both (M = 256, each
// CTA holding 128 rows of A, half of the N columns of B and 128 lanes of the accumulator)
template <int PREC, int CG>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if (CG == 1 && PREC == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else if (CG == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else if (PREC == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
// completion of the MMAs issued so far arrives once on `bar`; with CG = 2 on the barrier at
// the same offset in both CTAs of the pair
template <int CG>
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  if (CG == 1) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  } else {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(smem_u32(bar)),
        "h"(uint16_t(3))
        : "memory");
  }
}
// completion of one CTA's MMAs issued so far arrives once on the barrier at `bar`'s offset
// in every CTA of `mask`
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  if (CG == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  } else {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
}
template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t cols) {
  if (CG == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
  else asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}
// 16 columns of 32 lanes; the caller waits with tmem_wait_ld before using r
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 8 columns of 32 lanes
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// Instruction descriptor for kind::tf32 (A/B format 2) or kind::f16 with bf16 (format 1),
// FP32 accumulator, both operands K-major, M = 128.
template <int PREC, int BM, int BN>
__device__ __forceinline__ constexpr uint32_t idesc() {
  return (1u << 4) | (uint32_t(PREC == 1 ? 2 : 1) << 7) | (uint32_t(PREC == 1 ? 2 : 1) << 10) |
         (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

// float <-> double by IEEE-754 bit manipulation on the integer pipes: this GPU has few FP64
// units, and a conversion on them costs as much as an FP64 add.  Values outside the
// normal range of float (zero, subnormals, overflow, inf, nan) take the hardware
// conversion.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 255u) {
    if ((u << 1) == 0u) return __longlong_as_double(int64_t(uint64_t(u) << 32));  // signed zero
    return double(f);
  }
  return __longlong_as_double(int64_t((uint64_t(u & 0x80000000u) << 32) | (uint64_t(e + 896u) << 52) |
                                      (uint64_t(u & 0x7FFFFFu) << 29)));
}
// round to nearest, ties to even
__device__ __forceinline__ float d2f_bits(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  if ((b << 1) == 0u) return __uint_as_float(uint32_t(b >> 32));  // signed zero
  const int e = int((b >> 52) & 0x7FFu) - 896;                     // biased float exponent
  if (e <= 0 || e >= 255) return __double2float_rn(x);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  uint32_t f = (uint32_t(b >> 32) & 0x80000000u) | (uint32_t(e) << 23) | uint32_t(m >> 29);
  const uint64_t rem = m & 0x1FFFFFFFull, half = 0x10000000ull;
  if (rem > half || (rem == half && (f & 1u))) f += 1u;  // a carry into the exponent rounds correctly
  return __uint_as_float(f);
}

struct TcArgs {
  DevModes mC;  // s1 = C stride of each M mode
  DevModes nC;  // s1 = C stride of each N mode
  int64_t M, N;
  int kb_per_split, nkb;
  int mtiles, ntiles;  // output tiles, walked in groups of GROUP_M row panels
  int split;           // K ranges per tile; work unit u = split index * tiles + tile
  double alpha, beta;
  int atomic;
  int n_contig;  // the C offset of output column n is n (the N modes run contiguously in C)
  double* C;
};

// Packed pairs of floats (sm_100+ f32x2 arithmetic, round to nearest in each lane).
__device__ __forceinline__ uint64_t pk(uint32_t lo, uint32_t hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}
__device__ __forceinline__ void unpk(uint64_t x, uint32_t& lo, uint32_t& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(x));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// (hi, lo) += v for two lanes at once: Knuth's TwoSum of hi and v, its error added to lo.
__device__ __forceinline__ void two_sum_acc2(uint64_t& hi, uint64_t& lo, uint64_t v) {
  const uint64_t s = add2(hi, v);
  const uint64_t bb = sub2(s, hi);
  const uint64_t e = add2(sub2(hi, sub2(s, bb)), sub2(v, bb));
  lo = add2(lo, e);
  hi = s;
}

// K stages ahead of the producer whose operand boxes are prefetched into L2 (0: none)
#ifndef TATRG_L2_PREFETCH
#define TATRG_L2_PREFETCH 0
#endif

// Output tile of work unit u: grouped raster (GROUP_M consecutive row panels sweep all
// column panels together, so the CTAs working at one time share a few A and B panels
// that stay in L2) and the K range of its split index.
struct Unit {
  int64_t m0, n0;
  int kb0, nk;
};
#ifndef TATRG_GROUP_M
#define TATRG_GROUP_M 8
#endif
template <int TILE_M>
__device__ __forceinline__ Unit unit_of(const TcArgs& g, int u) {
  constexpr int GROUP_M = TATRG_GROUP_M;
  const int tiles = g.mtiles * g.ntiles;
  const int sidx = u / tiles, b = u - sidx * tiles;
  const int per_group = GROUP_M * g.ntiles;
  const int first = (b / per_group) * GROUP_M;
  const int gsize = min(g.mtiles - first, GROUP_M);
  const int mt = first + (b % per_group) % gsize;
  const int nt = (b % per_group) / gsize;
  Unit w;
  w.m0 = int64_t(mt) * TILE_M;
  w.n0 = int64_t(nt) * TC_BN;
  w.kb0 = sidx * g.kb_per_split;
  w.nk = min(g.nkb, w.kb0 + g.kb_per_split) - w.kb0;
  return w;
}

// Persistent kernel: CTA b processes work units b, b + gridDim.x, ...; each unit is a
// 128 x 128 output tile over one K range.  The K loop is cut into chunks of KC stages;
// each chunk accumulates in one of NBUF TMEM buffers of 128 columns while the sixteen
// epilogue warps drain finished ones into per-thread double-float (hi, lo) sums, so no FP32
// accumulation chain in the tensor memory is longer than KC * 64 bytes of K.  The shared
// memory ring, the TMEM buffers and their barriers run on across units, so the loads and
// MMAs of the next unit overlap the drain and the stores of the current one.
constexpr int EPI_WARPS = 16;
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;

// AND of p over the epilogue warps (named barrier 1); every epilogue thread must call it.
__device__ __forceinline__ bool epilogue_all(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, 1, %2, a;\n"
      " selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"(uint32_t(p)), "r"(EPI_WARPS * 32)
      : "memory");
  return r != 0;
}

// PAIR: the CTAs of a cluster of two share each 256 x 128 tile: CTA r loads rows
// m0 + 128 r .. of A and rows n0 + 64 r .. of B (half of the tile's N) into its own shared
// memory, its tensor memory holds rows m0 + 128 r .. of the accumulator, and its epilogue
// writes them.  The first CTA (rank 0) issues the MMAs of both (cta_group::2); the second
// CTA's warp 1 tells it, through a barrier in the first CTA's shared memory, when each of
// its stages has landed, and the second CTA's epilogue warps arrive on the first CTA's
// accumulator-empty barriers.  Per SM this halves the B operand traffic of each MMA.
// NS slices per operand (2: hi, lo; 3: hi, mid, lo); the products kept are those whose
// slice indices (0 = hi) sum to at most NS - 1, issued smallest first
//   NS = 2: lo*hi, hi*lo, hi*hi;  NS = 3: lo*hi, hi*lo, mid*mid, mid*hi, hi*mid, hi*hi
template <int NS>
struct Products {
  static constexpr int n = NS == 2 ? 3 : 6;
  __device__ __forceinline__ static constexpr int a(int t) {
    return NS == 2 ? (t == 0 ? 1 : 0) : (t == 0 ? 2 : t == 1 ? 0 : t == 2 ? 1 : t == 3 ? 1 : 0);
  }
  __device__ __forceinline__ static constexpr int b(int t) {
    return NS == 2 ? (t == 1 ? 1 : 0) : (t == 0 ? 0 : t == 1 ? 2 : t == 2 ? 1 : t == 3 ? 0 : t == 4 ? 1 : 0);
  }
};

struct TcMaps {
  CUtensorMap a[3], b[3];  // slice panels of A and B (the first NS are used)
};

// Tile forms: FORM 0, one CTA per 128 x 128 tile; FORM 1, CTA pairs (cta_group::2: one MMA
// for a 256 x 128 tile, each CTA holding 128 rows of A and half of B); FORM 2, clusters of
// two CTAs with a 128 x 128 tile each, stacked in M, sharing the B tile: each CTA loads half
// of B's rows and multicasts them to both, so every CTA reads 3/4 of the operand bytes of
// FORM 0 from L2 for the same output.
template <int PREC, int NS, int KC, int STAGES, int NBUF, int FORM>
__global__ void __maxnreg__(96)  // 18 warps x 96 registers fit one SM's register file
    tc_gemm_kernel(const __grid_constant__ TcMaps maps, TcArgs g) {
  constexpr bool PAIR = FORM == 1, MC = FORM == 2, CLU = FORM != 0;
  constexpr int CG = PAIR ? 2 : 1;
  constexpr int BN = TC_BN;
  constexpr int TILE_M = CLU ? 2 * TC_BM : TC_BM;  // output rows per work unit
  constexpr int B_ROWS = PAIR ? BN / 2 : BN;       // rows of B (output columns) in a CTA's stage
  constexpr int B_LOAD = CLU ? BN / 2 : BN;        // rows of B a CTA loads per stage
  constexpr int A_TILE = TC_BM * KSLICE;    // bytes
  constexpr int B_TILE = B_ROWS * KSLICE;
  constexpr int STAGE = NS * (A_TILE + B_TILE);
  constexpr int KELEM = PREC == 1 ? KSLICE / 4 : KSLICE / 2;  // K elements per stage
  constexpr int TMEM_COLS = NBUF * BN + 2 * BN;  // chunk buffers, running hi, running lo
  static_assert(TMEM_COLS == 512, "the tensor memory holds exactly 512 columns");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], peer_full[STAGES], acc_full[NBUF],
      acc_empty[NBUF], fin_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int64_t col_off[BN];
  // per epilogue warp: a 32-row x 8-column slice of doubles (XOR-swizzled by row), through
  // which the warp turns its row-per-lane values into row-contiguous stores
  __shared__ __align__(16) double epi_stage[EPI_WARPS * 32 * 8];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = g.mtiles * g.ntiles * g.split;
  const uint32_t rank = CLU ? cluster_rank() : 0u;
  const int first = CLU ? int(blockIdx.x >> 1) : int(blockIdx.x);  // this CTA's (cluster's) first unit
  const int stride = CLU ? int(gridDim.x >> 1) : int(gridDim.x);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], MC ? 2 : 1);  // FORM 2: both CTAs' MMAs read the stage's B
      mbar_init(&peer_full[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], CG * EPI_WARPS);
    }
    mbar_init(&fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (CLU) cluster_sync_all();  // both CTAs' barriers exist before any remote arrive or copy
  if (warp == 1) tmem_alloc<CG>(&tmem_base_s, uint32_t(TMEM_COLS));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;  // stage uses, continued across units
      bool ok = true;
      for (int u = first; u < units && ok; u += stride) {
        const Unit w = unit_of<TILE_M>(g, u);
        const int ya = int(w.m0) + int(rank) * TC_BM, yb = int(w.n0) + int(rank) * B_LOAD;
        auto prefetch = [&](int j) {
#pragma unroll
          for (int p = 0; p < NS; ++p) {
            tma_prefetch_2d(&maps.a[p], (w.kb0 + j) * KELEM, ya);
            tma_prefetch_2d(&maps.b[p], (w.kb0 + j) * KELEM, yb);
          }
        };
        if (TATRG_L2_PREFETCH > 0)
          for (int j = 0; j < min(TATRG_L2_PREFETCH, w.nk); ++j) prefetch(j);
        for (int i = 0; i < w.nk; ++i, ++it) {
          if (TATRG_L2_PREFETCH > 0 && i + TATRG_L2_PREFETCH < w.nk) prefetch(i + TATRG_L2_PREFETCH);
          const int s = it % STAGES, round = it / STAGES;
          if (round > 0 && !mbar_wait<CLU>(&empty_bar[s], (round - 1) & 1, now_ns() + WAIT_NS)) { ok = false; break; }
          uint8_t* st = smem + s * STAGE;
          mbar_expect_tx(&full_bar[s], STAGE);  // FORM 2: half of B comes from the other CTA
          const int kx = (w.kb0 + i) * KELEM;
#pragma unroll
          for (int p = 0; p < NS; ++p) {
            tma_load_2d(st + p * A_TILE, &maps.a[p], &full_bar[s], kx, ya);
            if (MC)
              tma_load_2d_mc(st + NS * A_TILE + p * B_TILE + int(rank) * B_LOAD * KSLICE, &maps.b[p], &full_bar[s],
                             kx, yb, uint16_t(3));
            else
              tma_load_2d(st + NS * A_TILE + p * B_TILE, &maps.b[p], &full_bar[s], kx, yb);
          }
        }
      }
      // drain: the last loads issued into each stage must have landed before the CTA exits
      const uint64_t drain = now_ns() + WAIT_NS;
      for (int i = max(0, it - STAGES); i < it; ++i)
        mbar_wait(&full_bar[i % STAGES], (i / STAGES) & 1, drain);
    }
  } else if (warp == 1 && (!PAIR || rank == 0)) {
    if (lane == 0) {
      constexpr uint32_t id = idesc<PREC, PAIR ? 2 * TC_BM : TC_BM, BN>();
      int it = 0, cc = 0;  // stage uses and chunks, continued across units
      bool ok = true;
      for (int u = first; u < units && ok; u += stride) {
        const Unit w = unit_of<TILE_M>(g, u);
        const int nchunks = (w.nk + KC - 1) / KC;
        for (int c = 0; c < nchunks && ok; ++c, ++cc) {
          const int b = cc % NBUF, use = cc / NBUF;
          if (use > 0 && !mbar_wait<PAIR>(&acc_empty[b], (use - 1) & 1, now_ns() + WAIT_NS)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acc = tmem + uint32_t(b * BN);
          const int i_end = min(w.nk, (c + 1) * KC);
          for (int i = c * KC; i < i_end; ++i, ++it) {
            const int s = it % STAGES, round = it / STAGES;
            if (!mbar_wait(&full_bar[s], round & 1, now_ns() + WAIT_NS)) { ok = false; break; }
            if (PAIR && !mbar_wait<true>(&peer_full[s], round & 1, now_ns() + WAIT_NS)) { ok = false; break; }
            tc_fence_after();
            // descriptors of the stage's slices, formed once (the issuing thread is on the
            // critical path of every MMA)
            const uint64_t d0 = sdesc_sw(smem_u32(smem + s * STAGE));
            uint64_t ad[NS], bd[NS];
#pragma unroll
            for (int p = 0; p < NS; ++p) {
              ad[p] = d0 + uint64_t((p * A_TILE) >> 4);
              bd[p] = d0 + uint64_t((NS * A_TILE + p * B_TILE) >> 4);
            }
#pragma unroll
            for (int kk = 0; kk < KSLICE / 32; ++kk) {  // 32 bytes of K per instruction
              const uint64_t off = uint64_t(kk * 2);
#pragma unroll
              for (int t = 0; t < Products<NS>::n; ++t)
                mma<PREC, CG>(acc, ad[Products<NS>::a(t)] + off, bd[Products<NS>::b(t)] + off, id,
                              (i > c * KC || kk > 0 || t > 0) ? 1u : 0u);
            }
            if (MC) mma_commit_mc(&empty_bar[s], uint16_t(3));  // both CTAs wrote this stage's B
            else mma_commit<CG>(&empty_bar[s]);
          }
          if (ok) mma_commit<CG>(&acc_full[b]);
        }
      }
      // drain: every MMA issued by this thread completes before TMEM is released
      mma_commit<CG>(&fin_bar);
      mbar_wait<PAIR>(&fin_bar, 0, now_ns() + WAIT_NS);
    }
  } else if (warp == 1) {  // PAIR, rank 1
    if (lane == 0) {
      // second CTA of a pair: forward "stage landed" to the first CTA, which issues the MMAs
      const uint32_t peer0 = cluster_addr(&peer_full[0], 0);
      int it = 0;
      bool ok = true;
      for (int u = first; u < units && ok; u += stride) {
        const Unit w = unit_of<TILE_M>(g, u);
        for (int i = 0; i < w.nk; ++i, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (!mbar_wait(&full_bar[s], round & 1, now_ns() + WAIT_NS)) { ok = false; break; }
          mbar_arrive_remote(peer0 + uint32_t(s * sizeof(uint64_t)));
        }
      }
      // the first CTA's final commit also arrives here: its MMAs into this CTA's tensor
      // memory are complete before the memory is released
      mbar_wait<true>(&fin_bar, 0, now_ns() + WAIT_NS);
    }
  } else {
    // epilogue warps 2..17: TMEM lane quarter q = warp % 4 (the lanes a warp may access),
    // column quarter h.  The running double-float sums of the tile live in TMEM columns
    // [NBUF*BN, NBUF*BN + BN) (hi) and [NBUF*BN + BN, NBUF*BN + 2*BN) (lo), so the drain
    // needs few registers.
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = int(rank) * TC_BM + q * 32 + lane;  // row of the tile
    const uint32_t lanes = tmem + (uint32_t(q * 32) << 16);
    const uint32_t t_hi = lanes + uint32_t(NBUF * BN + h * 32);
    const uint32_t t_lo = lanes + uint32_t(NBUF * BN + BN + h * 32);
    const uint32_t empty0 = PAIR ? cluster_addr(&acc_empty[0], 0) : 0u;
    int cc = 0;
    bool ok = true;
#pragma unroll 1
    for (int u = first; u < units && ok; u += stride) {
      const Unit w = unit_of<TILE_M>(g, u);
      // per-column C offsets of this tile (the previous tile's stores are done with them)
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      for (int j = threadIdx.x - 64; j < BN; j += EPI_WARPS * 32) {
        int64_t a = 0, c = 0;
        if (w.n0 + j < g.N) mode_offsets(g.nC, w.n0 + j, a, c);
        col_off[j] = c;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      const int nchunks = (w.nk + KC - 1) / KC;
#pragma unroll 1
      for (int c = 0; c < nchunks; ++c, ++cc) {
        const int b = cc % NBUF, use = cc / NBUF;
        ok = __all_sync(0xffffffffu, (ok && mbar_wait<PAIR>(&acc_full[b], use & 1, now_ns() + WAIT_NS)) ? 1 : 0) != 0;
        if (!ok) break;
        tc_fence_after();
        const uint32_t ta = lanes + uint32_t(b * BN + h * 32);
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          uint32_t v[16], vh[16], vl[16];
          tmem_ld16_nowait(ta + uint32_t(16 * part), v);
          if (c > 0) {
            tmem_ld16_nowait(t_hi + uint32_t(16 * part), vh);
            tmem_ld16_nowait(t_lo + uint32_t(16 * part), vl);
          }
          tmem_wait_ld();
          if (part == 1) {  // the whole slice has been read: hand the buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (PAIR) mbar_arrive_remote(empty0 + uint32_t(b * sizeof(uint64_t)));
              else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
            }
          }
          if (c == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) { vh[j] = v[j]; vl[j] = 0u; }
          } else {
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              uint64_t h2 = pk(vh[j], vh[j + 1]), l2 = pk(vl[j], vl[j + 1]);
              two_sum_acc2(h2, l2, pk(v[j], v[j + 1]));
              unpk(h2, vh[j], vh[j + 1]);
              unpk(l2, vl[j], vl[j + 1]);
            }
          }
          tmem_st16(t_hi + uint32_t(16 * part), vh);
          tmem_st16(t_lo + uint32_t(16 * part), vl);
        }
        tmem_wait_st();
      }
      // one decision for all epilogue warps (a wait that ran out in any of them stops all)
      ok = epilogue_all(ok);
      if (ok) {
        const bool in_rows = (w.m0 + row) < g.M;
        int64_t roff = 0, dummy = 0;
        if (in_rows) mode_offsets(g.mC, w.m0 + row, dummy, roff);
        const double alpha = g.alpha, beta = g.beta;
        const int mode = g.atomic ? 2 : (beta != 0.0 ? 1 : 0);
        if (g.n_contig && mode != 2) {
          // coalesced: each slice of 8 columns goes through shared memory so that eight
          // lanes write 64 contiguous bytes of one row (four rows per store instruction)
          double* const stg = epi_stage + (warp - 2) * 256;
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            if (w.n0 + h * 32 + 16 * part >= g.N) break;  // the rest of this warp's columns are padding
            uint32_t vh[16], vl[16];
            tmem_ld16_nowait(t_hi + uint32_t(16 * part), vh);
            tmem_ld16_nowait(t_lo + uint32_t(16 * part), vl);
            tmem_wait_ld();
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              if (w.n0 + h * 32 + 16 * part + 8 * half >= g.N) break;
              __syncwarp();
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                const int j = 8 * half + c;
                double x = f2d_bits(__uint_as_float(vh[j])) + f2d_bits(__uint_as_float(vl[j]));
                if (alpha != 1.0) x *= alpha;
                stg[lane * 8 + (c ^ (lane & 7))] = x;
              }
              __syncwarp();
              const int cb = h * 32 + 16 * part + 8 * half;  // tile column of the slice
              const int c = lane & 7;
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int r = (lane >> 3) + 4 * i;  // row of the warp's 32
                const int64_t rb = __shfl_sync(0xffffffffu, roff, r);
                const int rin = __shfl_sync(0xffffffffu, in_rows ? 1 : 0, r);
                const double v = stg[r * 8 + (c ^ (r & 7))];
                if (rin && w.n0 + cb + c < g.N) {
                  double* p = g.C + rb + col_off[cb + c];
                  *p = (mode == 1) ? fma(beta, *p, v) : v;
                }
              }
            }
          }
        } else {
          double* const crow = g.C + roff;
          const int64_t rem_ = g.N - (w.n0 + h * 32);
          const int ncols = !in_rows ? 0 : (rem_ < 32 ? int(rem_) : 32);
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            uint32_t vh[16], vl[16];
            tmem_ld16_nowait(t_hi + uint32_t(16 * part), vh);
            tmem_ld16_nowait(t_lo + uint32_t(16 * part), vl);
            tmem_wait_ld();
            const int64_t* const co = col_off + h * 32 + 16 * part;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (16 * part + j < ncols) {
                double* p = crow + co[j];
                double x = f2d_bits(__uint_as_float(vh[j])) + f2d_bits(__uint_as_float(vl[j]));
                if (alpha != 1.0) x *= alpha;
                if (mode == 2) atomicAdd(p, x);
                else if (mode == 1) *p = fma(beta, *p, x);
                else *p = x;
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // a cluster: no CTA releases its tensor memory or exits while the other may still arrive
  // on its barriers or copy into its shared memory
  if (CLU) cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem, uint32_t(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------------
// Operand packing: dst[r * Kp + k] for r < Rp, k < Kp, zero outside the R x K operand.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One block packs a strip of PK_R rows x PK_K K-elements per iteration (grid-stride over
// strips).  The row and K offsets of the strip are decomposed once into shared memory.
// K-contiguous sources are read and written with the lanes along K (no staging);
// row-contiguous sources are read with the lanes along the rows into a shared tile and
// written from it with the lanes along K.
constexpr int PK_R = 32, PK_K = 128;

// destinations of the NS slices of a packed operand
struct PackDst {
  void* p[3];
};

template <int PREC, int NS>
__device__ __forceinline__ void pack_store(const PackDst& dst, int64_t o, double x) {
  // split the float nearest to x (its 24 bits hold more than hi + lo keep; hi + mid + lo of
  // bf16 keep all of them); each residual is exact in float
  const float f = d2f_bits(x);
  if (PREC == 1) {
    const float h = tf32_rna(f);
    const float l = tf32_rna(__fsub_rn(f, h));
    reinterpret_cast<float*>(dst.p[0])[o] = h;
    reinterpret_cast<float*>(dst.p[1])[o] = l;
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    const float r = __fsub_rn(f, __bfloat162float(h));
    const __nv_bfloat16 m = __float2bfloat16_rn(r);
    reinterpret_cast<__nv_bfloat16*>(dst.p[0])[o] = h;
    reinterpret_cast<__nv_bfloat16*>(dst.p[1])[o] = m;
    if (NS == 3) reinterpret_cast<__nv_bfloat16*>(dst.p[2])[o] = __float2bfloat16_rn(__fsub_rn(r, __bfloat162float(m)));
  }
}

// GEN: the operand is the Gaussian sketch whose element index is the offset the modes
// give (philox.cuh, float Box-Muller); src is not read.
template <int PREC, bool GEN>
__device__ __forceinline__ double operand_at(const double* __restrict__ src, const GaussSrc& gs,
                                             int64_t off) {
  if (GEN) {
    float z0, z1;
    gauss_pair_f32(gs.seed, gs.sid, gs.replica, off >> 1, z0, z1);
    return double((off & 1) ? z1 : z0);
  }
  return __ldg(src + off);
}

template <int PREC, int NS, bool GEN>
__global__ void __launch_bounds__(256) pack_kernel(const double* __restrict__ src, DevModes rm,
                                                   DevModes km, int64_t R, int64_t K, int64_t Kp,
                                                   int64_t ktiles, int64_t ntiles, PackDst dst,
                                                   int r_contig, GaussSrc gs) {
  __shared__ int64_t roff[PK_R], koff[PK_K];
  __shared__ double tile[PK_R][PK_K + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;  // 8 warps
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / ktiles) * PK_R, k0 = (t % ktiles) * PK_K;
    __syncthreads();  // the previous strip is done with roff, koff and tile
    if (tid < PK_R) {
      int64_t a = 0, b = 0;
      if (r0 + tid < R) mode_offsets(rm, r0 + tid, a, b);
      roff[tid] = a;
    } else if (tid < PK_R + PK_K) {
      const int j = tid - PK_R;
      int64_t a = 0, b = 0;
      if (k0 + j < K) mode_offsets(km, k0 + j, a, b);
      koff[j] = a;
    }
    __syncthreads();
    if (GEN) {
      // generated sketch: warp w takes the row pairs (2w, 2w + 1), (2w + 16, 2w + 17); when
      // the two rows hold consecutive sketch elements 2c, 2c + 1 (the row mode is the
      // innermost one), one Philox call gives both
#pragma unroll
      for (int i = 0; i < PK_R / 16; ++i) {
        const int rr = 2 * (warp + 8 * i);
        const int64_t r = r0 + rr;
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int kk = lane + 32 * j;
          const int64_t k = k0 + kk;
          if (k >= Kp) continue;
          double v0 = 0.0, v1 = 0.0;
          if (k < K) {
            const int64_t o0 = roff[rr] + koff[kk], o1 = roff[rr + 1] + koff[kk];
            if (r < R && r + 1 < R && o1 == o0 + 1 && (o0 & 1) == 0) {
              float z0, z1;
              gauss_pair_f32(gs.seed, gs.sid, gs.replica, o0 >> 1, z0, z1);
              v0 = double(z0);
              v1 = double(z1);
            } else {
              if (r < R) v0 = operand_at<PREC, true>(src, gs, o0);
              if (r + 1 < R) v1 = operand_at<PREC, true>(src, gs, o1);
            }
          }
          pack_store<PREC, NS>(dst, r * Kp + k, v0);
          pack_store<PREC, NS>(dst, (r + 1) * Kp + k, v1);
        }
      }
    } else if (!r_contig) {
      // warp w: rows w, w + 8, ...; lanes along K (coalesced reads and writes)
#pragma unroll
      for (int i = 0; i < PK_R / 8; ++i) {
        const int rr = warp + 8 * i;
        const int64_t r = r0 + rr;
        double v[PK_K / 32];
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int kk = lane + 32 * j;
          v[j] = (r < R && k0 + kk < K) ? operand_at<PREC, GEN>(src, gs, roff[rr] + koff[kk]) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int64_t k = k0 + lane + 32 * j;
          if (k < Kp) pack_store<PREC, NS>(dst, r * Kp + k, v[j]);
        }
      }
    } else {
      // lanes along the rows for the reads (the source is contiguous in r)
#pragma unroll
      for (int i = 0; i < PK_K / 8; ++i) {
        const int kk = warp + 8 * i;
        const bool ok = (r0 + lane < R) && (k0 + kk < K);
        tile[lane][kk] = ok ? operand_at<PREC, GEN>(src, gs, roff[lane] + koff[kk]) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PK_R / 8; ++i) {
        const int rr = warp + 8 * i;
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int64_t k = k0 + lane + 32 * j;
          if (k < Kp) pack_store<PREC, NS>(dst, (r0 + rr) * Kp + k, tile[rr][lane + 32 * j]);
        }
      }
    }
  }
}

__global__ void scale_c_kernel(double* C, DevModes m, DevModes n, int64_t M, int64_t N, double beta) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < M * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = e / N, j = e - (e / N) * N, a, c, b, d;
    mode_offsets(m, i, a, c);
    mode_offsets(n, j, b, d);
    double* p = C + c + d;
    *p = beta == 0.0 ? 0.0 : beta * *p;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {  // once, thread-safe
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

CUtensorMap make_map(void* base, int64_t rows, int64_t kp, int esize, int box_rows, int prec,
                     int kslice = KSLICE) {
  CUtensorMap m;
  cuuint64_t dims[2] = {cuuint64_t(kp), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(kp * esize)};
  cuuint32_t box[2] = {cuuint32_t(kslice / esize), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, prec == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           kslice == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TATRG_CHECK(r == CUDA_SUCCESS, TATRG_ECUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

// ---------------------------------------------------------------------------------
// Near-FP64 contractions from exact tensor-core products: the error-free splitting of a
// matrix product into products of slices (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms
// 59, 2012), with bf16 slices and FP32 accumulation.  Every row of A (every column of B)
// is scaled by 2^-e, e the exponent of its largest entry, and written as OZ_NS balanced
// base-2^7 digits: x = 2^e sum_{s=1..5} a_s 2^(-7s) + O(2^(e-36)), |a_1| <= 128,
// |a_s| <= 64 otherwise.  Slice s is stored as a_s 2^(-7(s-1)) (exact in bf16), so a slice
// product of level s + t carries the weight 2^(-7(s+t-2)) of its level.  Over a chunk of
// OZ_CHUNK K elements the level-2 product sum is an integer below 2^24, and the level-3
// sum a multiple of 2^-7 below 2^16: both exact in the FP32 accumulator.  The 15 products
// with s + t <= 6 are kept: levels 2 and 3 in one exact accumulator each, levels 4..6
// together (that sum is ~2^-14 of the result, so its float rounding is ~2^-38 relative).
// Each chunk is combined exactly (TwoSum) and added into double-float sums in tensor
// memory; the output is alpha 2^(e_row + e_col - 14) (hi + lo).
constexpr int OZ_NS = 5;                       // slices per operand
constexpr int OZ_BN = 64;                      // output columns per tile
constexpr int OZ_KS = 64;                      // bytes of K per stage row (SWIZZLE_64B)
constexpr int OZ_KELEM = OZ_KS / 2;            // bf16 K elements per stage
constexpr int OZ_STAGES = 3;
constexpr int OZ_CHUNK = 512;                  // 2 * 2^13 * 512 < 2^24: level-3 sums stay exact
constexpr int OZ_KC = OZ_CHUNK / OZ_KELEM;     // stages per chunk
constexpr int OZ_A_TILE = TC_BM * OZ_KS;       // bytes
constexpr int OZ_B_TILE = OZ_BN * OZ_KS;
constexpr int OZ_STAGE = OZ_NS * (OZ_A_TILE + OZ_B_TILE);
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;
constexpr int OZ_EXP_NONE = -1061109568;       // exponent of an all-zero row (bytes 0xC0)

// slice indices (0 = most significant) and accumulator of product t, smallest level first
__device__ __forceinline__ constexpr int oz_a(int t) {
  return t == 0 ? 4 : t == 1 ? 0 : t == 2 ? 3 : t == 3 ? 1 : t == 4 ? 2 : t == 5 ? 3 : t == 6 ? 0 : t == 7 ? 2
       : t == 8 ? 1 : t == 9 ? 2 : t == 10 ? 0 : t == 11 ? 1 : t == 12 ? 1 : 0;
}
__device__ __forceinline__ constexpr int oz_b(int t) {
  return t == 0 ? 0 : t == 1 ? 4 : t == 2 ? 1 : t == 3 ? 3 : t == 4 ? 2 : t == 5 ? 0 : t == 6 ? 3 : t == 7 ? 1
       : t == 8 ? 2 : t == 9 ? 0 : t == 10 ? 2 : t == 11 ? 1 : t == 12 ? 0 : t == 13 ? 1 : 0;
}
__device__ __forceinline__ constexpr int oz_acc(int t) { return t < 12 ? 2 : t < 14 ? 1 : 0; }
__device__ __forceinline__ constexpr bool oz_first(int t) { return t == 0 || t == 12 || t == 14; }

// K-major operand tile with 64-byte rows, SWIZZLE_64B (8-row atoms of 512 bytes)
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFF) >> 4);
  d |= uint64_t(1) << 16;
  d |= uint64_t((8 * OZ_KS) >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(4) << 61;  // SWIZZLE_64B
  return d;
}

// frexp exponent of a nonzero finite double from its bits (|x| < 2^e, e the result)
__device__ __forceinline__ int oz_exponent(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int ex = int((b >> 52) & 0x7FF);
  return ex == 0 ? OZ_EXP_NONE : ex - 1022;  // zero and subnormals count as zero
}

// the five balanced base-2^7 digits of x 2^(35 - e) rounded to an integer (integer
// arithmetic on the IEEE fields: this GPU has few FP64 units)
__device__ __forceinline__ void oz_digits(double x, int e, int (&d)[OZ_NS]) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int ex = int((b >> 52) & 0x7FF);
#pragma unroll
  for (int s = 0; s < OZ_NS; ++s) d[s] = 0;
  if (ex == 0 || e == OZ_EXP_NONE) return;
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (uint64_t(1) << 52);  // |x| = M 2^(ex - 1075)
  const int sh = 1040 - ex + e;                                          // >= 18 since |x| < 2^e
  int64_t F = sh >= 63 ? 0 : int64_t((M + (uint64_t(1) << (sh - 1))) >> sh);
  if (b >> 63) F = -F;
#pragma unroll
  for (int s = OZ_NS - 1; s > 0; --s) {
    const int64_t dd = ((F + 64) & 127) - 64;
    d[s] = int(dd);
    F = (F - dd) >> 7;
  }
  d[0] = int(F);
}

// Largest exponent of every row of a multi-mode operand (rows rm, K km): one block per
// strip of PK_R rows x PK_K K elements (grid-stride); row-contiguous sources are read with
// the lanes along the rows, the others with the lanes along K.
__global__ void __launch_bounds__(256) oz_exp_kernel(const double* __restrict__ src, DevModes rm, DevModes km,
                                                     int64_t R, int64_t K, int64_t ktiles, int64_t ntiles,
                                                     int* __restrict__ exps, int r_contig) {
  __shared__ int64_t roff[PK_R], koff[PK_K];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / ktiles) * PK_R, k0 = (t % ktiles) * PK_K;
    __syncthreads();
    if (tid < PK_R) {
      int64_t a = 0, c = 0;
      if (r0 + tid < R) mode_offsets(rm, r0 + tid, a, c);
      roff[tid] = a;
    } else if (tid < PK_R + PK_K) {
      const int j = tid - PK_R;
      int64_t a = 0, c = 0;
      if (k0 + j < K) mode_offsets(km, k0 + j, a, c);
      koff[j] = a;
    }
    __syncthreads();
    if (r_contig) {  // lane = row; warp w takes K elements w, w + 8, ...
      int m = OZ_EXP_NONE;
      if (r0 + lane < R)
        for (int kk = warp; kk < PK_K && k0 + kk < K; kk += 8) m = max(m, oz_exponent(__ldg(src + roff[lane] + koff[kk])));
      if (m != OZ_EXP_NONE) atomicMax(exps + r0 + lane, m);
    } else {  // warp w takes rows w, w + 8, ...; lanes along K
      for (int rr = warp; rr < PK_R; rr += 8) {
        if (r0 + rr >= R) break;
        int m = OZ_EXP_NONE;
        for (int kk = lane; kk < PK_K && k0 + kk < K; kk += 32) m = max(m, oz_exponent(__ldg(src + roff[rr] + koff[kk])));
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m != OZ_EXP_NONE) atomicMax(exps + r0 + rr, m);
      }
    }
  }
}

// The digit planes of a multi-mode operand: dst.p[s][r * Kp + k] = a_s of element (r, k),
// zero outside the R x K operand (same strip structure as pack_kernel).
__global__ void __launch_bounds__(256) oz_pack_kernel(const double* __restrict__ src, DevModes rm, DevModes km,
                                                      int64_t R, int64_t K, int64_t Kp, int64_t ktiles,
                                                      int64_t ntiles, const int* __restrict__ exps,
                                                      PackDst dst, PackDst dst2, int r_contig) {
  __shared__ int64_t roff[PK_R], koff[PK_K];
  __shared__ int rexp[PK_R];
  __shared__ double tile[PK_R][PK_K + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto store = [&](int64_t o, double x, int e) {
    int d[OZ_NS];
    oz_digits(x, e, d);
    __nv_bfloat16* const p[OZ_NS] = {reinterpret_cast<__nv_bfloat16*>(dst.p[0]),
                                     reinterpret_cast<__nv_bfloat16*>(dst.p[1]),
                                     reinterpret_cast<__nv_bfloat16*>(dst.p[2]),
                                     reinterpret_cast<__nv_bfloat16*>(dst2.p[0]),
                                     reinterpret_cast<__nv_bfloat16*>(dst2.p[1])};
    float w = 1.0f;  // 2^(-7 s): the level weight of slice s (exact: |d| <= 128)
#pragma unroll
    for (int s = 0; s < OZ_NS; ++s, w *= 0.0078125f) p[s][o] = __float2bfloat16_rn(float(d[s]) * w);
  };
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / ktiles) * PK_R, k0 = (t % ktiles) * PK_K;
    __syncthreads();
    if (tid < PK_R) {
      int64_t a = 0, c = 0;
      if (r0 + tid < R) mode_offsets(rm, r0 + tid, a, c);
      roff[tid] = a;
      rexp[tid] = r0 + tid < R ? exps[r0 + tid] : OZ_EXP_NONE;
    } else if (tid < PK_R + PK_K) {
      const int j = tid - PK_R;
      int64_t a = 0, c = 0;
      if (k0 + j < K) mode_offsets(km, k0 + j, a, c);
      koff[j] = a;
    }
    __syncthreads();
    if (!r_contig) {
#pragma unroll
      for (int i = 0; i < PK_R / 8; ++i) {
        const int rr = warp + 8 * i;
        const int64_t r = r0 + rr;
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int kk = lane + 32 * j;
          const int64_t k = k0 + kk;
          if (k >= Kp) continue;
          const double v = (r < R && k < K) ? __ldg(src + roff[rr] + koff[kk]) : 0.0;
          store(r * Kp + k, v, rexp[rr]);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < PK_K / 8; ++i) {
        const int kk = warp + 8 * i;
        const bool ok = (r0 + lane < R) && (k0 + kk < K);
        tile[lane][kk] = ok ? __ldg(src + roff[lane] + koff[kk]) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PK_R / 8; ++i) {
        const int rr = warp + 8 * i;
#pragma unroll
        for (int j = 0; j < PK_K / 32; ++j) {
          const int64_t k = k0 + lane + 32 * j;
          if (k < Kp) store((r0 + rr) * Kp + k, tile[rr][lane + 32 * j], rexp[rr]);
        }
      }
    }
  }
}

struct OzArgs {
  TcArgs g;           // mtiles over 128-row tiles, ntiles over OZ_BN-column tiles
  const int* ea;      // exponent of every packed row of A
  const int* eb;      // exponent of every packed row of B (output column)
};
struct OzMaps {
  CUtensorMap a[OZ_NS], b[OZ_NS];
};

__device__ __forceinline__ Unit oz_unit_of(const TcArgs& g, int u) {
  constexpr int GROUP_M = TATRG_GROUP_M;
  const int tiles = g.mtiles * g.ntiles;
  const int sidx = u / tiles, b = u - sidx * tiles;
  const int per_group = GROUP_M * g.ntiles;
  const int first = (b / per_group) * GROUP_M;
  const int gsize = min(g.mtiles - first, GROUP_M);
  const int mt = first + (b % per_group) % gsize;
  const int nt = (b % per_group) / gsize;
  Unit w;
  w.m0 = int64_t(mt) * TC_BM;
  w.n0 = int64_t(nt) * OZ_BN;
  w.kb0 = sidx * g.kb_per_split;
  w.nk = min(g.nkb, w.kb0 + g.kb_per_split) - w.kb0;
  return w;
}

// Persistent kernel with the roles of tc_gemm_kernel (warp 0 TMA, one thread of warp 1
// MMA, 16 epilogue warps); tensor memory: two buffers of three 64-column accumulators
// (columns 0..383), running hi (384..447) and lo (448..511).
__global__ void __maxnreg__(96) oz_gemm_kernel(const __grid_constant__ OzMaps maps, OzArgs args) {
  constexpr int NACC = 3, ACC_COLS = NACC * OZ_BN, HI = 2 * ACC_COLS, LO = HI + OZ_BN;
  static_assert(LO + OZ_BN == 512, "the tensor memory holds exactly 512 columns");
  const TcArgs& g = args.g;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[OZ_STAGES], empty_bar[OZ_STAGES], acc_full[2], acc_empty[2], fin_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int64_t col_off[OZ_BN];
  __shared__ int col_exp[OZ_BN];
  __shared__ __align__(16) double epi_stage[EPI_WARPS * 32 * 8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = g.mtiles * g.ntiles * g.split;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);
    }
    mbar_init(&fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<1>(&tmem_base_s, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const Unit w = oz_unit_of(g, u);
        for (int i = 0; i < w.nk; ++i, ++it) {
          const int s = it % OZ_STAGES, round = it / OZ_STAGES;
          if (round > 0 && !mbar_wait(&empty_bar[s], (round - 1) & 1, now_ns() + WAIT_NS)) { ok = false; break; }
          uint8_t* st = smem + s * OZ_STAGE;
          mbar_expect_tx(&full_bar[s], OZ_STAGE);
          const int kx = (w.kb0 + i) * OZ_KELEM;
#pragma unroll
          for (int p = 0; p < OZ_NS; ++p) {
            tma_load_2d(st + p * OZ_A_TILE, &maps.a[p], &full_bar[s], kx, int(w.m0));
            tma_load_2d(st + OZ_NS * OZ_A_TILE + p * OZ_B_TILE, &maps.b[p], &full_bar[s], kx, int(w.n0));
          }
        }
      }
      const uint64_t drain = now_ns() + WAIT_NS;
      for (int i = max(0, it - OZ_STAGES); i < it; ++i) mbar_wait(&full_bar[i % OZ_STAGES], (i / OZ_STAGES) & 1, drain);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id = idesc<2, TC_BM, OZ_BN>();
      int it = 0, cc = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const Unit w = oz_unit_of(g, u);
        const int nchunks = (w.nk + OZ_KC - 1) / OZ_KC;
        for (int c = 0; c < nchunks && ok; ++c, ++cc) {
          const int b = cc & 1, use = cc >> 1;
          if (use > 0 && !mbar_wait(&acc_empty[b], (use - 1) & 1, now_ns() + WAIT_NS)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acc = tmem + uint32_t(b * ACC_COLS);
          const int i_end = min(w.nk, (c + 1) * OZ_KC);
          for (int i = c * OZ_KC; i < i_end; ++i, ++it) {
            const int s = it % OZ_STAGES, round = it / OZ_STAGES;
            if (!mbar_wait(&full_bar[s], round & 1, now_ns() + WAIT_NS)) { ok = false; break; }
            tc_fence_after();
            const uint64_t d0 = sdesc_sw64(smem_u32(smem + s * OZ_STAGE));
            uint64_t ad[OZ_NS], bd[OZ_NS];
#pragma unroll
            for (int p = 0; p < OZ_NS; ++p) {
              ad[p] = d0 + uint64_t((p * OZ_A_TILE) >> 4);
              bd[p] = d0 + uint64_t((OZ_NS * OZ_A_TILE + p * OZ_B_TILE) >> 4);
            }
#pragma unroll
            for (int kk = 0; kk < OZ_KS / 32; ++kk) {  // 16 bf16 of K per instruction
              const uint64_t off = uint64_t(kk * 2);
#pragma unroll
              for (int t = 0; t < 15; ++t)
                mma<2, 1>(acc + uint32_t(oz_acc(t) * OZ_BN), ad[oz_a(t)] + off, bd[oz_b(t)] + off, id,
                          (i > c * OZ_KC || kk > 0 || !oz_first(t)) ? 1u : 0u);
            }
            mma_commit<1>(&empty_bar[s]);
          }
          if (ok) mma_commit<1>(&acc_full[b]);
        }
      }
      mma_commit<1>(&fin_bar);
      mbar_wait(&fin_bar, 0, now_ns() + WAIT_NS);
    }
  } else {
    // epilogue warps 2..17: lane quarter q, column quarter h (16 of the 64 columns)
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t lanes = tmem + (uint32_t(q * 32) << 16);
    int cc = 0;
    bool ok = true;
#pragma unroll 1
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const Unit w = oz_unit_of(g, u);
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      for (int j = threadIdx.x - 64; j < OZ_BN; j += EPI_WARPS * 32) {
        int64_t a = 0, c = 0;
        if (w.n0 + j < g.N) mode_offsets(g.nC, w.n0 + j, a, c);
        col_off[j] = c;
        const int e = args.eb[w.n0 + j];
        col_exp[j] = e == OZ_EXP_NONE ? 0 : e;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      const int nchunks = (w.nk + OZ_KC - 1) / OZ_KC;
#pragma unroll 1
      for (int c = 0; c < nchunks; ++c, ++cc) {
        const int b = cc & 1, use = cc >> 1;
        ok = __all_sync(0xffffffffu, (ok && mbar_wait(&acc_full[b], use & 1, now_ns() + WAIT_NS)) ? 1 : 0) != 0;
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const uint32_t col = uint32_t(h * 16 + part * 8);
          uint32_t v0[8], v1[8], v2[8], vh[8], vl[8];
          tmem_ld8_nowait(lanes + uint32_t(b * ACC_COLS) + col, v0);
          tmem_ld8_nowait(lanes + uint32_t(b * ACC_COLS + OZ_BN) + col, v1);
          tmem_ld8_nowait(lanes + uint32_t(b * ACC_COLS + 2 * OZ_BN) + col, v2);
          if (c > 0) {
            tmem_ld8_nowait(lanes + uint32_t(HI) + col, vh);
            tmem_ld8_nowait(lanes + uint32_t(LO) + col, vl);
          }
          tmem_wait_ld();
          if (part == 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
              asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // the chunk: level 2 (exact) + level 3 (exact) + levels 4..6, each already in
            // units of the level-2 weight
            const float x0 = __uint_as_float(v0[j]), x1 = __uint_as_float(v1[j]);
            const float sum = __fadd_rn(x0, x1), bb = __fsub_rn(sum, x0);
            float err = __fadd_rn(__fsub_rn(x0, __fsub_rn(sum, bb)), __fsub_rn(x1, bb));
            err = __fadd_rn(err, __uint_as_float(v2[j]));
            if (c == 0) {
              vh[j] = __float_as_uint(sum);
              vl[j] = __float_as_uint(err);
            } else {
              const float hi = __uint_as_float(vh[j]);
              const float t2 = __fadd_rn(hi, sum), b2 = __fsub_rn(t2, hi);
              const float e2 = __fadd_rn(__fsub_rn(hi, __fsub_rn(t2, b2)), __fsub_rn(sum, b2));
              vh[j] = __float_as_uint(t2);
              vl[j] = __float_as_uint(__fadd_rn(__uint_as_float(vl[j]), __fadd_rn(e2, err)));
            }
          }
          tmem_st8(lanes + uint32_t(HI) + col, vh);
          tmem_st8(lanes + uint32_t(LO) + col, vl);
        }
        tmem_wait_st();
      }
      ok = epilogue_all(ok);
      if (ok) {
        const bool in_rows = (w.m0 + row) < g.M;
        int64_t roff = 0, dummy = 0;
        if (in_rows) mode_offsets(g.mC, w.m0 + row, dummy, roff);
        const int er0 = args.ea[w.m0 + row];
        const int er = (er0 == OZ_EXP_NONE ? 0 : er0) - 14;
        const double alpha = g.alpha, beta = g.beta;
        const int mode = g.atomic ? 2 : (beta != 0.0 ? 1 : 0);
        double* const stg = epi_stage + (warp - 2) * 256;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const int cb = h * 16 + part * 8;  // tile column of the slice
          if (w.n0 + cb >= g.N) break;
          uint32_t vh[8], vl[8];
          tmem_ld8_nowait(lanes + uint32_t(HI + cb), vh);
          tmem_ld8_nowait(lanes + uint32_t(LO + cb), vl);
          tmem_wait_ld();
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            double x = f2d_bits(__uint_as_float(vh[c])) + f2d_bits(__uint_as_float(vl[c]));
            x = ldexp(x, er + col_exp[cb + c]);
            if (alpha != 1.0) x *= alpha;
            stg[lane * 8 + (c ^ (lane & 7))] = x;
          }
          __syncwarp();
          const int c = lane & 7;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = (lane >> 3) + 4 * i;
            const int64_t rb = __shfl_sync(0xffffffffu, roff, r);
            const int rin = __shfl_sync(0xffffffffu, in_rows ? 1 : 0, r);
            const double v = stg[r * 8 + (c ^ (r & 7))];
            if (rin && w.n0 + cb + c < g.N) {
              double* p = g.C + rb + col_off[cb + c];
              if (mode == 2) atomicAdd(p, v);
              else *p = (mode == 1) ? fma(beta, *p, v) : v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<1>(tmem, 512u);
  }
}

// Shared-memory ring of the kernel: stages of the NS slices of A and of B.
// launch policy for the two-CTA tile forms: 0 = the autotuner decides (single CTAs
// untuned), 1 = CTA pairs (FORM 1) wherever they apply, 2 = multicast clusters (FORM 2)
// wherever they apply, -1 = never
std::atomic<int> g_pair_mode{0};

template <int NS, int FORM>
constexpr int stage_bytes() { return NS * (TC_BM * KSLICE + (FORM == 1 ? TC_BN / 2 : TC_BN) * KSLICE); }

// Largest number of CTAs (of clusters) that are resident at once, per device.
template <int PREC, int NS, int FORM>
int resident_units(const void* kfn, int smem) {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  TATRG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> l(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  TATRG_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int n = 0;
  if (FORM != 0) {
    TATRG_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * unsigned(sm_count() / 2));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TATRG_CUDA(cudaOccupancyMaxActiveClusters(&n, kfn, &cfg));
  } else {
    int per_sm = 0;
    TATRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, TC_THREADS, smem));
    n = per_sm >= 1 ? sm_count() : 0;  // one CTA per SM: the ring admits no second one
  }
  TATRG_CHECK(n >= 1, TATRG_ECUDA, "gemm_tc: the tensor-core kernel does not fit on the device");
  cache[dev] = n;
  return n;
}

template <int PREC, int NS, int FORM>
void launch(const TcMaps& maps, const TcArgs& a, int64_t units, cudaStream_t s) {
  constexpr int STAGE = stage_bytes<NS, FORM>();
  constexpr int STAGES = SMEM_BUDGET / STAGE;
  static_assert(STAGES >= 2, "the ring needs two stages");
  constexpr int KC_ = TATRG_CHAIN_K / (PREC == 1 ? KSLICE / 4 : KSLICE / 2);  // stages per FP32 chain
  constexpr int KC = KC_ > 0 ? KC_ : 1;  // at least one stage
  constexpr int SMEM = STAGES * STAGE + 1024;
  auto k = tc_gemm_kernel<PREC, NS, KC, STAGES, 2, FORM>;
  const int resident = resident_units<PREC, NS, FORM>(reinterpret_cast<const void*>(k), SMEM);
  // persistent: every CTA (cluster) walks units b, b + grid, ...; no more than are resident
  const unsigned n = unsigned(std::min<int64_t>(units, resident));
  if (FORM == 0) {
    k<<<n, TC_THREADS, SMEM, s>>>(maps, a);
  } else {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * n);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = size_t(SMEM);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TATRG_CUDA(cudaLaunchKernelEx(&cfg, k, maps, a));
  }
  TATRG_CUDA(cudaGetLastError());
}

// The two-CTA tile forms for the contractions with many 256-row tiles (set TATRG_CTA_PAIR=0
// to use single CTAs everywhere, e.g. to compare).
bool pairs_enabled() {
  static const bool on = []() {
    const char* e = getenv("TATRG_CTA_PAIR");
    return !(e && e[0] == '0');
  }();
  return on && g_pair_mode.load() >= 0;
}

}  // namespace

bool tc_available() {
  // per device ordinal: a process may drive several GPUs
  static std::mutex mu;
  static std::map<int, bool> ok_on;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> l(mu);
  auto it = ok_on.find(dev);
  if (it != ok_on.end()) return it->second;
  int major = 0, minor = 0;
  const bool ok = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess &&
                  major == 10 && minor == 3 && encode_fn() != nullptr;
  ok_on[dev] = ok;
  return ok;
}

void set_pair_mode(int mode) { g_pair_mode.store(mode); }

int tc_error_flag(bool reset) {
  int h = 0;
  cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int));
  if (reset && h) {
    int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  }
  return h;
}

namespace {
// Autotuner of the launch configuration: the first time a large contraction of a given
// shape is seen on a device (and its output is overwritten, beta = 0), every candidate --
// each tile form, the split-K heuristic's factor, half and twice it -- runs once
// on the real operands, timed with CUDA events; the fastest is kept for that shape.  Each
// candidate computes the whole result, so the output of the last one stands.  Smaller
// contractions, and shapes not yet tuned whose output is accumulated into, take the
// heuristic on single CTAs.  TATRG_AUTOTUNE=0 turns tuning off.
struct TcChoice {
  int form = 0;  // tile form of tc_gemm_kernel
  int split = 1;
};

constexpr double kTuneFlops = 2e11;  // contractions below this are not tuned

template <class Heur, class Run>
TcChoice tuned_choice(int prec, int64_t M, int64_t N, int64_t K, int n_contig, bool pair_ok, bool may_tune,
                      Heur& heuristic, Run& run, cudaStream_t s) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int64_t, int64_t, int64_t, int, bool>, TcChoice> cache;
  static const bool on = []() {
    const char* e = getenv("TATRG_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  int dev = 0;
  TATRG_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, prec, M, N, K, n_contig, pair_ok);
  {
    std::lock_guard<std::mutex> l(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  TcChoice def;  // untuned: single CTAs
  def.form = 0;
  def.split = heuristic(false);
  const int mode = g_pair_mode.load();
  if (pair_ok && (mode == 1 || mode == 2)) return TcChoice{mode, heuristic(true)};
  if (!on || !may_tune || 2.0 * double(M) * double(N) * double(K) < kTuneFlops) return def;
  std::vector<TcChoice> cand;
  for (int f = 0; f <= (pair_ok ? 2 : 0); ++f) {
    const int h = heuristic(f != 0);
    for (int sp : {h, std::max(1, h / 2), std::min(512, 2 * h)}) {
      bool dup = false;
      for (const auto& c : cand) dup = dup || (c.form == f && c.split == sp);
      if (!dup) cand.push_back(TcChoice{f, sp});
    }
  }
  cudaEvent_t ev[2];
  TATRG_CUDA(cudaEventCreate(&ev[0]));
  TATRG_CUDA(cudaEventCreate(&ev[1]));
  TcChoice best = def;
  float best_ms = 1e30f;
  for (const auto& c : cand) {
    TATRG_CUDA(cudaEventRecord(ev[0], s));
    run(c.form, c.split);
    TATRG_CUDA(cudaEventRecord(ev[1], s));
    TATRG_CUDA(cudaEventSynchronize(ev[1]));
    float ms = 0.f;
    TATRG_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  static const bool log = []() {
    const char* e = getenv("TATRG_AUTOTUNE_LOG");
    return e && e[0] == '1';
  }();
  if (log)
    fprintf(stderr, "tatrg autotune: M=%lld N=%lld K=%lld prec=%d -> %s split %d (%.3f ms of %zu candidates)\n",
            (long long)M, (long long)N, (long long)K, prec,
            best.form == 2 ? "multicast cluster" : best.form == 1 ? "pair" : "single", best.split, best_ms,
            cand.size());
  std::lock_guard<std::mutex> l(mu);
  cache[key] = best;
  return best;
}
}  // namespace

void gemm_tc(const GemmDesc& d, const double* A, const double* B, double* C, int prec,
             cudaStream_t s, Stats* st, const GaussSrc* gen_b) {
  TATRG_CHECK(prec >= 1 && prec <= 3, TATRG_EINVAL, "gemm_tc: precision must be TF32X3, BF16X3 or BF16X6");
  TATRG_CHECK(tc_available(), TATRG_ENOTIMPL, "gemm_tc: tcgen05 path needs an sm_103 GPU");
  const int64_t M = d.m.total(), N = d.n.total(), K = d.k.total();
  if (M == 0 || N == 0) return;
  if (gen_b) {
    TATRG_CHECK(B == nullptr, TATRG_EINVAL, "gemm_tc: a generated B operand takes no pointer");
    check_extent(A, max_off0(d.m) + max_off0(d.k), sizeof(double), "operand A");
    check_extent(C, max_off1(d.m) + max_off1(d.n), sizeof(double), "result C");
  } else {
    check_gemm(d, A, B, C);
  }
  const GaussSrc no_gen{};
  const int kind = prec == 1 ? 1 : 2;  // kind::tf32 or kind::f16 (bf16)
  const int ns = prec == 3 ? 3 : 2;    // slices per operand
  const int esize = kind == 1 ? 4 : 2;
  const int kelem = KSLICE / esize;
  const int BN = TC_BN;
  // CTA pairs are a candidate when there are many 256-row tiles (the last tile row is then
  // less than half padding); the A panel is padded for them either way
  const bool pair_ok = pairs_enabled() && M >= 1024;
  const int64_t Mp = cdiv(M, pair_ok ? 2 * TC_BM : TC_BM) * (pair_ok ? 2 * TC_BM : TC_BM);
  const int64_t Np = cdiv(N, BN) * BN, Kp = cdiv(K, kelem) * kelem;
  TATRG_CHECK(Mp < (int64_t(1) << 31) && Np < (int64_t(1) << 31), TATRG_EINVAL, "gemm_tc: operand too large");
  // packed operands (ns slices each) in one allocation
  const size_t abytes = size_t(Mp) * Kp * esize, bbytes = size_t(Np) * Kp * esize;
  DevBuf pk(ns * (abytes + bbytes), s);
  uint8_t* base = pk.as<uint8_t>();
  PackDst da{}, db{};
  for (int p = 0; p < ns; ++p) {
    da.p[p] = base + p * abytes;
    db.p[p] = base + ns * abytes + p * bbytes;
  }
  auto pack = [&](const double* src, const DevModes& rm, const DevModes& km, int64_t R, int64_t tiles,
                  const PackDst& dst, int rc, bool gen) {
    const int grid = int(std::min<int64_t>(tiles, int64_t(sm_count()) * 6));
    const int64_t kt = cdiv(Kp, PK_K);
    const GaussSrc& gs = gen ? *gen_b : no_gen;
    if (kind == 1 && gen) pack_kernel<1, 2, true><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    else if (kind == 1) pack_kernel<1, 2, false><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    else if (ns == 2 && gen) pack_kernel<2, 2, true><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    else if (ns == 2) pack_kernel<2, 2, false><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    else if (gen) pack_kernel<2, 3, true><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    else pack_kernel<2, 3, false><<<grid, 256, 0, s>>>(src, rm, km, R, K, Kp, kt, tiles, dst, rc, gs);
    TATRG_CUDA(cudaGetLastError());
  };
  {
    // A: rows = m (stride s0), k (stride s0);  B: rows = n (s0), k (s1)
    DevModes rm = dev(d.m), km = dev(d.k);
    const int rc = (d.m.n > 0 && d.m.s0[d.m.n - 1] == 1 && !(d.k.n > 0 && d.k.s0[d.k.n - 1] == 1)) ? 1 : 0;
    pack(A, rm, km, M, (Mp / PK_R) * cdiv(Kp, PK_K), da, rc, false);
    // a Gram (B is A read the same way) reuses A's panels
    bool same = !gen_b && (A == B) && Np == Mp && d.m.n == d.n.n && d.k.n > 0;
    for (int i = 0; same && i < d.m.n; ++i) same = d.m.ext[i] == d.n.ext[i] && d.m.s0[i] == d.n.s0[i];
    for (int i = 0; same && i < d.k.n; ++i) same = d.k.s0[i] == d.k.s1[i];
    if (same) {
      db = da;
    } else {
      DevModes rn = dev(d.n), kn = dev(d.k);
      for (int i = 0; i < kMaxModes; ++i) kn.s0[i] = kn.s1[i];  // B's k strides
      const int rcb = (d.n.n > 0 && d.n.s0[d.n.n - 1] == 1 && !(d.k.n > 0 && d.k.s1[d.k.n - 1] == 1)) ? 1 : 0;
      pack(gen_b ? nullptr : B, rn, kn, N, (Np / PK_R) * cdiv(Kp, PK_K), db, gen_b ? 0 : rcb, gen_b != nullptr);
    }
  }
  TcMaps maps1{}, maps2{};  // B boxes of a whole tile's columns (single CTAs) or half (clusters)
  for (int p = 0; p < ns; ++p) {
    maps1.a[p] = maps2.a[p] = make_map(da.p[p], Mp, Kp, esize, TC_BM, kind);
    maps1.b[p] = make_map(db.p[p], Np, Kp, esize, BN, kind);
    if (pair_ok) maps2.b[p] = make_map(db.p[p], Np, Kp, esize, BN / 2, kind);
  }
  const int nkb = int(Kp / kelem);
  TcArgs a;
  a.mC = dev(d.m);
  a.nC = dev(d.n);
  a.M = M;
  a.N = N;
  a.nkb = nkb;
  a.alpha = d.alpha;
  a.beta = d.beta;
  {
    // C offset of column n equals n when the N modes chain contiguously in C
    bool contig = d.n.n >= 1 && d.n.s1[d.n.n - 1] == 1;
    for (int i = 0; contig && i + 1 < d.n.n; ++i) contig = d.n.s1[i] == d.n.s1[i + 1] * d.n.ext[i + 1];
    a.n_contig = contig ? 1 : 0;
  }
  a.C = C;
  a.ntiles = int(Np / BN);
  // one launch of configuration (tile form, split): C is rewritten whole (zeroed first when
  // K is split, the CTAs then add their partial sums)
  auto run = [&](int form, int split) {
    const int tile_m = form != 0 ? 2 * TC_BM : TC_BM;
    TcArgs g = a;
    g.mtiles = int(cdiv(M, tile_m));
    const int per = int(cdiv(nkb, split));
    g.split = int(cdiv(nkb, per));
    g.kb_per_split = per;
    g.atomic = g.split > 1 ? 1 : 0;
    if (g.split > 1) {
      scale_c_kernel<<<int(std::min<int64_t>(cdiv(M * N, 256), 4096)), 256, 0, s>>>(C, dev(d.m), dev(d.n), M, N, d.beta);
      TATRG_CUDA(cudaGetLastError());
    }
    const int64_t units = int64_t(g.mtiles) * g.ntiles * g.split;
    TATRG_CHECK(units < (int64_t(1) << 31), TATRG_EINVAL, "gemm_tc: too many work units");
    const TcMaps& mp = form != 0 ? maps2 : maps1;
    if (prec == 1 && form == 1) launch<1, 2, 1>(mp, g, units, s);
    else if (prec == 1 && form == 2) launch<1, 2, 2>(mp, g, units, s);
    else if (prec == 1) launch<1, 2, 0>(mp, g, units, s);
    else if (prec == 2 && form == 1) launch<2, 2, 1>(mp, g, units, s);
    else if (prec == 2 && form == 2) launch<2, 2, 2>(mp, g, units, s);
    else if (prec == 2) launch<2, 2, 0>(mp, g, units, s);
    else if (form == 1) launch<2, 3, 1>(mp, g, units, s);
    else if (form == 2) launch<2, 3, 2>(mp, g, units, s);
    else launch<2, 3, 0>(mp, g, units, s);
    return g.split;
  };
  // the split-K heuristic: enough work units for two per CTA (pair)
  auto heuristic = [&](bool pair) {
    const int64_t tiles = cdiv(M, pair ? 2 * TC_BM : TC_BM) * a.ntiles;
    const int64_t workers = pair ? sm_count() / 2 : sm_count();
    int split = 1;
    if (tiles < 2 * workers && nkb >= 8) split = int(std::min<int64_t>(cdiv(2 * workers, tiles), nkb / 4));
    return std::max(1, std::min(split, 512));
  };
  const TcChoice ch = tuned_choice(prec, M, N, K, a.n_contig, pair_ok, d.beta == 0.0, heuristic, run, s);
  const bool timed = st && st->timing;
  if (timed) TATRG_CUDA(cudaEventRecord(st->next_event(), s));
  const int split = run(ch.form, ch.split);
  if (timed) TATRG_CUDA(cudaEventRecord(st->next_event(), s));
  if (st) {
    st->launches += 3 + (split > 1);
    st->tc_launches += 1;
    st->flops_tc += 2.0 * double(M) * double(N) * double(K);
  }
}

void gemm_oz(const GemmDesc& d, const double* A, const double* B, double* C, cudaStream_t s, Stats* st) {
  TATRG_CHECK(tc_available(), TATRG_ENOTIMPL, "gemm_oz: tcgen05 path needs an sm_103 GPU");
  const int64_t M = d.m.total(), N = d.n.total(), K = d.k.total();
  if (M == 0 || N == 0) return;
  check_gemm(d, A, B, C);
  const int64_t Mp = cdiv(M, TC_BM) * TC_BM, Np = cdiv(N, OZ_BN) * OZ_BN, Kp = cdiv(K, OZ_KELEM) * OZ_KELEM;
  TATRG_CHECK(Mp < (int64_t(1) << 31) && Np < (int64_t(1) << 31), TATRG_EINVAL, "gemm_oz: operand too large");
  // row exponents (all-zero rows keep the 0xC0 bytes) and the digit planes
  DevBuf ex(size_t(Mp + Np) * sizeof(int), s);
  TATRG_CUDA(cudaMemsetAsync(ex.d(), 0xC0, size_t(Mp + Np) * sizeof(int), s));
  int* ea = ex.as<int>();
  int* eb = ea + Mp;
  const size_t abytes = size_t(Mp) * Kp * 2, bbytes = size_t(Np) * Kp * 2;
  DevBuf pk(OZ_NS * (abytes + bbytes), s);
  uint8_t* base = pk.as<uint8_t>();
  void* pa[OZ_NS];
  void* pb[OZ_NS];
  for (int p = 0; p < OZ_NS; ++p) {
    pa[p] = base + p * abytes;
    pb[p] = base + OZ_NS * abytes + p * bbytes;
  }
  const int sms = sm_count();
  auto slice = [&](const double* src, const DevModes& rm, const DevModes& km, int64_t R, int64_t Rp, int* exps,
                   void* const* planes, int rc) {
    const int64_t kt = cdiv(K, PK_K), nt = cdiv(R, PK_R) * kt;
    oz_exp_kernel<<<int(std::min<int64_t>(nt, int64_t(sms) * 6)), 256, 0, s>>>(src, rm, km, R, K, kt, nt, exps, rc);
    TATRG_CUDA(cudaGetLastError());
    const int64_t kt2 = cdiv(Kp, PK_K), nt2 = (Rp / PK_R) * kt2;
    PackDst d1{}, d2{};
    d1.p[0] = planes[0];
    d1.p[1] = planes[1];
    d1.p[2] = planes[2];
    d2.p[0] = planes[3];
    d2.p[1] = planes[4];
    oz_pack_kernel<<<int(std::min<int64_t>(nt2, int64_t(sms) * 6)), 256, 0, s>>>(src, rm, km, R, K, Kp, kt2, nt2,
                                                                                  exps, d1, d2, rc);
    TATRG_CUDA(cudaGetLastError());
  };
  {
    DevModes rm = dev(d.m), km = dev(d.k);
    const int rc = (d.m.n > 0 && d.m.s0[d.m.n - 1] == 1 && !(d.k.n > 0 && d.k.s0[d.k.n - 1] == 1)) ? 1 : 0;
    slice(A, rm, km, M, Mp, ea, pa, rc);
    DevModes rn = dev(d.n), kn = dev(d.k);
    for (int i = 0; i < kMaxModes; ++i) kn.s0[i] = kn.s1[i];  // B's k strides
    const int rcb = (d.n.n > 0 && d.n.s0[d.n.n - 1] == 1 && !(d.k.n > 0 && d.k.s1[d.k.n - 1] == 1)) ? 1 : 0;
    slice(B, rn, kn, N, Np, eb, pb, rcb);
  }
  OzMaps maps;
  for (int p = 0; p < OZ_NS; ++p) {
    maps.a[p] = make_map(pa[p], Mp, Kp, 2, TC_BM, 2, OZ_KS);
    maps.b[p] = make_map(pb[p], Np, Kp, 2, OZ_BN, 2, OZ_KS);
  }
  OzArgs oa;
  TcArgs& g = oa.g;
  g.mC = dev(d.m);
  g.nC = dev(d.n);
  g.M = M;
  g.N = N;
  g.nkb = int(Kp / OZ_KELEM);
  g.alpha = d.alpha;
  g.beta = d.beta;
  g.n_contig = 0;
  g.C = C;
  g.mtiles = int(Mp / TC_BM);
  g.ntiles = int(Np / OZ_BN);
  const int64_t tiles = int64_t(g.mtiles) * g.ntiles;
  int split = 1;
  if (tiles < 2 * sms && g.nkb >= 8) split = int(std::min<int64_t>(cdiv(2 * sms, tiles), g.nkb / 4));
  split = std::max(1, std::min(split, 512));
  g.kb_per_split = int(cdiv(g.nkb, split));
  g.split = int(cdiv(g.nkb, g.kb_per_split));
  g.atomic = g.split > 1 ? 1 : 0;
  oa.ea = ea;
  oa.eb = eb;
  if (g.split > 1) {
    scale_c_kernel<<<int(std::min<int64_t>(cdiv(M * N, 256), 4096)), 256, 0, s>>>(C, dev(d.m), dev(d.n), M, N, d.beta);
    TATRG_CUDA(cudaGetLastError());
  }
  const int64_t units = tiles * g.split;
  TATRG_CHECK(units < (int64_t(1) << 31), TATRG_EINVAL, "gemm_oz: too many work units");
  {
    static std::mutex mu;
    static std::map<int, int> fits;
    int dev_ = 0;
    TATRG_CUDA(cudaGetDevice(&dev_));
    std::lock_guard<std::mutex> l(mu);
    if (!fits.count(dev_)) {
      TATRG_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
      int n = 0;
      TATRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, oz_gemm_kernel, TC_THREADS, OZ_SMEM));
      fits[dev_] = n;
    }
    TATRG_CHECK(fits[dev_] >= 1, TATRG_ECUDA, "gemm_oz: the kernel does not fit on an SM");
  }
  const bool timed = st && st->timing;
  if (timed) TATRG_CUDA(cudaEventRecord(st->next_event(), s));
  oz_gemm_kernel<<<unsigned(std::min<int64_t>(units, sms)), TC_THREADS, OZ_SMEM, s>>>(maps, oa);
  TATRG_CUDA(cudaGetLastError());
  if (timed) TATRG_CUDA(cudaEventRecord(st->next_event(), s));
  if (st) {
    st->launches += 5 + (g.split > 1);
    st->tc_launches += 1;
    st->flops_tc += 2.0 * double(M) * double(N) * double(K);
  }
}

}  // namespace tatrg
