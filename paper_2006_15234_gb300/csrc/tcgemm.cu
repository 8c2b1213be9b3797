// Tensor-core (tcgen05, kind::tf32) GEMM for the dense contractions of the
// implicit products (Sec. IV-A: A X and A^H Y as chains of contractions; with
// the intermediate layouts chosen by the planner each stage is one GEMM whose
// two operands are contiguous along the contracted index).
//
//   C(m, n) (+)= alpha * sum_k opA(A[m][k]) * opB(B[n][k])
//
// A and B are row-major with K contiguous (real, or complex interleaved
// re/im).  Tiles arrive by TMA with the 128-byte swizzle; the accumulators
// live in tensor memory.  A complex product runs as ONE real MMA chain: A's
// interleaved rows (ar, ai) are used as they are, and each complex row b of
// B becomes two real rows,
//   (br, sr*bi) -> Re C,     (s1*bi, s2*br) -> Im C,
// the signs encoding the conjugation of A and/or B.  The accumulator then
// holds (Re, Im) column pairs, i.e. C's interleaved layout, and A is read
// once per k step for both parts.
// SPLIT3 ("3xTF32") splits each operand into a TF32 head (round to nearest)
// and an FP32 tail and accumulates head*head + tail*head + head*tail,
// recovering FP32-level products on TF32 tensor cores.  Plain TF32 products
// round both operands to the nearest TF32 value first (unbiased).
// SPLIT3 operands:
//  * A (128 rows per tile) goes to tensor memory: the worker warps read each
//    raw row from shared memory, split it in registers and store head and
//    tail with tcgen05.st; the MMA takes A from tensor memory (A stages after
//    the two accumulator buffers), so the tensor core reads only B from
//    shared memory;
//  * B is expanded (complex) and split once before the GEMM into a scratch
//    buffer (tc_expand_kernel, "bpre") and TMA delivers MMA-ready head and
//    tail tiles; where B is too large for that (the Grams) the workers expand
//    and split it in shared memory per 16-byte chunk, which commutes with the
//    swizzle up to the row-dependent chunk permutation the rewrite applies.
// The tensor core's FP32 accumulator drops the bits of each addend below the
// running sum's last place (measured: a relative bias of about 1e-8 per
// accumulated K value, growing linearly with K).  SPLIT3 products therefore
// accumulate only CK k blocks at a time in tensor memory (two buffers, so the
// MMAs of one chunk overlap the read-back of the previous one) and the worker
// warps add each chunk into FP32 registers with round-to-nearest.
//
// Roles: warp 0 issues TMA, warp 1 owns tensor memory and issues MMAs from
// one thread, warps 2-9 prepare operands, fold accumulator chunks and run the
// epilogue (tensor memory or registers -> global through an arbitrary
// mixed-radix index map; warp w owns lane quarter w % 4 and column half
// (w - 2) / 4).  An item's epilogue runs after the first k blocks of the next
// item are prepared, so that its MMAs overlap the epilogue.  Every mbarrier
// wait is bounded: on expiry the kernel raises a status bit, lets its own TMA
// copies and MMAs drain (again bounded), frees its tensor memory and returns.
// Decisions to leave a loop are taken by all worker threads together (a
// barrier reduction; a warp vote inside k loops that reach no named
// barrier), so no worker is left at a named barrier.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tcgemm.h"

namespace peps {

namespace {

constexpr int BM = 128;
constexpr int BKF = 32;              // floats of K per stage (one 128-byte swizzle row)
constexpr int NWORK = 256;           // worker threads (warps 2..9)
constexpr int NTHREADS = 64 + NWORK;
constexpr uint32_t kWaitLimit = 1u << 24;   // polls of a teardown drain (~1 s)
constexpr uint64_t kWaitNs = 2000000000ull;  // a pipeline wait gives up after 2 s
constexpr uint32_t kSuspendNs = 1000;        // suspend-time hint of one pipeline poll
constexpr int CK = 2;                // k blocks per tensor-memory accumulation chunk (SPLIT3)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// One poll that may suspend the thread (up to the hint) until the phase completes.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait (limit_ns of global time, checked every 16 polls or, for limits
// under 64 us, after every poll; and at most 2^26 polls); false (and the abort
// flag raised) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  const uint32_t every = limit_ns < 65536 ? 0u : 15u;
  for (uint32_t i = 1; i < (1u << 26); ++i) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((i & every) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns) break;
    }
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (tcgen05 descriptor version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulate, TF32 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// A from tensor memory: row i of the 128 x 8 operand in lane i, one 32-bit
// column per K element, starting at column address a_tmem
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// this warp's 32 lanes, 8 consecutive columns from taddr
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 columns without the wait (the caller waits once for several loads)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// nearest TF32 value (ties away from zero): exact input to the tensor core
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ int64_t map_index(const DigitMap &m, int64_t i64) {
  uint32_t i = (uint32_t)i64;      // row / column indices are below 2^31
  int64_t off = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (d >= m.n) break;
    // q = i / radix: t + i < 2^32 since t <= i < 2^31
    const uint32_t q = (__umulhi(i, m.mul[d]) + i) >> m.shr[d];
    off += (int64_t)(i - q * (uint32_t)m.radix[d]) * m.stride[d];
    i = q;
  }
  return off;
}

// AND over the worker threads (barrier 3); every worker must call it.
__device__ __forceinline__ bool workers_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.and.pred q, 3, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void workers_sync(int id) {
  asm volatile("barrier.cta.sync %0, 256;" ::"r"(id) : "memory");
}

__device__ __forceinline__ float4 head4(float4 v) {
  return make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

template <int NMMA, bool CPLX, bool SPLIT3, bool FOLD_, bool BPRE_> struct Layout {
  static constexpr int BNR = CPLX ? NMMA / 2 : NMMA;   // output columns (complex or real) per tile
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = NMMA * 128;           // MMA-ready B tile
  static constexpr int RAW_BYTES = BNR * 128;          // B tile as TMA lands it
  // SPLIT3: A's head and tail go to tensor memory (ATMEM); only the raw A
  // tile sits in shared memory.  Otherwise A is rounded in place.
  static constexpr bool ATMEM = SPLIT3;
  // B arrives as MMA-ready head and tail tiles (expanded and split beforehand)
  static constexpr bool BPRE = SPLIT3 && BPRE_;
  static constexpr int NB = SPLIT3 ? 2 : 1;            // B head, B tail
  // complex: the raw B tile lands in the tail tile (read out before the tail
  // is written) or, without SPLIT3, in a buffer of its own
  static constexpr bool RAW_SEP = CPLX && !SPLIT3;
  static constexpr int STAGE = A_BYTES + NB * B_BYTES + (RAW_SEP ? RAW_BYTES : 0);
  static constexpr int STAGES = (200 * 1024) / STAGE >= 4 ? 4 : (200 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static constexpr bool FOLD = SPLIT3 && FOLD_;          // chunked accumulation (long K)
  static constexpr int ACC_COLS = NMMA;                // one accumulator set
  static constexpr int HALF = NMMA / 2;                // columns per epilogue thread
  // tensor-memory A stages after the two accumulator buffers: 32 head and 32
  // tail columns (one 32-float k block of 128 rows) each
  static constexpr int A_COLS = 64;
  static constexpr int SA_FIT = ATMEM ? (512 - 2 * NMMA) / A_COLS : 0;
  static constexpr int SA = SA_FIT > 4 ? 4 : SA_FIT;
  static constexpr int A_COL0 = 2 * NMMA;
  static constexpr int TMEM_NEED = 2 * NMMA + SA * A_COLS;
  static constexpr int TMEM_COLS = TMEM_NEED <= 64 ? 64 : TMEM_NEED <= 128 ? 128 : TMEM_NEED <= 256 ? 256 : 512;
  static_assert(STAGES >= 2, "two pipeline stages at least");
  static_assert(!ATMEM || SA >= 2, "two tensor-memory A stages at least");
  static_assert(TMEM_NEED <= 512, "tensor memory holds 512 columns");
  static_assert(NMMA % 16 == 0 && NMMA >= 16 && NMMA <= 256, "tcgen05 N for M = 128");
};

// 10 warps: each SM sub-partition (16K registers) holds 3 of them, so at most
// 168 registers per thread
template <int NMMA, bool CPLX, bool SPLIT3, bool FOLD_, bool BPRE_>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_kernel(const __grid_constant__ TcDesc g) {
  using L = Layout<NMMA, CPLX, SPLIT3, FOLD_, BPRE_>;
  constexpr int STAGES = L::STAGES;
  constexpr bool FOLD = L::FOLD;
  constexpr int HALF = L::HALF;
  constexpr int SAD = L::SA > 0 ? L::SA : 1;   // tensor-memory A stages (ATMEM)
  __shared__ __align__(8) uint64_t full_bar[STAGES], ready_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t a_empty[L::SA > 0 ? L::SA : 1];   // tensor-memory A stage free again
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int64_t col_off[L::BNR];
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // persistent: this CTA takes work items blockIdx.x, + gridDim.x, ...; an
  // item is one output tile (and one K chunk when K is split)
  const int ntile = g.tiles_m * g.tiles_n;
  const int total = ntile * (g.ksplit > 1 ? g.ksplit : 1);
  const int nkb_all = (g.Kr + BKF - 1) / BKF;
  struct Item { int m0, n0, kb0, nkb; };
  auto item = [&](int w) {
    const int tile = w % ntile, kc = w / ntile;
    Item it;
    // N tiles of one M tile are neighbours: the CTAs sharing an A tile run together (L2 reuse)
    it.m0 = (tile / g.tiles_n) * BM;
    it.n0 = (tile % g.tiles_n) * L::BNR;
    it.kb0 = g.ksplit > 1 ? kc * g.kb_per_split : 0;
    it.nkb = g.ksplit > 1 ? min(g.kb_per_split, nkb_all - it.kb0) : nkb_all;
    return it;
  };
  // accumulation chunks of an item: CK k blocks (SPLIT3) or the whole item
  auto nchunks_of = [&](int nkb) { return FOLD ? (nkb + CK - 1) / CK : 1; };

  auto a_tile = [&](int s) { return smem + s * L::STAGE; };
  auto b_tile = [&](int s, int which) { return smem + s * L::STAGE + L::A_BYTES + which * L::B_BYTES; };
  auto raw_tile = [&](int s) {
    if constexpr (!CPLX) return b_tile(s, 0);
    else if constexpr (L::RAW_SEP) return smem + s * L::STAGE + L::A_BYTES + L::NB * L::B_BYTES;
    else return b_tile(s, 1);
  };

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&ready_bar[s], NWORK);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], NWORK);
    }
    for (int a = 0; a < L::SA; ++a) mbar_init(&a_empty[a], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)L::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint64_t wns = g.wait_ns ? g.wait_ns : kWaitNs;

  int issued = 0;          // producer: k blocks whose TMA was issued (over all items)
  bool mma_any = false;    // MMA thread: at least one MMA issued

  // workers: lane quarter q (tensor-memory lanes 32q..32q+31), column half h
  const int q = warp & 3, h = warp >= 2 ? (warp - 2) >> 2 : 0;
  int folded = 0;          // workers: chunks read back so far (over all items)
  float facc[FOLD ? HALF : 1];
  // add chunk `folded` (whose completion was awaited) into facc
  auto fold_body = [&]() {
    const int b = folded & 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * L::ACC_COLS + h * HALF);
#pragma unroll
    for (int c0 = 0; c0 < (FOLD ? HALF : 0); c0 += 16) {
      float v[16];
      tmem_ld16(base + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) facc[c0 + i] += v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(&acc_empty[b]);
    ++folded;
  };
  auto acc_wait = [&]() -> bool {
    return !abort_flag && mbar_wait(&acc_full[folded & 1], (folded >> 1) & 1, &abort_flag, wns);
  };

  if (warp == 0) {
    if (lane == 0) {
      int gk = 0;
      for (int w = blockIdx.x; w < total && !abort_flag; w += gridDim.x) {
        const Item it = item(w);
        for (int kb = 0; kb < it.nkb && !abort_flag; ++kb, ++gk) {
          const int s = gk % STAGES;
          if (gk >= STAGES && !mbar_wait(&empty_bar[s], ((gk / STAGES) - 1) & 1, &abort_flag, wns)) break;
          const int x = (it.kb0 + kb) * BKF;
          if constexpr (L::BPRE) {
            const int nr0 = CPLX ? 2 * it.n0 : it.n0;      // first MMA row of B (Re / Im rows when complex)
            mbar_expect_tx(&full_bar[s], (uint32_t)(L::A_BYTES + 2 * L::B_BYTES));
            tma_load_2d(a_tile(s), &g.ta, x, it.m0, &full_bar[s]);
            tma_load_2d(b_tile(s, 0), &g.tb, x, nr0, &full_bar[s]);
            tma_load_2d(b_tile(s, 1), &g.tb2, x, nr0, &full_bar[s]);
          } else {
            mbar_expect_tx(&full_bar[s], (uint32_t)(L::A_BYTES + L::RAW_BYTES));
            tma_load_2d(a_tile(s), &g.ta, x, it.m0, &full_bar[s]);
            tma_load_2d(raw_tile(s), &g.tb, x, it.n0, &full_bar[s]);
          }
          issued = gk + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(NMMA);
      int gk = 0, gch = 0;
      bool alive = true;
      for (int w = blockIdx.x; w < total && alive; w += gridDim.x) {
        const Item it = item(w);
        for (int kb = 0; kb < it.nkb; ++kb, ++gk) {
          const int s = gk % STAGES;
          const bool first = FOLD ? (kb % CK == 0) : (kb == 0);
          const bool last = FOLD ? (kb % CK == CK - 1 || kb == it.nkb - 1) : (kb == it.nkb - 1);
          const int buf = gch & 1;
          // a buffer is reused once the workers have read back the chunk two before
          if (first && gch >= 2 && !mbar_wait(&acc_empty[buf], ((gch >> 1) - 1) & 1, &abort_flag, wns)) { alive = false; break; }
          if (!mbar_wait(&ready_bar[s], (gk / STAGES) & 1, &abort_flag, wns)) { alive = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t tacc = tmem + (uint32_t)(buf * L::ACC_COLS);
          const uint32_t b0 = smem_u32(b_tile(s, 0));
          if constexpr (L::ATMEM) {
            // A head and tail from tensor memory stage gk % SA; B head and tail from shared memory
            const uint32_t ah = tmem + (uint32_t)(L::A_COL0 + (gk % SAD) * L::A_COLS), at = ah + 32;
            const uint32_t bt = smem_u32(b_tile(s, 1));
#pragma unroll
            for (int kk = 0; kk < BKF / 8; ++kk) {
              const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
              const uint32_t off = kk * 32;
              mma_tf32_ta(tacc, ah + kk * 8, sw128_desc(b0 + off), idesc, acc);
              mma_tf32_ta(tacc, at + kk * 8, sw128_desc(b0 + off), idesc, 1u);
              mma_tf32_ta(tacc, ah + kk * 8, sw128_desc(bt + off), idesc, 1u);
            }
          } else {
            const uint32_t a0 = smem_u32(a_tile(s));
#pragma unroll
            for (int kk = 0; kk < BKF / 8; ++kk) {
              const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
              const uint32_t off = kk * 32;
              mma_tf32(tacc, sw128_desc(a0 + off), sw128_desc(b0 + off), idesc, acc);
            }
          }
          mma_any = true;
          mma_commit(&empty_bar[s]);
          if (L::ATMEM) mma_commit(&a_empty[gk % SAD]);
          if (last) { mma_commit(&acc_full[buf]); ++gch; }
        }
      }
      if (mma_any) mma_commit(&done_bar);
    }
  } else {
    // ---- workers: operand rewrites, chunk read-back, epilogue ----
    const int t = threadIdx.x - 64;
    float sr = 1.f, s1 = 1.f, s2 = 1.f;
    if (CPLX) {
      if (!g.conjA && !g.conjB) { sr = -1.f; s1 = 1.f; s2 = 1.f; }
      else if (g.conjA && !g.conjB) { sr = 1.f; s1 = 1.f; s2 = -1.f; }
      else if (!g.conjA && g.conjB) { sr = 1.f; s1 = -1.f; s2 = 1.f; }
      else { sr = -1.f; s1 = -1.f; s2 = -1.f; }
    }
    double alpha = g.alpha;
    if (g.alpha_dev) alpha *= *g.alpha_dev;
    const float alpha_f = (float)alpha;       // single-precision outputs: no FP64 multiplies per element
    bool alive = workers_all(!abort_flag);
    int gk = 0, items = 0;
    // one k block: wait for its tiles (and, at a chunk boundary, read back the
    // chunk before the last one), then prepare its operands for the MMA
    auto kblock = [&](int kb) -> bool {
      const int s = gk % STAGES;
      bool ok = mbar_wait(&full_bar[s], (gk / STAGES) & 1, &abort_flag, wns);
      const bool fold_now = FOLD && kb % CK == 0 && kb >= 2 * CK;
      if (fold_now) ok = ok && acc_wait();
      // the tensor-memory A stage of this k block was last read by k block gk - SA
      if (L::ATMEM && gk >= SAD)
        ok = ok && mbar_wait(&a_empty[gk % SAD], ((gk / SAD) - 1) & 1, &abort_flag, wns);
      // a warp-wide decision suffices when no named barrier follows in the k loop (BPRE)
      if (!(L::BPRE ? __all_sync(0xffffffffu, ok) : workers_all(ok))) return false;
      if (fold_now) fold_body();
      {
        if constexpr (L::ATMEM) {
          // A row r = 32q + lane, floats 16h .. 16h + 15 of the k block (swizzled
          // 16-byte chunks 4h .. 4h + 3): head and tail into tensor memory
          const int r = q * 32 + lane;
          const unsigned char *arow = a_tile(s) + r * 128;
          const uint32_t tcol = tmem + ((uint32_t)(q * 32) << 16) +
                                (uint32_t)(L::A_COL0 + (gk % SAD) * L::A_COLS + h * 16);
#pragma unroll
          for (int hv = 0; hv < 2; ++hv) {
            const int c0 = 4 * h + 2 * hv;
            const float4 x0 = *(const float4 *)(arow + ((c0 ^ (r & 7)) << 4));
            const float4 x1 = *(const float4 *)(arow + (((c0 + 1) ^ (r & 7)) << 4));
            const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            float hd[8], tl[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              hd[i] = tf32_head(xv[i]);
              tl[i] = xv[i] - hd[i];
            }
            tmem_st8(tcol + hv * 8, hd);
            tmem_st8(tcol + 32 + hv * 8, tl);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        } else {
          // A: nearest TF32 in place
          float4 *A0 = (float4 *)a_tile(s);
#pragma unroll
          for (int c = t; c < L::A_BYTES / 16; c += NWORK) A0[c] = head4(A0[c]);
        }
        if constexpr (L::BPRE) {
        } else if constexpr (CPLX) {
          // B: complex row n -> real rows 2n (Re) and 2n+1 (Im), chunk by chunk
          constexpr int RAWC = L::RAW_BYTES / 16;
          constexpr int PER = (RAWC + NWORK - 1) / NWORK;
          const unsigned char *raw = raw_tile(s);
          unsigned char *BH = b_tile(s, 0);
          unsigned char *BT = b_tile(s, 1);
          float4 v[PER];
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int i = t + u * NWORK;
            if (i < RAWC) v[u] = ((const float4 *)raw)[i];
          }
          if (!L::RAW_SEP) workers_sync(2);    // raw tile is the tail tile: read out before writing
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int i = t + u * NWORK;
            if (i >= RAWC) continue;
            const int n = i >> 3, c = (i & 7) ^ (n & 7);           // logical chunk of row n
            const float4 x = v[u];
            const float4 re = make_float4(x.x, sr * x.y, x.z, sr * x.w);
            const float4 im = make_float4(s1 * x.y, s2 * x.x, s1 * x.w, s2 * x.z);
            const int r0 = 2 * n, r1 = 2 * n + 1;
            const float4 reh = head4(re), imh = head4(im);
            *(float4 *)(BH + r0 * 128 + ((c ^ (r0 & 7)) << 4)) = reh;
            *(float4 *)(BH + r1 * 128 + ((c ^ (r1 & 7)) << 4)) = imh;
            if (SPLIT3) {
              *(float4 *)(BT + r0 * 128 + ((c ^ (r0 & 7)) << 4)) = sub4(re, reh);
              *(float4 *)(BT + r1 * 128 + ((c ^ (r1 & 7)) << 4)) = sub4(im, imh);
            }
          }
        } else {
          float4 *B0 = (float4 *)b_tile(s, 0);
          float4 *B1 = (float4 *)b_tile(s, 1);
#pragma unroll
          for (int c = t; c < L::B_BYTES / 16; c += NWORK) {
            const float4 v = B0[c];
            const float4 hd = head4(v);
            if (SPLIT3) B1[c] = sub4(v, hd);
            B0[c] = hd;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (L::ATMEM) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      mbar_arrive(&ready_bar[s]);
      ++gk;
      return true;
    };
    // final read-back and epilogue of an item whose k blocks were all prepared
    auto finish = [&](const Item &it, int chunk_end) -> bool {
      if (FOLD) {
        bool live = true;
        while (live && folded < chunk_end) {
          live = workers_all(acc_wait());
          if (live) fold_body();
        }
        if (!live) return false;
      } else if (!workers_all(acc_wait())) {
        return false;
      }
      // ---- epilogue of this item ----
      workers_sync(1);                        // previous item's column offsets no longer read
      for (int c = t; c < L::BNR; c += NWORK) col_off[c] = it.n0 + c < g.N ? map_index(g.mn, it.n0 + c) : 0;
      workers_sync(1);
      const int m = it.m0 + q * 32 + lane;
      const int64_t row_off = m < g.M ? map_index(g.mm, m) : 0;
      // local accumulator column j of this half -> output column
      auto store = [&](int j, float v0, float v1) {
        const int cl = CPLX ? (h * HALF + j) >> 1 : h * HALF + j;
        if (it.n0 + cl >= g.N) return;
        const int64_t off = row_off + col_off[cl];
        if (g.atomic64) {
          if (CPLX) {
            double2 *C = (double2 *)g.C + off;
            atomicAdd(&C->x, alpha * (double)v0);
            atomicAdd(&C->y, (g.conjC ? -alpha : alpha) * (double)v1);
          } else {
            atomicAdd((double *)g.C + off, alpha * (double)v0);
          }
        } else if (CPLX) {
          float2 v = make_float2(alpha_f * v0, alpha_f * v1);
          if (g.conjC) v.y = -v.y;
          float2 *C = (float2 *)g.C + off;
          if (g.accumulate) { const float2 o = *C; v.x += o.x; v.y += o.y; }
          *C = v;
        } else {
          float v = alpha_f * v0;
          float *C = (float *)g.C + off;
          if (g.accumulate) v += *C;
          *C = v;
        }
      };
      constexpr int STEP = CPLX ? 2 : 1;
      if (FOLD) {
        if (m < g.M) {
#pragma unroll
          for (int j = 0; j < HALF; j += STEP) store(j, facc[j], CPLX ? facc[(j + 1) % HALF] : 0.f);
        }
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((folded & 1) * L::ACC_COLS + h * HALF);
        // up to 96 columns per round of loads (one wait per round)
        constexpr int GRP = HALF > 96 ? 64 : HALF;
#pragma unroll 1
        for (int g0 = 0; g0 < HALF; g0 += GRP) {
          float v[GRP];
#pragma unroll
          for (int c0 = 0; c0 < GRP; c0 += 16) tmem_ld16_nowait(base + g0 + c0, &v[c0]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (m < g.M) {
#pragma unroll
            for (int i = 0; i < GRP; i += STEP) store(g0 + i, v[i], CPLX ? v[i + 1] : 0.f);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&acc_empty[folded & 1]);
        ++folded;
      }
      return true;
    };
    // The epilogue of item i runs after the first k blocks of item i + 1 are
    // prepared (lag: one chunk when folding, else the tensor-memory A stages),
    // so that the MMAs of item i + 1 overlap it.  Every worker reaches the
    // barrier reductions between the two k loops and at the item's end the
    // same number of times, whichever k block it left at.
    bool pend = false;
    Item pit{};
    int pend_end = 0, chunk_next = 0;
    for (int w = blockIdx.x; w < total && alive; w += gridDim.x, ++items) {
      const Item it = item(w);
      const int chunk_end = chunk_next + nchunks_of(it.nkb);
      chunk_next = chunk_end;
      const int lag = min(it.nkb, FOLD ? CK : SAD);
      bool ok = true;
      for (int kb = 0; kb < lag && ok; ++kb) ok = kblock(kb);
      if (!workers_all(ok)) { alive = false; break; }
      if (pend && !finish(pit, pend_end)) { alive = false; break; }
      pend = false;
#pragma unroll
      for (int i = 0; i < (FOLD ? HALF : 1); ++i) facc[i] = 0.f;
      for (int kb = lag; kb < it.nkb && ok; ++kb) ok = kblock(kb);
      if (!workers_all(ok)) { alive = false; break; }
      pend = true;
      pit = it;
      pend_end = chunk_end;
    }
    if (alive && pend) alive = finish(pit, pend_end);
    // the MMA thread's final completion signal lands before the CTA may exit
    if (alive && items > 0) mbar_wait(&done_bar, 0, &abort_flag, wns);
  }

  // ---- teardown: drain own copies and MMAs if a wait gave up ----
  __syncthreads();
  if (abort_flag) {
    if (threadIdx.x == 0 && g.status) atomicOr(g.status, STATUS_TIMEOUT);
    if (warp == 0 && lane == 0)
      for (int k = issued > STAGES ? issued - STAGES : 0; k < issued; ++k)
        for (uint32_t i = 0; i < kWaitLimit && !mbar_test(&full_bar[k % STAGES], (k / STAGES) & 1); ++i) {
        }
    if (warp == 1 && lane == 0 && mma_any)
      for (uint32_t i = 0; i < kWaitLimit && !mbar_test(&done_bar, 0); ++i) {
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)L::TMEM_COLS));
  }
}

template <int NMMA, bool CPLX, bool SPLIT3, bool FOLD, bool BPRE>
void launch_tc(const TcDesc &d, cudaStream_t s) {
  using L = Layout<NMMA, CPLX, SPLIT3, FOLD, BPRE>;
  auto kern = tc_gemm_kernel<NMMA, CPLX, SPLIT3, FOLD, BPRE>;
  static int resident = 0;     // CTAs of this instantiation that fit the whole GPU at once
  if (!resident) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NTHREADS, L::SMEM);
    resident = std::max(1, sms) * std::max(1, per);
  }
  const int64_t items = (int64_t)d.tiles_m * d.tiles_n * (d.ksplit > 1 ? d.ksplit : 1);
  const unsigned blocks = (unsigned)std::min<int64_t>(items, resident);
  if (blocks) kern<<<blocks, NTHREADS, L::SMEM, s>>>(d);
}

template <int NMMA, bool CPLX, bool FOLD> void launch_split3(const TcDesc &d, cudaStream_t s) {
  if (d.bpre) launch_tc<NMMA, CPLX, true, FOLD, true>(d, s);
  else launch_tc<NMMA, CPLX, true, FOLD, false>(d, s);
}

template <int NMMA> void launch_n(const TcDesc &d, cudaStream_t s) {
  // SPLIT3 items longer than two chunks fold; shorter ones keep one tensor-memory accumulation
  const bool fold = tc_folds(d.split3 != 0, d.Kr, d.ksplit > 1 ? d.kb_per_split : 0);
  if constexpr (NMMA > 192) {
    if (d.cplx) launch_tc<NMMA, true, false, false, false>(d, s);
    else launch_tc<NMMA, false, false, false, false>(d, s);
  } else if (d.cplx) {
    if (!d.split3) launch_tc<NMMA, true, false, false, false>(d, s);
    else if (fold) launch_split3<NMMA, true, true>(d, s);
    else launch_split3<NMMA, true, false>(d, s);
  } else {
    if (!d.split3) launch_tc<NMMA, false, false, false, false>(d, s);
    else if (fold) launch_split3<NMMA, false, true>(d, s);
    else launch_split3<NMMA, false, false>(d, s);
  }
}

// B -> Bx (bpre): each 16-byte chunk of B (two complex values, or four real
// ones) gives its head and tail chunks; a complex row n becomes the real rows
// 2n = (br, sr*bi) and 2n+1 = (s1*bi, s2*br), the signs encoding the
// conjugation of A and/or B as in the in-kernel expansion.
__global__ void tc_expand_kernel(const float4 *__restrict__ B, float4 *__restrict__ Bx, int64_t n, int64_t kr4,
                                 int cplx, float sr, float s1, float s2) {
  const int64_t total = n * kr4;
  const int64_t nr = cplx ? 2 * n : n;       // MMA rows of one part (head or tail)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / kr4, c = i - row * kr4;
    const float4 x = B[i];
    if (cplx) {
      const float4 re = make_float4(x.x, sr * x.y, x.z, sr * x.w);
      const float4 im = make_float4(s1 * x.y, s2 * x.x, s1 * x.w, s2 * x.z);
      const float4 reh = head4(re), imh = head4(im);
      Bx[(2 * row) * kr4 + c] = reh;
      Bx[(2 * row + 1) * kr4 + c] = imh;
      Bx[(nr + 2 * row) * kr4 + c] = sub4(re, reh);
      Bx[(nr + 2 * row + 1) * kr4 + c] = sub4(im, imh);
    } else {
      const float4 hd = head4(x);
      Bx[row * kr4 + c] = hd;
      Bx[(nr + row) * kr4 + c] = sub4(x, hd);
    }
  }
}

void launch_expand(const TcDesc &d, cudaStream_t s) {
  float sr = 1.f, s1 = 1.f, s2 = 1.f;
  if (d.cplx) {
    if (!d.conjA && !d.conjB) { sr = -1.f; s1 = 1.f; s2 = 1.f; }
    else if (d.conjA && !d.conjB) { sr = 1.f; s1 = 1.f; s2 = -1.f; }
    else if (!d.conjA && d.conjB) { sr = 1.f; s1 = -1.f; s2 = 1.f; }
    else { sr = -1.f; s1 = -1.f; s2 = -1.f; }
  }
  const int64_t kr4 = d.Kr / 4, total = (int64_t)d.N * kr4;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (blocks > 0)
    tc_expand_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float4 *)d.Braw, (float4 *)d.Bx, d.N, kr4, d.cplx,
                                                       sr, s1, s2);
}

}  // namespace

bool tc_folds(bool split3, int64_t kr, int kb_per_split) {
  const int64_t nkb = kb_per_split > 0 ? kb_per_split : (kr + BKF - 1) / BKF;
  return split3 && nkb > 2 * CK;
}

int tc_pick_nmma(int N, bool cplx, bool split3) {
  // fewest padded columns, a tile's fixed cost (its A split) counted as 32
  // columns; SPLIT3 kernels hold two accumulator buffers and the A stages in
  // tensor memory (and folding ones half a tile row in registers): at most 192
  static const int cand[4] = {64, 128, 192, 256};
  int best = 64;
  int64_t best_cost = -1;
  for (int nm : cand) {
    if (split3 && nm > 192) continue;
    const int64_t bnr = cplx ? nm / 2 : nm;
    const int64_t tiles = (N + bnr - 1) / bnr;
    const int64_t cost = tiles * (bnr + 32);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = nm; }
  }
  return best;
}

// multiply-shift constants of the index maps' radices
static void fill_div(DigitMap &m) {
  for (int d = 0; d < 4; ++d) div_magic(m.radix[d] > 0 ? (uint64_t)m.radix[d] : 0, &m.mul[d], &m.shr[d]);
}

void launch_tc_gemm(const TcDesc &desc, int nmma, cudaStream_t s) {
  TcDesc d = desc;
  fill_div(d.mm);
  fill_div(d.mn);
  if (d.bpre) {
    if (!d.split3 || nmma > 192) return;   // never planned
    launch_expand(d, s);
  }
  switch (nmma) {
    case 64: launch_n<64>(d, s); break;
    case 128: launch_n<128>(d, s); break;
    case 192: launch_n<192>(d, s); break;
    default:
      if (d.split3) return;   // never planned: tc_pick_nmma caps SPLIT3 at 192
      launch_n<256>(d, s);
      break;
  }
}

}  // namespace peps
