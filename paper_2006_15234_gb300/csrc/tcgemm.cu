// Tensor-core (tcgen05, kind::tf32) GEMM for the dense contractions of the
// implicit products (Sec. IV-A: A X and A^H Y as chains of contractions; with
// the intermediate layouts chosen by the planner each stage is one GEMM whose
// two operands are contiguous along the contracted index).
//
//   C(m, n) (+)= alpha * sum_k opA(A[m][k]) * opB(B[n][k])
//
// A and B are row-major with K contiguous (real, or complex interleaved
// re/im).  Tiles arrive by TMA with the 128-byte swizzle; the accumulators
// live in tensor memory.  Complex products run as real MMAs on a rewritten A
// tile: with b = (br, bi) interleaved along K,
//   Re C = sum [ar, sr*ai] . [br, bi],   Im C = sum [s1*ai, s2*ar] . [br, bi]
// where the signs encode the conjugation of A and/or B; both rewrites act
// inside each 16-byte chunk, so they commute with the TMA swizzle and four
// worker warps apply them in shared memory between the TMA and the MMAs.
// SPLIT3 ("3xTF32") splits each operand into a TF32 head and an FP32 tail
// and accumulates head*head + tail*head + head*tail, recovering FP32-level
// products on TF32 tensor cores.  Plain TF32 products round both operands to
// the nearest TF32 value first (unbiased, half the error of truncation).
// The tensor core's FP32 accumulator drops the bits of each addend below the
// running sum's last place (measured: a relative bias of about 1e-8 per
// accumulated K value, growing linearly with K).  SPLIT3 products therefore
// accumulate only CK k blocks at a time in tensor memory (two buffers, so the
// MMAs of one chunk overlap the read-back of the previous one) and the worker
// warps add each chunk into FP32 registers with round-to-nearest.
//
// Roles: warp 0 issues TMA, warp 1 owns tensor memory and issues MMAs from
// one thread, warps 2-5 rewrite operand tiles and run the epilogue (tensor
// memory -> registers -> global through an arbitrary mixed-radix index map).
// Every mbarrier wait is bounded: on expiry the kernel raises a status bit,
// lets its own TMA copies and MMAs drain (again bounded), frees its tensor
// memory and returns.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgemm.h"

namespace peps {

namespace {

constexpr int BM = 128;
constexpr int BKF = 32;              // floats of K per stage (one 128-byte swizzle row)
constexpr int NTHREADS = 192;
constexpr uint32_t kWaitLimit = 1u << 24;   // polls before a wait gives up (~1 s)
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
// Bounded wait; false (and the abort flag raised) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 1023) == 1023 && *abort_flag) return false;
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

// nearest TF32 value (ties away from zero): exact input to the tensor core
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float4 round4(float4 v) {
  return make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
}

__device__ __forceinline__ int64_t map_index(const DigitMap &m, int64_t i) {
  int64_t off = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (d >= m.n) break;
    const int64_t r = m.radix[d];
    off += (i % r) * m.stride[d];
    i /= r;
  }
  return off;
}

template <int BN, bool CPLX, bool SPLIT3> struct Layout {
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int NA = (CPLX ? 2 : 1) * (SPLIT3 ? 2 : 1);   // A_re, A_im, A_re_s, A_im_s
  static constexpr int NB = SPLIT3 ? 2 : 1;                      // B (head), B tail
  static constexpr int STAGE = NA * A_BYTES + NB * B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE >= 4 ? 4 : ((200 * 1024) / STAGE >= 2 ? (200 * 1024) / STAGE : 1);
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static constexpr int ACC_COLS = CPLX ? 2 * BN : (BN < 32 ? 32 : BN);   // one accumulator set
  static constexpr bool FOLD = SPLIT3;                                     // chunked accumulation
  static constexpr int TMEM_COLS = FOLD ? 2 * ACC_COLS : ACC_COLS;
  static_assert(!FOLD || ACC_COLS <= 128, "register accumulators hold at most 128 columns");
};

template <int BN, bool CPLX, bool SPLIT3>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_kernel(const __grid_constant__ TcDesc g) {
  using L = Layout<BN, CPLX, SPLIT3>;
  constexpr int STAGES = L::STAGES;
  constexpr bool FOLD = L::FOLD;
  __shared__ __align__(8) uint64_t full_bar[STAGES], ready_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int64_t col_off[BN];
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = g.tiles_m * g.tiles_n;
  const int tile = blockIdx.x % ntile, kc = blockIdx.x / ntile;
  const int tm = tile % g.tiles_m, tn = tile / g.tiles_m;
  const int m0 = tm * BM, n0 = tn * BN;
  const int nkb_all = (g.Kr + BKF - 1) / BKF;
  const int kb0 = g.ksplit > 1 ? kc * g.kb_per_split : 0;
  const int nkb = g.ksplit > 1 ? min(g.kb_per_split, nkb_all - kb0) : nkb_all;

  auto a_tile = [&](int s, int which) { return smem + s * L::STAGE + which * L::A_BYTES; };
  auto b_tile = [&](int s, int which) { return smem + s * L::STAGE + L::NA * L::A_BYTES + which * L::B_BYTES; };

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&ready_bar[s], 128);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
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

  int issued = 0;          // producer: k blocks whose TMA was issued
  bool mma_any = false;    // MMA thread: at least one MMA issued

  // SPLIT3 workers: per-row FP32 sums of the chunks read back from tensor memory
  const int q = warp & 3;  // tensor-memory lane quarter a worker warp may access
  const int nchunks = (nkb + CK - 1) / CK;
  int folded = 0;
  float facc[FOLD ? L::ACC_COLS : 1];
#pragma unroll
  for (int i = 0; i < (FOLD ? L::ACC_COLS : 1); ++i) facc[i] = 0.f;
  auto fold = [&]() -> bool {       // add chunk `folded` into facc (warp-collective)
    const int b = folded & 1;
    bool ok = !abort_flag && mbar_wait(&acc_full[b], (folded >> 1) & 1, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * L::ACC_COLS);
#pragma unroll
    for (int c0 = 0; c0 < (FOLD ? L::ACC_COLS : 0); c0 += 16) {
      float v[16];
      tmem_ld16(base + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) facc[c0 + i] += v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(&acc_empty[b]);
    ++folded;
    return true;
  };

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb && !abort_flag; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty_bar[s], ((kb / STAGES) - 1) & 1, &abort_flag)) break;
        mbar_expect_tx(&full_bar[s], (uint32_t)(L::A_BYTES + L::B_BYTES));
        tma_load_2d(a_tile(s, 0), &g.ta, (kb0 + kb) * BKF, m0, &full_bar[s]);
        tma_load_2d(b_tile(s, 0), &g.tb, (kb0 + kb) * BKF, n0, &full_bar[s]);
        issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(BN);
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const int chunk = kb / CK, buf = FOLD ? (chunk & 1) : 0;
        const bool first = FOLD ? (kb % CK == 0) : (kb == 0);
        // a buffer is reused once the workers have read back the chunk two before
        if (FOLD && first && chunk >= 2 && !mbar_wait(&acc_empty[buf], ((chunk >> 1) - 1) & 1, &abort_flag)) break;
        if (!mbar_wait(&ready_bar[s], (kb / STAGES) & 1, &abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t t_re = tmem + (uint32_t)(buf * L::ACC_COLS), t_im = t_re + BN;
        const uint32_t a0 = smem_u32(a_tile(s, 0)), a1 = smem_u32(a_tile(s, 1));
        const uint32_t b0 = smem_u32(b_tile(s, 0));
#pragma unroll
        for (int kk = 0; kk < BKF / 8; ++kk) {
          const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
          const uint32_t off = kk * 32;
          mma_tf32(t_re, sw128_desc(a0 + off), sw128_desc(b0 + off), idesc, acc);
          if (CPLX) mma_tf32(t_im, sw128_desc(a1 + off), sw128_desc(b0 + off), idesc, acc);
          if (SPLIT3) {
            const uint32_t as = smem_u32(a_tile(s, CPLX ? 2 : 1));
            const uint32_t bs = smem_u32(b_tile(s, 1));
            mma_tf32(t_re, sw128_desc(as + off), sw128_desc(b0 + off), idesc, 1u);
            mma_tf32(t_re, sw128_desc(a0 + off), sw128_desc(bs + off), idesc, 1u);
            if (CPLX) {
              const uint32_t ais = smem_u32(a_tile(s, 3));
              mma_tf32(t_im, sw128_desc(ais + off), sw128_desc(b0 + off), idesc, 1u);
              mma_tf32(t_im, sw128_desc(a1 + off), sw128_desc(bs + off), idesc, 1u);
            }
          }
        }
        mma_any = true;
        mma_commit(&empty_bar[s]);
        if (FOLD && (kb % CK == CK - 1 || kb == nkb - 1)) mma_commit(&acc_full[buf]);
      }
      if (mma_any) mma_commit(&done_bar);
    }
  } else {
    // rewrite workers: 128 threads over the A tile (and the B tile for SPLIT3)
    const int t = threadIdx.x - 64;
    float sr = 1.f, s1 = 1.f, s2 = 1.f;
    if (CPLX) {
      if (!g.conjA && !g.conjB) { sr = -1.f; s1 = 1.f; s2 = 1.f; }
      else if (g.conjA && !g.conjB) { sr = 1.f; s1 = -1.f; s2 = 1.f; }
      else if (!g.conjA && g.conjB) { sr = 1.f; s1 = 1.f; s2 = -1.f; }
      else { sr = -1.f; s1 = -1.f; s2 = -1.f; }
    }
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      // warp-uniform exit: the read-backs below are warp-collective
      if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[s], (kb / STAGES) & 1, &abort_flag))) break;
      {
        float4 *A0 = (float4 *)a_tile(s, 0);
        float4 *A1 = (float4 *)a_tile(s, 1);
        for (int c = t; c < L::A_BYTES / 16; c += 128) {
          const float4 v = A0[c];
          if (CPLX) {
            float4 re = make_float4(v.x, sr * v.y, v.z, sr * v.w);
            float4 imv = make_float4(s1 * v.y, s2 * v.x, s1 * v.w, s2 * v.z);
            if (!SPLIT3) {
              re = round4(re);
              imv = round4(imv);
            }
            if (SPLIT3) {
              float4 *A2 = (float4 *)a_tile(s, 2);
              float4 *A3 = (float4 *)a_tile(s, 3);
              const float4 rh = make_float4(tf32_head(re.x), tf32_head(re.y), tf32_head(re.z), tf32_head(re.w));
              const float4 ih = make_float4(tf32_head(imv.x), tf32_head(imv.y), tf32_head(imv.z), tf32_head(imv.w));
              A2[c] = make_float4(re.x - rh.x, re.y - rh.y, re.z - rh.z, re.w - rh.w);
              A3[c] = make_float4(imv.x - ih.x, imv.y - ih.y, imv.z - ih.z, imv.w - ih.w);
              re = rh;
              imv = ih;
            }
            A0[c] = re;
            A1[c] = imv;
          } else if (SPLIT3) {
            // real SPLIT3: head in place, tail to tile 1
            const float4 h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
            A1[c] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            A0[c] = h;
          } else {
            A0[c] = round4(v);
          }
        }
        if (!SPLIT3) {
          // TF32 products: round B to nearest as well (the tensor core would truncate)
          float4 *B0 = (float4 *)b_tile(s, 0);
          for (int c = t; c < L::B_BYTES / 16; c += 128) B0[c] = round4(B0[c]);
        }
        if (SPLIT3) {
          float4 *B0 = (float4 *)b_tile(s, 0);
          float4 *B1 = (float4 *)b_tile(s, 1);
          for (int c = t; c < L::B_BYTES / 16; c += 128) {
            const float4 v = B0[c];
            const float4 h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
            B1[c] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            B0[c] = h;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      mbar_arrive(&ready_bar[s]);
      // with the next chunk's operands ready, read back the chunk before it
      if (FOLD && kb % CK == CK - 1 && kb >= 2 * CK - 1 && !fold()) break;
    }
  }

  // ---- epilogue (warps 2..5 own tensor-memory lane quarters 2, 3, 0, 1) ----
  if (warp >= 2) {
    // output offsets of this tile's columns, once per tile
    for (int c = threadIdx.x - 64; c < BN; c += 128) col_off[c] = n0 + c < g.N ? map_index(g.mn, n0 + c) : 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    bool ok = __all_sync(0xffffffffu, !abort_flag);
    if (FOLD)
      while (ok && folded < nchunks) ok = fold();
    // done_bar also tracks the last MMAs' completion signal, which must land before exit
    ok = ok && mbar_wait(&done_bar, 0, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);      // tensor-memory loads are warp-collective
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = m0 + q * 32 + lane;
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      double alpha = g.alpha;
      if (g.alpha_dev) alpha *= *g.alpha_dev;
      const int64_t row_off = m < g.M ? map_index(g.mm, m) : 0;
      auto store = [&](int cl, float re, float im) {
        if (n0 + cl >= g.N) return;
        const int64_t off = row_off + col_off[cl];
        if (g.atomic64) {
          if (CPLX) {
            double2 *C = (double2 *)g.C + off;
            atomicAdd(&C->x, alpha * (double)re);
            atomicAdd(&C->y, (g.conjC ? -alpha : alpha) * (double)im);
          } else {
            atomicAdd((double *)g.C + off, alpha * (double)re);
          }
        } else if (CPLX) {
          float2 v = make_float2((float)(alpha * re), (float)(alpha * im));
          if (g.conjC) v.y = -v.y;
          float2 *C = (float2 *)g.C + off;
          if (g.accumulate) { const float2 o = *C; v.x += o.x; v.y += o.y; }
          *C = v;
        } else {
          float v = (float)(alpha * re);
          float *C = (float *)g.C + off;
          if (g.accumulate) v += *C;
          *C = v;
        }
      };
      if (FOLD) {
        if (m < g.M) {
#pragma unroll
          for (int c = 0; c < BN; ++c) store(c, facc[c], CPLX ? facc[(BN + c) % L::ACC_COLS] : 0.f);
        }
      } else {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float re[16], imv[16];
          tmem_ld16(lane_base + c0, re);
          if (CPLX) tmem_ld16(lane_base + BN + c0, imv);
          if (m >= g.M) continue;
#pragma unroll
          for (int i = 0; i < 16; ++i) store(c0 + i, re[i], CPLX ? imv[i] : 0.f);
        }
      }
    }
  }

  // ---- teardown: drain own copies and MMAs if a wait gave up ----
  __syncthreads();
  if (abort_flag) {
    if (threadIdx.x == 0 && g.status) atomicOr(g.status, STATUS_TIMEOUT);
    if (warp == 0 && lane == 0)
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        for (uint32_t i = 0; i < kWaitLimit && !mbar_test(&full_bar[kb % STAGES], (kb / STAGES) & 1); ++i) {
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

template <int BN, bool CPLX, bool SPLIT3> void launch_tc(const TcDesc &d, cudaStream_t s) {
  using L = Layout<BN, CPLX, SPLIT3>;
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(tc_gemm_kernel<BN, CPLX, SPLIT3>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    set = true;
  }
  const unsigned blocks = (unsigned)(d.tiles_m * d.tiles_n * (d.ksplit > 1 ? d.ksplit : 1));
  if (blocks) tc_gemm_kernel<BN, CPLX, SPLIT3><<<blocks, NTHREADS, L::SMEM, s>>>(d);
}

}  // namespace

int tc_block_n(int N, bool cplx, bool split3) { return N <= 64 || (cplx && split3) ? 64 : 128; }

void launch_tc_gemm(const TcDesc &d, int bn, cudaStream_t s) {
  if (bn == 64) {
    if (d.cplx) { if (d.split3) launch_tc<64, true, true>(d, s); else launch_tc<64, true, false>(d, s); }
    else { if (d.split3) launch_tc<64, false, true>(d, s); else launch_tc<64, false, false>(d, s); }
  } else {
    // (tc_block_n never gives 128 for complex SPLIT3)
    if (d.cplx) { if (!d.split3) launch_tc<128, true, false>(d, s); }
    else { if (d.split3) launch_tc<128, false, true>(d, s); else launch_tc<128, false, false>(d, s); }
  }
}

}  // namespace peps
