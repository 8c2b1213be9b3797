// Descriptor of the tensor-core GEMM (tcgemm.cu) and its host helpers.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace peps {

// index -> sum_d digit_d * stride_d, digit 0 least significant (radix[d]).
// mul / shr: division by radix[d] as a multiply-high and shift (filled by
// the launcher; exact for indices below 2^31).
struct DigitMap {
  int32_t n;
  int32_t radix[4];
  int64_t stride[4];
  uint32_t mul[4], shr[4];
};

// C(m, n) (+)= alpha * sum_k opA(A[m][k]) opB(B[n][k]); A, B row-major with K
// contiguous, complex interleaved when cplx.  C's element (m, n) sits at
// C + mm(m) + mn(n) (elements of the output type: float2 or float).
// bpre (SPLIT3 only): before the GEMM, B is rewritten once into Bx as the
// MMA's real operand rows, head rows [0, NR) and tail rows [NR, 2 NR)
// (NR = 2N for complex data: Re and Im rows of each complex row; N for real
// data), so that the GEMM's B tiles arrive by TMA ready for the MMA (tb over
// the head rows, tb2 over the tail rows).
struct TcDesc {
  CUtensorMap ta;
  CUtensorMap tb;
  CUtensorMap tb2;
  int32_t M, N, Kr;        // Kr = K extent in floats (2K for complex data)
  int32_t cplx, conjA, conjB, split3;
  int32_t tiles_m, tiles_n;
  DigitMap mm, mn;
  void *C;
  double alpha;
  const double *alpha_dev;
  int32_t accumulate, conjC;
  int32_t atomic64;        // C holds FP64 accumulators (double / double2): atomicAdd
  int32_t ksplit, kb_per_split;   // K cut into ksplit chunks of kb_per_split 32-float blocks
  int32_t bpre;
  const void *Braw;        // bpre: B as given (N rows of Kr floats)
  void *Bx;                // bpre: tc_bx_bytes(N, Kr, cplx) bytes
  uint32_t *status;        // STATUS_TIMEOUT is or-ed in when a wait gives up (may be NULL)
  uint64_t wait_ns;        // limit of one pipeline wait in ns (0: the default of 2 s)
};

// bytes of the pre-expanded B operand (head and tail rows)
inline int64_t tc_bx_bytes(int64_t n, int64_t kr, bool cplx) { return n * kr * 4 * 2 * (cplx ? 2 : 1); }

// MMA width (64, 128, 192 or 256 accumulator columns; SPLIT3 at most 192) for
// an N extent: a tile covers nmma output columns (real) or nmma / 2 (complex,
// Re/Im pairs).
// Whether a SPLIT3 product folds its accumulation chunks (K longer than two
// chunks); kb_per_split > 0 when K is split across CTAs.
bool tc_folds(bool split3, int64_t kr, int kb_per_split);
int tc_pick_nmma(int N, bool cplx, bool split3);
inline int tc_tile_cols(int nmma, bool cplx) { return cplx ? nmma / 2 : nmma; }
void launch_tc_gemm(const TcDesc &d, int nmma, cudaStream_t s);

// Encode a 2-D TMA map over rows x cols FP32 values (row pitch in bytes) with
// a box of 32 floats x box_rows and the 128-byte swizzle.  Returns false when
// the driver entry point is unavailable (no GPU driver) or encoding fails.
bool tc_encode_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t pitch_bytes,
                   int box_rows);
// Whether a K-contiguous operand can be fed by TMA (alignment rules).
bool tc_operand_ok(const void *base, int64_t pitch_bytes);

// Division by an invariant integer r >= 1 as multiply-high, add and shift
// (Granlund and Montgomery, 1994): with l = ceil(log2 r) and
// mul = floor(2^32 (2^l - r) / r) + 1, i / r = (umulhi(i, mul) + i) >> l for
// every i < 2^31 (the sum then fits in 32 bits).
inline void div_magic(uint64_t r, uint32_t *mul, uint32_t *shr) {
  if (r == 0) r = 0x7fffffffull;
  uint32_t l = 0;
  while ((1ull << l) < r) ++l;
  *mul = (uint32_t)(((1ull << 32) * ((1ull << l) - r)) / r + 1);
  *shr = l;
}

inline DigitMap digits1(int64_t stride) {
  DigitMap d{};
  d.n = 1;
  d.radix[0] = 0x7fffffff;
  d.stride[0] = stride;
  return d;
}

}  // namespace peps
