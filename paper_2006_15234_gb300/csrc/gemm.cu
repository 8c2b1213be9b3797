// Grouped, strided, batched GEMM on CUDA cores (the PLAIN arithmetic path).
//
// Serves every dense contraction of one einsumsvd step whose operands are
// already laid out as matrices: the two m^2 stages of the implicit product
// (boundary site S and carry V, Sec. IV-A / Table 2), their adjoints, the
// Gram matrices of CholeskyQR (64-term partial sums folded into FP64, split
// over K and combined atomically in FP64),
// the R^-1 applications and the U = P U~, W = U~^H B epilogue (Algorithm 4's
// last lines).  Strides are arbitrary; each tile load picks the coalesced
// direction from the unit stride.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int BM = kGemmBM, BN = kGemmBN, BK = 16, NT = 256;
constexpr int kFoldTiles = 4;   // K tiles per single-precision partial sum of a Gram

__device__ __forceinline__ int find_desc(const int64_t *prefix, int nd, int64_t blk) {
  int lo = 0, hi = nd - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T> __device__ __forceinline__ T ldg_(const T *p) { return *p; }

template <class T, bool ATOMIC>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmDesc *__restrict__ descs,
                                                  const int64_t *__restrict__ prefix, int nd) {
  using Acc = typename Traits<T>::Acc;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];

  const int64_t blk = blockIdx.x;
  const int di = find_desc(prefix, nd, blk);
  const GemmDesc &g = descs[di];
  // 32-bit block arithmetic (block indices and tile counts fit; 64-bit
  // division runs through FP64 operations)
  uint32_t local = (uint32_t)(blk - prefix[di]);
  const uint32_t mn = (uint32_t)g.tiles_m * (uint32_t)g.tiles_n, per_batch = (uint32_t)g.ksplit * mn;
  const int bi = (int)(local / per_batch);
  local -= (uint32_t)bi * per_batch;
  const int kc = (int)(local / mn);
  local -= (uint32_t)kc * mn;
  const int tm = (int)(local / (uint32_t)g.tiles_n);
  const int tn = (int)(local % (uint32_t)g.tiles_n);
  const int m0 = tm * BM, n0 = tn * BN;
  const int kbeg = kc * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);

  const T *A = (const T *)g.A + (int64_t)bi * g.sAb;
  const T *B = (const T *)g.B + (int64_t)bi * g.sBb;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const bool conjA = g.conjA, conjB = g.conjB;
  const bool a_kc = (g.sAk == 1), a_mc = (g.sAm == 1);
  const bool b_nc = (g.sBn == 1), b_kc = (g.sBk == 1);

  // Store mode accumulates in the working type.  Gram (atomic) mode keeps
  // short partial sums (kFoldTiles K tiles) in the working type and folds
  // them into FP64 accumulators, so rounding does not grow with K.
  T acc[4][4];
  Acc acc64[ATOMIC ? 4 : 1][ATOMIC ? 4 : 1];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
#pragma unroll
  for (int i = 0; i < (ATOMIC ? 4 : 1); ++i)
#pragma unroll
    for (int j = 0; j < (ATOMIC ? 4 : 1); ++j) acc64[i][j] = Acc{};

  int tile_count = 0;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      const int idx = tid + r * NT;
      int mm, kk;
      if (a_kc || !a_mc) { kk = idx & (BK - 1); mm = idx >> 4; }
      else { mm = idx & (BM - 1); kk = idx >> 6; }
      const int m = m0 + mm, k = k0 + kk;
      T v = zero<T>();
      if (m < g.M && k < kend) v = cj(A[(int64_t)m * g.sAm + (int64_t)k * g.sAk], conjA);
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      const int idx = tid + r * NT;
      int nn, kk;
      if (b_nc || !b_kc) { nn = idx & (BN - 1); kk = idx >> 6; }
      else { kk = idx & (BK - 1); nn = idx >> 4; }
      const int n = n0 + nn, k = k0 + kk;
      T v = zero<T>();
      if (n < g.N && k < kend) v = cj(B[(int64_t)k * g.sBk + (int64_t)n * g.sBn], conjB);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma_(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if constexpr (ATOMIC) {
      if ((++tile_count % kFoldTiles) == 0 || k0 + BK >= kend) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc64[i][j] = add(acc64[i][j], widen(acc[i][j]));
            acc[i][j] = zero<T>();
          }
      }
    }
  }

  double alpha = g.alpha;
  if (g.alpha_dev) alpha *= *g.alpha_dev;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      const int64_t off = (int64_t)bi * g.sCb + (int64_t)m * g.sCm + (int64_t)n * g.sCn;
      if constexpr (ATOMIC) {
        Acc v = acc64[i][j];
        if (g.conjC) v = conj_(v);
        atomic_add_acc((Acc *)g.C + off, scale(v, alpha));
      } else {
        T v = scale(acc[i][j], (typename Traits<T>::Real)alpha);
        if (g.conjC) v = conj_(v);
        T *C = (T *)g.C + off;
        if (g.accumulate) v = add(v, *C);
        *C = v;
      }
    }
  }
}

template <class T>
void launch_t(bool atomic, const GemmDesc *d, const int64_t *prefix, int nd, int64_t blocks,
              cudaStream_t s) {
  if (blocks <= 0) return;
  if (atomic)
    gemm_kernel<T, true><<<(unsigned)blocks, NT, 0, s>>>(d, prefix, nd);
  else
    gemm_kernel<T, false><<<(unsigned)blocks, NT, 0, s>>>(d, prefix, nd);
}

}  // namespace

void launch_gemm(int dt, bool atomic, const GemmDesc *d, const int64_t *prefix, int nd,
                 int64_t blocks, cudaStream_t s) {
  switch (dt) {
    case DT_R32: launch_t<float>(atomic, d, prefix, nd, blocks, s); break;
    case DT_C64: launch_t<float2>(atomic, d, prefix, nd, blocks, s); break;
    case DT_R64: launch_t<double>(atomic, d, prefix, nd, blocks, s); break;
    case DT_C128: launch_t<double2>(atomic, d, prefix, nd, blocks, s); break;
  }
}

}  // namespace peps
