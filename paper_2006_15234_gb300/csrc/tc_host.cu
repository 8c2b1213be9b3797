// Host side of the tensor-core GEMM: TMA map encoding through the driver
// entry point (no link-time dependency on libcuda) and a self-contained
// verification entry point of the C ABI.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/libpeps.h"
#include "common.cuh"
#include "tcgemm.h"

namespace peps {

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  }
  return fn;
}
}  // namespace

bool tc_operand_ok(const void *base, int64_t pitch_bytes) {
  return ((uintptr_t)base % 16 == 0) && (pitch_bytes % 16 == 0) && pitch_bytes > 0;
}

bool tc_encode_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t pitch_bytes,
                   int box_rows) {
  std::memset(map, 0, sizeof(*map));
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tc_operand_ok(base, pitch_bytes)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace peps

using namespace peps;

extern "C" peps_status peps_debug_tc_gemm(int32_t cplx, int32_t conjA, int32_t conjB, int32_t split3, int32_t M,
                                          int32_t N, int32_t K, const void *A, const void *B, void *C,
                                          void *scratch, void *stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || split3 < 0 || split3 > 2) return PEPS_ERR_ARG;
  if (split3 == 2 && !scratch) return PEPS_ERR_ARG;
  const int64_t kr = (int64_t)K * (cplx ? 2 : 1);
  const int64_t pitch = kr * 4;
  TcDesc d;
  std::memset(&d, 0, sizeof d);
  const int nmma = tc_pick_nmma(N, cplx != 0, split3 != 0);
  const int bn = tc_tile_cols(nmma, cplx != 0);
  if (!tc_encode_map(&d.ta, A, M, kr, pitch, 128)) return PEPS_ERR_UNSUPPORTED;
  if (split3 == 2) {
    const int64_t nr = (int64_t)N * (cplx ? 2 : 1);
    if (!tc_encode_map(&d.tb, scratch, nr, kr, pitch, nmma) ||
        !tc_encode_map(&d.tb2, (char *)scratch + nr * pitch, nr, kr, pitch, nmma))
      return PEPS_ERR_UNSUPPORTED;
    d.bpre = 1;
    d.Braw = B;
    d.Bx = scratch;
  } else if (!tc_encode_map(&d.tb, B, N, kr, pitch, bn)) {
    return PEPS_ERR_UNSUPPORTED;
  }
  d.M = M; d.N = N; d.Kr = (int32_t)kr;
  d.cplx = cplx; d.conjA = conjA; d.conjB = conjB; d.split3 = split3 != 0;
  d.tiles_m = (M + 127) / 128;
  d.tiles_n = (N + bn - 1) / bn;
  d.mm = digits1(N);
  d.mn = digits1(1);
  d.C = C;
  d.alpha = 1.0;
  launch_tc_gemm(d, nmma, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? PEPS_OK : PEPS_ERR_CUDA;
}
