// Two-layer site stage of the implicit product (PLAIN arithmetic path).
//
// For the implicit matrix of a zip-up einsumsvd step (Algorithm 3 with
// Algorithm 4 applied implicitly, Sec. IV-A) the product A X starts by
// contracting the block X with the ket site K over its (down, right) bonds
// and with the conjugated bra site Kb over (physical, down, right): the two
// d*D^6 terms of Table 2's two-layer IBMPS column.  For every sketch column
// j and old-boundary bond b this is a "sandwich" of small matrices,
//   out_{j,b} = sum_s K_s X_{j,b} Kb_s^H        (forward)
//   out_{j,b} = sum_s K_s^H Z_{j,b} Kb_s        (adjoint, for A^H Y)
// with K_s the [(l,u)][(x,e)] slice.  One block stages K and Kb in shared
// memory once and walks a run of (j, b) items; each thread owns a 4 x 4
// register tile of the two chained small products.
#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int find_desc64(const int64_t *prefix, int nd, int64_t blk) {
  int lo = 0, hi = nd - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }

// acc[ii][jj] += sum_k A[k*lda + i0+ii] * B[k*ldb + j0+jj]
template <class T>
__device__ __forceinline__ void tile_mm(const T *A, int lda, const T *B, int ldb, int K, int i0,
                                        int j0, T (&acc)[4][4]) {
  for (int k = 0; k < K; ++k) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = A[k * lda + i0 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = B[k * ldb + j0 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma_(a[i], b[j], acc[i][j]);
  }
}

template <class T> __device__ __forceinline__ void clear(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
}

// Shared-memory layout (elements), forward:
//   KT  [d][Q1][P1p]   KT[s][k][r]  = K[s][r][k]          r=(l,u), k=(x,e)
//   KbT [d][Q2][P2p]   KbT[s][k][c] = conj(Kb[s][c][k])    c=(L,U), k=(X,E)
//   Xs  [Q1][Q2p]      item slab X_{j,b}[(x,e)][(X,E)]
//   T1T [Q2][P1p]      (K_s X_{j,b})^T
// adjoint:
//   KcT [d][P1][Q1p]   KcT[s][r][k] = conj(K[s][r][k])
//   KbS [d][P2][Q2p]   KbS[s][c][k] = Kb[s][c][k]
//   ZsT [P2][P1p]      item slab Z_{j,b}[(l,u)][(L,U)] transposed
//   T1p [P1][Q2p]      Z_{j,b} Kb_s
struct Dims {
  int d, P1, Q1, P2, Q2, P1p, Q1p, P2p, Q2p;
};

__host__ __device__ inline Dims make_dims(const SandwichDesc &g) {
  Dims z;
  z.d = g.d;
  z.P1 = g.Dl * g.Du;
  z.Q1 = g.Dx * g.De;
  z.P2 = g.DL * g.DU;
  z.Q2 = g.DX * g.DE;
  z.P1p = pad4(z.P1);
  z.Q1p = pad4(z.Q1);
  z.P2p = pad4(z.P2);
  z.Q2p = pad4(z.Q2);
  return z;
}

__host__ __device__ inline int64_t smem_elems(const SandwichDesc &g) {
  Dims z = make_dims(g);
  if (!g.adjoint)
    return (int64_t)z.d * z.Q1 * z.P1p + (int64_t)z.d * z.Q2 * z.P2p + (int64_t)z.Q1 * z.Q2p +
           (int64_t)z.Q2 * z.P1p;
  return (int64_t)z.d * z.P1 * z.Q1p + (int64_t)z.d * z.P2 * z.Q2p + (int64_t)z.P2 * z.P1p +
         (int64_t)z.P1 * z.Q2p;
}

template <class T>
__global__ void __launch_bounds__(NT) sandwich_kernel(const SandwichDesc *__restrict__ descs,
                                                      const int64_t *__restrict__ prefix, int nd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int di = find_desc64(prefix, nd, blockIdx.x);
  const SandwichDesc &g = descs[di];
  const Dims z = make_dims(g);
  const int tid = threadIdx.x;
  const T *K = (const T *)g.K;
  const T *Kb = (const T *)g.Kb;
  const int64_t items = (int64_t)g.ell * g.B;
  const int64_t it0 = (int64_t)(blockIdx.x - prefix[di]) * g.items_per_block;
  const int64_t it1 = min(items, it0 + g.items_per_block);
  const int Dv = g.Du * g.DU;                 // vertical (ket, bra) pair size

  if (!g.adjoint) {
    T *KT = sm;
    T *KbT = KT + z.d * z.Q1 * z.P1p;
    T *Xs = KbT + z.d * z.Q2 * z.P2p;
    T *T1T = Xs + z.Q1 * z.Q2p;
    for (int i = tid; i < z.d * z.Q1 * z.P1p; i += NT) {
      const int s = i / (z.Q1 * z.P1p), rem = i % (z.Q1 * z.P1p);
      const int k = rem / z.P1p, r = rem % z.P1p;
      KT[i] = r < z.P1 ? K[((int64_t)s * z.P1 + r) * z.Q1 + k] : zero<T>();
    }
    for (int i = tid; i < z.d * z.Q2 * z.P2p; i += NT) {
      const int s = i / (z.Q2 * z.P2p), rem = i % (z.Q2 * z.P2p);
      const int k = rem / z.P2p, c = rem % z.P2p;
      KbT[i] = c < z.P2 ? conj_(Kb[((int64_t)s * z.P2 + c) * z.Q2 + k]) : zero<T>();
    }
    // pads of the item buffers stay zero
    for (int i = tid; i < z.Q1 * z.Q2p; i += NT) Xs[i] = zero<T>();
    for (int i = tid; i < z.Q2 * z.P1p; i += NT) T1T[i] = zero<T>();
    __syncthreads();
    const int tA = (z.P1p / 4) * (z.Q2p / 4);   // tiles of T1 (r x k2)
    const int tB = (z.P1p / 4) * (z.P2p / 4);   // tiles of out (r x c)
    for (int64_t it = it0; it < it1; ++it) {
      const int64_t j = it / g.B;
      const int b = (int)(it % g.B);
      const T *X = (const T *)g.in + j * g.ld_in;
      for (int i = tid; i < z.Q1 * z.Q2; i += NT) {
        const int k = i / z.Q2, c2 = i % z.Q2;
        const int x = k / g.De, e = k % g.De, X_ = c2 / g.DE, E = c2 % g.DE;
        Xs[k * z.Q2p + c2] = X[((((int64_t)x * g.DX + X_) * g.B + b) * g.De + e) * g.DE + E];
      }
      T acc[4][4];
      clear(acc);
      for (int s = 0; s < z.d; ++s) {
        __syncthreads();
        if (tid < tA) {
          const int r0 = (tid / (z.Q2p / 4)) * 4, c0 = (tid % (z.Q2p / 4)) * 4;
          T t[4][4];
          clear(t);
          tile_mm(KT + s * z.Q1 * z.P1p, z.P1p, Xs, z.Q2p, z.Q1, r0, c0, t);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
              if (c0 + jj < z.Q2) T1T[(c0 + jj) * z.P1p + r0 + i] = t[i][jj];
        }
        __syncthreads();
        if (tid < tB) {
          const int r0 = (tid / (z.P2p / 4)) * 4, c0 = (tid % (z.P2p / 4)) * 4;
          tile_mm(T1T, z.P1p, KbT + s * z.Q2 * z.P2p, z.P2p, z.Q2, r0, c0, acc);
        }
      }
      if (tid < tB) {
        const int r0 = (tid / (z.P2p / 4)) * 4, c0 = (tid % (z.P2p / 4)) * 4;
        T *O = (T *)g.out + j * g.ld_out;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = r0 + i;
          if (r >= z.P1) continue;
          const int l = r / g.Du, u = r % g.Du;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int c = c0 + jj;
            if (c >= z.P2) continue;
            const int L = c / g.DU, U = c % g.DU;
            O[(((int64_t)l * g.DL + L) * Dv + u * g.DU + U) * g.B + b] = acc[i][jj];
          }
        }
      }
      __syncthreads();
    }
  } else {
    T *KcT = sm;
    T *KbS = KcT + z.d * z.P1 * z.Q1p;
    T *ZsT = KbS + z.d * z.P2 * z.Q2p;
    T *T1p = ZsT + z.P2 * z.P1p;
    for (int i = tid; i < z.d * z.P1 * z.Q1p; i += NT) {
      const int s = i / (z.P1 * z.Q1p), rem = i % (z.P1 * z.Q1p);
      const int r = rem / z.Q1p, k = rem % z.Q1p;
      KcT[i] = k < z.Q1 ? conj_(K[((int64_t)s * z.P1 + r) * z.Q1 + k]) : zero<T>();
    }
    for (int i = tid; i < z.d * z.P2 * z.Q2p; i += NT) {
      const int s = i / (z.P2 * z.Q2p), rem = i % (z.P2 * z.Q2p);
      const int c = rem / z.Q2p, k = rem % z.Q2p;
      KbS[i] = k < z.Q2 ? Kb[((int64_t)s * z.P2 + c) * z.Q2 + k] : zero<T>();
    }
    for (int i = tid; i < z.P2 * z.P1p; i += NT) ZsT[i] = zero<T>();
    for (int i = tid; i < z.P1 * z.Q2p; i += NT) T1p[i] = zero<T>();
    __syncthreads();
    const int tA = (z.P1p / 4) * (z.Q2p / 4);   // tiles of T1p (r x k2)
    const int tB = (z.Q1p / 4) * (z.Q2p / 4);   // tiles of out (k x k2)
    for (int64_t it = it0; it < it1; ++it) {
      const int64_t j = it / g.B;
      const int b = (int)(it % g.B);
      const T *Zin = (const T *)g.in + j * g.ld_in;
      for (int i = tid; i < z.P1 * z.P2; i += NT) {
        const int r = i / z.P2, c = i % z.P2;
        const int l = r / g.Du, u = r % g.Du, L = c / g.DU, U = c % g.DU;
        ZsT[c * z.P1p + r] = Zin[(((int64_t)l * g.DL + L) * Dv + u * g.DU + U) * g.B + b];
      }
      T acc[4][4];
      clear(acc);
      for (int s = 0; s < z.d; ++s) {
        __syncthreads();
        if (tid < tA) {
          const int r0 = (tid / (z.Q2p / 4)) * 4, c0 = (tid % (z.Q2p / 4)) * 4;
          T t[4][4];
          clear(t);
          tile_mm(ZsT, z.P1p, KbS + s * z.P2 * z.Q2p, z.Q2p, z.P2, r0, c0, t);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (r0 + i < z.P1)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) T1p[(r0 + i) * z.Q2p + c0 + jj] = t[i][jj];
        }
        __syncthreads();
        if (tid < tB) {
          const int k0 = (tid / (z.Q2p / 4)) * 4, c0 = (tid % (z.Q2p / 4)) * 4;
          tile_mm(KcT + s * z.P1 * z.Q1p, z.Q1p, T1p, z.Q2p, z.P1, k0, c0, acc);
        }
      }
      if (tid < tB) {
        const int k0 = (tid / (z.Q2p / 4)) * 4, c0 = (tid % (z.Q2p / 4)) * 4;
        T *O = (T *)g.out + j * g.ld_out;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int k = k0 + i;
          if (k >= z.Q1) continue;
          const int x = k / g.De, e = k % g.De;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int c2 = c0 + jj;
            if (c2 >= z.Q2) continue;
            const int X_ = c2 / g.DE, E = c2 % g.DE;
            O[((((int64_t)x * g.DX + X_) * g.B + b) * g.De + e) * g.DE + E] = acc[i][jj];
          }
        }
      }
      __syncthreads();
    }
  }
}

template <class T>
void launch_t(const SandwichDesc *d, const int64_t *prefix, int nd, int64_t blocks, int smem,
              cudaStream_t s) {
  if (blocks <= 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(sandwich_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set = true;
  }
  sandwich_kernel<T><<<(unsigned)blocks, NT, smem, s>>>(d, prefix, nd);
}

}  // namespace

int sandwich_smem_bytes(int dt, const SandwichDesc &d) {
  return (int)(smem_elems(d) * dtype_size(dt));
}

void launch_sandwich(int dt, const SandwichDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                     int smem, cudaStream_t s) {
  switch (dt) {
    case DT_R32: launch_t<float>(d, prefix, nd, blocks, smem, s); break;
    case DT_C64: launch_t<float2>(d, prefix, nd, blocks, smem, s); break;
    case DT_R64: launch_t<double>(d, prefix, nd, blocks, smem, s); break;
    case DT_C128: launch_t<double2>(d, prefix, nd, blocks, smem, s); break;
  }
}

}  // namespace peps
