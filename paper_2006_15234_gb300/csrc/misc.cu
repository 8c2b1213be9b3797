// Sketch generation and the small per-row kernels of the boundary sweep.
//
//  * sketch: Philox4x64-10 (Salmon et al., SC'11) draw of Algorithm 4's start
//    block, counter (block, instance, tag, 0), key (seed, 0); element
//    e = j*N + n; Box-Muller on word pairs (real: 4 normals per block;
//    complex: 2 values per block, scaled by 1/sqrt 2).  The uniform is
//    ((x >> 11) + 1/2) 2^-53, rounded once to the working precision.
//  * site: the untruncated first row of the two-layer network (Algorithm 2,
//    first line) and the zip-up start V1 = S1 O1 (Algorithm 3, first line).
//  * scalar: the final contraction of a boundary with trivial vertical bonds
//    (Algorithm 2, last line), returned as log|v| plus the carried logs.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace peps {

namespace {

__device__ __forceinline__ int find_desc(const int64_t *prefix, int nd, int64_t blk) {
  int lo = 0, hi = nd - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr uint64_t PH_M0 = 0xD2E7470EE14C6C93ull, PH_M1 = 0xCA5A826395121157ull;
constexpr uint64_t PH_W0 = 0x9E3779B97F4A7C15ull, PH_W1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(PH_M0, c[0]), lo0 = PH_M0 * c[0];
    const uint64_t hi1 = __umul64hi(PH_M1, c[2]), lo1 = PH_M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += PH_W0; k1 += PH_W1;
  }
}

template <class R> struct Uni;
template <> struct Uni<double> {
  __device__ static double u(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }
  __device__ static void bm(double u0, double u1, double &a, double &b) {
    const double r = sqrt(-2.0 * log(u0));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    a = r * cs; b = r * sn;
  }
};
template <> struct Uni<float> {
  // same 53-bit uniform as the double path, ((x >> 11) + 1/2) 2^-53 =
  // (2 (x >> 11) + 1) 2^-54 exactly, rounded once to 24 bits by the integer
  // conversion (the scaling by a power of two is exact)
  __device__ static float u(uint64_t x) {
    return __ull2float_rn(((x >> 11) << 1) | 1ull) * 0x1.0p-54f;
  }
  __device__ static void bm(float u0, float u1, float &a, float &b) {
    const float r = sqrtf(-2.0f * logf(u0));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    a = r * cs; b = r * sn;
  }
};

template <class T>
__global__ void sketch_kernel(const SketchDesc *__restrict__ descs, const int64_t *__restrict__ prefix,
                              int nd) {
  using R = typename Traits<T>::Real;
  constexpr bool CPLX = Traits<T>::cplx;
  constexpr int PER = CPLX ? 2 : 4;
  const int di = find_desc(prefix, nd, blockIdx.x);
  const SketchDesc &g = descs[di];
  const int64_t total = g.N * g.ell;
  const int64_t blk = (int64_t)(blockIdx.x - prefix[di]) * blockDim.x + threadIdx.x;
  if (blk * PER >= total) return;
  uint64_t c[4] = {(uint64_t)blk, g.instance, (uint64_t)g.tag, 0ull};
  philox4x64_10(c, g.seed, 0ull);
  R v[4];
  if (g.kind == 0) {
    Uni<R>::bm(Uni<R>::u(c[0]), Uni<R>::u(c[1]), v[0], v[1]);
    Uni<R>::bm(Uni<R>::u(c[2]), Uni<R>::u(c[3]), v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (R)2 * Uni<R>::u(c[i]) - (R)1;
  }
  T *X = (T *)g.X;
  const bool small = total < (1ll << 31);      // 32-bit index arithmetic (multiply-shift division)
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t e = blk * PER + r;
    if (e >= total) break;
    if (small) {
      const uint32_t e32 = (uint32_t)e;
      const uint32_t j = (__umulhi(e32, g.nmul) + e32) >> g.nshr;
      uint32_t n = e32 - j * (uint32_t)g.N;
      T val;
      if constexpr (CPLX) {
        const R sc = g.kind == 0 ? (R)0.70710678118654752440 : (R)1;
        val = from_parts<T>((double)(v[2 * r] * sc), (double)(v[2 * r + 1] * sc));
      } else {
        val = from_parts<T>((double)v[r], 0.0);
      }
      int64_t off = n;
      if (g.nd) {
        off = 0;
        for (int d = 0; d < g.nd; ++d) {
          const uint32_t q = (__umulhi(n, g.rmul[d]) + n) >> g.rshr[d];
          off += (int64_t)(n - q * (uint32_t)g.radix[d]) * g.stride[d];
          n = q;
        }
      }
      X[(int64_t)j * g.ld + off] = val;
      continue;
    }
    const int64_t j = e / g.N, n = e % g.N;
    T val;
    if constexpr (CPLX) {
      const R sc = g.kind == 0 ? (R)0.70710678118654752440 : (R)1;
      val = from_parts<T>((double)(v[2 * r] * sc), (double)(v[2 * r + 1] * sc));
    } else {
      val = from_parts<T>((double)v[r], 0.0);
    }
    int64_t off = n;
    if (g.nd) {
      off = 0;
      int64_t r = n;
      for (int d = 0; d < g.nd; ++d) {
        off += (r % g.radix[d]) * g.stride[d];
        r /= g.radix[d];
      }
    }
    X[j * g.ld + off] = val;
  }
}

// Tiled 32 x 32 transpose of the (r, c) index pair; the inner block q is
// carried along (q == 1 for plain matrix transposes).
template <class T>
__global__ void permute_kernel(const PermuteDesc *__restrict__ descs, const int64_t *__restrict__ prefix,
                               int nd) {
  __shared__ T tile[32][33];
  const int di = find_desc(prefix, nd, blockIdx.x);
  const PermuteDesc &g = descs[di];
  // block coordinates in 32-bit arithmetic (a block index and the tile counts
  // fit; 64-bit division runs through FP64 operations, 1/64 rate here)
  const uint32_t tr = (uint32_t)((g.R + 31) / 32), tc = (uint32_t)((g.Cc + 31) / 32), Q = (uint32_t)g.Q;
  uint32_t blk = (uint32_t)(blockIdx.x - prefix[di]);
  const int64_t q = blk % Q; blk /= Q;
  const int64_t cb = blk % tc; blk /= tc;
  const int64_t rb = blk % tr; blk /= tr;
  const int64_t b = blk;
  const T *in = (const T *)g.in + b * g.R * g.Cc * g.Q;
  T *out = (T *)g.out + b * g.R * g.Cc * g.Q;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = rb * 32 + i, c = cb * 32 + tx;
    if (r < g.R && c < g.Cc) tile[i][tx] = in[(r * g.Cc + c) * g.Q + q];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t c = cb * 32 + i, r = rb * 32 + tx;
    if (r < g.R && c < g.Cc) {
      T v = tile[tx][i];
      if (g.conj) v = conj_(v);
      out[(c * g.R + r) * g.Q + q] = v;
    }
  }
}

template <class T>
__global__ void site_kernel(const SiteDesc *__restrict__ descs, const int64_t *__restrict__ prefix,
                            int nd) {
  const int di = find_desc(prefix, nd, blockIdx.x);
  const SiteDesc &g = descs[di];
  const int64_t idx = (int64_t)(blockIdx.x - prefix[di]) * blockDim.x + threadIdx.x;
  if (idx >= g.total) return;
  const T *K = (const T *)g.K, *Kb = (const T *)g.Kb;
  // K strides for [d][Dl][Du][Dx][De]
  const int64_t kE = 1, kX = g.De, kU = (int64_t)g.Dx * g.De, kL = kU * g.Du, kS = kL * g.Dl;
  const int64_t bE = 1, bX = g.DE, bU = (int64_t)g.DX * g.DE, bL = bU * g.DU, bS = bL * g.DL;
  using Acc = typename Traits<T>::Acc;      // FP64 sums: these sites start every row's sweep
  Acc acc = zero<Acc>();
  if (g.mode == 0) {
    // out[(l,L)][(x,X)][(e,E)], u = U = 0
    int64_t r = idx;
    const int E = r % g.DE; r /= g.DE;
    const int e = r % g.De; r /= g.De;
    const int X_ = r % g.DX; r /= g.DX;
    const int x = r % g.Dx; r /= g.Dx;
    const int L = r % g.DL; r /= g.DL;
    const int l = (int)r;
    for (int s = 0; s < g.d; ++s)
      acc = fma_(widen(K[s * kS + l * kL + x * kX + e * kE]),
                 conj_(widen(Kb[s * bS + L * bL + X_ * bX + E * bE])), acc);
  } else {
    // out[(x,X)][b][(e,E)] = sum S1[0][(u,U)][b] K[s,0,u,x,e] conj(Kb[s,0,U,X,E])
    const T *S = (const T *)g.S;
    int64_t r = idx;
    const int E = r % g.DE; r /= g.DE;
    const int e = r % g.De; r /= g.De;
    const int b = r % g.B; r /= g.B;
    const int X_ = r % g.DX; r /= g.DX;
    const int x = (int)r;
    for (int u = 0; u < g.Du; ++u)
      for (int U = 0; U < g.DU; ++U) {
        const Acc sv = widen(S[((int64_t)u * g.DU + U) * g.B + b]);
        Acc t = zero<Acc>();
        for (int s = 0; s < g.d; ++s)
          t = fma_(widen(K[s * kS + u * kU + x * kX + e * kE]),
                   conj_(widen(Kb[s * bS + U * bU + X_ * bX + E * bE])), t);
        acc = fma_(sv, t, acc);
      }
  }
  ((T *)g.out)[idx] = narrow<T>(acc);
}

template <class T>
__global__ void pad_kernel(const PadDesc *__restrict__ descs, const int64_t *__restrict__ prefix, int nd) {
  const int di = find_desc(prefix, nd, blockIdx.x);
  const PadDesc &g = descs[di];
  const int64_t o = (int64_t)(blockIdx.x - prefix[di]) * kPadPerBlock + threadIdx.x;
  if (o >= g.total) return;
  int64_t off = 0;
  bool in_range = true;
  if (g.total < ((int64_t)1 << 31)) {
    // 32-bit digits (a 64-bit division runs through FP64 operations)
    uint32_t r = (uint32_t)o;
    for (int d = g.nd - 1; d >= 0; --d) {
      const uint32_t dim = (uint32_t)g.dims[d], dig = r % dim;
      r /= dim;
      in_range = in_range && (int)dig < g.lim[d];
      off += (int64_t)dig * g.in_stride[d];
    }
  } else {
    int64_t r = o;
    for (int d = g.nd - 1; d >= 0; --d) {
      const int64_t dig = r % g.dims[d];
      r /= g.dims[d];
      in_range = in_range && dig < g.lim[d];
      off += dig * g.in_stride[d];
    }
  }
  ((T *)g.out)[o] = in_range ? ((const T *)g.in)[off] : zero<T>();
}

__global__ void zero_kernel(const ZeroDesc *__restrict__ descs, const int64_t *__restrict__ prefix,
                            int nd) {
  const int di = find_desc(prefix, nd, blockIdx.x);
  const ZeroDesc &g = descs[di];
  const int64_t w0 = (int64_t)(blockIdx.x - prefix[di]) * kZeroWordsPerBlock;
  uint64_t *p = (uint64_t *)g.p;
  for (int64_t i = w0 + threadIdx.x; i < min(g.words, w0 + kZeroWordsPerBlock); i += blockDim.x) p[i] = 0ull;
}

template <class T> __global__ void fill_kernel(T *p, int64_t n, double value) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = from_parts<T>(value, 0.0);
}

// v_{q+1}[r] = sum_l v_q[l] S_q[l][0][r] in FP64; one block, sequential sites.
template <class T> __global__ void scalar_kernel(ScalarDesc g) {
  using Acc = typename Traits<T>::Acc;
  Acc *v = (Acc *)g.scratch;
  int maxb = 1;
  for (int q = 0; q < g.ncol; ++q) maxb = max(maxb, max(g.left[q], g.right[q]));
  Acc *w = v + maxb;
  if (threadIdx.x == 0) v[0] = widen(from_parts<T>(1.0, 0.0));
  __syncthreads();
  for (int q = 0; q < g.ncol; ++q) {
    const T *S = (const T *)g.sites[q];
    const int L = g.left[q], R = g.right[q];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      Acc a = widen(zero<T>());
      for (int l = 0; l < L; ++l) a = fma_(v[l], widen(S[(int64_t)l * R + r]), a);
      w[r] = a;
    }
    __syncthreads();
    Acc *t = v; v = w; w = t;
  }
  if (threadIdx.x == 0) {
    double lg = 0.0;
    for (int i = 0; i < g.nlogs; ++i) lg += g.logs[i];
    const Acc x = v[0];
    const double mag = sqrt(abs2(x));
    g.out[0] = (mag > 0 ? log(mag) : -INFINITY) + lg;
    g.out[1] = atan2((double)im(x), (double)re(x));
  }
}

}  // namespace

void sketch_set_div(SketchDesc &s) {
  div_magic((uint64_t)s.N, &s.nmul, &s.nshr);
  for (int d = 0; d < 5; ++d) div_magic(s.radix[d] > 0 ? (uint64_t)s.radix[d] : 0, &s.rmul[d], &s.rshr[d]);
}

namespace {

template <class T>
void sketch_t(const SketchDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s) {
  if (blocks > 0) sketch_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd);
}
template <class T>
void site_t(const SiteDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s) {
  if (blocks > 0) site_kernel<T><<<(unsigned)blocks, kSiteThreads, 0, s>>>(d, prefix, nd);
}

}  // namespace

void launch_sketch(int dt, const SketchDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                   cudaStream_t s) {
  switch (dt) {
    case DT_R32: sketch_t<float>(d, prefix, nd, blocks, s); break;
    case DT_C64: sketch_t<float2>(d, prefix, nd, blocks, s); break;
    case DT_R64: sketch_t<double>(d, prefix, nd, blocks, s); break;
    case DT_C128: sketch_t<double2>(d, prefix, nd, blocks, s); break;
  }
}

namespace {
__global__ void narrow_kernel(const double *__restrict__ in, float *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}
}  // namespace

void launch_narrow(const double *in, float *out, int64_t n, cudaStream_t s) {
  if (n > 0) narrow_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(in, out, n);
}

namespace {
template <class T> __global__ void absorb_kernel(AbsorbDesc g) {
  const int64_t nu = g.M * g.k, total = nu + (int64_t)g.k * g.N;
  const double s0 = g.sigma[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nu) {
      const int c = (int)(i % g.k);
      T *u = (T *)g.U + i;
      *u = scale(*u, (typename Traits<T>::Real)(s0 > 0.0 ? g.sigma[c] / s0 : 0.0));
    } else {
      const int64_t j = i - nu;
      const int c = (int)(j / g.N);
      const double sc = g.sigma[c];
      T *w = (T *)g.W + j;
      *w = scale(*w, (typename Traits<T>::Real)(sc > 0.0 ? s0 / sc : 0.0));
    }
  }
}
}  // namespace

void launch_absorb(int dt, const AbsorbDesc &d, cudaStream_t s) {
  const int64_t total = d.M * d.k + (int64_t)d.k * d.N;
  if (total <= 0) return;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16);
  switch (dt) {
    case DT_R32: absorb_kernel<float><<<blocks, 256, 0, s>>>(d); break;
    case DT_C64: absorb_kernel<float2><<<blocks, 256, 0, s>>>(d); break;
    case DT_R64: absorb_kernel<double><<<blocks, 256, 0, s>>>(d); break;
    case DT_C128: absorb_kernel<double2><<<blocks, 256, 0, s>>>(d); break;
  }
}

void launch_pad(int dt, const PadDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s) {
  if (blocks <= 0) return;
  switch (dt) {
    case DT_R32: pad_kernel<float><<<(unsigned)blocks, kPadPerBlock, 0, s>>>(d, prefix, nd); break;
    case DT_C64: pad_kernel<float2><<<(unsigned)blocks, kPadPerBlock, 0, s>>>(d, prefix, nd); break;
    case DT_R64: pad_kernel<double><<<(unsigned)blocks, kPadPerBlock, 0, s>>>(d, prefix, nd); break;
    case DT_C128: pad_kernel<double2><<<(unsigned)blocks, kPadPerBlock, 0, s>>>(d, prefix, nd); break;
  }
}

void launch_site(int dt, const SiteDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                 cudaStream_t s) {
  switch (dt) {
    case DT_R32: site_t<float>(d, prefix, nd, blocks, s); break;
    case DT_C64: site_t<float2>(d, prefix, nd, blocks, s); break;
    case DT_R64: site_t<double>(d, prefix, nd, blocks, s); break;
    case DT_C128: site_t<double2>(d, prefix, nd, blocks, s); break;
  }
}

int64_t permute_blocks(const PermuteDesc &d) {
  return d.nb * ceil_div(d.R, 32) * ceil_div(d.Cc, 32) * d.Q;
}

void launch_permute(int dt, const PermuteDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                    cudaStream_t s) {
  if (blocks <= 0) return;
  switch (dt) {
    case DT_R32: permute_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd); break;
    case DT_C64: permute_kernel<float2><<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd); break;
    case DT_R64: permute_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd); break;
    case DT_C128: permute_kernel<double2><<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd); break;
  }
}

void launch_zero(const ZeroDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s) {
  if (blocks > 0) zero_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, prefix, nd);
}

void launch_fill(int dt, void *p, int64_t n, double value, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned blocks = (unsigned)ceil_div(n, 256);
  switch (dt) {
    case DT_R32: fill_kernel<float><<<blocks, 256, 0, s>>>((float *)p, n, value); break;
    case DT_C64: fill_kernel<float2><<<blocks, 256, 0, s>>>((float2 *)p, n, value); break;
    case DT_R64: fill_kernel<double><<<blocks, 256, 0, s>>>((double *)p, n, value); break;
    case DT_C128: fill_kernel<double2><<<blocks, 256, 0, s>>>((double2 *)p, n, value); break;
  }
}

void launch_scalar(int dt, const ScalarDesc *d, cudaStream_t s) {
  switch (dt) {
    case DT_R32: scalar_kernel<float><<<1, 256, 0, s>>>(*d); break;
    case DT_C64: scalar_kernel<float2><<<1, 256, 0, s>>>(*d); break;
    case DT_R64: scalar_kernel<double><<<1, 256, 0, s>>>(*d); break;
    case DT_C128: scalar_kernel<double2><<<1, 256, 0, s>>>(*d); break;
  }
}

}  // namespace peps
