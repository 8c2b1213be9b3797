// Small dense factorisations of one einsumsvd step (l x l, l = sketch width).
//
// Arithmetic is the data's own precision: single-precision data factorise in
// FP32, FP64 data in FP64 (GB300 runs FP64 at ~1/58 of the FP32 rate, and
// the Gram matrices these kernels start from are already accumulated with
// FP64 partial sums).  Matrices live in shared memory when they fit and in
// the caller's global scratch otherwise.
//
//  * chol: the factor of CholeskyQR (Gram-matrix orthogonalisation, the role
//    of Algorithm 5 with a Cholesky factor in place of its eigen route).
//    A relative diagonal shift may be added first (shifted CholeskyQR, so a
//    single-precision factorisation cannot break down on an ill-conditioned
//    block; a second pass restores orthogonality).  A pivot <= tol * max diag
//    marks the column as numerically inside the span of the earlier ones: its
//    row of R and column of R^+ are zero, exactly Gram-Schmidt with deletion.
//    Outputs R, T = R^+ and optionally R * Rprev (CholeskyQR2's R).
//  * jacobi: one-sided (Hestenes) Jacobi SVD of Rb^H in round-robin order,
//    one warp per column pair.  The singular values of Algorithm 4's small
//    matrix P^H A are those of Rb^H, Rb being the R factor of (P^H A)^H.
//  * finalize: sort, truncate to k, zero directions below rtol * sigma_1 and
//    fix the phase of each singular vector against a Philox vector g.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int NT = 512;
constexpr int kSmemLimit = 200 * 1024;
constexpr int kCholCTAs = 8;     // CTAs of the cluster Cholesky

// Where a Cholesky of size n runs: one CTA with the matrix in shared memory,
// a cluster holding the rows in distributed shared memory, or one CTA on the
// caller's global scratch (too large for either).
enum CholRoute { kCholSmem = 0, kCholCluster = 1, kCholGlobal = 2 };
// Shared memory of the cluster Cholesky with panels of nb rows: the CTA's
// rows of W (and T), one panel of nb rows and an nb x nb block.
__host__ __device__ inline int64_t chol_cluster_bytes_nb(int n, int es, bool needT, int nb) {
  const int64_t cap = (n + kCholCTAs - 1) / kCholCTAs;
  return ((needT ? 2 : 1) * cap * n + (int64_t)nb * n + (int64_t)nb * nb) * es;
}
// widest panel (16, 8, 4, 2 or 1 rows) that fits
__host__ __device__ inline int chol_cluster_nb(int n, int es, bool needT) {
  int nb = 16;
  while (nb > 1 && chol_cluster_bytes_nb(n, es, needT, nb) > kSmemLimit) nb >>= 1;
  return nb;
}
__host__ __device__ inline int64_t chol_cluster_bytes(int n, int es, bool needT) {
  return chol_cluster_bytes_nb(n, es, needT, chol_cluster_nb(n, es, needT));
}
__host__ __device__ inline int chol_route(int n, int es, bool needT) {
  if ((int64_t)n * n * es <= kSmemLimit) return kCholSmem;
  return chol_cluster_bytes(n, es, needT) <= kSmemLimit ? kCholCluster : kCholGlobal;
}

template <class T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 5.9604644775390625e-08; };
template <> struct Eps<float2> { static constexpr double v = 5.9604644775390625e-08; };
template <> struct Eps<double> { static constexpr double v = 1.1102230246251565e-16; };
template <> struct Eps<double2> { static constexpr double v = 1.1102230246251565e-16; };

template <class T> __device__ __forceinline__ T warp_sum(T v);
template <> __device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <> __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <> __device__ __forceinline__ float2 warp_sum(float2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
template <> __device__ __forceinline__ double2 warp_sum(double2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

__device__ double block_max(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    red[0] = m;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m += red[i];
    red[0] = m;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

template <class T> __device__ __forceinline__ T real_scalar(double x) { return from_parts<T>(x, 0.0); }

template <class T> __device__ __forceinline__ T div_real(T a, double r) {
  return scale(a, (typename Traits<T>::Real)(1.0 / r));
}

// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(NT) chol_kernel(const CholDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  __shared__ double red[32];
  __shared__ unsigned char dead[1024];
  extern __shared__ __align__(16) unsigned char dyn[];
  const CholDesc &g = descs[blockIdx.x];
  const int n = g.n;
  if (chol_route(n, (int)sizeof(T), g.T != nullptr) == kCholCluster) return;
  const Acc *G = (const Acc *)g.G;
  const bool in_smem = (int64_t)n * n * sizeof(T) <= kSmemLimit;
  T *W = in_smem ? (T *)dyn : (T *)g.R;        // working matrix; its upper triangle becomes R
  T *R = (T *)g.R;

  double md = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double gi = re(G[(int64_t)i * n + i]);
    md = fmax(md, gi);
    // a NaN / Inf diagonal would otherwise count as a dead pivot and vanish
    if (!isfinite(gi) && g.status) atomicOr(g.status, STATUS_NONFINITE);
  }
  md = block_max(md, red);
  const double shift = g.shift * md;
  for (int t = threadIdx.x; t < n * n; t += NT) {
    const int i = (int)(t / n), k = (int)(t % n);
    T v = zero<T>();
    if (k >= i) {
      v = narrow<T>(G[t]);
      if (k == i) v = from_parts<T>(re(G[t]) + shift, 0.0);
    }
    W[t] = v;
  }
  __syncthreads();
  const double thr = g.tol * md;

  // the pivot's FP64 scalars are formed once by thread 0 and read by all
  // (FP64 square roots and divisions in every thread would cost 16 warps of
  // 1/64-rate FP64 work per pivot)
  __shared__ double piv[2];
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double dj = (double)re(W[(int64_t)j * n + j]);
      const bool isdead = !(dj > thr) || !(md > 0.0);
      dead[j] = isdead;
      piv[0] = isdead ? 0.0 : sqrt(dj);
      piv[1] = isdead ? 0.0 : 1.0 / piv[0];
    }
    __syncthreads();   // the pivot's scalars are published before row j is rewritten
    if (dead[j]) {
      for (int k = j + threadIdx.x; k < n; k += NT) W[(int64_t)j * n + k] = zero<T>();
      __syncthreads();
      continue;
    }
    const double r = piv[0];
    const typename Traits<T>::Real rinv = (typename Traits<T>::Real)piv[1];
    for (int k = j + threadIdx.x; k < n; k += NT)
      W[(int64_t)j * n + k] = k == j ? real_scalar<T>(r) : scale(W[(int64_t)j * n + k], rinv);
    __syncthreads();
    // trailing update of the upper triangle: W[i][k] -= conj(R[j][i]) R[j][k], j < i <= k
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * m; t += NT) {
      const int i = j + 1 + (int)(t / m), k = j + 1 + (int)(t % m);
      if (i > k) continue;
      W[(int64_t)i * n + k] = sub(W[(int64_t)i * n + k], mul(conj_(W[(int64_t)j * n + i]), W[(int64_t)j * n + k]));
    }
    __syncthreads();
  }
  // R (upper triangle of W, zero below) to global
  if (in_smem)
    for (int t = threadIdx.x; t < n * n; t += NT) {
      const int i = (int)(t / n), k = (int)(t % n);
      R[t] = k >= i ? W[t] : zero<T>();
    }
  else
    for (int t = threadIdx.x; t < n * n; t += NT)
      if ((int)(t % n) < (int)(t / n)) R[t] = zero<T>();
  __syncthreads();

  if constexpr (sizeof(typename Traits<T>::Real) == 8) {
    if (g.Rlow) {
      for (int t = threadIdx.x; t < n * n; t += NT) {
        if constexpr (sizeof(T) == 16) ((float2 *)g.Rlow)[t] = narrow<float2>(widen(R[t]));
        else ((float *)g.Rlow)[t] = narrow<float>(widen(R[t]));
      }
    }
  }
  if (!g.T) return;

  // T = R^+ row by row from the bottom: T[i][c] = -(sum_{k=i+1..c} R[i][k] T[k][c]) / R[i][i]
  T *Tm = (T *)g.T;
  const int warps = NT / 32, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = n - 1; i >= 0; --i) {
    if (dead[i]) {
      for (int c = threadIdx.x; c < n; c += NT) Tm[(int64_t)i * n + c] = zero<T>();
      __syncthreads();
      continue;
    }
    const double rii = re(R[(int64_t)i * n + i]);
    const typename Traits<T>::Real nrinv = (typename Traits<T>::Real)(-1.0 / rii);
    for (int c = threadIdx.x; c <= i; c += NT)
      Tm[(int64_t)i * n + c] = c == i ? real_scalar<T>(1.0 / rii) : zero<T>();
    for (int c = i + 1 + w; c < n; c += warps) {
      T s = zero<T>();
      for (int k = i + 1 + lane; k <= c; k += 32) s = fma_(R[(int64_t)i * n + k], Tm[(int64_t)k * n + c], s);
      s = warp_sum(s);
      if (lane == 0) Tm[(int64_t)i * n + c] = scale(s, nrinv);
    }
    __syncthreads();
  }
  if constexpr (sizeof(typename Traits<T>::Real) == 8) {
    if (g.Tlow) {
      for (int t = threadIdx.x; t < n * n; t += NT) {
        if constexpr (sizeof(T) == 16) ((float2 *)g.Tlow)[t] = narrow<float2>(widen(Tm[t]));
        else ((float *)g.Tlow)[t] = narrow<float>(widen(Tm[t]));
      }
    }
  }
  if (g.Rprev) {
    const T *P = (const T *)g.Rprev;
    T *O = (T *)g.Rout;
    for (int t = threadIdx.x; t < n * n; t += NT) {
      const int i = (int)(t / n), k = (int)(t % n);
      T s = zero<T>();
      for (int l = i; l <= k; ++l) s = fma_(R[(int64_t)i * n + l], P[(int64_t)l * n + k], s);
      O[t] = s;
    }
  }
}

// Cluster Cholesky for l beyond one CTA's shared memory: the rows of W (then
// R) and of T = R^+ are dealt round-robin to kCholCTAs CTAs (row i on CTA
// i mod kCholCTAs), each in its own shared memory.  Blocked right-looking
// over panels of nb pivots: after one cluster barrier every CTA copies the
// panel's rows through distributed shared memory, factors the panel itself
// (the same arithmetic in every CTA, so the copies agree), and applies the
// panel to its own rows below; the owners keep the final panel rows.  R^+ is
// formed the same way from the last panel up (a row of T is final once every
// later row has been added into it).  Each element receives its updates in
// the pivot order of the unblocked algorithm.  Same outputs and pivot rule as
// chol_kernel.
template <class T>
__global__ void __cluster_dims__(kCholCTAs, 1, 1) __launch_bounds__(NT)
    chol_cluster_kernel(const CholDesc *__restrict__ descs) {
  namespace cg = cooperative_groups;
  using Acc = typename Traits<T>::Acc;
  using Real = typename Traits<T>::Real;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const CholDesc &g = descs[blockIdx.x / kCholCTAs];
  const int n = g.n;
  const bool needT = g.T != nullptr;
  if (chol_route(n, (int)sizeof(T), needT) != kCholCluster) return;   // uniform over the cluster
  const int nb = chol_cluster_nb(n, (int)sizeof(T), needT);
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[32];
  __shared__ double piv[2];
  const int cap = (n + kCholCTAs - 1) / kCholCTAs;
  const int nloc = rank < n ? (n - rank + kCholCTAs - 1) / kCholCTAs : 0;   // rows rank + kCholCTAs * li
  T *Wl = (T *)dyn;
  T *Tl = Wl + (int64_t)cap * n;
  T *P = Tl + (needT ? (int64_t)cap * n : 0);    // nb panel rows, full width
  T *B = P + (int64_t)nb * n;                     // nb x nb block of R (inverse phase)
  const Acc *G = (const Acc *)g.G;
  // first local row index with global row >= r
  auto first_li = [&](int r) { return r - rank <= 0 ? 0 : (r - rank + kCholCTAs - 1) / kCholCTAs; };

  double md = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double gi = re(G[(int64_t)i * n + i]);
    md = fmax(md, gi);
    // a NaN / Inf diagonal would otherwise count as a dead pivot and vanish
    if (!isfinite(gi) && g.status) atomicOr(g.status, STATUS_NONFINITE);
  }
  md = block_max(md, red);
  const double shift = g.shift * md, thr = g.tol * md;
  for (int t = threadIdx.x; t < nloc * n; t += NT) {
    const int li = (int)(t / n), k = (int)(t % n), i = rank + kCholCTAs * li;
    T v = zero<T>();
    if (k >= i) {
      const Acc a = G[(int64_t)i * n + k];
      v = k == i ? from_parts<T>(re(a) + shift, 0.0) : narrow<T>(a);
    }
    Wl[t] = v;
    if (needT) Tl[t] = zero<T>();
  }

  // panel rows of this CTA back into its rows (after every CTA has copied the panel)
  auto keep_panel = [&](T *dst, int j0, int jb, int c0) {
    for (int p = 0; p < jb; ++p) {
      const int j = j0 + p;
      if (j % kCholCTAs != rank) continue;
      T *row = dst + (int64_t)(j / kCholCTAs) * n;
      for (int k = c0 + threadIdx.x; k < n; k += NT) row[k] = P[(int64_t)p * n + k];
    }
  };

  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = min(nb, n - j0);
    cluster.sync();                    // earlier panels applied everywhere and copied by everyone
    if (j0 > 0) keep_panel(Wl, j0 - nb, nb, j0 - nb);
    __syncthreads();                   // the panel buffer is read out
    const int w = n - j0;
    for (int t = threadIdx.x; t < jb * w; t += NT) {
      const int p = (int)(t / w), k = j0 + (int)(t % w), j = j0 + p;
      P[(int64_t)p * n + k] = cluster.map_shared_rank(Wl, j % kCholCTAs)[(int64_t)(j / kCholCTAs) * n + k];
    }
    __syncthreads();
    for (int p = 0; p < jb; ++p) {
      const int j = j0 + p;
      T *row = P + (int64_t)p * n;
      // the pivot's FP64 scalars, formed once by thread 0 and read by all
      if (threadIdx.x == 0) {
        const double dj = re(row[j]);
        const bool dead = !(dj > thr) || !(md > 0.0);
        piv[0] = dead ? -1.0 : sqrt(dj);
        piv[1] = dead ? 0.0 : 1.0 / piv[0];
      }
      __syncthreads();                 // the scalars are published before the row changes
      const bool dead = piv[0] < 0.0;
      if (dead) {
        for (int k = j + threadIdx.x; k < n; k += NT) row[k] = zero<T>();
      } else {
        const double r = piv[0];
        const Real rinv = (Real)piv[1];
        for (int k = j + threadIdx.x; k < n; k += NT) row[k] = k == j ? real_scalar<T>(r) : scale(row[k], rinv);
      }
      __syncthreads();
      // later rows of the panel: W[i][k] -= conj(R[j][i]) R[j][k], k >= i
      const int rem = jb - p - 1;
      for (int t = threadIdx.x; t < rem * w; t += NT) {
        const int pp = p + 1 + (int)(t / w), k = j0 + (int)(t % w), i = j0 + pp;
        if (k < i) continue;
        T *x = P + (int64_t)pp * n + k;
        *x = sub(*x, mul(conj_(row[i]), row[k]));
      }
      __syncthreads();
    }
    // this CTA's rows below the panel
    const int li0 = first_li(j0 + jb);
    for (int t = threadIdx.x; t < (nloc - li0) * n; t += NT) {
      const int li = li0 + (int)(t / n), k = (int)(t % n), i = rank + kCholCTAs * li;
      if (k < i) continue;
      T x = Wl[(int64_t)li * n + k];
      for (int p = 0; p < jb; ++p) x = sub(x, mul(conj_(P[(int64_t)p * n + i]), P[(int64_t)p * n + k]));
      Wl[(int64_t)li * n + k] = x;
    }
  }
  cluster.sync();                      // the last panel copied by everyone
  {
    const int j0 = ((n - 1) / nb) * nb;
    keep_panel(Wl, j0, n - j0, j0);
  }

  if (needT) {
    cluster.sync();                    // every row of R final
    // panels of rows [k0, k0 + kb) from the bottom; Tl rows hold
    // sum_{l > i, l done} R[i][l] T[l][c] until row i is finalised
    int prev0 = -1, prevb = 0;
    for (int k1 = n; k1 > 0; k1 -= nb) {
      const int k0 = max(0, k1 - nb), kb = k1 - k0;
      if (prev0 >= 0) {
        cluster.sync();                // previous panel applied everywhere and copied by everyone
        keep_panel(Tl, prev0, prevb, prev0);
        __syncthreads();               // the panel buffer is read out
      }
      const int w = n - k0;
      for (int t = threadIdx.x; t < kb * w; t += NT) {
        const int p = (int)(t / w), c = k0 + (int)(t % w), k = k0 + p;
        const int64_t o = (int64_t)(k / kCholCTAs) * n;
        P[(int64_t)p * n + c] = cluster.map_shared_rank(Tl, k % kCholCTAs)[o + c];
        if (c < k1) B[p * nb + (c - k0)] = cluster.map_shared_rank(Wl, k % kCholCTAs)[o + c];
      }
      __syncthreads();
      for (int p = kb - 1; p >= 0; --p) {
        const int k = k0 + p;
        T *trow = P + (int64_t)p * n;
        const double rkk = re(B[p * nb + p]);
        if (rkk == 0.0) {
          for (int c = k + threadIdx.x; c < n; c += NT) trow[c] = zero<T>();
        } else {
          const Real ninv = (Real)(-1.0 / rkk);
          for (int c = k + threadIdx.x; c < n; c += NT) trow[c] = c == k ? real_scalar<T>(1.0 / rkk) : scale(trow[c], ninv);
        }
        __syncthreads();
        // earlier rows of the panel: T[i][c] += R[i][k] T[k][c], c >= k
        const int m = n - k;
        for (int t = threadIdx.x; t < p * m; t += NT) {
          const int pi = (int)(t / m), c = k + (int)(t % m);
          T *x = P + (int64_t)pi * n + c;
          *x = fma_(B[pi * nb + p], trow[c], *x);
        }
        __syncthreads();
      }
      // this CTA's rows above the panel
      const int li1 = first_li(k0);    // rows i < k0: local indices below li1
      for (int t = threadIdx.x; t < li1 * w; t += NT) {
        const int li = (int)(t / w), c = k0 + (int)(t % w);
        T x = Tl[(int64_t)li * n + c];
        for (int p = kb - 1; p >= 0; --p) {
          const int k = k0 + p;
          if (c >= k) x = fma_(Wl[(int64_t)li * n + k], P[(int64_t)p * n + c], x);
        }
        Tl[(int64_t)li * n + c] = x;
      }
      prev0 = k0;
      prevb = kb;
    }
    cluster.sync();
    keep_panel(Tl, prev0, prevb, prev0);
  }
  __syncthreads();

  // outputs: R (upper, zero below), T, R * Rprev, R in single precision
  T *R = (T *)g.R;
  T *Tg = (T *)g.T;
  for (int t = threadIdx.x; t < nloc * n; t += NT) {
    const int li = (int)(t / n), k = (int)(t % n), i = rank + kCholCTAs * li;
    const int64_t o = (int64_t)i * n + k;
    R[o] = Wl[t];
    if (needT) Tg[o] = Tl[t];
    if constexpr (sizeof(Real) == 8) {
      if (g.Rlow) {
        if constexpr (sizeof(T) == 16) ((float2 *)g.Rlow)[o] = narrow<float2>(widen(Wl[t]));
        else ((float *)g.Rlow)[o] = narrow<float>(widen(Wl[t]));
      }
      if (needT && g.Tlow) {
        if constexpr (sizeof(T) == 16) ((float2 *)g.Tlow)[o] = narrow<float2>(widen(Tl[t]));
        else ((float *)g.Tlow)[o] = narrow<float>(widen(Tl[t]));
      }
    }
    if (g.Rprev) {
      const T *Rp = (const T *)g.Rprev;
      T sacc = zero<T>();
      for (int l = i; l <= k; ++l) sacc = fma_(Wl[(int64_t)li * n + l], Rp[(int64_t)l * n + k], sacc);
      ((T *)g.Rout)[o] = sacc;
    }
  }
  cluster.sync();   // peers may still read this CTA's shared memory until here
}

// Hestenes rotation of columns a, b (length n) in place.  Rotates when
// |a^H b| > tol |a| |b|; returns that relative off-diagonal measure.  The
// rotation scalars use the data's own precision (FP64 divide / square root
// run at a small fraction of the FP32 rate on this GPU).
template <class T>
__device__ __forceinline__ float jacobi_rotate_params(typename Traits<T>::Real al, typename Traits<T>::Real be, T ga,
                                                      float tol, typename Traits<T>::Real &c,
                                                      typename Traits<T>::Real &sn, T &ph, bool &rot) {
  using R = typename Traits<T>::Real;
  const R gm = sqrt(abs2(ga));
  const R nrm = sqrt(al * be);
  const float rel = nrm > (R)0 ? (float)(gm / nrm) : 0.f;
  rot = gm > (R)tol * nrm && gm != (R)0;
  if (!rot) return rel;
  const R zeta = (be - al) / ((R)2 * gm);
  const R t = (zeta >= (R)0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
  c = (R)1 / sqrt((R)1 + t * t);
  sn = c * t;
  // e^{-i phi} with gamma = |gamma| e^{i phi}
  if constexpr (Traits<T>::cplx) ph = from_parts<T>(re(ga) / gm, -im(ga) / gm);
  else ph = re(ga) > (R)0 ? (R)1 : (R)-1;
  return rel;
}

// kRegs: columns of up to 32 * kRegs rows stay in registers
template <class T, int kRegs = (sizeof(T) <= 8 ? 16 : 8)>
__device__ float jacobi_pair(T *a, T *b, int n, float tol) {
  using R = typename Traits<T>::Real;
  const int lane = threadIdx.x & 31;
  R al = 0, be = 0;
  T ga = zero<T>();
  R c = 0, sn = 0;
  T ph = zero<T>();
  bool rot = false;
  float rel;
  if (n <= 32 * kRegs) {
    // both columns read once (all loads issued back to back), rotated in registers
    T x[kRegs], y[kRegs];
#pragma unroll
    for (int i = 0; i < kRegs; ++i) {
      const int r = lane + 32 * i;
      x[i] = r < n ? a[r] : zero<T>();
      y[i] = r < n ? b[r] : zero<T>();
    }
#pragma unroll
    for (int i = 0; i < kRegs; ++i) {
      al += abs2(x[i]);
      be += abs2(y[i]);
      ga = fma_(conj_(x[i]), y[i], ga);
    }
    al = warp_sum(al);
    be = warp_sum(be);
    ga = warp_sum(ga);
    rel = jacobi_rotate_params<T>(al, be, ga, tol, c, sn, ph, rot);
    if (!rot) return rel;
#pragma unroll
    for (int i = 0; i < kRegs; ++i) {
      const int r = lane + 32 * i;
      if (r < n) {
        const T yy = mul(y[i], ph);
        a[r] = sub(scale(x[i], c), scale(yy, sn));
        b[r] = add(scale(x[i], sn), scale(yy, c));
      }
    }
    return rel;
  }
  for (int r = lane; r < n; r += 32) {
    const T x = a[r], y = b[r];
    al += abs2(x);
    be += abs2(y);
    ga = fma_(conj_(x), y, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  rel = jacobi_rotate_params<T>(al, be, ga, tol, c, sn, ph, rot);
  if (!rot) return rel;
  for (int r = lane; r < n; r += 32) {
    const T x = a[r];
    const T y = mul(b[r], ph);
    a[r] = sub(scale(x, c), scale(y, sn));
    b[r] = add(scale(x, sn), scale(y, c));
  }
  return rel;
}

template <class T>
__global__ void __launch_bounds__(NT) jacobi_kernel(const JacobiDesc *__restrict__ descs) {
  __shared__ float sweep_max;
  extern __shared__ __align__(16) unsigned char dyn[];
  const JacobiDesc &g = descs[blockIdx.x];
  const int n = g.n;
  const bool in_smem = (int64_t)n * n * sizeof(T) <= kSmemLimit;
  if (!in_smem) return;                                      // cluster kernel
  const T *Rb = (const T *)g.Rb;
  T *Mg = (T *)g.Mw;
  T *M = in_smem ? (T *)dyn : Mg;
  // column c of Rb^H = conj(row c of Rb)
  for (int t = threadIdx.x; t < n * n; t += NT) M[t] = conj_(Rb[t]);
  __syncthreads();
  const int n2 = n + (n & 1);
  const int warps = NT / 32, w = threadIdx.x >> 5;
  // rotate above the rounding level of the dot products; stop once a whole
  // sweep found nothing above a few times that level
  const double tol = 2.0 * sqrt((double)n) * Eps<T>::v;
  const double stop_tol = 8.0 * tol;
  int sweep = 0;
  for (; sweep < g.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) sweep_max = 0.f;
    __syncthreads();
    float mine = 0.f;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int i = w; i < n2 / 2; i += warps) {
        int a, b;
        if (i == 0) { a = r; b = n2 - 1; }
        else { a = (r + i) % (n2 - 1); b = (r - i + (n2 - 1)) % (n2 - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= n) continue;
        mine = fmaxf(mine, jacobi_pair(M + (int64_t)a * n, M + (int64_t)b * n, n, (float)tol));
      }
      __syncthreads();
    }
    if ((threadIdx.x & 31) == 0) atomicMax((int *)&sweep_max, __float_as_int(mine));
    __syncthreads();
    const bool done = sweep_max <= (float)stop_tol;
    __syncthreads();
    if (done) break;
  }
  if (sweep == g.max_sweeps && threadIdx.x == 0 && g.status) atomicOr(g.status, STATUS_JACOBI_NOCONV);
  for (int c = w; c < n; c += warps) {
    double s2 = 0.0;
    for (int r = threadIdx.x & 31; r < n; r += 32) s2 += (double)abs2(M[(int64_t)c * n + r]);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) g.sig[c] = sqrt(s2);
  }
  if (in_smem)
    for (int t = threadIdx.x; t < n * n; t += NT) Mg[t] = M[t];
}


// One-sided Jacobi on a thread-block cluster: for l x l matrices too large for
// one SM's shared memory, eight CTAs hold the columns in distributed shared
// memory and all column pairs of a round-robin round rotate in parallel (one
// warp per pair, any CTA reaching any column through the cluster window),
// with a cluster barrier between rounds (for l whose four column blocks do
// not fit the block-cyclic kernel below).  18 warps per CTA: the 144 warps of
// the cluster take every pair of a round at once up to l = 288, with columns
// of up to 288 rows (160 in FP64 complex) held in registers.
constexpr int kClusterCTAs = 8;
constexpr int NTJ = 576;
template <class T> __host__ __device__ constexpr int jacobi_regs() { return sizeof(T) <= 8 ? 9 : 5; }
// column blocks of the block-cyclic cluster Jacobi (below)
constexpr int kJB = 2 * kClusterCTAs;
__host__ __device__ inline int jacobi_bs(int n) { return (n + kJB - 1) / kJB; }
__host__ __device__ inline int64_t jacobi_block_bytes(int n, int es) { return 4LL * jacobi_bs(n) * n * es; }
// 0: one CTA; 1: block-cyclic cluster; 2: column-window cluster
__host__ __device__ inline int jacobi_route(int n, int es) {
  if ((int64_t)n * n * es <= kSmemLimit) return 0;
  return jacobi_block_bytes(n, es) <= kSmemLimit ? 1 : 2;
}

template <class T>
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(NTJ)
    jacobi_cluster_kernel(const JacobiDesc *__restrict__ descs) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const JacobiDesc &g = descs[blockIdx.x / kClusterCTAs];
  const int n = g.n;
  if (jacobi_route(n, (int)sizeof(T)) != 2) return;         // one CTA, or the block-cyclic kernel
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ float cta_max;
  __shared__ float cluster_max;
  T *local = (T *)dyn;
  const int cpc = (n + kClusterCTAs - 1) / kClusterCTAs;     // columns per CTA
  const T *Rb = (const T *)g.Rb;
  for (int t = threadIdx.x; t < cpc * n; t += NTJ) {
    const int lc = (int)(t / n), r = (int)(t % n), c = rank * cpc + lc;
    local[t] = c < n ? conj_(Rb[(int64_t)c * n + r]) : zero<T>();
  }
  if (threadIdx.x == 0) cluster_max = 0.f;
  cluster.sync();
  auto col = [&](int c) -> T * {
    T *base = cluster.map_shared_rank(local, c / cpc);
    return base + (int64_t)(c % cpc) * n;
  };
  const int n2 = n + (n & 1);
  const int lane = threadIdx.x & 31;
  const int gw = rank * (NTJ / 32) + (threadIdx.x >> 5), nwarps = kClusterCTAs * NTJ / 32;
  const double tol = 2.0 * sqrt((double)n) * Eps<T>::v;
  const double stop_tol = 8.0 * tol;
  float *root_max = cluster.map_shared_rank(&cluster_max, 0);
  int sweep = 0;
  for (; sweep < g.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) cta_max = 0.f;
    __syncthreads();
    float mine = 0.f;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int i = gw; i < n2 / 2; i += nwarps) {
        int a, b;
        if (i == 0) { a = r; b = n2 - 1; }
        else { a = (r + i) % (n2 - 1); b = (r - i + (n2 - 1)) % (n2 - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= n) continue;
        mine = fmaxf(mine, jacobi_pair<T, jacobi_regs<T>()>(col(a), col(b), n, (float)tol));
      }
      cluster.sync();
    }
    if (lane == 0) atomicMax((int *)&cta_max, __float_as_int(mine));
    __syncthreads();
    if (threadIdx.x == 0) atomicMax((int *)root_max, __float_as_int(cta_max));
    cluster.sync();
    const bool done = *root_max <= (float)stop_tol;
    cluster.sync();                                          // all read before the reset
    if (rank == 0 && threadIdx.x == 0) cluster_max = 0.f;
    cluster.sync();
    if (done) break;
  }
  if (sweep == g.max_sweeps && rank == 0 && threadIdx.x == 0 && g.status)
    atomicOr(g.status, STATUS_JACOBI_NOCONV);
  T *Mg = (T *)g.Mw;
  const int w = threadIdx.x >> 5;
  for (int lc = w; lc < cpc; lc += NTJ / 32) {
    const int c = rank * cpc + lc;
    if (c >= n) break;
    double s2 = 0.0;
    for (int r = lane; r < n; r += 32) {
      const T v = local[(int64_t)lc * n + r];
      Mg[(int64_t)c * n + r] = v;
      s2 += (double)abs2(v);
    }
    s2 = warp_sum(s2);
    if (lane == 0) g.sig[c] = sqrt(s2);
  }
  cluster.sync();   // keep this CTA's shared memory alive until every peer is done with it
}

// Block-cyclic one-sided Jacobi on a cluster: the l columns form 16 blocks;
// each CTA holds two of them in its own shared memory and rotates all pairs
// between (and once per sweep within) its two blocks with block-level
// synchronisation only; between these stages the blocks move to other CTAs
// on a round-robin tournament (block position p >= 1 goes to p + 1, 15 wraps
// to 1), so that after 15 moves every pair of blocks has met once and each
// block is back home.  One cluster barrier per move instead of one per
// round, and column data crosses the cluster only when blocks move.

template <class T>
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(NTJ)
    jacobi_block_kernel(const JacobiDesc *__restrict__ descs) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const JacobiDesc &g = descs[blockIdx.x / kClusterCTAs];
  const int n = g.n;
  if (jacobi_route(n, (int)sizeof(T)) != 1) return;          // uniform over the cluster
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ float cta_max;
  __shared__ float cluster_max;
  const int bs = jacobi_bs(n);
  const int64_t bsz = (int64_t)bs * n;                       // elements of one block
  T *const set0 = (T *)dyn, *const set1 = (T *)dyn + 2 * bsz; // current and next (two slots each)
  const int pos0 = rank, pos1 = kJB - 1 - rank;               // tournament positions of the two slots
  // block at position p after s moves (block b starts at position b)
  auto block_at = [&](int p, int s) { return p == 0 ? 0 : 1 + ((p - 1 - s) % (kJB - 1) + (kJB - 1)) % (kJB - 1); };
  auto valid = [&](int b) { return max(0, min(bs, n - b * bs)); };
  const T *Rb = (const T *)g.Rb;
  T *cs = set0;
  for (int sl = 0; sl < 2; ++sl)
    for (int t = threadIdx.x; t < (int)bsz; t += NTJ) {
      const int j = (int)(t / n), r = (int)(t % n), c = (sl ? pos1 : pos0) * bs + j;
      cs[sl * bsz + t] = c < n ? conj_(Rb[(int64_t)c * n + r]) : zero<T>();
    }
  if (threadIdx.x == 0) cluster_max = 0.f;
  cluster.sync();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nw = NTJ / 32;
  const double tol = 2.0 * sqrt((double)n) * Eps<T>::v;
  const double stop_tol = 8.0 * tol;
  float *root_max = cluster.map_shared_rank(&cluster_max, 0);
  int sweep = 0;
  for (; sweep < g.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) cta_max = 0.f;
    __syncthreads();
    float mine = 0.f;
    {
      // pairs within each of the two blocks (round robin, a dummy player for odd sizes)
      const int bsp = bs + (bs & 1), ppr = bsp / 2;
      const int nva = valid(block_at(pos0, 0)), nvb = valid(block_at(pos1, 0));
      for (int rr = 0; rr < bsp - 1; ++rr) {
        for (int i = w; i < 2 * ppr; i += nw) {
          const int sl = i / ppr, k = i % ppr;
          int a, b;
          if (k == 0) { a = rr; b = bsp - 1; }
          else { a = (rr + k) % (bsp - 1); b = (rr - k + bsp - 1) % (bsp - 1); }
          if (a > b) { const int t = a; a = b; b = t; }
          if (b >= (sl ? nvb : nva)) continue;
          T *base = cs + sl * bsz;
          mine = fmaxf(mine, jacobi_pair<T, jacobi_regs<T>()>(base + (int64_t)a * n, base + (int64_t)b * n, n,
                                                               (float)tol));
        }
        __syncthreads();
      }
    }
    for (int s = 0; s < kJB - 1; ++s) {
      // every pair between the two blocks: bs rounds of bs disjoint pairs
      const int nv0 = valid(block_at(pos0, s)), nv1 = valid(block_at(pos1, s));
      for (int t = 0; t < bs; ++t) {
        for (int i = w; i < bs; i += nw) {
          const int b = (i + t) % bs;
          if (i >= nv0 || b >= nv1) continue;
          mine = fmaxf(mine, jacobi_pair<T, jacobi_regs<T>()>(cs + (int64_t)i * n, cs + bsz + (int64_t)b * n, n,
                                                               (float)tol));
        }
        __syncthreads();
      }
      // move: pull the blocks of the next positions into the other set
      cluster.sync();                                        // every CTA is done with its current blocks
      T *nx = cs == set0 ? set1 : set0;
      const T *src0 = rank == 0   ? cs
                      : rank == 1 ? cluster.map_shared_rank(cs, 0) + bsz
                                  : cluster.map_shared_rank(cs, rank - 1);
      const T *src1 = rank <= kClusterCTAs - 2 ? cluster.map_shared_rank(cs, rank + 1) + bsz
                                               : cluster.map_shared_rank(cs, kClusterCTAs - 1);
      for (int t = threadIdx.x; t < (int)bsz; t += NTJ) {
        nx[t] = src0[t];
        nx[bsz + t] = src1[t];
      }
      cs = nx;
      __syncthreads();
    }
    if (lane == 0) atomicMax((int *)&cta_max, __float_as_int(mine));
    __syncthreads();
    if (threadIdx.x == 0) atomicMax((int *)root_max, __float_as_int(cta_max));
    cluster.sync();
    const bool done = *root_max <= (float)stop_tol;
    cluster.sync();                                          // all read before the reset
    if (rank == 0 && threadIdx.x == 0) cluster_max = 0.f;
    cluster.sync();
    if (done) break;
  }
  if (sweep == g.max_sweeps && rank == 0 && threadIdx.x == 0 && g.status)
    atomicOr(g.status, STATUS_JACOBI_NOCONV);
  // every block is home again: slot 0 holds block pos0, slot 1 block pos1
  T *Mg = (T *)g.Mw;
  for (int i = w; i < 2 * bs; i += nw) {
    const int sl = i / bs, j = i % bs, c = (sl ? pos1 : pos0) * bs + j;
    if (c >= n) continue;
    const T *col = cs + sl * bsz + (int64_t)j * n;
    double s2 = 0.0;
    for (int r = lane; r < n; r += 32) {
      const T v = col[r];
      Mg[(int64_t)c * n + r] = v;
      s2 += (double)abs2(v);
    }
    s2 = warp_sum(s2);
    if (lane == 0) g.sig[c] = sqrt(s2);
  }
  cluster.sync();   // keep this CTA's shared memory alive until every peer is done with it
}

// Singular values recomputed from the converged directions.  With Mw = Rb^H
// rotated to Mw J = [sigma_c u_c] (J unitary), Rb u_c = sigma_c j_c, so
// sigma_c = |Rb u_c| for the unit column u_c.  Each rotation's rounding
// (cosine and sine not exactly on the unit circle, a phase of modulus
// 1 + O(eps)) scales the columns it touches, and over the ~n rotations per
// sweep per column that drift reaches ~n eps relative; the product with the
// unrotated upper-triangular Rb, summed in FP64, carries Rb's rounding only.
// One CTA per column; its warps take rows round-robin.
template <class T>
__global__ void __launch_bounds__(NT) sigma_refine_kernel(const JacobiDesc *__restrict__ descs, int cols) {
  using Acc = typename Traits<T>::Acc;
  __shared__ double red[32];
  const JacobiDesc &g = descs[blockIdx.x / cols];
  const int n = g.n;
  const int c = blockIdx.x % cols;
  if (c >= n) return;                              // uniform over the CTA
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T *m = (const T *)g.Mw + (int64_t)c * n;
  const T *Rb = (const T *)g.Rb;
  double s2 = 0.0;
  for (int k = threadIdx.x; k < n; k += NT) s2 += (double)abs2(m[k]);
  s2 = block_sum(s2, red);
  double v2 = 0.0;
  if (s2 > 0.0) {
    for (int i = w; i < n; i += NT / 32) {
      Acc d = zero<Acc>();
      for (int k = i + lane; k < n; k += 32) d = fma_(widen(Rb[(int64_t)i * n + k]), widen(m[k]), d);
      d = warp_sum(d);
      v2 += abs2(d);                               // identical in every lane
    }
  }
  if (lane != 0) v2 = 0.0;
  v2 = block_sum(v2, red);
  if (threadIdx.x == 0) g.sig[c] = s2 > 0.0 ? sqrt(v2 / s2) : 0.0;
}

// Gauge projections h_j = sum_m conj(P[j][m]) g[m] (P = the M-side basis,
// g = the Philox gauge vector): one CTA per j, products exact and sums in
// FP64 (the gauge phase fixes the next step's sketch, so h carries only P's
// own rounding), partial sums in a fixed order.
template <class T>
__global__ void __launch_bounds__(NT) gauge_h_kernel(const FinalizeDesc *__restrict__ descs, int cols) {
  using Acc = typename Traits<T>::Acc;
  __shared__ Acc part[NT / 32];
  const FinalizeDesc &g = descs[blockIdx.x / cols];
  const int j = blockIdx.x % cols;
  if (j >= g.n) return;                            // uniform over the CTA
  const T *P = (const T *)g.P + (int64_t)j * g.M;
  const T *gv = (const T *)g.g;
  Acc acc = zero<Acc>();
  for (int64_t m = threadIdx.x; m < g.M; m += NT) acc = fma_(conj_(widen(P[m])), widen(gv[m]), acc);
  acc = warp_sum(acc);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[w] = acc;
  __syncthreads();
  if (w == 0) {
    Acc v = lane < NT / 32 ? part[lane] : zero<Acc>();
    v = warp_sum(v);
    if (lane == 0) ((Acc *)g.h)[j] = v;
  }
}

template <class T>
__global__ void __launch_bounds__(NT) finalize_kernel(const FinalizeDesc *__restrict__ descs) {
  const FinalizeDesc &g = descs[blockIdx.x];
  const int n = g.n, k = g.k;
  extern __shared__ __align__(16) unsigned char dyn[];
  using Acc = typename Traits<T>::Acc;
  int *order = (int *)dyn;                                   // n
  Acc *h = (Acc *)(dyn + ((n * sizeof(int) + 15) & ~15));    // n
  T *rho = (T *)(h + n);                                     // k
  const double *sig = g.sig;
  const T *M = (const T *)g.Mw;
  for (int c = threadIdx.x; c < n; c += NT) {
    int rank = 0;
    const double sc = sig[c];
    for (int c2 = 0; c2 < n; ++c2) {
      const double s2 = sig[c2];
      rank += (s2 > sc) || (s2 == sc && c2 < c);
    }
    order[rank] = c;
  }
  // h_j = sum_m conj(P[j][m]) g[m], formed by gauge_h_kernel
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < n; j += NT) h[j] = ((const Acc *)g.h)[j];
  __syncthreads();
  const double s1 = sig[order[0]];
  // phi_i = sum_j conj(h_j) u_{j,i}, u_i = M[:, order[i]] / sigma_i
  for (int i = w; i < k; i += NT / 32) {
    const int c = order[i];
    const double si = sig[c];
    const bool zero_dir = !(si > g.rtol * s1);
    Acc s = zero<Acc>();
    double nrm2 = 0.0;
    if (!zero_dir)
      for (int j = lane; j < n; j += 32) {
        const T mv = M[(int64_t)c * n + j];
        s = fma_(conj_(h[j]), widen(mv), s);
        nrm2 += (double)abs2(mv);
      }
    s = warp_sum(s);
    nrm2 = warp_sum(nrm2);
    if (lane == 0) {
      T r;
      const double mag = sqrt((double)abs2(s));
      if constexpr (Traits<T>::cplx)
        r = mag > 0 ? from_parts<T>(re(s) / mag, im(s) / mag) : from_parts<T>(1.0, 0.0);
      else
        r = re(s) < 0 ? from_parts<T>(-1.0, 0.0) : from_parts<T>(1.0, 0.0);
      // coefficient of column c of Mw in Ut: the phase over the column's own
      // norm (the rotated column's length, not the refined sigma), so u_i is
      // a unit vector; zero for dropped directions
      rho[i] = zero_dir || !(nrm2 > 0.0) ? zero<T>() : div_real(conj_(r), sqrt(nrm2));
      g.sigma_out[i] = zero_dir ? 0.0 : si;
    }
  }
  __syncthreads();
  T *Ut = (T *)g.Ut;
  for (int t = threadIdx.x; t < n * k; t += NT) {
    const int j = (int)(t / k), i = (int)(t % k);
    Ut[t] = mul(M[(int64_t)order[i] * n + j], rho[i]);
  }
  if (threadIdx.x == 0) {
    *g.log_out = s1 > 0 ? log(s1) : -INFINITY;
    *g.inv_s1 = s1 > 0 ? 1.0 / s1 : 1.0;
    if (!isfinite(s1) && g.status) atomicOr(g.status, STATUS_NONFINITE);
  }
}

template <class K> void set_smem(K kernel, int bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class T> void chol_t(const CholDesc *d, int nd, int smem, int cluster_smem, cudaStream_t s) {
  static bool set = false;
  if (!set) {
    set_smem(chol_kernel<T>, kSmemLimit);
    set_smem(chol_cluster_kernel<T>, kSmemLimit);
    set = true;
  }
  chol_kernel<T><<<nd, NT, smem, s>>>(d);
  if (cluster_smem > 0) chol_cluster_kernel<T><<<nd * kCholCTAs, NT, cluster_smem, s>>>(d);
}
template <class T>
void jacobi_t(const JacobiDesc *d, int nd, int smem, int block_smem, int cluster_smem, int nmax, cudaStream_t s) {
  static bool set = false;
  if (!set) {
    set_smem(jacobi_kernel<T>, kSmemLimit);
    set_smem(jacobi_block_kernel<T>, kSmemLimit);
    set_smem(jacobi_cluster_kernel<T>, kSmemLimit);
    set = true;
  }
  if (smem >= 0) jacobi_kernel<T><<<nd, NT, smem, s>>>(d);
  if (block_smem > 0) jacobi_block_kernel<T><<<nd * kClusterCTAs, NTJ, block_smem, s>>>(d);
  if (cluster_smem > 0) jacobi_cluster_kernel<T><<<nd * kClusterCTAs, NTJ, cluster_smem, s>>>(d);
  if (nmax > 0) sigma_refine_kernel<T><<<nd * nmax, NT, 0, s>>>(d, nmax);
}
template <class T> void finalize_t(const FinalizeDesc *d, int nd, int nmax, cudaStream_t s) {
  // order (n ints) + h (n, FP64) + rho (k <= n): n <= 1024
  const int smem = 4096 + 16 + 1024 * (int)(sizeof(typename Traits<T>::Acc) + sizeof(T));
  static bool set = false;
  if (!set) { set_smem(finalize_kernel<T>, smem); set = true; }
  if (nmax > 0) gauge_h_kernel<T><<<nd * nmax, NT, 0, s>>>(d, nmax);
  finalize_kernel<T><<<nd, NT, smem, s>>>(d);
}

}  // namespace

int small_smem_bytes(int dt, int n) {
  const int64_t b = (int64_t)n * n * dtype_size(dt);
  return b <= kSmemLimit ? (int)b : 0;
}

int jacobi_block_smem_bytes(int dt, int n) {
  return jacobi_route(n, dtype_size(dt)) == 1 ? (int)jacobi_block_bytes(n, dtype_size(dt)) : 0;
}

int jacobi_cluster_smem_bytes(int dt, int n) {
  if (jacobi_route(n, dtype_size(dt)) != 2) return 0;
  const int64_t cpc = (n + kClusterCTAs - 1) / kClusterCTAs;
  return (int)(cpc * n * dtype_size(dt));
}

int chol_cluster_smem_bytes(int dt, int n, bool needT) {
  return chol_route(n, dtype_size(dt), needT) == kCholCluster ? (int)chol_cluster_bytes(n, dtype_size(dt), needT)
                                                              : 0;
}

void launch_chol(int dt, const CholDesc *d, int nd, int smem, int cluster_smem, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: chol_t<float>(d, nd, smem, cluster_smem, s); break;
    case DT_C64: chol_t<float2>(d, nd, smem, cluster_smem, s); break;
    case DT_R64: chol_t<double>(d, nd, smem, cluster_smem, s); break;
    case DT_C128: chol_t<double2>(d, nd, smem, cluster_smem, s); break;
  }
}

void launch_jacobi(int dt, const JacobiDesc *d, int nd, int smem, int block_smem, int cluster_smem, int nmax,
                   cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: jacobi_t<float>(d, nd, smem, block_smem, cluster_smem, nmax, s); break;
    case DT_C64: jacobi_t<float2>(d, nd, smem, block_smem, cluster_smem, nmax, s); break;
    case DT_R64: jacobi_t<double>(d, nd, smem, block_smem, cluster_smem, nmax, s); break;
    case DT_C128: jacobi_t<double2>(d, nd, smem, block_smem, cluster_smem, nmax, s); break;
  }
}

void launch_finalize(int dt, const FinalizeDesc *d, int nd, int nmax, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: finalize_t<float>(d, nd, nmax, s); break;
    case DT_C64: finalize_t<float2>(d, nd, nmax, s); break;
    case DT_R64: finalize_t<double>(d, nd, nmax, s); break;
    case DT_C128: finalize_t<double2>(d, nd, nmax, s); break;
  }
}

}  // namespace peps
