// Small dense factorisations of one einsumsvd step, in FP64.
//
//  * chol: CholeskyQR's factor of a Gram matrix G = Y^H Y (the Gram-matrix
//    orthogonalisation of Algorithm 5, with a Cholesky factor in place of
//    its eigendecomposition).  A pivot <= tol * max diag means the column is
//    numerically inside the span of the earlier ones: it is skipped (its row
//    of R and column of R^+ are zero), which drops the direction exactly as
//    Gram-Schmidt with deletion would.  Outputs R (FP64), T = R^+ in the
//    working type, and optionally R * Rprev (the accumulated R of CholeskyQR2).
//  * jacobi: one-sided (Hestenes) Jacobi SVD of Rb^H in round-robin order,
//    one warp per column pair; the singular values of Algorithm 4's small
//    matrix P^H A are those of Rb^H, where Rb is the R factor of (P^H A)^H.
//  * finalize: sort, truncate to k, zero directions below rtol * sigma_1 and
//    fix the phase of each singular vector against a Philox vector g.
#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
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

// divide by a positive real
PEPS_HD double divr(double a, double r) { return a / r; }
PEPS_HD double2 divr(double2 a, double r) { return make_double2(a.x / r, a.y / r); }
PEPS_HD double neg(double a) { return -a; }
PEPS_HD double2 neg(double2 a) { return make_double2(-a.x, -a.y); }

template <class T>
__global__ void __launch_bounds__(NT) chol_kernel(const CholDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  __shared__ double red[32];
  __shared__ double maxd_s;
  const CholDesc &g = descs[blockIdx.x];
  const int n = g.n;
  Acc *G = (Acc *)g.G;
  Acc *R = (Acc *)g.R;
  extern __shared__ unsigned char dyn[];
  unsigned char *dead = dyn;   // n flags

  double md = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) md = fmax(md, re(G[(int64_t)i * n + i]));
  md = block_max(md, red);
  if (threadIdx.x == 0) maxd_s = md;
  for (int i = threadIdx.x; i < n * n; i += NT) R[i] = widen(zero<T>());
  __syncthreads();
  const double thr = g.tol * maxd_s;

  for (int j = 0; j < n; ++j) {
    const double dj = re(G[(int64_t)j * n + j]);
    const bool isdead = !(dj > thr) || !(maxd_s > 0.0);
    if (threadIdx.x == 0) dead[j] = isdead;
    if (!isdead) {
      const double r = sqrt(dj);
      for (int k = j + threadIdx.x; k < n; k += NT)
        R[(int64_t)j * n + k] = k == j ? widen(from_parts<T>(r, 0.0)) : divr(G[(int64_t)j * n + k], r);
    }
    __syncthreads();
    if (!isdead) {
      // trailing update of the upper triangle: G[i][k] -= conj(R[j][i]) R[j][k], j < i <= k
      const int m = n - j - 1;
      const int64_t cnt = (int64_t)m * m;
      for (int64_t t = threadIdx.x; t < cnt; t += NT) {
        const int row = j + 1 + (int)(t / m), col = j + 1 + (int)(t % m);
        if (row > col) continue;
        const Acc a = conj_(R[(int64_t)j * n + row]);
        const Acc b = R[(int64_t)j * n + col];
        Acc &dst = G[(int64_t)row * n + col];
        dst = sub(dst, mul(a, b));
      }
    }
    __syncthreads();
  }

  // T = R^+ by back substitution (one thread per column), FP64 in G's storage
  Acc *Ti = G;
  for (int c = threadIdx.x; c < n; c += NT) {
    for (int i = 0; i < n; ++i) Ti[(int64_t)i * n + c] = widen(zero<T>());
    if (dead[c]) continue;
    Ti[(int64_t)c * n + c] = widen(from_parts<T>(1.0 / re(R[(int64_t)c * n + c]), 0.0));
    for (int i = c - 1; i >= 0; --i) {
      if (dead[i]) continue;
      Acc s = widen(zero<T>());
      for (int k = i + 1; k <= c; ++k) s = fma_(R[(int64_t)i * n + k], Ti[(int64_t)k * n + c], s);
      Ti[(int64_t)i * n + c] = divr(neg(s), re(R[(int64_t)i * n + i]));
    }
  }
  __syncthreads();
  T *Tout = (T *)g.T;
  for (int i = threadIdx.x; i < n * n; i += NT) Tout[i] = narrow<T>(Ti[i]);
  if (g.Rprev) {
    const Acc *P = (const Acc *)g.Rprev;
    Acc *O = (Acc *)g.Rout;
    for (int t = threadIdx.x; t < n * n; t += NT) {
      const int i = t / n, k = t % n;
      Acc s = widen(zero<T>());
      for (int l = i; l <= k; ++l) s = fma_(R[(int64_t)i * n + l], P[(int64_t)l * n + k], s);
      O[t] = s;
    }
  }
}

// Hestenes rotation of columns a, b (length n, FP64) in place.
template <class Acc>
__device__ bool jacobi_pair(Acc *a, Acc *b, int n, double tol) {
  const int lane = threadIdx.x & 31;
  double al = 0.0, be = 0.0;
  Acc ga = {};
  for (int r = lane; r < n; r += 32) {
    const Acc x = a[r], y = b[r];
    al += abs2(x);
    be += abs2(y);
    ga = fma_(conj_(x), y, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  const double g = sqrt(abs2(ga));
  if (!(g > tol * sqrt(al * be)) || g == 0.0) return false;
  const double zeta = (be - al) / (2.0 * g);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double s = c * t;
  // e^{-i phi} with gamma = |gamma| e^{i phi}
  Acc ph;
  if constexpr (sizeof(Acc) == 16) ph = make_double2(ga.x / g, -ga.y / g);
  else ph = ga > 0 ? 1.0 : -1.0;
  for (int r = lane; r < n; r += 32) {
    const Acc x = a[r];
    const Acc y = mul(b[r], ph);
    a[r] = sub(scale(x, c), scale(y, s));
    b[r] = add(scale(x, s), scale(y, c));
  }
  return true;
}

template <class T>
__global__ void __launch_bounds__(NT) jacobi_kernel(const JacobiDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  __shared__ int rotated;
  const JacobiDesc &g = descs[blockIdx.x];
  const int n = g.n;
  const Acc *Rb = (const Acc *)g.Rb;
  Acc *M = (Acc *)g.Mw;
  // column c of Rb^H = conj(row c of Rb)
  for (int t = threadIdx.x; t < n * n; t += NT) M[t] = conj_(Rb[t]);
  __syncthreads();
  const int n2 = n + (n & 1);
  const int warps = NT / 32, w = threadIdx.x >> 5;
  const double tol = 4.0 * n * 1.1102230246251565e-16;
  int sweep = 0;
  for (; sweep < g.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    int mine = 0;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int i = w; i < n2 / 2; i += warps) {
        int a, b;
        if (i == 0) { a = r; b = n2 - 1; }
        else { a = (r + i) % (n2 - 1); b = (r - i + (n2 - 1)) % (n2 - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= n) continue;
        if (jacobi_pair(M + (int64_t)a * n, M + (int64_t)b * n, n, tol)) mine = 1;
      }
      __syncthreads();
    }
    if (mine && (threadIdx.x & 31) == 0) rotated = 1;
    __syncthreads();
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == g.max_sweeps && threadIdx.x == 0 && g.status) atomicOr(g.status, STATUS_JACOBI_NOCONV);
  for (int c = w; c < n; c += warps) {
    double s2 = 0.0;
    for (int r = threadIdx.x & 31; r < n; r += 32) s2 += abs2(M[(int64_t)c * n + r]);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) g.sig[c] = sqrt(s2);
  }
}

template <class T>
__global__ void __launch_bounds__(NT) finalize_kernel(const FinalizeDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  const FinalizeDesc &g = descs[blockIdx.x];
  const int n = g.n, k = g.k;
  extern __shared__ __align__(16) unsigned char dyn[];
  int *order = (int *)dyn;                                   // n
  Acc *h = (Acc *)(dyn + ((n * sizeof(int) + 15) & ~15));    // n
  Acc *rho = h + n;                                          // k
  const double *sig = g.sig;
  const Acc *M = (const Acc *)g.Mw;
  for (int c = threadIdx.x; c < n; c += NT) {
    int rank = 0;
    const double sc = sig[c];
    for (int c2 = 0; c2 < n; ++c2) {
      const double s2 = sig[c2];
      rank += (s2 > sc) || (s2 == sc && c2 < c);
    }
    order[rank] = c;
  }
  // h_j = sum_m conj(P[j][m]) g[m]
  const T *P = (const T *)g.P;
  const T *gv = (const T *)g.g;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < n; j += NT / 32) {
    Acc s = widen(zero<T>());
    for (int64_t m = lane; m < g.M; m += 32)
      s = fma_(widen(conj_(P[(int64_t)j * g.M + m])), widen(gv[m]), s);
    s = warp_sum(s);
    if (lane == 0) h[j] = s;
  }
  __syncthreads();
  const double s1 = sig[order[0]];
  // phi_i = sum_j conj(h_j) u_{j,i}, u_i = M[:, order[i]] / sigma
  for (int i = w; i < k; i += NT / 32) {
    const int c = order[i];
    const double si = sig[c];
    const bool zero_dir = !(si > g.rtol * s1);
    Acc s = widen(zero<T>());
    if (!zero_dir)
      for (int j = lane; j < n; j += 32) s = fma_(conj_(h[j]), M[(int64_t)c * n + j], s);
    s = warp_sum(s);
    if (lane == 0) {
      Acc r;
      const double mag = sqrt(abs2(s));
      if constexpr (Traits<T>::cplx) r = mag > 0 ? make_double2(s.x / mag, s.y / mag) : make_double2(1.0, 0.0);
      else r = re(s) < 0 ? -1.0 : 1.0;
      // coefficient of u_i in Ut: conj(rho) / sigma_i (zero for dropped directions)
      rho[i] = zero_dir ? widen(zero<T>()) : scale(conj_(r), 1.0 / si);
      g.sigma_out[i] = zero_dir ? 0.0 : si;
    }
  }
  __syncthreads();
  T *Ut = (T *)g.Ut;
  for (int t = threadIdx.x; t < n * k; t += NT) {
    const int j = t / k, i = t % k;
    Ut[t] = narrow<T>(mul(M[(int64_t)order[i] * n + j], rho[i]));
  }
  if (threadIdx.x == 0) {
    *g.log_out = s1 > 0 ? log(s1) : -INFINITY;
    *g.inv_s1 = s1 > 0 ? 1.0 / s1 : 1.0;
    if (!isfinite(s1) && g.status) atomicOr(g.status, STATUS_NONFINITE);
  }
}

template <class T> void chol_t(const CholDesc *d, int nd, cudaStream_t s) {
  // dead flags: n bytes of dynamic shared memory (n <= 4096 enforced on the host)
  chol_kernel<T><<<nd, NT, 4096, s>>>(d);
}
template <class T> void jacobi_t(const JacobiDesc *d, int nd, cudaStream_t s) {
  jacobi_kernel<T><<<nd, NT, 0, s>>>(d);
}
template <class T> void finalize_t(const FinalizeDesc *d, int nd, cudaStream_t s) {
  // order (n ints) + h (n) + rho (k <= n) in FP64 complex at most: n <= 1024
  const int smem = 4096 + 2 * 1024 * 16;
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(finalize_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    set = true;
  }
  finalize_kernel<T><<<nd, NT, smem, s>>>(d);
}

}  // namespace

void launch_chol(int dt, const CholDesc *d, int nd, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: chol_t<float>(d, nd, s); break;
    case DT_C64: chol_t<float2>(d, nd, s); break;
    case DT_R64: chol_t<double>(d, nd, s); break;
    case DT_C128: chol_t<double2>(d, nd, s); break;
  }
}

void launch_jacobi(int dt, const JacobiDesc *d, int nd, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: jacobi_t<float>(d, nd, s); break;
    case DT_C64: jacobi_t<float2>(d, nd, s); break;
    case DT_R64: jacobi_t<double>(d, nd, s); break;
    case DT_C128: jacobi_t<double2>(d, nd, s); break;
  }
}

void launch_finalize(int dt, const FinalizeDesc *d, int nd, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: finalize_t<float>(d, nd, s); break;
    case DT_C64: finalize_t<float2>(d, nd, s); break;
    case DT_R64: finalize_t<double>(d, nd, s); break;
    case DT_C128: finalize_t<double2>(d, nd, s); break;
  }
}

}  // namespace peps
