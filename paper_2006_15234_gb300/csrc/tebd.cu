// Operator application by QR-SVD (Algorithm 1) on the bonds of one TEBD
// pass: the kernels that the generic ones (strided copies, Gram GEMMs,
// Cholesky, apply GEMMs, Philox draws) leave.
//
//  * theta: Theta[(r1, i1)][(r2, i2)] = sum_{j1, j2, b} G[i1 i2, j1 j2]
//    R1[r1][(j1, b)] R2[r2][(j2, b)] (Algorithm 1's einsumsvd input, Eq. 5
//    contracted with the two R factors), FP64 sums.
//  * svd_small: truncated SVD of Theta by one-sided Jacobi in FP64 (one CTA
//    per bond, Theta in shared memory, one warp per column pair of a
//    round-robin round); singular values sorted descending, the first k kept,
//    Sigma split evenly: R1t = U sqrt(Sigma) [(r1, i1)][k] and
//    R2t = (sqrt(Sigma) V^H)^T as [(r2, i2)][k] (Sigma / sigma_1 for
//    normalised bonds); directions at or below
//    16 max(rows, cols) eps64 sigma_1 are zero.  Theta is scaled to unit
//    Frobenius norm first, and a column whose norm falls to eps64 or below
//    is set to zero and leaves the rotations: a Theta with more columns than
//    rows (or of lower rank) has columns that can only become orthogonal by
//    vanishing, and without this they shrink every sweep until their norms
//    underflow.  Zeroing them changes Theta by at most
//    sqrt(cols) eps64 ||Theta||_F, below the zero rule above.
//  * site_op: a one-site operator on the physical index of a site (Eq. 4),
//    in place, each thread holding one column of the site's d values.
//  * site_gauge: the phase of every new bond direction c fixed on the
//    updated first site N1 [(outer, s)][k]: rho_c = <g, N1[:, c]> / |.|,
//    N1[:, c] *= conj(rho_c), N2[:, c] *= rho_c (real data: a sign).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
__global__ void theta_kernel(const ThetaDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  const ThetaDesc &g = descs[blockIdx.x];
  const int d = g.d, Db = g.Db, rows = g.r1 * d, cols = g.r2 * d, n = d * Db;
  const T *R1 = (const T *)g.R1, *R2 = (const T *)g.R2, *G = (const T *)g.G;
  T *Th = (T *)g.Theta;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int row = e / cols, col = e % cols;
    const int r1 = row / d, i1 = row % d, r2 = col / d, i2 = col % d;
    Acc acc = zero<Acc>();
    for (int j1 = 0; j1 < d; ++j1)
      for (int j2 = 0; j2 < d; ++j2) {
        const Acc gv = widen(G[(int64_t)(i1 * d + i2) * d * d + j1 * d + j2]);
        Acc s = zero<Acc>();
        for (int b = 0; b < Db; ++b)
          s = fma_(widen(R1[(int64_t)r1 * n + j1 * Db + b]), widen(R2[(int64_t)r2 * n + j2 * Db + b]), s);
        acc = fma_(gv, s, acc);
      }
    Th[(int64_t)row * cols + col] = narrow<T>(acc);
  }
}

template <class R> __device__ __forceinline__ R wsum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the single-precision type of an FP64 scalar type
template <class A> struct Lo;
template <> struct Lo<double> { using type = float; };
template <> struct Lo<double2> { using type = float2; };

// One-sided (Hestenes) Jacobi on A (mr x mc, column-major, column j at
// j * mr) with the rotations accumulated into V (mc x mc, column-major):
// round-robin pairs, one warp per pair, one barrier per round.  A pair is
// rotated when |<a_p, a_q>| > tol |a_p| |a_q|; a column of squared norm <=
// dead2 is set to zero and leaves the rotations (A is scaled to unit
// Frobenius norm by the caller).  Stops after the first sweep whose largest
// rotated off-diagonal is <= stop, or after max_sweeps.
template <class S>
__device__ bool jacobi_sweeps(S *A, S *V, int mr, int mc, int max_sweeps, double tol, double stop, double dead2,
                              float *off_max) {
  using R = typename Traits<S>::Real;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n2 = mc + (mc & 1);
  const R rtol = (R)tol, rdead = (R)dead2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *off_max = 0.f;
    __syncthreads();
    float mine = 0.f;
    for (int rr = 0; rr < n2 - 1; ++rr) {
      for (int i = warp; i < n2 / 2; i += nwarps) {
        int p, q;
        if (i == 0) { p = rr; q = n2 - 1; }
        else { p = (rr + i) % (n2 - 1); q = (rr - i + (n2 - 1)) % (n2 - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= mc) continue;
        S *ap = A + (int64_t)p * mr, *aq = A + (int64_t)q * mr;
        R al = 0, be = 0;
        S ga = zero<S>();
        for (int r = lane; r < mr; r += 32) {
          al += abs2(ap[r]);
          be += abs2(aq[r]);
          ga = fma_(conj_(ap[r]), aq[r], ga);
        }
        al = wsum_r(al);
        be = wsum_r(be);
        ga = from_parts<S>(wsum_r(re(ga)), wsum_r(im(ga)));
        if (al <= rdead || be <= rdead) {
          for (int r = lane; r < mr; r += 32) {
            if (al <= rdead) ap[r] = zero<S>();
            if (be <= rdead) aq[r] = zero<S>();
          }
          continue;
        }
        // the rotation test on squares: a converged pair costs no square root
        const R gm2 = abs2(ga), n2 = al * be;
        if (!(gm2 > rtol * rtol * n2)) continue;
        const R gm = sqrt(gm2), nrm = sqrt(n2);
        mine = fmaxf(mine, (float)(gm / nrm));
        // one reciprocal of |gamma| serves the phase and zeta, and the cosine
        // comes from rsqrt: FP64 divisions and square roots are the expensive
        // part of a rotation on this GPU
        const R ig = (R)1 / gm;
        // b_q = e^{-i phi} a_q makes <a_p, b_q> = |gamma| real; then the real rotation
        const S ph = scale(conj_(ga), ig);
        const R zeta = (be - al) * ((R)0.5 * ig), az = fabs(zeta);
        const R t = az > (R)1e15 ? (R)0.5 / zeta : (zeta >= 0 ? (R)1 : (R)-1) / (az + sqrt((R)1 + zeta * zeta));
        const R c = rsqrt((R)1 + t * t), sn = c * t;
        for (int r = lane; r < mr; r += 32) {
          const S x = ap[r], y = mul(ph, aq[r]);
          ap[r] = sub(scale(x, c), scale(y, sn));
          aq[r] = add(scale(x, sn), scale(y, c));
        }
        S *vp = V + (int64_t)p * mc, *vq = V + (int64_t)q * mc;
        for (int r = lane; r < mc; r += 32) {
          const S x = vp[r], y = mul(ph, vq[r]);
          vp[r] = sub(scale(x, c), scale(y, sn));
          vq[r] = add(scale(x, sn), scale(y, c));
        }
      }
      __syncthreads();
    }
    if (lane == 0) atomicMax((int *)off_max, __float_as_int(mine));
    __syncthreads();
    const bool done = *off_max <= (float)stop;
    __syncthreads();
    if (done) return true;
  }
  return false;
}

// Truncated SVD of one Theta.  GB300 runs FP64 at 1/64 of the FP32 rate, so
// the Jacobi runs in two phases: FP32 sweeps until the columns are
// orthogonal to ~1e-6, then V is made unitary in FP64 (two Newton-Schulz
// steps V <- V (3 I - V^H V) / 2), A = Theta V is formed in FP64 and FP64
// sweeps finish it (two or three, the convergence being quadratic).  The
// result is the FP64 SVD of the stored Theta.  A Theta with fewer rows than
// columns is factorised as Theta^H (mr >= mc always).
template <class T>
__global__ void svd_small_kernel(const SvdSmallDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;      // double or double2
  using S32 = typename Lo<Acc>::type;       // float or float2
  const SvdSmallDesc &g = descs[blockIdx.x];
  const int rows = g.rows, cols = g.cols, k = g.k;
  const bool tr = rows < cols;
  const int mr = tr ? cols : rows, mc = tr ? rows : cols;
  extern __shared__ __align__(16) unsigned char dyn[];
  Acc *A = (Acc *)dyn;                      // mr x mc, column-major
  Acc *Vm = A + (int64_t)mr * mc;           // mc x mc, column-major
  S32 *A32 = (S32 *)(Vm + (int64_t)mc * mc);
  S32 *V32 = A32 + (int64_t)mr * mc;
  Acc *W = (Acc *)A32;                      // mc x mc FP64 temporary over the FP32 copies (mr >= mc)
  __shared__ double sig[kSvdSmallMax];
  __shared__ int order[kSvdSmallMax];
  __shared__ float off_max;
  __shared__ double part[32];
  const T *Th = (const T *)g.Theta;         // row-major rows x cols
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // working matrix X = Theta, or Theta^H when Theta is wide
  auto X = [&](int i, int j) -> Acc {
    return tr ? conj_(widen(Th[(int64_t)j * cols + i])) : widen(Th[(int64_t)i * cols + j]);
  };
  // ||Theta||_F
  double f2 = 0.0;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) f2 += abs2(widen(Th[e]));
  f2 = wsum_r(f2);
  if (lane == 0) part[warp] = f2;
  __syncthreads();
  f2 = 0.0;
  for (int w = 0; w < nwarps; ++w) f2 += part[w];
  const double fro = sqrt(f2);
  T *R1t = (T *)g.R1t, *R2t = (T *)g.R2t;
  if (!(fro > 0.0) || !isfinite(fro)) {
    // an all-zero Theta gives a zero bond; a non-finite one is flagged and
    // carried into the sites
    const T fill = fro == 0.0 ? zero<T>() : from_parts<T>(fro, 0.0);
    if (fro != 0.0 && threadIdx.x == 0 && g.status) atomicOr(g.status, STATUS_NONFINITE);
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x) R1t[e] = fill;
    for (int e = threadIdx.x; e < cols * k; e += blockDim.x) R2t[e] = fill;
    if (g.sigma)
      for (int c = threadIdx.x; c < k; c += blockDim.x) g.sigma[c] = fro;
    return;
  }
  const double inv = 1.0 / fro;
  // phase 1: FP32 sweeps on X / ||X||_F
  for (int e = threadIdx.x; e < mr * mc; e += blockDim.x) {
    const int j = e / mr, i = e % mr;
    A32[e] = narrow<S32>(scale(X(i, j), inv));
  }
  for (int e = threadIdx.x; e < mc * mc; e += blockDim.x)
    V32[e] = (e / mc == e % mc) ? from_parts<S32>(1.0, 0.0) : zero<S32>();
  __syncthreads();
  const double eps32 = 5.9604644775390625e-08, eps64 = 1.1102230246251565e-16;
  jacobi_sweeps<S32>(A32, V32, mr, mc, 30, 16.0 * eps32, 64.0 * eps32, 4.0 * eps32 * eps32, &off_max);
  // phase 2: V unitary in FP64
  for (int e = threadIdx.x; e < mc * mc; e += blockDim.x) Vm[e] = widen(V32[e]);
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    // Gm = V^H V into A's space (mc x mc, column-major)
    for (int e = threadIdx.x; e < mc * mc; e += blockDim.x) {
      const int a = e % mc, b = e / mc;
      Acc s = zero<Acc>();
      for (int r = 0; r < mc; ++r) s = fma_(conj_(Vm[(int64_t)a * mc + r]), Vm[(int64_t)b * mc + r], s);
      A[e] = s;
    }
    __syncthreads();
    // W = V (3 I - Gm) / 2
    for (int e = threadIdx.x; e < mc * mc; e += blockDim.x) {
      const int i = e % mc, b = e / mc;
      Acc s = zero<Acc>();
      for (int a = 0; a < mc; ++a) s = fma_(Vm[(int64_t)a * mc + i], A[(int64_t)b * mc + a], s);
      W[e] = sub(scale(Vm[e], 1.5), scale(s, 0.5));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mc * mc; e += blockDim.x) Vm[e] = W[e];
    __syncthreads();
  }
  // phase 3: A = X V / ||X||_F in FP64, then FP64 sweeps
  for (int e = threadIdx.x; e < mr * mc; e += blockDim.x) {
    const int j = e / mr, i = e % mr;
    Acc s = zero<Acc>();
    for (int c = 0; c < mc; ++c) s = fma_(X(i, c), Vm[(int64_t)j * mc + c], s);
    A[e] = scale(s, inv);
  }
  __syncthreads();
  if (!jacobi_sweeps<Acc>(A, Vm, mr, mc, 60, 4.0 * eps64, 32.0 * eps64, 4.0 * eps64 * eps64, &off_max) &&
      threadIdx.x == 0 && g.status)
    atomicOr(g.status, STATUS_JACOBI_NOCONV);
  // singular values and their descending order (ties by index)
  for (int j = warp; j < mc; j += nwarps) {
    double s2 = 0.0;
    for (int r = lane; r < mr; r += 32) s2 += abs2(A[(int64_t)j * mr + r]);
    s2 = wsum_r(s2);
    if (lane == 0) sig[j] = sqrt(s2) * fro;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < mc; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < mc; ++i) rank += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    order[rank] = j;
  }
  __syncthreads();
  const double s1 = sig[order[0]];
  const double zt = 16.0 * (double)max(rows, cols) * 2.220446049250313e-16 * s1;
  // the split weight w_j: sigma_j, or sigma_j / sigma_1 for normalised bonds;
  // left factor column j: A_j fro / sigma_j (X's U) or V_j (when X = Theta^H)
  const double wdiv = g.unit ? s1 : 1.0;
  for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    T v = zero<T>();
    if (c < mc) {
      const int j = order[c];
      const double sv = sig[j];
      if (sv > zt)
        v = tr ? narrow<T>(scale(Vm[(int64_t)j * mc + r], sqrt(sv / wdiv)))
               : narrow<T>(scale(A[(int64_t)j * mr + r], fro / sv * sqrt(sv / wdiv)));
    }
    R1t[e] = v;
  }
  // right factor (sqrt(w) V^H)^T: conj(V_j) sqrt(w_j), V = X's V or X's U when X = Theta^H
  for (int e = threadIdx.x; e < cols * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    T v = zero<T>();
    if (c < mc) {
      const int j = order[c];
      const double sv = sig[j];
      if (sv > zt)
        v = tr ? narrow<T>(scale(conj_(A[(int64_t)j * mr + r]), fro / sv * sqrt(sv / wdiv)))
               : narrow<T>(scale(conj_(Vm[(int64_t)j * mc + r]), sqrt(sv / wdiv)));
    }
    R2t[e] = v;
  }
  if (g.sigma)
    for (int c = threadIdx.x; c < k; c += blockDim.x)
      g.sigma[c] = (c < mc && sig[order[c]] > zt) ? sig[order[c]] : 0.0;
}

template <class T>
__global__ void site_gauge_kernel(const SiteGaugeDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  const SiteGaugeDesc &g = descs[blockIdx.x];
  const int k = g.k;
  T *N1 = (T *)g.N1, *N2 = (T *)g.N2;
  const T *gv = (const T *)g.g;
  __shared__ double2 rho[kSvdSmallMax];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int c = warp; c < k; c += nwarps) {
    Acc s = zero<Acc>();
    for (int64_t r = lane; r < g.rows1; r += 32) s = fma_(conj_(widen(gv[r])), widen(N1[r * k + c]), s);
    const double sr = wsum(re(s)), si = wsum(im(s));
    if (lane == 0) {
      double2 p = make_double2(1.0, 0.0);
      if (Traits<T>::cplx) {
        const double m = sqrt(sr * sr + si * si);
        if (m > 0.0) p = make_double2(sr / m, si / m);
      } else if (sr < 0.0) {
        p = make_double2(-1.0, 0.0);
      }
      rho[c] = p;
    }
  }
  __syncthreads();
  // (32-bit element indices: a site matrix holds far fewer than 2^31 values)
  for (int e = threadIdx.x; e < (int)(g.rows1 * k); e += blockDim.x) {
    const double2 p = rho[e % k];
    N1[e] = mul(N1[e], from_parts<T>(p.x, -p.y));
  }
  for (int e = threadIdx.x; e < (int)(g.rows2 * k); e += blockDim.x) {
    const double2 p = rho[e % k];
    N2[e] = mul(N2[e], from_parts<T>(p.x, p.y));
  }
}

// one-site operator, in place: thread r owns column r of M as [d][rest]
template <class T>
__global__ void site_op_kernel(const SiteOpDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;
  const SiteOpDesc &g = descs[blockIdx.y];
  const int d = g.d;
  T *M = (T *)g.M;
  const T *G = (const T *)g.g;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < g.rest; r += (int64_t)gridDim.x * blockDim.x) {
    Acc x[kSiteOpMaxPhys];
    for (int j = 0; j < d; ++j) x[j] = widen(M[(int64_t)j * g.rest + r]);
    for (int i = 0; i < d; ++i) {
      Acc acc = zero<Acc>();
      for (int j = 0; j < d; ++j) acc = fma_(widen(G[i * d + j]), x[j], acc);
      M[(int64_t)i * g.rest + r] = narrow<T>(acc);
    }
  }
}

template <class T> void tebd_launch(int kind, const void *d, int nd, int aux, cudaStream_t s) {
  if (nd <= 0) return;
  if (kind == 0) {
    theta_kernel<T><<<nd, 256, 0, s>>>((const ThetaDesc *)d);
  } else if (kind == 1) {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(svd_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set = true;
    }
    svd_small_kernel<T><<<nd, 256, aux, s>>>((const SvdSmallDesc *)d);
  } else if (kind == 2) {
    site_gauge_kernel<T><<<nd, 256, 0, s>>>((const SiteGaugeDesc *)d);
  } else {
    // grid.y: one row per site; grid.x: aux column blocks (strided loop)
    site_op_kernel<T><<<dim3((unsigned)aux, (unsigned)nd), 256, 0, s>>>((const SiteOpDesc *)d);
  }
}

}  // namespace

int svd_small_smem_bytes(int dt, int rows, int cols) {
  // FP64 A (mr x mc) and V (mc x mc), and their FP32 copies; mr >= mc
  const int as = acc_size(dt), mc = rows < cols ? rows : cols;
  return as * (rows * cols + mc * mc) * 3 / 2;
}

void launch_tebd(int dt, int kind, const void *d, int nd, int aux, cudaStream_t s) {
  switch (dt) {
    case DT_R32: tebd_launch<float>(kind, d, nd, aux, s); break;
    case DT_C64: tebd_launch<float2>(kind, d, nd, aux, s); break;
    case DT_R64: tebd_launch<double>(kind, d, nd, aux, s); break;
    case DT_C128: tebd_launch<double2>(kind, d, nd, aux, s); break;
  }
}

}  // namespace peps
