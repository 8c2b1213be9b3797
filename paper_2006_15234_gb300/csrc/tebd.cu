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
//    R2t = (sqrt(Sigma) V^H)^T as [(r2, i2)][k]; directions at or below
//    16 max(rows, cols) eps64 sigma_1 are zero.  Theta is scaled to unit
//    Frobenius norm first, and a column whose norm falls to eps64 or below
//    is set to zero and leaves the rotations: a Theta with more columns than
//    rows (or of lower rank) has columns that can only become orthogonal by
//    vanishing, and without this they shrink every sweep until their norms
//    underflow.  Zeroing them changes Theta by at most
//    sqrt(cols) eps64 ||Theta||_F, below the zero rule above.
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

// complex helpers on double2 / double for the FP64 Jacobi
template <class A> struct CJ;
template <> struct CJ<double> {
  __device__ static double conj(double a) { return a; }
  __device__ static double abs2(double a) { return a * a; }
};
template <> struct CJ<double2> {
  __device__ static double2 conj(double2 a) { return make_double2(a.x, -a.y); }
  __device__ static double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
};

template <class T>
__global__ void svd_small_kernel(const SvdSmallDesc *__restrict__ descs) {
  using Acc = typename Traits<T>::Acc;      // double or double2
  const SvdSmallDesc &g = descs[blockIdx.x];
  const int rows = g.rows, cols = g.cols, k = g.k;
  const int n2 = cols + (cols & 1);
  extern __shared__ __align__(16) unsigned char dyn[];
  Acc *A = (Acc *)dyn;                      // column-major rows x cols (column j at j * rows)
  Acc *Vm = A + (int64_t)rows * cols;       // column-major cols x cols
  __shared__ double sig[kSvdSmallMax];
  __shared__ int order[kSvdSmallMax];
  __shared__ float off_max;
  __shared__ double part[32];
  const T *Th = (const T *)g.Theta;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // ||Theta||_F
  double f2 = 0.0;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) f2 += CJ<Acc>::abs2(widen(Th[e]));
  f2 = wsum(f2);
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
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int r = e / cols, c = e % cols;
    A[(int64_t)c * rows + r] = scale(widen(Th[e]), inv);
  }
  for (int e = threadIdx.x; e < cols * cols; e += blockDim.x)
    Vm[e] = (e / cols == e % cols) ? widen(from_parts<T>(1.0, 0.0)) : zero<Acc>();
  __syncthreads();
  const double tol = 4.0 * 1.1102230246251565e-16;
  const double dead2 = 2.220446049250313e-16 * 2.220446049250313e-16;   // (eps64 ||Theta||_F)^2, scaled
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) off_max = 0.f;
    __syncthreads();
    float mine = 0.f;
    for (int rr = 0; rr < n2 - 1; ++rr) {
      for (int i = warp; i < n2 / 2; i += nwarps) {
        int p, q;
        if (i == 0) { p = rr; q = n2 - 1; }
        else { p = (rr + i) % (n2 - 1); q = (rr - i + (n2 - 1)) % (n2 - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= cols) continue;
        Acc *ap = A + (int64_t)p * rows, *aq = A + (int64_t)q * rows;
        double al = 0.0, be = 0.0;
        Acc ga = zero<Acc>();
        for (int r = lane; r < rows; r += 32) {
          al += CJ<Acc>::abs2(ap[r]);
          be += CJ<Acc>::abs2(aq[r]);
          ga = fma_(CJ<Acc>::conj(ap[r]), aq[r], ga);
        }
        al = wsum(al);
        be = wsum(be);
        ga = from_parts<Acc>(wsum(re(ga)), wsum(im(ga)));
        if (al <= dead2 || be <= dead2) {
          for (int r = lane; r < rows; r += 32) {
            if (al <= dead2) ap[r] = zero<Acc>();
            if (be <= dead2) aq[r] = zero<Acc>();
          }
          continue;
        }
        const double gm = sqrt(CJ<Acc>::abs2(ga));
        if (!(gm > tol * sqrt(al * be)) || gm == 0.0) continue;
        mine = fmaxf(mine, (float)(gm / sqrt(al * be)));
        // b_q = e^{-i phi} a_q makes <a_p, b_q> = |gamma|; then the real rotation
        const Acc ph = scale(CJ<Acc>::conj(ga), 1.0 / gm);         // e^{-i phi}
        const double zeta = (be - al) / (2.0 * gm);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int r = lane; r < rows; r += 32) {
          const Acc x = ap[r], y = mul(ph, aq[r]);
          ap[r] = sub(scale(x, c), scale(y, s));
          aq[r] = add(scale(x, s), scale(y, c));
        }
        Acc *vp = Vm + (int64_t)p * cols, *vq = Vm + (int64_t)q * cols;
        for (int r = lane; r < cols; r += 32) {
          const Acc x = vp[r], y = mul(ph, vq[r]);
          vp[r] = sub(scale(x, c), scale(y, s));
          vq[r] = add(scale(x, s), scale(y, c));
        }
      }
      __syncthreads();
    }
    if (lane == 0) atomicMax((int *)&off_max, __float_as_int(mine));
    __syncthreads();
    const bool done = off_max <= (float)(8.0 * tol);
    __syncthreads();
    if (done) break;
  }
  // singular values and their descending order (ties by index)
  for (int j = warp; j < cols; j += nwarps) {
    double s2 = 0.0;
    for (int r = lane; r < rows; r += 32) s2 += CJ<Acc>::abs2(A[(int64_t)j * rows + r]);
    s2 = wsum(s2);
    if (lane == 0) sig[j] = sqrt(s2) * fro;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < cols; ++i) rank += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    order[rank] = j;
  }
  __syncthreads();
  const double s1 = sig[order[0]];
  const double zt = 16.0 * (double)max(rows, cols) * 2.220446049250313e-16 * s1;
  for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
    const int r = e / k, c = e % k, j = order[c];
    const double sv = sig[j];
    // U sqrt(S) = A_j / sigma_j * sqrt(sigma_j) = A_j / sqrt(sigma_j), A_j = fro x the scaled column
    R1t[e] = sv > zt ? narrow<T>(scale(A[(int64_t)j * rows + r], fro / sqrt(sv))) : zero<T>();
  }
  for (int e = threadIdx.x; e < cols * k; e += blockDim.x) {
    const int r = e / k, c = e % k, j = order[c];
    const double sv = sig[j];
    // (sqrt(S) V^H)[c][r] = sqrt(sigma_j) conj(V[r][j])
    R2t[e] = sv > zt ? narrow<T>(scale(CJ<Acc>::conj(Vm[(int64_t)j * cols + r]), sqrt(sv))) : zero<T>();
  }
  if (g.sigma)
    for (int c = threadIdx.x; c < k; c += blockDim.x) g.sigma[c] = sig[order[c]] > zt ? sig[order[c]] : 0.0;
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
  for (int64_t e = threadIdx.x; e < g.rows1 * k; e += blockDim.x) {
    const double2 p = rho[e % k];
    N1[e] = mul(N1[e], from_parts<T>(p.x, -p.y));
  }
  for (int64_t e = threadIdx.x; e < g.rows2 * k; e += blockDim.x) {
    const double2 p = rho[e % k];
    N2[e] = mul(N2[e], from_parts<T>(p.x, p.y));
  }
}

template <class T> void tebd_launch(int kind, const void *d, int nd, int smem, cudaStream_t s) {
  if (nd <= 0) return;
  if (kind == 0) {
    theta_kernel<T><<<nd, 256, 0, s>>>((const ThetaDesc *)d);
  } else if (kind == 1) {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(svd_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set = true;
    }
    svd_small_kernel<T><<<nd, 256, smem, s>>>((const SvdSmallDesc *)d);
  } else {
    site_gauge_kernel<T><<<nd, 256, 0, s>>>((const SiteGaugeDesc *)d);
  }
}

}  // namespace

int svd_small_smem_bytes(int dt, int rows, int cols) {
  const int as = acc_size(dt);
  return as * (rows * cols + cols * cols);
}

void launch_tebd(int dt, int kind, const void *d, int nd, int smem, cudaStream_t s) {
  switch (dt) {
    case DT_R32: tebd_launch<float>(kind, d, nd, smem, s); break;
    case DT_C64: tebd_launch<float2>(kind, d, nd, smem, s); break;
    case DT_R64: tebd_launch<double>(kind, d, nd, smem, s); break;
    case DT_C128: tebd_launch<double2>(kind, d, nd, smem, s); break;
  }
}

}  // namespace peps
