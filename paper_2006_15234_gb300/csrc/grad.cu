// Small kernels of the einsumsvd adjoint (reverse mode of Algorithm 4 with
// the sketch held fixed), real data:
//  * svd_bwd: the l x l core of the SVD adjoint.  With B = U~ S V~^T the
//    l x N matrix of Algorithm 4, the step's outputs use U~_k (through
//    U = P U~_k and W = U~_k^T B / sigma_1) and sigma_1; given their
//    cotangents, B's cotangent is H B (+ the direct term of W), with
//    H = U~ C S^-1 U~^T, C = (F o (U~^T Ubar - Ubar^T U~)) S + diag(sbar),
//    F_ij = 1 / (s_j^2 - s_i^2) (i != j).
//  * copyltu: the symmetric matrix built from the lower triangle, used by the
//    QR adjoint  Ybar = (Qbar + Q copyltu(-Qbar^T Q)) R^-T.
//  * tensor_grad: cotangents of the two site tensors from the rank-P
//    factorisation Abar = sum_j L_j R_j^T of A's cotangent (direct sums; the
//    site tensors are the smallest operands).
#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int NTG = 256;

template <class T>
__global__ void __launch_bounds__(NTG) svd_bwd_kernel(SvdBwdDesc g) {
  const int n = g.n, k = g.k;
  const T *Mw = (const T *)g.Mw, *Ut = (const T *)g.Ut, *Ub = (const T *)g.Utbar, *WW = (const T *)g.WW;
  double *Uf = g.scratch;               // n x n, column i = i-th singular vector (sorted)
  double *C = Uf + (size_t)n * n;       // n x n
  double *Tq = C + (size_t)n * n;       // n x n: C S^-1 U~^T
  double *s = Tq + (size_t)n * n;       // n
  int *order = (int *)(s + n);          // n
  for (int c = threadIdx.x; c < n; c += NTG) {
    int rank = 0;
    const double sc = g.sig[c];
    for (int c2 = 0; c2 < n; ++c2) {
      const double s2 = g.sig[c2];
      rank += (s2 > sc) || (s2 == sc && c2 < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  // singular vectors: the gauge-fixed Ut for the kept k, unit columns of Mw for the rest
  for (int i = threadIdx.x; i < n; i += NTG) {
    const int c = order[i];
    s[i] = g.sig[c];
    if (i < k) {
      for (int r = 0; r < n; ++r) Uf[(size_t)r * n + i] = (double)Ut[(size_t)r * k + i];
    } else {
      double nrm = 0.0;
      for (int r = 0; r < n; ++r) nrm += (double)Mw[(size_t)c * n + r] * (double)Mw[(size_t)c * n + r];
      nrm = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
      for (int r = 0; r < n; ++r) Uf[(size_t)r * n + i] = (double)Mw[(size_t)c * n + r] * nrm;
    }
  }
  __syncthreads();
  // C = (F o (A1 - A1^T)) S + diag(sbar), A1 = U~^T [Utbar, 0]
  double trw = 0.0;
  for (int i = 0; i < k; ++i) trw += (double)WW[(size_t)i * k + i];
  const double sbar0 = (*g.lbar - trw) * *g.inv_s1;
  for (int t = threadIdx.x; t < n * n; t += NTG) {
    const int i = t / n, j = t % n;
    double v = 0.0;
    if (i != j) {
      double a_ij = 0.0, a_ji = 0.0;        // (U~^T Ubar)_ij and _ji
      for (int r = 0; r < n; ++r) {
        if (j < k) a_ij += Uf[(size_t)r * n + i] * (double)Ub[(size_t)r * k + j];
        if (i < k) a_ji += Uf[(size_t)r * n + j] * (double)Ub[(size_t)r * k + i];
      }
      const double den = s[j] * s[j] - s[i] * s[i];
      v = den != 0.0 ? (a_ij - a_ji) / den * s[j] : 0.0;
    } else if (i == 0) {
      v = sbar0;
    }
    C[t] = v;
  }
  __syncthreads();
  // H = U~ (C S^-1 U~^T)
  for (int t = threadIdx.x; t < n * n; t += NTG) {
    const int i = t / n, b = t % n;
    double w = 0.0;
    for (int j = 0; j < n; ++j)
      if (s[j] > 0.0) w += C[(size_t)i * n + j] / s[j] * Uf[(size_t)b * n + j];
    Tq[t] = w;
  }
  __syncthreads();
  T *H = (T *)g.H;
  for (int t = threadIdx.x; t < n * n; t += NTG) {
    const int a = t / n, b = t % n;
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += Uf[(size_t)a * n + i] * Tq[(size_t)i * n + b];
    H[t] = (T)v;
  }
}

template <class T> __global__ void copyltu_kernel(const T *M, T *out, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  out[t] = i >= j ? M[t] : M[(size_t)j * n + i];
}

// Kbar[s,l,u,x,e]  = sum_{j,b,L,U,X,E} Z2[j][(l,L)][(u,U),b] Kb[s,L,U,X,E] R[j][(x,X,b,e,E)]
// Kbbar[s,L,U,X,E] = sum_{j,b,l,u,x,e} Z2[j][(l,L)][(u,U),b] K[s,l,u,x,e]  R[j][(x,X,b,e,E)]
template <class T> __global__ void __launch_bounds__(NTG) tensor_grad_kernel(TensorGradDesc g) {
  const int d = g.d, Dl = g.Dl, Du = g.Du, Dx = g.Dx, De = g.De, DL = g.DL, DU = g.DU, DX = g.DX, DE = g.DE,
            b = g.b;
  const int64_t nk = (int64_t)d * Dl * Du * Dx * De, nkb = (int64_t)d * DL * DU * DX * DE;
  const int64_t t = (int64_t)blockIdx.x * NTG + threadIdx.x;
  if (t >= nk + nkb) return;
  const T *Z2 = (const T *)g.Z2, *R = (const T *)g.R, *K = (const T *)g.K, *Kb = (const T *)g.Kb;
  const int h = Dl * DL, v = Du * DU;
  const int64_t ldz = (int64_t)h * v * b, N = (int64_t)Dx * DX * b * De * DE;
  double acc = 0.0;
  if (t < nk) {
    int64_t r = t;
    const int e = (int)(r % De); r /= De;
    const int x = (int)(r % Dx); r /= Dx;
    const int u = (int)(r % Du); r /= Du;
    const int l = (int)(r % Dl); r /= Dl;
    const int s = (int)r;
    for (int j = 0; j < g.P; ++j)
      for (int bb = 0; bb < b; ++bb)
        for (int L = 0; L < DL; ++L)
          for (int U = 0; U < DU; ++U) {
            const double z = (double)Z2[j * ldz + ((int64_t)(l * DL + L) * v + u * DU + U) * b + bb];
            if (z == 0.0) continue;
            double w = 0.0;
            for (int X = 0; X < DX; ++X)
              for (int E = 0; E < DE; ++E)
                w += (double)Kb[(((int64_t)(s * DL + L) * DU + U) * DX + X) * DE + E] *
                     (double)R[j * N + ((((int64_t)x * DX + X) * b + bb) * De + e) * DE + E];
            acc += z * w;
          }
    ((T *)g.Kbar)[t] = (T)acc;
  } else {
    int64_t r = t - nk;
    const int E = (int)(r % DE); r /= DE;
    const int X = (int)(r % DX); r /= DX;
    const int U = (int)(r % DU); r /= DU;
    const int L = (int)(r % DL); r /= DL;
    const int s = (int)r;
    for (int j = 0; j < g.P; ++j)
      for (int bb = 0; bb < b; ++bb)
        for (int l = 0; l < Dl; ++l)
          for (int u = 0; u < Du; ++u) {
            const double z = (double)Z2[j * ldz + ((int64_t)(l * DL + L) * v + u * DU + U) * b + bb];
            if (z == 0.0) continue;
            double w = 0.0;
            for (int x = 0; x < Dx; ++x)
              for (int e = 0; e < De; ++e)
                w += (double)K[(((int64_t)(s * Dl + l) * Du + u) * Dx + x) * De + e] *
                     (double)R[j * N + ((((int64_t)x * DX + X) * b + bb) * De + e) * DE + E];
            acc += z * w;
          }
    ((T *)g.Kbbar)[t - nk] = (T)acc;
  }
}

}  // namespace

void launch_svd_bwd(int dt, const SvdBwdDesc &d, cudaStream_t s) {
  if (dt == DT_R32) svd_bwd_kernel<float><<<1, NTG, 0, s>>>(d);
  else if (dt == DT_R64) svd_bwd_kernel<double><<<1, NTG, 0, s>>>(d);
}

void launch_copyltu(int dt, const void *M, void *out, int n, cudaStream_t s) {
  const int blocks = (n * n + 255) / 256;
  if (blocks <= 0) return;
  if (dt == DT_R32) copyltu_kernel<float><<<blocks, 256, 0, s>>>((const float *)M, (float *)out, n);
  else if (dt == DT_R64) copyltu_kernel<double><<<blocks, 256, 0, s>>>((const double *)M, (double *)out, n);
}

void launch_tensor_grad(int dt, const TensorGradDesc &d, cudaStream_t s) {
  const int64_t n = (int64_t)d.d * (d.Dl * d.Du * d.Dx * d.De + d.DL * d.DU * d.DX * d.DE);
  const unsigned blocks = (unsigned)((n + NTG - 1) / NTG);
  if (!blocks) return;
  if (dt == DT_R32) tensor_grad_kernel<float><<<blocks, NTG, 0, s>>>(d);
  else if (dt == DT_R64) tensor_grad_kernel<double><<<blocks, NTG, 0, s>>>(d);
}

}  // namespace peps
