// Adjoint kernels of the network layer (real data): the strip contraction
// of the cached-environment expectation value (Eq. 6), the two row-start
// site contractions of the boundary sweep (Algorithm 2's first row and
// Algorithm 3's first zip-up carry), and an accumulate.  Cotangents are
// added into their targets with atomics (several strips and steps feed the
// same boundary sites and PEPS tensors).
#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int NTB = 256;

template <class T> __device__ __forceinline__ void add_to(void *p, int64_t i, double v) {
  atomicAdd((T *)p + i, (T)v);
}

// One strip: left blocks L_0..L_n, right blocks R_n..R_0, then per column the
// cotangents of its four tensors, scaled by the strip's cotangent.
template <class T>
__global__ void __launch_bounds__(NTB) strip_bwd_kernel(const StripDesc *__restrict__ descs,
                                                        const StripCol *__restrict__ cols,
                                                        const StripBwdCol *__restrict__ bcols,
                                                        const double *__restrict__ ops, const double *__restrict__ sbar,
                                                        StripBwdScratch sc) {
  const StripDesc &g = descs[blockIdx.x];
  const double w = sbar[blockIdx.x];
  const int n = g.ncol;
  double *base = sc.base + (size_t)blockIdx.x * sc.per_strip;
  double *Lb = base;                                  // (n+1) x blk
  double *Rb = Lb + (size_t)(n + 1) * sc.blk;         // (n+1) x blk
  double *A1 = Rb + (size_t)(n + 1) * sc.blk;
  double *A2 = A1 + sc.big;
  double *A3 = A2 + sc.big;
  double *B1 = A3 + sc.big;
  double *B2 = B1 + sc.big;
  double *B3 = B2 + sc.big;
  auto L = [&](int q) { return Lb + (size_t)q * sc.blk; };
  auto R = [&](int q) { return Rb + (size_t)q * sc.blk; };
  if (threadIdx.x == 0) { L(0)[0] = 1.0; R(n)[0] = 1.0; }
  __syncthreads();
  // K' = op K on the physical index (op may be absent)
  auto kp = [&](const T *K, const double *op, int d, int64_t rest, int s, int64_t idx) -> double {
    if (!op) return (double)K[(int64_t)s * rest + idx];
    double v = 0.0;
    for (int s2 = 0; s2 < d; ++s2) v += op[s * d + s2] * (double)K[(int64_t)s2 * rest + idx];
    return v;
  };
  // ---- forward stages of column q from left block Lq (writes A1, A2, A3) ----
  auto fwd = [&](int q, const double *Lq) {
    const StripCol &c = cols[g.col0 + q];
    const T *Tu = (const T *)c.up, *K = (const T *)c.ket;
    const int a = c.a, b = c.b, cc = c.c, d = c.d, Dl = c.Dl, Du = c.Du, Dx = c.Dx, De = c.De;
    const int vu = Du * Du;
    const int64_t rest = (int64_t)Dl * Du * Dx * De;
    const double *op = g.op[q] >= 0 ? ops + (int64_t)g.op[q] * d * d : nullptr;
    for (int64_t t = threadIdx.x; t < (int64_t)Dl * Dl * cc * vu * b; t += NTB) {
      int64_t r = t;
      const int bb = (int)(r % b); r /= b;
      const int uU = (int)(r % vu); r /= vu;
      const int c_ = (int)(r % cc); r /= cc;
      const int lL = (int)r;
      double s = 0.0;
      for (int a_ = 0; a_ < a; ++a_)
        s += Lq[((int64_t)a_ * Dl * Dl + lL) * cc + c_] * (double)Tu[((int64_t)a_ * vu + uU) * b + bb];
      A1[t] = s;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)Dl * cc * Du * b * d * Dx * De; t += NTB) {
      int64_t r = t;
      const int e = (int)(r % De); r /= De;
      const int x = (int)(r % Dx); r /= Dx;
      const int s_ = (int)(r % d); r /= d;
      const int bb = (int)(r % b); r /= b;
      const int U = (int)(r % Du); r /= Du;
      const int c_ = (int)(r % cc); r /= cc;
      const int Lq_ = (int)r;
      double acc = 0.0;
      for (int l = 0; l < Dl; ++l)
        for (int u = 0; u < Du; ++u)
          acc += A1[((((int64_t)(l * Dl + Lq_) * cc + c_) * Du + u) * Du + U) * b + bb] *
                 kp(K, op, d, rest, s_, (((int64_t)l * Du + u) * Dx + x) * De + e);
      A2[t] = acc;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)cc * b * De * Dx * Dx * De; t += NTB) {
      int64_t r = t;
      const int E = (int)(r % De); r /= De;
      const int X = (int)(r % Dx); r /= Dx;
      const int x = (int)(r % Dx); r /= Dx;
      const int e = (int)(r % De); r /= De;
      const int bb = (int)(r % b); r /= b;
      const int c_ = (int)r;
      double acc = 0.0;
      for (int s_ = 0; s_ < d; ++s_)
        for (int Lq_ = 0; Lq_ < Dl; ++Lq_)
          for (int U = 0; U < Du; ++U)
            acc += A2[((((((int64_t)Lq_ * cc + c_) * Du + U) * b + bb) * d + s_) * Dx + x) * De + e] *
                   (double)K[((((int64_t)s_ * Dl + Lq_) * Du + U) * Dx + X) * De + E];
      A3[t] = acc;
    }
    __syncthreads();
  };
  // ---- right stages of column q from right block Rq = R_{q+1} (writes B1, B2, B3) ----
  auto bwd = [&](int q, const double *Rq) {
    const StripCol &c = cols[g.col0 + q];
    const T *Bl = (const T *)c.lo, *K = (const T *)c.ket;
    const int b = c.b, cc = c.c, f = c.f, d = c.d, Dl = c.Dl, Du = c.Du, Dx = c.Dx, De = c.De;
    const int vd = Dx * Dx;
    const int64_t rest = (int64_t)Dl * Du * Dx * De;
    const double *op = g.op[q] >= 0 ? ops + (int64_t)g.op[q] * d * d : nullptr;
    // B1[c][x][X][b][e][E] = sum_f Bl[c][(x,X)][f] Rq[b][e][E][f]
    for (int64_t t = threadIdx.x; t < (int64_t)cc * Dx * Dx * b * De * De; t += NTB) {
      int64_t r = t;
      const int E = (int)(r % De); r /= De;
      const int e = (int)(r % De); r /= De;
      const int bb = (int)(r % b); r /= b;
      const int X = (int)(r % Dx); r /= Dx;
      const int x = (int)(r % Dx); r /= Dx;
      const int c_ = (int)r;
      double acc = 0.0;
      for (int ff = 0; ff < f; ++ff)
        acc += (double)Bl[((int64_t)c_ * vd + x * Dx + X) * f + ff] * Rq[(((int64_t)bb * De + e) * De + E) * f + ff];
      B1[t] = acc;
    }
    __syncthreads();
    // B2[c][x][b][e][s][L][U] = sum_{X,E} B1[c][x][X][b][e][E] K[s][L][U][X][E]
    for (int64_t t = threadIdx.x; t < (int64_t)cc * Dx * b * De * d * Dl * Du; t += NTB) {
      int64_t r = t;
      const int U = (int)(r % Du); r /= Du;
      const int Lq_ = (int)(r % Dl); r /= Dl;
      const int s_ = (int)(r % d); r /= d;
      const int e = (int)(r % De); r /= De;
      const int bb = (int)(r % b); r /= b;
      const int x = (int)(r % Dx); r /= Dx;
      const int c_ = (int)r;
      double acc = 0.0;
      for (int X = 0; X < Dx; ++X)
        for (int E = 0; E < De; ++E)
          acc += B1[((((((int64_t)c_ * Dx + x) * Dx + X) * b + bb) * De + e) * De + E)] *
                 (double)K[((((int64_t)s_ * Dl + Lq_) * Du + U) * Dx + X) * De + E];
      B2[t] = acc;
    }
    __syncthreads();
    // B3[c][b][L][U][l][u] = sum_{s,x,e} B2[c][x][b][e][s][L][U] K'[s][l][u][x][e]
    for (int64_t t = threadIdx.x; t < (int64_t)cc * b * Dl * Du * Dl * Du; t += NTB) {
      int64_t r = t;
      const int u = (int)(r % Du); r /= Du;
      const int l = (int)(r % Dl); r /= Dl;
      const int U = (int)(r % Du); r /= Du;
      const int Lq_ = (int)(r % Dl); r /= Dl;
      const int bb = (int)(r % b); r /= b;
      const int c_ = (int)r;
      double acc = 0.0;
      for (int s_ = 0; s_ < d; ++s_)
        for (int x = 0; x < Dx; ++x)
          for (int e = 0; e < De; ++e)
            acc += B2[((((((int64_t)c_ * Dx + x) * b + bb) * De + e) * d + s_) * Dl + Lq_) * Du + U] *
                   kp(K, op, d, rest, s_, (((int64_t)l * Du + u) * Dx + x) * De + e);
      B3[t] = acc;
    }
    __syncthreads();
  };
  // left blocks
  for (int q = 0; q < n; ++q) {
    const StripCol &c = cols[g.col0 + q];
    fwd(q, L(q));
    double *Ln = L(q + 1);
    const int b = c.b, f = c.f, De = c.De, cc = c.c, Dx = c.Dx;
    const T *Bl = (const T *)c.lo;
    for (int64_t t = threadIdx.x; t < (int64_t)b * De * De * f; t += NTB) {
      int64_t r = t;
      const int ff = (int)(r % f); r /= f;
      const int E = (int)(r % De); r /= De;
      const int e = (int)(r % De); r /= De;
      const int bb = (int)r;
      double acc = 0.0;
      for (int c_ = 0; c_ < cc; ++c_)
        for (int x = 0; x < Dx; ++x)
          for (int X = 0; X < Dx; ++X)
            acc += A3[((((int64_t)c_ * b + bb) * De + e) * Dx + x) * Dx * De + (int64_t)X * De + E] *
                   (double)Bl[((int64_t)c_ * Dx * Dx + x * Dx + X) * f + ff];
      Ln[t] = acc;
    }
    __syncthreads();
  }
  // right blocks: R_q[a][l][L][c] = sum_{u,U,b} T[a][(u,U)][b] B3[c][b][L][U][l][u]
  for (int q = n - 1; q >= 0; --q) {
    const StripCol &c = cols[g.col0 + q];
    bwd(q, R(q + 1));
    double *Rn = R(q);
    const int a = c.a, b = c.b, cc = c.c, Dl = c.Dl, Du = c.Du;
    const T *Tu = (const T *)c.up;
    for (int64_t t = threadIdx.x; t < (int64_t)a * Dl * Dl * cc; t += NTB) {
      int64_t r = t;
      const int c_ = (int)(r % cc); r /= cc;
      const int Lq_ = (int)(r % Dl); r /= Dl;
      const int l = (int)(r % Dl); r /= Dl;
      const int a_ = (int)r;
      double acc = 0.0;
      for (int u = 0; u < Du; ++u)
        for (int U = 0; U < Du; ++U)
          for (int bb = 0; bb < b; ++bb)
            acc += (double)Tu[((int64_t)a_ * Du * Du + u * Du + U) * b + bb] *
                   B3[(((((int64_t)c_ * b + bb) * Dl + Lq_) * Du + U) * Dl + l) * Du + u];
      Rn[t] = acc;
    }
    __syncthreads();
  }
  // per column: cotangents of up, lo, ket (ket and bra slots are the same tensor)
  for (int q = 0; q < n; ++q) {
    const StripCol &c = cols[g.col0 + q];
    const StripBwdCol &o = bcols[g.col0 + q];
    fwd(q, L(q));
    bwd(q, R(q + 1));
    const double *Lq = L(q), *Rq = R(q + 1);
    const int a = c.a, b = c.b, cc = c.c, f = c.f, d = c.d, Dl = c.Dl, Du = c.Du, Dx = c.Dx, De = c.De;
    const double *op = g.op[q] >= 0 ? ops + (int64_t)g.op[q] * d * d : nullptr;
    if (o.cot_up)
      for (int64_t t = threadIdx.x; t < (int64_t)a * Du * Du * b; t += NTB) {
        int64_t r = t;
        const int bb = (int)(r % b); r /= b;
        const int U = (int)(r % Du); r /= Du;
        const int u = (int)(r % Du); r /= Du;
        const int a_ = (int)r;
        double acc = 0.0;
        for (int l = 0; l < Dl; ++l)
          for (int Lq_ = 0; Lq_ < Dl; ++Lq_)
            for (int c_ = 0; c_ < cc; ++c_)
              acc += Lq[(((int64_t)a_ * Dl + l) * Dl + Lq_) * cc + c_] *
                     B3[(((((int64_t)c_ * b + bb) * Dl + Lq_) * Du + U) * Dl + l) * Du + u];
        add_to<T>(o.cot_up, t, w * acc);
      }
    if (o.cot_lo)
      for (int64_t t = threadIdx.x; t < (int64_t)cc * Dx * Dx * f; t += NTB) {
        int64_t r = t;
        const int ff = (int)(r % f); r /= f;
        const int X = (int)(r % Dx); r /= Dx;
        const int x = (int)(r % Dx); r /= Dx;
        const int c_ = (int)r;
        double acc = 0.0;
        for (int bb = 0; bb < b; ++bb)
          for (int e = 0; e < De; ++e)
            for (int E = 0; E < De; ++E)
              acc += A3[((((int64_t)c_ * b + bb) * De + e) * Dx + x) * Dx * De + (int64_t)X * De + E] *
                     Rq[(((int64_t)bb * De + e) * De + E) * f + ff];
        add_to<T>(o.cot_lo, t, w * acc);
      }
    // env of K' (ket slot) and of K (bra slot), both [s][l][u][x][e]
    for (int64_t t = threadIdx.x; t < (int64_t)d * Dl * Du * Dx * De; t += NTB) {
      int64_t r = t;
      const int e = (int)(r % De); r /= De;
      const int x = (int)(r % Dx); r /= Dx;
      const int u = (int)(r % Du); r /= Du;
      const int l = (int)(r % Dl); r /= Dl;
      const int s_ = (int)r;
      // bra slot: sum_{c,b,x',e'} A2[L=l][c][U=u][b][s][x'][e'] B1[c][x'][X=x][b][e'][E=e]
      double bra = 0.0;
      for (int c_ = 0; c_ < cc; ++c_)
        for (int bb = 0; bb < b; ++bb)
          for (int x2 = 0; x2 < Dx; ++x2)
            for (int e2 = 0; e2 < De; ++e2)
              bra += A2[((((((int64_t)l * cc + c_) * Du + u) * b + bb) * d + s_) * Dx + x2) * De + e2] *
                     B1[((((((int64_t)c_ * Dx + x2) * Dx + x) * b + bb) * De + e2) * De + e)];
      // ket slot env_K'[s][l][u][x][e] = sum_{L,c,U,b} A1[l][L][c][u][U][b] B2[c][x][b][e][s][L][U];
      // d/dK[s2] of K'[s] = op[s][s2]: ket part at s = sum_{s'} op[s'][s] env_K'[s']
      double ket = 0.0;
      for (int s2 = 0; s2 < d; ++s2) {
        const double coef = op ? op[s2 * d + s_] : (s2 == s_ ? 1.0 : 0.0);
        if (coef == 0.0) continue;
        double env = 0.0;
        for (int Lq_ = 0; Lq_ < Dl; ++Lq_)
          for (int c_ = 0; c_ < cc; ++c_)
            for (int U = 0; U < Du; ++U)
              for (int bb = 0; bb < b; ++bb)
                env += A1[((((int64_t)(l * Dl + Lq_) * cc + c_) * Du + u) * Du + U) * b + bb] *
                       B2[((((((int64_t)c_ * Dx + x) * b + bb) * De + e) * d + s2) * Dl + Lq_) * Du + U];
        ket += coef * env;
      }
      add_to<T>(o.cot_ket, t, w * (ket + bra));
    }
    __syncthreads();
  }
}

// Row one: S[(l,L)][(x,X)][(e,E)] = sum_s K[s,l,0,x,e] K[s,L,0,X,E] (up bond 1)
template <class T> __global__ void first_row_bwd_kernel(SiteBwdDesc g) {
  const int d = g.d, Dl = g.Dl, Dx = g.Dx, De = g.De;
  const T *K = (const T *)g.K, *cot = (const T *)g.cot;
  const int64_t n = (int64_t)d * Dl * Dx * De;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int64_t r = t;
  const int e = (int)(r % De); r /= De;
  const int x = (int)(r % Dx); r /= Dx;
  const int l = (int)(r % Dl); r /= Dl;
  const int s = (int)r;
  double acc = 0.0;   // ket and bra slots of the same tensor give the same sum (cot read both ways)
  for (int L = 0; L < Dl; ++L)
    for (int X = 0; X < Dx; ++X)
      for (int E = 0; E < De; ++E) {
        const double kv = (double)K[(((int64_t)s * Dl + L) * Dx + X) * De + E];
        acc += kv * ((double)cot[(((int64_t)(l * Dl + L) * Dx * Dx + x * Dx + X) * De * De) + e * De + E] +
                     (double)cot[(((int64_t)(L * Dl + l) * Dx * Dx + X * Dx + x) * De * De) + E * De + e]);
      }
  add_to<T>(g.Kbar, (((int64_t)s * Dl + l) * 1 + 0) * Dx * De + (int64_t)x * De + e, acc);
}

// First zip-up carry: V[(x,X)][b][(e,E)] = sum_{u,U} S[(u,U)][b] sum_s K[s,0,u,x,e] K[s,0,U,X,E] (left bond 1)
template <class T> __global__ void zipup_start_bwd_kernel(SiteBwdDesc g) {
  const int d = g.d, Du = g.Du, Dx = g.Dx, De = g.De, B = g.B;
  const T *K = (const T *)g.K, *S = (const T *)g.S, *cot = (const T *)g.cot;
  const int64_t nk = (int64_t)d * Du * Dx * De, ns = (int64_t)Du * Du * B;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto Kv = [&](int s, int u, int x, int e) { return (double)K[(((int64_t)s * Du + u) * Dx + x) * De + e]; };
  auto C = [&](int x, int X, int b, int e, int E) {
    return (double)cot[((((int64_t)x * Dx + X) * B + b) * De + e) * De + E];
  };
  if (t < nk) {
    int64_t r = t;
    const int e = (int)(r % De); r /= De;
    const int x = (int)(r % Dx); r /= Dx;
    const int u = (int)(r % Du); r /= Du;
    const int s = (int)r;
    double acc = 0.0;   // ket slot + bra slot of the same tensor
    for (int U = 0; U < Du; ++U)
      for (int b = 0; b < B; ++b)
        for (int X = 0; X < Dx; ++X)
          for (int E = 0; E < De; ++E) {
            const double kv = Kv(s, U, X, E);
            acc += kv * ((double)S[((int64_t)u * Du + U) * B + b] * C(x, X, b, e, E) +
                         (double)S[((int64_t)U * Du + u) * B + b] * C(X, x, b, E, e));
          }
    add_to<T>(g.Kbar, t, acc);
  } else if (t < nk + ns) {
    int64_t r = t - nk;
    const int b = (int)(r % B); r /= B;
    const int U = (int)(r % Du); r /= Du;
    const int u = (int)r;
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int x = 0; x < Dx; ++x)
        for (int X = 0; X < Dx; ++X)
          for (int e = 0; e < De; ++e)
            for (int E = 0; E < De; ++E) acc += C(x, X, b, e, E) * Kv(s, u, x, e) * Kv(s, U, X, E);
    add_to<T>(g.Sbar, ((int64_t)u * Du + U) * B + b, acc);
  }
}

template <class T> __global__ void axpy_kernel(const T *x, T *y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

}  // namespace

void launch_strip_bwd(int dt, const StripDesc *d, const StripCol *cols, const StripBwdCol *bcols, const double *ops,
                      const double *sbar, const StripBwdScratch &sc, int nd, cudaStream_t s) {
  if (nd <= 0) return;
  if (dt == DT_R32) strip_bwd_kernel<float><<<nd, NTB, 0, s>>>(d, cols, bcols, ops, sbar, sc);
  else if (dt == DT_R64) strip_bwd_kernel<double><<<nd, NTB, 0, s>>>(d, cols, bcols, ops, sbar, sc);
}

void launch_site_bwd(int dt, const SiteBwdDesc &d, cudaStream_t s) {
  const int64_t n = d.mode == 0 ? (int64_t)d.d * d.Dl * d.Dx * d.De
                                : (int64_t)d.d * d.Du * d.Dx * d.De + (int64_t)d.Du * d.Du * d.B;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (!blocks) return;
  if (d.mode == 0) {
    if (dt == DT_R32) first_row_bwd_kernel<float><<<blocks, 256, 0, s>>>(d);
    else if (dt == DT_R64) first_row_bwd_kernel<double><<<blocks, 256, 0, s>>>(d);
  } else {
    if (dt == DT_R32) zipup_start_bwd_kernel<float><<<blocks, 256, 0, s>>>(d);
    else if (dt == DT_R64) zipup_start_bwd_kernel<double><<<blocks, 256, 0, s>>>(d);
  }
}

void launch_axpy(int dt, const void *x, void *y, int64_t n, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (!blocks) return;
  if (dt == DT_R32) axpy_kernel<float><<<blocks, 256, 0, s>>>((const float *)x, (float *)y, n);
  else if (dt == DT_R64) axpy_kernel<double><<<blocks, 256, 0, s>>>((const double *)x, (double *)y, n);
}

}  // namespace peps
