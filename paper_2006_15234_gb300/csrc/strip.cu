// Exact strip contractions of the cached-environment expectation value
// (Eq. 6 with the environments of Sec. IV-B): for a row r, the boundary MPS
// above it, the row's ket and bra sites (one-site operators applied to the
// ket's physical index where a term acts) and the boundary below it are
// contracted left to right into one scalar.
//
// The running left block L[a][l][L][c] (upper bond a, ket bond l, bra bond L,
// lower bond c) absorbs one column per step in four contractions:
//   A1[l][L][c][u][U][b]      = sum_a       L[a][l][L][c] T[a][(u,U)][b]
//   A2[L][c][U][b][s][x][e]   = sum_{l,u}   A1 K'[s][l][u][x][e]
//   A3[c][b][e][x][X][E]      = sum_{s,L,U} A2 conj(K[s][L][U][X][E])
//   L'[b][e][E][f]            = sum_{c,x,X} A3 Bl[c][(x,X)][f]
// with K' = op K on the physical index.  One CTA per strip; the blocks live
// in a per-strip slice of global scratch (they are small: m^2 D^4 values at
// most); every sum is accumulated in FP64.  Element indices are decomposed in
// 32-bit arithmetic (the planner keeps every block below 2^31 elements; a
// 64-bit division runs through FP64 operations, which this GPU issues at
// 1/64 of the FP32 rate).
#include "common.cuh"
#include "kernels.h"

namespace peps {

namespace {

constexpr int kStripThreads = 256;

template <class T>
__global__ void __launch_bounds__(kStripThreads) strip_kernel(const StripDesc *__restrict__ descs,
                                                              const StripCol *__restrict__ cols,
                                                              const void *__restrict__ op_table) {
  using Acc = typename Traits<T>::Acc;
  const StripDesc &g = descs[blockIdx.x];
  Acc *Lb = (Acc *)g.scratch;
  Acc *A1 = Lb + g.l_cap;
  Acc *A2 = A1 + g.a1_cap;
  Acc *A3 = A2 + g.a2_cap;
  const Acc *ops = (const Acc *)op_table;
  if (threadIdx.x == 0) Lb[0] = from_parts<Acc>(1.0, 0.0);
  __syncthreads();
  for (int q = 0; q < g.ncol; ++q) {
    const StripCol &c = cols[g.col0 + q];
    const T *Tu = (const T *)c.up, *Bl = (const T *)c.lo, *K = (const T *)c.ket;
    const int a = c.a, b = c.b, cc = c.c, f = c.f, d = c.d;
    const int Dl = c.Dl, Du = c.Du, Dx = c.Dx, De = c.De;   // ket = bra shapes
    const int vu = Du * Du, vd = Dx * Dx;
    const Acc *op = g.op[q] >= 0 ? ops + (int64_t)g.op[q] * d * d : nullptr;
    // A1[l][L][c][u][U][b]
    {
      const int64_t n = (int64_t)Dl * Dl * cc * vu * b;
      for (uint32_t t = threadIdx.x; t < (uint32_t)n; t += kStripThreads) {
        uint32_t r = t;
        const int bb = (int)(r % b); r /= b;
        const int uU = (int)(r % vu); r /= vu;
        const int c_ = (int)(r % cc); r /= cc;
        const int lL = (int)r;                                  // l * Dl + L
        Acc s = zero<Acc>();
        for (int a_ = 0; a_ < a; ++a_)
          s = fma_(Lb[((int64_t)a_ * Dl * Dl + lL) * cc + c_], widen(Tu[((int64_t)a_ * vu + uU) * b + bb]), s);
        A1[t] = s;
      }
    }
    __syncthreads();
    // A2[L][c][U][b][s][x][e]
    {
      const int64_t n = (int64_t)Dl * cc * Du * b * d * Dx * De;
      for (uint32_t t = threadIdx.x; t < (uint32_t)n; t += kStripThreads) {
        uint32_t r = t;
        const int e = (int)(r % De); r /= De;
        const int x = (int)(r % Dx); r /= Dx;
        const int s_ = (int)(r % d); r /= d;
        const int bb = (int)(r % b); r /= b;
        const int U = (int)(r % Du); r /= Du;
        const int c_ = (int)(r % cc); r /= cc;
        const int L = (int)r;
        Acc acc = zero<Acc>();
        for (int l = 0; l < Dl; ++l)
          for (int u = 0; u < Du; ++u) {
            Acc kv;
            if (op) {
              kv = zero<Acc>();
              for (int s2 = 0; s2 < d; ++s2)
                kv = fma_(op[s_ * d + s2], widen(K[((((int64_t)s2 * Dl + l) * Du + u) * Dx + x) * De + e]), kv);
            } else {
              kv = widen(K[((((int64_t)s_ * Dl + l) * Du + u) * Dx + x) * De + e]);
            }
            const Acc a1 = A1[((((int64_t)(l * Dl + L) * cc + c_) * Du + u) * Du + U) * b + bb];
            acc = fma_(a1, kv, acc);
          }
        A2[t] = acc;
      }
    }
    __syncthreads();
    // A3[c][b][e][x][X][E]
    {
      const int64_t n = (int64_t)cc * b * De * Dx * Dx * De;
      for (uint32_t t = threadIdx.x; t < (uint32_t)n; t += kStripThreads) {
        uint32_t r = t;
        const int E = (int)(r % De); r /= De;
        const int X = (int)(r % Dx); r /= Dx;
        const int x = (int)(r % Dx); r /= Dx;
        const int e = (int)(r % De); r /= De;
        const int bb = (int)(r % b); r /= b;
        const int c_ = (int)r;
        Acc acc = zero<Acc>();
        for (int s_ = 0; s_ < d; ++s_)
          for (int L = 0; L < Dl; ++L)
            for (int U = 0; U < Du; ++U) {
              const Acc a2 = A2[((((((int64_t)L * cc + c_) * Du + U) * b + bb) * d + s_) * Dx + x) * De + e];
              const Acc kb = conj_(widen(K[((((int64_t)s_ * Dl + L) * Du + U) * Dx + X) * De + E]));
              acc = fma_(a2, kb, acc);
            }
        A3[t] = acc;
      }
    }
    __syncthreads();
    // L'[b][e][E][f]
    {
      const int64_t n = (int64_t)b * De * De * f;
      for (uint32_t t = threadIdx.x; t < (uint32_t)n; t += kStripThreads) {
        uint32_t r = t;
        const int ff = (int)(r % f); r /= f;
        const int E = (int)(r % De); r /= De;
        const int e = (int)(r % De); r /= De;
        const int bb = (int)r;
        Acc acc = zero<Acc>();
        for (int c_ = 0; c_ < cc; ++c_)
          for (int x = 0; x < Dx; ++x)
            for (int X = 0; X < Dx; ++X) {
              const Acc a3 = A3[((((int64_t)c_ * b + bb) * De + e) * Dx + x) * Dx * De + (int64_t)X * De + E];
              acc = fma_(a3, widen(Bl[((int64_t)c_ * vd + x * Dx + X) * f + ff]), acc);
            }
        Lb[t] = acc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ((Acc *)g.out)[0] = Lb[0];
}

}  // namespace

void launch_strip(int dt, const StripDesc *d, const StripCol *cols, const void *ops, int nd, cudaStream_t s) {
  if (nd <= 0) return;
  switch (dt) {
    case DT_R32: strip_kernel<float><<<nd, kStripThreads, 0, s>>>(d, cols, ops); break;
    case DT_C64: strip_kernel<float2><<<nd, kStripThreads, 0, s>>>(d, cols, ops); break;
    case DT_R64: strip_kernel<double><<<nd, kStripThreads, 0, s>>>(d, cols, ops); break;
    case DT_C128: strip_kernel<double2><<<nd, kStripThreads, 0, s>>>(d, cols, ops); break;
  }
}

}  // namespace peps
