// Scalar helpers shared by the libpeps kernels: one set of overloads for the
// four element types (float, double, float2 = complex float, double2 =
// complex double) so every kernel is written once as a template.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PEPS_HD __host__ __device__ __forceinline__

namespace peps {

template <class T> struct Traits;
template <> struct Traits<float>   { using Real = float;  using Acc = double;  static constexpr bool cplx = false; };
template <> struct Traits<double>  { using Real = double; using Acc = double;  static constexpr bool cplx = false; };
template <> struct Traits<float2>  { using Real = float;  using Acc = double2; static constexpr bool cplx = true; };
template <> struct Traits<double2> { using Real = double; using Acc = double2; static constexpr bool cplx = true; };

// ---- construction -------------------------------------------------------
template <class T> PEPS_HD T zero();
template <> PEPS_HD float zero<float>() { return 0.f; }
template <> PEPS_HD double zero<double>() { return 0.0; }
template <> PEPS_HD float2 zero<float2>() { return make_float2(0.f, 0.f); }
template <> PEPS_HD double2 zero<double2>() { return make_double2(0.0, 0.0); }

template <class T> PEPS_HD T from_parts(double re, double im);
template <> PEPS_HD float from_parts<float>(double re, double) { return (float)re; }
template <> PEPS_HD double from_parts<double>(double re, double) { return re; }
template <> PEPS_HD float2 from_parts<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> PEPS_HD double2 from_parts<double2>(double re, double im) { return make_double2(re, im); }

// ---- parts --------------------------------------------------------------
PEPS_HD float re(float a) { return a; }
PEPS_HD double re(double a) { return a; }
PEPS_HD float re(float2 a) { return a.x; }
PEPS_HD double re(double2 a) { return a.x; }
PEPS_HD float im(float) { return 0.f; }
PEPS_HD double im(double) { return 0.0; }
PEPS_HD float im(float2 a) { return a.y; }
PEPS_HD double im(double2 a) { return a.y; }

// ---- arithmetic ----------------------------------------------------------
PEPS_HD float conj_(float a) { return a; }
PEPS_HD double conj_(double a) { return a; }
PEPS_HD float2 conj_(float2 a) { return make_float2(a.x, -a.y); }
PEPS_HD double2 conj_(double2 a) { return make_double2(a.x, -a.y); }

PEPS_HD float add(float a, float b) { return a + b; }
PEPS_HD double add(double a, double b) { return a + b; }
PEPS_HD float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
PEPS_HD double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

PEPS_HD float sub(float a, float b) { return a - b; }
PEPS_HD double sub(double a, double b) { return a - b; }
PEPS_HD float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
PEPS_HD double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

PEPS_HD float mul(float a, float b) { return a * b; }
PEPS_HD double mul(double a, double b) { return a * b; }
PEPS_HD float2 mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
PEPS_HD double2 mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// c + a * b
PEPS_HD float fma_(float a, float b, float c) { return fmaf(a, b, c); }
PEPS_HD double fma_(double a, double b, double c) { return fma(a, b, c); }
PEPS_HD float2 fma_(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.y, b.y, fmaf(a.x, b.x, c.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, c.y)));
}
PEPS_HD double2 fma_(double2 a, double2 b, double2 c) {
  return make_double2(fma(-a.y, b.y, fma(a.x, b.x, c.x)), fma(a.y, b.x, fma(a.x, b.y, c.y)));
}

PEPS_HD float scale(float a, float s) { return a * s; }
PEPS_HD double scale(double a, double s) { return a * s; }
PEPS_HD float2 scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
PEPS_HD double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

PEPS_HD float abs2(float a) { return a * a; }
PEPS_HD double abs2(double a) { return a * a; }
PEPS_HD float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
PEPS_HD double abs2(double2 a) { return a.x * a.x + a.y * a.y; }

// conditional conjugate
template <class T> PEPS_HD T cj(T a, bool c) { return c ? conj_(a) : a; }

// ---- widening / narrowing between working and accumulation types ---------
PEPS_HD double widen(float a) { return (double)a; }
PEPS_HD double widen(double a) { return a; }
PEPS_HD double2 widen(float2 a) { return make_double2(a.x, a.y); }
PEPS_HD double2 widen(double2 a) { return a; }

template <class T> PEPS_HD T narrow(double a);
template <class T> PEPS_HD T narrow(double2 a);
template <> PEPS_HD float narrow<float>(double a) { return (float)a; }
template <> PEPS_HD double narrow<double>(double a) { return a; }
template <> PEPS_HD float2 narrow<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> PEPS_HD double2 narrow<double2>(double2 a) { return a; }

PEPS_HD bool finite_(float a) { return isfinite(a); }
PEPS_HD bool finite_(double a) { return isfinite(a); }
PEPS_HD bool finite_(float2 a) { return isfinite(a.x) && isfinite(a.y); }
PEPS_HD bool finite_(double2 a) { return isfinite(a.x) && isfinite(a.y); }

#ifdef __CUDACC__
__device__ __forceinline__ void atomic_add_acc(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_acc(double2 *p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}
#endif

// Integer helpers
PEPS_HD int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device status word bits (written by kernels, read back by the host).
enum : uint32_t {
  STATUS_NONFINITE = 1u << 0,   // a non-finite Gram / singular value met
  STATUS_JACOBI_NOCONV = 1u << 1,
  STATUS_TIMEOUT = 1u << 2,
};

}  // namespace peps
