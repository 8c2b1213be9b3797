// C ABI of libpeps (declared in include/libpeps.h): argument checking, plan
// objects, descriptor upload and launch of the static schedules built by
// step.cu (one einsumsvd) and by the boundary sweep below (Algorithms 2, 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/libpeps.h"
#include "common.cuh"
#include "plan.h"
#include "tcgemm.h"

using namespace peps;

namespace {

thread_local std::string g_last_error;

peps_status fail(peps_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(PEPS_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
  } while (0)

bool valid_dtype(int dt) { return dt >= 0 && dt <= 3; }

peps_status check_opts(const peps_rsvd_opts *o) {
  if (!o) return fail(PEPS_ERR_ARG, "opts is NULL");
  if (o->m < 1) return fail(PEPS_ERR_ARG, "m must be >= 1 (got %d)", o->m);
  if (o->p < 0) return fail(PEPS_ERR_ARG, "p must be >= 0 (got %d)", o->p);
  if (o->q < 0) return fail(PEPS_ERR_ARG, "q must be >= 0 (got %d)", o->q);
  if (o->sketch != PEPS_SKETCH_GAUSS && o->sketch != PEPS_SKETCH_UNIFORM)
    return fail(PEPS_ERR_ARG, "unknown sketch kind %d", o->sketch);
  if (o->prec != PEPS_PREC_PLAIN && o->prec != PEPS_PREC_MIXED && o->prec != PEPS_PREC_FAST)
    return fail(PEPS_ERR_ARG, "unknown precision %d", o->prec);
  if (o->flags & ~PEPS_FLAG_ORTH_Q) return fail(PEPS_ERR_ARG, "unknown flag bits %#x", o->flags);
  return PEPS_OK;
}

RsvdOpts to_opts(const peps_rsvd_opts *o) {
  RsvdOpts r;
  r.m = o->m; r.p = o->p; r.q = o->q; r.seed = o->seed; r.sketch = o->sketch; r.prec = o->prec;
  r.orth_q = (o->flags & PEPS_FLAG_ORTH_Q) != 0;
  return r;
}

bool in_capture(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// ---- network bookkeeping --------------------------------------------------

struct SiteDims { int d, Dl, Du, Dx, De; };

struct Net {
  int nrow, ncol, d, dt;
  std::vector<SiteDims> dims;           // row-major
  std::vector<const void *> site;
  const SiteDims &at(int p, int q) const { return dims[(size_t)p * ncol + q]; }
  const void *ptr(int p, int q) const { return site[(size_t)p * ncol + q]; }
};

peps_status read_net(const peps_network *n, Net &out, const char *which) {
  if (!n) return fail(PEPS_ERR_ARG, "%s network is NULL", which);
  if (n->nrow < 1 || n->ncol < 1 || n->d < 1)
    return fail(PEPS_ERR_SHAPE, "%s: nrow, ncol and d must be >= 1", which);
  if (!valid_dtype(n->dtype)) return fail(PEPS_ERR_ARG, "%s: bad dtype %d", which, n->dtype);
  if (!n->site) return fail(PEPS_ERR_ARG, "%s: site array is NULL", which);
  if ((n->ncol > 1 && !n->bond_h) || (n->nrow > 1 && !n->bond_v))
    return fail(PEPS_ERR_ARG, "%s: bond arrays are NULL", which);
  out.nrow = n->nrow; out.ncol = n->ncol; out.d = n->d; out.dt = n->dtype;
  out.dims.resize((size_t)n->nrow * n->ncol);
  out.site.resize((size_t)n->nrow * n->ncol);
  for (int p = 0; p < n->nrow; ++p)
    for (int q = 0; q < n->ncol; ++q) {
      SiteDims s;
      s.d = n->d;
      s.Dl = q > 0 ? n->bond_h[(size_t)p * (n->ncol - 1) + q - 1] : 1;
      s.De = q < n->ncol - 1 ? n->bond_h[(size_t)p * (n->ncol - 1) + q] : 1;
      s.Du = p > 0 ? n->bond_v[(size_t)(p - 1) * n->ncol + q] : 1;
      s.Dx = p < n->nrow - 1 ? n->bond_v[(size_t)p * n->ncol + q] : 1;
      if (s.Dl < 1 || s.De < 1 || s.Du < 1 || s.Dx < 1)
        return fail(PEPS_ERR_SHAPE, "%s: bond dimensions must be >= 1", which);
      out.dims[(size_t)p * n->ncol + q] = s;
      out.site[(size_t)p * n->ncol + q] = n->site[(size_t)p * n->ncol + q];
      if (!n->site[(size_t)p * n->ncol + q]) return fail(PEPS_ERR_ARG, "%s: site (%d,%d) is NULL", which, p, q);
    }
  return PEPS_OK;
}

}  // namespace

// ---- plans ------------------------------------------------------------------

struct peps_plan {
  enum Kind { EINSUMSVD, CONTRACT } kind;
  int dt = 0;
  RsvdOpts opts{};
  // einsumsvd
  std::vector<Inst> insts;
  std::vector<peps_einsumsvd_io> io_cache;
  // contraction
  Net ket, bra;
  bool one_layer = false;
  int direction = 0;
  int64_t nsigma = 0;
  size_t result_off = 0, sigma_off = 0;
  // built schedule
  uintptr_t built_base = 0;
  bool built = false;
  std::vector<Op> ops;
  std::vector<uint8_t> blob;
  size_t blob_off = 0;
  size_t ws_bytes = 0;
};

namespace {

size_t finish(Builder &B, size_t *blob_off) {
  *blob_off = (B.top + 255) & ~(size_t)255;
  return *blob_off + B.blob.size();
}

// Build the einsumsvd schedule (io may be null while sizing).
std::string build_einsumsvd(peps_plan *P, uintptr_t base, const peps_einsumsvd_io *io, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  std::vector<Inst *> ptrs;
  for (size_t i = 0; i < P->insts.size(); ++i) {
    Inst &I = P->insts[i];
    inst_alloc_scratch(B, I, P->dt);
    I.logp = (double *)B.buf(8);
    if (io) {
      I.V = io[i].V; I.S = io[i].S; I.K = io[i].ket; I.Kb = io[i].bra;
      I.U = io[i].U; I.W = io[i].W; I.sigma = io[i].sigma;
      if (io[i].log_scale) I.logp = io[i].log_scale;
    }
    ptrs.push_back(&I);
  }
  emit_einsumsvd(B, ptrs, P->opts);
  return "";
}

// Boundary sweep of Algorithms 2 and 3 over the whole network.
std::string build_contract(peps_plan *P, uintptr_t base, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  const Net &K = P->ket;
  const int nrow = K.nrow, ncol = K.ncol, dt = P->dt;
  const size_t es = dtype_size(dt);
  auto bra_dims = [&](int p, int q) -> SiteDims {
    if (P->one_layer) return SiteDims{1, 1, 1, 1, 1};
    return P->bra.at(p, q);
  };
  // --- shapes of every boundary site and einsumsvd step
  struct Site { int left, vert, right; };
  std::vector<std::vector<Site>> bound(nrow);
  std::vector<std::vector<Inst>> steps(nrow);
  for (int q = 0; q < ncol; ++q) {
    const SiteDims k = K.at(0, q), b = bra_dims(0, q);
    bound[0].push_back(Site{k.Dl * b.Dl, k.Dx * b.Dx, k.De * b.De});
  }
  size_t max_site = 0, max_carry = 0;
  for (auto &s : bound[0]) max_site = std::max(max_site, (size_t)s.left * s.vert * s.right);
  int64_t nsteps = 0, nsigma = 0;
  for (int r = 1; r < nrow; ++r) {
    bound[r].resize(ncol);
    // V1 = [1][t0][b0][h0]
    const SiteDims k0 = K.at(r, 0), b0 = bra_dims(r, 0);
    {
      const Site &s0 = bound[r - 1][0];
      if (s0.vert != k0.Du * b0.Du) return "vertical bond mismatch between rows";
      max_carry = std::max(max_carry, (size_t)k0.Dx * b0.Dx * s0.right * k0.De * b0.De);
    }
    int kprev = 1;
    for (int i = 1; i < ncol; ++i) {
      const SiteDims kp = K.at(r, i - 1), bp = bra_dims(r, i - 1);
      const SiteDims kc = K.at(r, i), bc = bra_dims(r, i);
      const Site &S = bound[r - 1][i];
      Inst I{};
      I.kL = kprev; I.t = kp.Dx * bp.Dx; I.a = S.left; I.b = S.right;
      I.d = kc.d; I.Dl = kc.Dl; I.Du = kc.Du; I.Dx = kc.Dx; I.De = kc.De;
      I.DL = bc.Dl; I.DU = bc.Du; I.DX = bc.Dx; I.DE = bc.De;
      if (kp.De != kc.Dl || bp.De != bc.Dl) return "horizontal bond mismatch";
      if (S.vert != kc.Du * bc.Du) return "vertical bond mismatch between rows";
      if (!P->one_layer && kc.d != bc.d) return "ket and bra physical dimensions differ";
      inst_derive(I, P->opts);
      std::string e = inst_check(I, dt);
      if (!e.empty()) return e;
      I.instance = ((uint64_t)P->direction << 32) | ((uint64_t)r << 16) | (uint64_t)i;
      I.tc = P->opts.prec != PEPS_PREC_PLAIN && inst_tc_ok(I, dt);
      bound[r][i - 1] = Site{I.kL, I.t, I.k};
      max_carry = std::max(max_carry, (size_t)I.kL * I.t * I.a * I.h);
      max_carry = std::max(max_carry, (size_t)I.k * I.N);
      steps[r].push_back(I);
      kprev = I.k;
      ++nsteps;
      nsigma += I.k;
    }
    const SiteDims kl = K.at(r, ncol - 1), bl = bra_dims(r, ncol - 1);
    bound[r][ncol - 1] = Site{kprev, kl.Dx * bl.Dx, 1};
    for (auto &s : bound[r]) max_site = std::max(max_site, (size_t)s.left * s.vert * s.right);
  }
  P->nsigma = nsigma;
  // --- buffers
  Inst owner{};
  {
    // scratch sized by the largest step in each dimension
    int64_t xN = 0, t2 = 0, t3 = 0, yM = 0, ell = 1, kk = 1;
    for (auto &row : steps)
      for (auto &I : row) {
        xN = std::max<int64_t>(xN, (int64_t)I.ell * I.N);
        t2 = std::max<int64_t>(t2, (int64_t)I.ell * I.h * I.v * I.b);
        t3 = std::max<int64_t>(t3, (int64_t)I.ell * I.a * I.h);
        yM = std::max<int64_t>(yM, (int64_t)I.ell * I.M);
        ell = std::max<int64_t>(ell, I.ell);
        kk = std::max<int64_t>(kk, I.k);
      }
    const size_t as = acc_size(dt);
    owner.X = B.buf(xN * es); owner.Z = B.buf(xN * es);
    owner.T2 = B.buf(t2 * es); owner.T3 = B.buf(t3 * es);
    owner.Y = B.buf(yM * es); owner.P = B.buf(yM * es);
    owner.g = B.buf(std::max<int64_t>(yM, 1) * es);
    owner.Tm = B.buf(ell * ell * es); owner.Ut = B.buf(ell * kk * es);
    owner.G = B.buf(ell * ell * as); owner.R1 = B.buf(ell * ell * as); owner.R2 = B.buf(ell * ell * as);
    owner.Rout = B.buf(ell * ell * as); owner.Mw = B.buf(ell * ell * as);
    owner.sig = (double *)B.buf(ell * 8); owner.inv_s1 = (double *)B.buf(8);
    int64_t t1 = 0, vt = 0, st = 0, ut = 0, kt = 0, kb = 0;
    for (auto &row : steps)
      for (auto &I : row) {
        if (!I.tc) continue;
        const int64_t P1 = (int64_t)I.Dl * I.Du, Q1 = (int64_t)I.Dx * I.De, P2 = (int64_t)I.DL * I.DU,
                      Q2 = (int64_t)I.DX * I.DE;
        t1 = std::max<int64_t>(t1, (int64_t)I.ell * I.b * I.d * P1 * Q2);
        vt = std::max<int64_t>(vt, I.M * I.a * I.h);
        st = std::max<int64_t>(st, (int64_t)I.a * I.v * I.b);
        ut = std::max<int64_t>(ut, (int64_t)I.k * I.M);
        kt = std::max<int64_t>(kt, Q1 * I.d * P1);
        kb = std::max<int64_t>(kb, (int64_t)I.d * P2 * Q2);
      }
    owner.T1 = t1 ? B.buf(t1 * es) : nullptr;
    owner.VT = vt ? B.buf(vt * es) : nullptr;
    owner.ST = st ? B.buf(st * es) : nullptr;
    owner.UT = ut ? B.buf(ut * es) : nullptr;
    owner.KT = kt ? B.buf(kt * es) : nullptr;
    owner.KbP = kb ? B.buf(kb * es) : nullptr;
    owner.KbT = kb ? B.buf(kb * es) : nullptr;
  }
  void *Sbuf[2][64];
  if (ncol > 64) return "ncol above 64 is not supported";
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q < ncol; ++q) Sbuf[c][q] = B.buf(max_site * es);
  void *Vbuf[2] = {B.buf(std::max<size_t>(max_carry, 1) * es), B.buf(std::max<size_t>(max_carry, 1) * es)};
  double *logs = (double *)B.buf(std::max<int64_t>(nsteps, 1) * 8);
  P->sigma_off = B.alloc(std::max<int64_t>(nsigma, 1) * 8);
  double *sigma = (double *)B.ptr(P->sigma_off);
  P->result_off = B.alloc(16);
  double *result = (double *)B.ptr(P->result_off);
  int maxbond = 1;
  for (int q = 0; q < ncol; ++q)
    maxbond = std::max(maxbond, std::max(bound[nrow - 1][q].left, bound[nrow - 1][q].right));
  void *sc_scratch = B.buf((size_t)2 * maxbond * acc_size(dt));
  void *ones = B.buf(es);

  // --- ops
  auto bra_ptr = [&](int p, int q) -> const void * { return P->one_layer ? ones : P->bra.ptr(p, q); };
  if (P->one_layer) {
    Op f;
    f.kind = Op::FILL; f.fill_ptr = ones; f.fill_n = 1; f.fill_value = 1.0; f.tag = "init";
    B.ops.push_back(f);
  }
  auto push_site = [&](std::vector<SiteDesc> &d, const char *tag) {
    std::vector<int64_t> bl;
    std::vector<int64_t> prefix;
    int64_t tot = 0;
    for (auto &s : d) {
      prefix.push_back(tot);
      bl.push_back(ceil_div(s.total, kSiteThreads));
      tot += bl.back();
    }
    Op op;
    op.kind = Op::SITE; op.desc_off = B.put(d); op.prefix_off = B.put(prefix);
    op.nd = (int)d.size(); op.blocks = tot; op.tag = tag;
    B.ops.push_back(op);
  };
  {
    std::vector<SiteDesc> d;
    for (int q = 0; q < ncol; ++q) {
      const SiteDims k = K.at(0, q), b = bra_dims(0, q);
      SiteDesc s{};
      s.K = K.ptr(0, q); s.Kb = bra_ptr(0, q); s.S = nullptr; s.out = Sbuf[0][q]; s.mode = 0;
      s.d = k.d; s.Dl = k.Dl; s.Du = k.Du; s.Dx = k.Dx; s.De = k.De;
      s.DL = b.Dl; s.DU = b.Du; s.DX = b.Dx; s.DE = b.De; s.B = 1;
      s.total = (int64_t)k.Dl * b.Dl * k.Dx * b.Dx * k.De * b.De;
      d.push_back(s);
    }
    push_site(d, "first_row");
  }
  int cur = 0;
  int64_t step_idx = 0, sig_pos = 0;
  for (int r = 1; r < nrow; ++r) {
    const int nxt = 1 - cur;
    {
      const SiteDims k = K.at(r, 0), b = bra_dims(r, 0);
      SiteDesc s{};
      s.K = K.ptr(r, 0); s.Kb = bra_ptr(r, 0); s.S = Sbuf[cur][0];
      s.out = ncol == 1 ? Sbuf[nxt][0] : Vbuf[0];
      s.mode = 1;
      s.d = k.d; s.Dl = k.Dl; s.Du = k.Du; s.Dx = k.Dx; s.De = k.De;
      s.DL = b.Dl; s.DU = b.Du; s.DX = b.Dx; s.DE = b.De; s.B = bound[r - 1][0].right;
      s.total = (int64_t)k.Dx * b.Dx * s.B * k.De * b.De;
      std::vector<SiteDesc> d{s};
      push_site(d, "zipup_start");
    }
    int cv = 0;
    for (int i = 1; i < ncol; ++i) {
      Inst &I = steps[r][i - 1];
      inst_share_scratch(I, owner);
      I.V = Vbuf[cv];
      I.S = Sbuf[cur][i];
      I.K = K.ptr(r, i);
      I.Kb = bra_ptr(r, i);
      I.U = Sbuf[nxt][i - 1];
      I.W = (i == ncol - 1) ? Sbuf[nxt][ncol - 1] : Vbuf[1 - cv];
      I.sigma = sigma + sig_pos;
      I.logp = logs + step_idx;
      sig_pos += I.k;
      ++step_idx;
      std::vector<Inst *> one{&I};
      emit_einsumsvd(B, one, P->opts);
      cv = 1 - cv;
    }
    cur = nxt;
  }
  // --- final scalar
  std::vector<const void *> sp(ncol);
  std::vector<int32_t> lb(ncol), rb(ncol);
  for (int q = 0; q < ncol; ++q) {
    sp[q] = Sbuf[cur][q];
    lb[q] = bound[nrow - 1][q].left;
    rb[q] = bound[nrow - 1][q].right;
    if (bound[nrow - 1][q].vert != 1) return "last row has open vertical bonds";
  }
  Op sc;
  sc.kind = Op::SCALAR;
  sc.aux_off[0] = B.put(sp);
  sc.aux_off[1] = B.put(lb);
  sc.aux_off[2] = B.put(rb);
  sc.scalar.ncol = ncol;
  sc.scalar.logs = logs;
  sc.scalar.nlogs = (int)nsteps;
  sc.scalar.scratch = sc_scratch;
  sc.scalar.out = result;
  sc.tag = "scalar";
  B.ops.push_back(sc);
  return "";
}


// ---- host-side access validator ---------------------------------------------
// Recomputes, from every launch descriptor, the byte range each kernel may
// read or write and checks it lies inside the workspace or a caller tensor.
struct Extent { uintptr_t lo, hi; const char *what; };

struct Checker {
  std::vector<Extent> ext;
  std::string err;
  void need(const void *p, double nbytes, const char *op, const char *field) {
    if (!err.empty() || nbytes <= 0) return;
    if (!p) { err = std::string(op) + "." + field + " is NULL"; return; }
    const uintptr_t lo = (uintptr_t)p, hi = lo + (uintptr_t)nbytes;
    for (auto &e : ext)
      if (lo >= e.lo && hi <= e.hi) return;
    char b[256];
    snprintf(b, sizeof b, "%s.%s: [%#lx, +%.0f bytes) outside every buffer", op, field,
             (unsigned long)lo, nbytes);
    err = b;
  }
};

std::string validate_ops(const peps_plan *P, uintptr_t ws, size_t ws_bytes, Checker &C) {
  C.ext.push_back(Extent{ws, ws + ws_bytes, "workspace"});
  const int dt = P->dt;
  const double es = dtype_size(dt), as = acc_size(dt);
  const uint8_t *blob = P->blob.data();
  for (const Op &op : P->ops) {
    const char *tag = op.tag.c_str();
    const void *d = blob + op.desc_off;
    switch (op.kind) {
      case Op::GEMM:
      case Op::GEMM_ATOMIC:
        for (int i = 0; i < op.nd; ++i) {
          const GemmDesc &g = ((const GemmDesc *)d)[i];
          if (g.ksplit * (int64_t)g.kchunk < g.K) C.err = std::string(tag) + ": K chunks do not cover K";
          C.need(g.A, es * ((g.batch - 1) * (double)g.sAb + (g.M - 1) * (double)g.sAm + (g.K - 1) * (double)g.sAk + 1), tag, "A");
          C.need(g.B, es * ((g.batch - 1) * (double)g.sBb + (g.K - 1) * (double)g.sBk + (g.N - 1) * (double)g.sBn + 1), tag, "B");
          C.need(g.C, (op.kind == Op::GEMM_ATOMIC ? as : es) *
                          ((g.batch - 1) * (double)g.sCb + (g.M - 1) * (double)g.sCm + (g.N - 1) * (double)g.sCn + 1), tag, "C");
          if (g.alpha_dev) C.need(g.alpha_dev, 8, tag, "alpha_dev");
        }
        break;
      case Op::SANDWICH:
        for (int i = 0; i < op.nd; ++i) {
          const SandwichDesc &w = ((const SandwichDesc *)d)[i];
          const double N = (double)w.Dx * w.DX * w.B * w.De * w.DE;
          const double T2 = (double)w.Dl * w.DL * w.Du * w.DU * w.B;
          const double nin = w.adjoint ? T2 : N, nout = w.adjoint ? N : T2;
          if (w.ld_in < nin || w.ld_out < nout) C.err = std::string(tag) + ": leading dimension too small";
          C.need(w.in, es * ((w.ell - 1) * (double)w.ld_in + nin), tag, "in");
          C.need(w.out, es * ((w.ell - 1) * (double)w.ld_out + nout), tag, "out");
          C.need(w.K, es * w.d * w.Dl * w.Du * w.Dx * w.De, tag, "K");
          C.need(w.Kb, es * w.d * w.DL * w.DU * w.DX * w.DE, tag, "Kb");
          if ((int64_t)w.nblocks * w.items_per_block < (int64_t)w.ell * w.B) C.err = std::string(tag) + ": items not covered";
        }
        break;
      case Op::SKETCH:
        for (int i = 0; i < op.nd; ++i) {
          const SketchDesc &k = ((const SketchDesc *)d)[i];
          C.need(k.X, es * ((k.ell - 1) * (double)k.ld + k.N), tag, "X");
        }
        break;
      case Op::CHOL:
        for (int i = 0; i < op.nd; ++i) {
          const CholDesc &c = ((const CholDesc *)d)[i];
          const double n2 = (double)c.n * c.n;
          const double ws_ = op.wide ? as : es;        // working-type size
          C.need(c.G, as * n2, tag, "G");
          if (c.T) C.need(c.T, ws_ * n2, tag, "T");
          C.need(c.R, ws_ * n2, tag, "R");
          if (c.Rprev) { C.need(c.Rprev, ws_ * n2, tag, "Rprev"); C.need(c.Rout, ws_ * n2, tag, "Rout"); }
          if (c.Rlow) C.need(c.Rlow, es * n2, tag, "Rlow");
          if (c.Rlow && !op.wide) C.err = std::string(tag) + ": Rlow needs an FP64 factorisation";
          if (c.n > 1024) C.err = std::string(tag) + ": n above the pivot-flag buffer";
          if (op.smem < small_smem_bytes(op.wide ? (dt | 2) : dt, c.n))
            C.err = std::string(tag) + ": shared memory too small";
          if (op.smem2 < chol_cluster_smem_bytes(op.wide ? (dt | 2) : dt, c.n, c.T != nullptr))
            C.err = std::string(tag) + ": cluster shared memory too small";
        }
        break;
      case Op::JACOBI:
        for (int i = 0; i < op.nd; ++i) {
          const JacobiDesc &j = ((const JacobiDesc *)d)[i];
          C.need(j.Rb, es * (double)j.n * j.n, tag, "Rb");
          C.need(j.Mw, es * (double)j.n * j.n, tag, "Mw");
          if (op.smem < small_smem_bytes(dt, j.n)) C.err = std::string(tag) + ": shared memory too small";
          if (op.smem2 < jacobi_cluster_smem_bytes(dt, j.n)) C.err = std::string(tag) + ": cluster shared memory too small";
          if (op.blocks < j.n) C.err = std::string(tag) + ": sigma refinement grid too small";
          C.need(j.sig, 8.0 * j.n, tag, "sig");
        }
        break;
      case Op::FINALIZE:
        for (int i = 0; i < op.nd; ++i) {
          const FinalizeDesc &f = ((const FinalizeDesc *)d)[i];
          C.need(f.Mw, es * (double)f.n * f.n, tag, "Mw");
          C.need(f.sig, 8.0 * f.n, tag, "sig");
          C.need(f.P, es * (double)f.n * f.M, tag, "P");
          C.need(f.g, es * (double)f.M, tag, "g");
          C.need(f.Ut, es * (double)f.n * f.k, tag, "Ut");
          C.need(f.sigma_out, 8.0 * f.k, tag, "sigma_out");
          C.need(f.log_out, 8, tag, "log_out");
          C.need(f.inv_s1, 8, tag, "inv_s1");
          if (f.k > f.n || f.n > 1024) C.err = std::string(tag) + ": k > n or n > 1024";
        }
        break;
      case Op::ZERO:
        for (int i = 0; i < op.nd; ++i) {
          const ZeroDesc &z = ((const ZeroDesc *)d)[i];
          C.need(z.p, 8.0 * z.words, tag, "p");
        }
        break;
      case Op::SITE:
        for (int i = 0; i < op.nd; ++i) {
          const SiteDesc &s = ((const SiteDesc *)d)[i];
          C.need(s.K, es * s.d * s.Dl * s.Du * s.Dx * s.De, tag, "K");
          C.need(s.Kb, es * s.d * s.DL * s.DU * s.DX * s.DE, tag, "Kb");
          if (s.mode == 1) C.need(s.S, es * (double)s.Du * s.DU * s.B, tag, "S");
          C.need(s.out, es * (double)s.total, tag, "out");
        }
        break;
      case Op::SCALAR: {
        const ScalarDesc &sd = op.scalar;
        const void *const *sites = (const void *const *)(blob + op.aux_off[0]);
        const int32_t *lb = (const int32_t *)(blob + op.aux_off[1]);
        const int32_t *rb = (const int32_t *)(blob + op.aux_off[2]);
        int maxb = 1;
        for (int q = 0; q < sd.ncol; ++q) {
          C.need(sites[q], es * (double)lb[q] * rb[q], tag, "site");
          maxb = std::max(maxb, std::max(lb[q], rb[q]));
        }
        C.need(sd.scratch, 2.0 * maxb * as, tag, "scratch");
        C.need(sd.out, 16, tag, "out");
        C.need(sd.logs, 8.0 * sd.nlogs, tag, "logs");
        break;
      }
      case Op::FILL:
        C.need(op.fill_ptr, es * (double)op.fill_n, tag, "ptr");
        break;
      case Op::TC: {
        const TcDesc &t = op.tc;
        C.need(op.tcA, 4.0 * op.tcA_rows * op.tc_kr, tag, "A");
        C.need(op.tcB, 4.0 * op.tcB_rows * op.tc_kr, tag, "B");
        auto span = [](const DigitMap &m, int64_t extent) {
          double mx = 0;
          int64_t rest = extent - 1;
          for (int d = 0; d < m.n; ++d) {
            const int64_t dig = d == m.n - 1 ? rest : std::min<int64_t>(rest, (int64_t)m.radix[d] - 1);
            mx += (double)dig * m.stride[d];
            rest = d == m.n - 1 ? 0 : rest / m.radix[d];
          }
          return mx;
        };
        C.need(t.C, (t.atomic64 ? as : es) * (span(t.mm, t.M) + span(t.mn, t.N) + 1), tag, "C");
        if (t.ksplit > 1 && (int64_t)t.ksplit * t.kb_per_split * 32 < t.Kr)
          C.err = std::string(tag) + ": K chunks do not cover K";
        if (t.alpha_dev) C.need(t.alpha_dev, 8, tag, "alpha_dev");
        if (op.tc_kr % 4 || t.Kr != op.tc_kr) C.err = std::string(tag) + ": TMA rows not 16-byte aligned";
        break;
      }
      case Op::PERMUTE:
        for (int i = 0; i < op.nd; ++i) {
          const PermuteDesc &q = ((const PermuteDesc *)d)[i];
          const double n = (double)q.nb * q.R * q.Cc * q.Q;
          C.need(q.in, es * n, tag, "in");
          C.need(q.out, es * n, tag, "out");
        }
        break;
    }
    if (!C.err.empty()) return C.err;
  }
  if (P->blob_off + P->blob.size() > ws_bytes) return "descriptor blob beyond the workspace";
  return "";
}

peps_status rebuild(peps_plan *P, void *ws, const peps_einsumsvd_io *io, bool encode = false) {
  Builder B;
  B.encode = encode;
  std::string e = P->kind == peps_plan::EINSUMSVD ? build_einsumsvd(P, (uintptr_t)ws, io, B)
                                                   : build_contract(P, (uintptr_t)ws, B);
  if (!e.empty()) return fail(PEPS_ERR_SHAPE, "%s", e.c_str());
  if (!B.err.empty()) return fail(PEPS_ERR_UNSUPPORTED, "%s", B.err.c_str());
  P->ws_bytes = finish(B, &P->blob_off);   // needs the blob size: before the move
  P->ops = std::move(B.ops);
  P->blob = std::move(B.blob);
  return PEPS_OK;
}

peps_status enqueue(peps_plan *P, void *ws, size_t ws_bytes, cudaStream_t s, bool upload,
                    cudaEvent_t *events = nullptr) {
  if (!ws) return fail(PEPS_ERR_WORKSPACE, "workspace is NULL");
  if ((uintptr_t)ws & 255) return fail(PEPS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < P->ws_bytes)
    return fail(PEPS_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", ws_bytes, P->ws_bytes);
  uint8_t *blob = (uint8_t *)ws + P->blob_off;
  if (upload) {
    if (in_capture(s))
      return fail(PEPS_ERR_CAPTURE, "descriptor upload during stream capture; run once before capturing");
    CUDA_TRY(cudaMemcpyAsync(blob, P->blob.data(), P->blob.size(), cudaMemcpyHostToDevice, s));
  }
  const int dt = P->dt;
  if (events) CUDA_TRY(cudaEventRecord(events[0], s));
  for (const Op &op : P->ops) {
    const void *d = blob + op.desc_off;
    const int64_t *pre = (const int64_t *)(blob + op.prefix_off);
    switch (op.kind) {
      case Op::SKETCH: launch_sketch(dt, (const SketchDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::GEMM: launch_gemm(dt, false, (const GemmDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::GEMM_ATOMIC: launch_gemm(dt, true, (const GemmDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::SANDWICH:
        launch_sandwich(dt, (const SandwichDesc *)d, pre, op.nd, op.blocks, op.smem, s);
        break;
      case Op::CHOL: launch_chol(op.wide ? (dt | 2) : dt, (const CholDesc *)d, op.nd, op.smem, op.smem2, s); break;
      case Op::JACOBI: launch_jacobi(dt, (const JacobiDesc *)d, op.nd, op.smem, op.smem2, (int)op.blocks, s); break;
      case Op::FINALIZE: launch_finalize(dt, (const FinalizeDesc *)d, op.nd, s); break;
      case Op::ZERO: launch_zero((const ZeroDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::SITE: launch_site(dt, (const SiteDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::SCALAR: {
        ScalarDesc sd = op.scalar;
        sd.sites = (const void *const *)(blob + op.aux_off[0]);
        sd.left = (const int32_t *)(blob + op.aux_off[1]);
        sd.right = (const int32_t *)(blob + op.aux_off[2]);
        launch_scalar(dt, &sd, s);
        break;
      }
      case Op::FILL: launch_fill(dt, op.fill_ptr, op.fill_n, op.fill_value, s); break;
      case Op::TC: launch_tc_gemm(op.tc, op.tc_bn, s); break;
      case Op::PERMUTE: launch_permute(dt, (const PermuteDesc *)d, pre, op.nd, op.blocks, s); break;
    }
    if (events) CUDA_TRY(cudaEventRecord(events[&op - P->ops.data() + 1], s));
  }
  CUDA_TRY(cudaGetLastError());
  return PEPS_OK;
}

}  // namespace

extern "C" {

const char *peps_status_string(peps_status s) {
  switch (s) {
    case PEPS_OK: return "PEPS_OK";
    case PEPS_ERR_ARG: return "PEPS_ERR_ARG";
    case PEPS_ERR_SHAPE: return "PEPS_ERR_SHAPE";
    case PEPS_ERR_UNSUPPORTED: return "PEPS_ERR_UNSUPPORTED";
    case PEPS_ERR_CUDA: return "PEPS_ERR_CUDA";
    case PEPS_ERR_WORKSPACE: return "PEPS_ERR_WORKSPACE";
    case PEPS_ERR_NUMERIC: return "PEPS_ERR_NUMERIC";
    case PEPS_ERR_TIMEOUT: return "PEPS_ERR_TIMEOUT";
    case PEPS_ERR_CAPTURE: return "PEPS_ERR_CAPTURE";
    default: return "PEPS_ERR_UNKNOWN";
  }
}

const char *peps_last_error(void) { return g_last_error.c_str(); }
const char *peps_version(void) { return "libpeps 0.1 (sm_103a)"; }

peps_status peps_einsumsvd_plan(peps_plan **out, peps_dtype dtype, int32_t batch,
                                const peps_einsumsvd_shape *shapes, const uint64_t *instance_ids,
                                const peps_rsvd_opts *opts, size_t *workspace_bytes) {
  g_last_error.clear();
  if (!out || !shapes || !workspace_bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (!valid_dtype(dtype)) return fail(PEPS_ERR_ARG, "bad dtype %d", (int)dtype);
  if (batch < 1) return fail(PEPS_ERR_ARG, "batch must be >= 1");
  if (peps_status s = check_opts(opts)) return s;
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::EINSUMSVD;
  P->dt = dtype;
  P->opts = to_opts(opts);
  for (int i = 0; i < batch; ++i) {
    const peps_einsumsvd_shape &s = shapes[i];
    Inst I{};
    I.kL = s.kL; I.t = s.t; I.a = s.a; I.b = s.b; I.d = s.d;
    I.Dl = s.Dl; I.Du = s.Du; I.Dx = s.Dx; I.De = s.De;
    I.DL = s.DL; I.DU = s.DU; I.DX = s.DX; I.DE = s.DE;
    std::string e = inst_check(I, dtype);
    if (!e.empty()) return fail(PEPS_ERR_SHAPE, "instance %d: %s", i, e.c_str());
    inst_derive(I, P->opts);
    I.instance = instance_ids ? instance_ids[i] : (uint64_t)i;
    I.tc = P->opts.prec != PEPS_PREC_PLAIN && inst_tc_ok(I, dtype);
    P->insts.push_back(I);
  }
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_einsumsvd_rank(const peps_plan *plan, int32_t i, int32_t *k) {
  if (!plan || !k) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EINSUMSVD) return fail(PEPS_ERR_ARG, "not an einsumsvd plan");
  if (i < 0 || i >= (int)plan->insts.size()) return fail(PEPS_ERR_ARG, "instance index out of range");
  *k = plan->insts[i].k;
  return PEPS_OK;
}

peps_status peps_einsumsvd_execute(peps_plan *plan, const peps_einsumsvd_io *io, void *workspace,
                                   size_t workspace_bytes, void *stream) {
  g_last_error.clear();
  if (!plan || !io) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EINSUMSVD) return fail(PEPS_ERR_ARG, "not an einsumsvd plan");
  const size_t n = plan->insts.size();
  for (size_t i = 0; i < n; ++i)
    if (!io[i].V || !io[i].S || !io[i].ket || !io[i].bra || !io[i].U || !io[i].W || !io[i].sigma)
      return fail(PEPS_ERR_ARG, "instance %zu: NULL tensor pointer", i);
  bool same = plan->built && plan->built_base == (uintptr_t)workspace && plan->io_cache.size() == n;
  for (size_t i = 0; same && i < n; ++i)
    same = memcmp(&plan->io_cache[i], &io[i], sizeof(peps_einsumsvd_io)) == 0;
  if (!same) {
    if (peps_status s = rebuild(plan, workspace, io, true)) return s;
    plan->io_cache.assign(io, io + n);
    plan->built_base = (uintptr_t)workspace;
    plan->built = true;
  }
  return enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, !same);
}

peps_status peps_plan_destroy(peps_plan *plan) {
  delete plan;
  return PEPS_OK;
}

peps_status peps_contract_plan(peps_plan **out, const peps_network *ket, const peps_network *bra,
                               const peps_rsvd_opts *opts, int32_t direction, size_t *workspace_bytes) {
  g_last_error.clear();
  if (!out || !workspace_bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (peps_status s = check_opts(opts)) return s;
  if (direction < 0 || direction > 0xFFFF) return fail(PEPS_ERR_ARG, "direction out of range");
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::CONTRACT;
  P->opts = to_opts(opts);
  P->direction = direction;
  if (peps_status s = read_net(ket, P->ket, "ket")) return s;
  P->dt = P->ket.dt;
  if (bra) {
    if (peps_status s = read_net(bra, P->bra, "bra")) return s;
    if (P->bra.nrow != P->ket.nrow || P->bra.ncol != P->ket.ncol)
      return fail(PEPS_ERR_SHAPE, "ket and bra lattices differ");
    if (P->bra.dt != P->ket.dt) return fail(PEPS_ERR_ARG, "ket and bra dtypes differ");
    if (P->bra.d != P->ket.d) return fail(PEPS_ERR_SHAPE, "ket and bra physical dimensions differ");
  } else {
    if (P->ket.d != 1) return fail(PEPS_ERR_SHAPE, "one-layer contraction needs d = 1");
    P->one_layer = true;
  }
  if (P->ket.nrow > 0xFFFF || P->ket.ncol > 64) return fail(PEPS_ERR_UNSUPPORTED, "lattice too large");
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_contract_execute(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream) {
  g_last_error.clear();
  if (!plan) return fail(PEPS_ERR_ARG, "plan is NULL");
  if (plan->kind != peps_plan::CONTRACT) return fail(PEPS_ERR_ARG, "not a contraction plan");
  const bool same = plan->built && plan->built_base == (uintptr_t)workspace;
  if (!same) {
    if (peps_status s = rebuild(plan, workspace, nullptr, true)) return s;
    plan->built_base = (uintptr_t)workspace;
    plan->built = true;
  }
  return enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, !same);
}

peps_status peps_contract_sigma_count(const peps_plan *plan, int64_t *count) {
  if (!plan || !count) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::CONTRACT) return fail(PEPS_ERR_ARG, "not a contraction plan");
  *count = plan->nsigma;
  return PEPS_OK;
}

peps_status peps_contract_result(peps_plan *plan, void *workspace, void *stream, double *log_abs,
                                 double *phase, double *sigma_out) {
  g_last_error.clear();
  if (!plan || !workspace) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::CONTRACT) return fail(PEPS_ERR_ARG, "not a contraction plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "result read during stream capture");
  double res[2];
  CUDA_TRY(cudaMemcpyAsync(res, (uint8_t *)workspace + plan->result_off, 16, cudaMemcpyDeviceToHost, s));
  if (sigma_out && plan->nsigma > 0)
    CUDA_TRY(cudaMemcpyAsync(sigma_out, (uint8_t *)workspace + plan->sigma_off, plan->nsigma * 8,
                             cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (log_abs) *log_abs = res[0];
  if (phase) *phase = res[1];
  if (!std::isfinite(res[0]) && res[0] != -INFINITY)
    return fail(PEPS_ERR_NUMERIC, "non-finite contraction result");
  return PEPS_OK;
}

peps_status peps_boundary_workspace(const peps_network *ket, const peps_network *bra,
                                    const peps_rsvd_opts *opts, size_t *workspace_bytes) {
  peps_plan *p = nullptr;
  peps_status s = peps_contract_plan(&p, ket, bra, opts, 0, workspace_bytes);
  if (s == PEPS_OK) peps_plan_destroy(p);
  return s;
}

peps_status peps_boundary_contract(const peps_network *ket, const peps_network *bra,
                                   const peps_rsvd_opts *opts, void *workspace, size_t workspace_bytes,
                                   void *stream, double *log_abs, double *phase) {
  peps_plan *p = nullptr;
  size_t need = 0;
  peps_status s = peps_contract_plan(&p, ket, bra, opts, 0, &need);
  if (s != PEPS_OK) return s;
  s = peps_contract_execute(p, workspace, workspace_bytes, stream);
  if (s == PEPS_OK) s = peps_contract_result(p, workspace, stream, log_abs, phase, nullptr);
  peps_plan_destroy(p);
  return s;
}

peps_status peps_plan_launch_count(const peps_plan *plan, int64_t *count) {
  if (!plan || !count) return fail(PEPS_ERR_ARG, "NULL argument");
  *count = (int64_t)plan->ops.size();
  return PEPS_OK;
}

peps_status peps_plan_launch_info(const peps_plan *plan, int64_t i, const char **tag, double *flops,
                                  double *bytes) {
  if (!plan) return fail(PEPS_ERR_ARG, "NULL argument");
  if (i < 0 || i >= (int64_t)plan->ops.size()) return fail(PEPS_ERR_ARG, "launch index out of range");
  const Op &op = plan->ops[i];
  if (tag) *tag = op.tag.c_str();
  if (flops) *flops = op.flops;
  if (bytes) *bytes = op.bytes;
  return PEPS_OK;
}

peps_status peps_plan_profile(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream,
                              double *ms) {
  g_last_error.clear();
  if (!plan || !ms) return fail(PEPS_ERR_ARG, "NULL argument");
  if (!plan->built || plan->built_base != (uintptr_t)workspace)
    return fail(PEPS_ERR_ARG, "execute the plan on this workspace before profiling it");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "profiling during stream capture");
  const size_t n = plan->ops.size();
  std::vector<cudaEvent_t> ev(n + 1);
  for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
  peps_status st = enqueue(plan, workspace, workspace_bytes, s, false, ev.data());
  if (st == PEPS_OK) {
    cudaError_t e = cudaEventSynchronize(ev[n]);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] = t;
    }
    if (e != cudaSuccess) st = fail(PEPS_ERR_CUDA, "profiling events: %s", cudaGetErrorString(e));
  }
  for (auto &e : ev) cudaEventDestroy(e);
  return st;
}

peps_status peps_plan_validate(peps_plan *plan, void *workspace, size_t workspace_bytes,
                               const peps_einsumsvd_io *io) {
  g_last_error.clear();
  if (!plan || !workspace) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind == peps_plan::EINSUMSVD && !io) return fail(PEPS_ERR_ARG, "einsumsvd plans need io");
  if (peps_status s = rebuild(plan, workspace, plan->kind == peps_plan::EINSUMSVD ? io : nullptr)) return s;
  plan->built = false;            // force an upload at the next execute
  Checker C;
  const double es = dtype_size(plan->dt);
  if (plan->kind == peps_plan::EINSUMSVD) {
    for (size_t i = 0; i < plan->insts.size(); ++i) {
      const Inst &I = plan->insts[i];
      auto add = [&](const void *p, double n) { C.ext.push_back(Extent{(uintptr_t)p, (uintptr_t)p + (uintptr_t)n, "io"}); };
      add(io[i].V, es * I.kL * I.t * I.a * I.h);
      add(io[i].S, es * I.a * I.v * I.b);
      add(io[i].ket, es * I.d * I.Dl * I.Du * I.Dx * I.De);
      add(io[i].bra, es * I.d * I.DL * I.DU * I.DX * I.DE);
      add(io[i].U, es * (double)I.M * I.k);
      add(io[i].W, es * (double)I.k * I.N);
      add(io[i].sigma, 8.0 * I.k);
      if (io[i].log_scale) add(io[i].log_scale, 8);
    }
  } else {
    for (const Net *n : {&plan->ket, &plan->bra}) {
      if (n == &plan->bra && plan->one_layer) continue;
      for (size_t i = 0; i < n->site.size(); ++i) {
        const SiteDims &d = n->dims[i];
        C.ext.push_back(Extent{(uintptr_t)n->site[i],
                               (uintptr_t)n->site[i] + (uintptr_t)(es * d.d * d.Dl * d.Du * d.Dx * d.De), "site"});
      }
    }
  }
  std::string e = validate_ops(plan, (uintptr_t)workspace, workspace_bytes, C);
  if (!e.empty()) return fail(PEPS_ERR_ARG, "%s", e.c_str());
  return PEPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Contraction into the library's own device array (no allocation anywhere).
// Some callers cannot allocate device memory: a plugin given only its input
// and output buffers by a host application that owns every allocator, a
// process whose memory another framework's caching allocator already holds,
// or a latency-bound loop that cannot pay for cudaMalloc's device-wide
// synchronisation.  They get the same sweep with this fixed scratch instead.
// ---------------------------------------------------------------------------
// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[PEPS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
peps_status static_scratch(void **addr) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PEPS_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    if (!p || ((uintptr_t)p & 255)) return fail(PEPS_ERR_CUDA, "static scratch address %p unusable", p);
    g_static_addr[dev] = p;
  }
  *addr = g_static_addr[dev];
  return PEPS_OK;
}

}  // namespace

extern "C" peps_status peps_boundary_contract_static(const peps_network *ket, const peps_network *bra,
                                                     const peps_rsvd_opts *opts, void *stream,
                                                     double *log_abs, double *phase) {
  g_last_error.clear();
  peps_plan *raw = nullptr;
  size_t need = 0;
  if (peps_status s = peps_contract_plan(&raw, ket, bra, opts, 0, &need)) return s;
  std::unique_ptr<peps_plan> plan(raw);
  if (need > PEPS_STATIC_SCRATCH_BYTES)
    return fail(PEPS_ERR_WORKSPACE,
                "contraction needs %zu bytes of workspace, more than the %zu-byte static scratch; "
                "call peps_boundary_contract with caller memory instead",
                need, (size_t)PEPS_STATIC_SCRATCH_BYTES);
  void *ws = nullptr;
  if (peps_status s = static_scratch(&ws)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // the array holds the previous call's values: start this one from zeros
  CUDA_TRY(cudaMemsetAsync(ws, 0, need, st));
  if (peps_status s = peps_contract_execute(plan.get(), ws, PEPS_STATIC_SCRATCH_BYTES, stream)) return s;
  return peps_contract_result(plan.get(), ws, stream, log_abs, phase, nullptr);
}
