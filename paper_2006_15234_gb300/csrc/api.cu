// C ABI of libpeps (declared in include/libpeps.h): argument checking, plan
// objects, descriptor upload and launch of the static schedules built by
// step.cu (one einsumsvd) and by the boundary sweep below (Algorithms 2, 3).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <map>
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
  if (o->flags & ~(PEPS_FLAG_ORTH_Q | PEPS_FLAG_FP64_SMALL | PEPS_FLAG_ALTERNATE | PEPS_FLAG_UNIT_BOND))
    return fail(PEPS_ERR_ARG, "unknown flag bits %#x", o->flags);
  return PEPS_OK;
}

RsvdOpts to_opts(const peps_rsvd_opts *o) {
  RsvdOpts r;
  r.m = o->m; r.p = o->p; r.q = o->q; r.seed = o->seed; r.sketch = o->sketch; r.prec = o->prec;
  r.orth_q = (o->flags & PEPS_FLAG_ORTH_Q) != 0;
  r.fp64_small = (o->flags & PEPS_FLAG_FP64_SMALL) != 0;
  r.alternate = (o->flags & PEPS_FLAG_ALTERNATE) != 0;
  r.unit_bond = (o->flags & PEPS_FLAG_UNIT_BOND) != 0;
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
  enum Kind { EINSUMSVD, CONTRACT, EXPECT, EGRAD, GRAD, TEBD } kind;
  int dt = 0;
  RsvdOpts opts{};
  // einsumsvd
  std::vector<Inst> insts;
  std::vector<Inst> embeds;                 // zero-padded copies of instances with embed set
  int branches = 16;                        // side streams of the tensor-core chains
  // side streams of the plan's branches and their fork / join events
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_ev;
  ~peps_plan() {
    for (cudaEvent_t e : side_ev) cudaEventDestroy(e);
    for (cudaStream_t st : side) cudaStreamDestroy(st);
  }
  std::vector<peps_einsumsvd_io> io_cache;
  // einsumsvd adjoint (one instance)
  peps_einsumsvd_cotangent ct{};
  peps_einsumsvd_grads gr{};
  bool grad_bound = false;
  // contraction
  Net ket, bra;
  bool one_layer = false;
  int direction = 0;
  int64_t nsigma = 0;
  size_t result_off = 0, sigma_off = 0;
  // expectation value
  struct Term { int nsite; int site[2]; std::vector<double> op; double coeff; };
  std::vector<Term> terms;
  bool use_cache = true;
  // two-rank split of the cached expectation: op ranges of part 0 (top-down
  // sweeps), 1 (bottom-up sweeps), 2 (strips), and the workspace region
  // [lo, hi) holding each sweep part's environments, logs and sigmas
  std::vector<std::pair<size_t, size_t>> part_ops[3];
  size_t env_lo[2] = {0, 0}, env_hi[2] = {0, 0};
  bool splittable = false;
  int64_t nstrips = 0;
  size_t strip_off = 0;                     // strip values (accumulation type)
  std::vector<std::vector<std::pair<int64_t, int64_t>>> term_strips;   // per term: (component strip, norm strip)
  int64_t lognorm_strip = 0;                // row 0 norm strip of the original lattice
  size_t lognorm_logs_off = 0;              // logs of the sweep below row 0
  int64_t lognorm_nlogs = 0;
  // TEBD layer: the two-site operators, then the one-site operators, in the
  // working type (raw bytes)
  std::vector<uint8_t> gate;
  int64_t ngates = 0, nsite_gates = 0;
  // energy gradient: caller's gradient tensors, phase split, strip cotangents
  std::vector<void *> grad_site;
  size_t split = 0;                         // ops[0, split): forward; ops[split, end): reverse sweep
  size_t sbar_off = 0;
  // device status word (STATUS_* bits) at this workspace offset, cleared by
  // the first launch of every execute; limit of one tensor-core pipeline wait
  size_t status_off = 0;
  uint64_t wait_ns = 0;
  // autotuned MMA width per tensor-core GEMM shape (tc_signature -> width)
  std::map<std::string, int> tune;
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

// Side streams of a batched plan's tensor-core chains (default and limit).
constexpr int kBranches = 16;
constexpr int kMaxBranches = 64;

// Multiply-adds of one implicit product of an instance (Table 2's two-layer
// terms): the cost the tensor-core chains are balanced on.
double inst_cost(const Inst &q) {
  const double P1 = (double)q.Dl * q.Du, Q1 = (double)q.Dx * q.De, P2 = (double)q.DL * q.DU,
               Q2 = (double)q.DX * q.DE;
  return (double)q.ell * ((double)q.b * q.d * (P1 * Q1 * Q2 + P1 * Q2 * P2) + (double)q.a * q.h * q.v * q.b +
                          (double)q.M * q.a * q.h);
}

// Build the einsumsvd schedule (io may be null while sizing).  Instances on
// the CUDA cores share grouped launches on the caller's stream (branch 0).
// Instances on the tensor cores (extents aligned, or through a zero-padded
// copy) each run as one chain of launches; the chains are dealt to
// P->branches side streams by longest-processing-time-first on their product
// cost, so that independent chains overlap on the GPU, and the chains of
// one branch, which run one after the other, share one scratch region.
std::string build_einsumsvd(peps_plan *P, uintptr_t base, const peps_einsumsvd_io *io, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  const size_t n = P->insts.size();
  P->embeds.assign(n, Inst{});
  std::vector<Inst *> simt;
  std::vector<size_t> chains;
  for (size_t i = 0; i < n; ++i) {
    Inst &I = P->insts[i];
    I.logp = (double *)B.buf(8);
    if (io) {
      I.V = io[i].V; I.S = io[i].S; I.K = io[i].ket; I.Kb = io[i].bra;
      I.U = io[i].U; I.W = io[i].W; I.sigma = io[i].sigma;
      if (io[i].log_scale) I.logp = io[i].log_scale;
    }
    if (I.embed && !inst_embed_dims(I, P->dt, P->opts, P->embeds[i])) return "padded copy out of range";
    if (I.tc || I.embed) {
      chains.push_back(i);
    } else {
      inst_alloc_scratch(B, I, P->dt);
      simt.push_back(&I);
    }
  }
  if (!simt.empty()) emit_einsumsvd_simt(B, simt, P->opts);
  if (chains.empty()) return "";
  auto exec = [&](size_t i) -> Inst & { return P->insts[i].embed ? P->embeds[i] : P->insts[i]; };
  std::sort(chains.begin(), chains.end(), [&](size_t x, size_t y) {
    const double cx = inst_cost(exec(x)), cy = inst_cost(exec(y));
    return cx != cy ? cx > cy : x < y;
  });
  const int nb = (int)std::min<size_t>(P->branches, chains.size());
  std::vector<double> load(nb, 0.0);
  std::vector<std::vector<size_t>> br(nb);
  for (size_t i : chains) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[b] += inst_cost(exec(i));
    br[b].push_back(i);
  }
  for (int b = 0; b < nb; ++b) {
    const size_t region = B.alloc(0);
    size_t end = region;
    for (size_t i : br[b]) {
      B.top = region;
      Inst &I = P->insts[i];
      if (I.embed) inst_embed_alloc(B, P->embeds[i], P->dt);
      else inst_alloc_scratch(B, I, P->dt);
      end = std::max(end, B.top);
      const size_t first = B.ops.size();
      if (I.embed) emit_einsumsvd_embedded(B, I, P->embeds[i], P->opts);
      else emit_einsumsvd_tc_one(B, I, P->opts);
      for (size_t k = first; k < B.ops.size(); ++k) B.ops[k].branch = b + 1;
    }
    B.top = end;
  }
  return "";
}

// One einsumsvd with its adjoint: forward keeping the power iteration's
// bases, then the reverse sweep into the operand cotangents.
std::string build_egrad(peps_plan *P, uintptr_t base, const peps_einsumsvd_io *io, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  Inst &I = P->insts[0];
  inst_alloc_scratch(B, I, P->dt);
  I.logp = (double *)B.buf(8);
  GradBufs G;
  grad_alloc(B, I, P->opts, G, P->dt);
  double *lzero = (double *)B.buf(8);
  if (io) {
    I.V = io->V; I.S = io->S; I.K = io->ket; I.Kb = io->bra;
    I.U = io->U; I.W = io->W; I.sigma = io->sigma;
    if (io->log_scale) I.logp = io->log_scale;
  }
  const double *lbar = P->ct.log_scale_bar ? P->ct.log_scale_bar : lzero;
  {
    std::vector<std::pair<void *, int64_t>> z{{lzero, 1}};
    std::vector<ZeroDesc> d{ZeroDesc{lzero, 1}};
    std::vector<int64_t> prefix{0};
    Op op;
    op.kind = Op::ZERO; op.desc_off = B.put(d); op.prefix_off = B.put(prefix); op.nd = 1; op.blocks = 1;
    op.tag = "init";
    B.ops.push_back(op);
  }
  emit_einsumsvd_save(B, I, P->opts, G);
  emit_einsumsvd_bwd(B, I, P->opts, G, P->ct.U_bar, P->ct.W_bar, lbar, P->gr.V_bar, P->gr.S_bar, P->gr.ket_bar,
                     P->gr.bra_bar);
  return "";
}

// ---- boundary sweeps (Algorithms 2 and 3) -----------------------------------
// A sweep contracts rows 0..last of a lattice into a boundary MPS, keeping the
// boundary after each row in caller-chosen buffers (ping-pong for a plain
// contraction, one set per row for cached environments).

struct BSite { int left, vert, right; };

struct Sweep {
  const Net *ket = nullptr, *bra = nullptr;   // bra NULL: one-layer
  int last = 0;                               // last row contracted into the boundary
  int direction = 0;
  std::vector<std::vector<BSite>> bound;      // [r][q] boundary after row r
  std::vector<std::vector<Inst>> steps;       // [r] einsumsvd steps of row r (r >= 1)
  size_t max_site = 0, max_carry = 0;
  int64_t nsteps = 0, nsigma = 0;
};

SiteDims sweep_bra_dims(const Sweep &S, int p, int q) {
  if (!S.bra) return SiteDims{1, 1, 1, 1, 1};
  return S.bra->at(p, q);
}

// Shapes of every boundary site and einsumsvd step of rows 0..S.last.
std::string sweep_shapes(Sweep &S, const RsvdOpts &opts, int dt) {
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  S.bound.assign(S.last + 1, {});
  S.steps.assign(S.last + 1, {});
  for (int q = 0; q < ncol; ++q) {
    const SiteDims k = K.at(0, q), b = sweep_bra_dims(S, 0, q);
    S.bound[0].push_back(BSite{k.Dl * b.Dl, k.Dx * b.Dx, k.De * b.De});
  }
  for (auto &x : S.bound[0]) S.max_site = std::max(S.max_site, (size_t)x.left * x.vert * x.right);
  for (int r = 1; r <= S.last; ++r) {
    S.bound[r].resize(ncol);
    const SiteDims k0 = K.at(r, 0), b0 = sweep_bra_dims(S, r, 0);
    {
      const BSite &s0 = S.bound[r - 1][0];
      if (s0.vert != k0.Du * b0.Du) return "vertical bond mismatch between rows";
      S.max_carry = std::max(S.max_carry, (size_t)k0.Dx * b0.Dx * s0.right * k0.De * b0.De);
    }
    int kprev = 1;
    for (int i = 1; i < ncol; ++i) {
      const SiteDims kp = K.at(r, i - 1), bp = sweep_bra_dims(S, r, i - 1);
      const SiteDims kc = K.at(r, i), bc = sweep_bra_dims(S, r, i);
      const BSite &B0 = S.bound[r - 1][i];
      Inst I{};
      I.kL = kprev; I.t = kp.Dx * bp.Dx; I.a = B0.left; I.b = B0.right;
      I.d = kc.d; I.Dl = kc.Dl; I.Du = kc.Du; I.Dx = kc.Dx; I.De = kc.De;
      I.DL = bc.Dl; I.DU = bc.Du; I.DX = bc.Dx; I.DE = bc.De;
      if (kp.De != kc.Dl || bp.De != bc.Dl) return "horizontal bond mismatch";
      if (B0.vert != kc.Du * bc.Du) return "vertical bond mismatch between rows";
      if (S.bra && kc.d != bc.d) return "ket and bra physical dimensions differ";
      inst_derive(I, opts);
      std::string e = inst_check(I, dt);
      if (!e.empty()) return e;
      I.instance = ((uint64_t)S.direction << 32) | ((uint64_t)r << 16) | (uint64_t)i;
      I.tc = opts.prec != PEPS_PREC_PLAIN && inst_tc_ok(I, dt);
      S.bound[r][i - 1] = BSite{I.kL, I.t, I.k};
      S.max_carry = std::max(S.max_carry, (size_t)I.kL * I.t * I.a * I.h);
      S.max_carry = std::max(S.max_carry, (size_t)I.k * I.N);
      S.steps[r].push_back(I);
      kprev = I.k;
      ++S.nsteps;
      S.nsigma += I.k;
    }
    const SiteDims kl = K.at(r, ncol - 1), bl = sweep_bra_dims(S, r, ncol - 1);
    S.bound[r][ncol - 1] = BSite{kprev, kl.Dx * bl.Dx, 1};
    for (auto &x : S.bound[r]) S.max_site = std::max(S.max_site, (size_t)x.left * x.vert * x.right);
  }
  return "";
}

// One set of einsumsvd scratch, sized by the largest step of all sweeps.
void sweep_owner_scratch(Builder &B, const std::vector<Sweep *> &sw, int dt, Inst &owner) {
  const size_t es = dtype_size(dt), as = acc_size(dt);
  int64_t xN = 0, t2 = 0, t3 = 0, yM = 0, ell = 1, kk = 1;
  int64_t t1 = 0, vt = 0, st = 0, ut = 0, kt = 0, kb = 0;
  for (Sweep *S : sw)
    for (auto &row : S->steps)
      for (auto &I : row) {
        xN = std::max<int64_t>(xN, (int64_t)I.ell * I.N);
        t2 = std::max<int64_t>(t2, (int64_t)I.ell * I.h * I.v * I.b);
        t3 = std::max<int64_t>(t3, (int64_t)I.ell * I.a * I.h);
        yM = std::max<int64_t>(yM, (int64_t)I.ell * I.M);
        ell = std::max<int64_t>(ell, I.ell);
        kk = std::max<int64_t>(kk, I.k);
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
  owner.X = B.buf(xN * es); owner.Z = B.buf(xN * es);
  owner.T2 = B.buf(t2 * es); owner.T3 = B.buf(t3 * es);
  owner.Y = B.buf(yM * es); owner.P = B.buf(yM * es);
  owner.g = B.buf(std::max<int64_t>(yM, 1) * es);
  owner.Tm = B.buf(ell * ell * es); owner.Ut = B.buf(ell * kk * es);
  owner.G = B.buf(ell * ell * as); owner.R1 = B.buf(ell * ell * as); owner.R2 = B.buf(ell * ell * as);
  owner.Rout = B.buf(ell * ell * as); owner.Mw = B.buf(ell * ell * as);
  owner.sig = (double *)B.buf(ell * 8); owner.inv_s1 = (double *)B.buf(8);
  owner.T1 = t1 ? B.buf(t1 * es) : nullptr;
  owner.VT = vt ? B.buf(vt * es) : nullptr;
  owner.ST = st ? B.buf(st * es) : nullptr;
  owner.UT = ut ? B.buf(ut * es) : nullptr;
  owner.KT = kt ? B.buf(kt * es) : nullptr;
  owner.KbP = kb ? B.buf(kb * es) : nullptr;
  owner.KbT = kb ? B.buf(kb * es) : nullptr;
}

void push_site(Builder &B, std::vector<SiteDesc> &d, const char *tag) {
  std::vector<int64_t> prefix;
  int64_t tot = 0;
  for (auto &x : d) {
    prefix.push_back(tot);
    tot += ceil_div(x.total, kSiteThreads);
  }
  Op op;
  op.kind = Op::SITE; op.desc_off = B.put(d); op.prefix_off = B.put(prefix);
  op.nd = (int)d.size(); op.blocks = tot; op.tag = tag;
  B.ops.push_back(op);
}

// Ops of a sweep: row[r][q] receives the boundary after row r; logs (one per
// step, sweep order) and sigma (the planned ranks' values) are written too.
void emit_sweep(Builder &B, const Sweep &S, const RsvdOpts &opts, const void *ones,
                const std::vector<std::vector<void *>> &row, void *const Vbuf[2], double *logs, double *sigma,
                Inst &owner) {
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  auto bra_ptr = [&](int p, int q) -> const void * { return S.bra ? S.bra->ptr(p, q) : ones; };
  {
    std::vector<SiteDesc> d;
    for (int q = 0; q < ncol; ++q) {
      const SiteDims k = K.at(0, q), b = sweep_bra_dims(S, 0, q);
      SiteDesc x{};
      x.K = K.ptr(0, q); x.Kb = bra_ptr(0, q); x.S = nullptr; x.out = row[0][q]; x.mode = 0;
      x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De;
      x.DL = b.Dl; x.DU = b.Du; x.DX = b.Dx; x.DE = b.De; x.B = 1;
      x.total = (int64_t)k.Dl * b.Dl * k.Dx * b.Dx * k.De * b.De;
      d.push_back(x);
    }
    push_site(B, d, "first_row");
  }
  int64_t step_idx = 0, sig_pos = 0;
  for (int r = 1; r <= S.last; ++r) {
    {
      const SiteDims k = K.at(r, 0), b = sweep_bra_dims(S, r, 0);
      SiteDesc x{};
      x.K = K.ptr(r, 0); x.Kb = bra_ptr(r, 0); x.S = row[r - 1][0];
      x.out = ncol == 1 ? row[r][0] : Vbuf[0];
      x.mode = 1;
      x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De;
      x.DL = b.Dl; x.DU = b.Du; x.DX = b.Dx; x.DE = b.De; x.B = S.bound[r - 1][0].right;
      x.total = (int64_t)k.Dx * b.Dx * x.B * k.De * b.De;
      std::vector<SiteDesc> d{x};
      push_site(B, d, "zipup_start");
    }
    int cv = 0;
    for (int i = 1; i < ncol; ++i) {
      Inst I = S.steps[r][i - 1];
      inst_share_scratch(I, owner);
      I.V = Vbuf[cv];
      I.S = row[r - 1][i];
      I.K = K.ptr(r, i);
      I.Kb = bra_ptr(r, i);
      I.U = row[r][i - 1];
      I.W = (i == ncol - 1) ? row[r][ncol - 1] : Vbuf[1 - cv];
      I.sigma = sigma + sig_pos;
      I.logp = logs + step_idx;
      sig_pos += I.k;
      ++step_idx;
      std::vector<Inst *> one{&I};
      emit_einsumsvd(B, one, opts);
      if (opts.alternate && r % 2 == 0) {
        // alternating canonicalisation: Sigma / sigma_1 into the finished site
        Op op;
        op.kind = Op::ABSORB; op.tag = "epilogue_u";
        op.absorb = AbsorbDesc{I.U, I.W, I.sigma, I.M, I.N, I.k};
        op.bytes = 2.0 * dtype_size(B.dt) * ((double)I.M * I.k + (double)I.k * I.N);
        B.ops.push_back(op);
      }
      cv = 1 - cv;
    }
  }
}

// Boundary sweep of Algorithms 2 and 3 over the whole network.
std::string build_contract(peps_plan *P, uintptr_t base, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  const Net &K = P->ket;
  const int nrow = K.nrow, ncol = K.ncol, dt = P->dt;
  const size_t es = dtype_size(dt);
  if (ncol > 64) return "ncol above 64 is not supported";
  Sweep S;
  S.ket = &K;
  S.bra = P->one_layer ? nullptr : &P->bra;
  S.last = nrow - 1;
  S.direction = P->direction;
  std::string e = sweep_shapes(S, P->opts, dt);
  if (!e.empty()) return e;
  P->nsigma = S.nsigma;
  Inst owner{};
  sweep_owner_scratch(B, {&S}, dt, owner);
  std::vector<void *> Sbuf[2];
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q < ncol; ++q) Sbuf[c].push_back(B.buf(S.max_site * es));
  std::vector<std::vector<void *>> row(nrow);
  for (int r = 0; r < nrow; ++r) row[r] = Sbuf[r & 1];
  void *Vbuf[2] = {B.buf(std::max<size_t>(S.max_carry, 1) * es), B.buf(std::max<size_t>(S.max_carry, 1) * es)};
  double *logs = (double *)B.buf(std::max<int64_t>(S.nsteps, 1) * 8);
  P->sigma_off = B.alloc(std::max<int64_t>(S.nsigma, 1) * 8);
  double *sigma = (double *)B.ptr(P->sigma_off);
  P->result_off = B.alloc(16);
  double *result = (double *)B.ptr(P->result_off);
  int maxbond = 1;
  for (int q = 0; q < ncol; ++q)
    maxbond = std::max(maxbond, std::max(S.bound[nrow - 1][q].left, S.bound[nrow - 1][q].right));
  void *sc_scratch = B.buf((size_t)2 * maxbond * acc_size(dt));
  void *ones = B.buf(es);

  if (P->one_layer) {
    Op f;
    f.kind = Op::FILL; f.fill_ptr = ones; f.fill_n = 1; f.fill_value = 1.0; f.tag = "init";
    B.ops.push_back(f);
  }
  emit_sweep(B, S, P->opts, ones, row, Vbuf, logs, sigma, owner);
  // --- final scalar
  const std::vector<void *> &last = row[nrow - 1];
  std::vector<const void *> sp(ncol);
  std::vector<int32_t> lb(ncol), rb(ncol);
  for (int q = 0; q < ncol; ++q) {
    sp[q] = last[q];
    lb[q] = S.bound[nrow - 1][q].left;
    rb[q] = S.bound[nrow - 1][q].right;
    if (S.bound[nrow - 1][q].vert != 1) return "last row has open vertical bonds";
  }
  Op sc;
  sc.kind = Op::SCALAR;
  sc.aux_off[0] = B.put(sp);
  sc.aux_off[1] = B.put(lb);
  sc.aux_off[2] = B.put(rb);
  sc.scalar.ncol = ncol;
  sc.scalar.logs = logs;
  sc.scalar.nlogs = (int)S.nsteps;
  sc.scalar.scratch = sc_scratch;
  sc.scalar.out = result;
  sc.tag = "scalar";
  B.ops.push_back(sc);
  return "";
}


// ---- expectation values (Eq. 6 with cached environments, Sec. IV-B) --------

// A lattice the sweeps read: the caller's network, or a permuted copy of it
// (rows read bottom-up, rows and columns exchanged) in the workspace.
struct LatticeCopy {
  Net net;                                   // site pointers into the workspace
  std::vector<PermuteDesc> perm;             // how the copy is made
};

void push_permute(Builder &B, std::vector<PermuteDesc> &d, const char *tag) {
  if (d.empty()) return;
  std::vector<int64_t> prefix;
  int64_t tot = 0;
  for (auto &x : d) {
    prefix.push_back(tot);
    tot += permute_blocks(x);
  }
  Op op;
  op.kind = Op::PERMUTE; op.desc_off = B.put(d); op.prefix_off = B.put(prefix);
  op.nd = (int)d.size(); op.blocks = tot; op.tag = tag;
  B.ops.push_back(op);
}

PermuteDesc mk_permute(const void *in, void *out, int64_t nb, int64_t R, int64_t C, int64_t Q) {
  PermuteDesc p{};
  p.in = in; p.out = out; p.nb = nb; p.R = R; p.Cc = C; p.Q = Q; p.conj = 0;
  return p;
}

int64_t site_elems(const SiteDims &x) { return (int64_t)x.d * x.Dl * x.Du * x.Dx * x.De; }

// Rows reversed, up and down bonds exchanged: [d][l][u][x][e] -> [d][l][x][u][e].
LatticeCopy flip_copy(Builder &B, const Net &src, size_t es) {
  LatticeCopy L;
  L.net.nrow = src.nrow; L.net.ncol = src.ncol; L.net.d = src.d; L.net.dt = src.dt;
  L.net.dims.resize(src.dims.size());
  L.net.site.resize(src.site.size());
  for (int p = 0; p < src.nrow; ++p)
    for (int q = 0; q < src.ncol; ++q) {
      const SiteDims x = src.at(src.nrow - 1 - p, q);
      void *out = B.buf(site_elems(x) * es);
      L.perm.push_back(mk_permute(src.ptr(src.nrow - 1 - p, q), out, (int64_t)x.d * x.Dl, x.Du, x.Dx, x.De));
      L.net.dims[(size_t)p * src.ncol + q] = SiteDims{x.d, x.Dl, x.Dx, x.Du, x.De};
      L.net.site[(size_t)p * src.ncol + q] = out;
    }
  return L;
}

// Rows and columns exchanged: [d][l][u][x][e] -> [d][u][l][e][x] (two passes).
LatticeCopy transpose_copy(Builder &B, const Net &src, size_t es, std::vector<PermuteDesc> &first_pass) {
  LatticeCopy L;
  L.net.nrow = src.ncol; L.net.ncol = src.nrow; L.net.d = src.d; L.net.dt = src.dt;
  L.net.dims.resize(src.dims.size());
  L.net.site.resize(src.site.size());
  for (int p = 0; p < src.nrow; ++p)
    for (int q = 0; q < src.ncol; ++q) {
      const SiteDims x = src.at(p, q);
      void *tmp = B.buf(site_elems(x) * es);
      void *out = B.buf(site_elems(x) * es);
      first_pass.push_back(mk_permute(src.ptr(p, q), tmp, x.d, x.Dl, x.Du, (int64_t)x.Dx * x.De));
      L.perm.push_back(mk_permute(tmp, out, (int64_t)x.d * x.Du * x.Dl, x.Dx, x.De, 1));
      L.net.dims[(size_t)q * src.nrow + p] = SiteDims{x.d, x.Du, x.Dl, x.De, x.Dx};
      L.net.site[(size_t)q * src.nrow + p] = out;
    }
  return L;
}

// ---- energy gradient: sweeps that keep every step, and their reverse -------

struct StepRec {
  Inst I;
  GradBufs G;
  void *tmpS = nullptr, *tmpK = nullptr, *tmpKb = nullptr;
};

struct SweepGrad {
  std::vector<std::vector<void *>> crow;             // cotangents of the boundary after row r
  std::vector<std::vector<void *>> carry, ccarry;    // [r][i]: carry entering step i (i >= 1) and its cotangent
  std::vector<std::vector<StepRec>> steps;           // [r][i-1]
  std::vector<std::vector<void *>> gsite;            // [r][q]: cotangent of the lattice's site tensors
};

void push_copy(Builder &B, void *dst, const void *src, int64_t bytes, const char *tag) {
  Op op;
  op.kind = Op::COPY; op.fill_ptr = dst; op.aux_ptr = src; op.fill_n = bytes; op.tag = tag;
  B.ops.push_back(op);
}

void push_memset(Builder &B, void *p, int64_t bytes, const char *tag) {
  Op op;
  op.kind = Op::MEMSET; op.fill_ptr = p; op.fill_n = bytes; op.tag = tag;
  B.ops.push_back(op);
}

void push_axpy(Builder &B, const void *x, void *y, int64_t n, const char *tag) {
  Op op;
  op.kind = Op::AXPY; op.aux_ptr = x; op.fill_ptr = y; op.fill_n = n; op.tag = tag;
  B.ops.push_back(op);
}

int64_t bsite_elems(const BSite &x) { return (int64_t)x.left * x.vert * x.right; }

// Buffers of a sweep's gradient pass with per-row checkpointing: the
// boundary after every row (the cached environments) is the checkpoint; a
// row's einsumsvd steps keep their forward data only while that row is being
// reversed, so every row's step at column i (its scratch, saved bases, carry
// and carry cotangent) is carved out of one region per column that all rows
// share.  The boundary cotangents stay per row (they accumulate across rows).
void sweep_grad_alloc(Builder &B, const Sweep &S, const RsvdOpts &opts, int dt, SweepGrad &SG) {
  const size_t es = dtype_size(dt);
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  SG.crow.assign(S.last + 1, {});
  for (int r = 0; r <= S.last; ++r)
    for (auto &x : S.bound[r]) SG.crow[r].push_back(B.buf(bsite_elems(x) * es));
  SG.carry.assign(S.last + 1, std::vector<void *>(ncol + 1, nullptr));
  SG.ccarry.assign(S.last + 1, std::vector<void *>(ncol + 1, nullptr));
  SG.steps.assign(S.last + 1, {});
  for (int i = 1; i < ncol; ++i) {
    const size_t region = B.alloc(0);
    size_t end = region;
    for (int r = 1; r <= S.last; ++r) {
      B.top = region;
      const Inst &I0 = S.steps[r][i - 1];
      const int64_t vsz = (int64_t)I0.kL * I0.t * I0.a * I0.h;
      SG.carry[r][i] = B.buf(vsz * es);
      SG.ccarry[r][i] = B.buf(vsz * es);
      StepRec rec;
      rec.I = I0;
      inst_alloc_scratch(B, rec.I, dt);
      rec.I.logp = (double *)B.buf(8);
      grad_alloc(B, rec.I, opts, rec.G, dt);
      rec.tmpS = B.buf((int64_t)I0.a * I0.v * I0.b * es);
      rec.tmpK = B.buf((int64_t)I0.d * I0.Dl * I0.Du * I0.Dx * I0.De * es);
      rec.tmpKb = B.buf((int64_t)I0.d * I0.DL * I0.DU * I0.DX * I0.DE * es);
      SG.steps[r].push_back(rec);
      end = std::max(end, B.top);
    }
    B.top = end;
  }
  SG.gsite.assign(K.nrow, std::vector<void *>(ncol, nullptr));
}

// Row r of a sweep (r >= 1) keeping every step's forward data: the zip-up
// start from the boundary after row r - 1, then the einsumsvd steps.
void emit_row_save(Builder &B, const Sweep &S, const RsvdOpts &opts, const std::vector<std::vector<void *>> &row,
                   SweepGrad &SG, double *logs, double *sigma, int r) {
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  int64_t step_idx = 0, sig_pos = 0;
  for (int rr = 1; rr < r; ++rr)
    for (const Inst &I : S.steps[rr]) {
      ++step_idx;
      sig_pos += I.k;
    }
  {
    const SiteDims k = K.at(r, 0), b = sweep_bra_dims(S, r, 0);
    SiteDesc x{};
    x.K = K.ptr(r, 0); x.Kb = S.bra->ptr(r, 0); x.S = row[r - 1][0];
    x.out = ncol == 1 ? row[r][0] : SG.carry[r][1];
    x.mode = 1;
    x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De;
    x.DL = b.Dl; x.DU = b.Du; x.DX = b.Dx; x.DE = b.De; x.B = S.bound[r - 1][0].right;
    x.total = (int64_t)k.Dx * b.Dx * x.B * k.De * b.De;
    std::vector<SiteDesc> d{x};
    push_site(B, d, "zipup_start");
  }
  for (int i = 1; i < ncol; ++i) {
    StepRec &rec = SG.steps[r][i - 1];
    Inst &I = rec.I;
    I.V = SG.carry[r][i];
    I.S = row[r - 1][i];
    I.K = K.ptr(r, i);
    I.Kb = S.bra->ptr(r, i);
    I.U = row[r][i - 1];
    I.W = (i == ncol - 1) ? row[r][ncol - 1] : SG.carry[r][i + 1];
    I.sigma = sigma + sig_pos;
    I.logp = logs + step_idx;
    sig_pos += I.k;
    ++step_idx;
    emit_einsumsvd_save(B, I, opts, rec.G);
  }
}

// Forward of a sweep (same ops as emit_sweep otherwise); the last row's
// steps leave their forward data in place for the reverse sweep.
void emit_sweep_save(Builder &B, const Sweep &S, const RsvdOpts &opts, const std::vector<std::vector<void *>> &row,
                     SweepGrad &SG, double *logs, double *sigma) {
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  {
    std::vector<SiteDesc> d;
    for (int q = 0; q < ncol; ++q) {
      const SiteDims k = K.at(0, q), b = sweep_bra_dims(S, 0, q);
      SiteDesc x{};
      x.K = K.ptr(0, q); x.Kb = S.bra->ptr(0, q); x.S = nullptr; x.out = row[0][q]; x.mode = 0;
      x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De;
      x.DL = b.Dl; x.DU = b.Du; x.DX = b.Dx; x.DE = b.De; x.B = 1;
      x.total = (int64_t)k.Dl * b.Dl * k.Dx * b.Dx * k.De * b.De;
      d.push_back(x);
    }
    push_site(B, d, "first_row");
  }
  for (int r = 1; r <= S.last; ++r) emit_row_save(B, S, opts, row, SG, logs, sigma, r);
}

// Reverse of a sweep: boundary cotangents SG.crow (complete for every row the
// strips and later rows feed) to the lattice's site cotangents SG.gsite.
void emit_sweep_bwd(Builder &B, const Sweep &S, const RsvdOpts &opts, const std::vector<std::vector<void *>> &row,
                    SweepGrad &SG, const double *lzero, double *logs, double *sigma) {
  const Net &K = *S.ket;
  const int ncol = K.ncol;
  const char *tag = "sweep_reverse";
  for (int r = S.last; r >= 1; --r) {
    // checkpoint restart: row r's forward again from the boundary after row
    // r - 1 (the same kernels on the same inputs rewrite the same values);
    // the last row's forward data are still in place
    if (r < S.last) emit_row_save(B, S, opts, row, SG, logs, sigma, r);
    for (int i = ncol - 1; i >= 1; --i) {
      StepRec &rec = SG.steps[r][i - 1];
      Inst &I = rec.I;
      const void *Ub = SG.crow[r][i - 1];
      const void *Wb = (i == ncol - 1) ? SG.crow[r][ncol - 1] : SG.ccarry[r][i + 1];
      emit_einsumsvd_bwd(B, I, opts, rec.G, Ub, Wb, lzero, SG.ccarry[r][i], rec.tmpS, rec.tmpK, rec.tmpKb);
      push_axpy(B, rec.tmpS, SG.crow[r - 1][i], (int64_t)I.a * I.v * I.b, tag);
      const int64_t nk = (int64_t)I.d * I.Dl * I.Du * I.Dx * I.De;
      push_axpy(B, rec.tmpK, SG.gsite[r][i], nk, tag);
      push_axpy(B, rec.tmpKb, SG.gsite[r][i], nk, tag);
    }
    // first zip-up carry of row r
    const SiteDims k = K.at(r, 0);
    SiteBwdDesc x{};
    x.K = K.ptr(r, 0); x.S = row[r - 1][0];
    x.cot = ncol == 1 ? SG.crow[r][0] : SG.ccarry[r][1];
    x.Kbar = SG.gsite[r][0]; x.Sbar = SG.crow[r - 1][0];
    x.mode = 1; x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De; x.B = S.bound[r - 1][0].right;
    Op op;
    op.kind = Op::SITEBWD; op.desc_off = B.put(std::vector<SiteBwdDesc>{x}); op.nd = 1; op.tag = tag;
    B.ops.push_back(op);
  }
  for (int q = 0; q < ncol; ++q) {
    const SiteDims k = K.at(0, q);
    SiteBwdDesc x{};
    x.K = K.ptr(0, q); x.cot = SG.crow[0][q]; x.Kbar = SG.gsite[0][q];
    x.mode = 0; x.d = k.d; x.Dl = k.Dl; x.Du = k.Du; x.Dx = k.Dx; x.De = k.De; x.B = 1;
    Op op;
    op.kind = Op::SITEBWD; op.desc_off = B.put(std::vector<SiteBwdDesc>{x}); op.nd = 1; op.tag = tag;
    B.ops.push_back(op);
  }
}

// Cached environments of one lattice: boundaries above every row (top-down
// sweep) and below every row (sweep of the row-reversed copy).
struct EnvSet {
  Sweep top, bot;
  bool has_top = false, has_bot = false;
  std::unique_ptr<SweepGrad> tg, bg;      // energy gradient only
  std::vector<std::vector<void *>> top_rows, bot_rows;
  double *top_logs = nullptr, *bot_logs = nullptr;
  double *top_sigma = nullptr, *bot_sigma = nullptr;
};

std::string build_expect(peps_plan *P, uintptr_t base, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  const int dt = P->dt;
  const size_t es = dtype_size(dt), as = acc_size(dt);
  const bool cplx = dtype_complex(dt);
  const Net &H = P->ket;
  const int d = H.d;
  const bool grad = P->kind == peps_plan::GRAD;
  if (d > 4) return "physical dimension above 4 is not supported by the strip kernel";
  if (H.ncol > kStripMaxCols || H.nrow > kStripMaxCols) return "lattice side above 32 is not supported";

  // --- terms -> strips: (lattice 0 = as given, 1 = transposed; row; column -> operator)
  struct Comp { int lat, row; std::vector<std::pair<int, int>> ops; };   // (column, op table index)
  std::vector<std::vector<double>> optab;     // d x d matrices (re, im interleaved when complex)
  auto add_op = [&](const std::vector<double> &m) { optab.push_back(m); return (int)optab.size() - 1; };
  const int vals = cplx ? 2 : 1;
  std::vector<std::vector<Comp>> comps(P->terms.size());
  bool need_v = false;
  for (size_t t = 0; t < P->terms.size(); ++t) {
    const auto &T = P->terms[t];
    const int r0 = T.site[0] / H.ncol, c0 = T.site[0] % H.ncol;
    if (T.nsite == 1) {
      std::vector<double> m(T.op.begin(), T.op.end());
      comps[t].push_back(Comp{0, r0, {{c0, add_op(m)}}});
      continue;
    }
    const int r1 = T.site[1] / H.ncol, c1 = T.site[1] % H.ncol;
    const bool horiz = r1 == r0 && c1 == c0 + 1;
    if (!horiz) need_v = true;
    // O[(a,s'),(b,s)] = sum_{a,b} E_ab (x) O^(a,b): one component per nonzero block
    const int dd = d * d;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        std::vector<double> blk((size_t)dd * vals);
        bool nz = false;
        for (int s2 = 0; s2 < d; ++s2)
          for (int t2 = 0; t2 < d; ++t2)
            for (int v = 0; v < vals; ++v) {
              const double x = T.op[((size_t)(a * d + s2) * dd + (b * d + t2)) * vals + v];
              blk[((size_t)s2 * d + t2) * vals + v] = x;
              nz = nz || x != 0.0;
            }
        if (!nz) continue;
        std::vector<double> e((size_t)dd * vals, 0.0);
        e[((size_t)a * d + b) * vals] = 1.0;
        const int ia = add_op(e), ib = add_op(blk);
        if (horiz) comps[t].push_back(Comp{0, r0, {{c0, ia}, {c1, ib}}});
        else comps[t].push_back(Comp{1, c0, {{r0, ia}, {r1, ib}}});
      }
  }

  // --- lattices
  const Net *lat[2] = {&H, nullptr};
  LatticeCopy Vt, Hf, Vf;
  std::vector<PermuteDesc> tpass;
  Hf = flip_copy(B, H, es);
  if (need_v) {
    Vt = transpose_copy(B, H, es, tpass);
    lat[1] = &Vt.net;
    Vf = flip_copy(B, Vt.net, es);
  }
  const Net *flat[2] = {&Hf.net, need_v ? &Vf.net : nullptr};

  // --- sweeps: cached (one top and one bottom sweep per lattice) or one
  // pair per row that holds strips (uncached: the environments are
  // recomputed for every row, with the same sketches)
  std::vector<bool> rows_used[2];
  for (int l = 0; l < 2; ++l) rows_used[l].assign(lat[l] ? lat[l]->nrow : 0, false);
  rows_used[0][0] = true;                  // log-norm strip
  for (auto &cv : comps)
    for (auto &c : cv) rows_used[c.lat][c.row] = true;
  // env[l][r]: environment set used by row r of lattice l (index into envs)
  std::vector<std::unique_ptr<EnvSet>> envs;
  std::vector<int> env_of[2];
  for (int l = 0; l < 2; ++l) {
    if (!lat[l]) continue;
    const int nrow = lat[l]->nrow;
    env_of[l].assign(nrow, -1);
    auto make = [&](int top_last, int bot_last) {
      auto E = std::make_unique<EnvSet>();
      if (top_last >= 0) {
        E->has_top = true;
        E->top.ket = lat[l]; E->top.bra = lat[l]; E->top.last = top_last; E->top.direction = 2 * l;
      }
      if (bot_last >= 0) {
        E->has_bot = true;
        E->bot.ket = flat[l]; E->bot.bra = flat[l]; E->bot.last = bot_last; E->bot.direction = 2 * l + 1;
      }
      envs.push_back(std::move(E));
      return (int)envs.size() - 1;
    };
    if (P->use_cache || grad) {
      const int e = make(nrow - 2, nrow - 2);
      for (int r = 0; r < nrow; ++r) env_of[l][r] = e;
    } else {
      for (int r = 0; r < nrow; ++r)
        if (rows_used[l][r]) env_of[l][r] = make(r - 1, nrow - 2 - r);
    }
  }
  std::vector<Sweep *> all;
  for (auto &E : envs) {
    if (E->has_top) {
      std::string e = sweep_shapes(E->top, P->opts, dt);
      if (!e.empty()) return e;
      all.push_back(&E->top);
    }
    if (E->has_bot) {
      std::string e = sweep_shapes(E->bot, P->opts, dt);
      if (!e.empty()) return e;
      all.push_back(&E->bot);
    }
  }
  // the cached schedule's sweeps (top-down and bottom-up, of the lattice and
  // of its transpose) are independent: each runs on a graph branch of its
  // own with its own scratch, and the strips follow the join
  const bool par = !grad && P->use_cache && all.size() > 1;
  std::map<const Sweep *, int> branch_of;
  // (branches 1..n: the caller's stream keeps the prelude and the strips)
  std::vector<Inst> owners(par ? all.size() + 1 : 1);
  std::vector<std::array<void *, 2>> vbufs(owners.size());
  for (size_t i = 0; i < all.size(); ++i) branch_of[all[i]] = par ? (int)i + 1 : 0;
  if (par) {
    for (size_t i = 0; i < all.size(); ++i) {
      sweep_owner_scratch(B, {all[i]}, dt, owners[i + 1]);
      vbufs[i + 1] = {B.buf(all[i]->max_carry * es), B.buf(all[i]->max_carry * es)};
    }
  } else {
    if (!grad) sweep_owner_scratch(B, all, dt, owners[0]);
    size_t max_carry = 1;
    for (Sweep *S : all) max_carry = std::max(max_carry, S->max_carry);
    vbufs[0] = {B.buf(max_carry * es), B.buf(max_carry * es)};
  }
  void *ones = B.buf(es);
  auto rows_for = [&](const Sweep &S) {
    std::vector<std::vector<void *>> rows(S.last + 1);
    for (int r = 0; r <= S.last; ++r)
      for (auto &x : S.bound[r]) rows[r].push_back(B.buf((size_t)x.left * x.vert * x.right * es));
    return rows;
  };
  // the top-down environments of every set, then the bottom-up ones: each
  // sweep direction's results form one contiguous workspace region (the
  // unit a two-rank split exchanges)
  B.alloc(0);
  P->env_lo[0] = (B.top + 255) & ~(size_t)255;
  for (auto &E : envs)
    if (E->has_top) {
      E->top_rows = rows_for(E->top);
      E->top_logs = (double *)B.buf(std::max<int64_t>(E->top.nsteps, 1) * 8);
      E->top_sigma = (double *)B.buf(std::max<int64_t>(E->top.nsigma, 1) * 8);
    }
  P->env_hi[0] = B.top;
  P->env_lo[1] = (B.top + 255) & ~(size_t)255;
  for (auto &E : envs)
    if (E->has_bot) {
      E->bot_rows = rows_for(E->bot);
      E->bot_logs = (double *)B.buf(std::max<int64_t>(E->bot.nsteps, 1) * 8);
      E->bot_sigma = (double *)B.buf(std::max<int64_t>(E->bot.nsigma, 1) * 8);
    }
  P->env_hi[1] = B.top;
  // energy gradient: site cotangents of the four lattices (0 H, 1 Vt, 2 Hf, 3 Vf) and the sweeps' buffers
  std::vector<std::vector<void *>> gl[4];
  const Net *glat[4] = {&H, need_v ? &Vt.net : nullptr, &Hf.net, need_v ? &Vf.net : nullptr};
  if (grad) {
    for (int l = 0; l < 4; ++l) {
      if (!glat[l]) continue;
      gl[l].assign(glat[l]->nrow, std::vector<void *>(glat[l]->ncol, nullptr));
      for (int r = 0; r < glat[l]->nrow; ++r)
        for (int q = 0; q < glat[l]->ncol; ++q) gl[l][r][q] = B.buf(site_elems(glat[l]->at(r, q)) * es);
    }
    for (int l = 0; l < 2; ++l) {
      if (!lat[l]) continue;
      EnvSet &E = *envs[env_of[l][0]];
      if (E.has_top && !E.tg) {
        E.tg = std::make_unique<SweepGrad>();
        sweep_grad_alloc(B, E.top, P->opts, dt, *E.tg);
        E.tg->gsite = gl[l];
      }
      if (E.has_bot && !E.bg) {
        E.bg = std::make_unique<SweepGrad>();
        sweep_grad_alloc(B, E.bot, P->opts, dt, *E.bg);
        E.bg->gsite = gl[l + 2];
      }
    }
  }

  // --- strips
  std::vector<StripCol> cols;
  std::vector<StripBwdCol> bcols;
  std::vector<StripDesc> sd;
  int64_t l_cap = 1, a1_cap = 1, a2_cap = 1, a3_cap = 1;
  // column table of row r of lattice l (shared by all strips of that row)
  std::map<std::pair<int, int>, int> row_cols;
  auto columns = [&](int l, int r) -> std::string {
    if (row_cols.count({l, r})) return "";
    const Net &L = *lat[l];
    const EnvSet &E = *envs[env_of[l][r]];
    const int nrow = L.nrow;
    row_cols[{l, r}] = (int)cols.size();
    for (int q = 0; q < L.ncol; ++q) {
      const SiteDims x = L.at(r, q);
      StripCol c{};
      c.ket = L.ptr(r, q);
      c.d = x.d; c.Dl = x.Dl; c.Du = x.Du; c.Dx = x.Dx; c.De = x.De;
      if (r > 0) {
        const BSite &u = E.top.bound[r - 1][q];
        if (u.vert != x.Du * x.Du) return "environment above does not match the row";
        c.up = E.top_rows[r - 1][q]; c.a = u.left; c.b = u.right;
      } else {
        c.up = ones; c.a = 1; c.b = 1;
      }
      if (r < nrow - 1) {
        const BSite &w = E.bot.bound[nrow - 2 - r][q];
        if (w.vert != x.Dx * x.Dx) return "environment below does not match the row";
        c.lo = E.bot_rows[nrow - 2 - r][q]; c.c = w.left; c.f = w.right;
      } else {
        c.lo = ones; c.c = 1; c.f = 1;
      }
      const int64_t vu = (int64_t)x.Du * x.Du;
      l_cap = std::max<int64_t>(l_cap, (int64_t)c.a * x.Dl * x.Dl * c.c);
      l_cap = std::max<int64_t>(l_cap, (int64_t)c.b * x.De * x.De * c.f);
      a1_cap = std::max<int64_t>(a1_cap, (int64_t)x.Dl * x.Dl * c.c * vu * c.b);
      a2_cap = std::max<int64_t>(a2_cap, (int64_t)x.Dl * c.c * x.Du * c.b * x.d * x.Dx * x.De);
      a3_cap = std::max<int64_t>(a3_cap, (int64_t)c.c * c.b * x.De * x.Dx * x.Dx * x.De);
      cols.push_back(c);
      StripBwdCol bc{};
      if (grad) {
        bc.cot_up = r > 0 ? E.tg->crow[r - 1][q] : nullptr;
        bc.cot_lo = r < nrow - 1 ? E.bg->crow[nrow - 2 - r][q] : nullptr;
        bc.cot_ket = gl[l][r][q];
      }
      bcols.push_back(bc);
    }
    return "";
  };
  std::map<std::pair<int, int>, int64_t> norm_strip;
  auto add_strip = [&](int l, int r, const std::vector<std::pair<int, int>> &ops) -> int64_t {
    StripDesc x{};
    x.col0 = row_cols[{l, r}];
    x.ncol = lat[l]->ncol;
    for (int q = 0; q < kStripMaxCols; ++q) x.op[q] = -1;
    for (auto &o : ops) x.op[o.first] = o.second;
    sd.push_back(x);
    return (int64_t)sd.size() - 1;
  };
  auto norm_of = [&](int l, int r) -> std::string {
    if (norm_strip.count({l, r})) return "";
    std::string e = columns(l, r);
    if (!e.empty()) return e;
    norm_strip[{l, r}] = add_strip(l, r, {});
    return "";
  };
  {
    std::string e = norm_of(0, 0);
    if (!e.empty()) return e;
  }
  P->term_strips.assign(P->terms.size(), {});
  for (size_t t = 0; t < comps.size(); ++t)
    for (auto &c : comps[t]) {
      std::string e = norm_of(c.lat, c.row);
      if (!e.empty()) return e;
      const int64_t k = add_strip(c.lat, c.row, c.ops);
      P->term_strips[t].push_back({k, norm_strip[{c.lat, c.row}]});
    }
  P->nstrips = (int64_t)sd.size();
  P->lognorm_strip = norm_strip[{0, 0}];
  if (std::max(std::max(l_cap, a1_cap), std::max(a2_cap, a3_cap)) >= ((int64_t)1 << 31))
    return "strip blocks of 2^31 elements or more are not supported";
  const int64_t per = l_cap + a1_cap + a2_cap + a3_cap;
  void *scr = B.buf((size_t)P->nstrips * per * as);
  P->strip_off = B.alloc((size_t)P->nstrips * as);
  for (int64_t i = 0; i < P->nstrips; ++i) {
    sd[i].scratch = (uint8_t *)scr + (size_t)i * per * as;
    sd[i].l_cap = l_cap; sd[i].a1_cap = a1_cap; sd[i].a2_cap = a2_cap; sd[i].a3_cap = a3_cap;
    sd[i].out = (uint8_t *)B.ptr(P->strip_off) + (size_t)i * as;
  }
  // log |<psi|psi>| from row 0: its strip and the scales of the sweep below it
  {
    const EnvSet &E = *envs[env_of[0][0]];
    P->lognorm_nlogs = E.has_bot ? E.bot.nsteps : 0;
    P->lognorm_logs_off = E.has_bot ? (size_t)((uintptr_t)E.bot_logs - base) : 0;
  }

  // --- ops: lattice copies, sweeps, strips
  {
    Op f;
    f.kind = Op::FILL; f.fill_ptr = ones; f.fill_n = 1; f.fill_value = 1.0; f.tag = "init";
    B.ops.push_back(f);
  }
  push_permute(B, Hf.perm, "lattice_copy");
  if (need_v) {
    push_permute(B, tpass, "lattice_copy");
    push_permute(B, Vt.perm, "lattice_copy");
    push_permute(B, Vf.perm, "lattice_copy");
  }
  // op ranges of the split: the prelude (status word, lattice copies) runs in
  // both sweep parts
  for (auto &r : P->part_ops) r.clear();
  const size_t prelude_end = B.ops.size();
  P->part_ops[0].push_back({0, prelude_end});
  P->part_ops[1].push_back({0, prelude_end});
  for (auto &E : envs) {
    if (grad) {
      if (E->has_top) emit_sweep_save(B, E->top, P->opts, E->top_rows, *E->tg, E->top_logs, E->top_sigma);
      if (E->has_bot) emit_sweep_save(B, E->bot, P->opts, E->bot_rows, *E->bg, E->bot_logs, E->bot_sigma);
      continue;
    }
    if (E->has_top) {
      const size_t a = B.ops.size();
      const int b = branch_of[&E->top];
      emit_sweep(B, E->top, P->opts, ones, E->top_rows, vbufs[b].data(), E->top_logs, E->top_sigma, owners[b]);
      for (size_t k = a; k < B.ops.size(); ++k) B.ops[k].branch = b;
      P->part_ops[0].push_back({a, B.ops.size()});
    }
    if (E->has_bot) {
      const size_t a = B.ops.size();
      const int b = branch_of[&E->bot];
      emit_sweep(B, E->bot, P->opts, ones, E->bot_rows, vbufs[b].data(), E->bot_logs, E->bot_sigma, owners[b]);
      for (size_t k = a; k < B.ops.size(); ++k) B.ops[k].branch = b;
      P->part_ops[1].push_back({a, B.ops.size()});
    }
  }
  P->splittable = !grad && P->use_cache;
  // operator table in the accumulation type
  std::vector<double> opflat;
  for (auto &m : optab) opflat.insert(opflat.end(), m.begin(), m.end());
  if (opflat.empty()) opflat.push_back(0.0);
  Op st;
  st.kind = Op::STRIP;
  st.desc_off = B.put(sd);
  st.aux_off[0] = B.put(cols);
  st.aux_off[1] = B.put(opflat);
  st.nd = (int)P->nstrips;
  st.tag = "strips";
  P->part_ops[2].assign(1, {B.ops.size(), B.ops.size() + 1});
  B.ops.push_back(st);
  if (!grad) return "";

  // ---- reverse sweep (second phase: the host sets the strip cotangents) ----
  P->split = B.ops.size();
  P->sbar_off = B.alloc((size_t)P->nstrips * 8);
  double *lzero = (double *)B.buf(8);
  push_memset(B, lzero, 8, "reverse_init");
  for (int l = 0; l < 4; ++l)
    for (int r = 0; r < (int)gl[l].size(); ++r)
      for (int q = 0; q < (int)gl[l][r].size(); ++q)
        push_memset(B, gl[l][r][q], site_elems(glat[l]->at(r, q)) * (int64_t)es, "reverse_init");
  for (auto &E : envs)
    for (SweepGrad *SGp : {E->tg.get(), E->bg.get()}) {
      if (!SGp) continue;
      const Sweep &S = SGp == E->tg.get() ? E->top : E->bot;
      for (int r = 0; r <= S.last; ++r)
        for (size_t q = 0; q < SGp->crow[r].size(); ++q)
          push_memset(B, SGp->crow[r][q], bsite_elems(S.bound[r][q]) * (int64_t)es, "reverse_init");
    }
  {
    const int64_t blk = l_cap, big = std::max(a1_cap, std::max(a2_cap, a3_cap));
    int maxc = 1;
    for (auto &x : sd) maxc = std::max(maxc, x.ncol);
    StripBwdScratch sc{};
    sc.blk = blk; sc.big = big;
    sc.per_strip = 2 * (int64_t)(maxc + 1) * blk + 6 * big;
    sc.base = (double *)B.buf((size_t)P->nstrips * sc.per_strip * 8);
    Op sb;
    sb.kind = Op::STRIPBWD;
    sb.desc_off = st.desc_off;
    sb.aux_off[0] = st.aux_off[0];
    sb.aux_off[1] = st.aux_off[1];
    sb.aux_off[2] = B.put(bcols);
    sb.nd = (int)P->nstrips;
    sb.sbar = (const double *)B.ptr(P->sbar_off);
    sb.sbs = sc;
    sb.tag = "strips_reverse";
    B.ops.push_back(sb);
  }
  for (auto &E : envs) {
    if (E->has_top) emit_sweep_bwd(B, E->top, P->opts, E->top_rows, *E->tg, lzero, E->top_logs, E->top_sigma);
    if (E->has_bot) emit_sweep_bwd(B, E->bot, P->opts, E->bot_rows, *E->bg, lzero, E->bot_logs, E->bot_sigma);
  }
  // lattice copies back onto the caller's lattice: un-flip (the same axis swap), un-transpose
  auto unflip = [&](const Net &src_dims, std::vector<std::vector<void *>> &gsrc, std::vector<std::vector<void *>> &gdst) {
    // gsrc on the flipped lattice (row p = original row nrow-1-p, [d][l][x][u][e])
    const int nrow = src_dims.nrow;
    for (int p = 0; p < nrow; ++p)
      for (int q = 0; q < src_dims.ncol; ++q) {
        const SiteDims f = src_dims.at(p, q);        // flipped dims: Du = original Dx, Dx = original Du
        void *tmp = B.buf(site_elems(f) * es);
        std::vector<PermuteDesc> pd{mk_permute(gsrc[p][q], tmp, (int64_t)f.d * f.Dl, f.Du, f.Dx, f.De)};
        push_permute(B, pd, "lattice_reverse");
        push_axpy(B, tmp, gdst[nrow - 1 - p][q], site_elems(f), "lattice_reverse");
      }
  };
  if (need_v) {
    unflip(Vf.net, gl[3], gl[1]);
    // Vt site (q,p) = [d][u][l][e][x] of H site (p,q): undo the (e,x) swap, then the (u,l) swap
    for (int p = 0; p < H.nrow; ++p)
      for (int q = 0; q < H.ncol; ++q) {
        const SiteDims x = H.at(p, q);
        void *t1 = B.buf(site_elems(x) * es), *t2 = B.buf(site_elems(x) * es);
        std::vector<PermuteDesc> a{mk_permute(gl[1][q][p], t1, (int64_t)x.d * x.Du * x.Dl, x.De, x.Dx, 1)};
        push_permute(B, a, "lattice_reverse");
        std::vector<PermuteDesc> b{mk_permute(t1, t2, x.d, x.Du, x.Dl, (int64_t)x.Dx * x.De)};
        push_permute(B, b, "lattice_reverse");
        push_axpy(B, t2, gl[0][p][q], site_elems(x), "lattice_reverse");
      }
  }
  unflip(Hf.net, gl[2], gl[0]);
  for (int p = 0; p < H.nrow; ++p)
    for (int q = 0; q < H.ncol; ++q) {
      void *dst = P->grad_site.empty() ? nullptr : P->grad_site[(size_t)p * H.ncol + q];
      if (dst) push_copy(B, dst, gl[0][p][q], site_elems(H.at(p, q)) * (int64_t)es, "gradient_out");
    }
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
          if (c.Tlow) C.need(c.Tlow, es * n2, tag, "Tlow");
          if (c.Tlow && (!op.wide || !c.T)) C.err = std::string(tag) + ": Tlow needs an FP64 factorisation with T";
          if (c.n > 1024) C.err = std::string(tag) + ": n above the pivot-flag buffer";
          if (c.status) C.need(c.status, 4, tag, "status");
          if (op.smem < small_smem_bytes(op.wide ? (dt | 2) : dt, c.n))
            C.err = std::string(tag) + ": shared memory too small";
          if (op.smem2 < chol_cluster_smem_bytes(op.wide ? (dt | 2) : dt, c.n, c.T != nullptr))
            C.err = std::string(tag) + ": cluster shared memory too small";
        }
        break;
      case Op::JACOBI:
        for (int i = 0; i < op.nd; ++i) {
          const JacobiDesc &j = ((const JacobiDesc *)d)[i];
          const int jdt = op.wide ? (dt | 2) : dt;
          const double jes = dtype_size(jdt);
          C.need(j.Rb, jes * (double)j.n * j.n, tag, "Rb");
          C.need(j.Mw, jes * (double)j.n * j.n, tag, "Mw");
          if (op.smem < small_smem_bytes(jdt, j.n)) C.err = std::string(tag) + ": shared memory too small";
          if (op.smem2 < jacobi_block_smem_bytes(jdt, j.n) || op.smem3 < jacobi_cluster_smem_bytes(jdt, j.n))
            C.err = std::string(tag) + ": cluster shared memory too small";
          if (op.blocks < j.n) C.err = std::string(tag) + ": sigma refinement grid too small";
          C.need(j.sig, 8.0 * j.n, tag, "sig");
          if (j.status) C.need(j.status, 4, tag, "status");
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
          C.need(f.h, as * (double)f.n, tag, "h");
          if (f.status) C.need(f.status, 4, tag, "status");
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
        if (t.status) C.need(t.status, 4, tag, "status");
        if (op.tc_kr % 4 || t.Kr != op.tc_kr) C.err = std::string(tag) + ": TMA rows not 16-byte aligned";
        if (t.bpre) {
          if (t.Braw != op.tcB || !t.split3 || op.tc_bn > 192) C.err = std::string(tag) + ": bad B pre-expansion";
          C.need(t.Bx, (double)tc_bx_bytes(op.tcB_rows, op.tc_kr, t.cplx != 0), tag, "Bx");
        }
        break;
      }
      case Op::COPY:
        C.need(op.aux_ptr, (double)op.fill_n, tag, "src");
        C.need(op.fill_ptr, (double)op.fill_n, tag, "dst");
        break;
      case Op::MEMSET:
        C.need(op.fill_ptr, (double)op.fill_n, tag, "dst");
        break;
      case Op::NARROW:
        C.need(op.aux_ptr, 8.0 * op.fill_n, tag, "src");
        C.need(op.fill_ptr, 4.0 * op.fill_n, tag, "dst");
        break;
      case Op::BLOBCOPY:
        C.need(op.fill_ptr, (double)op.fill_n, tag, "dst");
        if (op.aux_off[0] + (size_t)op.fill_n > P->blob.size()) C.err = std::string(tag) + ": source beyond the blob";
        break;
      case Op::THETA:
        for (int i = 0; i < op.nd; ++i) {
          const ThetaDesc &t = ((const ThetaDesc *)d)[i];
          const double n = (double)t.d * t.Db;
          C.need(t.R1, es * t.r1 * n, tag, "R1");
          C.need(t.R2, es * t.r2 * n, tag, "R2");
          C.need(t.G, es * (double)t.d * t.d * t.d * t.d, tag, "G");
          C.need(t.Theta, es * (double)t.r1 * t.d * t.r2 * t.d, tag, "Theta");
        }
        break;
      case Op::SVDSMALL:
        for (int i = 0; i < op.nd; ++i) {
          const SvdSmallDesc &v = ((const SvdSmallDesc *)d)[i];
          if (v.rows > kSvdSmallMax || v.cols > kSvdSmallMax || v.k > v.rows || v.k > v.cols || v.k < 1)
            C.err = std::string(tag) + ": Theta size out of range";
          if (op.smem < svd_small_smem_bytes(dt, v.rows, v.cols)) C.err = std::string(tag) + ": shared memory too small";
          C.need(v.Theta, es * (double)v.rows * v.cols, tag, "Theta");
          C.need(v.R1t, es * (double)v.rows * v.k, tag, "R1t");
          C.need(v.R2t, es * (double)v.cols * v.k, tag, "R2t");
          if (v.sigma) C.need(v.sigma, 8.0 * v.k, tag, "sigma");
          if (v.status) C.need(v.status, 4, tag, "status");
        }
        break;
      case Op::SITEOP:
        if (op.blocks < 1 || op.blocks > 65535 || op.nd > 65535) C.err = std::string(tag) + ": grid out of range";
        for (int i = 0; i < op.nd; ++i) {
          const SiteOpDesc &x = ((const SiteOpDesc *)d)[i];
          if (x.d < 1 || x.d > kSiteOpMaxPhys) C.err = std::string(tag) + ": physical dimension out of range";
          C.need(x.M, es * (double)x.d * x.rest, tag, "M");
          C.need(x.g, es * (double)x.d * x.d, tag, "g");
        }
        break;
      case Op::SITEGAUGE:
        for (int i = 0; i < op.nd; ++i) {
          const SiteGaugeDesc &g = ((const SiteGaugeDesc *)d)[i];
          if (g.k > kSvdSmallMax) C.err = std::string(tag) + ": bond above the phase buffer";
          C.need(g.N1, es * (double)g.rows1 * g.k, tag, "N1");
          C.need(g.N2, es * (double)g.rows2 * g.k, tag, "N2");
          C.need(g.g, es * (double)g.rows1, tag, "g");
        }
        break;
      case Op::ABSORB:
        C.need(op.absorb.U, es * (double)op.absorb.M * op.absorb.k, tag, "U");
        C.need(op.absorb.W, es * (double)op.absorb.k * op.absorb.N, tag, "W");
        C.need(op.absorb.sigma, 8.0 * op.absorb.k, tag, "sigma");
        break;
      case Op::AXPY:
        C.need(op.aux_ptr, es * (double)op.fill_n, tag, "x");
        C.need(op.fill_ptr, es * (double)op.fill_n, tag, "y");
        break;
      case Op::SITEBWD: {
        const SiteBwdDesc &x = *(const SiteBwdDesc *)d;
        if (x.mode == 0) {
          const double nk = (double)x.d * x.Dl * x.Dx * x.De;
          C.need(x.K, es * nk, tag, "K");
          C.need(x.Kbar, es * nk, tag, "Kbar");
          C.need(x.cot, es * (double)x.Dl * x.Dl * x.Dx * x.Dx * x.De * x.De, tag, "cot");
        } else {
          const double nk = (double)x.d * x.Du * x.Dx * x.De, ns = (double)x.Du * x.Du * x.B;
          C.need(x.K, es * nk, tag, "K");
          C.need(x.Kbar, es * nk, tag, "Kbar");
          C.need(x.S, es * ns, tag, "S");
          C.need(x.Sbar, es * ns, tag, "Sbar");
          C.need(x.cot, es * (double)x.Dx * x.Dx * x.B * x.De * x.De, tag, "cot");
        }
        break;
      }
      case Op::STRIPBWD: {
        const StripCol *cl = (const StripCol *)(blob + op.aux_off[0]);
        const StripBwdCol *bl = (const StripBwdCol *)(blob + op.aux_off[2]);
        C.need(op.sbar, 8.0 * op.nd, tag, "sbar");
        C.need(op.sbs.base, 8.0 * op.nd * op.sbs.per_strip, tag, "scratch");
        for (int i = 0; i < op.nd; ++i) {
          const StripDesc &x = ((const StripDesc *)d)[i];
          if (2 * (int64_t)(x.ncol + 1) * op.sbs.blk + 6 * op.sbs.big > op.sbs.per_strip)
            C.err = std::string(tag) + ": scratch slice too small";
          for (int q = 0; q < x.ncol && q < kStripMaxCols; ++q) {
            const StripCol &c = cl[x.col0 + q];
            const StripBwdCol &b = bl[x.col0 + q];
            const double vu = (double)c.Du * c.Du, vd = (double)c.Dx * c.Dx;
            if (b.cot_up) C.need(b.cot_up, es * c.a * vu * c.b, tag, "cot_up");
            if (b.cot_lo) C.need(b.cot_lo, es * c.c * vd * c.f, tag, "cot_lo");
            C.need(b.cot_ket, es * (double)c.d * c.Dl * c.Du * c.Dx * c.De, tag, "cot_ket");
            const double blk = std::max((double)c.a * c.Dl * c.Dl * c.c, (double)c.b * c.De * c.De * c.f);
            const double big = std::max({(double)c.Dl * c.Dl * c.c * vu * c.b,
                                         (double)c.Dl * c.c * c.Du * c.b * c.d * c.Dx * c.De,
                                         (double)c.c * c.b * c.De * c.Dx * c.Dx * c.De});
            if (blk > op.sbs.blk || big > op.sbs.big) C.err = std::string(tag) + ": scratch blocks too small";
          }
        }
        break;
      }
      case Op::LTU:
        C.need(op.aux_ptr, es * (double)op.fill_n * op.fill_n, tag, "M");
        C.need(op.fill_ptr, es * (double)op.fill_n * op.fill_n, tag, "out");
        break;
      case Op::SVDBWD: {
        const SvdBwdDesc &x = *(const SvdBwdDesc *)d;
        const double n = x.n, k = x.k;
        C.need(x.Mw, es * n * n, tag, "Mw");
        C.need(x.sig, 8 * n, tag, "sig");
        C.need(x.Ut, es * n * k, tag, "Ut");
        C.need(x.Utbar, es * n * k, tag, "Utbar");
        C.need(x.WW, es * k * k, tag, "WW");
        C.need(x.H, es * n * n, tag, "H");
        C.need(x.scratch, 8 * (3 * n * n + n) + 4 * n, tag, "scratch");
        C.need(x.lbar, 8, tag, "lbar");
        C.need(x.inv_s1, 8, tag, "inv_s1");
        break;
      }
      case Op::TGRAD: {
        const TensorGradDesc &x = *(const TensorGradDesc *)d;
        const double nk = (double)x.d * x.Dl * x.Du * x.Dx * x.De, nkb = (double)x.d * x.DL * x.DU * x.DX * x.DE;
        const double N = (double)x.Dx * x.DX * x.b * x.De * x.DE;
        C.need(x.Z2, es * x.P * (double)x.Dl * x.DL * x.Du * x.DU * x.b, tag, "Z2");
        C.need(x.R, es * x.P * N, tag, "R");
        C.need(x.K, es * nk, tag, "K");
        C.need(x.Kb, es * nkb, tag, "Kb");
        C.need(x.Kbar, es * nk, tag, "Kbar");
        C.need(x.Kbbar, es * nkb, tag, "Kbbar");
        break;
      }
      case Op::STRIP: {
        const StripCol *cl = (const StripCol *)(blob + op.aux_off[0]);
        for (int i = 0; i < op.nd; ++i) {
          const StripDesc &x = ((const StripDesc *)d)[i];
          if (x.ncol > kStripMaxCols) C.err = std::string(tag) + ": too many columns";
          for (int q = 0; q < x.ncol && q < kStripMaxCols; ++q) {
            const StripCol &c = cl[x.col0 + q];
            C.need(c.up, es * (double)c.a * c.Du * c.Du * c.b, tag, "up");
            C.need(c.lo, es * (double)c.c * c.Dx * c.Dx * c.f, tag, "lo");
            C.need(c.ket, es * (double)c.d * c.Dl * c.Du * c.Dx * c.De, tag, "ket");
            const double vu = (double)c.Du * c.Du;
            if ((double)c.a * c.Dl * c.Dl * c.c > x.l_cap || (double)c.b * c.De * c.De * c.f > x.l_cap ||
                (double)c.Dl * c.Dl * c.c * vu * c.b > x.a1_cap ||
                (double)c.Dl * c.c * c.Du * c.b * c.d * c.Dx * c.De > x.a2_cap ||
                (double)c.c * c.b * c.De * c.Dx * c.Dx * c.De > x.a3_cap)
              C.err = std::string(tag) + ": strip scratch too small";
          }
          C.need(x.scratch, as * ((double)x.l_cap + x.a1_cap + x.a2_cap + x.a3_cap), tag, "scratch");
          C.need(x.out, as, tag, "out");
        }
        break;
      }
      case Op::PAD:
        for (int i = 0; i < op.nd; ++i) {
          const PadDesc &q = ((const PadDesc *)d)[i];
          double tot = 1, span = 0;
          bool ok = q.nd >= 1 && q.nd <= 6;
          for (int k = 0; ok && k < q.nd; ++k) {
            ok = q.dims[k] >= 1 && q.lim[k] >= 1 && q.lim[k] <= q.dims[k] && q.in_stride[k] >= 0;
            tot *= q.dims[k];
            span += (double)(q.lim[k] - 1) * q.in_stride[k];
          }
          if (!ok || tot != (double)q.total) { C.err = std::string(tag) + ": bad pad descriptor"; break; }
          C.need(q.in, es * (span + 1), tag, "in");
          C.need(q.out, es * tot, tag, "out");
        }
        break;
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

// One TEBD layer (Algorithm 1 on every bond): two horizontal passes (bonds
// starting at even, then odd columns) and two vertical ones, the bonds of a
// pass disjoint; each pass's launches are grouped over its bonds.  The sites
// are updated in place; the gate is copied from the descriptor blob into
// the workspace by the first launch.
std::string build_tebd(peps_plan *P, uintptr_t base, Builder &B) {
  B.base = base;
  B.dt = P->dt;
  const Net &H = P->ket;
  const int nrow = H.nrow, ncol = H.ncol;
  void *gate = B.buf(P->gate.size());
  {
    Op op;
    op.kind = Op::BLOBCOPY; op.fill_ptr = gate; op.aux_off[0] = B.put_bytes(P->gate.data(), P->gate.size());
    op.fill_n = (int64_t)P->gate.size(); op.tag = "tebd_gate";
    B.ops.push_back(op);
  }
  const int d = H.d, es = dtype_size(P->dt);
  const size_t g2 = (size_t)d * d * d * d * es, g1 = (size_t)d * d * es;
  auto site = [&](int i, int *dims) {
    const SiteDims &s = H.dims[i];
    dims[0] = s.d; dims[1] = s.Dl; dims[2] = s.Du; dims[3] = s.Dx; dims[4] = s.De;
    return const_cast<void *>(H.site[i]);
  };
  // one-site operators (Eq. 4) before the bonds
  if (P->nsite_gates) {
    std::vector<SiteOpDesc> so;
    const uint8_t *g0 = (const uint8_t *)gate + P->ngates * g2;
    for (int i = 0; i < nrow * ncol; ++i) {
      int dims[5];
      SiteOpDesc x{};
      x.M = site(i, dims);
      x.g = g0 + (P->nsite_gates == 1 ? 0 : (size_t)i * g1);
      x.d = dims[0];
      x.rest = (int64_t)dims[1] * dims[2] * dims[3] * dims[4];
      so.push_back(x);
    }
    emit_site_ops(B, so);
  }
  // position of the bond a-b in bond order (horizontal by left site, then vertical by upper site)
  auto bond_gate = [&](int a, int b) {
    if (P->ngates == 1) return (const void *)gate;
    const int p = a / ncol, q = a % ncol;
    const int64_t idx = b == a + 1 ? (int64_t)p * (ncol - 1) + q : (int64_t)nrow * (ncol - 1) + (int64_t)p * ncol + q;
    return (const void *)((const uint8_t *)gate + idx * g2);
  };
  for (int vertical = 0; vertical < 2; ++vertical)
    for (int start = 0; start < 2; ++start) {
      std::vector<TebdBond> bonds;
      if (!vertical) {
        for (int p = 0; p < nrow; ++p)
          for (int q = start; q < ncol - 1; q += 2) {
            TebdBond t;
            t.a = p * ncol + q; t.b = t.a + 1;
            bonds.push_back(t);
          }
      } else {
        for (int p = start; p < nrow - 1; p += 2)
          for (int q = 0; q < ncol; ++q) {
            TebdBond t;
            t.a = p * ncol + q; t.b = t.a + ncol; t.vertical = true;
            bonds.push_back(t);
          }
      }
      if (bonds.empty()) continue;
      for (TebdBond &t : bonds) {
        t.M1 = site(t.a, t.s1);
        t.M2 = site(t.b, t.s2);
        std::string e = tebd_bond_shape(t);
        if (!e.empty()) return e;
        tebd_alloc(B, t, P->dt);
        t.gate = bond_gate(t.a, t.b);
      }
      emit_tebd_pass(B, bonds, P->opts.seed, P->opts.unit_bond);
    }
  return "";
}

peps_status rebuild(peps_plan *P, void *ws, const peps_einsumsvd_io *io, bool encode = false) {
  Builder B;
  B.encode = encode;
  // the status word first (workspace offset 0), cleared by the first launch
  B.base = (uintptr_t)ws;
  B.dt = P->dt;
  P->status_off = B.alloc(256);
  B.status = (uint32_t *)B.ptr(P->status_off);
  {
    std::vector<ZeroDesc> d{ZeroDesc{B.status, 1}};
    std::vector<int64_t> prefix{0};
    Op op;
    op.kind = Op::ZERO; op.desc_off = B.put(d); op.prefix_off = B.put(prefix); op.nd = 1; op.blocks = 1;
    op.tag = "status";
    B.ops.push_back(op);
  }
  std::string e = P->kind == peps_plan::EINSUMSVD ? build_einsumsvd(P, (uintptr_t)ws, io, B)
                  : P->kind == peps_plan::CONTRACT ? build_contract(P, (uintptr_t)ws, B)
                  : P->kind == peps_plan::EGRAD    ? build_egrad(P, (uintptr_t)ws, io, B)
                  : P->kind == peps_plan::TEBD     ? build_tebd(P, (uintptr_t)ws, B)
                                                   : build_expect(P, (uintptr_t)ws, B);
  if (!e.empty()) return fail(PEPS_ERR_SHAPE, "%s", e.c_str());
  tc_finish(B);
  if (!B.err.empty()) return fail(PEPS_ERR_UNSUPPORTED, "%s", B.err.c_str());
  for (Op &op : B.ops) {
    if (op.kind != Op::TC) continue;
    op.tc.wait_ns = P->wait_ns;
    if (!encode || P->tune.empty()) continue;
    auto it = P->tune.find(tc_signature(op));
    if (it != P->tune.end() && it->second != op.tc_bn && !tc_retile(op, it->second))
      return fail(PEPS_ERR_UNSUPPORTED, "tuned MMA width %d not encodable for %s", it->second, op.tag.c_str());
  }
  P->ws_bytes = finish(B, &P->blob_off);   // needs the blob size: before the move
  P->ops = std::move(B.ops);
  P->blob = std::move(B.blob);
  return PEPS_OK;
}

// Status of the device word read back after a synchronisation: a wait that
// gave up outranks a non-finite value; Jacobi non-convergence alone is not an
// error (peps_poll reports it).
static_assert(PEPS_STATUS_NONFINITE == STATUS_NONFINITE && PEPS_STATUS_JACOBI_NOCONV == STATUS_JACOBI_NOCONV &&
                  PEPS_STATUS_TIMEOUT == STATUS_TIMEOUT,
              "status bits of the ABI and the kernels differ");
peps_status status_of(uint32_t w) {
  if (w & STATUS_TIMEOUT) return fail(PEPS_ERR_TIMEOUT, "a tensor-core pipeline wait gave up (status 0x%x)", w);
  if (w & STATUS_NONFINITE) return fail(PEPS_ERR_NUMERIC, "non-finite singular value met (status 0x%x)", w);
  return PEPS_OK;
}

peps_status enqueue(peps_plan *P, void *ws, size_t ws_bytes, cudaStream_t s0, bool upload,
                    cudaEvent_t *events = nullptr, size_t first = 0, size_t last = SIZE_MAX) {
  cudaStream_t s = s0;
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
  last = std::min(last, P->ops.size());
  // branches > 0 run on the plan's side streams, forked from the caller's
  // stream just before the first op of a branch > 0 (so they see every
  // earlier op of the range, e.g. the status word's clear and the lattice
  // copies) and joined back after the last launch (the profiling replay
  // keeps every launch on the caller's stream, one after the other)
  int nbr = 1;
  for (size_t oi = first; oi < last; ++oi) nbr = std::max(nbr, P->ops[oi].branch + 1);
  const bool fork = nbr > 1 && !events;
  size_t fork_at = last;
  if (fork) {
    while ((int)P->side.size() < nbr - 1) {
      cudaStream_t st = nullptr;
      CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      P->side.push_back(st);
    }
    while ((int)P->side_ev.size() < nbr) {
      cudaEvent_t ev = nullptr;
      CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      P->side_ev.push_back(ev);
    }
    for (size_t oi = first; oi < last; ++oi)
      if (P->ops[oi].branch > 0) { fork_at = oi; break; }
  }
  for (size_t oi = first; oi < last; ++oi) {
    if (fork && oi == fork_at) {
      CUDA_TRY(cudaEventRecord(P->side_ev[0], s0));
      for (int b = 1; b < nbr; ++b) CUDA_TRY(cudaStreamWaitEvent(P->side[b - 1], P->side_ev[0], 0));
    }
    const Op &op = P->ops[oi];
    s = fork && op.branch > 0 ? P->side[op.branch - 1] : s0;
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
      case Op::JACOBI:
        launch_jacobi(op.wide ? (dt | 2) : dt, (const JacobiDesc *)d, op.nd, op.smem, op.smem2, op.smem3,
                      (int)op.blocks, s);
        break;
      case Op::NARROW: launch_narrow((const double *)op.aux_ptr, (float *)op.fill_ptr, op.fill_n, s); break;
      case Op::FINALIZE: launch_finalize(dt, (const FinalizeDesc *)d, op.nd, (int)op.blocks, s); break;
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
      case Op::PAD: launch_pad(dt, (const PadDesc *)d, pre, op.nd, op.blocks, s); break;
      case Op::STRIP:
        launch_strip(dt, (const StripDesc *)d, (const StripCol *)(blob + op.aux_off[0]), blob + op.aux_off[1], op.nd,
                     s);
        break;
      case Op::COPY:
        CUDA_TRY(cudaMemcpyAsync(op.fill_ptr, op.aux_ptr, (size_t)op.fill_n, cudaMemcpyDeviceToDevice, s));
        break;
      case Op::SVDBWD: launch_svd_bwd(dt, *(const SvdBwdDesc *)(P->blob.data() + op.desc_off), s); break;
      case Op::LTU: launch_copyltu(dt, op.aux_ptr, op.fill_ptr, (int)op.fill_n, s); break;
      case Op::TGRAD: launch_tensor_grad(dt, *(const TensorGradDesc *)(P->blob.data() + op.desc_off), s); break;
      case Op::MEMSET: CUDA_TRY(cudaMemsetAsync(op.fill_ptr, 0, (size_t)op.fill_n, s)); break;
      case Op::AXPY: launch_axpy(dt, op.aux_ptr, op.fill_ptr, op.fill_n, s); break;
      case Op::ABSORB: launch_absorb(dt, op.absorb, s); break;
      case Op::THETA: launch_tebd(dt, 0, d, op.nd, 0, s); break;
      case Op::SVDSMALL: launch_tebd(dt, 1, d, op.nd, op.smem, s); break;
      case Op::SITEGAUGE: launch_tebd(dt, 2, d, op.nd, 0, s); break;
      case Op::SITEOP: launch_tebd(dt, 3, d, op.nd, (int)op.blocks, s); break;
      case Op::BLOBCOPY:
        CUDA_TRY(cudaMemcpyAsync(op.fill_ptr, blob + op.aux_off[0], (size_t)op.fill_n, cudaMemcpyDeviceToDevice, s));
        break;
      case Op::SITEBWD: launch_site_bwd(dt, *(const SiteBwdDesc *)(P->blob.data() + op.desc_off), s); break;
      case Op::STRIPBWD:
        launch_strip_bwd(dt, (const StripDesc *)d, (const StripCol *)(blob + op.aux_off[0]),
                         (const StripBwdCol *)(blob + op.aux_off[2]), (const double *)(blob + op.aux_off[1]), op.sbar,
                         op.sbs, op.nd, s);
        break;
    }
    if (events) CUDA_TRY(cudaEventRecord(events[&op - P->ops.data() + 1], s));
  }
  if (fork)
    for (int b = 1; b < nbr; ++b) {
      CUDA_TRY(cudaEventRecord(P->side_ev[b], P->side[b - 1]));
      CUDA_TRY(cudaStreamWaitEvent(s0, P->side_ev[b], 0));
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
  if (opts->flags & PEPS_FLAG_UNIT_BOND)
    return fail(PEPS_ERR_UNSUPPORTED, "PEPS_FLAG_UNIT_BOND applies to TEBD plans only");
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::EINSUMSVD;
  P->dt = dtype;
  P->opts = to_opts(opts);
  if (P->opts.alternate)
    return fail(PEPS_ERR_UNSUPPORTED, "alternating canonicalisation applies to contraction plans only");
  for (int i = 0; i < batch; ++i) {
    const peps_einsumsvd_shape &s = shapes[i];
    Inst I{};
    I.kL = s.kL; I.t = s.t; I.a = s.a; I.b = s.b; I.d = s.d;
    I.Dl = s.Dl; I.Du = s.Du; I.Dx = s.Dx; I.De = s.De;
    I.DL = s.DL; I.DU = s.DU; I.DX = s.DX; I.DE = s.DE;
    std::string e = inst_check(I, dtype);
    if (!e.empty()) return fail(PEPS_ERR_SHAPE, "instance %d: %s", i, e.c_str());
    if (s.m < 0) return fail(PEPS_ERR_ARG, "instance %d: negative rank", i);
    RsvdOpts oi = P->opts;
    if (s.m > 0) oi.m = s.m;
    inst_derive(I, oi);
    I.instance = instance_ids ? instance_ids[i] : (uint64_t)i;
    I.tc = P->opts.prec != PEPS_PREC_PLAIN && inst_tc_ok(I, dtype);
    Inst E{};
    I.embed = P->opts.prec != PEPS_PREC_PLAIN && !I.tc && inst_embed_dims(I, dtype, oi, E);
    P->insts.push_back(I);
  }
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_einsumsvd_set_branches(peps_plan *plan, int32_t branches, size_t *workspace_bytes) {
  g_last_error.clear();
  if (!plan || !workspace_bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EINSUMSVD) return fail(PEPS_ERR_ARG, "not an einsumsvd plan");
  if (branches < 1 || branches > kMaxBranches) return fail(PEPS_ERR_ARG, "branches must be in 1..%d", kMaxBranches);
  plan->branches = branches;
  plan->built = false;
  if (peps_status s = rebuild(plan, nullptr, nullptr)) return s;
  *workspace_bytes = plan->ws_bytes;
  return PEPS_OK;
}

peps_status peps_einsumsvd_rank(const peps_plan *plan, int32_t i, int32_t *k) {
  if (!plan || !k) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EINSUMSVD && plan->kind != peps_plan::EGRAD)
    return fail(PEPS_ERR_ARG, "not an einsumsvd plan");
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

peps_status peps_einsumsvd_grad_plan(peps_plan **out, peps_dtype dtype, const peps_einsumsvd_shape *shape,
                                     const peps_rsvd_opts *opts, size_t *workspace_bytes) {
  g_last_error.clear();
  if (!out || !shape || !workspace_bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (dtype != PEPS_R32 && dtype != PEPS_R64) return fail(PEPS_ERR_UNSUPPORTED, "the adjoint takes real data");
  if (peps_status s = check_opts(opts)) return s;
  if (opts->flags & PEPS_FLAG_UNIT_BOND)
    return fail(PEPS_ERR_UNSUPPORTED, "PEPS_FLAG_UNIT_BOND applies to TEBD plans only");
  if (opts->prec != PEPS_PREC_PLAIN) return fail(PEPS_ERR_UNSUPPORTED, "the adjoint runs the plain arithmetic");
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::EGRAD;
  P->dt = dtype;
  P->opts = to_opts(opts);
  if (P->opts.alternate)
    return fail(PEPS_ERR_UNSUPPORTED, "alternating canonicalisation applies to contraction plans only");
  const peps_einsumsvd_shape &s = *shape;
  Inst I{};
  I.kL = s.kL; I.t = s.t; I.a = s.a; I.b = s.b; I.d = s.d;
  I.Dl = s.Dl; I.Du = s.Du; I.Dx = s.Dx; I.De = s.De;
  I.DL = s.DL; I.DU = s.DU; I.DX = s.DX; I.DE = s.DE;
  std::string e = inst_check(I, dtype);
  if (!e.empty()) return fail(PEPS_ERR_SHAPE, "%s", e.c_str());
  if (s.m < 0) return fail(PEPS_ERR_ARG, "negative rank");
  RsvdOpts oi = P->opts;
  if (s.m > 0) oi.m = s.m;
  inst_derive(I, oi);
  I.instance = 0;
  I.tc = false;
  P->insts.push_back(I);
  if (peps_status st = rebuild(P.get(), nullptr, nullptr)) return st;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_einsumsvd_grad_bind(peps_plan *plan, const peps_einsumsvd_cotangent *ct,
                                     const peps_einsumsvd_grads *gr) {
  if (!plan || !ct || !gr) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EGRAD) return fail(PEPS_ERR_ARG, "not an adjoint plan");
  plan->ct = *ct;
  plan->gr = *gr;
  plan->built = false;
  return PEPS_OK;
}

peps_status peps_einsumsvd_grad_execute(peps_plan *plan, const peps_einsumsvd_io *io,
                                        const peps_einsumsvd_cotangent *ct, const peps_einsumsvd_grads *gr,
                                        void *workspace, size_t workspace_bytes, void *stream) {
  g_last_error.clear();
  if (!plan || !io || !ct || !gr) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EGRAD) return fail(PEPS_ERR_ARG, "not an adjoint plan");
  if (!io->V || !io->S || !io->ket || !io->bra || !io->U || !io->W || !io->sigma)
    return fail(PEPS_ERR_ARG, "NULL tensor pointer");
  if (!gr->V_bar || !gr->S_bar || !gr->ket_bar || !gr->bra_bar) return fail(PEPS_ERR_ARG, "NULL gradient pointer");
  if (!ct->U_bar || !ct->W_bar) return fail(PEPS_ERR_ARG, "U_bar and W_bar are required (pass zeros for none)");
  bool same = plan->built && plan->built_base == (uintptr_t)workspace && plan->io_cache.size() == 1 &&
              memcmp(&plan->io_cache[0], io, sizeof *io) == 0 && memcmp(&plan->ct, ct, sizeof *ct) == 0 &&
              memcmp(&plan->gr, gr, sizeof *gr) == 0;
  if (!same) {
    plan->ct = *ct;
    plan->gr = *gr;
    if (peps_status s = rebuild(plan, workspace, io, true)) return s;
    plan->io_cache.assign(io, io + 1);
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
  if (opts->flags & PEPS_FLAG_UNIT_BOND)
    return fail(PEPS_ERR_UNSUPPORTED, "PEPS_FLAG_UNIT_BOND applies to TEBD plans only");
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

peps_status peps_tebd_plan(peps_plan **out, const peps_network *net, const double *gates, int64_t ngates,
                           const double *site_gates, int64_t nsite_gates, const peps_rsvd_opts *opts,
                           size_t *workspace_bytes) {
  g_last_error.clear();
  if (!out || !workspace_bytes || !gates) return fail(PEPS_ERR_ARG, "NULL argument");
  if (nsite_gates < 0 || (nsite_gates > 0 && !site_gates)) return fail(PEPS_ERR_ARG, "bad one-site operators");
  if (peps_status s = check_opts(opts)) return s;
  if (opts->prec != PEPS_PREC_PLAIN) return fail(PEPS_ERR_UNSUPPORTED, "the TEBD layer runs the plain arithmetic");
  if (opts->flags & ~PEPS_FLAG_UNIT_BOND)
    return fail(PEPS_ERR_UNSUPPORTED, "only PEPS_FLAG_UNIT_BOND applies to the TEBD layer");
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::TEBD;
  P->opts = to_opts(opts);
  if (peps_status s = read_net(net, P->ket, "network")) return s;
  P->dt = P->ket.dt;
  if (P->ket.nrow > 0xFFFF || P->ket.ncol > 0xFFFF || (int64_t)P->ket.nrow * P->ket.ncol > 0xFFFF)
    return fail(PEPS_ERR_UNSUPPORTED, "lattice too large");
  const int d = P->ket.d;
  const int64_t nr = P->ket.nrow, nc = P->ket.ncol;
  const int64_t nbonds = nr * (nc - 1) + (nr - 1) * nc, nsites = nr * nc;
  if (ngates != 1 && ngates != nbonds)
    return fail(PEPS_ERR_ARG, "ngates = %lld: 1 or the number of bonds (%lld)", (long long)ngates,
                (long long)nbonds);
  if (nsite_gates != 0 && nsite_gates != 1 && nsite_gates != nsites)
    return fail(PEPS_ERR_ARG, "nsite_gates = %lld: 0, 1 or the number of sites (%lld)", (long long)nsite_gates,
                (long long)nsites);
  if (nsite_gates && d > kSiteOpMaxPhys)
    return fail(PEPS_ERR_UNSUPPORTED, "one-site operators need d <= %d", kSiteOpMaxPhys);
  const int64_t n2 = (int64_t)d * d * d * d, n1 = (int64_t)d * d;
  const bool cplx = dtype_complex(P->dt), dbl = dtype_double(P->dt);
  const int es = dtype_size(P->dt);
  P->ngates = ngates;
  P->nsite_gates = nsite_gates;
  P->gate.resize((size_t)(ngates * n2 + nsite_gates * n1) * es);
  auto put = [&](const double *src, int64_t count, uint8_t *dst) {
    for (int64_t i = 0; i < count; ++i, dst += es) {
      const double re_ = src[cplx ? 2 * i : i], im_ = cplx ? src[2 * i + 1] : 0.0;
      if (dbl) {
        memcpy(dst, &re_, 8);
        if (cplx) memcpy(dst + 8, &im_, 8);
      } else {
        const float fr = (float)re_, fi = (float)im_;
        memcpy(dst, &fr, 4);
        if (cplx) memcpy(dst + 4, &fi, 4);
      }
    }
  };
  put(gates, ngates * n2, P->gate.data());
  if (nsite_gates) put(site_gates, nsite_gates * n1, P->gate.data() + ngates * n2 * es);
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_tebd_execute(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream) {
  g_last_error.clear();
  if (!plan) return fail(PEPS_ERR_ARG, "plan is NULL");
  if (plan->kind != peps_plan::TEBD) return fail(PEPS_ERR_ARG, "not a TEBD plan");
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

peps_status peps_poll(const peps_plan *plan, const void *workspace, void *stream, uint32_t *flags) {
  g_last_error.clear();
  if (!plan || !workspace) return fail(PEPS_ERR_ARG, "NULL argument");
  if (!plan->built) return fail(PEPS_ERR_ARG, "plan was never executed");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "status read during stream capture");
  uint32_t word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, (const uint8_t *)workspace + plan->status_off, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (flags) *flags = word;
  return status_of(word);
}

peps_status peps_plan_autotune(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream,
                               int32_t reps) {
  g_last_error.clear();
  if (!plan || !workspace) return fail(PEPS_ERR_ARG, "NULL argument");
  if (!plan->built || plan->built_base != (uintptr_t)workspace)
    return fail(PEPS_ERR_ARG, "execute the plan with this workspace before tuning it");
  if (workspace_bytes < plan->ws_bytes) return fail(PEPS_ERR_WORKSPACE, "workspace too small");
  if (reps < 1 || reps > 100) return fail(PEPS_ERR_ARG, "reps must be in 1..100");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "tuning during stream capture");
  // one representative launch per shape; every candidate width timed on it
  std::map<std::string, std::vector<size_t>> groups;
  for (size_t i = 0; i < plan->ops.size(); ++i)
    if (plan->ops[i].kind == Op::TC) groups[tc_signature(plan->ops[i])].push_back(i);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  peps_status st = PEPS_OK;
  for (auto &g : groups) {
    Op &rep = plan->ops[g.second.front()];
    const int orig = rep.tc_bn;
    int best = orig;
    float best_ms = -1.f;
    for (int c : tc_candidates(rep)) {
      if (!tc_retile(rep, c)) continue;
      launch_tc_gemm(rep.tc, rep.tc_bn, s);           // warm-up (and first-launch set-up)
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) launch_tc_gemm(rep.tc, rep.tc_bn, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(PEPS_ERR_CUDA, "tuning launch failed"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = c; }
    }
    if (st != PEPS_OK) break;
    for (size_t i : g.second)
      if (plan->ops[i].tc_bn != best && !tc_retile(plan->ops[i], best)) {
        st = fail(PEPS_ERR_UNSUPPORTED, "MMA width %d not encodable", best);
        break;
      }
    if (st != PEPS_OK) break;
    plan->tune[g.first] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == PEPS_OK) CUDA_TRY(cudaGetLastError());
  return st;
}

peps_status peps_plan_tune_table(const peps_plan *plan, char *buf, size_t cap, size_t *len) {
  if (!plan || !len) return fail(PEPS_ERR_ARG, "NULL argument");
  std::string t;
  for (auto &kv : plan->tune) t += kv.first + " = " + std::to_string(kv.second) + "\n";
  *len = t.size() + 1;
  if (buf && cap) {
    const size_t n = std::min(cap - 1, t.size());
    memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return PEPS_OK;
}

peps_status peps_plan_set_tune_table(peps_plan *plan, const char *table) {
  g_last_error.clear();
  if (!plan || !table) return fail(PEPS_ERR_ARG, "NULL argument");
  std::map<std::string, int> t;
  const char *p = table;
  while (*p) {
    const char *e = strchr(p, '\n');
    std::string line(p, e ? (size_t)(e - p) : strlen(p));
    p = e ? e + 1 : p + line.size();
    if (line.empty()) continue;
    const size_t eq = line.rfind(" = ");
    int w = 0;
    if (eq == std::string::npos || sscanf(line.c_str() + eq + 3, "%d", &w) != 1 ||
        (w != 64 && w != 128 && w != 192 && w != 256))
      return fail(PEPS_ERR_ARG, "bad tuning line \"%s\"", line.c_str());
    t[line.substr(0, eq)] = w;
  }
  plan->tune = t;
  plan->built = false;        // the next execute rebuilds with the table
  return PEPS_OK;
}

peps_status peps_plan_set_wait_limit(peps_plan *plan, uint64_t ns) {
  g_last_error.clear();
  if (!plan) return fail(PEPS_ERR_ARG, "plan is NULL");
  plan->wait_ns = ns;
  for (Op &op : plan->ops)
    if (op.kind == Op::TC) op.tc.wait_ns = ns;
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
  uint32_t word = 0;
  CUDA_TRY(cudaMemcpyAsync(res, (uint8_t *)workspace + plan->result_off, 16, cudaMemcpyDeviceToHost, s));
  if (sigma_out && plan->nsigma > 0)
    CUDA_TRY(cudaMemcpyAsync(sigma_out, (uint8_t *)workspace + plan->sigma_off, plan->nsigma * 8,
                             cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&word, (uint8_t *)workspace + plan->status_off, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (log_abs) *log_abs = res[0];
  if (phase) *phase = res[1];
  if (peps_status st = status_of(word)) return st;
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

peps_status peps_expectation_plan(peps_plan **out, const peps_network *ket, const peps_term *terms,
                                  int32_t nterms, const peps_rsvd_opts *opts, int32_t use_cache,
                                  size_t *workspace_bytes) {
  g_last_error.clear();
  if (!out || !workspace_bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (nterms < 0 || (nterms > 0 && !terms)) return fail(PEPS_ERR_ARG, "terms missing");
  if (peps_status s = check_opts(opts)) return s;
  if (opts->flags & PEPS_FLAG_UNIT_BOND)
    return fail(PEPS_ERR_UNSUPPORTED, "PEPS_FLAG_UNIT_BOND applies to TEBD plans only");
  std::unique_ptr<peps_plan> P(new (std::nothrow) peps_plan());
  if (!P) return fail(PEPS_ERR_ARG, "out of host memory");
  P->kind = peps_plan::EXPECT;
  P->opts = to_opts(opts);
  if (P->opts.alternate)
    return fail(PEPS_ERR_UNSUPPORTED, "alternating canonicalisation applies to contraction plans only");
  P->use_cache = use_cache != 0;
  if (peps_status s = read_net(ket, P->ket, "ket")) return s;
  P->dt = P->ket.dt;
  const Net &H = P->ket;
  const int d = H.d, vals = dtype_complex(P->dt) ? 2 : 1;
  for (int t = 0; t < nterms; ++t) {
    const peps_term &T = terms[t];
    if (T.nsite != 1 && T.nsite != 2) return fail(PEPS_ERR_ARG, "term %d: nsite must be 1 or 2", t);
    if (!T.op) return fail(PEPS_ERR_ARG, "term %d: operator is NULL", t);
    const int nsites = H.nrow * H.ncol;
    for (int k = 0; k < T.nsite; ++k)
      if (T.site[k] < 0 || T.site[k] >= nsites) return fail(PEPS_ERR_ARG, "term %d: site out of range", t);
    if (T.nsite == 2) {
      const int r0 = T.site[0] / H.ncol, c0 = T.site[0] % H.ncol;
      const int r1 = T.site[1] / H.ncol, c1 = T.site[1] % H.ncol;
      if (!((r1 == r0 && c1 == c0 + 1) || (c1 == c0 && r1 == r0 + 1)))
        return fail(PEPS_ERR_UNSUPPORTED, "term %d: only nearest-neighbour bonds, left-to-right or top-down", t);
    }
    peps_plan::Term X;
    X.nsite = T.nsite;
    X.site[0] = T.site[0];
    X.site[1] = T.nsite == 2 ? T.site[1] : -1;
    const int64_t n = T.nsite == 1 ? d : (int64_t)d * d;
    X.op.assign(T.op, T.op + n * n * vals);
    X.coeff = T.coeff;
    P->terms.push_back(X);
  }
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_expectation_execute(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream) {
  g_last_error.clear();
  if (!plan) return fail(PEPS_ERR_ARG, "plan is NULL");
  if (plan->kind != peps_plan::EXPECT) return fail(PEPS_ERR_ARG, "not an expectation plan");
  const bool same = plan->built && plan->built_base == (uintptr_t)workspace;
  if (!same) {
    if (peps_status s = rebuild(plan, workspace, nullptr, true)) return s;
    plan->built_base = (uintptr_t)workspace;
    plan->built = true;
  }
  if (!plan->splittable) return enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, !same);
  // the sweeps (on their branches, joined at the end of the first call), then the strips
  const size_t strips = plan->part_ops[2][0].first;
  if (peps_status s = enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, !same, nullptr, 0, strips))
    return s;
  return enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, false, nullptr, strips);
}

peps_status peps_expectation_env_region(const peps_plan *plan, int32_t part, size_t *offset, size_t *bytes) {
  g_last_error.clear();
  if (!plan || !offset || !bytes) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EXPECT) return fail(PEPS_ERR_ARG, "not an expectation plan");
  if (!plan->splittable) return fail(PEPS_ERR_UNSUPPORTED, "the split applies to the cached schedule only");
  if (part != 0 && part != 1) return fail(PEPS_ERR_ARG, "part %d: 0 (top-down) or 1 (bottom-up)", (int)part);
  *offset = plan->env_lo[part];
  *bytes = plan->env_hi[part] - plan->env_lo[part];
  return PEPS_OK;
}

peps_status peps_expectation_execute_part(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream,
                                          int32_t part) {
  g_last_error.clear();
  if (!plan) return fail(PEPS_ERR_ARG, "plan is NULL");
  if (plan->kind != peps_plan::EXPECT) return fail(PEPS_ERR_ARG, "not an expectation plan");
  if (!plan->splittable) return fail(PEPS_ERR_UNSUPPORTED, "the split applies to the cached schedule only");
  if (part < 0 || part > 2) return fail(PEPS_ERR_ARG, "part %d: 0, 1 or 2", (int)part);
  const bool same = plan->built && plan->built_base == (uintptr_t)workspace;
  if (!same) {
    if (peps_status s = rebuild(plan, workspace, nullptr, true)) return s;
    plan->built_base = (uintptr_t)workspace;
    plan->built = true;
  }
  bool upload = !same;
  for (const auto &r : plan->part_ops[part]) {
    if (peps_status s = enqueue(plan, workspace, workspace_bytes, (cudaStream_t)stream, upload, nullptr, r.first,
                                r.second))
      return s;
    upload = false;
  }
  return PEPS_OK;
}

peps_status peps_expectation_result(peps_plan *plan, void *workspace, void *stream, double *energy,
                                    double *log_norm, double *term_values) {
  g_last_error.clear();
  if (!plan || !workspace) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::EXPECT) return fail(PEPS_ERR_ARG, "not an expectation plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "result read during stream capture");
  const bool cplx = dtype_complex(plan->dt);
  const int vals = cplx ? 2 : 1;
  std::vector<double> sv((size_t)plan->nstrips * vals);
  std::vector<double> lg((size_t)std::max<int64_t>(plan->lognorm_nlogs, 1));
  CUDA_TRY(cudaMemcpyAsync(sv.data(), (uint8_t *)workspace + plan->strip_off, sv.size() * 8, cudaMemcpyDeviceToHost,
                           s));
  if (plan->lognorm_nlogs > 0)
    CUDA_TRY(cudaMemcpyAsync(lg.data(), (uint8_t *)workspace + plan->lognorm_logs_off,
                             (size_t)plan->lognorm_nlogs * 8, cudaMemcpyDeviceToHost, s));
  uint32_t word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, (uint8_t *)workspace + plan->status_off, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (peps_status st = status_of(word)) return st;
  auto re_ = [&](int64_t i) { return sv[(size_t)i * vals]; };
  auto im_ = [&](int64_t i) { return cplx ? sv[(size_t)i * vals + 1] : 0.0; };
  double e = 0.0;
  for (size_t t = 0; t < plan->terms.size(); ++t) {
    double num_re = 0.0, num_im = 0.0;
    int64_t nrm = -1;
    for (auto &pr : plan->term_strips[t]) {
      num_re += re_(pr.first);
      num_im += im_(pr.first);
      nrm = pr.second;
    }
    double v = 0.0;
    if (nrm >= 0) {
      const double dr = re_(nrm), di = im_(nrm), den = dr * dr + di * di;
      if (!(den > 0.0)) return fail(PEPS_ERR_NUMERIC, "term %zu: vanishing strip norm", t);
      v = (num_re * dr + num_im * di) / den;       // Re(num / norm)
    }
    v *= plan->terms[t].coeff;
    if (term_values) term_values[t] = v;
    e += v;
  }
  if (energy) *energy = e;
  if (log_norm) {
    const double dr = re_(plan->lognorm_strip), di = im_(plan->lognorm_strip);
    double l = 0.5 * std::log(dr * dr + di * di);
    for (int64_t i = 0; i < plan->lognorm_nlogs; ++i) l += lg[(size_t)i];
    *log_norm = l;
  }
  if (!std::isfinite(e)) return fail(PEPS_ERR_NUMERIC, "non-finite expectation value");
  return PEPS_OK;
}

peps_status peps_grad_plan(peps_plan **out, const peps_network *ket, const peps_term *terms, int32_t nterms,
                           const peps_rsvd_opts *opts, size_t *workspace_bytes) {
  g_last_error.clear();
  if (!ket) return fail(PEPS_ERR_ARG, "NULL argument");
  if (ket->dtype != PEPS_R32 && ket->dtype != PEPS_R64)
    return fail(PEPS_ERR_UNSUPPORTED, "the energy gradient takes real networks");
  if (!opts) return fail(PEPS_ERR_ARG, "opts is NULL");
  if (opts->prec != PEPS_PREC_PLAIN) return fail(PEPS_ERR_UNSUPPORTED, "the energy gradient runs the plain arithmetic");
  if (ket->nrow < 2 || ket->ncol < 2) return fail(PEPS_ERR_UNSUPPORTED, "the energy gradient needs 2 rows and 2 columns");
  peps_plan *p = nullptr;
  if (peps_status s = peps_expectation_plan(&p, ket, terms, nterms, opts, 1, workspace_bytes)) return s;
  std::unique_ptr<peps_plan> P(p);
  P->kind = peps_plan::GRAD;
  if (peps_status s = rebuild(P.get(), nullptr, nullptr)) return s;
  *workspace_bytes = P->ws_bytes;
  *out = P.release();
  return PEPS_OK;
}

peps_status peps_grad_execute(peps_plan *plan, void *const *grad_site, void *workspace, size_t workspace_bytes,
                              void *stream, double *energy) {
  g_last_error.clear();
  if (!plan || !grad_site) return fail(PEPS_ERR_ARG, "NULL argument");
  if (plan->kind != peps_plan::GRAD) return fail(PEPS_ERR_ARG, "not a gradient plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (in_capture(s)) return fail(PEPS_ERR_CAPTURE, "the gradient reads the strips back mid-way: no capture");
  const size_t ns = (size_t)plan->ket.nrow * plan->ket.ncol;
  for (size_t i = 0; i < ns; ++i)
    if (!grad_site[i]) return fail(PEPS_ERR_ARG, "gradient tensor %zu is NULL", i);
  bool same = plan->built && plan->built_base == (uintptr_t)workspace && plan->grad_site.size() == ns &&
              std::equal(plan->grad_site.begin(), plan->grad_site.end(), grad_site);
  if (!same) {
    plan->grad_site.assign(grad_site, grad_site + ns);
    if (peps_status st = rebuild(plan, workspace, nullptr, true)) return st;
    plan->built_base = (uintptr_t)workspace;
    plan->built = true;
  }
  // phase 1: forward (sweeps keeping every step, strips)
  if (peps_status st = enqueue(plan, workspace, workspace_bytes, s, !same, nullptr, 0, plan->split)) return st;
  // strip cotangents of E = sum_t c_t sum_x s_{t,x} / s_norm(t) on the host
  std::vector<double> sv((size_t)plan->nstrips), sb((size_t)plan->nstrips, 0.0);
  CUDA_TRY(cudaMemcpyAsync(sv.data(), (uint8_t *)workspace + plan->strip_off, sv.size() * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double e = 0.0;
  for (size_t t = 0; t < plan->terms.size(); ++t) {
    double num = 0.0;
    int64_t nrm = -1;
    for (auto &pr : plan->term_strips[t]) { num += sv[(size_t)pr.first]; nrm = pr.second; }
    if (nrm < 0) continue;
    const double den = sv[(size_t)nrm], c = plan->terms[t].coeff;
    if (!(den != 0.0)) return fail(PEPS_ERR_NUMERIC, "term %zu: vanishing strip norm", t);
    e += c * num / den;
    for (auto &pr : plan->term_strips[t]) sb[(size_t)pr.first] += c / den;
    sb[(size_t)nrm] -= c * num / (den * den);
  }
  if (energy) *energy = e;
  CUDA_TRY(cudaMemcpyAsync((uint8_t *)workspace + plan->sbar_off, sb.data(), sb.size() * 8, cudaMemcpyHostToDevice, s));
  // phase 2: reverse sweep into the site cotangents; synchronise (sb is host memory)
  if (peps_status st = enqueue(plan, workspace, workspace_bytes, s, false, nullptr, plan->split)) return st;
  uint32_t word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, (uint8_t *)workspace + plan->status_off, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (peps_status st = status_of(word)) return st;
  if (!std::isfinite(e)) return fail(PEPS_ERR_NUMERIC, "non-finite energy");
  return PEPS_OK;
}

peps_status peps_grad(const peps_network *ket, const peps_term *terms, int32_t nterms, const peps_rsvd_opts *opts,
                      void *const *grad_site, void *workspace, size_t workspace_bytes, void *stream, double *energy) {
  peps_plan *p = nullptr;
  size_t need = 0;
  peps_status s = peps_grad_plan(&p, ket, terms, nterms, opts, &need);
  if (s != PEPS_OK) return s;
  s = peps_grad_execute(p, grad_site, workspace, workspace_bytes, stream, energy);
  peps_plan_destroy(p);
  return s;
}

peps_status peps_expectation_workspace(const peps_network *ket, const peps_term *terms, int32_t nterms,
                                       const peps_rsvd_opts *opts, int32_t use_cache, size_t *workspace_bytes) {
  peps_plan *p = nullptr;
  peps_status s = peps_expectation_plan(&p, ket, terms, nterms, opts, use_cache, workspace_bytes);
  if (s == PEPS_OK) peps_plan_destroy(p);
  return s;
}

peps_status peps_expectation(const peps_network *ket, const peps_term *terms, int32_t nterms,
                             const peps_rsvd_opts *opts, int32_t use_cache, void *workspace, size_t workspace_bytes,
                             void *stream, double *energy, double *log_norm) {
  peps_plan *p = nullptr;
  size_t need = 0;
  peps_status s = peps_expectation_plan(&p, ket, terms, nterms, opts, use_cache, &need);
  if (s != PEPS_OK) return s;
  s = peps_expectation_execute(p, workspace, workspace_bytes, stream);
  if (s == PEPS_OK) s = peps_expectation_result(p, workspace, stream, energy, log_norm, nullptr);
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

peps_status peps_plan_kernel_launches(const peps_plan *plan, int64_t *count) {
  if (!plan || !count) return fail(PEPS_ERR_ARG, "NULL argument");
  int64_t n = 0;
  for (const Op &op : plan->ops) {
    switch (op.kind) {
      case Op::JACOBI: n += 1 + (op.smem2 > 0) + (op.smem3 > 0) + (op.blocks > 0); break;   // one CTA, clusters, refinement
      case Op::CHOL: n += 1 + (op.smem2 > 0); break;                         // one CTA, cluster
      case Op::FINALIZE: n += 1 + (op.blocks > 0); break;                    // gauge projections, finalize
      case Op::TC: n += (op.tc.tiles_m * op.tc.tiles_n > 0) + (op.tc.bpre != 0); break;   // B expansion, GEMM
      case Op::COPY: case Op::MEMSET: case Op::BLOBCOPY: break;             // copies, not kernels
      case Op::SKETCH: case Op::GEMM: case Op::GEMM_ATOMIC: case Op::SANDWICH: case Op::ZERO: case Op::SITE:
      case Op::PERMUTE: case Op::PAD: n += op.blocks > 0; break;
      default: n += 1; break;
    }
  }
  *count = n;
  return PEPS_OK;
}

peps_status peps_plan_launch_kernel(const peps_plan *plan, int64_t i, const char **kernel) {
  if (!plan || !kernel) return fail(PEPS_ERR_ARG, "NULL argument");
  if (i < 0 || i >= (int64_t)plan->ops.size()) return fail(PEPS_ERR_ARG, "launch index out of range");
  switch (plan->ops[i].kind) {
    case Op::SKETCH: *kernel = "sketch"; break;
    case Op::GEMM: *kernel = "gemm"; break;
    case Op::GEMM_ATOMIC: *kernel = "gemm_gram"; break;
    case Op::SANDWICH: *kernel = "sandwich"; break;
    case Op::CHOL: *kernel = "chol"; break;
    case Op::JACOBI: *kernel = "jacobi"; break;
    case Op::FINALIZE: *kernel = "finalize"; break;
    case Op::ZERO: *kernel = "zero"; break;
    case Op::SITE: *kernel = "site"; break;
    case Op::SCALAR: *kernel = "scalar"; break;
    case Op::FILL: *kernel = "fill"; break;
    case Op::TC: *kernel = "tc_gemm"; break;
    case Op::PERMUTE: *kernel = "permute"; break;
    case Op::PAD: *kernel = "pad"; break;
    case Op::NARROW: *kernel = "narrow"; break;
    case Op::ABSORB: *kernel = "absorb"; break;
    case Op::THETA: *kernel = "theta"; break;
    case Op::SITEOP: *kernel = "site_op"; break;
    case Op::SVDSMALL: *kernel = "svd_small"; break;
    case Op::SITEGAUGE: *kernel = "site_gauge"; break;
    case Op::BLOBCOPY: *kernel = "copy"; break;
    case Op::STRIP: *kernel = "strip"; break;
    case Op::COPY: *kernel = "copy"; break;
    case Op::SVDBWD: *kernel = "svd_bwd"; break;
    case Op::LTU: *kernel = "copyltu"; break;
    case Op::TGRAD: *kernel = "tensor_grad"; break;
    case Op::MEMSET: *kernel = "memset"; break;
    case Op::AXPY: *kernel = "axpy"; break;
    case Op::SITEBWD: *kernel = "site_reverse"; break;
    case Op::STRIPBWD: *kernel = "strip_reverse"; break;
    default: *kernel = "unknown"; break;
  }
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
  if ((plan->kind == peps_plan::EINSUMSVD || plan->kind == peps_plan::EGRAD) && !io)
    return fail(PEPS_ERR_ARG, "einsumsvd plans need io");
  const bool with_io = plan->kind == peps_plan::EINSUMSVD || plan->kind == peps_plan::EGRAD;
  if (peps_status s = rebuild(plan, workspace, with_io ? io : nullptr)) return s;
  plan->built = false;            // force an upload at the next execute
  Checker C;
  const double es = dtype_size(plan->dt);
  if (plan->kind == peps_plan::EGRAD) {
    const Inst &I = plan->insts[0];
    auto add = [&](const void *p, double n) {
      if (p) C.ext.push_back(Extent{(uintptr_t)p, (uintptr_t)p + (uintptr_t)n, "operand"});
    };
    add(plan->ct.U_bar, es * (double)I.M * I.k);
    add(plan->ct.W_bar, es * (double)I.k * I.N);
    add(plan->ct.log_scale_bar, 8);
    add(plan->gr.V_bar, es * I.kL * I.t * I.a * I.h);
    add(plan->gr.S_bar, es * I.a * I.v * I.b);
    add(plan->gr.ket_bar, es * I.d * I.Dl * I.Du * I.Dx * I.De);
    add(plan->gr.bra_bar, es * I.d * I.DL * I.DU * I.DX * I.DE);
  }
  if (plan->kind == peps_plan::EINSUMSVD || plan->kind == peps_plan::EGRAD) {
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

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

std::mutex g_static_mu;
struct StaticSlot {
  CUcontext ctx = nullptr;  // context the address was looked up in
  void *addr = nullptr;
};
StaticSlot g_static_slot[kMaxDevices];

// The driver's cuCtxGetCurrent, fetched through the runtime (no libcuda link).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (CtxGetCurrentFn)p;
  }();
  return fn;
}

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// the device current and cached per device ordinal AND context: a device reset
// (or a primary context torn down and made again) reloads the module, and the
// array may then sit at another address, which the new context's lookup finds.
peps_status static_scratch(void **addr) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PEPS_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return fail(PEPS_ERR_CUDA, "cannot identify the current CUDA context");
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return fail(PEPS_ERR_CUDA, "cuCtxGetCurrent failed");
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticSlot &slot = g_static_slot[dev];
  if (!ctx || slot.ctx != ctx || !slot.addr) {
    void *p = nullptr;
    // with the device current; also makes its primary context current if none was
    CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    if (!p || ((uintptr_t)p & 255)) return fail(PEPS_ERR_CUDA, "static scratch address %p unusable", p);
    if (!ctx && (get(&ctx) != CUDA_SUCCESS || !ctx))
      return fail(PEPS_ERR_CUDA, "no current CUDA context after the symbol lookup");
    slot.ctx = ctx;
    slot.addr = p;
  }
  *addr = slot.addr;
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
  cudaStream_t st = (cudaStream_t)stream;
  // refused here, before the memset, as the plan's first execute would refuse it
  if (in_capture(st)) return fail(PEPS_ERR_CAPTURE, "contraction during stream capture");
  void *ws = nullptr;
  if (peps_status s = static_scratch(&ws)) return s;
  // the array holds the previous call's values: start this one from zeros
  CUDA_TRY(cudaMemsetAsync(ws, 0, need, st));
  if (peps_status s = peps_contract_execute(plan.get(), ws, PEPS_STATIC_SCRATCH_BYTES, stream)) return s;
  return peps_contract_result(plan.get(), ws, stream, log_abs, phase, nullptr);
}

// ---------------------------------------------------------------------------
// Verification entry of the sketch generator (Algorithm 4's first line).
// ---------------------------------------------------------------------------
extern "C" peps_status peps_debug_sketch(int32_t dtype, int64_t N, int32_t ell, uint64_t seed, uint64_t instance,
                                         int32_t tag, int32_t kind, void *X, void *desc_scratch, void *stream) {
  g_last_error.clear();
  if (!X || !desc_scratch) return fail(PEPS_ERR_ARG, "NULL argument");
  if (dtype < PEPS_R32 || dtype > PEPS_C128) return fail(PEPS_ERR_ARG, "bad dtype %d", dtype);
  if (N < 1 || ell < 1) return fail(PEPS_ERR_ARG, "N and ell must be >= 1");
  if (kind != PEPS_SKETCH_GAUSS && kind != PEPS_SKETCH_UNIFORM) return fail(PEPS_ERR_ARG, "bad kind %d", kind);
  if (tag < 0) return fail(PEPS_ERR_ARG, "bad tag %d", tag);
  if (((uintptr_t)desc_scratch & 15) != 0) return fail(PEPS_ERR_ARG, "desc_scratch must be 16-byte aligned");
  const int per = dtype_complex(dtype) ? 2 : 4;
  const int64_t total = N * (int64_t)ell;
  const int64_t blocks = ceil_div(ceil_div(total, per), 256);
  if (blocks > 0x7fffffffll) return fail(PEPS_ERR_UNSUPPORTED, "block too large");
  SketchDesc d{};
  d.X = X; d.N = N; d.ld = N; d.ell = ell; d.tag = tag; d.kind = kind;
  d.seed = seed; d.instance = instance; d.nblocks = blocks; d.nd = 0;
  sketch_set_div(d);
  struct { SketchDesc d; int64_t prefix[2]; } host{d, {0, blocks}};
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(desc_scratch, &host, sizeof host, cudaMemcpyHostToDevice, s));
  uint8_t *dev = (uint8_t *)desc_scratch;
  launch_sketch(dtype, (const SketchDesc *)dev, (const int64_t *)(dev + offsetof(decltype(host), prefix)), 1, blocks, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));   // the host copy of the descriptor dies with this call
  return PEPS_OK;
}
