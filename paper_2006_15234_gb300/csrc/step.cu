// Launch schedule of one einsumsvd (Algorithm 3's einsumsvd line with
// Algorithm 4 applied to the implicit operator of Sec. IV-A), emitted as
// grouped launches over any number of instances:
//
//   X <- Omega (Philox), g <- gauge vector
//   Y <- A X;              P <- orth(Y)            (CholeskyQR2)
//   repeat q:  Z <- A^H P; Q <- orth(Z);  Y <- A Q;  P <- orth(Y)
//   Z <- A^H P  (= (P^H A)^H);  R_B <- R factor of Z (CholeskyQR2)
//   U~, Sigma <- one-sided Jacobi SVD of R_B^H;  sort / truncate / gauge
//   U <- P U~;   W <- U~^H P^H A / sigma_1
//
// A X runs as the two-layer site "sandwich" (ket and bra over their down and
// right bonds) followed by the boundary-site and carry contractions; A^H Y
// is the same chain reversed (Table 2's two-layer IBMPS contraction order).
#include <algorithm>
#include <cmath>

#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "plan.h"

namespace peps {

namespace {

constexpr int kSMs = 152;

int64_t gemm_blocks(GemmDesc &g) {
  g.tiles_m = (int)ceil_div(g.M, kGemmBM);
  g.tiles_n = (int)ceil_div(g.N, kGemmBN);
  return (int64_t)g.batch * g.ksplit * g.tiles_m * g.tiles_n;
}

GemmDesc mk_gemm(int M, int N, int K, int batch, const void *A, int64_t sAm, int64_t sAk, int64_t sAb,
                 bool conjA, const void *B, int64_t sBk, int64_t sBn, int64_t sBb, bool conjB, void *C,
                 int64_t sCm, int64_t sCn, int64_t sCb) {
  GemmDesc g{};
  g.A = A; g.B = B; g.C = C;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.ksplit = 1; g.kchunk = K;
  g.sAm = sAm; g.sAk = sAk; g.sAb = sAb;
  g.sBk = sBk; g.sBn = sBn; g.sBb = sBb;
  g.sCm = sCm; g.sCn = sCn; g.sCb = sCb;
  g.alpha = 1.0; g.alpha_dev = nullptr;
  g.conjA = conjA; g.conjB = conjB; g.conjC = 0; g.accumulate = 0;
  return g;
}

// split K of an atomic Gram so the launch fills the machine a few times over
void set_ksplit(GemmDesc &g, int ndesc) {
  const int64_t tiles = ceil_div(g.M, kGemmBM) * ceil_div(g.N, kGemmBN) * (int64_t)g.batch * ndesc;
  int64_t ks = std::max<int64_t>(1, (4 * kSMs + tiles - 1) / tiles);
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, g.K / 256));
  g.kchunk = (int)(ceil_div(ceil_div(g.K, ks), 16) * 16);
  g.ksplit = (int)ceil_div(g.K, g.kchunk);
}

void push_grouped(Builder &B, Op::Kind kind, const void *descs, size_t desc_size, int nd,
                  const std::vector<int64_t> &blocks, const char *tag, int smem = 0) {
  std::vector<int64_t> prefix(nd);
  int64_t tot = 0;
  for (int i = 0; i < nd; ++i) { prefix[i] = tot; tot += blocks[i]; }
  Op op;
  op.kind = kind;
  op.desc_off = B.put_bytes(descs, desc_size * nd);
  op.prefix_off = B.put(prefix);
  op.nd = nd;
  op.blocks = tot;
  op.smem = smem;
  op.tag = tag;
  if (nd > 0 && tot > 0) B.ops.push_back(op);
}

void push_gemm(Builder &B, std::vector<GemmDesc> &d, bool atomic, const char *tag) {
  std::vector<int64_t> bl(d.size());
  double fl = 0, by = 0;
  const double mult = dtype_complex(B.dt) ? 8.0 : 2.0, es = dtype_size(B.dt);
  for (size_t i = 0; i < d.size(); ++i) {
    bl[i] = gemm_blocks(d[i]);
    const GemmDesc &g = d[i];
    fl += mult * (double)g.M * g.N * g.K * g.batch;
    by += es * ((double)g.M * g.K * (g.sAb ? g.batch : 1) + (double)g.K * g.N * (g.sBb ? g.batch : 1)) +
          (atomic ? acc_size(B.dt) : es) * (double)g.M * g.N * g.batch;
  }
  const size_t before = B.ops.size();
  push_grouped(B, atomic ? Op::GEMM_ATOMIC : Op::GEMM, d.data(), sizeof(GemmDesc), (int)d.size(), bl, tag);
  if (B.ops.size() > before) { B.ops.back().flops = fl; B.ops.back().bytes = by; }
}

void push_zero(Builder &B, const std::vector<std::pair<void *, int64_t>> &regions, const char *tag) {
  std::vector<ZeroDesc> d;
  std::vector<int64_t> bl;
  for (auto &r : regions) {
    d.push_back(ZeroDesc{r.first, r.second});
    bl.push_back(ceil_div(r.second, kZeroWordsPerBlock));
  }
  push_grouped(B, Op::ZERO, d.data(), sizeof(ZeroDesc), (int)d.size(), bl, tag);
}

// ---- stages ---------------------------------------------------------------

void emit_sketch(Builder &B, std::vector<Inst *> &I, const RsvdOpts &o) {
  std::vector<SketchDesc> d;
  std::vector<int64_t> bl;
  const int per = dtype_complex(B.dt) ? 2 : 4;
  for (Inst *p : I) {
    SketchDesc s{};
    s.X = p->X; s.N = p->N; s.ld = p->N; s.ell = p->ell; s.tag = 0; s.kind = o.sketch;
    s.seed = o.seed; s.instance = p->instance;
    s.nblocks = ceil_div(ceil_div(s.N * s.ell, per), 256);
    sketch_set_div(s);
    d.push_back(s); bl.push_back(s.nblocks);
    SketchDesc gg = s;
    gg.X = p->g; gg.N = p->M; gg.ld = p->M; gg.ell = 1; gg.tag = 1; gg.kind = 0;
    gg.nblocks = ceil_div(ceil_div(gg.N, per), 256);
    sketch_set_div(gg);
    d.push_back(gg); bl.push_back(gg.nblocks);
  }
  push_grouped(B, Op::SKETCH, d.data(), sizeof(SketchDesc), (int)d.size(), bl, "sketch");
  double by = 0;
  for (auto &s : d) by += (double)dtype_size(B.dt) * s.N * s.ell;
  B.ops.back().bytes = by;
}

SandwichDesc mk_sandwich(const Inst &I, const void *in, void *out, bool adjoint) {
  SandwichDesc s{};
  s.in = in; s.out = out; s.K = I.K; s.Kb = I.Kb;
  s.d = I.d; s.Dl = I.Dl; s.Du = I.Du; s.Dx = I.Dx; s.De = I.De;
  s.DL = I.DL; s.DU = I.DU; s.DX = I.DX; s.DE = I.DE;
  s.B = I.b; s.ell = I.ell; s.adjoint = adjoint;
  const int64_t ldT2 = (int64_t)I.h * I.v * I.b;
  s.ld_in = adjoint ? ldT2 : I.N;
  s.ld_out = adjoint ? I.N : ldT2;
  return s;
}

void push_sandwich(Builder &B, std::vector<SandwichDesc> &d, const char *tag) {
  int64_t items = 0;
  int smem = 0;
  for (auto &s : d) {
    items += (int64_t)s.ell * s.B;
    smem = std::max(smem, sandwich_smem_bytes(B.dt, s));
  }
  const int64_t per = std::max<int64_t>(1, std::min<int64_t>(32, items / (4 * kSMs)));
  std::vector<int64_t> bl;
  for (auto &s : d) {
    s.items_per_block = (int)per;
    s.nblocks = (int)ceil_div((int64_t)s.ell * s.B, per);
    bl.push_back(s.nblocks);
  }
  double fl = 0, by = 0;
  const double mult = dtype_complex(B.dt) ? 8.0 : 2.0, es = dtype_size(B.dt);
  for (auto &s : d) {
    const double P1 = s.Dl * s.Du, Q1 = s.Dx * s.De, P2 = s.DL * s.DU, Q2 = s.DX * s.DE;
    const double items_s = (double)s.ell * s.B;
    fl += mult * items_s * s.d * (s.adjoint ? (P1 * P2 * Q2 + Q1 * P1 * Q2) : (P1 * Q1 * Q2 + P1 * Q2 * P2));
    by += es * items_s * (P1 * P2 + Q1 * Q2);
  }
  const size_t before = B.ops.size();
  push_grouped(B, Op::SANDWICH, d.data(), sizeof(SandwichDesc), (int)d.size(), bl, tag, smem);
  if (B.ops.size() > before) { B.ops.back().flops = fl; B.ops.back().bytes = by; }
}

// Y <- A X (src N-side [j][n] -> dst M-side [j][mrow])
void emit_product(Builder &B, std::vector<Inst *> &I, bool from_x) {
  std::vector<SandwichDesc> sw;
  std::vector<GemmDesc> g3, g4;
  for (Inst *p : I) {
    const Inst &q = *p;
    sw.push_back(mk_sandwich(q, from_x ? q.X : q.Z, q.T2, false));
    const int64_t vb = (int64_t)q.v * q.b, hvb = (int64_t)q.h * vb, ah = (int64_t)q.a * q.h;
    // T3_j[a][h] = sum_(v,b) S[a][(v,b)] T2_j[h][(v,b)]
    g3.push_back(mk_gemm(q.a, q.h, (int)vb, q.ell, q.S, vb, 1, 0, false, q.T2, 1, vb, hvb, false, q.T3,
                         q.h, 1, ah));
    // Y[j][mrow] = sum_(a,h) T3[j][(a,h)] V[mrow][(a,h)]
    g4.push_back(mk_gemm(q.ell, (int)q.M, (int)ah, 1, q.T3, ah, 1, 0, false, q.V, 1, ah, 0, false, q.Y,
                         q.M, 1, 0));
  }
  push_sandwich(B, sw, "product_sites");
  push_gemm(B, g3, false, "product_boundary");
  push_gemm(B, g4, false, "product_carry");
}

// Z <- A^H Y (the chain reversed)
void emit_adjoint(Builder &B, std::vector<Inst *> &I) {
  std::vector<SandwichDesc> sw;
  std::vector<GemmDesc> g4, g3;
  for (Inst *p : I) {
    const Inst &q = *p;
    const int64_t vb = (int64_t)q.v * q.b, hvb = (int64_t)q.h * vb, ah = (int64_t)q.a * q.h;
    // Z3[j][(a,h)] = sum_mrow P[j][mrow] conj(V[mrow][(a,h)])
    g4.push_back(mk_gemm(q.ell, (int)ah, (int)q.M, 1, q.Y, q.M, 1, 0, false, q.V, ah, 1, 0, true, q.T3,
                         ah, 1, 0));
    // Z2_j[h][(v,b)] = sum_a Z3_j[a][h] conj(S[a][(v,b)])
    g3.push_back(mk_gemm(q.h, (int)vb, q.a, q.ell, q.T3, 1, q.h, ah, false, q.S, vb, 1, 0, true, q.T2,
                         vb, 1, hvb));
    sw.push_back(mk_sandwich(q, q.T2, q.Z, true));
  }
  push_gemm(B, g4, false, "adjoint_carry");
  push_gemm(B, g3, false, "adjoint_boundary");
  push_sandwich(B, sw, "adjoint_sites");
}

double chol_tol(int dt, int ell) {
  // Gram pivots below tol * max diag are numerically zero directions.  With
  // FP64 data the Gram is accurate to ~eps64; with single-precision data only
  // a breakdown (non-positive pivot) is treated as a zero direction.
  return dtype_double(dt) ? 64.0 * ell * 2.220446049250313e-16 : 0.0;
}

double chol_shift(int dt, int ell, bool first_pass) {
  // Shifted CholeskyQR: a single-precision factorisation of an
  // ill-conditioned block gets a diagonal shift of a few n*eps so it cannot
  // break down; the next pass restores orthogonality.  FP64 data: no shift.
  if (dtype_double(dt) || !first_pass) return 0.0;
  return 4.0 * ell * 5.9604644775390625e-08;
}

void emit_gram_tc(Builder &B, Inst &q, const void *src, int64_t L, const char *tag);
void emit_tc(Builder &B, const char *tag, const void *A, int64_t rowsA, const void *Bm, int64_t rowsB, int64_t K,
             bool conjA, bool conjB, bool split3, void *C, DigitMap mm, DigitMap mn, bool conjC,
             const double *alpha_dev, bool bpre);
void emit_permute(Builder &B, const char *tag, std::vector<PermuteDesc> d);
PermuteDesc mk_perm(const void *in, void *out, int64_t nb, int64_t R, int64_t C, int64_t Q, bool conj);
DigitMap mkmap(std::initializer_list<std::pair<int64_t, int64_t>> l);
constexpr int64_t BIG = 0x7fffffff;          // radix of an index map's last digit

// CholeskyQR pass: G <- src^H src; T <- R^+; dst <- src T.  tc_gram: the Gram
// of a single tensor-core instance runs on the tensor cores (3xTF32, FP64
// accumulation across K chunks), and so does the M-side apply (src and T
// transposed into free scratch first: the sketch block X, which the M-side
// orthogonalisation never reads, and the Jacobi matrix).
// wide (single-precision data): the Cholesky runs in FP64 on the FP64 Gram,
// R into the FP64-sized Rdst, T = R^+ in FP64 into R2 and rounded once into
// Tm for the apply (R2 is free during the orthogonalisations).
void emit_cqr_pass(Builder &B, std::vector<Inst *> &I, bool mside, void *Inst::*src, void *Inst::*dst,
                   void *Inst::*Rdst, void *Inst::*Rprev, void *Inst::*Rout, bool apply, const char *tag,
                   bool first_pass, bool tc_gram = false, bool wide = false) {
  wide = wide && !dtype_double(B.dt) && !Rprev;
  const int as = acc_size(B.dt);
  std::vector<std::pair<void *, int64_t>> z;
  std::vector<GemmDesc> gram, app;
  std::vector<CholDesc> ch;
  for (Inst *p : I) {
    Inst &q = *p;
    const int64_t L = mside ? q.M : q.N;
    z.push_back({q.G, (int64_t)q.ell * q.ell * as / 8});
    GemmDesc g = mk_gemm(q.ell, q.ell, (int)L, 1, q.*src, L, 1, 0, true, q.*src, 1, L, 0, false, q.G,
                         q.ell, 1, 0);
    gram.push_back(g);
    CholDesc c{};
    c.G = q.G; c.T = q.Tm; c.R = q.*Rdst; c.n = q.ell; c.tol = chol_tol(B.dt, q.ell);
    c.shift = chol_shift(B.dt, q.ell, first_pass);
    c.Rprev = Rprev ? q.*Rprev : nullptr;
    c.Rout = Rout ? q.*Rout : nullptr;
    c.status = B.status;
    if (wide) {
      c.T = q.R2;
      c.Tlow = q.Tm;
    }
    ch.push_back(c);
    if (apply)
      app.push_back(mk_gemm(q.ell, (int)L, q.ell, 1, q.Tm, 1, q.ell, 0, false, q.*src, L, 1, 0, false,
                            q.*dst, L, 1, 0));
  }
  const int64_t Lr = I.empty() ? 0 : (mside ? I[0]->M : I[0]->N);
  if (tc_gram && I.size() == 1 && (Lr * dtype_size(B.dt)) % 16 == 0) {
    emit_gram_tc(B, *I[0], I[0]->*src, Lr, tag);
  } else {
    for (auto &g : gram) set_ksplit(g, (int)gram.size());
    push_zero(B, z, tag);
    push_gemm(B, gram, true, tag);
  }
  Op op;
  op.kind = Op::CHOL;
  op.desc_off = B.put(ch);
  op.nd = (int)ch.size();
  op.tag = tag;
  op.wide = wide;
  const int fdt = wide ? (B.dt | 2) : B.dt;
  const double mult = dtype_complex(B.dt) ? 8.0 : 2.0;
  for (auto &c : ch) {
    op.smem = std::max(op.smem, small_smem_bytes(fdt, c.n));
    op.smem2 = std::max(op.smem2, chol_cluster_smem_bytes(fdt, c.n, c.T != nullptr));
    const double n = c.n;
    // factor n^3/3 MACs (+ n^3/6 for R^+); Gram in, R (and R^+) out
    op.flops += mult * (n * n * n / 3.0 + (c.T ? n * n * n / 6.0 : 0.0));
    op.bytes += n * n * (acc_size(B.dt) + dtype_size(fdt) * (c.T ? 2.0 : 1.0));
  }
  B.ops.push_back(op);
  if (!apply) return;
  // (X holds l x N elements: room for the transposed M x l block when M <= N)
  if (tc_gram && mside && I.size() == 1 && I[0]->M <= I[0]->N && (Lr * dtype_size(B.dt)) % 16 == 0 &&
      ((int64_t)I[0]->ell * dtype_size(B.dt)) % 16 == 0) {
    // dst[i][n] = sum_j T[j][i] src[j][n] as C(n, i) = sum_j srcT[n][j] TT[i][j]
    Inst &q = *I[0];
    emit_permute(B, tag, {mk_perm(q.*src, q.X, 1, q.ell, Lr, 1, false), mk_perm(q.Tm, q.Mw, 1, q.ell, q.ell, 1, false)});
    emit_tc(B, tag, q.X, Lr, q.Mw, q.ell, q.ell, false, false, true, q.*dst, mkmap({{BIG, 1}}), mkmap({{BIG, Lr}}),
            false, nullptr, true);
    return;
  }
  push_gemm(B, app, false, tag);
}

void emit_jacobi_finalize(Builder &B, std::vector<Inst *> &I, bool wide = false);

void emit_orth(Builder &B, std::vector<Inst *> &I, bool mside, bool tc_gram = false, bool wide = false) {
  void *Inst::*a = mside ? &Inst::Y : &Inst::Z;
  void *Inst::*t = mside ? &Inst::P : &Inst::X;
  const char *tag = mside ? "orth_m" : "orth_n";
  emit_cqr_pass(B, I, mside, a, t, &Inst::R1, nullptr, nullptr, true, tag, true, tc_gram, wide);
  emit_cqr_pass(B, I, mside, t, a, &Inst::R1, nullptr, nullptr, true, tag, false, tc_gram, wide);
}

// FP64 Cholesky of the FP64 Gram of Z (no apply): R_B in FP64 into R2 and
// rounded once into Rout.
void emit_rb_wide(Builder &B, std::vector<Inst *> &I, const char *tag) {
  const int wdt = B.dt | 2;
  std::vector<CholDesc> ch;
  for (Inst *p : I) {
    Inst &q = *p;
    CholDesc c{};
    c.G = q.G; c.T = nullptr; c.R = q.R2; c.n = q.ell; c.tol = chol_tol(B.dt, q.ell);
    c.Rlow = q.Rout;
    c.status = B.status;
    ch.push_back(c);
  }
  Op op;
  op.kind = Op::CHOL; op.desc_off = B.put(ch); op.nd = (int)ch.size(); op.tag = tag;
  op.wide = true;
  for (auto &c : ch) {
    op.smem = std::max(op.smem, small_smem_bytes(wdt, c.n));
    op.smem2 = std::max(op.smem2, chol_cluster_smem_bytes(wdt, c.n, false));
  }
  B.ops.push_back(op);
}

void emit_small_svd(Builder &B, std::vector<Inst *> &I, bool wide = false) {
  // R_B: CholeskyQR2 of Z = (P^H A)^H (R_B = R2 R1, R_B^H R_B = B B^H with
  // B = P^H A, so its singular values are those of B).  FP64 data: one
  // Cholesky of the FP64 Gram is already accurate; so is one FP64 Cholesky
  // of the FP64-accumulated Gram for single-precision data (wide).
  if (dtype_double(B.dt)) {
    emit_cqr_pass(B, I, false, &Inst::Z, nullptr, &Inst::Rout, nullptr, nullptr, false, "svd_qr", false);
  } else if (wide) {
    const int as = acc_size(B.dt);
    std::vector<std::pair<void *, int64_t>> z;
    std::vector<GemmDesc> gram;
    for (Inst *p : I) {
      Inst &q = *p;
      z.push_back({q.G, (int64_t)q.ell * q.ell * as / 8});
      gram.push_back(mk_gemm(q.ell, q.ell, (int)q.N, 1, q.Z, q.N, 1, 0, true, q.Z, 1, q.N, 0, false, q.G, q.ell, 1,
                             0));
    }
    for (auto &g : gram) set_ksplit(g, (int)gram.size());
    push_zero(B, z, "svd_qr");
    push_gemm(B, gram, true, "svd_qr");
    emit_rb_wide(B, I, "svd_qr");
    emit_jacobi_finalize(B, I, true);
    return;
  } else {
    emit_cqr_pass(B, I, false, &Inst::Z, &Inst::X, &Inst::R1, nullptr, nullptr, true, "svd_qr", true);
    emit_cqr_pass(B, I, false, &Inst::X, nullptr, &Inst::R2, &Inst::R1, &Inst::Rout, false, "svd_qr", false);
  }
  emit_jacobi_finalize(B, I);
}

// wide (single-precision data whose R_B was factored in FP64 into R2): the
// Jacobi SVD runs in FP64 on R2 (Mw in FP64), its result is rounded once into
// R1 for the finalize.
void emit_jacobi_finalize(Builder &B, std::vector<Inst *> &I, bool wide) {
  wide = wide && !dtype_double(B.dt);
  std::vector<JacobiDesc> jd;
  std::vector<FinalizeDesc> fd;
  for (Inst *p : I) {
    Inst &q = *p;
    JacobiDesc j{};
    j.Rb = wide ? q.R2 : q.Rout; j.Mw = q.Mw; j.sig = q.sig; j.n = q.ell; j.max_sweeps = 30; j.status = B.status;
    jd.push_back(j);
    FinalizeDesc f{};
    f.Mw = wide ? q.R1 : q.Mw; f.sig = q.sig; f.P = q.Y; f.g = q.g; f.Ut = q.Ut; f.sigma_out = q.sigma;
    f.h = q.G;                     // the Gram buffer is free once R_B is factored
    f.log_out = q.logp; f.inv_s1 = q.inv_s1; f.n = q.ell; f.k = q.k; f.M = q.M;
    f.rtol = 16.0 * q.ell * 2.220446049250313e-16; f.status = B.status;
    fd.push_back(f);
  }
  Op oj;
  oj.kind = Op::JACOBI; oj.desc_off = B.put(jd); oj.nd = (int)jd.size(); oj.tag = "svd_jacobi";
  oj.wide = wide;
  const int jdt = wide ? (B.dt | 2) : B.dt;
  for (auto &j : jd) {
    oj.smem = std::max(oj.smem, small_smem_bytes(jdt, j.n));
    oj.smem2 = std::max(oj.smem2, jacobi_block_smem_bytes(jdt, j.n));
    oj.smem3 = std::max(oj.smem3, jacobi_cluster_smem_bytes(jdt, j.n));
    oj.blocks = std::max<int64_t>(oj.blocks, j.n);       // largest n: column blocks of the sigma refinement
  }
  B.ops.push_back(oj);
  if (wide)
    for (Inst *p : I) {
      Op on;
      on.kind = Op::NARROW; on.tag = "svd_jacobi";
      on.aux_ptr = p->Mw; on.fill_ptr = p->R1;
      on.fill_n = (int64_t)p->ell * p->ell * (dtype_complex(B.dt) ? 2 : 1);
      on.bytes = 12.0 * on.fill_n;
      B.ops.push_back(on);
    }
  Op of;
  of.kind = Op::FINALIZE; of.desc_off = B.put(fd); of.nd = (int)fd.size(); of.tag = "svd_finalize";
  for (auto &f : fd) of.blocks = std::max<int64_t>(of.blocks, f.n);
  B.ops.push_back(of);
}

void emit_epilogue(Builder &B, std::vector<Inst *> &I) {
  std::vector<GemmDesc> gu, gw;
  for (Inst *p : I) {
    Inst &q = *p;
    // U[mrow][c] = sum_j P[j][mrow] Ut[j][c]
    gu.push_back(mk_gemm((int)q.M, q.k, q.ell, 1, q.Y, 1, q.M, 0, false, q.Ut, q.k, 1, 0, false, q.U, q.k,
                         1, 0));
    // W[c][n] = sum_j conj(Ut[j][c]) conj(Z[j][n]) / sigma_1
    GemmDesc w = mk_gemm(q.k, (int)q.N, q.ell, 1, q.Ut, 1, q.k, 0, true, q.Z, q.N, 1, 0, true, q.W, q.N, 1, 0);
    w.alpha_dev = q.inv_s1;
    gw.push_back(w);
  }
  push_gemm(B, gu, false, "epilogue_u");
  push_gemm(B, gw, false, "epilogue_w");
}


// ===========================================================================
// Tensor-core path (PEPS_PREC_MIXED).  Every stage of A X and A^H Y is one
// K-contiguous GEMM on tcgen05 through layout maps:
//   N-side block layout XL: [j][b][(X,E)][(x,e)]
//   A X :  S1  T1[(j,l,u,b)][(s,X,E)] = X (.) K          over (x,e)
//          S2  T2[j][(l,L)][(u,U,b)]  = T1 (.) conj(Kb)  over (s,X,E)
//          S3  T3[j][(a,h)]           = T2 (.) S         over (u,U,b)
//          S4  Y[j][mrow]             = V (.) T3         over (a,h)
//   A^H Y: S4' Z3[(j,h)][a]           = conj(V^T) (.) Y  over mrow
//          S3' Z2[(j,b,l,u)][(U,L)]   = Z3 (.) conj(S^T) over a
//          S2' T1[(j,b,X,E)][(s,l,u)] = Z2 (.) Kb^T      over (U,L)
//          S1' Z[(j,b,X,E)][(x,e)]    = T1 (.) conj(K^T) over (s,l,u)
// ===========================================================================

DigitMap mkmap(std::initializer_list<std::pair<int64_t, int64_t>> l) {
  DigitMap m{};
  m.n = 0;
  for (auto &p : l) {
    m.radix[m.n] = (int32_t)std::min<int64_t>(p.first, BIG);
    m.stride[m.n] = p.second;
    ++m.n;
  }
  return m;
}

// bpre: B expanded and split into the plan's B scratch before the GEMM (all
// SPLIT3 products but the Grams, whose B is the whole N x l block)
void emit_tc(Builder &B, const char *tag, const void *A, int64_t rowsA, const void *Bm, int64_t rowsB, int64_t K,
             bool conjA, bool conjB, bool split3, void *C, DigitMap mm, DigitMap mn, bool conjC,
             const double *alpha_dev, bool bpre = true) {
  Op op;
  op.kind = Op::TC;
  op.tag = tag;
  TcDesc &d = op.tc;
  std::memset(&d, 0, sizeof d);
  const bool cplx = dtype_complex(B.dt);
  const int64_t kr = K * (cplx ? 2 : 1);
  const int nmma = tc_pick_nmma((int)rowsB, cplx, split3);
  const int bn = tc_tile_cols(nmma, cplx);
  bpre = bpre && split3;
  if (B.encode) {
    // bpre: B's maps point into the B scratch, encoded once its address is known (tc_finish)
    const bool ok = tc_encode_map(&d.ta, A, rowsA, kr, kr * 4, 128) &&
                    (bpre || tc_encode_map(&d.tb, Bm, rowsB, kr, kr * 4, bn));
    if (!ok && B.err.empty()) B.err = std::string("TMA map encoding failed for ") + tag;
  }
  if (bpre) {
    d.bpre = 1;
    d.Braw = Bm;
    B.bx_need = std::max<size_t>(B.bx_need, (size_t)tc_bx_bytes(rowsB, kr, cplx));
  }
  d.M = (int32_t)rowsA; d.N = (int32_t)rowsB; d.Kr = (int32_t)kr;
  d.cplx = cplx; d.conjA = conjA; d.conjB = conjB; d.split3 = split3;
  d.tiles_m = (int32_t)ceil_div(rowsA, 128);
  d.tiles_n = (int32_t)ceil_div(rowsB, bn);
  d.mm = mm; d.mn = mn;
  d.C = C;
  d.alpha = 1.0;
  d.alpha_dev = alpha_dev;
  d.conjC = conjC;
  d.status = B.status;
  op.tc_bn = nmma;
  op.tcA = A; op.tcB = Bm; op.tcA_rows = rowsA; op.tcB_rows = rowsB; op.tc_kr = kr;
  const double mult = cplx ? 8.0 : 2.0, es = dtype_size(B.dt);
  op.flops = mult * (double)rowsA * rowsB * K;
  op.bytes = es * ((double)rowsA * K + (double)rowsB * K + (double)rowsA * rowsB);
  B.ops.push_back(op);
}

}  // namespace

// The plan's B scratch (after every buffer of the schedule) and the TMA maps
// of the pre-expanded B operands, which point into it.
void tc_finish(Builder &B) {
  if (!B.bx_need) return;
  // one B scratch per branch (chains of different branches may run at once)
  std::vector<size_t> need(B.branches(), 0);
  for (const Op &op : B.ops)
    if (op.kind == Op::TC && op.tc.bpre)
      need[op.branch] = std::max<size_t>(need[op.branch], (size_t)tc_bx_bytes(op.tcB_rows, op.tc_kr, op.tc.cplx != 0));
  std::vector<void *> bxs(need.size(), nullptr);
  for (size_t b = 0; b < need.size(); ++b)
    if (need[b]) bxs[b] = B.buf(need[b]);
  for (Op &op : B.ops) {
    if (op.kind != Op::TC || !op.tc.bpre) continue;
    TcDesc &d = op.tc;
    void *bx = bxs[op.branch];
    d.Bx = bx;
    if (!B.encode) continue;
    const int64_t nr = (int64_t)d.N * (d.cplx ? 2 : 1), pitch = (int64_t)d.Kr * 4;
    const bool ok = tc_encode_map(&d.tb, bx, nr, d.Kr, pitch, op.tc_bn) &&
                    tc_encode_map(&d.tb2, (char *)bx + nr * pitch, nr, d.Kr, pitch, op.tc_bn);
    if (!ok && B.err.empty()) B.err = std::string("TMA map encoding failed for ") + op.tag;
  }
}

std::string tc_signature(const Op &op) {
  const TcDesc &d = op.tc;
  char b[160];
  snprintf(b, sizeof b, "c%d s%d p%d a%d f%d M%lld N%d K%d k%d", d.cplx, d.split3, d.bpre, d.atomic64,
           tc_folds(d.split3 != 0, d.Kr, d.kb_per_split) ? 1 : 0, (long long)op.tcA_rows, d.N, d.Kr,
           d.ksplit > 1 ? d.kb_per_split : 0);
  return b;
}

std::vector<int> tc_candidates(const Op &op) {
  std::vector<int> c{64, 128, 192};
  if (!op.tc.split3) c.push_back(256);
  return c;
}

bool tc_retile(Op &op, int nmma) {
  TcDesc &d = op.tc;
  const bool cplx = d.cplx != 0;
  if (d.split3 && nmma > 192) return false;
  const int bn = tc_tile_cols(nmma, cplx);
  const int64_t pitch = (int64_t)d.Kr * 4;
  if (d.bpre) {
    const int64_t nr = (int64_t)d.N * (cplx ? 2 : 1);
    if (!tc_encode_map(&d.tb, d.Bx, nr, d.Kr, pitch, nmma) ||
        !tc_encode_map(&d.tb2, (char *)d.Bx + nr * pitch, nr, d.Kr, pitch, nmma))
      return false;
  } else if (!tc_encode_map(&d.tb, op.tcB, op.tcB_rows, d.Kr, pitch, bn)) {
    return false;
  }
  op.tc_bn = nmma;
  d.tiles_n = (int32_t)ceil_div(d.N, bn);
  return true;
}

namespace {

// G = src^H src for an l x L block stored [j][n] (any order of n), FP64
// accumulators, split over K.
void emit_gram_tc(Builder &B, Inst &q, const void *src, int64_t L, const char *tag) {
  const int as = acc_size(B.dt);
  std::vector<std::pair<void *, int64_t>> zr{{q.G, (int64_t)q.ell * q.ell * as / 8}};
  push_zero(B, zr, tag);
  emit_tc(B, tag, src, q.ell, src, q.ell, L, true, false, true, q.G, mkmap({{BIG, q.ell}}), mkmap({{BIG, 1}}),
          false, nullptr, false);
  Op &op = B.ops.back();
  const int64_t kr = op.tc_kr;
  const int64_t nkb = ceil_div(kr, 32);
  // K chunks of at most 128 K blocks, and small enough that about two items
  // per SM exist; 8 K blocks at least
  const int64_t tiles = (int64_t)op.tc.tiles_m * op.tc.tiles_n;
  const int64_t want = std::max<int64_t>(1, ceil_div(2 * kSMs, tiles));
  const int64_t chunk_kb = std::max<int64_t>(std::min<int64_t>(8, nkb), std::min<int64_t>(128, ceil_div(nkb, want)));
  op.tc.atomic64 = 1;
  op.tc.kb_per_split = (int32_t)chunk_kb;
  op.tc.ksplit = (int32_t)ceil_div(nkb, chunk_kb);
  op.bytes = dtype_size(B.dt) * (double)q.ell * L + acc_size(B.dt) * (double)q.ell * q.ell;
}

void emit_permute(Builder &B, const char *tag, std::vector<PermuteDesc> d) {
  std::vector<int64_t> bl;
  double by = 0;
  for (auto &p : d) {
    bl.push_back(permute_blocks(p));
    by += 2.0 * dtype_size(B.dt) * p.nb * p.R * p.Cc * p.Q;
  }
  const size_t before = B.ops.size();
  push_grouped(B, Op::PERMUTE, d.data(), sizeof(PermuteDesc), (int)d.size(), bl, tag);
  if (B.ops.size() > before) B.ops.back().bytes = by;
}

PermuteDesc mk_perm(const void *in, void *out, int64_t nb, int64_t R, int64_t C, int64_t Q, bool conj = false) {
  PermuteDesc p{};
  p.in = in; p.out = out; p.nb = nb; p.R = R; p.Cc = C; p.Q = Q; p.conj = conj;
  return p;
}

struct Dims6 {
  int64_t l, b, P1, Q1, P2, Q2, d, h, v, a, M, N;
};
Dims6 dims_of(const Inst &q, int64_t ncols) {
  return Dims6{ncols, q.b, (int64_t)q.Dl * q.Du, (int64_t)q.Dx * q.De, (int64_t)q.DL * q.DU,
               (int64_t)q.DX * q.DE, q.d, q.h, q.v, q.a, q.M, q.N};
}

// per-step operand preparation: K^T, Kb permutes, S^T, V^T
void emit_tc_prep(Builder &B, Inst &q) {
  const Dims6 z = dims_of(q, q.ell);
  // Kb [s][L][U][(X,E)] -> KbT [s][(X,E)][U][L]: swap L and U, then move (X,E) ahead
  emit_permute(B, "tc_prep", {mk_perm(q.K, q.KT, 1, z.d * z.P1, z.Q1, 1),
                              mk_perm(q.Kb, q.KbP, z.d, q.DL, q.DU, z.Q2),
                              mk_perm(q.S, q.ST, 1, z.a, z.v * z.b, 1),
                              mk_perm(q.V, q.VT, 1, z.M, z.a * z.h, 1)});
  emit_permute(B, "tc_prep", {mk_perm(q.KbP, q.KbT, z.d, z.P2, z.Q2, 1)});
  // Kb [s][(L,U)][(X,E)] -> KbP [(L,U)][s][(X,E)] (forward stage S2)
  emit_permute(B, "tc_prep", {mk_perm(q.Kb, q.KbP, 1, z.d, z.P2, z.Q2)});
}

// Algorithmic flops and bytes of the last launch recomputed for the extents a
// padded copy stands in for (the padding is not algorithmic work).
void relabel(Builder &B, int64_t rowsA, int64_t rowsB, int64_t K) {
  Op &op = B.ops.back();
  const double mult = dtype_complex(B.dt) ? 8.0 : 2.0, es = dtype_size(B.dt);
  op.flops = mult * (double)rowsA * rowsB * K;
  op.bytes = es * ((double)rowsA * K + (double)rowsB * K + (double)rowsA * rowsB);
}

void emit_product_tc(Builder &B, Inst &q, const void *src, void *dst, bool split3, const Inst *lg = nullptr) {
  const Dims6 z = dims_of(q, q.ell);
  const Dims6 y = lg ? dims_of(*lg, q.ell) : z;
  // T1 rows (j, l, u, b) with b fastest, columns (s, X, E)
  emit_tc(B, "product_sites", src, z.l * z.b * z.Q2, q.K, z.d * z.P1, z.Q1, false, false, split3, q.T1,
          mkmap({{z.Q2, 1}, {z.b, z.d * z.Q2}, {BIG, z.P1 * z.b * z.d * z.Q2}}),
          mkmap({{z.P1, z.b * z.d * z.Q2}, {BIG, z.Q2}}), false, nullptr);
  if (lg) relabel(B, y.l * y.b * y.Q2, y.d * y.P1, y.Q1);
  emit_tc(B, "product_sites", q.T1, z.l * z.b * z.P1, q.KbP, z.P2, z.d * z.Q2, false, true, split3, q.T2,
          mkmap({{z.b, 1}, {q.Du, (int64_t)q.DU * z.b}, {q.Dl, (int64_t)q.DL * z.v * z.b}, {BIG, z.h * z.v * z.b}}),
          mkmap({{q.DU, z.b}, {BIG, z.v * z.b}}), false, nullptr);
  if (lg) relabel(B, y.l * y.b * y.P1, y.P2, y.d * y.Q2);
  emit_tc(B, "product_boundary", q.T2, z.l * z.h, q.S, z.a, z.v * z.b, false, false, split3, q.T3,
          mkmap({{z.h, 1}, {BIG, z.a * z.h}}), mkmap({{BIG, z.h}}), false, nullptr);
  if (lg) relabel(B, y.l * y.h, y.a, y.v * y.b);
  emit_tc(B, "product_carry", q.V, z.M, q.T3, z.l, z.a * z.h, false, false, split3, dst, mkmap({{BIG, 1}}),
          mkmap({{BIG, z.M}}), false, nullptr);
  if (lg) relabel(B, y.M, y.l, y.a * y.h);
}

// A^H P for ncols columns of P ([j][mrow]); result in the XL layout, or (W
// mode) conjugated, scaled by 1/sigma_1 and written in the carry layout.
void emit_adjoint_tc(Builder &B, Inst &q, const void *Pin, int64_t ncols, void *dst, bool wmode, bool split3,
                     const Inst *lg = nullptr) {
  const Dims6 z = dims_of(q, ncols);
  const Dims6 y = lg ? dims_of(*lg, ncols) : z;
  emit_tc(B, "adjoint_carry", q.VT, z.a * z.h, Pin, z.l, z.M, true, false, split3, q.T3,
          mkmap({{z.h, z.a}, {BIG, 1}}), mkmap({{BIG, z.h * z.a}}), false, nullptr);
  if (lg) relabel(B, y.a * y.h, y.l, y.M);
  // Z2 rows (j, b, l, u) with u fastest, columns (U, L) with L fastest;
  // computed as Z3 (.) conj(S^T) so that lanes write along L
  emit_tc(B, "adjoint_boundary", q.T3, z.l * z.h, q.ST, z.v * z.b, z.a, false, true, split3, q.T2,
          mkmap({{q.DL, 1}, {q.Dl, (int64_t)q.Du * z.P2}, {BIG, z.b * z.P1 * z.P2}}),
          mkmap({{z.b, z.P1 * z.P2}, {q.DU, q.DL}, {BIG, z.P2}}), false, nullptr);
  if (lg) relabel(B, y.l * y.h, y.v * y.b, y.a);
  emit_tc(B, "adjoint_sites", q.T2, z.l * z.b * z.P1, q.KbT, z.d * z.Q2, z.P2, false, false, split3, q.T1,
          mkmap({{q.Du, 1}, {q.Dl, q.Du}, {z.b, z.Q2 * z.d * z.P1}, {BIG, z.b * z.Q2 * z.d * z.P1}}),
          mkmap({{z.Q2, z.d * z.P1}, {BIG, z.P1}}), false, nullptr);
  if (lg) relabel(B, y.l * y.b * y.P1, y.d * y.Q2, y.P2);
  if (!wmode)
    emit_tc(B, "adjoint_sites", q.T1, z.l * z.b * z.Q2, q.KT, z.Q1, z.d * z.P1, false, true, split3, dst,
            mkmap({{BIG, z.Q1}}), mkmap({{BIG, 1}}), false, nullptr);
  else
    emit_tc(B, "epilogue_w", q.T1, z.l * z.b * z.Q2, q.KT, z.Q1, z.d * z.P1, false, true, split3, dst,
            mkmap({{q.DE, 1}, {q.DX, z.b * q.De * q.DE}, {z.b, (int64_t)q.De * q.DE}, {BIG, z.N}}),
            mkmap({{q.De, q.DE}, {BIG, (int64_t)q.DX * z.b * q.De * q.DE}}), true, q.inv_s1);
  if (lg) relabel(B, y.l * y.b * y.Q2, y.Q1, y.d * y.P1);
}

// Sketch in the XL layout: logical n = (x, X, b, e, E), least significant E.
void emit_sketch_xl(Builder &B, Inst &q, const RsvdOpts &o) {
  std::vector<Inst *> one{&q};
  const size_t before = B.ops.size();
  emit_sketch(B, one, o);
  if (B.ops.size() == before) return;
  SketchDesc *d = (SketchDesc *)(B.blob.data() + B.ops.back().desc_off);
  const int64_t Q1 = (int64_t)q.Dx * q.De;
  d[0].nd = 5;
  const int64_t rad[5] = {q.DE, q.De, q.b, q.DX, BIG};
  const int64_t str[5] = {Q1, 1, (int64_t)q.DX * q.DE * Q1, (int64_t)q.DE * Q1, q.De};
  for (int i = 0; i < 5; ++i) { d[0].radix[i] = (int32_t)rad[i]; d[0].stride[i] = str[i]; }
  sketch_set_div(d[0]);
}

// Sketch and gauge vector of the padded copy E drawn at the caller instance
// I's element numbering: element e = j N + n of I's stream (n = (x, X, b, e,
// E) in I's extents) lands at its place in E's XL layout, gauge entry (k, t)
// at row k t_E + t; every padded position is zero.
void emit_sketch_embedded(Builder &B, const Inst &I, Inst &E, const RsvdOpts &o) {
  const int es = dtype_size(B.dt);
  push_zero(B, {{E.X, (int64_t)E.ell * E.N * es / 8}, {E.g, E.M * es / 8}}, "sketch");
  const int per = dtype_complex(B.dt) ? 2 : 4;
  SketchDesc s{};
  s.X = E.X; s.N = I.N; s.ld = E.N; s.ell = I.ell; s.tag = 0; s.kind = o.sketch;
  s.seed = o.seed; s.instance = I.instance;
  s.nblocks = ceil_div(ceil_div(s.N * s.ell, per), 256);
  const int64_t Q1 = (int64_t)E.Dx * E.De;
  s.nd = 5;
  const int64_t rad[5] = {I.DE, I.De, I.b, I.DX, BIG};
  const int64_t str[5] = {Q1, 1, (int64_t)E.DX * E.DE * Q1, (int64_t)E.DE * Q1, E.De};
  for (int i = 0; i < 5; ++i) { s.radix[i] = (int32_t)rad[i]; s.stride[i] = str[i]; }
  sketch_set_div(s);
  SketchDesc gg{};
  gg.X = E.g; gg.N = I.M; gg.ld = E.M; gg.ell = 1; gg.tag = 1; gg.kind = 0;
  gg.seed = o.seed; gg.instance = I.instance;
  gg.nblocks = ceil_div(ceil_div(gg.N, per), 256);
  gg.nd = 2;
  gg.radix[0] = I.t; gg.stride[0] = 1;
  gg.radix[1] = (int32_t)BIG; gg.stride[1] = E.t;
  sketch_set_div(gg);
  std::vector<SketchDesc> d{s, gg};
  std::vector<int64_t> bl{s.nblocks, gg.nblocks};
  push_grouped(B, Op::SKETCH, d.data(), sizeof(SketchDesc), 2, bl, "sketch");
  B.ops.back().bytes = (double)es * ((double)s.N * s.ell + gg.N);
}

void emit_einsumsvd_tc(Builder &B, Inst &q, const RsvdOpts &o, const Inst *logical = nullptr) {
  std::vector<Inst *> one{&q};
  emit_tc_prep(B, q);
  if (logical) emit_sketch_embedded(B, *logical, q, o);
  else emit_sketch_xl(B, q, o);
  // 3xTF32 (FP32-level) products throughout; the FAST precision runs the
  // products before the last A Q of the power iteration on plain TF32
  const bool fast = o.prec == 2;
  emit_product_tc(B, q, q.X, q.Y, !fast || o.q == 0, logical);
  emit_orth(B, one, true, true, o.fp64_small);
  for (int it = 0; it < o.q; ++it) {
    const bool last = it == o.q - 1;
    emit_adjoint_tc(B, q, q.Y, q.ell, q.Z, false, !fast, logical);
    if (o.orth_q) emit_orth(B, one, false, false, o.fp64_small);
    emit_product_tc(B, q, q.Z, q.Y, !fast || last, logical);
    emit_orth(B, one, true, true, o.fp64_small);
  }
  emit_adjoint_tc(B, q, q.Y, q.ell, q.Z, false, true, logical);      // Z = A^H P = B^H
  // R_B: Cholesky factor of the Gram Z^H Z (= B B^H, B = P^H A).  3xTF32
  // tensor-core products, FP32 partial sums over chunks of 2048 K values,
  // chunks combined in FP64, so the factor carries Z's own error only (a Gram
  // formed from P^H (A Z) would square the product error into the singular
  // values).
  emit_gram_tc(B, q, q.Z, q.N, "svd_gram");
  {
    // FP64 Cholesky of the FP64 Gram (its backward error then stays far
    // below the Gram's own, so sigma_i carries only O(u sigma_1^2 / sigma_i)
    // from Z; an FP32 factorisation would add O(sqrt(l) u sigma_1^2 / sigma_i)),
    // R_B rounded once to the working precision for the Jacobi SVD.
    const int wdt = B.dt | 2;   // R32 -> R64, C64 -> C128
    std::vector<CholDesc> ch(1);
    ch[0] = CholDesc{};
    ch[0].G = q.G; ch[0].T = nullptr; ch[0].R = q.R2; ch[0].n = q.ell; ch[0].tol = chol_tol(B.dt, q.ell);
    ch[0].Rlow = wdt != B.dt ? q.Rout : nullptr;
    ch[0].status = B.status;
    if (wdt == B.dt) ch[0].R = q.Rout;
    Op op;
    op.kind = Op::CHOL; op.desc_off = B.put(ch); op.nd = 1; op.tag = "svd_gram";
    op.wide = wdt != B.dt;
    op.smem = small_smem_bytes(wdt, q.ell);
    op.smem2 = chol_cluster_smem_bytes(wdt, q.ell, false);
    B.ops.push_back(op);
  }
  emit_jacobi_finalize(B, one, o.fp64_small);
  // U = P U~ and its transpose (input of the W adjoint)
  {
    std::vector<GemmDesc> gu{mk_gemm((int)q.M, q.k, q.ell, 1, q.Y, 1, q.M, 0, false, q.Ut, q.k, 1, 0, false, q.U,
                                     q.k, 1, 0)};
    push_gemm(B, gu, false, "epilogue_u");
    emit_permute(B, "epilogue_u", {mk_perm(q.U, q.UT, 1, q.M, q.k, 1)});
  }
  emit_adjoint_tc(B, q, q.UT, q.k, q.W, true, true, logical);        // W = U^H A / sigma_1
}

}  // namespace

void inst_derive(Inst &I, const RsvdOpts &o) {
  I.h = I.Dl * I.DL;
  I.v = I.Du * I.DU;
  I.M = (int64_t)I.kL * I.t;
  I.N = (int64_t)I.Dx * I.DX * I.b * I.De * I.DE;
  I.k = (int)std::min<int64_t>(o.m, std::min(I.M, I.N));
  I.ell = (int)std::min<int64_t>((int64_t)I.k + o.p, std::min(I.M, I.N));
}

size_t inst_scratch_bytes(const Inst &I, int dt) {
  const size_t es = dtype_size(dt), as = acc_size(dt);
  const size_t l = I.ell;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t s = 0;
  s += 2 * al(l * I.N * es);                              // X, Z
  s += al(l * (size_t)I.h * I.v * I.b * es);              // T2
  s += al(l * (size_t)I.a * I.h * es);                    // T3
  s += 2 * al(l * I.M * es);                              // Y, P
  s += al(I.M * es);                                      // g
  s += al(l * l * es) + al(l * I.k * es);                 // Tm, Ut
  s += 5 * al(l * l * as);                                // G, R1, R2, Rout, Mw
  s += al(l * 8) + al(8);                                 // sig, inv_s1
  if (I.tc) {
    const size_t P1 = (size_t)I.Dl * I.Du, Q1 = (size_t)I.Dx * I.De, P2 = (size_t)I.DL * I.DU,
                 Q2 = (size_t)I.DX * I.DE;
    s += al(l * I.b * I.d * P1 * Q2 * es) + al((size_t)I.M * I.a * I.h * es) + al((size_t)I.a * I.v * I.b * es);
    s += al((size_t)I.k * I.M * es) + al(Q1 * I.d * P1 * es) + 2 * al((size_t)I.d * P2 * Q2 * es);
  }
  return s;
}

void inst_alloc_scratch(Builder &B, Inst &I, int dt) {
  const size_t es = dtype_size(dt), as = acc_size(dt);
  const size_t l = I.ell;
  I.X = B.buf(l * I.N * es);
  I.Z = B.buf(l * I.N * es);
  I.T2 = B.buf(l * (size_t)I.h * I.v * I.b * es);
  I.T3 = B.buf(l * (size_t)I.a * I.h * es);
  I.Y = B.buf(l * I.M * es);
  I.P = B.buf(l * I.M * es);
  I.g = B.buf(I.M * es);
  I.Tm = B.buf(l * l * es);
  I.Ut = B.buf(l * I.k * es);
  I.G = B.buf(l * l * as);
  I.R1 = B.buf(l * l * as);
  I.R2 = B.buf(l * l * as);
  I.Rout = B.buf(l * l * as);
  I.Mw = B.buf(l * l * as);
  I.sig = (double *)B.buf(l * 8);
  I.inv_s1 = (double *)B.buf(8);
  I.T1 = I.VT = I.ST = I.UT = I.KT = I.KbP = I.KbT = nullptr;
  if (I.tc) {
    const size_t P1 = (size_t)I.Dl * I.Du, Q1 = (size_t)I.Dx * I.De, P2 = (size_t)I.DL * I.DU,
                 Q2 = (size_t)I.DX * I.DE;
    I.T1 = B.buf(l * I.b * I.d * P1 * Q2 * es);
    I.VT = B.buf((size_t)I.M * I.a * I.h * es);
    I.ST = B.buf((size_t)I.a * I.v * I.b * es);
    I.UT = B.buf((size_t)I.k * I.M * es);
    I.KT = B.buf(Q1 * I.d * P1 * es);
    I.KbP = B.buf((size_t)I.d * P2 * Q2 * es);
    I.KbT = B.buf((size_t)I.d * P2 * Q2 * es);
  }
}

void inst_share_scratch(Inst &I, const Inst &o) {
  I.X = o.X; I.Z = o.Z; I.T2 = o.T2; I.T3 = o.T3; I.Y = o.Y; I.P = o.P; I.g = o.g; I.Tm = o.Tm;
  I.Ut = o.Ut; I.G = o.G; I.R1 = o.R1; I.R2 = o.R2; I.Rout = o.Rout; I.Mw = o.Mw; I.sig = o.sig;
  I.inv_s1 = o.inv_s1;
  I.T1 = o.T1; I.VT = o.VT; I.ST = o.ST; I.UT = o.UT; I.KT = o.KT; I.KbP = o.KbP; I.KbT = o.KbT;
}

bool inst_tc_ok(const Inst &I, int dt) {
  if (dtype_double(dt)) return false;
  const int64_t align = dtype_complex(dt) ? 2 : 4;    // K multiple: rows 16-byte aligned
  const int64_t P1 = (int64_t)I.Dl * I.Du, Q1 = (int64_t)I.Dx * I.De, P2 = (int64_t)I.DL * I.DU,
                Q2 = (int64_t)I.DX * I.DE;
  const int64_t ks[] = {Q1, (int64_t)I.d * Q2, (int64_t)I.v * I.b, (int64_t)I.a * I.h, I.M, I.a, P2,
                        (int64_t)I.d * P1};
  for (int64_t k : ks)
    if (k % align) return false;
  return true;
}

namespace {
int round_up(int x, int q) { return (x + q - 1) / q * q; }
void push_pad(Builder &B, std::vector<PadDesc> &d, const char *tag) {
  std::vector<int64_t> bl;
  double by = 0;
  for (auto &p : d) {
    bl.push_back(ceil_div(p.total, kPadPerBlock));
    by += 2.0 * dtype_size(B.dt) * p.total;
  }
  const size_t before = B.ops.size();
  push_grouped(B, Op::PAD, d.data(), sizeof(PadDesc), (int)d.size(), bl, tag);
  if (B.ops.size() > before) B.ops.back().bytes = by;
}
PadDesc mk_pad(const void *in, void *out, std::initializer_list<int> dims, std::initializer_list<int> lim,
               std::initializer_list<int64_t> in_stride) {
  PadDesc p{};
  p.in = in; p.out = out; p.nd = (int32_t)dims.size(); p.total = 1;
  int i = 0;
  for (int x : dims) { p.dims[i++] = x; p.total *= x; }
  i = 0;
  for (int x : lim) p.lim[i++] = x;
  i = 0;
  for (int64_t x : in_stride) p.in_stride[i++] = x;
  return p;
}
}  // namespace

bool inst_embed_dims(const Inst &I, int dt, const RsvdOpts &o, Inst &E) {
  if (dtype_double(dt)) return false;
  const int q = dtype_complex(dt) ? 2 : 4;
  E = I;
  E.embed = false;
  E.Dl = round_up(I.Dl, 2); E.Du = round_up(I.Du, 2); E.Dx = round_up(I.Dx, 2); E.De = round_up(I.De, 2);
  E.DL = round_up(I.DL, 2); E.DU = round_up(I.DU, 2); E.DX = round_up(I.DX, 2); E.DE = round_up(I.DE, 2);
  E.t = round_up(I.t, q);
  E.a = round_up(I.a, q);
  inst_derive(E, o);
  E.k = I.k;                      // the caller's rank and sketch width
  E.ell = I.ell;
  E.tc = true;
  return inst_check(E, dt).empty() && inst_tc_ok(E, dt);
}

size_t inst_embed_bytes(const Inst &E, int dt) {
  const size_t es = dtype_size(dt);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return inst_scratch_bytes(E, dt) + al((size_t)E.kL * E.t * E.a * E.h * es) + al((size_t)E.a * E.v * E.b * es) +
         al((size_t)E.d * E.Dl * E.Du * E.Dx * E.De * es) + al((size_t)E.d * E.DL * E.DU * E.DX * E.DE * es) +
         al((size_t)E.M * E.k * es) + al((size_t)E.k * E.N * es);
}

void inst_embed_alloc(Builder &B, Inst &E, int dt) {
  const size_t es = dtype_size(dt);
  inst_alloc_scratch(B, E, dt);
  E.V = B.buf((size_t)E.kL * E.t * E.a * E.h * es);
  E.S = B.buf((size_t)E.a * E.v * E.b * es);
  E.K = B.buf((size_t)E.d * E.Dl * E.Du * E.Dx * E.De * es);
  E.Kb = B.buf((size_t)E.d * E.DL * E.DU * E.DX * E.DE * es);
  E.U = B.buf((size_t)E.M * E.k * es);
  E.W = B.buf((size_t)E.k * E.N * es);
}

void emit_einsumsvd_embedded(Builder &B, Inst &I, Inst &E, const RsvdOpts &o) {
  E.instance = I.instance;
  E.sigma = I.sigma;
  E.logp = I.logp;
  // operands into the padded extents (zeros elsewhere)
  std::vector<PadDesc> in{
      mk_pad(I.V, (void *)E.V, {E.kL, E.t, E.a, E.Dl, E.DL}, {I.kL, I.t, I.a, I.Dl, I.DL},
             {(int64_t)I.t * I.a * I.h, (int64_t)I.a * I.h, I.h, I.DL, 1}),
      mk_pad(I.S, (void *)E.S, {E.a, E.Du, E.DU, E.b}, {I.a, I.Du, I.DU, I.b},
             {(int64_t)I.v * I.b, (int64_t)I.DU * I.b, I.b, 1}),
      mk_pad(I.K, (void *)E.K, {E.d, E.Dl, E.Du, E.Dx, E.De}, {I.d, I.Dl, I.Du, I.Dx, I.De},
             {(int64_t)I.Dl * I.Du * I.Dx * I.De, (int64_t)I.Du * I.Dx * I.De, (int64_t)I.Dx * I.De, I.De, 1}),
      mk_pad(I.Kb, (void *)E.Kb, {E.d, E.DL, E.DU, E.DX, E.DE}, {I.d, I.DL, I.DU, I.DX, I.DE},
             {(int64_t)I.DL * I.DU * I.DX * I.DE, (int64_t)I.DU * I.DX * I.DE, (int64_t)I.DX * I.DE, I.DE, 1})};
  push_pad(B, in, "pad");
  const size_t first = B.ops.size();
  emit_einsumsvd_tc(B, E, o, &I);
  // the orthogonalisations and Grams count the caller's extents too
  const double fm = (double)I.M / E.M, fn = (double)I.N / E.N;
  for (size_t i = first; i < B.ops.size(); ++i) {
    Op &op = B.ops[i];
    const double f = (op.tag == "orth_m" || op.tag == "epilogue_u") ? fm
                     : (op.tag == "orth_n" || op.tag == "svd_gram") ? fn : 1.0;
    op.flops *= f;
    op.bytes *= f;
  }
  // U [kL][t][k] and W [k][(x,X)][b][(e,E)] cut out of the padded results
  std::vector<PadDesc> out{
      mk_pad(E.U, I.U, {I.kL, I.t, I.k}, {I.kL, I.t, I.k}, {(int64_t)E.t * E.k, E.k, 1}),
      mk_pad(E.W, I.W, {I.k, I.Dx, I.DX, I.b, I.De, I.DE}, {I.k, I.Dx, I.DX, I.b, I.De, I.DE},
             {E.N, (int64_t)E.DX * E.b * E.De * E.DE, (int64_t)E.b * E.De * E.DE, (int64_t)E.De * E.DE, E.DE, 1})};
  push_pad(B, out, "pad");
}

void emit_einsumsvd_tc_one(Builder &B, Inst &q, const RsvdOpts &o) { emit_einsumsvd_tc(B, q, o); }

std::string inst_check(const Inst &I, int dt) {
  const int dims[] = {I.kL, I.t, I.a, I.b, I.d, I.Dl, I.Du, I.Dx, I.De, I.DL, I.DU, I.DX, I.DE};
  for (int x : dims)
    if (x < 1) return "every dimension must be >= 1";
  auto p4 = [](int x) { return (x + 3) / 4; };
  const int P1 = I.Dl * I.Du, Q1 = I.Dx * I.De, P2 = I.DL * I.DU, Q2 = I.DX * I.DE;
  if (p4(P1) * p4(Q2) > 256 || p4(P1) * p4(P2) > 256 || p4(Q1) * p4(Q2) > 256)
    return "site bond products (left*up, down*right) above 64 are not supported";
  SandwichDesc s{};
  s.d = I.d; s.Dl = I.Dl; s.Du = I.Du; s.Dx = I.Dx; s.De = I.De; s.DL = I.DL; s.DU = I.DU; s.DX = I.DX;
  s.DE = I.DE;
  for (int adj = 0; adj < 2; ++adj) {
    s.adjoint = adj;
    if (sandwich_smem_bytes(dt, s) > 227 * 1024) return "site tensors too large for shared memory";
  }
  if (I.ell > 1024) return "sketch width l = min(k+p, M, N) above 1024 is not supported";
  if (I.M > (1ll << 31) || I.N > (1ll << 31)) return "matrix dimension above 2^31";
  return "";
}

// ===========================================================================
// einsumsvd adjoint (plain path, real data).  Reverse mode of the same
// function the forward computes, the sketch held fixed:
//   Y0 = A Om, P0 R0 = Y0;  Z_i = A^T P_{i-1}, Q_i S_i = Z_i, Y_i = A Q_i,
//   P_i R_i = Y_i;  Z = A^T P_q, B = Z^T = U~ S V~^T;  U = P_q Ut, W = Ut^T B / s1,
//   log s1  (Ut = the kept, gauge-fixed U~ columns)
// Cotangent of A: sum over the pairs (L_t, R_t) of L_t R_t^T, contracted
// into the operands at the end.
// ===========================================================================

namespace {

void push_copy(Builder &B, void *dst, const void *src, int64_t bytes, const char *tag) {
  Op op;
  op.kind = Op::COPY; op.fill_ptr = dst; op.aux_ptr = src; op.fill_n = bytes; op.tag = tag;
  B.ops.push_back(op);
}

GemmDesc gemm_acc(GemmDesc g, bool acc) {
  g.accumulate = acc ? 1 : 0;
  return g;
}

void push_one(Builder &B, GemmDesc g, const char *tag) {
  std::vector<GemmDesc> v{g};
  push_gemm(B, v, false, tag);
}

// CholeskyQR2 of src into dst (M- or N-side), saving R^-1 = T1 T2 in Tsave.
void orth_save(Builder &B, Inst &q, bool mside, void *Tsave, GradBufs &G) {
  std::vector<Inst *> one{&q};
  void *Inst::*a = mside ? &Inst::Y : &Inst::Z;
  void *Inst::*t = mside ? &Inst::P : &Inst::X;
  const char *tag = mside ? "orth_m" : "orth_n";
  const int64_t es = dtype_size(B.dt), l = q.ell;
  emit_cqr_pass(B, one, mside, a, t, &Inst::R1, nullptr, nullptr, true, tag, true);
  push_copy(B, G.T1s, q.Tm, l * l * es, tag);
  emit_cqr_pass(B, one, mside, t, a, &Inst::R1, nullptr, nullptr, true, tag, false);
  // Tsave = T1 T2 (row-major l x l)
  push_one(B, mk_gemm((int)l, (int)l, (int)l, 1, G.T1s, l, 1, 0, false, q.Tm, l, 1, 0, false, Tsave, l, 1, 0), tag);
}

// QR adjoint on the [j][row] layout: Ybar = (Qbar + Q copyltu(-Qbar^T Q)) R^-T,
// R^-1 = T; rows = M or N.
void qr_bwd(Builder &B, GradBufs &G, int64_t l, int64_t rows, const void *Q, const void *Qbar, const void *T,
            void *Ybar, const char *tag) {
  // Ms[a][b] = -sum_r Qbar[a][r] Q[b][r]
  GemmDesc m = mk_gemm((int)l, (int)l, (int)rows, 1, Qbar, rows, 1, 0, false, Q, 1, rows, 0, false, G.Ms, l, 1, 0);
  m.alpha = -1.0;
  push_one(B, m, tag);
  Op lt;
  lt.kind = Op::LTU; lt.aux_ptr = G.Ms; lt.fill_ptr = G.Cq; lt.fill_n = l; lt.tag = tag;
  B.ops.push_back(lt);
  // Xbar[j][r] = Qbar[j][r] + sum_i Cq[i][j] Q[i][r]
  push_copy(B, G.Xbar, Qbar, l * rows * dtype_size(B.dt), tag);
  push_one(B, gemm_acc(mk_gemm((int)l, (int)rows, (int)l, 1, G.Cq, 1, l, 0, false, Q, rows, 1, 0, false, G.Xbar,
                               rows, 1, 0), true), tag);
  // Ybar[j][r] = sum_i T[j][i] Xbar[i][r]
  push_one(B, mk_gemm((int)l, (int)rows, (int)l, 1, T, l, 1, 0, false, G.Xbar, rows, 1, 0, false, Ybar, rows, 1, 0),
           tag);
}

}  // namespace

void grad_alloc(Builder &B, const Inst &q, const RsvdOpts &o, GradBufs &G, int dt) {
  const int64_t es = dtype_size(dt), l = q.ell, M = q.M, N = q.N, k = q.k;
  G.Ps.clear(); G.Qs.clear(); G.Tp.clear(); G.Tq.clear();
  for (int i = 0; i <= o.q; ++i) { G.Ps.push_back(B.buf(M * l * es)); G.Tp.push_back(B.buf(l * l * es)); }
  for (int i = 0; i < o.q; ++i) { G.Qs.push_back(B.buf(N * l * es)); G.Tq.push_back(B.buf(l * l * es)); }
  G.Om = B.buf(N * l * es);
  G.T1s = B.buf(l * l * es);
  G.Pbar = B.buf(M * l * es);
  G.Xbar = B.buf(std::max(M, N) * l * es);
  G.Qbar = B.buf(N * l * es);
  G.Utbar = B.buf(l * k * es);
  G.WW = B.buf(k * k * es);
  G.H = B.buf(l * l * es);
  G.Ms = B.buf(l * l * es);
  G.Cq = B.buf(l * l * es);
  G.svd_scr = (double *)B.buf((3 * l * l + l) * 8 + l * 4);
  G.Pw = (int)((2 * o.q + 2) * l);
  const int64_t Pw = G.Pw;
  G.Lall = B.buf(Pw * M * es);
  G.Rall = B.buf(Pw * N * es);
  G.T2g = B.buf(Pw * q.h * q.v * q.b * es);
  G.T3g = B.buf(Pw * q.a * q.h * es);
  G.Z3g = B.buf(Pw * q.a * q.h * es);
  G.Z3p = B.buf(Pw * q.a * q.h * es);
  G.Z2g = B.buf(Pw * q.h * q.v * q.b * es);
}

void emit_einsumsvd_save(Builder &B, Inst &q, const RsvdOpts &o, GradBufs &G) {
  std::vector<Inst *> one{&q};
  const int64_t es = dtype_size(B.dt), l = q.ell;
  emit_sketch(B, one, o);
  push_copy(B, G.Om, q.X, q.N * l * es, "sketch");
  emit_product(B, one, true);
  orth_save(B, q, true, G.Tp[0], G);
  push_copy(B, G.Ps[0], q.Y, q.M * l * es, "orth_m");
  for (int it = 0; it < o.q; ++it) {
    emit_adjoint(B, one);
    orth_save(B, q, false, G.Tq[it], G);
    push_copy(B, G.Qs[it], q.Z, q.N * l * es, "orth_n");
    emit_product(B, one, false);
    orth_save(B, q, true, G.Tp[it + 1], G);
    push_copy(B, G.Ps[it + 1], q.Y, q.M * l * es, "orth_m");
  }
  emit_adjoint(B, one);
  emit_small_svd(B, one);
  emit_epilogue(B, one);
}

void emit_einsumsvd_bwd(Builder &B, Inst &q, const RsvdOpts &o, GradBufs &G, const void *Ubar, const void *Wbar,
                        const double *lbar, void *dV, void *dS, void *dK, void *dKb) {
  const int64_t es = dtype_size(B.dt), l = q.ell, M = q.M, N = q.N, k = q.k;
  const char *tag = "backward";
  auto Lslot = [&](int t) { return (uint8_t *)G.Lall + (size_t)t * l * M * es; };
  auto Rslot = [&](int t) { return (uint8_t *)G.Rall + (size_t)t * l * N * es; };
  // views of the instance whose products read / write the adjoint's buffers
  auto product_into = [&](const void *src, void *dst) {
    Inst v = q;
    v.Z = (void *)src; v.Y = dst;
    std::vector<Inst *> one{&v};
    emit_product(B, one, false);
  };
  auto adjoint_into = [&](const void *src, void *dst) {
    Inst v = q;
    v.Y = (void *)src; v.Z = dst;
    std::vector<Inst *> one{&v};
    emit_adjoint(B, one);
  };
  const void *Pq = G.Ps[o.q];
  // Utbar = Pq^T Ubar + Z^T Wbar^T / s1      ([j][c])
  push_one(B, mk_gemm((int)l, (int)k, (int)M, 1, Pq, M, 1, 0, false, Ubar, k, 1, 0, false, G.Utbar, k, 1, 0), tag);
  {
    GemmDesc g = mk_gemm((int)l, (int)k, (int)N, 1, q.Z, N, 1, 0, false, Wbar, 1, N, 0, false, G.Utbar, k, 1, 0);
    g.alpha_dev = q.inv_s1;
    push_one(B, gemm_acc(g, true), tag);
  }
  // WW = Wbar W^T (k x k)
  push_one(B, mk_gemm((int)k, (int)k, (int)N, 1, Wbar, N, 1, 0, false, q.W, 1, N, 0, false, G.WW, k, 1, 0), tag);
  {
    SvdBwdDesc d{};
    d.Mw = q.Mw; d.sig = q.sig; d.Ut = q.Ut; d.Utbar = G.Utbar; d.WW = G.WW; d.lbar = lbar; d.inv_s1 = q.inv_s1;
    d.H = G.H; d.scratch = G.svd_scr; d.n = (int)l; d.k = (int)k;
    Op op;
    op.kind = Op::SVDBWD; op.desc_off = B.put(std::vector<SvdBwdDesc>{d}); op.nd = 1; op.tag = tag;
    B.ops.push_back(op);
  }
  // Zbar = Z H^T + Wbar^T Ut^T / s1, written as pair 0's right factor ([j][n])
  void *Zbar = Rslot(0);
  push_one(B, mk_gemm((int)l, (int)N, (int)l, 1, G.H, l, 1, 0, false, q.Z, N, 1, 0, false, Zbar, N, 1, 0), tag);
  {
    GemmDesc g = mk_gemm((int)l, (int)N, (int)k, 1, q.Ut, k, 1, 0, false, Wbar, N, 1, 0, false, Zbar, N, 1, 0);
    g.alpha_dev = q.inv_s1;
    push_one(B, gemm_acc(g, true), tag);
  }
  push_copy(B, Lslot(0), Pq, M * l * es, tag);
  // Pbar = A Zbar + Ubar Ut^T     ([j][m])
  product_into(Zbar, G.Pbar);
  push_one(B, gemm_acc(mk_gemm((int)l, (int)M, (int)k, 1, q.Ut, k, 1, 0, false, Ubar, 1, k, 0, false, G.Pbar, M, 1, 0),
                       true), tag);
  int slot = 1;
  for (int i = o.q; i >= 1; --i) {
    void *Ybar = Lslot(slot);
    qr_bwd(B, G, l, M, G.Ps[i], G.Pbar, G.Tp[i], Ybar, tag);
    push_copy(B, Rslot(slot), G.Qs[i - 1], N * l * es, tag);
    ++slot;
    adjoint_into(Ybar, G.Qbar);
    void *Zb = Rslot(slot);
    qr_bwd(B, G, l, N, G.Qs[i - 1], G.Qbar, G.Tq[i - 1], Zb, tag);
    push_copy(B, Lslot(slot), G.Ps[i - 1], M * l * es, tag);
    ++slot;
    product_into(Zb, G.Pbar);
  }
  qr_bwd(B, G, l, M, G.Ps[0], G.Pbar, G.Tp[0], Lslot(slot), tag);
  push_copy(B, Rslot(slot), G.Om, N * l * es, tag);
  // ---- operand cotangents from Abar = Lall^T-pairs ----
  const int64_t Pw = G.Pw, ah = (int64_t)q.a * q.h, vb = (int64_t)q.v * q.b, hvb = (int64_t)q.h * vb;
  {
    // T2g, T3g: the first three product stages applied to Rall
    Inst v = q;
    v.ell = (int)Pw; v.X = G.Rall; v.T2 = G.T2g; v.T3 = G.T3g;
    std::vector<SandwichDesc> sw{mk_sandwich(v, G.Rall, G.T2g, false)};
    push_sandwich(B, sw, tag);
    std::vector<GemmDesc> g3{mk_gemm(q.a, q.h, (int)vb, (int)Pw, q.S, vb, 1, 0, false, G.T2g, 1, vb, hvb, false,
                                     G.T3g, q.h, 1, ah)};
    push_gemm(B, g3, false, tag);
  }
  // dV[m][(a,h)] = sum_j Lall[j][m] T3g[j][(a,h)]
  push_one(B, mk_gemm((int)M, (int)ah, (int)Pw, 1, G.Lall, 1, M, 0, false, G.T3g, ah, 1, 0, false, dV, ah, 1, 0), tag);
  // Z3g[j][(a,h)] = sum_m Lall[j][m] V[m][(a,h)];  Z2g[j][h][(v,b)] = sum_a Z3g[j][a][h] S[a][(v,b)]
  push_one(B, mk_gemm((int)Pw, (int)ah, (int)M, 1, G.Lall, M, 1, 0, false, q.V, ah, 1, 0, false, G.Z3g, ah, 1, 0), tag);
  {
    std::vector<GemmDesc> g3{mk_gemm(q.h, (int)vb, q.a, (int)Pw, G.Z3g, 1, q.h, ah, false, q.S, vb, 1, 0, false,
                                     G.Z2g, vb, 1, hvb)};
    push_gemm(B, g3, false, tag);
  }
  // dS[a][(v,b)] = sum_{j,h} Z3g[j][a][h] T2g[j][h][(v,b)]  (Z3g regrouped to [a][(j,h)])
  {
    std::vector<PermuteDesc> pd(1);
    pd[0] = PermuteDesc{};
    pd[0].in = G.Z3g; pd[0].out = G.Z3p; pd[0].nb = 1; pd[0].R = Pw; pd[0].Cc = q.a; pd[0].Q = q.h; pd[0].conj = 0;
    std::vector<int64_t> bl{permute_blocks(pd[0])};
    push_grouped(B, Op::PERMUTE, pd.data(), sizeof(PermuteDesc), 1, bl, tag);
    push_one(B, mk_gemm(q.a, (int)vb, (int)(Pw * q.h), 1, G.Z3p, Pw * q.h, 1, 0, false, G.T2g, vb, 1, 0, false, dS,
                        vb, 1, 0), tag);
  }
  {
    TensorGradDesc d{};
    d.Z2 = G.Z2g; d.R = G.Rall; d.K = q.K; d.Kb = q.Kb; d.Kbar = dK; d.Kbbar = dKb;
    d.P = (int)Pw; d.b = q.b; d.d = q.d; d.Dl = q.Dl; d.Du = q.Du; d.Dx = q.Dx; d.De = q.De;
    d.DL = q.DL; d.DU = q.DU; d.DX = q.DX; d.DE = q.DE;
    Op op;
    op.kind = Op::TGRAD; op.desc_off = B.put(std::vector<TensorGradDesc>{d}); op.nd = 1; op.tag = tag;
    B.ops.push_back(op);
  }
}

void emit_einsumsvd(Builder &B, std::vector<Inst *> &I, const RsvdOpts &o) {
  // tensor-core instances run one by one; the rest share grouped launches
  std::vector<Inst *> simt;
  for (Inst *p : I) {
    if (p->tc) emit_einsumsvd_tc(B, *p, o);
    else simt.push_back(p);
  }
  if (simt.empty()) return;
  emit_einsumsvd_simt(B, simt, o);
}

void emit_einsumsvd_simt(Builder &B, std::vector<Inst *> &I, const RsvdOpts &o) {
  emit_sketch(B, I, o);
  emit_product(B, I, true);
  emit_orth(B, I, true, false, o.fp64_small);
  for (int it = 0; it < o.q; ++it) {
    emit_adjoint(B, I);
    emit_orth(B, I, false, false, o.fp64_small);
    emit_product(B, I, false);
    emit_orth(B, I, true, false, o.fp64_small);
  }
  emit_adjoint(B, I);
  emit_small_svd(B, I, o.fp64_small);
  emit_epilogue(B, I);
}


// ===========================================================================
// Operator application by QR-SVD (Algorithm 1) on one TEBD pass.
// Site matrices (Algorithm 1's "QR(M)"): horizontal bond, M1 as
// [(l,u,x)][(s,e)] and M2 as [(u,x,e)][(s,l)]; vertical bond, M1 as
// [(l,u,e)][(s,x)] and M2 as [(l,x,e)][(s,u)].  A side with more outer entries
// than n = d Db is factorised by CholeskyQR2 (Grams in FP64 accumulators), a
// side with fewer is its own R (Q = identity).
// ===========================================================================

std::string tebd_bond_shape(TebdBond &t) {
  const int *a = t.s1, *b = t.s2;
  t.d = a[0];
  if (b[0] != t.d) return "sites of a bond have different physical dimensions";
  t.Db = t.vertical ? a[3] : a[4];
  if ((t.vertical ? b[2] : b[1]) != t.Db) return "bond dimensions of neighbouring sites differ";
  t.O1 = t.vertical ? (int64_t)a[1] * a[2] * a[4] : (int64_t)a[1] * a[2] * a[3];
  t.O2 = t.vertical ? (int64_t)b[1] * b[3] * b[4] : (int64_t)b[2] * b[3] * b[4];
  const int n = t.d * t.Db;
  t.f1 = t.O1 > n;
  t.f2 = t.O2 > n;
  t.r1 = t.f1 ? n : (int)t.O1;
  t.r2 = t.f2 ? n : (int)t.O2;
  t.k = t.Db;
  if (t.r1 * t.d > kSvdSmallMax || t.r2 * t.d > kSvdSmallMax)
    return "QR rank times physical dimension above 64 is not supported";
  if (t.k > t.r1 * t.d || t.k > t.r2 * t.d) return "bond above the rank of the two-site operator";
  return "";
}

void tebd_alloc(Builder &B, TebdBond &t, int dt) {
  const size_t es = dtype_size(dt), as = acc_size(dt);
  const size_t n = (size_t)t.d * t.Db, rows = (size_t)t.r1 * t.d, cols = (size_t)t.r2 * t.d;
  t.A1 = B.buf(t.O1 * n * es);
  t.A2 = B.buf(t.O2 * n * es);
  auto side = [&](bool f, int64_t O, void *&Qa, void *&Q, void *&G, void *&Ra, void *&Rb, void *&R, void *&T) {
    if (!f) return;
    Qa = B.buf(O * n * es);
    Q = B.buf(O * n * es);
    G = B.buf(n * n * as);
    Ra = B.buf(n * n * as);
    Rb = B.buf(n * n * as);
    R = B.buf(n * n * as);
    T = B.buf(n * n * as);
  };
  side(t.f1, t.O1, t.Qa1, t.Q1, t.G1, t.Ra1, t.Rb1, t.R1, t.T1);
  side(t.f2, t.O2, t.Qa2, t.Q2, t.G2, t.Ra2, t.Rb2, t.R2, t.T2);
  t.Theta = B.buf(rows * cols * es);
  t.R1t = B.buf(rows * t.k * es);
  t.R2t = B.buf(cols * t.k * es);
  t.N1 = t.f1 ? B.buf(t.O1 * t.d * t.k * es) : t.R1t;
  t.N2 = t.f2 ? B.buf(t.O2 * t.d * t.k * es) : t.R2t;
  t.g = B.buf(t.O1 * t.d * es);
  t.sigma = (double *)B.buf(t.k * 8);
}

namespace {

// in_stride of a [d][l][u][x][e] site for each of its five axes
void site_strides(const int *sd, int64_t st[5]) {
  st[4] = 1;
  for (int i = 3; i >= 0; --i) st[i] = st[i + 1] * sd[i + 1];
}

// CholeskyQR2 of the factorised sides: Q = A R^-1 with R = R_b R_a
void emit_tebd_qr(Builder &B, std::vector<TebdBond> &bonds) {
  const int as = acc_size(B.dt);
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<std::pair<void *, int64_t>> z;
    std::vector<GemmDesc> gram, app;
    std::vector<CholDesc> ch;
    auto add = [&](TebdBond &t, bool f, int64_t O, void *A, void *Qa, void *Q, void *G, void *Ra, void *Rb, void *R,
                   void *T) {
      if (!f) return;
      const int n = t.d * t.Db;
      const void *src = pass == 0 ? A : Qa;
      z.push_back({G, (int64_t)n * n * as / 8});
      // G[i][j] = sum_o conj(src[o][i]) src[o][j]
      gram.push_back(mk_gemm(n, n, (int)O, 1, src, 1, n, 0, true, src, n, 1, 0, false, G, n, 1, 0));
      CholDesc c{};
      c.G = G; c.T = T; c.n = n; c.tol = chol_tol(B.dt, n); c.status = B.status;
      if (pass == 0) {
        c.R = Ra;
        c.shift = chol_shift(B.dt, n, true);
      } else {
        c.R = Rb; c.Rprev = Ra; c.Rout = R;
      }
      ch.push_back(c);
      app.push_back(mk_gemm((int)O, n, n, 1, src, n, 1, 0, false, T, n, 1, 0, false, pass == 0 ? Qa : Q, n, 1, 0));
    };
    for (TebdBond &t : bonds) {
      add(t, t.f1, t.O1, t.A1, t.Qa1, t.Q1, t.G1, t.Ra1, t.Rb1, t.R1, t.T1);
      add(t, t.f2, t.O2, t.A2, t.Qa2, t.Q2, t.G2, t.Ra2, t.Rb2, t.R2, t.T2);
    }
    if (ch.empty()) return;
    for (auto &g : gram) set_ksplit(g, (int)gram.size());
    push_zero(B, z, "tebd_qr");
    push_gemm(B, gram, true, "tebd_qr");
    Op op;
    op.kind = Op::CHOL; op.desc_off = B.put(ch); op.nd = (int)ch.size(); op.tag = "tebd_qr";
    for (auto &c : ch) {
      op.smem = std::max(op.smem, small_smem_bytes(B.dt, c.n));
      op.smem2 = std::max(op.smem2, chol_cluster_smem_bytes(B.dt, c.n, true));
    }
    B.ops.push_back(op);
    push_gemm(B, app, false, "tebd_qr");
  }
}

template <class D> void push_small(Builder &B, Op::Kind kind, const std::vector<D> &d, const char *tag, int smem = 0) {
  if (d.empty()) return;
  Op op;
  op.kind = kind; op.desc_off = B.put(d); op.nd = (int)d.size(); op.tag = tag; op.smem = smem;
  B.ops.push_back(op);
}

}  // namespace

void emit_site_ops(Builder &B, const std::vector<SiteOpDesc> &d) {
  if (d.empty()) return;
  int64_t rest = 1;
  for (const SiteOpDesc &x : d) rest = std::max(rest, x.rest);
  Op op;
  op.kind = Op::SITEOP; op.desc_off = B.put(d); op.nd = (int)d.size(); op.tag = "tebd_site_op";
  op.blocks = std::min<int64_t>(ceil_div(rest, 256), 1024);     // column blocks per site
  const int es = dtype_size(B.dt);
  const double mult = dtype_complex(B.dt) ? 8.0 : 2.0;
  for (const SiteOpDesc &x : d) {
    op.flops += mult * (double)x.d * x.d * x.rest;
    op.bytes += 2.0 * es * (double)x.d * x.rest;
  }
  B.ops.push_back(op);
}

void emit_tebd_pass(Builder &B, std::vector<TebdBond> &bonds, uint64_t seed, bool unit_bond) {
  const int es = dtype_size(B.dt);
  // 1. site matrices (Algorithm 1's QR input), outer bonds first
  std::vector<PadDesc> in;
  for (TebdBond &t : bonds) {
    int64_t a[5], b[5];
    site_strides(t.s1, a);
    site_strides(t.s2, b);
    const int *x = t.s1, *y = t.s2;
    if (t.vertical) {
      in.push_back(mk_pad(t.M1, t.A1, {x[1], x[2], x[4], x[0], x[3]}, {x[1], x[2], x[4], x[0], x[3]},
                          {a[1], a[2], a[4], a[0], a[3]}));
      in.push_back(mk_pad(t.M2, t.A2, {y[1], y[3], y[4], y[0], y[2]}, {y[1], y[3], y[4], y[0], y[2]},
                          {b[1], b[3], b[4], b[0], b[2]}));
    } else {
      in.push_back(mk_pad(t.M1, t.A1, {x[1], x[2], x[3], x[0], x[4]}, {x[1], x[2], x[3], x[0], x[4]},
                          {a[1], a[2], a[3], a[0], a[4]}));
      in.push_back(mk_pad(t.M2, t.A2, {y[2], y[3], y[4], y[0], y[1]}, {y[2], y[3], y[4], y[0], y[1]},
                          {b[2], b[3], b[4], b[0], b[1]}));
    }
  }
  push_pad(B, in, "tebd_site");
  // 2. QR factorisations
  emit_tebd_qr(B, bonds);
  // 3. Theta, 4. its truncated SVD
  std::vector<ThetaDesc> th;
  std::vector<SvdSmallDesc> sv;
  int smem = 0;
  for (TebdBond &t : bonds) {
    ThetaDesc x{};
    x.R1 = t.f1 ? t.R1 : t.A1; x.R2 = t.f2 ? t.R2 : t.A2; x.G = t.gate; x.Theta = t.Theta;
    x.r1 = t.r1; x.r2 = t.r2; x.d = t.d; x.Db = t.Db;
    th.push_back(x);
    SvdSmallDesc y{};
    y.Theta = t.Theta; y.R1t = t.R1t; y.R2t = t.R2t; y.sigma = t.sigma;
    y.rows = t.r1 * t.d; y.cols = t.r2 * t.d; y.k = t.k; y.status = B.status; y.unit = unit_bond ? 1 : 0;
    sv.push_back(y);
    smem = std::max(smem, svd_small_smem_bytes(B.dt, y.rows, y.cols));
  }
  push_small(B, Op::THETA, th, "tebd_theta");
  push_small(B, Op::SVDSMALL, sv, "tebd_svd", smem);
  // 5. N = Q R~ on the factorised sides
  std::vector<GemmDesc> nq;
  for (TebdBond &t : bonds) {
    const int n = t.d * t.Db, dk = t.d * t.k;
    if (t.f1) nq.push_back(mk_gemm((int)t.O1, dk, n, 1, t.Q1, n, 1, 0, false, t.R1t, dk, 1, 0, false, t.N1, dk, 1, 0));
    if (t.f2) nq.push_back(mk_gemm((int)t.O2, dk, n, 1, t.Q2, n, 1, 0, false, t.R2t, dk, 1, 0, false, t.N2, dk, 1, 0));
  }
  if (!nq.empty()) push_gemm(B, nq, false, "tebd_apply");
  // 6. gauge vectors (one Philox stream per bond, tag 1) and phases
  std::vector<SketchDesc> sk;
  std::vector<int64_t> bl;
  std::vector<SiteGaugeDesc> ga;
  const int per = dtype_complex(B.dt) ? 2 : 4;
  for (TebdBond &t : bonds) {
    SketchDesc s{};
    s.X = t.g; s.N = t.O1 * t.d; s.ld = s.N; s.ell = 1; s.tag = 1; s.kind = 0;
    s.seed = seed; s.instance = (4ull << 32) | ((uint64_t)t.a << 16) | (uint64_t)t.b;
    s.nblocks = ceil_div(ceil_div(s.N, per), 256);
    sketch_set_div(s);
    sk.push_back(s);
    bl.push_back(s.nblocks);
    SiteGaugeDesc g{};
    g.N1 = t.N1; g.N2 = t.N2; g.g = t.g; g.rows1 = t.O1 * t.d; g.rows2 = t.O2 * t.d; g.k = t.k;
    ga.push_back(g);
  }
  push_grouped(B, Op::SKETCH, sk.data(), sizeof(SketchDesc), (int)sk.size(), bl, "tebd_gauge");
  push_small(B, Op::SITEGAUGE, ga, "tebd_gauge");
  // 7. back into the site layouts, in place
  std::vector<PadDesc> out;
  for (TebdBond &t : bonds) {
    const int *x = t.s1, *y = t.s2;
    const int64_t k = t.k, dk = (int64_t)t.d * k;
    if (t.vertical) {
      // N1 [l][u][e][s][k] -> [s][l][u][k][e];  N2 [l][x][e][s][k] -> [s][l][k][x][e]
      out.push_back(mk_pad(t.N1, t.M1, {x[0], x[1], x[2], t.k, x[4]}, {x[0], x[1], x[2], t.k, x[4]},
                           {k, x[2] * x[4] * dk, x[4] * dk, 1, dk}));
      out.push_back(mk_pad(t.N2, t.M2, {y[0], y[1], t.k, y[3], y[4]}, {y[0], y[1], t.k, y[3], y[4]},
                           {k, y[3] * y[4] * dk, 1, y[4] * dk, dk}));
    } else {
      // N1 [l][u][x][s][k] -> [s][l][u][x][k];  N2 [u][x][e][s][k] -> [s][k][u][x][e]
      out.push_back(mk_pad(t.N1, t.M1, {x[0], x[1], x[2], x[3], t.k}, {x[0], x[1], x[2], x[3], t.k},
                           {k, x[2] * x[3] * dk, x[3] * dk, dk, 1}));
      out.push_back(mk_pad(t.N2, t.M2, {y[0], t.k, y[2], y[3], y[4]}, {y[0], t.k, y[2], y[3], y[4]},
                           {k, 1, y[3] * y[4] * dk, y[4] * dk, dk}));
    }
  }
  push_pad(B, out, "tebd_site");
  (void)es;
}

}  // namespace peps
