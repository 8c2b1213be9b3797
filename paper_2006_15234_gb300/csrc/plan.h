// Host-side launch schedule of libpeps: a plan is a static list of grouped
// kernel launches whose descriptors are built once per workspace address and
// uploaded into the workspace, so an execute is a fixed kernel sequence that
// can be replayed or captured in a CUDA graph.
#pragma once
#include <stdint.h>
#include <string.h>
#include <string>
#include <vector>

#include "kernels.h"
#include "tcgemm.h"

namespace peps {

struct Op {
  enum Kind { SKETCH, GEMM, GEMM_ATOMIC, SANDWICH, CHOL, JACOBI, FINALIZE, ZERO, SITE, SCALAR, FILL, TC,
              PERMUTE, STRIP, COPY, SVDBWD, LTU, TGRAD, MEMSET, STRIPBWD, SITEBWD, AXPY, PAD, NARROW, ABSORB, THETA, SVDSMALL, SITEGAUGE,
              BLOBCOPY, SITEOP } kind;
  size_t desc_off = 0;    // byte offset of the descriptor array in the blob
  size_t prefix_off = 0;  // byte offset of the int64 block prefix array in the blob
  int nd = 0;
  int64_t blocks = 0;
  int smem = 0;
  int smem2 = 0;          // second kernel of the launch (cluster Cholesky, block-cyclic cluster Jacobi)
  int smem3 = 0;          // third kernel of the launch (column-window cluster Jacobi)
  bool wide = false;      // CHOL, JACOBI: run in FP64 on single-precision data
  ScalarDesc scalar{};
  size_t aux_off[3] = {0, 0, 0};  // blob offsets of the scalar's device arrays
  void *fill_ptr = nullptr;
  const void *aux_ptr = nullptr;  // COPY / LTU / AXPY source
  StripBwdScratch sbs{};          // STRIPBWD scratch
  AbsorbDesc absorb{};            // ABSORB
  const double *sbar = nullptr;   // STRIPBWD strip cotangents
  int64_t fill_n = 0;             // FILL: elements; COPY, BLOBCOPY: bytes; LTU: n; NARROW: real values
  double fill_value = 0.0;
  std::string tag;        // stage name (profiling ledger)
  double flops = 0.0;     // algorithmic flops of the launch
  double bytes = 0.0;     // algorithmic DRAM bytes of the launch
  // independent chain the launch belongs to: 0 runs on the caller's stream,
  // b > 0 on the plan's side stream b (forked from and joined back into the
  // caller's stream, so a captured execute holds the chains as parallel
  // graph branches)
  int branch = 0;
  // tensor-core GEMM (kind TC): descriptor passed by value, operand spans
  TcDesc tc{};
  int tc_bn = 0;
  const void *tcA = nullptr, *tcB = nullptr;
  int64_t tcA_rows = 0, tcB_rows = 0, tc_kr = 0;
};

struct ZeroDesc {
  void *p;
  int64_t words;          // 8-byte words
};

void launch_zero(const ZeroDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s);
constexpr int kZeroWordsPerBlock = 256 * 8;

// Builds ops + descriptor blob for one workspace base address.
struct Builder {
  uintptr_t base = 0;
  size_t top = 0;                 // bump allocator over buffer space
  std::vector<uint8_t> blob;
  std::vector<Op> ops;
  int dt = 0;
  bool encode = false;            // encode TMA maps (real device pointers, driver present)
  std::string err;                // first encoding failure
  size_t bx_need = 0;             // B scratch of the pre-expanded tensor-core operands (bytes)
  uint32_t *status = nullptr;     // the plan's device status word (STATUS_* bits), in the workspace
  int branch = 0;                 // branch of the ops emitted next (Op::branch)
  std::vector<size_t> bx_branch;  // B scratch need per branch > 0 (bytes)

  size_t alloc(size_t bytes) {
    size_t o = (top + 255) & ~(size_t)255;
    top = o + bytes;
    return o;
  }
  void *ptr(size_t off) const { return (void *)(base + off); }
  void *buf(size_t bytes) { return ptr(alloc(bytes)); }
  int branches() const {
    int n = 1;
    for (const Op &o : ops) n = o.branch + 1 > n ? o.branch + 1 : n;
    return n;
  }

  size_t put_bytes(const void *p, size_t n) {
    size_t o = (blob.size() + 15) & ~(size_t)15;
    blob.resize(o + n);
    memcpy(blob.data() + o, p, n);
    return o;
  }
  template <class D> size_t put(const std::vector<D> &v) { return put_bytes(v.data(), v.size() * sizeof(D)); }
};

}  // namespace peps

namespace peps {

// One einsumsvd instance (Algorithm 3's einsumsvd line, Algorithm 4 inside):
// shape, operand / output pointers and the scratch buffers its stages use.
struct Inst {
  int kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE;
  int h, v;
  int64_t M, N;
  int k, ell;
  uint64_t instance;
  const void *V, *S, *K, *Kb;
  void *U, *W;
  double *sigma, *logp;
  // scratch (working type unless noted)
  void *X, *Z, *T2, *T3, *Y, *P, *g, *Tm, *Ut;
  void *G, *R1, *R2, *Rout, *Mw;   // G: FP64 accumulators; the others working type
  double *sig, *inv_s1;
  // tensor-core path scratch
  void *T1, *VT, *ST, *UT, *KT, *KbP, *KbT;
  bool tc;                          // this instance runs its products on tensor cores
  // runs as a zero-padded copy whose extents meet the tensor cores' alignment
  // (set on the caller's instance; the copy is a separate Inst)
  bool embed;
};

struct RsvdOpts {
  int m, p, q;
  uint64_t seed;
  int sketch;
  int prec;
  bool orth_q;
  bool fp64_small;     // single-precision data: CholeskyQR2's factorisations and the Jacobi SVD in FP64
  bool alternate;      // contraction sweeps: Sigma into the finished site on even rows
  bool unit_bond;      // TEBD: each new bond's Sigma divided by sigma_1 before the split
};

// Shape bookkeeping shared by every planner.
void inst_derive(Inst &I, const RsvdOpts &o);
// Bytes of per-instance scratch.
size_t inst_scratch_bytes(const Inst &I, int dt);
// Carve per-instance scratch out of the builder.
void inst_alloc_scratch(Builder &B, Inst &I, int dt);
// the B scratch of the pre-expanded tensor-core operands and their TMA maps;
// called once after the whole schedule is emitted
void tc_finish(Builder &B);
// Shape signature of a tensor-core GEMM launch (the autotuner's table key),
// its candidate MMA widths, and a change of its MMA width (N tiling and the B
// operand's TMA boxes re-encoded; false if the maps cannot be encoded).
std::string tc_signature(const Op &op);
std::vector<int> tc_candidates(const Op &op);
bool tc_retile(Op &op, int nmma);
// Point I's scratch at another instance's buffers (the sweep reuses one set).
void inst_share_scratch(Inst &I, const Inst &owner);
// Check the shape against the kernels' limits; returns "" when supported.
std::string inst_check(const Inst &I, int dt);
// Whether every stage GEMM of the instance meets the TMA alignment rules.
bool inst_tc_ok(const Inst &I, int dt);
// Saved forward data and scratch of the einsumsvd adjoint (plain path, real
// data): the orthonormal bases P_i (M x l) and Q_i (N x l) of the power
// iteration with the inverses of their R factors, the sketch, and the
// buffers of the reverse sweep.
struct GradBufs {
  std::vector<void *> Ps, Qs, Tp, Tq;
  void *Om = nullptr, *T1s = nullptr;
  void *Pbar = nullptr, *Xbar = nullptr, *Qbar = nullptr, *Utbar = nullptr, *WW = nullptr, *H = nullptr;
  void *Ms = nullptr, *Cq = nullptr;
  double *svd_scr = nullptr;
  void *Lall = nullptr, *Rall = nullptr;
  void *T2g = nullptr, *T3g = nullptr, *Z3g = nullptr, *Z3p = nullptr, *Z2g = nullptr;
  int Pw = 0;
};
void grad_alloc(Builder &B, const Inst &q, const RsvdOpts &o, GradBufs &G, int dt);
// Forward of one plain-path instance that keeps what the adjoint needs.
void emit_einsumsvd_save(Builder &B, Inst &q, const RsvdOpts &o, GradBufs &G);
// Reverse sweep: cotangents of U ([M][k]), W ([k][N]) and log sigma_1 to
// those of V, S, K and Kb (same layouts as the operands).
void emit_einsumsvd_bwd(Builder &B, Inst &q, const RsvdOpts &o, GradBufs &G, const void *Ubar, const void *Wbar,
                        const double *lbar, void *dV, void *dS, void *dK, void *dKb);

// One bond of a TEBD pass (Algorithm 1): the two sites (updated in place),
// the geometry and the scratch of its QR factorisations and truncated SVD.
struct TebdBond {
  int a = 0, b = 0;                 // row-major site indices (the bond's Philox stream)
  bool vertical = false;
  int d = 0, Db = 0;                // physical dimension, shared bond (kept)
  int s1[5] = {}, s2[5] = {};       // site dims [d][l][u][x][e]
  void *M1 = nullptr, *M2 = nullptr;
  int64_t O1 = 0, O2 = 0;           // outer entries of each site matrix
  bool f1 = false, f2 = false;      // side factorised (more outer entries than d * Db)
  int r1 = 0, r2 = 0, k = 0;        // QR ranks, new bond (= Db)
  // scratch
  void *A1 = nullptr, *A2 = nullptr, *Qa1 = nullptr, *Qa2 = nullptr, *Q1 = nullptr, *Q2 = nullptr;
  void *G1 = nullptr, *G2 = nullptr;                       // FP64 Grams
  void *Ra1 = nullptr, *Ra2 = nullptr, *Rb1 = nullptr, *Rb2 = nullptr, *R1 = nullptr, *R2 = nullptr;
  void *T1 = nullptr, *T2 = nullptr;
  void *Theta = nullptr, *R1t = nullptr, *R2t = nullptr, *N1 = nullptr, *N2 = nullptr, *g = nullptr;
  double *sigma = nullptr;
  const void *gate = nullptr;       // this bond's d^2 x d^2 operator (device)
};
// Shapes of a bond from its two sites; "" or the reason it is not supported.
std::string tebd_bond_shape(TebdBond &t);
void tebd_alloc(Builder &B, TebdBond &t, int dt);
// One pass of disjoint bonds: every launch grouped over the pass's bonds.
void emit_tebd_pass(Builder &B, std::vector<TebdBond> &bonds, uint64_t seed, bool unit_bond);
// One-site operators (Eq. 4) on every listed site, in place: one launch.
void emit_site_ops(Builder &B, const std::vector<SiteOpDesc> &d);

// Emit every stage of one einsumsvd over a group of instances.
void emit_einsumsvd(Builder &B, std::vector<Inst *> &I, const RsvdOpts &o);
// Dimensions of the zero-padded copy of I that meets the tensor-core alignment
// (every bond even; t and a multiples of 4 real / 2 complex values), with
// I's rank k and sketch width l; false if the copy would exceed the kernels'
// limits.
bool inst_embed_dims(const Inst &I, int dt, const RsvdOpts &o, Inst &E);
// Bytes of E's scratch plus its padded operands and outputs.
size_t inst_embed_bytes(const Inst &E, int dt);
// Carve E's scratch, padded operands and outputs out of the builder.
void inst_embed_alloc(Builder &B, Inst &E, int dt);
// One instance through its padded copy E: operands zero-padded into E, the
// tensor-core einsumsvd of E with the sketch and gauge vector drawn at I's
// element numbering, U and W cut back into I's outputs.
void emit_einsumsvd_embedded(Builder &B, Inst &I, Inst &E, const RsvdOpts &o);
void emit_einsumsvd_tc_one(Builder &B, Inst &q, const RsvdOpts &o);
void emit_einsumsvd_simt(Builder &B, std::vector<Inst *> &I, const RsvdOpts &o);

}  // namespace peps
