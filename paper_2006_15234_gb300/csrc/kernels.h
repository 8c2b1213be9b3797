// Launch descriptors and launcher declarations of the libpeps kernels.
//
// Every kernel is "grouped": it reads an array of per-problem descriptors
// from device memory plus a prefix sum of the blocks each problem needs, so
// one launch serves one problem (a step of a boundary sweep) or hundreds of
// uneven ones (a batch of independent einsumsvd instances).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace peps {

enum DType : int32_t { DT_R32 = 0, DT_C64 = 1, DT_R64 = 2, DT_C128 = 3 };

inline int dtype_size(int dt) { return dt == DT_R32 ? 4 : (dt == DT_R64 || dt == DT_C64) ? 8 : 16; }
inline bool dtype_complex(int dt) { return dt == DT_C64 || dt == DT_C128; }
inline bool dtype_double(int dt) { return dt == DT_R64 || dt == DT_C128; }
// size of the FP64 accumulation element (double or double2)
inline int acc_size(int dt) { return dtype_complex(dt) ? 16 : 8; }

// C[b](m,n) = alpha * sum_k opA(A[b](m,k)) * opB(B[b](k,n))  (+ C if accumulate)
// with element (m,k) of A at A + b*sAb + m*sAm + k*sAk (likewise B, C).
// In "atomic" launches C points to FP64 accumulators (double / double2) and
// partial sums over K chunks are added atomically (split-K Gram matrices).
struct GemmDesc {
  const void *A, *B;
  void *C;
  int32_t M, N, K, batch;
  int32_t ksplit, kchunk;          // K is cut into ksplit chunks of kchunk
  int32_t tiles_m, tiles_n;
  int64_t sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
  double alpha;
  const double *alpha_dev;         // optional device factor (e.g. 1/sigma_1)
  int32_t conjA, conjB, conjC, accumulate;
};

// Two-layer site contraction of the implicit product (the two d*D^6 stages):
//  forward (adjoint=0), per (j, b):
//    out[j][(l,L)][(u,U,b)] = sum_s sum_{x,e,X,E} K[s,l,u,x,e] in[j][(x,X,b,e,E)] conj(Kb[s,L,U,X,E])
//  adjoint (adjoint=1), per (j, b):
//    out[j][(x,X,b,e,E)] = sum_s sum_{l,u,L,U} conj(K[s,l,u,x,e]) in[j][(l,L)][(u,U,b)] Kb[s,L,U,X,E]
struct SandwichDesc {
  const void *in;
  void *out;
  const void *K, *Kb;
  int32_t d, Dl, Du, Dx, De, DL, DU, DX, DE, B, ell;
  int32_t adjoint;
  int64_t ld_in, ld_out;           // per-j strides (elements)
  int32_t items_per_block;
  int32_t nblocks;
};

// Philox4x64-10 draw of an N x ell block stored as X[j*ld + map(n)]; map is
// the identity when nd == 0, else n's mixed-radix digits (least significant
// first) times their strides.
struct SketchDesc {
  void *X;
  int64_t N, ld;
  int32_t ell;
  int32_t tag, kind;               // kind 0 Gaussian, 1 uniform
  uint64_t seed, instance;
  int64_t nblocks;
  int32_t nd;
  int32_t radix[5];
  int64_t stride[5];
  // multiply-shift division by N and by each radix (sketch_set_div), used
  // when N * ell < 2^31
  uint32_t nmul, nshr;
  uint32_t rmul[5], rshr[5];
};
// fill the division constants of a sketch descriptor (after its radices)
void sketch_set_div(SketchDesc &s);

// out[b][c][r][q] = op(in[b][r][c][q]) for b < nb, r < R, c < Cc, q < Q
// (op = conjugate when conj): swaps two index groups of a tensor.
struct PermuteDesc {
  const void *in;
  void *out;
  int64_t nb, R, Cc, Q;
  int32_t conj;
};

// Strided copy with zero fill over up to 6 index digits (most significant
// first): out[o] for o < total (row-major over dims[]) takes
// in[sum_d digit_d * in_stride[d]] when every digit_d < lim[d], else 0.
// Zero-pads a tensor into larger bond dimensions (lim = source dims < dims)
// or cuts the padding off again (lim = dims, strides of the padded source).
struct PadDesc {
  const void *in;
  void *out;
  int32_t nd;
  int32_t dims[6], lim[6];
  int64_t in_stride[6];
  int64_t total;
};
constexpr int kPadPerBlock = 256;
void launch_pad(int dt, const PadDesc *d, const int64_t *prefix, int nd, int64_t blocks, cudaStream_t s);
// out[i] = in[i] rounded to single precision, i < n (real values)
void launch_narrow(const double *in, float *out, int64_t n, cudaStream_t s);

// Cholesky of a Hermitian Gram (FP64 accumulators, row-major n x n) with
// pivot skipping and an optional diagonal shift, in the working precision:
// upper factor R and T = R^+ (working type, n x n).  If Rprev != nullptr the
// product R * Rprev is written to Rout (working type).
struct CholDesc {
  void *G;
  void *T;
  void *R;
  const void *Rprev;
  void *Rout;
  int32_t n;
  double tol;       // pivot threshold relative to the largest diagonal entry
  double shift;     // diagonal shift relative to the largest diagonal entry
  void *Rlow;       // optional: R rounded to single precision (FP64 kernels only)
  uint32_t *status; // STATUS_NONFINITE when a Gram diagonal entry is not finite (may be NULL)
  void *Tlow;       // optional: T rounded to single precision (FP64 kernels only)
};

// One-sided Jacobi SVD of Mw = Rb^H (n x n, working type, column-major, built
// from the upper factor Rb by the kernel).  On return column c of Mw holds
// sigma_c u_c and sig[c] = sigma_c (unsorted, FP64).
struct JacobiDesc {
  const void *Rb;
  void *Mw;
  double *sig;
  int32_t n;
  int32_t max_sweeps;
  uint32_t *status;
};

// Sort, truncate, zero and gauge-fix the small SVD, then emit the ell x k
// coefficient block Ut (working type, row-major [j][c]) used for U = P Ut and
// W = conj(Ut^T Z) / sigma_1.
struct FinalizeDesc {
  const void *Mw;                  // working type n x n column-major, columns sigma_c u_c
  const double *sig;               // n unsorted singular values
  const void *P;                   // working type, [j][m], ld = M
  const void *g;                   // gauge vector, M entries
  void *Ut;                        // working type [j][c], n x k
  void *h;                         // FP64 (complex) n entries: h_j = sum_m conj(P[j][m]) g[m]
  double *sigma_out;               // k values
  double *log_out;                 // log sigma_1
  double *inv_s1;                  // 1 / sigma_1 (device scalar for the W GEMM)
  int32_t n, k;
  int64_t M;
  double rtol;
  uint32_t *status;
};

// Row one of the two-layer network (Algorithm 2, first line):
// S[(l,L)][(x,X)][(e,E)] = sum_s K[s,l,0,x,e] conj(Kb[s,L,0,X,E]).
// Zip-up start (Algorithm 3, first line), mode 1:
// V[0][(x,X)][b][(e,E)] = sum_{s,u,U} S1[0][(u,U)][b] K[s,0,u,x,e] conj(Kb[s,0,U,X,E]).
struct SiteDesc {
  const void *K, *Kb, *S;
  void *out;
  int32_t mode;
  int32_t d, Dl, Du, Dx, De, DL, DU, DX, DE, B;
  int64_t total;
};

// Sigma moved from the carry into the finished site (alternating
// canonicalisation): U[row][c] *= sigma_c / sigma_0 (U: M x k) and
// W[c][n] *= sigma_0 / sigma_c, 0 where sigma_c = 0 (W: k x N).
struct AbsorbDesc {
  void *U, *W;
  const double *sigma;
  int64_t M, N;
  int32_t k;
};
void launch_absorb(int dt, const AbsorbDesc &d, cudaStream_t s);

// ---- operator application by QR-SVD (Algorithm 1), one TEBD pass ----
constexpr int kSvdSmallMax = 64;   // largest side of Theta (d * QR rank)
// Theta[(r1, i1)][(r2, i2)] = sum_{j1, j2, b} G[i1 i2, j1 j2] R1[r1][(j1, b)] R2[r2][(j2, b)]
struct ThetaDesc {
  const void *R1, *R2;   // [r1][d * Db], [r2][d * Db] (working type, row-major)
  const void *G;         // d^2 x d^2 (working type), [out pair][in pair]
  void *Theta;           // [(r1 d)][(r2 d)]
  int32_t r1, r2, d, Db;
};
// Truncated SVD of Theta (rows x cols): R1t = U sqrt(S) [rows][k],
// R2t = (sqrt(S) V^H)^T [cols][k]; sigma (k values, may be NULL)
struct SvdSmallDesc {
  const void *Theta;
  void *R1t, *R2t;
  double *sigma;
  int32_t rows, cols, k;
  uint32_t *status;   // STATUS_NONFINITE for a non-finite Theta, STATUS_JACOBI_NOCONV at the
                      // FP64 sweep limit (may be NULL)
  int32_t unit;       // 1: split Sigma / sigma_1 instead of Sigma (sigma keeps the true values)
};
// One-site operator on a site tensor, in place (Eq. 4):
// M[i][r] <- sum_j g[i][j] M[j][r], r < rest, d <= kSiteOpMaxPhys
constexpr int kSiteOpMaxPhys = 16;
struct SiteOpDesc {
  void *M;
  const void *g;      // d x d (working type), [out][in]
  int64_t rest;       // product of the site's bond dimensions
  int32_t d;
};
// Phases of the new bond fixed on N1 [rows1][k] against g (rows1 entries);
// N2 [rows2][k] takes the opposite phase
struct SiteGaugeDesc {
  void *N1, *N2;
  const void *g;
  int64_t rows1, rows2;
  int32_t k;
};
// kind 0 theta, 1 svd_small, 2 site_gauge (descriptor arrays on the device)
// kind 0 theta, 1 svd_small (aux = dynamic shared memory bytes), 2 site_gauge,
// 3 site_op (aux = column blocks per site)
void launch_tebd(int dt, int kind, const void *d, int nd, int aux, cudaStream_t s);
int svd_small_smem_bytes(int dt, int rows, int cols);

// Contract a boundary MPS with trivial vertical bonds to a scalar:
// v = S_0[0,0,:] S_1[:,0,:] ... ; result log|v| + sum(logs), arg v.
struct ScalarDesc {
  const void *const *sites;        // device array of ncol site pointers
  const int32_t *left, *right;     // device arrays of bond dims
  int32_t ncol;
  const double *logs;              // nlogs per-step log sigma_1 values
  int32_t nlogs;
  void *scratch;                   // 2 * maxbond working elements
  double *out;                     // [log_abs, phase]
};

// ---- launchers (enqueue on stream; descriptor arrays live on the device) ----
void launch_gemm(int dt, bool atomic, const GemmDesc *d, const int64_t *prefix, int nd,
                 int64_t blocks, cudaStream_t s);
void launch_sandwich(int dt, const SandwichDesc *d, const int64_t *prefix, int nd,
                     int64_t blocks, int smem_bytes, cudaStream_t s);
void launch_sketch(int dt, const SketchDesc *d, const int64_t *prefix, int nd,
                   int64_t blocks, cudaStream_t s);
void launch_chol(int dt, const CholDesc *d, int nd, int smem, int cluster_smem, cudaStream_t s);
// per-CTA shared memory of the cluster Cholesky for n x n (0: not routed there)
int chol_cluster_smem_bytes(int dt, int n, bool needT);
void launch_jacobi(int dt, const JacobiDesc *d, int nd, int smem, int block_smem, int cluster_smem, int nmax,
                   cudaStream_t s);
// per-CTA shared memory of the block-cyclic / column-window cluster Jacobi (0: not used for n)
int jacobi_block_smem_bytes(int dt, int n);
int jacobi_cluster_smem_bytes(int dt, int n);
int small_smem_bytes(int dt, int n);   // shared memory of chol / jacobi for n x n (0: global)
// nmax: largest n of the descriptors (CTAs per instance of the gauge projections)
void launch_finalize(int dt, const FinalizeDesc *d, int nd, int nmax, cudaStream_t s);
void launch_site(int dt, const SiteDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                 cudaStream_t s);
void launch_scalar(int dt, const ScalarDesc *d, cudaStream_t s);
void launch_fill(int dt, void *p, int64_t n, double value, cudaStream_t s);
void launch_permute(int dt, const PermuteDesc *d, const int64_t *prefix, int nd, int64_t blocks,
                    cudaStream_t s);
int64_t permute_blocks(const PermuteDesc &d);

int sandwich_smem_bytes(int dt, const SandwichDesc &d);
constexpr int kGemmBM = 64, kGemmBN = 64;
constexpr int kSketchPerBlock = 256 * 4;   // elements per sketch block
constexpr int kSiteThreads = 256;
// One column of an expectation strip: boundary site above ([a][(u,U)][b]),
// the row's ket site (the bra is the same tensor, conjugated) and boundary
// site below ([c][(x,X)][f]).
struct StripCol {
  const void *up, *lo, *ket;
  int32_t a, b, c, f;
  int32_t d, Dl, Du, Dx, De;
};
constexpr int kStripMaxCols = 32;
// One strip: columns col0..col0+ncol-1 of the column table, a one-site
// operator index per column (-1: identity; d x d entries of the operator
// table, accumulation type), FP64 scratch blocks, the scalar result.
struct StripDesc {
  int32_t col0, ncol;
  int32_t op[kStripMaxCols];
  void *scratch;
  int64_t l_cap, a1_cap, a2_cap, a3_cap;
  void *out;
};
void launch_strip(int dt, const StripDesc *d, const StripCol *cols, const void *ops, int nd, cudaStream_t s);

// ---- einsumsvd adjoint (real data) ----
struct SvdBwdDesc {
  const void *Mw;          // Jacobi output, n x n column-major, columns sigma_c u_c (unsorted)
  const double *sig;       // n refined singular values (unsorted)
  const void *Ut;          // n x k gauge-fixed kept vectors [j][c]
  const void *Utbar;       // n x k cotangent of Ut
  const void *WW;          // k x k: Wbar W^T
  const double *lbar;      // cotangent of log sigma_1
  const double *inv_s1;    // 1 / sigma_1
  void *H;                 // out: n x n
  double *scratch;         // 3 n^2 + n doubles, then n ints
  int32_t n, k;
};
struct TensorGradDesc {
  const void *Z2;          // [P][(l,L)][(u,U),b]
  const void *R;           // [P][N], N = (x,X,b,e,E)
  const void *K, *Kb;
  void *Kbar, *Kbbar;
  int32_t P, b, d, Dl, Du, Dx, De, DL, DU, DX, DE;
};
void launch_svd_bwd(int dt, const SvdBwdDesc &d, cudaStream_t s);
void launch_copyltu(int dt, const void *M, void *out, int n, cudaStream_t s);
void launch_tensor_grad(int dt, const TensorGradDesc &d, cudaStream_t s);
// ---- network-layer adjoint (real data) ----
struct StripBwdCol { void *cot_up, *cot_lo, *cot_ket; };   // NULL: no target
struct StripBwdScratch {
  double *base;
  int64_t per_strip, blk, big;
};
// Row-start sites: mode 0 = first row (K is [d][Dl][1][Dx][De]), mode 1 =
// first zip-up carry (K is [d][1][Du][Dx][De], S the boundary site [1][(u,U)][B]).
struct SiteBwdDesc {
  const void *K, *S, *cot;
  void *Kbar, *Sbar;
  int32_t mode, d, Dl, Du, Dx, De, B;
};
void launch_strip_bwd(int dt, const StripDesc *d, const StripCol *cols, const StripBwdCol *bcols, const double *ops,
                      const double *sbar, const StripBwdScratch &sc, int nd, cudaStream_t s);
void launch_site_bwd(int dt, const SiteBwdDesc &d, cudaStream_t s);
void launch_axpy(int dt, const void *x, void *y, int64_t n, cudaStream_t s);


}  // namespace peps
