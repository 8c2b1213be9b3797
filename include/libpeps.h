/*
 * libpeps -- C ABI of the GB300 implicit-randomized-SVD PEPS contraction.
 *
 * The library implements the einsumsvd primitive of arXiv:2006.15234
 * (Sec. II-C "einsumsvd"; Algorithm 4 "Randomized SVD" applied to an implicit
 * operator, Sec. IV-A) and the boundary-MPS contraction that drives it
 * (Algorithm 2 "Boundary MPS", Algorithm 3 zip-up "ApproxApply", two-layer
 * form of Sec. III-B).
 *
 * Conventions shared by every entry point
 *  - Tensor pointers are DEVICE pointers owned by the caller.  The library
 *    never allocates, frees or retains device memory: all scratch lives in a
 *    caller-provided workspace whose size a *_workspace / *_plan call reports.
 *  - Work is enqueued on the caller's stream (a cudaStream_t passed as void*);
 *    calls return once the work is enqueued unless stated otherwise.
 *  - Every call returns a peps_status.  Shapes, dtypes and pointers are checked
 *    on the host before anything is enqueued; on error nothing is enqueued and
 *    peps_last_error() (thread-local) describes the failure.  No C++ exception
 *    crosses the ABI.
 *  - Layouts are row-major.  PEPS site tensors are [d][left][up][down][right]
 *    (edge bonds have dimension 1).  Boundary-MPS sites are
 *    [left][vert][right] with vert = (ket, bra) pair, ket-major.
 *  - Complex data are interleaved (re, im) pairs of the real type.
 */
#ifndef LIBPEPS_H
#define LIBPEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t peps_status;
#define PEPS_OK               0
#define PEPS_ERR_ARG          1  /* NULL pointer, bad option value            */
#define PEPS_ERR_SHAPE        2  /* inconsistent tensor shapes                */
#define PEPS_ERR_UNSUPPORTED  3  /* valid request the library does not handle */
#define PEPS_ERR_CUDA         4  /* a CUDA runtime call failed                */
#define PEPS_ERR_WORKSPACE    5  /* workspace missing, misaligned or too small */
#define PEPS_ERR_NUMERIC      6  /* non-finite value met on the device        */
#define PEPS_ERR_TIMEOUT      7  /* a bounded device wait expired             */
#define PEPS_ERR_CAPTURE      8  /* call not allowed during stream capture    */

/* Name of a status code (static string). */
const char *peps_status_string(peps_status s);
/* Detail of the last error raised on this host thread ("" if none). */
const char *peps_last_error(void);
/* Library version string. */
const char *peps_version(void);

/* Element type of every tensor handed to one call. */
typedef enum {
  PEPS_R32 = 0,   /* float                          */
  PEPS_C64 = 1,   /* complex float  (float re, im)  */
  PEPS_R64 = 2,   /* double                         */
  PEPS_C128 = 3   /* complex double (double re, im) */
} peps_dtype;

/* Arithmetic of the implicit products (Algorithm 4's A Q and A^H P).
 * PLAIN: CUDA-core arithmetic in the data type.
 * MIXED: tensor-core (tcgen05 kind::tf32) contraction GEMMs, every product
 *        formed from TF32 head + tail splits (3xTF32: FP32-level products,
 *        FP32 accumulation); single-precision data whose contracted extents
 *        meet the TMA alignment rules, PLAIN otherwise.
 * FAST:  as MIXED, but the products before the last A Q of the power
 *        iteration use single TF32 products (faster; singular values move by
 *        up to ~1e-4 relative on flat spectra, the contracted scalar by
 *        ~1e-6 on the tested workloads). */
typedef enum { PEPS_PREC_PLAIN = 0, PEPS_PREC_MIXED = 1, PEPS_PREC_FAST = 2 } peps_precision;

/* Sketch distribution of Algorithm 4's first line: Gaussian (default) or the
 * paper's uniform draw on [-1, 1]. */
typedef enum { PEPS_SKETCH_GAUSS = 0, PEPS_SKETCH_UNIFORM = 1 } peps_sketch;

/* Options of one randomized SVD (Algorithm 4) / boundary sweep (Algorithm 2).
 *  m     truncation rank (boundary bond), >= 1
 *  p     oversampling: the sketch has l = min(k + p, M, N) columns, >= 0
 *  q     power iterations (Algorithm 4's loop count), >= 0
 *  seed  Philox4x64-10 key of every sketch and gauge vector
 *  sketch, prec  see the enums above
 *  flags PEPS_FLAG_ORTH_Q: in the MIXED / FAST paths, orthogonalise A^H P
 *        explicitly (Algorithm 4 literally; the default feeds it to the next
 *        product directly, which spans the same subspace)
 *        PEPS_FLAG_FP64_SMALL: single-precision data only (ignored for FP64
 *        data and by the gradient plans): every Cholesky factorisation of
 *        CholeskyQR2 (Algorithm 4's "orthogonalize", both sides) and the
 *        one-sided Jacobi SVD of R_B (Algorithm 4's "SVD") run in FP64 on the
 *        FP64-accumulated Grams, their outputs rounded once to the working
 *        precision; the default runs them in single precision (with R_B's
 *        factor in FP64 on the MIXED / FAST paths)
 *        PEPS_FLAG_ALTERNATE: contraction plans only (PEPS_ERR_UNSUPPORTED
 *        elsewhere): alternating canonicalisation of the zip-up (Sec. III-A):
 *        on the even rows 2, 4, ... of a sweep every einsumsvd puts its
 *        singular values into the finished boundary site (U = U~ Sigma /
 *        sigma_1, carry W = V^H) instead of the carry
 *        PEPS_FLAG_UNIT_BOND: TEBD plans only: every updated bond's singular
 *        values are divided by the largest before the split (M1 <- Q1 U
 *        sqrt(Sigma / sigma_1), ...), so each bond update applies its
 *        operator up to one positive factor and the state's scale stays
 *        bounded over many steps of imaginary-time evolution */
typedef struct {
  int32_t m, p, q;
  uint64_t seed;
  int32_t sketch;
  int32_t prec;
  uint32_t flags;
} peps_rsvd_opts;
#define PEPS_FLAG_ORTH_Q 1u
#define PEPS_FLAG_FP64_SMALL 2u
#define PEPS_FLAG_ALTERNATE 4u
#define PEPS_FLAG_UNIT_BOND 8u

/* ------------------------------------------------------------------------
 * Batched einsumsvd (Algorithm 3's einsumsvd line, Algorithm 4 inside).
 *
 * One instance factorises the implicit matrix
 *   A[(k,t),(x,X,b,e,E)] = sum V[k,t,a,(l,L)] S[a,(u,U),b] K[s,l,u,x,e] conj(Kb[s,L,U,X,E])
 * with operands
 *   V   carry           [kL][t][a][Dl*DL]
 *   S   boundary site   [a][Du*DU][b]
 *   K   ket site        [d][Dl][Du][Dx][De]
 *   Kb  bra site        [d][DL][DU][DX][DE]
 * M = kL*t rows, N = Dx*DX*b*De*DE columns, k = min(m, M, N).  Outputs:
 *   U      [kL][t][k]            left factor, orthonormal columns (new boundary site)
 *   W      [k][Dx*DX][b][De*DE]  Sigma V^H divided by sigma_1 (new carry)
 *   sigma  k doubles             singular values, descending (not divided)
 *   log_scale  one double        log(sigma_1) (written, not accumulated)
 * Directions with sigma_c <= 16 l eps64 sigma_1 are returned as zero columns
 * of U / rows of W.  The phase of each U column is fixed so that <g, u_c> is
 * real and >= 0 for a Philox vector g (stream tag 1), W compensating.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t kL, t, a, b;
  int32_t d, Dl, Du, Dx, De;   /* ket site dims */
  int32_t DL, DU, DX, DE;      /* bra site dims */
  int32_t m;                   /* this instance's truncation rank; 0: opts->m */
} peps_einsumsvd_shape;

typedef struct {
  const void *V, *S, *ket, *bra;
  void *U, *W;
  double *sigma;
  double *log_scale;
} peps_einsumsvd_io;

typedef struct peps_plan peps_plan;

/* Plan `batch` independent instances.  shapes and instance_ids are HOST
 * arrays of length batch; instance_ids (Philox stream id of each instance's
 * sketch) may be NULL, meaning 0..batch-1.  *workspace_bytes receives the
 * required workspace size (256-byte aligned base required). */
peps_status peps_einsumsvd_plan(peps_plan **out, peps_dtype dtype, int32_t batch,
                                const peps_einsumsvd_shape *shapes,
                                const uint64_t *instance_ids,
                                const peps_rsvd_opts *opts, size_t *workspace_bytes);

/* Number of side streams (1..64, default 16) over which a batched plan deals
 * its tensor-core instances (longest-processing-time-first on each
 * instance's product cost); each runs its chains one after another in one
 * shared scratch region, and a captured execute holds them as parallel graph
 * branches.  Host only: rebuilds the schedule and writes the new workspace
 * size (more branches, more scratch regions) to *workspace_bytes. */
peps_status peps_einsumsvd_set_branches(peps_plan *plan, int32_t branches, size_t *workspace_bytes);

/* Output rank k of instance i of a plan (host query). */
peps_status peps_einsumsvd_rank(const peps_plan *plan, int32_t i, int32_t *k);

/* Run the planned instances.  io is a HOST array of `batch` pointer sets.
 * The first call for a given (io, workspace) pair uploads the launch
 * descriptors into the workspace (stream-ordered copy); later calls with the
 * same pointers enqueue kernels only and may be captured in a CUDA graph. */
peps_status peps_einsumsvd_execute(peps_plan *plan, const peps_einsumsvd_io *io,
                                   void *workspace, size_t workspace_bytes,
                                   void *stream);

peps_status peps_plan_destroy(peps_plan *plan);

/* ------------------------------------------------------------------------
 * einsumsvd adjoint (reverse mode of Algorithm 4 with the sketch held
 * fixed; the paper has no gradient, this carries the method toward
 * variational optimisation).  Real data (PEPS_R32, PEPS_R64), CUDA-core
 * arithmetic, one instance per plan.
 *
 * Given cotangents of the step's outputs U, W and log_scale, returns those of
 * its operands V, S, ket and bra: the gradient of
 *     L = <U_bar, U> + <W_bar, W> + log_scale_bar * log(sigma_1).
 * The forward (executed again by the call) keeps the orthonormal bases of
 * the power iteration and the inverses of their R factors; the reverse sweep
 * runs the QR and SVD adjoints
 *     Ybar = (Qbar + Q copyltu(-Qbar^T Q)) R^-T,
 *     Bbar = U~ [(F o (U~^T Ubar - Ubar^T U~)) S + diag(sbar)] S^-1 U~^T B
 *            (+ the direct dependence of W on B),  F_ij = 1/(s_j^2 - s_i^2),
 * accumulates A's cotangent as a sum of rank-l outer products (one per
 * product of the forward) and contracts it into the four operands with the
 * same stage kernels as the forward products.  Valid where the kept
 * singular values are distinct and nonzero (the gradient of a truncated SVD
 * is otherwise undefined).
 * ------------------------------------------------------------------------ */
typedef struct {
  const void *U_bar;              /* [kL][t][k], may be NULL (zero) */
  const void *W_bar;              /* [k][Dx*DX][b][De*DE], may be NULL (zero) */
  const double *log_scale_bar;    /* one double, may be NULL (zero) */
} peps_einsumsvd_cotangent;

typedef struct {
  void *V_bar, *S_bar, *ket_bar, *bra_bar;   /* operand shapes; overwritten */
} peps_einsumsvd_grads;

/* Plan one instance with its adjoint (opts->prec must be PEPS_PREC_PLAIN). */
peps_status peps_einsumsvd_grad_plan(peps_plan **out, peps_dtype dtype, const peps_einsumsvd_shape *shape,
                                     const peps_rsvd_opts *opts, size_t *workspace_bytes);

/* Host only: record the cotangent and gradient pointers in the plan without
 * enqueueing anything (peps_plan_validate then checks the adjoint's launches
 * against them; peps_einsumsvd_grad_execute records them too). */
peps_status peps_einsumsvd_grad_bind(peps_plan *plan, const peps_einsumsvd_cotangent *ct,
                                     const peps_einsumsvd_grads *gr);

/* Forward (outputs in io as for peps_einsumsvd_execute) and reverse sweep
 * (cotangents in gr); all pointers DEVICE pointers.  Same descriptor-upload
 * rule as the execute calls (keyed on io, ct, gr and the workspace). */
peps_status peps_einsumsvd_grad_execute(peps_plan *plan, const peps_einsumsvd_io *io,
                                        const peps_einsumsvd_cotangent *ct, const peps_einsumsvd_grads *gr,
                                        void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Boundary-MPS contraction of a PEPS network (Algorithms 2 and 3).
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t nrow, ncol, d;
  int32_t dtype;                 /* peps_dtype */
  const int32_t *bond_h;         /* HOST [nrow][ncol-1]: bond right of (p,q)  */
  const int32_t *bond_v;         /* HOST [nrow-1][ncol]: bond below (p,q)     */
  const void *const *site;       /* HOST array of nrow*ncol DEVICE pointers,
                                    row-major, each [d][left][up][down][right] */
} peps_network;

/* Plan the contraction of <bra|ket> (bra != NULL: two-layer, the bra layer
 * enters conjugated; pass the ket again for the norm) or of the one-layer
 * network ket (bra == NULL, ket.d must be 1).  `direction` selects the sketch
 * streams (stream id of the step at row r, column c is
 * direction<<32 | r<<16 | c). */
peps_status peps_contract_plan(peps_plan **out, const peps_network *ket,
                               const peps_network *bra, const peps_rsvd_opts *opts,
                               int32_t direction, size_t *workspace_bytes);

/* Enqueue the planned sweep.  Results land in the workspace and are read by
 * peps_contract_result(); same descriptor-upload rule as einsumsvd_execute. */
peps_status peps_contract_execute(peps_plan *plan, void *workspace,
                                  size_t workspace_bytes, void *stream);

/* Synchronise `stream` and read the scalar as log|v| and arg v.  If sigma_out
 * is non-NULL it receives, for every einsumsvd step in sweep order, the
 * planned rank's singular values (peps_contract_sigma_count doubles). */
peps_status peps_contract_result(peps_plan *plan, void *workspace, void *stream,
                                 double *log_abs, double *phase, double *sigma_out);

/* Number of doubles peps_contract_result writes to sigma_out. */
peps_status peps_contract_sigma_count(const peps_plan *plan, int64_t *count);

/* One-shot convenience: plan, execute, read the result and destroy. */
peps_status peps_boundary_contract(const peps_network *ket, const peps_network *bra,
                                   const peps_rsvd_opts *opts, void *workspace,
                                   size_t workspace_bytes, void *stream,
                                   double *log_abs, double *phase);

/* Workspace size of peps_boundary_contract for these arguments. */
peps_status peps_boundary_workspace(const peps_network *ket, const peps_network *bra,
                                    const peps_rsvd_opts *opts, size_t *workspace_bytes);

/* ------------------------------------------------------------------------
 * Operator application by QR-SVD (Algorithm 1) and one TEBD layer.
 *
 * One-site operators (Eq. 4; optional) act on every site first.  Then a
 * two-site operator G (gate) acts on every nearest-neighbour bond of the
 * network, in place: two passes over the horizontal bonds (those starting at
 * even, then at odd columns), then two over the vertical ones (starting at
 * even, then odd rows); the bonds of one pass share no site and run as
 * grouped launches.  On each bond (sites M1, M2; Eq. 5):
 *   Q1, R1 <- QR(M1 as [(outer bonds)][(s, shared bond)]), Q2, R2 likewise
 *     (CholeskyQR2 with FP64-accumulated Grams; a site with no more outer
 *     entries than d * bond is used as its own R),
 *   Theta[(r1, i1)][(r2, i2)] = sum G[i1 i2, j1 j2] R1[r1, (j1, b)] R2[r2, (j2, b)],
 *   its SVD truncated back to the bond's current dimension (one-sided
 *   Jacobi in FP64), Sigma split evenly between the two factors,
 *   M1 <- Q1 U sqrt(Sigma), M2 <- Q2 (sqrt(Sigma) V^H)^T,
 *   each new bond direction's phase fixed on M1: column c of M1 as
 *   [(outer bonds, s)][c] has a real non-negative inner product with the
 *   Philox vector of stream (4 << 32) | (a << 16) | b (sites a < b row-major,
 *   tag 1, key opts->seed); M2 takes the opposite phase.
 * Bond dimensions are kept (each must not exceed d times the smaller QR
 * rank); Theta's sides are at most 64.
 * ------------------------------------------------------------------------ */

/* Plan one TEBD layer on `net` (one step of imaginary-time evolution,
 * Sec. II-D, when the operators are exp(-tau H_j)).
 *   gates: HOST array of ngates operators of (d^2) x (d^2) values, each
 *     row-major [out pair][in pair] with the first site's index most
 *     significant: doubles for real networks, interleaved (re, im) doubles
 *     for complex ones.  ngates = 1: that operator on every bond; otherwise
 *     ngates must equal the number of bonds, listed in bond order: every
 *     horizontal bond by its left site in row-major order, then every
 *     vertical bond by its upper site in row-major order.
 *   site_gates: HOST array of nsite_gates one-site operators of d x d
 *     values (row-major [out][in], same element rule), applied before the
 *     bonds; nsite_gates = 0 (site_gates may be NULL), 1 (every site) or
 *     nrow * ncol (row-major per site).
 * Both arrays are copied.  opts: seed (gauge vectors); prec must be
 * PEPS_PREC_PLAIN; flags 0 or PEPS_FLAG_UNIT_BOND; m, p, q are not used.
 * Errors: PEPS_ERR_ARG (NULL pointers, bad counts), PEPS_ERR_SHAPE (bond
 * dimensions the update cannot keep), PEPS_ERR_UNSUPPORTED (precision,
 * flags, Theta sides above 64, lattices above 65535 sites). */
peps_status peps_tebd_plan(peps_plan **out, const peps_network *net, const double *gates, int64_t ngates,
                           const double *site_gates, int64_t nsite_gates, const peps_rsvd_opts *opts,
                           size_t *workspace_bytes);

/* Enqueue the layer: the network's site tensors are overwritten with the
 * updated ones (same shapes).  Same descriptor-upload rule as the other
 * execute calls.  The layer has no result call: peps_poll reads its status
 * word (PEPS_STATUS_NONFINITE for a non-finite Theta or Gram,
 * PEPS_STATUS_JACOBI_NOCONV when a bond's SVD reached its sweep limit). */
peps_status peps_tebd_execute(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Expectation values <psi|H|psi> / <psi|psi> with cached environments
 * (Eq. 6; Sec. IV-B).  Two boundary sweeps (top-down, and bottom-up on the
 * row-reversed lattice) keep the boundary MPS above and below every row;
 * every local term is then one exact strip contraction (environment above,
 * the term's row with the operator applied to the ket, environment below),
 * normalised by the same strip without operator:
 *     E = sum_t coeff_t * Re( strip_t(O_t) / strip_t(1) ).
 * Terms on vertical bonds use the same procedure on the transposed lattice
 * (sketch streams 2 and 3; the direct lattice uses 0 and 1).  The bra is
 * the ket conjugated.
 * ------------------------------------------------------------------------ */

/* One term coeff * O of H.  nsite = 1: O acts on site[0]; nsite = 2: a
 * nearest-neighbour bond, either horizontal (site[1] = site[0] + 1, same
 * row) or vertical (site[1] = site[0] + ncol).  Sites are numbered
 * p * ncol + q.  op is a HOST array of (d^nsite) x (d^nsite) values,
 * row-major [out][in], site[0]'s index most significant; doubles for real
 * networks, interleaved (re, im) doubles for complex ones.  It is copied
 * when the plan is made. */
typedef struct {
  int32_t nsite;
  int32_t site[2];
  const double *op;
  double coeff;
} peps_term;

/* Plan the expectation value of H = sum_t terms[t] on the network ket
 * (d <= 4, at most 32 rows and columns).  use_cache = 1 keeps the two
 * sweeps' boundaries for every row (the caching of Sec. IV-B); use_cache = 0
 * recomputes the environments of each row that holds a term with fresh
 * sweeps (same sketches, hence the same values, at O(rows) times the cost).
 * PEPS_ERR_UNSUPPORTED for terms that are not on nearest-neighbour bonds. */
peps_status peps_expectation_plan(peps_plan **out, const peps_network *ket, const peps_term *terms,
                                  int32_t nterms, const peps_rsvd_opts *opts, int32_t use_cache,
                                  size_t *workspace_bytes);

/* Enqueue the planned sweeps and strips (same descriptor-upload rule as
 * peps_einsumsvd_execute). */
peps_status peps_expectation_execute(peps_plan *plan, void *workspace, size_t workspace_bytes,
                                     void *stream);

/* Two-GPU split of the cached expectation (Sec. IV-B runs one top-down and
 * one bottom-up boundary sweep per lattice; the two directions are
 * independent).  part 0 = the top-down sweeps (of the lattice and of its
 * transpose when vertical terms exist), part 1 = the bottom-up sweeps, part
 * 2 = the strips, which read both parts' environments.  Protocol for two
 * ranks holding identical plans (same network shapes, terms and options):
 * rank r enqueues part r, the ranks exchange their region (an all-gather of
 * the bytes at [offset, offset + bytes) of each rank's workspace into the
 * same offsets of the other's), then both enqueue part 2 and read the
 * result.  One rank may also run parts 0, 1, 2 in turn (the same values as
 * peps_expectation_execute).  Cached schedule of an expectation plan only
 * (PEPS_ERR_UNSUPPORTED otherwise); the region of a part is fixed by the
 * plan.  The part calls follow peps_expectation_execute's upload rule. */
peps_status peps_expectation_env_region(const peps_plan *plan, int32_t part, size_t *offset, size_t *bytes);
peps_status peps_expectation_execute_part(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream,
                                          int32_t part);

/* Synchronise `stream` and read the results: energy = sum of the terms'
 * contributions, log_norm = log <psi|psi> (row 0's strip and the scales of
 * the boundary below it), term_values[t] (nterms doubles, optional) =
 * coeff_t * <O_t>.  Any output pointer may be NULL. */
peps_status peps_expectation_result(peps_plan *plan, void *workspace, void *stream, double *energy,
                                    double *log_norm, double *term_values);

/* Energy gradient (hand-written reverse mode; the paper has no gradient):
 * E = <psi|H|psi>/<psi|psi> as computed by peps_expectation (cached
 * environments) and dE/d(site) for every site tensor of a REAL network
 * (PEPS_R32 / PEPS_R64, plain arithmetic, at least 2 x 2).  The rows of
 * Algorithm 2 are the checkpoints: the forward keeps the boundary after every
 * row of the four sweeps (the cached environments) and the einsumsvd steps'
 * saved bases of the last row only; the reverse sweep runs the strip
 * adjoints, then every sweep backwards row by row, first recomputing the
 * row's zip-up from the boundary above it with its steps' forward data kept
 * (one row's worth of step scratch, shared by all rows), then the einsumsvd
 * adjoint of peps_einsumsvd_grad_execute per step and the row-start site
 * adjoints; finally it maps the row-reversed and transposed lattices' site
 * cotangents back.  Sketches are held fixed (the gradient of the function
 * the forward computes). */
peps_status peps_grad_plan(peps_plan **out, const peps_network *ket, const peps_term *terms, int32_t nterms,
                           const peps_rsvd_opts *opts, size_t *workspace_bytes);

/* Run forward and reverse; grad_site is a HOST array of nrow*ncol DEVICE
 * pointers (site shapes, overwritten with dE/d(site)); *energy receives E.
 * Synchronises `stream` (the strip values are read back between the two
 * phases), so it cannot be captured. */
peps_status peps_grad_execute(peps_plan *plan, void *const *grad_site, void *workspace,
                              size_t workspace_bytes, void *stream, double *energy);

/* One-shot convenience: plan, execute, destroy. */
peps_status peps_grad(const peps_network *ket, const peps_term *terms, int32_t nterms,
                      const peps_rsvd_opts *opts, void *const *grad_site, void *workspace,
                      size_t workspace_bytes, void *stream, double *energy);

/* Workspace size of peps_expectation for these arguments. */
peps_status peps_expectation_workspace(const peps_network *ket, const peps_term *terms, int32_t nterms,
                                       const peps_rsvd_opts *opts, int32_t use_cache,
                                       size_t *workspace_bytes);

/* One-shot convenience: plan, execute, read energy and log-norm, destroy. */
peps_status peps_expectation(const peps_network *ket, const peps_term *terms, int32_t nterms,
                             const peps_rsvd_opts *opts, int32_t use_cache, void *workspace,
                             size_t workspace_bytes, void *stream, double *energy, double *log_norm);

/* ------------------------------------------------------------------------
 * Device status word.  Every plan keeps one 32-bit word at the start of its
 * workspace; the first launch of every execute clears it and the kernels
 * or in these bits (Algorithm 4's operations whose failure they report):
 *   PEPS_STATUS_NONFINITE     a non-finite largest singular value (the
 *                             small SVD of Algorithm 4 met NaN / Inf data)
 *   PEPS_STATUS_JACOBI_NOCONV the one-sided Jacobi SVD stopped at its sweep
 *                             limit (30) before converging
 *   PEPS_STATUS_TIMEOUT       a bounded wait of the tensor-core GEMM gave
 *                             up; that kernel left its output incomplete,
 *                             drained its own copies, freed its tensor
 *                             memory and returned
 * The synchronising result calls (peps_contract_result,
 * peps_expectation_result, peps_grad_execute) read the word too and return
 * PEPS_ERR_TIMEOUT or PEPS_ERR_NUMERIC for the first two error bits (their
 * outputs are written all the same, but are not meaningful).
 * ------------------------------------------------------------------------ */
#define PEPS_STATUS_NONFINITE     1u
#define PEPS_STATUS_JACOBI_NOCONV 2u
#define PEPS_STATUS_TIMEOUT       4u

/* Synchronise `stream`, read the status word of the plan's last execute in
 * `workspace` into *flags (may be NULL) and return PEPS_ERR_TIMEOUT if the
 * TIMEOUT bit is set, else PEPS_ERR_NUMERIC if the NONFINITE bit is set,
 * else PEPS_OK.  PEPS_ERR_ARG if the plan was never executed;
 * PEPS_ERR_CAPTURE on a capturing stream. */
peps_status peps_poll(const peps_plan *plan, const void *workspace, void *stream, uint32_t *flags);

/* Limit of one wait of the tensor-core GEMM's pipeline (TMA arrival, MMA
 * completion, operand preparation) in nanoseconds; 0 restores the default
 * of 2 s.  Applies to the plan's later executes.  A wait that gives up sets
 * PEPS_STATUS_TIMEOUT (see above).  Host only. */
peps_status peps_plan_set_wait_limit(peps_plan *plan, uint64_t ns);

/* ------------------------------------------------------------------------
 * Autotuning of the tensor-core GEMM tiles.  Every tensor-core launch of a
 * plan has a shape signature (operand types, products, rows of A and B,
 * contracted extent, K split); its MMA width (64, 128, 192 or, without the
 * FP32-level split, 256 accumulator columns) fixes the N tiling.  The default
 * is a rule (fewest padded columns); the autotuner times every candidate
 * width on one launch of each signature and keeps the fastest.
 * ------------------------------------------------------------------------ */

/* Tune the plan's tensor-core launches on this device: for each shape
 * signature, time `reps` launches (1..100) of one representative with every
 * candidate width (CUDA events on `stream`, synchronising) and set the
 * fastest on every launch of that signature.  The plan must have been
 * executed with `workspace` (the launches read and write it; its contents are
 * not meaningful afterwards, the next execute recomputes them).  Results are
 * unchanged by the tiling (each output is accumulated over K in the same
 * order).  Execute the plan once more before capturing it in a CUDA graph.
 * PEPS_ERR_ARG if the plan was not executed with this workspace,
 * PEPS_ERR_CAPTURE on a capturing stream. */
peps_status peps_plan_autotune(peps_plan *plan, void *workspace, size_t workspace_bytes, void *stream,
                               int32_t reps);

/* The plan's tuning table as text, one "<signature> = <width>" line per shape
 * (*len receives the size including the terminating NUL; buf may be NULL to
 * query it; at most cap bytes are written, NUL-terminated). */
peps_status peps_plan_tune_table(const peps_plan *plan, char *buf, size_t cap, size_t *len);

/* Replace the plan's tuning table (text as peps_plan_tune_table writes it; a
 * stored table applies to every plan with launches of the same signatures).
 * The next execute rebuilds the launches with it.  PEPS_ERR_ARG on a
 * malformed line or a width other than 64, 128, 192, 256. */
peps_status peps_plan_set_tune_table(peps_plan *plan, const char *table);

/* ------------------------------------------------------------------------
 * Launch ledger (profiling).  A plan's execute is a fixed list of grouped
 * kernel launches, each tagged with the stage of Algorithm 4 it serves
 * ("product_sites", "orth_m", "svd_jacobi", ...).
 * ------------------------------------------------------------------------ */

/* Number of kernel launches one execute of the plan enqueues. */
peps_status peps_plan_launch_count(const peps_plan *plan, int64_t *count);

/* Stage tag (static for the plan's lifetime), algorithmic flops and
 * algorithmic DRAM bytes of launch i (0 <= i < count). */
peps_status peps_plan_launch_info(const peps_plan *plan, int64_t i, const char **tag,
                                  double *flops, double *bytes);

/* CUDA kernel launches one execute of the plan enqueues (an entry of the
 * ledger may launch more than one kernel: the Cholesky entry a one-CTA and a
 * cluster kernel, the Jacobi entry a one-CTA kernel, the cluster kernels its
 * sizes need and the singular value refinement, the finalize entry the gauge
 * projections first, a tensor-core GEMM entry the pre-expansion of its B
 * operand first). */
peps_status peps_plan_kernel_launches(const peps_plan *plan, int64_t *count);

/* Kernel family of launch i (static string): "tc_gemm" (tcgen05 GEMM),
 * "gemm", "gemm_gram", "sandwich", "chol", "jacobi", "finalize", "sketch",
 * "permute", "site", "strip", "scalar", "zero", "fill". */
peps_status peps_plan_launch_kernel(const peps_plan *plan, int64_t i, const char **kernel);

/* Execute once more (same rules as the execute calls; the plan must have
 * been executed before) with a CUDA event after every launch, synchronise,
 * and write launch i's device time in milliseconds to ms[i]. */
peps_status peps_plan_profile(peps_plan *plan, void *workspace, size_t workspace_bytes,
                              void *stream, double *ms);

/* Host-only check of a plan against concrete buffers: rebuilds the launch
 * descriptors for `workspace` (and io, for einsumsvd plans; NULL otherwise)
 * and verifies that every byte range any kernel may touch lies inside the
 * workspace or a caller tensor of the planned shape.  Enqueues nothing and
 * does not dereference any pointer, so it runs without a GPU; returns
 * PEPS_ERR_ARG naming the first offending launch and field. */
peps_status peps_plan_validate(peps_plan *plan, void *workspace, size_t workspace_bytes,
                               const peps_einsumsvd_io *io);

/* Verification entry point of the tensor-core GEMM that carries the dense
 * contraction stages (tcgen05 kind::tf32, operands fed by TMA):
 *   C[m][n] = sum_k opA(A[m][k]) * opB(B[n][k]),  m < M, n < N, k < K
 * A (M x K), B (N x K) and C (M x N) are row-major DEVICE arrays of float
 * (cplx = 0) or interleaved complex float (cplx = 1); opA / opB conjugate
 * when conjA / conjB.  split3 selects the products: 0 plain TF32; 1
 * FP32-level products from TF32 head and tail parts (3xTF32), B expanded and
 * split inside the GEMM; 2 the same products with B expanded and split
 * beforehand into `scratch`, a DEVICE buffer of 32*N*K bytes (complex) or
 * 8*N*K bytes (real), caller-owned, used for no other mode (may be NULL
 * then).  Rows must be 16-byte aligned (K even for complex, K % 4 == 0 for
 * real).  Enqueued on `stream`; PEPS_ERR_ARG for a NULL operand or a missing
 * scratch, PEPS_ERR_UNSUPPORTED if TMA maps cannot be encoded. */
peps_status peps_debug_tc_gemm(int32_t cplx, int32_t conjA, int32_t conjB, int32_t split3, int32_t M,
                               int32_t N, int32_t K, const void *A, const void *B, void *C,
                               void *scratch, void *stream);

/* Verification entry point of the sketch generator (Algorithm 4's first
 * line): writes elements e = j*N + n (n < N, j < ell) of the (instance, tag)
 * Philox4x64-10 stream (counter (block, instance, tag, 0), key (seed, 0))
 * to X[j*N + n], as the einsumsvd plans draw Omega (tag 0) and the gauge
 * vector (tag 1).  kind PEPS_SKETCH_GAUSS: Box-Muller normals (complex:
 * (a + i b)/sqrt 2 per pair); PEPS_SKETCH_UNIFORM: 2u - 1 with the 53-bit
 * uniform u = ((x >> 11) + 1/2) 2^-53, rounded once to single precision for
 * PEPS_R32 / PEPS_C64.  X is a DEVICE array of N*ell elements of dtype;
 * desc_scratch a DEVICE buffer of at least 256 bytes (16-byte aligned) for
 * the launch descriptor.  Synchronises `stream` before it returns.
 * PEPS_ERR_ARG for NULL buffers or bad sizes, kinds or dtypes. */
peps_status peps_debug_sketch(int32_t dtype, int64_t N, int32_t ell, uint64_t seed, uint64_t instance, int32_t tag,
                              int32_t kind, void *X, void *desc_scratch, void *stream);

/* ------------------------------------------------------------------------
 * Contraction without any allocation.  The paper has no counterpart: this
 * is a service of this library for callers that cannot obtain device
 * memory themselves.  Examples: a plugin whose host application hands it
 * only the input and output buffers and keeps every allocator to itself;
 * a process whose device memory is already reserved by another framework's
 * caching allocator, so that a cudaMalloc would fail; a latency-bound loop
 * that cannot afford cudaMalloc/cudaFree, which synchronise the device.
 * ------------------------------------------------------------------------ */

/* Size of the library's fixed device scratch array (32 MiB).  Every GPU
 * on which the library is loaded holds one such array until the process
 * exits. */
#define PEPS_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

/* Same contraction and result as peps_boundary_contract, but the workspace
 * is the library's static device array instead of caller memory, and the
 * call allocates no device memory (no cudaMalloc, cudaFree or allocating
 * library routine).  The site tensors in ket / bra are device arrays as for
 * peps_contract_plan; log_abs and phase are host pointers (either may be
 * NULL).  On success the call has synchronised `stream` before it returns;
 * on an error it returns the status without waiting for work already
 * enqueued.
 *  - PEPS_ERR_WORKSPACE, before anything is enqueued, when the contraction
 *    needs more than PEPS_STATIC_SCRATCH_BYTES of workspace (the need is
 *    what peps_boundary_workspace reports; the message states both sizes).
 *    Such contractions must use peps_boundary_contract with caller memory.
 *  - Set-up: the first call on a device looks up the array's device
 *    address, with that device current, and keeps it for later calls in
 *    the same CUDA context (a new context, e.g. after a device reset, looks
 *    it up again).  Make that first call before any stream capture begins.
 *  - Sharing: every call on a device uses the same array, which keeps what
 *    the previous call left in it.  Each call clears the bytes it uses
 *    before its kernels run.  Calls whose work can overlap on the GPU
 *    (different streams, or host threads with no ordering between their
 *    calls) race on the array and give wrong results: serialise them. */
peps_status peps_boundary_contract_static(const peps_network *ket, const peps_network *bra,
                                          const peps_rsvd_opts *opts, void *stream,
                                          double *log_abs, double *phase);

#ifdef __cplusplus
}
#endif
#endif /* LIBPEPS_H */
