/* strom.h — C ABI of the GB300-native STROM solver (sparse moment relaxation +
 * sGS-ADMM) of "Fast and Certifiable Trajectory Optimization" (Kang et al.).
 *
 * Conventions
 *   - Every call returns an int status (STROM_OK = 0, negative = error); the
 *     message of the last error on the calling thread is strom_last_error().
 *   - Opaque handles are created by *_create and freed by *_destroy; the
 *     caller owns them. Input arrays are borrowed for the duration of the call
 *     and copied; output arrays are caller-allocated with sizes from *_info.
 *   - Pointers named *_dev are CUDA device pointers on the current device;
 *     all other pointers are host pointers. `stream` is a cudaStream_t passed
 *     as void* (NULL = legacy default stream).
 *   - svec is the SDPT3 vectorisation: column-major upper triangle, off-diagonal
 *     entries multiplied by sqrt(2), so <A, B> = svec(A) . svec(B) (Sec. 4).
 *   - No C++ exception crosses this interface.
 */
#ifndef STROM_H
#define STROM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STROM_OK = 0,
  STROM_MAXITER = 1,          /* results valid, tolerance not reached */
  STROM_PENDING = 2,          /* a served request has not finished yet */
  STROM_ERR_INVALID = -1,     /* bad argument or malformed problem */
  STROM_ERR_OOM = -2,         /* device or host allocation failed */
  STROM_ERR_NOT_PD = -3,      /* A A^T not positive definite after row reduction */
  STROM_ERR_NUMERICAL = -4,   /* NaN / Inf met */
  STROM_ERR_TIMEOUT = -5,     /* time budget exhausted */
  STROM_ERR_CUDA = -6         /* a CUDA runtime call failed */
};

/* factorisations of the y-solve's Schur complement (strom_options.factor).
 * DENSE: one dense lower triangle per clique and a dense coupling block
 * (blocked substitution through inverted 32 x 32 diagonal blocks); SPARSE:
 * the sparse Cholesky factor of strom_sdp_factor_info (substitution in
 * blocks of 32 positions). Both take the same pivot decisions in the same
 * order and give the same y up to rounding. AUTO: DENSE when every clique
 * group has at most 800 rows and the dense factor takes at most a quarter
 * of the device's free memory at creation, else SPARSE. */
enum { STROM_FACTOR_AUTO = 0, STROM_FACTOR_DENSE = 1, STROM_FACTOR_SPARSE = 2 };

/* precision modes of the PSD projection */
enum {
  STROM_PREC_FP64 = 0,        /* Jacobi eigensolver in FP64 (plain) */
  STROM_PREC_FP32 = 1,        /* Jacobi eigensolver in FP32 */
  STROM_PREC_MIXED = 2        /* FP32 Jacobi, FP64 polish once eta <= polish_eta */
};

const char* strom_last_error(void);
const char* strom_version(void);

/* ------------------------------------------------------------------------
 * Problem: a polynomial optimization problem with chain-like sparsity
 * (Definition 1, eq. chain-sparse-pop) describing a trajectory problem
 * (eq. intro:trajopt). Clique k (0-based, k < N) has the n_v = 2 dx + du
 * variables z(I_k) = (x_{k-1}, u_{k-1}, x_k) (Sec. 2.1); consecutive cliques
 * overlap in x_k. Polynomials use clique-local exponents.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t nterms;
  const double* coef;        /* [nterms] */
  const uint8_t* expo;       /* [nterms * n_v], row-major: term t has expo[t*n_v + i] */
} strom_poly;

typedef struct {
  strom_poly f;              /* objective term f_k */
  int32_t ng;                /* inequalities g_{k,i} >= 0, degree 1 or 2 (Sec. 4 assumption iii) */
  const strom_poly* g;
  int32_t nh;                /* equalities h_{k,j} = 0, degree <= 2 kappa */
  const strom_poly* h;
} strom_clique;

typedef struct {
  int32_t N, dx, du;
  int32_t kappa;             /* relaxation order; must be 2 (Sec. 4 assumption i) */
  double R;                  /* bound |z_i| <= R on every variable (Theorem 1) */
  const strom_clique* cliques;   /* [N] */
} strom_problem_desc;

typedef struct strom_problem strom_problem;

/* Copies the description. Errors: INVALID (kappa != 2, a degree out of range,
 * an exponent tuple of the wrong length, N < 1, more than 21 variables per
 * clique). The relaxation builder takes cliques of up to 21 variables; the
 * solver takes blocks of up to 160 rows, i.e. cliques of up to 16 variables
 * (strom_solver_create refuses larger blocks). */
int strom_problem_create(const strom_problem_desc* desc, strom_problem** out);
void strom_problem_destroy(strom_problem* p);

/* ------------------------------------------------------------------------
 * Relaxation: the order-2 sparse moment relaxation (Prop. 1) written as the
 * PSD-only standard SDP  min <C,X> s.t. A(X) = b, X in Omega_+
 * (eq. standardsdp, Sec. 2.3). Blocks are ordered M_1, L_{1,1..}, M_2, ...;
 * rows are ordered by clique and inside a clique as A_mom, A_ineq, A_eq, the
 * phi_0 = 1 row, then the consensus rows A_sen with clique k+1. A monomial
 * of M_k is represented by its first occurrence in column-major upper order.
 * ---------------------------------------------------------------------- */
typedef struct strom_sdp strom_sdp;

typedef struct {
  int32_t N, nv, nblocks;
  int64_t nsvec;             /* length of svec(X) */
  int64_t m;                 /* rows of A (before row reduction) */
  int64_t nnz;               /* nonzeros of A */
  int64_t rows_by_kind[5];   /* A_mom, A_ineq, A_eq, phi_0, A_sen */
} strom_sdp_info;

enum { STROM_ROW_MOM = 0, STROM_ROW_INEQ = 1, STROM_ROW_EQ = 2, STROM_ROW_PHI0 = 3, STROM_ROW_CONS = 4 };

int strom_relax(const strom_problem* p, strom_sdp** out);
int strom_sdp_info_get(const strom_sdp* s, strom_sdp_info* info);
/* Any output pointer may be NULL to skip it. Sizes: block_* [nblocks],
 * C [nsvec], rowptr [m+1], col/val [nnz] (CSR, columns sorted), b/row_kind/
 * row_clique [m]. block_kind: 0 = moment, 1 = localizing. */
int strom_sdp_export(const strom_sdp* s, int32_t* block_n, int64_t* block_off, int8_t* block_kind,
                     int32_t* block_clique, double* C, int64_t* rowptr, int32_t* col, double* val,
                     double* b, int8_t* row_kind, int32_t* row_clique);
void strom_sdp_destroy(strom_sdp* s);

/* An SDP given by arrays in the layout strom_sdp_export writes, e.g. the
 * relaxation of Sec. 2.3 built by another implementation. Blocks are ordered
 * by clique, each clique led by its moment block of size s(2 dx + du, 2);
 * svec offsets are the running sums of n (n + 1) / 2. Rows are ordered by
 * clique; every row stays inside its clique's blocks except consensus rows,
 * which may also reach the next clique's moment block (the chain structure
 * of Definition 1); inside a clique the consensus rows come after every row
 * other than A_mom rows. Each A_mom row is s_p X_p - s_r X_r = 0 with b = 0,
 * the representative r first (column order) and s = 1 on the diagonal,
 * 1/sqrt(2) off it (svec scaling), and no entry is the duplicate of two rows.
 * The data of the y-solve's star elimination and clique groups are derived
 * from these rows. Arrays are copied. Errors: INVALID (with the first rule
 * broken in strom_last_error), OOM. */
typedef struct {
  int32_t N, dx, du;                /* horizon, state and control sizes: clique vars (x_{k-1}, u_{k-1}, x_k) */
  int32_t nblocks;
  const int32_t* block_n;           /* [nblocks] sizes 1..160 */
  const int8_t* block_kind;         /* [nblocks] 0 = moment, 1 = localizing */
  const int32_t* block_clique;      /* [nblocks] */
  const int32_t* block_index;       /* [nblocks] localizing constraint index in its clique, -1 for moment;
                                       NULL: localizing blocks are numbered in order */
  const double* C;                  /* [nsvec] */
  int64_t m;                        /* rows */
  const int64_t* rowptr;            /* [m + 1] CSR, rowptr[0] = 0 */
  const int32_t* col;               /* [nnz] strictly increasing inside a row */
  const double* val;                /* [nnz] */
  const double* b;                  /* [m] */
  const int8_t* row_kind;           /* [m] STROM_ROW_* */
  const int32_t* row_clique;        /* [m] */
} strom_sdp_desc;
int strom_sdp_import(const strom_sdp_desc* d, strom_sdp** out);

/* The star elimination the y-solve applies to the A_mom rows (each ties a
 * duplicate entry p of a moment matrix to the representative r of its
 * monomial): one class per representative with duplicates, cliques in
 * order and inside a clique in order of the class's first A_mom row. Per
 * class: rep (svec position), c = s_r^2, dsum = sum of 1/s_p^2 over its
 * rows, ptr [nclass + 1] into row / inv_s2 (its A_mom rows and their
 * 1/s_p^2). omega [nsvec]: weights of the Gram A_o diag(omega) A_o^T of the
 * other rows (1 / (occurrences s_r^2) at representatives, 0 at duplicates,
 * 1 on localizing blocks); inv_rep_s [nsvec]: 1/s_r at representatives of
 * moment blocks, else 0. *nclass, *nstar receive the sizes (call once with
 * NULL arrays to size them); any pointer may be NULL. */
int strom_sdp_star_export(const strom_sdp* s, int64_t* nclass, int64_t* nstar, int64_t* rep, double* c,
                          double* dsum, int32_t* ptr, int64_t* row, double* inv_s2, double* omega,
                          double* inv_rep_s);

/* Size of the sparse factor the y-solve uses for this SDP (host only, no GPU
 * needed). After the exact star elimination of the A_mom rows, the y-solve
 * factorises the Gram S of the other rows (eq. cholesky on the reduced
 * system) in the canonical order of the row reduction (cliques N..1, natural
 * order inside a clique), where S is block tridiagonal by clique and its
 * Cholesky factor L is block bidiagonal. Reported: the other rows (n_other;
 * the last group, the first clique's, starts at n_tail), the strictly lower
 * entries of S and of L (pattern without pivoting; dropped rows keep their
 * zero entries), the dependent steps of the forward and backward solves
 * (level schedules inside each clique's group, summed over groups), the
 * largest group, the longest column of L, the largest row distance inside
 * a column, and the entries of dense lower triangles of the groups (the
 * storage a dense per-clique factor would need). Errors: INVALID when the
 * rows are not chain-ordered. */
typedef struct {
  int64_t n_other, n_tail, nnz_S, nnz_L, dense_entries;
  int32_t levels_fwd, levels_bwd, max_group, max_col, max_span;
} strom_factor_info;
int strom_sdp_factor_info(const strom_sdp* s, strom_factor_info* out);

/* ------------------------------------------------------------------------
 * Solver: sGS-ADMM (Algorithm 1) on a batch of independent SDPs, all on the
 * current CUDA device. Creation uploads the data, removes linearly dependent
 * rows (pivot-skipping Cholesky of A A^T in the order cliques N..1, natural
 * row order inside a clique; a row is dropped when its pivot is at most
 * rank_tol times its squared norm) and factorises A A^T once (Sec. 4, hybrid
 * linear system solver; here entirely on the GPU).
 * ---------------------------------------------------------------------- */
typedef struct {
  double tol;                /* stop when max(eta_p, eta_d, eta_g) <= tol (eq. kkt-residual) */
  int32_t maxiter;
  double sigma0, tau;        /* Algorithm 1 inputs: sigma > 0, tau in (0, 2) */
  int32_t sigma_every;       /* sigma update cadence (iterations) */
  double sigma_ratio, sigma_factor, sigma_min, sigma_max;
  double rank_tol;           /* relative pivot threshold of the row reduction */
  int32_t precision;         /* STROM_PREC_* */
  double polish_eta;         /* MIXED: switch to the FP64 eigensolver once eta <= polish_eta; an
                                instance meeting tol in FP32 switches too, and it retires only
                                on an FP64 iterate with eta <= tol. It also switches when its
                                FP32 phase stalls: at eta <= 1e-4, less than 5 % progress over
                                200 iterations (the FP32 eigensolver's rounding can hold eta
                                above polish_eta) */
  int32_t check_every;       /* host checks for completion every this many iterations */
  double time_budget_s;      /* strom_solve only: wall-clock budget in seconds, checked every
                                check_every iterations; when spent, strom_solve returns
                                STROM_ERR_TIMEOUT with the state and results of the last
                                iteration run (valid, like MAXITER). <= 0: none */
  int32_t eig_warm_period;   /* FP32 eigensolver: start each block's sweeps from its eigenvectors of
                                the previous iteration, restarting cold every this many iterations
                                (0 = always cold); blocks of size <= 80 */
  int32_t share_tail;        /* 1: when every instance has the same constraint rows after the first
                                clique (e.g. one robot, different initial states), the factor of
                                cliques 2..N is computed once and shared (cliques are eliminated
                                N..1, so only the first clique's factor differs) */
  int32_t factor;            /* STROM_FACTOR_*: how A A^T is factorised for the y-solve */
  int32_t eig_reorth;        /* 1: a warm-started FP32 eigensolve of a block of 41..80 rows first
                                takes one Newton-Schulz step, V <- (3 V - V V^T V) / 2, towards
                                orthonormal stored eigenvectors (they drift in FP32 from one
                                iteration to the next); 0 (default): none */
} strom_options;

void strom_options_default(strom_options* o);

typedef struct strom_solver strom_solver;

typedef struct {
  int32_t status;            /* STROM_OK, STROM_MAXITER or an error */
  int32_t iterations;
  double pobj, dobj;         /* <C, X>, <b, y> */
  double eta_p, eta_d, eta_g;
  double sigma;
  int64_t m_kept;            /* rows kept by the row reduction */
} strom_result;

/* sdps: [count] relaxations (each may be different). Errors: INVALID, OOM,
 * NOT_PD (a pivot of a kept row became non-positive), CUDA. */
int strom_solver_create(const strom_sdp* const* sdps, int32_t count, const strom_options* opt,
                        strom_solver** out);
void strom_solver_destroy(strom_solver* s);
/* The factorisation the solver chose (STROM_FACTOR_DENSE or _SPARSE; -1 for
 * a NULL solver). */
int32_t strom_solver_factor_kind(const strom_solver* s);
int32_t strom_solver_count(const strom_solver* s);

/* Recomputes the row reduction and the factorisation of A A^T from the data
 * already on the device and resets every instance to X = S = y = 0,
 * sigma = sigma0 (the setup of Sec. 4, repeated; used to time a whole solve
 * with inputs resident in HBM). */
int strom_solver_factor(strom_solver* s, void* stream);

/* Runs Algorithm 1 until every instance meets tol or maxiter. Returns
 * STROM_OK when all converged, STROM_MAXITER otherwise, STROM_ERR_TIMEOUT
 * when opt.time_budget_s ran out first, STROM_ERR_NUMERICAL when an
 * instance met NaN / Inf. */
int strom_solve(strom_solver* s, void* stream);
/* Runs at most `iters` more iterations (instances that already met tol stay
 * frozen). *n_active receives the number of unconverged instances. */
int strom_solver_step(strom_solver* s, int32_t iters, void* stream, int32_t* n_active);
/* Resets instance i to (X, S, y, sigma) = (X0, S0, 0, sigma) (warm start,
 * Algorithm 1 input); NULL X0/S0 mean zero, sigma <= 0 means opt.sigma0. */
int strom_solver_reset(strom_solver* s, int32_t i, const double* X0, const double* S0, double sigma);

int strom_get_result(const strom_solver* s, int32_t i, strom_result* r);
/* Host copies of the state of instance i: X, S [nsvec], y [m] (dropped rows
 * hold 0). Any pointer may be NULL. */
int strom_get_state(const strom_solver* s, int32_t i, double* X, double* S, double* y);
/* Moment matrix M_k of instance i as a dense column-major n x n matrix. */
int strom_get_moment(const strom_solver* s, int32_t i, int32_t k, double* Mk);
/* Row keep-mask of instance i after the row reduction [m]. */
int strom_get_kept_rows(const strom_solver* s, int32_t i, uint8_t* keep);

/* ------------------------------------------------------------------------
 * Certificate (end of solve): rank-1 test of every M_k (Theorem 1 iii),
 * extraction of z_bar from the top eigenvectors (Sec. 2.2), a rollout that
 * clips the controls to [-R, R] and solves each clique's equalities for its
 * new state by Gauss-Newton (stands in for the paper's local solver), the
 * valid lower bound <b,y> + sum_beta R_beta min(0, lambda_min((C - A^T y)_beta))
 * (eq. valid-lowerbound, R_beta of App. C) and xi (eq. suboptimality-gap).
 * Eigenvalues are computed on the GPU in FP64.
 * ---------------------------------------------------------------------- */
typedef struct {
  double max_ratio;          /* max_k lambda_2 / lambda_1 of M_k */
  double lower_bound;
  double phat;               /* objective at the rolled-out point */
  double xi;
  double hmax, gmin;         /* max |h|, min g at the rolled-out point */
  int32_t feasible, rank_one, certified;
} strom_certificate;

/* zbar, zhat: optional host outputs of length N (dx + du) + dx. */
int strom_certify(strom_solver* s, int32_t i, const strom_problem* p, double rank_tol, double xi_tol,
                  strom_certificate* out, double* zbar, double* zhat);

/* The host half of the certificate, from eigen data computed elsewhere (no
 * GPU involved): the same extraction, rollout, lower bound and verdict as
 * strom_certify, given for one instance of problem p its nblocks blocks in
 * the builder's order (M_1, L_{1,*}, M_2, ...: block_n, block_kind 0 = moment
 * / 1 = localizing, block_clique 0-based), and, packed block after block at
 * offsets sum of previous block_n:
 *   lamX  eigenvalues of each block of X, ascending;
 *   topX  the eigenvector of each block's largest eigenvalue (any sign);
 *   lamZ  eigenvalues of each block of Z = C - A^T y, ascending;
 *   by    <b, y>.
 * Errors: INVALID when the block list does not match the problem (one
 * moment block of size (nv + 1)(nv + 2) / 2 per clique, as many localizing
 * blocks per clique as it has inequalities). */
int strom_certify_host(const strom_problem* p, int32_t nblocks, const int32_t* block_n, const int8_t* block_kind,
                       const int32_t* block_clique, const double* lamX, const double* topX, const double* lamZ,
                       double by, double rank_tol, double xi_tol, strom_certificate* out, double* zbar,
                       double* zhat);

/* The certificate of every instance of the solver; problems[i] describes
 * instance i. out: [count]. Eigenvalues of all blocks are computed in two
 * batched GPU launches; the rollout and bound run on the host. */
int strom_certify_batch(strom_solver* s, const strom_problem* const* problems, double rank_tol, double xi_tol,
                        strom_certificate* out);

/* Bookkeeping (no counterpart in the paper): number of CUDA kernels libstrom
 * has launched in this process (a graph launch counts each of its kernel
 * nodes). */
uint64_t strom_launch_count(void);
/* Bytes libstrom has copied host->device and device->host in this process. */
void strom_transfer_bytes(uint64_t* h2d, uint64_t* d2h);

/* ------------------------------------------------------------------------
 * Rank tests of one moment matrix beyond the rank-1 test (host only).
 * M: the n x n moment matrix of order 2 in nv clique variables (basis [z]_2
 * in graded lexicographic order, n = (nv + 1)(nv + 2) / 2), column-major,
 * e.g. from strom_get_moment. Numerical ranks count eigenvalues above
 * tol * lambda_max.
 *   rank, rank_low: of M and of its principal submatrix on [z]_1 (degree
 *     <= 1); flat = (rank == rank_low), the flat-extension condition that
 *     generalises rank 1 (Sec. 2.2): the moments then come from a measure
 *     with exactly `rank` atoms.
 *   ratio_sub: lambda_2 / lambda_1 of the principal submatrix on the
 *     monomials of the variables selected by vars (nv flags; NULL = all),
 *     the partial rank-1 test of the car back-in experiment, whose auxiliary
 *     variables keep M_k above rank 1 while the trajectory's submatrix is
 *     rank 1; zbar (nullable, [nv]) receives the degree-1 entries of that
 *     submatrix's top eigenvector scaled to a leading 1 (NaN for variables
 *     not selected).
 * nv in 1..21 (the cliques the builder takes). Errors: INVALID (bad sizes,
 * non-finite or non-symmetric M). */
typedef struct {
  int32_t n, rank, rank_low, flat, n_sub;
  double ratio_sub, lambda_max;
} strom_rank_test;
int strom_moment_rank_test(const double* M, int32_t nv, const uint8_t* vars, double tol, strom_rank_test* out,
                           double* zbar);

/* ------------------------------------------------------------------------
 * Serving by continuous batching. A batch owns `slots` solver slots for
 * SDPs with the structure of `tmpl` (same horizon, blocks, rows and sparsity
 * pattern; values of A, b and C may differ, as they do between initial
 * states). Submitted requests wait in a FIFO queue until a slot is free.
 * Each step admits queued requests into free slots (upload, row reduction
 * and factorisation of just those slots), runs `iters` iterations of
 * Algorithm 1 on every occupied slot, and retires the requests that met tol
 * or maxiter: their result and, when a problem was given, their certificate
 * are stored and the slot is reused at once. No slot waits for another, and
 * a request's arithmetic does not depend on what shares the batch with it.
 * Each slot runs Algorithm 1 with the certificate of Sec. 2.2 / eq.
 * (suboptimality-gap); the serving loop itself has no counterpart in the
 * paper, whose nearest use is the MPC loop of Sec. 5 (one warm-started solve
 * per control step).
 * ---------------------------------------------------------------------- */
typedef struct strom_batch strom_batch;

int strom_batch_create(const strom_sdp* tmpl, int32_t slots, const strom_options* opt, strom_batch** out);
/* Device bytes of a batch of this structure and options, measured on the
 * current device by building solvers of one and two slots (their set-up
 * included): *base_bytes once per batch, *slot_bytes per slot, and
 * *transient_bytes of scratch that the set-up holds for a moment. Either of
 * base_bytes / transient_bytes may be NULL. Admission by memory footprint
 * (serving by an HBM budget) has no counterpart in the paper. */
int strom_batch_slot_bytes(const strom_sdp* tmpl, const strom_options* opt, int64_t* base_bytes,
                           int64_t* slot_bytes, int64_t* transient_bytes);
/* A batch sized by a device-memory budget: as many slots as
 * base + transient + slots x slot_bytes <= budget_bytes allows
 * (strom_batch_slot_bytes); *slots_out (nullable) receives the count.
 * Requests beyond the slots wait in the batch's queue (host memory).
 * Errors: OOM when budget_bytes exceeds the device's free memory (nothing is
 * allocated then), INVALID when the budget holds less than one slot. */
int strom_batch_create_budget(const strom_sdp* tmpl, int64_t budget_bytes, const strom_options* opt,
                              strom_batch** out, int32_t* slots_out);
void strom_batch_destroy(strom_batch* b);
/* Copies the request. problem (nullable): certify the result on completion.
 * X0, S0 (nullable, length nsvec): warm start of Algorithm 1.
 * Errors: INVALID when the SDP's structure differs from the template. */
int strom_batch_submit(strom_batch* b, const strom_sdp* sdp, const strom_problem* problem, const double* X0,
                       const double* S0, uint64_t* ticket);
int strom_batch_step(strom_batch* b, int32_t iters, void* stream, int32_t* n_running, int32_t* n_queued);
/* STROM_OK once the request finished (outputs filled; c only if a problem
 * was given), STROM_PENDING before. latency_s: submit to retirement;
 * service_s: admission into a slot to retirement. Any output may be NULL.
 * A finished request's result (about 200 bytes) stays readable, and held,
 * until the batch is destroyed. */
int strom_batch_poll(strom_batch* b, uint64_t ticket, strom_result* r, strom_certificate* c, double* latency_s,
                     double* service_s);
/* ------------------------------------------------------------------------
 * Serving several structures (robots, horizons) behind one front within one
 * device-memory budget. The server routes each request to a class: the
 * structure of the first request of its kind and, when opt->share_tail is
 * set, that request's constraint values after the first clique; requests of
 * a known structure whose later constraints differ (other obstacles) go to
 * a second class of that structure without a shared tail factor. Each class
 * gets a strom_batch on the first step after its first request, with
 * min(max_slots, what the remaining budget holds) slots
 * (strom_batch_slot_bytes). When no slot fits, idle batches of other
 * classes are destroyed to make room (their results stay readable). A step
 * runs every batch with work for `iters` iterations, each from its own host
 * thread and stream, so different structures overlap on the device; each
 * request's arithmetic is the same as solving it alone. Inputs are copied at
 * submit. Latency counts the wait for a batch. A request whose structure
 * needs more than the whole budget for one slot finishes at the next step
 * with result status STROM_ERR_OOM. The paper has no
 * counterpart (its nearest use is the warm-started MPC loop of Sec. 5).
 * Errors: strom_server_create returns OOM (allocating nothing) when
 * budget_bytes exceeds the device's free memory.
 * ---------------------------------------------------------------------- */
typedef struct strom_server strom_server;
typedef struct {
  int32_t N;                 /* horizon of the class's structure */
  int32_t shared_tail;       /* its batch shares the factor of cliques 2..N */
  int64_t nsvec, m;
  int32_t slots;             /* slots of its current batch (0: none) */
  int32_t running, queued;   /* requests in the batch's slots / queue */
  int32_t waiting;           /* requests waiting for a batch */
  int32_t batches_created;
  int32_t pad;
  int64_t slot_bytes, reserved_bytes;
} strom_server_class;
int strom_server_create(int64_t budget_bytes, int32_t max_slots, const strom_options* opt, strom_server** out);
void strom_server_destroy(strom_server* s);
int strom_server_submit(strom_server* s, const strom_sdp* sdp, const strom_problem* problem, uint64_t* ticket);
/* *n_running: requests in batches (slots and batch queues); *n_waiting:
 * requests whose class has no batch yet. */
int strom_server_step(strom_server* s, int32_t iters, void* stream, int32_t* n_running, int32_t* n_waiting);
/* As strom_batch_poll. */
int strom_server_poll(strom_server* s, uint64_t ticket, strom_result* r, strom_certificate* c, double* latency_s,
                      double* service_s);
/* The first min(cap, classes) classes into out; *nclass = classes;
 * *used_bytes = budget bytes reserved by the current batches. */
int strom_server_info(const strom_server* s, int32_t cap, strom_server_class* out, int32_t* nclass,
                      int64_t* used_bytes);

/* ------------------------------------------------------------------------
 * Data-driven warm starts (Sec. 5, inverted pendulum initialised by a
 * nearest-neighbour search over stored solutions). A store holds solved
 * states (X, S, sigma) of one SDP structure in device memory (capacity x 2 x
 * nsvec doubles), each under a key of key_dim doubles: the parameters that
 * tell instances apart (e.g. the initial state), scaled by the caller so
 * that Euclidean distance compares them. A new instance starts from a convex
 * combination of stored states, chosen as follows. The stored keys are
 * ranked by distance to the new key (ties: lower index first) and the first
 * min(key_dim + 1, count) are the neighbours. A key equal to a stored key
 * takes that state alone. When there are key_dim + 1 neighbours, their keys
 * span a non-degenerate simplex and the new key lies in it (barycentric
 * coordinates >= -1e-12), the weights are those barycentric coordinates
 * (clipped at 0, renormalised): for keys on a grid and key_dim = 2 this is
 * the triangle of a Delaunay triangulation. Otherwise the weights are
 * proportional to 1 / distance. X0 = sum_j w_j X_j, S0 = sum_j w_j S_j,
 * y = 0, and sigma0 = prod_j sigma_j^{w_j}.
 * ---------------------------------------------------------------------- */
#define STROM_WARM_MAX_KEY 8
typedef struct strom_warm strom_warm;

/* The neighbour selection alone, on a host table keys [n x key_dim]
 * (row-major): idx, wt have room for key_dim + 1 entries; *k receives the
 * number used (0 when n = 0). Host only; no GPU needed. */
int strom_warm_select(const double* keys, int32_t n, int32_t key_dim, const double* key, int32_t* idx, double* wt,
                      int32_t* k);
/* key_dim 1..STROM_WARM_MAX_KEY, nsvec >= 1, capacity >= 1; allocates the
 * device store on the current device. Errors: INVALID, OOM, CUDA. */
int strom_warm_create(int32_t key_dim, int64_t nsvec, int32_t capacity, strom_warm** out);
void strom_warm_destroy(strom_warm* w);
/* Entries stored (-1 for a NULL store). */
int32_t strom_warm_count(const strom_warm* w);
/* Adds a state from host arrays X, S [nsvec] with sigma > 0; *index
 * (nullable) receives its index. INVALID when the store is full. */
int strom_warm_add(strom_warm* w, const double* key, const double* X, const double* S, double sigma, int32_t* index);
/* Adds the current (X, S, sigma) of instance i of a solver by device copies.
 * INVALID when the store is full or the instance's svec length differs. */
int strom_warm_add_from_solver(strom_warm* w, const strom_solver* s, int32_t i, const double* key, int32_t* index);
/* strom_warm_select over the stored keys. */
int strom_warm_query(const strom_warm* w, const double* key, int32_t* idx, double* wt, int32_t* k);
/* Host copies of entry j (any output may be NULL). */
int strom_warm_get(const strom_warm* w, int32_t j, double* key, double* X, double* S, double* sigma);
/* Resets instance i of a solver to the warm start for key (combined on the
 * device); an empty store leaves the cold start X = S = y = 0, sigma0. */
int strom_solver_warm_start(strom_solver* s, int32_t i, const strom_warm* w, const double* key);
/* Attaches a store to a batch (NULL detaches). Requests submitted with a
 * key start, at admission, from the store's combination for their key; with
 * record != 0 each keyed request that meets tol is added to the store at
 * retirement while it has room. The store must outlive its attachment. */
int strom_batch_set_warm(strom_batch* b, strom_warm* w, int32_t record);
/* strom_batch_submit with a warm-start key (key_dim doubles of the attached
 * store); INVALID when no store is attached. */
int strom_batch_submit_keyed(strom_batch* b, const strom_sdp* sdp, const strom_problem* problem, const double* key,
                             uint64_t* ticket);

/* ------------------------------------------------------------------------
 * Kernel-level entry points for parity tests (device pointers, caller's
 * stream). They use the solver's uploaded operator of the whole batch: x has
 * length strom_solver_nsvec_total, y and r have length strom_solver_m_total.
 * ---------------------------------------------------------------------- */
int64_t strom_solver_nsvec_total(const strom_solver* s);
int64_t strom_solver_m_total(const strom_solver* s);
/* Offsets of instance i inside the batch vectors. */
int strom_solver_offsets(const strom_solver* s, int32_t i, int64_t* svec_off, int64_t* row_off);
/* Ax_dev = A(x_dev) = (<A_i, X>)_i (Sec. 3); all rows, dropped ones included. */
int strom_kernel_A(const strom_solver* s, const double* x_dev, double* Ax_dev, void* stream);
/* x_dev = A^* y = sum_l y_l A_l over all rows (Sec. 3). */
int strom_kernel_At(const strom_solver* s, const double* y_dev, double* x_dev, void* stream);
/* The same products for an operator given by raw device arrays: y_dev =
 * M x_dev for a CSR matrix M of nrows rows (rowptr_dev: int64 [nrows + 1],
 * col_dev: int32 column indices, val_dev: FP64 values, all on the device,
 * borrowed for the call). With A's rows (strom_sdp_export) it is A(X); with
 * the CSR of A^T it is A^*(y) (Sec. 3). x_dev and y_dev may not alias;
 * nrows = 0 does nothing. Asynchronous on `stream`. Errors: INVALID. */
int strom_kernel_spmv_csr(const int64_t* rowptr_dev, const int32_t* col_dev, const double* val_dev,
                          int64_t nrows, const double* x_dev, double* y_dev, void* stream);
/* y_dev = (A_K A_K^T)^{-1} r_K on the kept rows K, zero on dropped rows
 * (eq. solve-y1 / solve-y2). r_dev entries of dropped rows are ignored. */
int strom_kernel_solve(const strom_solver* s, const double* r_dev, double* y_dev, void* stream);

/* ------------------------------------------------------------------------
 * Autotuning of the y-solve launch shape. Sec. 4 picks the implementation of
 * the linear-system solve by measuring the alternatives (its hybrid
 * CPU/GPU solve against GPU triangular solves); this call makes that choice
 * per batch, on the device. When the instances share the factor of cliques
 * 2..N (opt.share_tail), the chain solve can serve a tile of 1, 2, 4 or 8
 * instances per CTA; all tiles give bit-identical y, so only the time
 * differs. Each candidate tile (up to the batch size) runs the whole y-solve
 * `reps` times on a scratch right-hand side, timed with CUDA events on the
 * solver's stream; the fastest is kept for every later iteration (the
 * captured iteration graph is rebuilt on the next step). Without a shared
 * tail only the one-instance-per-CTA solve exists and nothing changes.
 * Then the eigensolver: each block-size class's launch is timed with each
 * of its thread counts (2 or 3 per class), in each precision the solver
 * uses, and the fastest is kept. The thread count changes only which
 * thread updates which entries, and the order in which the off-diagonal
 * sum of the stopping test is added up, so results agree to rounding.
 * The solver's state (X, S, y, sigma) is not touched. reps in 1..1000.
 * Allocates two scratch vectors of m_total doubles and two of nsvec_total
 * doubles for the duration of the call. Waits for `stream` (may be NULL)
 * before timing. */
typedef struct {
  int32_t ncand;             /* candidates timed */
  int32_t tile[4];           /* instances per CTA of each candidate */
  double ms[4];              /* mean time of one y-solve (milliseconds) */
  int32_t chosen;            /* tile kept */
  /* eigensolver: per precision ([0] FP64, [1] FP32, the latter only when the
   * solver uses it) and block-size class (n <= 16, 40, 80, 160), the threads
   * per CTA kept (0: no blocks in the class) and the mean time of that
   * class's launch with them (cold sweeps on a fixed pseudo-random input of
   * the solver's block layout) */
  int32_t eig_threads[2][4];
  double eig_ms[2][4];
} strom_tune_report;
int strom_solver_tune(strom_solver* s, int32_t reps, void* stream, strom_tune_report* out);

/* ------------------------------------------------------------------------
 * PSD projection of a list of symmetric blocks given in svec form
 * (Sec. 4, parallel PSD cone projection): P = Q max(0, W) Q^T per block.
 * A plan uploads the block table once; execute may be called many times.
 * blk_off[i] is the svec offset of block i, blk_n[i] its size (1..160).
 * ---------------------------------------------------------------------- */
typedef struct strom_psd_plan strom_psd_plan;
int strom_psd_plan_create(const int64_t* blk_off, const int32_t* blk_n, int32_t nblk, int32_t precision,
                          strom_psd_plan** out);
void strom_psd_plan_destroy(strom_psd_plan* p);
/* P_dev = Pi(Xb_dev) block by block; Xb_dev and P_dev may not alias.
 * Optionally lam_dev receives the eigenvalues (ascending) of each block,
 * packed at offsets sum of previous blk_n (NULL to skip). */
int strom_psd_execute(strom_psd_plan* p, const double* Xb_dev, double* P_dev, double* lam_dev, void* stream);
/* One-shot form (creates and destroys a plan). */
int strom_kernel_psd_project(const double* Xb_dev, const int64_t* blk_off, const int32_t* blk_n,
                             int32_t nblk, int32_t precision, double* P_dev, void* stream);

/* The same projection for callers that cannot allocate device memory (a host
 * framework that owns the whole device pool, a real-time loop that must not
 * allocate after start-up). It allocates nothing: the block table and the
 * FP64 eigenvector scratch live in a static device array of the library
 * (about 4.37 MB, held by every GPU that loads the library until exit).
 * The paper has no counterpart; this is a deployment variant.
 * Limits: nblk <= 65536 (else STROM_ERR_INVALID, nothing launched); block
 * sizes 1..160. Set-up: the first call on a device looks up the array's
 * device address (cudaGetSymbolAddress), caches it and loads the kernels it
 * launches; under CUDA's lazy module loading that loading is when the static
 * array and the kernels' code take their device memory. A call with nblk = 0
 * (all pointers may then be NULL) does the set-up alone: a caller that must
 * not allocate later makes it at start-up, before any stream capture.
 * All calls share the array, so calls that overlap on the GPU race; the
 * caller serialises them. Every call synchronises `stream` and returns after
 * the projection has finished. blk_off / blk_n are host arrays. */
int strom_kernel_psd_project_noalloc(const double* Xb_dev, const int64_t* blk_off, const int32_t* blk_n,
                                     int32_t nblk, int32_t precision, double* P_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STROM_H */
