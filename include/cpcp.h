/*
 * cpcp.h -- C ABI of the GB300 multilevel CPCP library.
 *
 * The library solves the compressive principal component pursuit program
 * (Sec. 2, eq. (cpcp)):
 *
 *     min_{L,S}  1/2 || P_Q[L + S - D] ||_F^2 + lambda_L ||L||_* + lambda_S ||S||_1
 *
 * with lambda_L = mu and lambda_S = lambda * mu, where lambda is the PCP weight
 * of eq. (rpca) and mu > 0 the nuclear-norm weight.  Q is a set of observed
 * entries (P_Q keeps them and zeroes the rest, Sec. 2); with Q = everything the
 * program is the penalised form of PCP (eq. (rpca)).
 *
 * Each iteration is one accelerated proximal-gradient step with the joint step
 * 1/2 fixed by the 2-Lipschitz gradient (Sec. 2.3, eq. (cpcp-grad-LS)).  Its
 * L-prox is the multilevel step of Alg. 4: restrict M to the coarse model
 * M_H = M R (Sec. 3.1), singular value thresholding there (Sec. 3.2, minimiser
 * of the coarse Lagrangian), and prolongation L = L_H R^T.  Its S-prox is the
 * soft threshold of Alg. 3.  R = R_n R_{n/2} ... R_{n_H} is the composite
 * linear-interpolation operator of eq. (Rx), scaled to unit spectral norm
 * (Assumption 4).  The solver starts on the coarsest level and moves one level
 * finer when the restricted gradient carries too small a share of the gradient
 * (coarse-gradient test) or the fine-level residual stalls; it always finishes
 * on the fine level, so single-level and multilevel runs share the optimum of
 * eq. (cpcp).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major with an explicit leading dimension in elements
 *     (ld >= number of columns).  "device" pointers are CUDA device pointers
 *     on the handle's device; "host" pointers are ordinary CPU memory.
 *   - Observation mask Q: bit-packed, row-major, ldq 32-bit words per row
 *     (ldq >= ceil(n/32)); bit (j % 32) of word [i * ldq + j / 32] set means
 *     entry (i, j) is observed.  NULL means every entry is observed (PCP).
 *     Unobserved entries of D are never used arithmetically (NaN is allowed).
 *   - dtype selects the storage and arithmetic type of D, L and S:
 *     CPCP_F64 (fp64 throughout) or CPCP_F32 (fp32 storage, contractions and
 *     small k x k factorisations; norms and residual reductions accumulate
 *     in fp64, the residual-check sums with compensated (Dot2) products).
 *   - All work is queued on the handle's stream.  Calls return after the
 *     result is complete unless stated otherwise.
 *   - No entry point aborts, exits or throws; every failure is a status code
 *     and a message retrievable with cpcp_last_error().
 *   - The library owns its workspace (device memory allocated on first use and
 *     grown as needed); callers own every buffer they pass.
 */
#ifndef CPCP_H
#define CPCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPCP_OK = 0,
    CPCP_ERR_INVALID_ARG = 1,    /* argument out of range, NULL where required */
    CPCP_ERR_NONFINITE_INPUT = 2,/* NaN/Inf in an observed entry of D */
    CPCP_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    CPCP_ERR_NOMEM = 4,          /* workspace allocation failed */
    CPCP_ERR_NOT_CONVERGED = 5,  /* iteration cap reached; best iterate returned */
    CPCP_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
    CPCP_ERR_NUMERIC = 7         /* unrecoverable numerical breakdown */
} cpcp_status;

typedef enum { CPCP_F32 = 0, CPCP_F64 = 1 } cpcp_dtype;

typedef struct cpcp_context *cpcp_handle;

/* Solver options.  Zero-initialised fields take the listed defaults. */
typedef struct {
    int max_iter;          /* iteration cap (default 5000) */
    int check_every;       /* c: iterations between fine residual checks (10) */
    double eta;            /* continuation factor, mu_k = max(mu0 eta^k, mu) (0.9) */
    double mu0;            /* first weight; <= 0 means ||P_Q D||_2 (estimated) */
    double switch_ratio;   /* move one level finer when rel-KKT > ratio * last (0.9) */
    int k_max;             /* cap on the subspace width of the coarse SVD (256) */
    int oversample;        /* p: extra subspace columns beyond the rank (10) */
    int power_iters;       /* q: power steps per coarse SVD (1) */
    int check_power_iters; /* power steps of the fine SVD in the residual check (2) */
    int start_level;       /* 0 (default): start on the coarsest level; s > 0: start
                              at min(s, levels) - 1 halvings (s = 1: fine level) */
    uint64_t seed;         /* seed of the random start block of the subspace (1) */
    double *trace;         /* optional host array: rel-KKT of each residual check */
    int trace_cap;         /* capacity of trace (entries written: info.checks) */
    int profile;           /* nonzero: time the phases with CUDA events (info.phase_*); 2: also
                              the kernel families of the iterations' SVT phase
                              (info.svt_detail_ms), with every kernel launched from the host
                              (no graph replay) */
    int precision;         /* CPCP_F32 solves only.  0: fp32 contractions.  1 (mixed):
                              the two passes over the restricted iterate in each
                              subspace step (M_H Omega and M_H^T Q) run on the tensor
                              cores with BF16 operands and fp32 accumulation, until the
                              fine rel-KKT falls to refine_at; then fp32 to the end
                              (momentum restarts at the switch).  Residual checks and
                              the small k x k factorisations are never BF16. */
    double refine_at;      /* rel-KKT at which the mixed path turns to fp32 (1e-3) */
    int batch_threads;     /* cpcp_solve_batched: threads per CTA, 256 or 512; 0 = the
                              tuned choice for this batch if one was measured, else 512 */
    int batch_autotune;    /* cpcp_solve_batched: nonzero = on the first call with a new
                              batch (sizes, levels, masks, tolerance, options), time every
                              pair of CTA size (256, 512 threads) and output tile of the CTA
                              products wider than 32 columns (64 x 64, 128 x 64) and keep the
                              fastest for that batch (info.batch_threads, info.batch_tile) */
    int unroll;            /* K > 0: cpcp_solve runs the differentiable program instead
                              (see cpcp_backward): exactly K steps at the deepest level with
                              an exact SVT, recording checkpoints for the reverse sweep */
    int ckpt_every;        /* steps between checkpoints of the unrolled run (10) */
    double rho;            /* unrolled run: mu_k = mu max(rho eta^k, 1); must be > 0 */
    int subspace_mode;     /* cpcp_solve: must be 0 (power_iters full range passes per
                              iteration); other values: INVALID_ARG.  (A half-step form that
                              projected onto the previous iteration's singular subspace without
                              re-orthonormalising it diverged once the width grew, and was
                              removed.) */
    int pass_simt;         /* cpcp_solve, fp32: nonzero runs the fused fine pass on the SIMT
                              cores.  0 (default): the tensor-core pass (tcgen05, each factor
                              entry split into three TF32 parts, the six products of order
                              >= 2^-22, small and large terms in separate fp32 accumulators)
                              wherever D and S meet its alignment rules (16-byte aligned base,
                              leading dimension a multiple of 4); else the SIMT pass */
    int plain_launches;    /* cpcp_solve: nonzero launches every kernel of every iteration from
                              the host; 0 (default) captures an iteration's kernels in a CUDA
                              graph the second time the same (level, buffer parity) comes up and
                              replays the graph for the iterations between residual checks */
    int transfer;          /* coarse levels of cpcp_solve, ML-IALM (cpcp_ialm) and ML-FWT (cpcp_fwt):
                              0 (default) = R scaled to unit spectral norm (the reading of
                              Assumption 4); 1 = R replaced by an orthonormal basis of its range,
                              R C^{-1} with R^T R = C^T C (C upper bidiagonal, R^T R being
                              tridiagonal), which makes the coarse L-step the exact minimiser over
                              {L_H R^T} (epsilon = 0 in Theorem LH-eps); applied to M_H (and the
                              restricted gradient of the level test) and to V by two bidiagonal
                              solves.  cpcp_solve rejects it with unroll > 0,
                              cpcp_solve_batched rejects it; other values than 0 and 1:
                              INVALID_ARG */
    int early_test;        /* cpcp_solve level rule: 0 (default) or 1 = the coarse-gradient test
                              (move one level finer when ||G R||_F < kappa ||G||_F) also runs after
                              the first iteration on each coarse level, so data whose gradient is
                              not coarse (no smooth column structure) leave the coarse levels at
                              once; -1 = only every check_every iterations.  A handover skips
                              that iteration's residual check.  Other values: INVALID_ARG */
    int products_tc;       /* fp32 products of the subspace iteration with the (restricted)
                              iterate, M_H Omega and M_H^T Q: 1 = on the tensor cores (tcgen05
                              kind::tf32 with the three-part TF32 split of the fused pass, each
                              accumulator drained into round-to-nearest fp32 sums every 32 of K,
                              the long K split over CTAs with fixed-order partial sums); -1 = on
                              the SIMT cores; 0 (default) = the tensor cores where the iterate
                              has at least 4096 rows, SIMT otherwise.  The tensor-core path is
                              taken only where the operands meet the TMA rules (16-byte aligned
                              bases and leading dimensions, width <= 128), else SIMT.  Other
                              values: INVALID_ARG */
    int cholqr_fused;      /* fp32 CholeskyQR2 of the subspace SVDs: 0 (default) = six launches
                              (Gram, Cholesky and product kernels per pass); nonzero = both passes
                              in one launch of a thread-block cluster (16 CTAs, or 8 where the
                              device refuses 16) whose partial Gram matrices meet in distributed
                              shared memory, CTA 0 factorising, where the device accepts it.  Same
                              arithmetic either way up to the summation order of the Gram
                              matrices.  Measured on GB300: 6% slower on the 2000 x 2000 workload
                              (k = 60), a few percent faster on the 19200 x 400 video shape */
    int check_serial;      /* cpcp_solve: nonzero runs every fine residual check before the next
                              iteration starts.  0 (default), with graph replay (plain_launches 0,
                              profile < 2): a check on the fine level (fp32 contractions) runs on a
                              second, low-priority stream from a copy of the checked iterate while
                              the solve stream computes up to five further iterations (none of
                              them a decision point; one where the last two checks' rate predicts
                              that this check stops the solve); they count if the check lets the
                              solve go on, and are dropped (the checked iterate restored) if it
                              stops it.
                              Same iterates, decisions and result either way; the overlap costs
                              two more m x n buffers */
    int chol_form;         /* fp32 Cholesky factorisations of CholeskyQR: 0 (default) = for widths
                              k > 32 by 16-column block rows, each eliminated by one warp in
                              registers (shuffles, no barrier inside the block) and applied to the
                              trailing matrix by the whole CTA in one rank-16 update, R^{-1} by
                              block back substitution; for k <= 32 the form of 2; 1 = one
                              elimination step per CTA barrier with column quarters per thread in
                              registers; 2 = one elimination step per barrier over S in shared
                              memory with rolled loops (small code: a one-CTA kernel fetches its
                              code from L2 on every launch).  Same arithmetic up to rounding order.
                              Other values: INVALID_ARG */
    int svd_serial;        /* cpcp_solve, fp32 with power_iters = 1.  1: each iteration's subspace
                              SVD runs in order on the solve stream.  0 (default) and 2: Z' = M^T Y
                              starts on a second stream as soon as Y = M Omega exists, beside the
                              CholeskyQR2 of Y (Gram matrix, Cholesky, and a second pass that is
                              one launch, returning at once when the first pass found Y nearly
                              orthogonal), and the solve stream forms Z = Z' R_Y^{-1} (equal to
                              M^T Q_Y); with 0, Q_Y, Q_Z and the next start block are also formed
                              on the second stream, beside the factorisation of Z and the core
                              Jacobi SVD; with 2 they stay on the solve stream.  Where M^T Y on the
                              tensor cores (sized to about one CTA per SM) would fill three quarters
                              of the SMs or more, it runs on three quarters of them beside the other
                              chain.  The rounding
                              of Z differs from the in-order form by a factor of the equilibrated
                              condition number of Y (near 1 once the subspace is warm-started).
                              With profile = 2 everything runs in order.  Other values:
                              INVALID_ARG */
    int gram_form;         /* fp32 Gram matrices X^T X of the CholeskyQR passes: 0 (default) = for
                              X of at least 4096 rows, by row ranges, each CTA staging 64 rows of
                              the live columns at a time in
                              shared memory and writing one partial slice (up to 16, summed in CTA
                              order by the Cholesky kernel), shorter X as with 1; 1 = the tiled
                              cluster-reduced kernel of the other tall products (64 x 64 output tiles
                              whatever the live width).  Other values: INVALID_ARG */
    int jacobi_lanes;      /* lanes per column pair in the rounds of the core Jacobi SVD for widths
                              k <= 64: 0 (default) or 16 = 16 lanes (the 32 pairs of a round over
                              512 threads); 8 = 8 lanes (half the warps, a shorter shuffle tree;
                              measured 2-7% slower per solve).  Wider k always take 8.  Other
                              values: INVALID_ARG */
    int jacobi_check;      /* core Jacobi SVD of the iterations' subspace steps (the residual checks
                              keep 0): 0 (default) = sweeps until the
                              largest rotated |x_p . x_q| / (|x_p| |x_q|) of a sweep is at most the
                              stop level (1e-2 while the continuation weight falls, 1e-4 after); 1 =
                              also, after a sweep that rotated more than that, measure every pair's
                              off-orthogonality in one parallel pass and end when the largest is at
                              most a tenth of the stop level, instead of running a sweep to confirm
                              it (measured: 153 -> 151 sweeps and no time gained on the 2000 x 2000
                              workload, whose second sweeps still rotate; -0.6% on the 4-level video
                              solve).  Other values: INVALID_ARG */
    int pdl_off;           /* cpcp_solve iterations in the two-stream subspace step (svd_serial):
                              0 (default) = programmatic dependent launch of the solve stream's
                              chain of small kernels (Gram matrices, Cholesky, second CholeskyQR
                              pass, Jacobi, schedule end): each starts while its predecessor runs
                              and waits for its results on the device, which hides a launch latency
                              per kernel (measured 25.0 -> 24.4 ms on the 2000 x 2000 workload,
                              results bit-identical); not with profile = 2, and not in the in-order
                              form (where it made the 4-level video solve 4% slower).  1 = ordinary
                              stream order.  Other values: INVALID_ARG */
} cpcp_options;

/* Phases timed when cpcp_options.profile is set. */
enum {
    CPCP_PHASE_PASS_COARSE = 0, /* fused iteration pass with restriction (level > 0) */
    CPCP_PHASE_PASS_FINE = 1,   /* fused iteration pass on the fine level */
    CPCP_PHASE_SVT = 2,         /* subspace SVD + SVT + prolongation of one iteration */
    CPCP_PHASE_CHECK = 3,       /* fine residual check (pass, fine SVD, difference) */
    CPCP_NUM_PHASES = 4
};

/* Per-solve report. */
typedef struct {
    int status;            /* cpcp_status of the solve */
    int iters;             /* iterations taken */
    int level_iters[8];    /* iterations spent at each number of halvings */
    int final_level;       /* halvings when the solve stopped (0 = fine) */
    int rank;              /* rank of the returned L */
    int checks;            /* fine residual checks performed */
    double relkkt;         /* last fine relative gradient-mapping residual */
    double mu0;            /* first continuation weight used */
    double pqd_fro;        /* ||P_Q D||_F */
    double seconds;        /* wall time of the solve (host clock) */
    double phase_ms[4];    /* device time per phase (profile only), CPCP_PHASE_* */
    int phase_count[4];    /* timed intervals per phase */
    long long launches;    /* CUDA kernels launched by the solve */
    int bf16_iters;        /* iterations whose contractions ran in BF16 (precision 1) */
    double svt_detail_ms[4]; /* the SVT phase split into the products with M, CholeskyQR, the
                                core Jacobi SVD and the factor products with the next start
                                block: cpcp_solve_batched (the instance's, SM cycle counter at the
                                nominal clock) and cpcp_solve with profile = 2 (the iterations',
                                CUDA events; residual checks excluded) */
    int jacobi_calls;      /* cpcp_solve: core Jacobi SVDs run (iterations and checks) */
    int jacobi_sweeps;     /* cpcp_solve: their sweeps, summed */
    int chol_factors;      /* cpcp_solve: Cholesky factorisations of CholeskyQR run (second
                              passes skipped on the device are not counted) */
    int batch_threads;     /* cpcp_solve_batched: threads per CTA of the launch (256 or 512) */
    int batch_tile;        /* cpcp_solve_batched: output tiles of the CTA products wider than 32
                              columns, 0 = 64 x 64, 1 = 128 x 64 (the autotuner's choice, or 0) */
    double level_ms[8];    /* cpcp_solve with profile: device time of the iterations at each
                              number of halvings (their pass and SVT phases; residual checks
                              excluded); divided by level_iters, the cost of one iteration there */
} cpcp_info;

/* One instance of cpcp_solve_batched (fp32, device pointers; conventions as
 * for cpcp_solve).  L and S may be NULL when not wanted. */
typedef struct {
    int m, n;              /* rows and columns of D */
    const float *D;        /* m x n, leading dimension ldd */
    int64_t ldd;
    const uint32_t *Q;     /* bit-packed observation mask (ldq words per row) or NULL */
    int64_t ldq;
    double lambda, mu;     /* weights as in cpcp_solve */
    int levels;            /* 1 .. 4 */
    float *L;              /* m x n output, leading dimension ldl, or NULL */
    int64_t ldl;
    float *S;              /* m x n output, leading dimension lds, or NULL */
    int64_t lds;
} cpcp_problem;

/* Returns a static description of a status code. */
const char *cpcp_status_string(cpcp_status s);

/* Last error message recorded on the handle (empty string if none).  The
 * pointer stays valid until the next call on the same handle. */
const char *cpcp_last_error(cpcp_handle h);

/*
 * Create a handle bound to CUDA device `device` and stream `stream` (a
 * cudaStream_t passed as void*, NULL = the legacy default stream).  opt may be
 * NULL for defaults; the options are copied.  *h receives the handle.
 * Errors: INVALID_ARG (h NULL, bad device), CUDA.
 */
cpcp_status cpcp_create(cpcp_handle *h, int device, void *stream, const cpcp_options *opt);

/* Release the handle and its workspace.  NULL is accepted and ignored. */
void cpcp_destroy(cpcp_handle h);

/*
 * Solve eq. (cpcp) for D (m x n, dtype, leading dimension ldd) with mask Q.
 *   lambda  > 0   weight ratio (lambda_S = lambda * mu)
 *   mu      > 0   nuclear-norm weight lambda_L (final continuation value)
 *   levels  >= 1  number of levels; 1 = single level, levels-1 halvings of n
 *   tol     > 0   stop when the fine relative residual (below) is <= tol
 *   L_out, S_out  m x n outputs (ldl, lds), may be NULL to skip
 * The relative residual is the gradient-mapping norm
 *   || (L - SVT_{mu/2}(L - G/2), S - shrink_{lambda mu/2}(S - G/2)) ||_F * 2
 *   / ||P_Q D||_F with G = P_Q[L + S - D]; it is zero iff (L, S) is optimal.
 * D, Q, L_out, S_out may be all device pointers or all host pointers (host
 * buffers are staged through device memory inside the call).
 * Validation (INVALID_ARG): m, n >= 1; lambda, mu, tol > 0; 1 <= levels <= 6;
 * the coarse width n_H after levels-1 halvings (ceil(n/2) per level) must be
 * >= 1 and, when levels > 1, n_H <= (m + 1) / 2 (Assumption 2).  If n > m
 * the transposed problem is solved and the results transposed back, with the
 * same rules applied to the transposed sizes.
 * Returns OK, NOT_CONVERGED (outputs hold the last iterate), NONFINITE_INPUT,
 * NOMEM, CUDA or NUMERIC.  info may be NULL.
 */
cpcp_status cpcp_solve(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd,
                       const uint32_t *Q, int64_t ldq, double lambda, double mu, int levels, double tol,
                       void *L_out, int64_t ldl, void *S_out, int64_t lds, cpcp_info *info);

/*
 * Frank-Wolfe Thresholding for eq. (cpcp): Alg. 3 (levels == 1) or ML-FWT,
 * Alg. 6 (levels > 1), on the epigraph form eq. (cpcp-fw),
 *   min 1/2 ||P_Q[L + S - D]||_F^2 + lambda_L t_L + lambda_S t_S,
 *   ||L||_* <= t_L <= U_L, ||S||_1 <= t_S <= U_S,
 * with lambda_L = mu and lambda_S = lambda * mu.  Each iteration takes the
 * linear minimisation oracles at G = P_Q[L + S - D] (nuclear ball: the top
 * singular pair of G, or of G R lifted by R for ML-FWT (of G R C^{-1} lifted
 * by R C^{-1} with cpcp_options.transfer = 1), from the subspace
 * SVD of cpcp_solve, block width min(oversample, k_max, n_H, m) and
 * power_iters passes, warm started from the last iteration's right vectors;
 * at full width it is exact; l1 ball: the first entry
 * of largest |G|), the exact minimiser of the objective over the two segments
 * toward them, the thresholding step S = shrink_{lambda_S}(S - P_Q[L+S-D])
 * with t_S = ||S||_1, and the bound updates U = f / lambda.  Starts from
 * L = S = 0.  Stops when the relative decrease |f_{k-1} - f_k| <= tol f_{k-1}
 * (OK; tol = 0 runs max_iter iterations, NOT_CONVERGED) or after max_iter
 * iterations.  D, Q (optional, bit-packed as in cpcp_solve), L_out, S_out:
 * device buffers (row-major, leading dimensions in elements).  ftrace
 * (optional, host, max_iter doubles) receives f after each iteration;
 * info->iters, relkkt (the last relative decrease), mu0 (the last f),
 * seconds and launches are filled.
 * Validation (INVALID_ARG): m, n >= 1; lambda, mu > 0; tol >= 0; max_iter >= 1;
 * 1 <= levels <= 6 with n_H >= 1; device buffers.
 */
cpcp_status cpcp_fwt(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, const uint32_t *Q,
                     int64_t ldq, double lambda, double mu, int levels, int max_iter, double tol, void *L_out,
                     int64_t ldl, void *S_out, int64_t lds, double *ftrace, cpcp_info *info);

/*
 * Inexact augmented Lagrangian method for PCP, eq. (rpca) (min ||L||_* +
 * lambda ||S||_1 subject to L + S = D): Alg. 1 (levels == 1) or its
 * multilevel form Alg. 4 (levels > 1; every iteration takes the low-rank step
 * on the coarse level, L = SVT_{1/mu_k}(M R) R^T with R the composite
 * restriction scaled to unit norm, or with the orthonormal basis R C^{-1} of
 * its range when cpcp_options.transfer = 1), with S_0 = Y_0 = 0 and
 *   M = D - S + Y / mu_k;  L = SVT_{1/mu_k}(M)  (or the coarse step);
 *   S = shrink_{lambda/mu_k}(D - L + Y / mu_k);  Y += mu_k (D - L - S).
 * Penalty schedule: rho > 1 gives mu_{k+1} = rho mu_k, otherwise mu_k =
 * mu0 (1 + k); mu0 <= 0 means 1.25 / ||D||_2 (estimated on the device).  The
 * SVT of each iteration uses the subspace-iteration SVD of cpcp_solve (warm
 * started, options power_iters, oversample, k_max).  Stops at the first
 * iteration whose feasibility gap ||D - L - S||_F / ||D||_F is <= tol, or
 * after max_iter iterations (NOT_CONVERGED); fg (optional, host, max_iter
 * doubles) receives the gap after each iteration.  D, L_out, S_out: m x n
 * device or host buffers as in cpcp_solve; requires n <= m (the restriction
 * acts on columns; pass the transpose otherwise).  info->iters, rank,
 * relkkt (the last gap), seconds and launches are filled.
 * Validation (INVALID_ARG): 1 <= n <= m; lambda, tol > 0; max_iter >= 1;
 * 1 <= levels <= 6 with n_H >= 1 and, when levels > 1, n_H <= (m + 1) / 2.
 */
cpcp_status cpcp_ialm(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, double lambda,
                      int levels, double mu0, double rho, int max_iter, double tol, void *L_out, int64_t ldl,
                      void *S_out, int64_t lds, double *fg, cpcp_info *info);

/*
 * One accelerated proximal-gradient step of the multilevel method (the hot
 * path of one iteration), on device buffers:
 *   Lhat = (1 + beta) A_k B_k^T - beta A_p B_p^T        (momentum on L)
 *   Shat = S_k + beta (S_k - S_p)                        (momentum on S)
 *   G    = P_Q[Lhat + Shat - D]                          (eq. (cpcp-grad-LS))
 *   S_out = shrink_{lambda mu_k / 2}(Shat - G/2)         (Alg. 3 threshold)
 *   M_H  = (Lhat - G/2) R,   L_H = SVT_{mu_k/2}(M_H),   L_out = L_H R^T
 *                                                        (Alg. 4, restrict/SVT/prolong)
 * Factors: A_k (m x r_k, lda), B_k (n x r_k, ldb), A_p (m x r_p, ldap),
 * B_p (n x r_p, ldbp) (a rank may be 0, its pointers are then unused).  R is the unit-norm composite operator
 * for `halvings` halvings of n (0 = fine level).
 * The coarse SVD runs subspace iteration with width k (1 <= k <= n_H) and q
 * power steps from the start block Omega0 (n_H x k, ldo; NULL = seeded random);
 * with k = n_H it is an exact SVD.
 * Outputs: S_out (m x n, lds); the new factors A_out (m x k, ldao) =
 * U diag(sigma - mu_k/2)_+ and B_out (n x k, ldbo) = R V; *r_out = number of
 * singular values above mu_k/2 (columns beyond r_out are zero); sigma_out
 * (k doubles, host or device; may be NULL) the coarse singular values.
 * With CPCP_F32 at halvings = 0 the fused pass runs on the tensor cores, as
 * in cpcp_solve, when the operands meet its TMA rules (D, S_k, S_p, S_out
 * 16-byte aligned with leading dimensions that are multiples of 4; lda = ldap
 * and ldb = ldbp, multiples of 4) and options.pass_simt is 0; otherwise on the
 * SIMT cores.
 * Requires n <= m (no internal transpose).  Errors: INVALID_ARG, NOMEM, CUDA,
 * TIMEOUT (a bounded wait of the tensor-core pass expired).
 */
cpcp_status cpcp_step(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, const uint32_t *Q,
                      int64_t ldq, double lambda, double mu_k, double beta, int halvings, const void *S_k,
                      const void *S_p, int64_t lds_in, const void *A_k, int64_t lda, const void *B_k, int64_t ldb,
                      int r_k, const void *A_p, int64_t ldap, const void *B_p, int64_t ldbp, int r_p, int k, int q,
                      const void *Omega0, int64_t ldo, void *S_out, int64_t lds, void *A_out, int64_t ldao,
                      void *B_out, int64_t ldbo, int *r_out, double *sigma_out);

/*
 * Restriction M_H = M R (Sec. 3.1; the coarse matrix of Alg. 4):
 * M (m x n, ldm) -> M_H (m x n_H, ldh), R the unit-norm composite operator for
 * `halvings` halvings of n.  Device buffers.  Errors: INVALID_ARG, CUDA.
 */
cpcp_status cpcp_restrict(cpcp_handle h, int m, int n, int halvings, cpcp_dtype dt, const void *M, int64_t ldm,
                          void *MH, int64_t ldh);

/*
 * Prolongation of right factors B = R V (Sec. 3.2, L = L_H R^T = U (R V)^T):
 * V (n_H x r, ldv) -> B (n x r, ldb).  Device buffers.
 */
cpcp_status cpcp_prolong(cpcp_handle h, int n, int halvings, int r, cpcp_dtype dt, const void *V, int64_t ldv,
                         void *B, int64_t ldb);

/*
 * Scale of the composite operator: *scale = 1 / ||R_printed||_2 for
 * `halvings` halvings of n, and *nh = n_H.  Host only.
 */
cpcp_status cpcp_transfer_info(int n, int halvings, double *scale, int *nh);

/*
 * The orthonormal-basis transfer of cpcp_options.transfer = 1 for
 * `halvings` >= 1 halvings of n: R^T R = C^T C with R the unit-norm composite
 * operator and C upper bidiagonal, C's diagonal into cd and super-diagonal into
 * ce (n_H doubles each, ce[n_H - 1] = 0; either may be NULL), and into *kappa
 * (may be NULL) the coarse-gradient test's threshold for R C^{-1}: the
 * geometric mean of ||R C^{-1}||_F / sqrt(n) and ||1^T R C^{-1}|| / sqrt(n).
 * Host only.  INVALID_ARG unless n >= 1 and 1 <= halvings <= 5.
 */
cpcp_status cpcp_transfer_orth(int n, int halvings, double *cd, double *ce, double *kappa);

/*
 * Truncated SVD of a device matrix M (m x n, ldm, m >= n) by subspace
 * iteration of width k (1 <= k <= n) with q power steps from Omega0 (n x k,
 * ldo; NULL = seeded random): M ~ U diag(sigma) V^T, U (m x k, ldu),
 * V (n x k, ldv), sigma (k doubles, device or host).  Singular values are in
 * descending order; with k = n the factorisation is exact up to rounding.
 * With options.precision = 1 (CPCP_F32 only) the two contractions with M of
 * each power step use BF16 operands on the tensor cores (see cpcp_gemm_bf16).
 */
cpcp_status cpcp_svd(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *M, int64_t ldm, int k, int q,
                     const void *Omega0, int64_t ldo, void *U, int64_t ldu, void *V, int64_t ldv, double *sigma);

/*
 * Reverse sweep of the last unrolled run on this handle (cpcp_solve with
 * options.unroll = K > 0, CPCP_F32, n <= m).  That run computes, from
 * L_0 = L_{-1} = S_0 = S_{-1} = 0, K steps of the proximal iteration at the
 * deepest level h = levels - 1 (Alg. 4 coarse step with an exact SVT of
 * M_H = (Lh - tau G) R by one-sided Jacobi, Alg. 3 shrink, FISTA momentum,
 * tau = 1/2) with weights mu_k = mu max(rho eta^k, 1), and returns L_K, S_K.
 * rho is a constant of the program; rho = ||P_Q D||_2 / mu reproduces the
 * continuation of cpcp_solve (for levels = 1 its first step then thresholds
 * tau P_Q D exactly at the top singular value, a point of non-smoothness).
 * Differentiation is not in the paper.
 *
 * Given the cotangents dL = d loss / d L_K (m x n, device, ldgl) and dS =
 * d loss / d S_K (device, ldgs, or NULL for zero), writes dD = d loss / d D
 * (device, m x n, ldgd; zero at unobserved entries) and the host scalars
 * *dlambda, *dmu.  The forward states are recomputed from the checkpoints
 * (every options.ckpt_every steps); the SVT is differentiated with the
 * singular-value-gap formula (the Jacobian of a proximal map is
 * self-adjoint), the shrink with its active set.  D and Q are copied by the
 * recording run.  Errors: INVALID_ARG (no recorded run, bad arguments), CUDA,
 * TIMEOUT (a bounded grid barrier of the SVD expired).
 */
cpcp_status cpcp_backward(cpcp_handle h, const float *dL, int64_t ldgl, const float *dS, int64_t ldgs, float *dD,
                          int64_t ldgd, double *dlambda, double *dmu);

/*
 * Solve `count` independent instances of eq. (cpcp) (fp32) in one persistent
 * launch.  Each CTA takes the next instance from a device work queue ordered by
 * decreasing size and runs the whole multilevel solve of cpcp_solve on it (the
 * same continuation, level switching, residual checks and tolerance), with the
 * instance's iterates resident in a device arena owned by the handle; a
 * problem with n > m is solved transposed.  Limits per instance: levels in
 * [1, 4]; min(m, n) <= 1024; subspace width at most 64 (rank + oversampling);
 * n_H <= (m + 1) / 2 when levels > 1 (Assumption 2).  The launch and the
 * read-back of the per-instance reports are captured in a CUDA graph that a
 * later call with the same sizes, levels, tolerance and options replays (the
 * instance descriptors, with the caller's pointers, are uploaded first on
 * every call).
 *   infos: host array of `count` reports (may be NULL); infos[i].status is
 *   instance i's status, the return value the first non-OK status in the order
 *   INVALID_ARG, NONFINITE_INPUT, NOT_CONVERGED (or OK).  seconds is the
 *   wall time of the whole batch, launches the kernels of the whole call;
 *   phase_ms is the instance's own device time per phase, from the SM cycle
 *   counter at the nominal clock (phase_count is 0).
 * Errors before any device work: INVALID_ARG (bad instance), NOMEM.
 */
cpcp_status cpcp_solve_batched(cpcp_handle h, int count, const cpcp_problem *probs, double tol, cpcp_info *infos);

/*
 * The contraction of the mixed-precision subspace iteration (options.precision
 * = 1), exposed for testing: C = bf16(A) bf16(B)^T with fp32 accumulation on
 * the tensor cores (tcgen05, TMEM accumulator).  This is the product form of
 * both passes over the restricted iterate in a power step (M_H Omega and
 * M_H^T Q, Sec. 4): the library stores both operands K-major.
 *   A (rows x K, lda) and B (N x K, ldb): fp32 device matrices, rounded to
 *   BF16 (nearest even) on the device; C (rows x N, ldc): fp32 device output.
 *   1 <= N <= 256; rows, K >= 1.  The K sum is split across CTAs and the
 *   partial sums are added in a fixed order, so the result is deterministic.
 * Errors: INVALID_ARG, NOMEM, CUDA, TIMEOUT (a bounded wait of the kernel
 * expired; the context stays usable).
 */
cpcp_status cpcp_gemm_bf16(cpcp_handle h, int rows, int K, int N, const float *A, int64_t lda, const float *B,
                           int64_t ldb, float *C, int64_t ldc);

/*
 * ||P_Q[D]||_F (fro, host double) and the number of observed entries of D
 * that are NaN or infinite (nonfinite, host int64, may be NULL), computed
 * without allocating any memory.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory while they run --
 * code whose device memory is all handed out up front by its own pool or
 * arena (a framework's caching allocator, an inference server with a fixed
 * budget), and latency-critical loops that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.  It needs no handle.
 *
 * D (m x n, dtype, ldd) and Q (bit-packed mask as in cpcp_solve, or NULL) are
 * device pointers on the current device; the work is queued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call synchronises that
 * stream: it returns after the results have been copied to the host.  The partial sums live in one static
 * device array of 1 MiB that every GPU loading the library holds until the
 * process exits; the largest accepted problem has ceil(m/64) * ceil(n/64) <=
 * 65536 tiles (for example 16384 x 16384) -- larger sizes return
 * CPCP_ERR_INVALID_ARG before any device work.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU (different streams or threads on
 * the same device) race and must be serialised by the caller.  Every slot a
 * call reads is written by the same call, so nothing needs clearing.
 * Returns OK, INVALID_ARG or CUDA (also when either kernel launch fails; the
 * results are then not written).
 */
cpcp_status cpcp_masked_norm_static(void *stream, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd,
                                    const uint32_t *Q, int64_t ldq, double *fro, int64_t *nonfinite);

#ifdef __cplusplus
}
#endif

#endif /* CPCP_H */
