// common.cuh -- shared device helpers and launch declarations of the CUDA
// library (not part of the public ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace cpcp {

// Number of kernels this library has launched in the process (reported per
// solve in cpcp_info.launches).
extern unsigned long long g_kernel_launches;
#define CPCP_COUNT_LAUNCH() (++::cpcp::g_kernel_launches)

// Programmatic dependent launch of the iteration's chain of small kernels:
// while g_pdl is set (by the solver, around launches that follow a kernel of
// the same stream), the launchers below ask for programmatic stream
// serialisation, so the next kernel starts while its predecessor runs and
// waits at pdl_enter() for the predecessor's completion and memory.  Every
// kernel such a launcher starts calls pdl_enter() before it reads anything
// (it does nothing for a kernel launched without the attribute).
extern thread_local int g_pdl;
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
struct PdlScope {
    int prev;
    explicit PdlScope(bool on) : prev(g_pdl) { g_pdl = on ? 1 : 0; }
    ~PdlScope() { g_pdl = prev; }
};
// kernel launch with the programmatic-serialisation attribute when g_pdl is set
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Device-resident scalars of one solve.  The per-iteration schedule (momentum
// weight, continuation weight, thresholds, ranks, subspace width) lives here
// so that an iteration needs no host round trip and can be graph-captured.
struct Ctrl {
    double tau;      // step 1/2 (2-Lipschitz gradient)
    double lam;      // lambda (lambda_S = lam * mu)
    double mu_bar;   // final weight mu
    double mu0;      // first continuation weight
    double eta;      // continuation factor
    double t;        // FISTA t_k
    double beta;     // momentum weight of the current iteration
    double mu_k;     // weight of the current iteration
    double theta_L;  // tau * mu_k
    double theta_S;  // tau * lam * mu_k
    double t_next;   // FISTA t_{k+1}
    int iter;        // iterations done
    int rk;          // rank of L_k factors
    int rp;          // rank of L_{k-1} factors
    int r_new;       // rank produced by the current iteration
    int k;           // active subspace width of the coarse SVD
    int k_next;      // width for the next iteration
    int kcap;        // min(n_H, k_max) on the current level
    int oversample;  // p
    int flags;       // bit 0: rank reached the width at least once
    int pad_;
    uint64_t seed;
    double eta_k;    // eta^iter (continuation factor so far; 1 at the start)
};

// shrink(x) = sign(x) max(|x| - th, 0), with a signed zero inside the band
template <typename T>
__device__ __forceinline__ T shrink(T x, T th)
{
    T a = fabs(x) - th;
    return a > T(0) ? copysign(a, x) : copysign(T(0), x);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// splitmix64 (Steele, Lea, Flood 2014) -> uniform in [-1, 1)
__host__ __device__ __forceinline__ double hash_uniform(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x = x ^ (x >> 31);
    return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Composite transfer operator of one level on the device: fine column j maps
// to coarse columns j0[j] (weight w0[j]) and j0[j] + 1 (weight w1[j]);
// coarse column c draws on the contiguous fine range [clo[c], chi[c]].
template <typename T>
struct TransferDev {
    int n, nh;
    double kappa;  // threshold of the coarse-gradient test (host use)
    const int *j0;
    const T *w0, *w1;
    const int *clo, *chi;
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files); all asynchronous on `st`
// ---------------------------------------------------------------------------

// Fused iteration pass (momentum, masked gradient, shrink, restriction).
template <typename T>
struct PassArgs {
    int m, n;
    const T *D;
    int64_t ldd;
    const uint32_t *Q;
    int64_t ldq;
    const T *Sk, *Sp;  // S_k, S_{k-1}
    int64_t lds;
    T *Sout;           // S_{k+1} (step) or nullptr
    int64_t ldso;
    const T *Ak, *Bk, *Ap, *Bp;  // low-rank factors (row-major)
    int64_t ldfa, ldfb;          // leading dimensions of Ak, Bk
    int64_t ldfap, ldfbp;        // leading dimensions of Ap, Bp
    const int *rk, *rp;          // device ranks of (Ak, Bk) and (Ap, Bp); may be null (= 0)
    const Ctrl *ctrl;
    T *M;              // fine output (level 0) or nullptr
    int64_t ldm;
    T *MH;             // coarse output (level > 0), zero on entry
    int64_t ldh;
    T *GH;             // optional (level > 0): G R, zero on entry, leading dimension ldh;
                       // then partial slot 0 of each block receives its share of ||G||_F^2
    TransferDev<T> tr;
    double *partial;   // per-block fp64 partial sums (check / norm passes)
};

// returns the number of blocks (partial sums written when a.GH is set)
template <typename T> int launch_step_pass(const PassArgs<T> &a, bool coarse, cudaStream_t st);
// the fine STEP pass on the tensor cores (k_pass_tc.cu); false, launching
// nothing, when an operand does not meet the TMA rules.  err: device flag set
// when a bounded wait of the kernel expired.
bool launch_pass_tc(const PassArgs<float> &p, int *err, cudaStream_t st);
// the products of the subspace iteration with M on the tensor cores
// (k_pass_tc.cu, three-part TF32 split): tn = 0 C = M B (M is P x K), tn = 1
// C = M^T B (M is K x P), B (K x k, k = *kdyn <= bcols_max <= 128); writes
// partial slices (returned count, 0 = not launched: an operand breaks the TMA
// rules) for launch_reduce_partial.  err: set when a bounded wait expired.
int launch_prod_tc(int tn, int P, int K, const float *M, int64_t ldm, const float *B, int64_t ldb, int bcols_max,
                   const int *kdyn, float *part, int64_t ldc, int64_t slice, int max_splits, int *err, cudaStream_t st,
                   int max_ctas = 0);
// CTAs that launch_prod_tc runs for a P-row output with K-long contraction
// (max_ctas > 0: at most that many instead of about one per SM)
int prod_tc_ctas(int P, int K, int max_splits, int max_ctas = 0);
// multiprocessors of the current device
int gpu_sm_count();
// per-block fp64 partial sums of squares of X (rows x cols); returns the block count
template <typename T> int launch_sumsq(int rows, int cols, const T *X, int64_t ld, double *partial, cudaStream_t st);
// check pass at (L_k, S_k) with weight mu_bar: writes M = L - tau G and
// per-block sums of ||S - shrink(S - tau G)||^2 (slot 0), ||P_Q D||^2 (slot 1),
// count of non-finite observed D (slot 2).
template <typename T> int launch_check_pass(const PassArgs<T> &a, cudaStream_t st);
// per-block sums of ||A_k B_k^T - A_p B_p^T||^2 (factors with ranks rk, rp from ctrl)
template <typename T> int launch_diff_pass(const PassArgs<T> &a, cudaStream_t st);
// dense L = A_k B_k^T into a.M (rank from a.rk)
template <typename T> void launch_reconstruct(const PassArgs<T> &a, cudaStream_t st);
void launch_sum_partials(const double *partial, int nblocks, int nslots, double *out, cudaStream_t st);

// dense GEMMs on row-major tall-skinny operands
template <typename T>
void launch_gemm_nn(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                    const int *kdyn_K, const int *kdyn_N, int kmaxN, cudaStream_t st);
template <typename T>
void launch_gemm_nn_splitk(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                           T *partial, const int *kdyn_N, int kmaxN, cudaStream_t st);
template <typename T>
int launch_gemm_tn_partial(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *partial,
                           const int *kdyn_N, int kmaxN, int kmaxK, cudaStream_t st, const int *skip = nullptr);
template <typename T>
void launch_reduce_partial(const T *partial, int splits, int K, int N, T *C, int64_t ldc, const int *kdyn_K,
                           const int *kdyn_N, cudaStream_t st);
template <typename T>
void launch_restrict(int m, int n, const T *M, int64_t ldm, T *MH, int64_t ldh, const TransferDev<T> &tr,
                     cudaStream_t st);
template <typename T>
void launch_prolong(int n, const T *V, int64_t ldv, T *B, int64_t ldb, const TransferDev<T> &tr, const int *kdyn,
                    int kmax, cudaStream_t st);
template <typename T>
void launch_restrict_rows(const T *B, int64_t ldb, T *Om, int64_t ldo, const TransferDev<T> &tr, const int *kdyn,
                          int kmax, cudaStream_t st);
template <typename T>
void launch_transpose(int rows, int cols, const T *A, int64_t lda, T *B, int64_t ldb, cudaStream_t st);
void launch_transpose_mask(int rows, int cols, const uint32_t *in, int64_t ldi, uint32_t *out, int64_t ldo,
                           cudaStream_t st);

// tall-skinny contractions with the split-K sums reduced inside a thread-block
// cluster (k_tsgemm.cu).  Each returns false (launching nothing) when an
// operand is not 16-byte aligned with a 16-byte multiple leading dimension.
// C = A B; K dynamic when kdyn_K is given (then kmaxK bounds it); skip: when
// *skip is set C = A (B is the identity; only with kdyn_K)
template <typename T>
bool launch_ts_nn(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                  const int *kdyn_K, const int *kdyn_N, int kmaxK, int kmaxN, const int *skip, cudaStream_t st);
// C (P x N) = A^T B with A K x P, B K x N
template <typename T>
bool launch_ts_tn(int P, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                  const int *kdyn_N, int kmaxN, cudaStream_t st);
// Gram X^T X (k = *kdyn) as partial slices of kmax x kmax; returns their
// number (-1: not aligned, nothing launched); skip: nothing when *skip is set
template <typename T>
int launch_ts_gram(int rows, const T *X, int64_t ldx, T *partial, const int *kdyn, int kmax, const int *skip,
                   cudaStream_t st);

// IALM / ML-IALM passes (k_ialm.cu): M = D - S + Y / mu; the S and Y steps
// with per-block partial sums of ||D - L - S||_F^2 (ialm_blocks() of them)
int ialm_blocks();
template <typename T>
void launch_ialm_m(int m, int n, const T *D, int64_t ldd, const T *S, const T *Y, int64_t lds, double mu, T *M,
                   int64_t ldm, cudaStream_t st);
template <typename T>
void launch_ialm_update(int m, int n, const T *D, int64_t ldd, const T *L, int64_t ldl, T *S, T *Y, int64_t lds,
                        double lam, double mu, double *partial, cudaStream_t st);
// end == 0: theta_L = 1 / mu into the control block; 1: width bookkeeping
void launch_ialm_ctrl(Ctrl *c, double mu, int end, cudaStream_t st);
// Device-resident scalars of an FW-T / ML-FWT run (k_fwt.cu): the epigraph
// objective, the bounds and variables t_L, t_S, U_L, U_S, the argmax of |G|,
// this iteration's vertices and step sizes, and the stop state.  Every kernel
// of an iteration reads them here, so an iteration needs no host round trip
// and can be replayed as a CUDA graph.
struct FwScal {
    double f, tL, tS, UL, US, gmax, rel;
    double cL, vs, VtL, VtS, a, b;  // V_L = cL u v^T, V_S = vs e_{i*}; step sizes
    double lamL, lamS, tol, margin;
    int64_t istar;
    int done;   // 0 running; 1 the relative decrease reached tol; 2 numeric failure
    int iters;  // iterations completed
};
// start: f and the argmax of |G| from fwt_grad's partials; t_L = t_S = 0
void launch_fwt_first(FwScal *sc, const double *partial, const double *amax_v, const int64_t *amax_i,
                      cudaStream_t st);
// the LMOs' vertices from the top singular value sig[0] and G[i*] (done = 2 when
// no finite entry of G exists)
template <typename T>
void launch_fwt_lmo(FwScal *sc, const T *sig, const T *G, int64_t ld, int m, int n, cudaStream_t st);
// the two-segment line search from fwt_coef's partials
void launch_fwt_ls(FwScal *sc, const double *partial, cudaStream_t st);
// after fwt_update: t_L, t_S, f, U_L, U_S, the argmax; trace[iters] = f; the stop test
void launch_fwt_post(FwScal *sc, const double *partial, const double *amax_v, const int64_t *amax_i, double *trace,
                     cudaStream_t st);
// Frank-Wolfe Thresholding passes (k_fwt.cu): fwt_blocks() per-block
// partials (1, 5 and 2 per block) and per-block argmax |G| (value, index)
int fwt_blocks();
template <typename T>
void launch_fwt_grad(int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const T *L, const T *S,
                     int64_t ld, T *G, double *partial, double *amax_v, int64_t *amax_i, cudaStream_t st);
template <typename T>
void launch_fwt_coef(int m, int n, const uint32_t *Q, int64_t ldq, const T *L, const T *S, const T *G, int64_t ld,
                     const T *u, int64_t ldu, const T *v, int64_t ldv, const FwScal *sc, double *partial,
                     cudaStream_t st);
template <typename T>
void launch_fwt_update(int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq, T *L, T *S, T *G,
                       int64_t ld, const T *u, int64_t ldu, const T *v, int64_t ldv, const FwScal *sc,
                       double *partial, double *amax_v, int64_t *amax_i, cudaStream_t st);
// the orthonormal-basis transfer of ML-IALM: C upper bidiagonal (diagonal cd,
// super-diagonal ce, nh entries each).  Right solve in place: X C = Y for the
// rows of X (rows x nh); left solve: Out = C^{-1} V for the first *kdyn
// columns of V (nh x k)
template <typename T>
void launch_bidiag_right_solve(int rows, int nh, T *X, int64_t ld, const T *cd, const T *ce, cudaStream_t st);
template <typename T>
void launch_bidiag_left_solve(int nh, const T *V, int64_t ldv, const int *kdyn, int kmax, const T *cd, const T *ce,
                              T *Out, int64_t ldo, cudaStream_t st);

// small dense kernels (one CTA)
// Cholesky pass of CholeskyQR: R = chol(X^T X) from row-split partial Gram
// matrices; well_out / skip_in implement the skip of a second pass.  form
// (fp32): 0 = by 16-column block rows, 1 = one elimination step per barrier
template <typename T>
void launch_chol(const T *partialG, int splits, int kmax, const int *kdyn, T *R, T *Rinv, const T *Rprev, T *Rtot,
                 int ldr, int *well_out, const int *skip_in, cudaStream_t st, int *stats = nullptr, int form = 0);
// ctrl (optional): skip rotations that cannot change SVT_{ctrl->theta_L};
// stats (optional): calls and sweeps are added to stats[0], stats[1];
// Us, svt (optional): the SVT of launch_svt_small fused into the epilogue
// CholeskyQR2 of X (rows x k, k = *kdyn <= KM, ld KM) in one thread-block
// cluster launch (k_small.cu): Q, and Rout (if given) with X = Q Rout; Q1, G,
// R1, R1i, R2, R2i are workspace (ld KM), well receives the first pass's
// skip flag, stats counts factorisations.  false (nothing launched): the
// fused form is not available and the caller runs the multi-launch form.
bool launch_cholqr2_cluster(int rows, const float *X, float *Q, float *Q1, int KM, const int *kdyn, float *G,
                            float *R1, float *R1i, float *R2, float *R2i, float *Rout, int *well, int *stats,
                            cudaStream_t st);
// The second CholeskyQR pass of X (rows x k, ld KM) after a first pass that
// left Rt = R1, Rti = R1^{-1} and the flag well (k_small.cu): nothing when
// *well is set, else Rt <- R2 Rt, Rti <- Rti R2^{-1} with R2 the Cholesky
// factor of the Gram matrix of X R1^{-1}.  Q1 (rows x KM), Gp (16 slices of
// KM x KM), G, R2, R2i (KM x KM): workspace; ticket: a zeroed counter that
// the launch leaves zeroed.  fp32.
// X^T X of a tall block X (rows x k, ld KM, k = *kdyn) as partial slices by row
// ranges (k_small.cu), loading only the live columns; returns the slice count
int launch_gram_rows(int rows, const float *X, int KM, const int *kdyn, float *part, cudaStream_t st);
void launch_cqr_pass2(int rows, const float *X, float *Q1, int KM, const int *kdyn, float *Rt, float *Rti,
                      const int *well, float *Gp, float *G, float *R2, float *R2i, unsigned *ticket, int *stats,
                      cudaStream_t st);
template <typename T>
void launch_jacobi(const T *Rz, int ldr, const int *kdyn, T *Ut, T *Wt, T *sig, int kmax, const Ctrl *ctrl,
                   cudaStream_t st, int *stats = nullptr, T *Us = nullptr, Ctrl *svt = nullptr, int lanes = 16,
                   int check = 0);
template <typename T>
void launch_svt_small(const T *Ut, const T *sig, int ldr, Ctrl *ctrl, T *Us, double *sig64, cudaStream_t st);
// all_cols = 1: fill columns [0, ctrl->k); else columns [ctrl->k, ctrl->k_next)
// and the columns whose sig is exactly zero
template <typename T>
void launch_fill_random(T *Omega, int64_t ldo, int rows, const Ctrl *ctrl, int all_cols, const T *sig, int kmax,
                        uint64_t salt, cudaStream_t st);
// launch_fill_random (columns [k, k_next) and zero-sigma columns of Omega) and
// launch_prolong (B = R Omega for the columns c < r_new) in one launch
template <typename T>
void launch_fill_prolong(T *Omega, int64_t ldo, int rows_o, const Ctrl *ctrl, const T *sig, int kmax, uint64_t salt,
                         int n, T *B, int64_t ldb, const TransferDev<T> &tr, cudaStream_t st);
int small_kmax_f32();
int small_kmax_f64();

void launch_ctrl_begin(Ctrl *c, cudaStream_t st);
void launch_ctrl_end(Ctrl *c, cudaStream_t st);
void launch_ctrl_take_width(Ctrl *c, cudaStream_t st);  // k = k_next
void launch_ctrl_set_check(Ctrl *chk, const Ctrl *it, double mu_c, cudaStream_t st);

// ---------------------------------------------------------------------------
// batched solve: one persistent launch, one CTA per instance at a time
// ---------------------------------------------------------------------------
constexpr int BATCH_KB = 64;     // widest subspace of a batched instance
constexpr int BATCH_NMAX = 1024; // widest oriented instance (n <= m)
constexpr int BATCH_LEVELS = 4;

// Device descriptor of one instance.  Oriented sizes: m >= n; when the user's
// problem is wider than tall (trans) the CTA solves its transpose, reading
// the user's D and mask through oriented copies Dw, Qw it makes first.
struct BatchInst {
    int m, n, trans, levels;
    int nh[BATCH_LEVELS];
    double kappa[BATCH_LEVELS];
    const float *D;      // user D (user orientation), ldd
    int64_t ldd;
    const uint32_t *Q;   // user mask or nullptr, ldq
    int64_t ldq;
    float *Lout, *Sout;  // user outputs (user orientation) or nullptr
    int64_t ldl, lds;
    double lam, mu;
    // arena (oriented)
    float *Dw;           // m x n copy of D^T (trans only), leading dimension ld
    uint32_t *Qw;        // m x ldqw mask words of Q^T (trans with mask only)
    int64_t ldqw;
    float *S[2], *L[2], *M, *MH;
    int64_t ld, ldh;     // leading dimensions of m x n and m x nh[1] arrays
    float *A, *B, *Ac, *Bc, *Om, *Omf, *Y, *Qy, *Q1, *Z, *Qz;  // rows x BATCH_KB
    float *R1, *R1i, *R2, *R2i, *Rz, *Ut, *Wt, *Us, *sig;      // BATCH_KB x BATCH_KB (sig: BATCH_KB)
    const int *j0[BATCH_LEVELS], *clo[BATCH_LEVELS], *chi[BATCH_LEVELS];
    const float *w0[BATCH_LEVELS], *w1[BATCH_LEVELS];
};

struct BatchResult {
    int status, iters, checks, rank, final_level, level_iters[BATCH_LEVELS];
    double relkkt, mu0, pqd;
    long long cycles[4];  // SM clock cycles per phase (CPCP_PHASE_* order)
    long long svt_cycles[4];  // the SVT phase split: products with M, CholeskyQR, Jacobi, factor products
};

struct BatchOpts {
    int max_iter, check_every, p, q, qc;
    int early;  // coarse-gradient test also at a coarse level's first iteration
    int tile;   // CTA GEMM output tiles for N > 32: 0 = 64 x 64, 1 = 128 x 64
    double eta, ratio, tol;
    uint64_t seed;
};

// Launch the persistent kernel with nt threads per CTA (256 or 512) over
// `count` instances taken in the order `order`; `next` is a zeroed counter.
// Returns cudaSuccess or the launch error.
cudaError_t launch_batched(const BatchInst *inst, BatchResult *res, const int *order, int count, int *next,
                           const BatchOpts &o, int nt, cudaStream_t st);
int batched_grid(int nt);  // CTAs of the persistent launch (all resident)

// unrolled (differentiable) iteration, fp32
void launch_unroll_step(int m, int n, const float *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const float *Lk,
                        const float *Lp, const float *Sk, const float *Sp, int64_t ld, float beta, float thS,
                        float *Sout, float *XL, cudaStream_t st);
int launch_unroll_adjoint(int m, int n, const float *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const float *Lk,
                          const float *Lp, const float *Sk, const float *Sp, int64_t ld, double beta, float thS,
                          const float *gXL, double *gLn, double *gSn, double *gLp, double *gSp, double *dD,
                          float *gL32, double *part, cudaStream_t st);
void launch_widen(int m, int n, const float *x, int64_t lx, double *y, int64_t ly, cudaStream_t st);
void launch_narrow(int m, int n, const double *x, int64_t lx, float *y, int64_t ly, cudaStream_t st);
void launch_row_prolong(int m, int n, int nh, const float *Y, int64_t ldy, const TransferDev<float> &tr, float *out,
                        int64_t ldo, cudaStream_t st);
int launch_full_svd(int m, int q, const float *M, int64_t ldm, float *U, int64_t ldu, float *V, int64_t ldv,
                    double *sig, float *X, float *Vc, double *nrm, int *pos, void *gs, int *err, cudaStream_t st);
size_t full_svd_sync_bytes();
void launch_svt_right(int q, const double *sig, const float *V, int64_t ldv, double theta, float *Bf, int64_t ldb,
                      cudaStream_t st);
int launch_svt_adjoint_core(int q, const float *A, int64_t lda, const double *sig, double theta, float *B, int64_t ldb,
                            double *gth_part, cudaStream_t st);
void launch_svt_adjoint_combine(int m, int q, const float *T, const float *P, const float *W, int64_t ld,
                                const double *sig, double theta, float *Z, cudaStream_t st);
void launch_unroll_scalars(const double *gthL_part, int nL, const double *gthS_part, int nS, double lam, double mu_k,
                           double dmu_k, double *out, cudaStream_t st);

// tensor-core (tcgen05) BF16 contractions of the mixed-precision path
int umma_pad_rows(int rows);  // rows rounded up to the 128-row tile
int umma_pad_k(int k);        // K rounded up to the 64-element stage
// BF16 copies of fp32 X (rows x cols): Xb (rows_b x ldb, same orientation)
// and/or Xt (rows_t x ldt, transposed); padding is written with zeros.
void launch_bf16_pair(int rows, int cols, const float *X, int64_t ldx, __nv_bfloat16 *Xb, int rows_b, int64_t ldb,
                      __nv_bfloat16 *Xt, int rows_t, int64_t ldt, cudaStream_t st);
// split-K partials of A B^T (A rows_pad x kpad, B nrows_b x kpad, both BF16
// K-major, zero padded) for the first *kdyn columns; returns the number of
// splits (partial: splits x rows x ldp fp32) or -1 if no tensor map could be made
int launch_umma_tn(int rows, int rows_pad, int kpad, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                   int nrows_b, int64_t ldb, int nbox, const int *kdyn, float *partial, int ldp, int max_splits,
                   int *err, cudaStream_t st);

}  // namespace cpcp
