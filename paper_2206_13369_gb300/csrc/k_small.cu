// k_small.cu -- the k x k stages of the subspace-iteration SVD and the
// per-iteration scalar schedule.  Each runs as a single CTA with its matrices
// in shared memory (k <= small_kmax<T>()).
//
//   chol      Gram reduction + Cholesky of the column-equilibrated Gram matrix
//             (CholeskyQR pass): X = Q R with Q = X R^{-1}.  Columns that are
//             numerically dependent are dropped (zero column in Q, zero row
//             in R) instead of breaking down.
//   jacobi    one-sided Jacobi SVD of the small triangular factor: the core
//             SVD of the Rayleigh-Ritz step, with singular values sorted.
//   svt_small singular value thresholding on the factors (Sec. 2.1, Alg. 1 /
//             Sec. 3.2): keeps sigma > theta, scales the kept left vectors by
//             sigma - theta, and picks the next subspace width.
//   ctrl      momentum weight, continuation weight and thresholds.
#include <cfloat>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace cpcp {

template <typename T>
constexpr int small_kmax()
{
    return sizeof(T) == 4 ? 128 : 80;
}

namespace {

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ float eps_of<float>()
{
    return FLT_EPSILON;
}
template <>
__device__ __forceinline__ double eps_of<double>()
{
    return DBL_EPSILON;
}

// 1/sqrt(x) for a threshold test (a few units of rounding are irrelevant)
__device__ __forceinline__ float rsqrt_of(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_of(double x) { return rsqrt(x); }
// 1/sqrt(y) for y in [1, 2]: the hardware estimate and one Newton step
// c <- c (3 - y c^2) / 2, which brings it to about one unit of rounding
__device__ __forceinline__ float rsqrt_nr(float y)
{
    float c = rsqrtf(y);
    return c * fmaf(-0.5f * y, c * c, 1.5f);
}
__device__ __forceinline__ double rsqrt_nr(double y) { return 1.0 / sqrt(y); }
// quotient for a rotation angle (denominator of magnitude at least |x|)
__device__ __forceinline__ float fast_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double fast_div(double x, double y) { return x / y; }

// ---------------------------------------------------------------------------
// Cholesky pass of CholeskyQR
// ---------------------------------------------------------------------------
constexpr int CHOL_NT = 512;

// Gram reduction + equilibrated Cholesky R = chol(X^T X) (upper) and its
// inverse.  well_out (optional): set to 1 when the equilibrated Gram matrix is
// within 0.5 of the identity in Frobenius norm: X D^{-1} is then well enough
// conditioned (kappa^2 <= 3) that one CholeskyQR pass is accurate to a few
// units of rounding and a second pass can be skipped.  skip_in (optional):
// when *skip_in is set this pass is not needed; R = I, Rinv = I, Rtot = Rprev.
// Rtot = R Rprev when Rprev is given.  A column whose pivot is not positive is
// dropped: zero row in R, zero column in Rinv (zero column of Q).  stats
// (optional) counts the factorisations run.
//
// The factorisation is right-looking: step j eliminates column j from the
// trailing upper triangle of G with the column operation E_j = I - e_j u_j^T
// (u_j = G[j][j+1:] / G[j][j]) and, in the same step, applies E_j to W
// (W = E_0 E_1 ... E_j).  At the end G = U^T P^2 U with U = W^{-1} unit upper
// triangular and P the pivots' square roots, so R = P U (row j of R is
// G[j][j:] / P_j) and R^{-1} = W P^{-1}.
//
// G and W live together in registers as one k x k array S: G in the upper
// triangle (with the pivots on the diagonal) and W^T in the strict lower one
// (S[x][y] = W[y][x] for x > y).  Thread (tr, tc) = (tid / 32, tid % 32) owns
// rows tr + 16 a and columns tc + 32 b.  Step j updates the positions (x, y)
// with x > j and either y <= j (W) or y >= x (G), in both cases by
// S[x][y] -= S[j][x] S'[j][y] / S[j][j] with S'[j][j] = 1: the step reads the
// single row j of S, which its owners publish into a double-buffered shared
// row at the end of step j - 1, so a step costs one barrier.  (A blocked
// variant with 16-column panels, one warp per diagonal block, measured about
// twice as slow at k = 60: its serial diagonal-block and triangular-solve
// chains leave the SM idle behind the barriers.)
template <typename T>
__device__ __forceinline__ T chol_gram_entry(const T *__restrict__ partial, int splits, int64_t slice, int kmax, int p,
                                             int c)
{
    // row-split partial sums in a fixed order (four independent chains keep
    // several loads in flight)
    const T *src = partial + (int64_t)p * kmax + c;
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int q = 0;
    for (; q + 3 < splits; q += 4) {
        s0 += src[q * slice];
        s1 += src[(q + 1) * slice];
        s2 += src[(q + 2) * slice];
        s3 += src[(q + 3) * slice];
    }
    for (; q < splits; q++) s0 += src[q * slice];
    return (s0 + s1) + (s2 + s3);
}

template <typename T, int RG, int RA, int CB, int NT = CHOL_NT>
__device__ __forceinline__ void chol_body(const T *__restrict__ partial, int splits, int kmax, int k,
                                          T *__restrict__ R, T *__restrict__ Rinv, const T *__restrict__ Rprev,
                                          T *__restrict__ Rtot, int ldr, int *well_out, T *sm, double *red)
{
    // RG warps take part in the elimination: thread (tr, tc) = (warp, lane)
    // owns rows tr + RG a (a < RA) and columns tc + 32 b (b < CB)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tr = warp, tc = lane;
    const bool active = warp < RG;
    T *d = sm;              // column scales of the equilibration
    T *piv = d + k;         // square roots of the pivots (0 = dropped)
    T *rows2 = piv + k;     // 2 x (k + 1): row j of S and, at [k], 1 / S[j][j] (0 = dropped)
    const int rl = k + 1;
    const int64_t slice = (int64_t)kmax * kmax;
    const T tol = eps_of<T>() * eps_of<T>();

    for (int c = tid; c < k; c += NT) {
        const T g = chol_gram_entry(partial, splits, slice, kmax, c, c);
        d[c] = (g > T(0) && isfinite(g)) ? sqrt(g) : T(0);
    }
    __syncthreads();

    T S[RA][CB];
    uint32_t upper[RA];  // bit b: position (a, b) is in the upper triangle (G), else W^T
    double defect = 0.0;
#pragma unroll
    for (int a = 0; a < RA; a++) {
        const int x = tr + RG * a;
        upper[a] = 0;
#pragma unroll
        for (int b = 0; b < CB; b++) {
            const int y = tc + 32 * b;
            T v = T(0);
            if (active && x < k && y < k && x <= y) {
                upper[a] |= 1u << b;
                const T dx = d[x], dy = d[y];
                v = (dx > T(0) && dy > T(0)) ? chol_gram_entry(partial, splits, slice, kmax, x, y) / dx / dy : T(0);
                const T ev = v - (x == y ? T(1) : T(0));
                defect += (x == y ? 1.0 : 2.0) * (double)(ev * ev);  // both triangles of the symmetric matrix
                if (x == 0 && y == 0) {
                    const bool dj = !(v > tol);
                    rows2[k] = dj ? T(0) : T(1) / v;
                    piv[0] = dj ? T(0) : sqrt(v);
                }
            }
            if (active && x == 0 && y < k) rows2[y] = v;  // row 0 of S for step 0
            S[a][b] = v;  // lower triangle: W^T = 0 off the diagonal
        }
    }
    defect = warp_sum(defect);
    if (lane == 0) red[warp] = defect;
    __syncthreads();
    if (tid == 0 && well_out != nullptr) {
        double tot = 0.0;
        for (int q = 0; q < NT / 32; q++) tot += red[q];
        *well_out = tot <= 0.25 ? 1 : 0;
    }

    // Only a non-positive (or denormal) pivot drops a column; a tiny positive
    // pivot gives a noise direction that the next CholeskyQR pass cleans up.
    // The owner of the next diagonal position publishes its reciprocal and
    // square root with the row, so a step reads one row and one scalar.  (Two
    // eliminations per barrier, each thread bringing the entries of row j + 1
    // it needs through step j itself, measured the same: the step is bound by
    // its per-position work, not by the barrier.)
    if (active) {
        for (int j = 0; j < k; j++) {
            const T *rw = rows2 + (j & 1) * rl;
            T *rn = rows2 + ((j + 1) & 1) * rl;
            const T inv = rw[k];
            T rxi[RA], rx[RA], cy[CB], cyi[CB];
            bool rowact[RA], selw[CB];
#pragma unroll
            for (int a = 0; a < RA; a++) {
                const int x = tr + RG * a;
                rowact[a] = x > j && x < k;
                rx[a] = rowact[a] ? rw[x] : T(0);  // G[j][x]
                rxi[a] = rx[a] * inv;
            }
#pragma unroll
            for (int b = 0; b < CB; b++) {
                const int y = tc + 32 * b;
                selw[b] = y <= j;
                cy[b] = y == j ? T(1) : (y < k ? rw[y] : T(0));  // G[j][y] (y > j) or W[y][j] (y <= j)
                cyi[b] = cy[b] * inv;
            }
#pragma unroll
            for (int a = 0; a < RA; a++) {
                if (!rowact[a]) continue;
#pragma unroll
                for (int b = 0; b < CB; b++) {
                    if (selw[b])
                        S[a][b] -= cyi[b] * rx[a];  // W[y][x] -= (W[y][j] / p_j) G[j][x]
                    else if ((upper[a] >> b) & 1u)
                        S[a][b] -= rxi[a] * cy[b];  // G[x][y] -= (G[j][x] / p_j) G[j][y]
                }
            }
#pragma unroll
            for (int a = 0; a < RA; a++) {
                const int x = tr + RG * a;
                if (x != j + 1) continue;
#pragma unroll
                for (int b = 0; b < CB; b++) {
                    const int y = tc + 32 * b;
                    if (y < k) rn[y] = S[a][b];
                    if (y == x) {
                        const T pv = S[a][b];
                        const bool dj = !(pv > tol);
                        rn[k] = dj ? T(0) : T(1) / pv;
                        piv[x] = dj ? T(0) : sqrt(pv);
                    }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(RG * 32) : "memory");
        }
    }
    __syncthreads();

    // undo the equilibration: R = Rt D with Rt = P U (row i of Rt is
    // G[i][i:] / P_i), R^{-1} = D^{-1} Rt^{-1} = D^{-1} W P^{-1} (dropped columns
    // zero); then Rtot = R Rprev
    T *Rs = rows2 + 2 * rl;     // k x (k + 1): R (upper), for Rtot
    T *Ps = Rs + k * (k + 1);   // k x (k + 1): Rprev
    const int ld = k + 1;
    if (active) {
#pragma unroll
        for (int a = 0; a < RA; a++) {
            const int x = tr + RG * a;
            if (x >= k) continue;
#pragma unroll
            for (int b = 0; b < CB; b++) {
                const int y = tc + 32 * b;
                if (y >= k) continue;
                if (x < y) {
                    const T p_x = piv[x], rx_ = p_x > T(0) ? T(1) / p_x : T(0);
                    const T rv = S[a][b] * rx_ * d[y];
                    R[(int64_t)x * ldr + y] = rv;
                    R[(int64_t)y * ldr + x] = T(0);
                    Rinv[(int64_t)y * ldr + x] = T(0);
                    if (Rprev != nullptr) {
                        Rs[x * ld + y] = rv;
                        Rtot[(int64_t)y * ldr + x] = T(0);
                    }
                } else if (x == y) {
                    const T p_x = piv[x];
                    const T rv = p_x * d[x];
                    R[(int64_t)x * ldr + x] = rv;
                    Rinv[(int64_t)x * ldr + x] = (p_x > T(0) && d[x] > T(0)) ? T(1) / p_x / d[x] : T(0);
                    if (Rprev != nullptr) Rs[x * ld + x] = rv;
                } else {
                    // S[x][y] = W[y][x]: entry (y, x) of R^{-1} = W[y][x] / P_x / d_y
                    Rinv[(int64_t)y * ldr + x] = (piv[x] > T(0) && d[y] > T(0)) ? S[a][b] / piv[x] / d[y] : T(0);
                }
            }
        }
    }
    if (Rprev == nullptr) return;
    for (int idx = tid; idx < k * k; idx += NT) {
        const int i = idx / k, c = idx - (idx / k) * k;
        Ps[i * ld + c] = Rprev[(int64_t)i * ldr + c];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        if (y < x) continue;
        T s = T(0);
        for (int p = x; p <= y; p++) s = fma(Rs[x * ld + p], Ps[p * ld + y], s);
        Rtot[(int64_t)x * ldr + y] = s;
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) chol_kernel(const T *__restrict__ partial, int splits, int kmax,
                                                       const int *kdyn, T *__restrict__ R, T *__restrict__ Rinv,
                                                       const T *__restrict__ Rprev, T *__restrict__ Rtot, int ldr,
                                                       int *well_out, const int *skip_in, int *stats)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[NT / 32];
    const int k = *kdyn;
    const int tid = threadIdx.x;
    if (skip_in != nullptr && *skip_in) {
        for (int idx = tid; idx < k * k; idx += NT) {
            int i = idx / k, c = idx % k;
            R[(int64_t)i * ldr + c] = (i == c) ? T(1) : T(0);
            Rinv[(int64_t)i * ldr + c] = (i == c) ? T(1) : T(0);
            if (Rtot != nullptr) Rtot[(int64_t)i * ldr + c] = Rprev[(int64_t)i * ldr + c];
        }
        return;
    }
    if (stats != nullptr && tid == 0) atomicAdd(stats, 1);
    T *sm = reinterpret_cast<T *>(smraw);
    // 16 warps x rows per warp x columns per lane: 4 x 2 covers k <= 64, 8 x 4
    // covers k <= 128.  (With 4 warps and 32 positions per thread a step took
    // three times as long: the step is latency-bound, and more warps hide it.)
    // NT / 32 warps in the elimination: 512 threads with 8 positions each, or
    // 1024 threads with 4 (k <= 64) or 16 (k <= 128) positions each
    if constexpr (NT == 1024) {
        if (k <= 64)
            chol_body<T, 32, 2, 2, NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, sm, red);
        else
            chol_body<T, 32, 4, 4, NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, sm, red);
    } else {
        if (k <= 64)
            chol_body<T, 16, 4, 2, NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, sm, red);
        else
            chol_body<T, 16, 8, 4, NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, sm, red);
    }
}

// ---------------------------------------------------------------------------
// The same factorisation in fp32 with column quarters per thread (k <= 64)
// ---------------------------------------------------------------------------
// Thread (q, y) = (tid / 64, tid % 64) of the 256 owns rows 16q .. 16q + 15
// of column y of S in registers (rows unrolled), so a step needs no
// per-position index logic: at step j the owners of columns y > j eliminate
// rows j < x <= y of the upper triangle (G[x][y] -= G[j][x] G[j][y] / p_j),
// and the owners of columns y <= j update every row x > j of W^T (W[y][x] -=
// W[y][j] G[j][x] / p_j, W[j][j] = 1).  Both are S[x][y] -= c_y S[j][x] with
// one coefficient per column, over rows (j, xmax(y)].  Row j of S goes
// through a double-buffered shared row, with a copy zeroed up to column j
// that serves as G[j][x] for x > j; one barrier per step.  A quarter wholly
// at or above row j skips the step (warp-uniform).  Wider subspaces
// (64 < k <= 128) take chol_body with 256 threads.  Same outputs, pivot
// rule, equilibration and well-conditioning test as chol_body.
constexpr int CQ_NT = 256;

size_t chol_q_smem(int kmax)
{
    const size_t narrow = (size_t)(2 * kmax * (kmax + 1) + 2 * kmax + 4 * 64 + 2) * sizeof(float) + 64;
    const size_t wide = (size_t)(4 * kmax + 2) * sizeof(float) + (size_t)2 * kmax * (kmax + 1) * sizeof(float) + 16;
    return std::max(narrow, wide);
}

__global__ void __launch_bounds__(CQ_NT, 1) chol_q_kernel(const float *__restrict__ partial, int splits, int kmax,
                                                           const int *kdyn, float *__restrict__ R,
                                                           float *__restrict__ Rinv, const float *__restrict__ Rprev,
                                                           float *__restrict__ Rtot, int ldr, int *well_out,
                                                           const int *skip_in, int *stats)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CQ_NT / 32];
    const int k = *kdyn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (skip_in != nullptr && *skip_in) {
        for (int idx = tid; idx < k * k; idx += CQ_NT) {
            const int i = idx / k, c = idx % k;
            R[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            Rinv[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            if (Rtot != nullptr) Rtot[(int64_t)i * ldr + c] = Rprev[(int64_t)i * ldr + c];
        }
        return;
    }
    if (stats != nullptr && tid == 0) atomicAdd(stats, 1);
    if (k > 64) {
        chol_body<float, 8, 16, 4, CQ_NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out,
                                          reinterpret_cast<float *>(smraw), red);
        return;
    }
    // shared: row buffers (16-byte aligned), then Gs and Ps (kmax x (kmax + 1)), scales, pivots
    float *rowf = reinterpret_cast<float *>(smraw);  // 2 x 64: row j of S
    float *rowg = rowf + 2 * 64;                      // 2 x 64: row j of S, zero in columns <= j
    const int ldg = kmax + 1;
    float *Gs = rowg + 2 * 64;     // equilibrated Gram (upper), the final columns of S, then R (upper)
    float *Ps = Gs + kmax * ldg;   // Rprev
    float *dsc = Ps + kmax * ldg;  // column scales
    float *piv = dsc + kmax;       // square roots of the pivots (0 = dropped)
    float *rinv = piv + kmax;      // 2: 1 / pivot of row j (0 = dropped)
    const int64_t slice = (int64_t)kmax * kmax;
    const float tol = FLT_EPSILON * FLT_EPSILON;

    // column scales, then the equilibrated Gram matrix and its distance from I
    for (int c = tid; c < k; c += CQ_NT) {
        const float g = chol_gram_entry(partial, splits, slice, kmax, c, c);
        dsc[c] = (g > 0.f && isfinite(g)) ? sqrtf(g) : 0.f;
    }
    for (int c = tid; c < 4 * 64; c += CQ_NT) rowf[c] = 0.f;  // rowf and rowg
    __syncthreads();
    // (eight entries per thread at a time, every load of a batch issued before
    // the first is used: the partials sit in L2, and one round trip per entry
    // was most of a small factorisation's time)
    double defect = 0.0;
    for (int base = 0; base < k * k; base += 8 * CQ_NT) {
        float acc[8];
        const float *src[8];
        bool use[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = base + u * CQ_NT + tid;
            const int x = idx / k, y = idx - (idx / k) * k;
            use[u] = idx < k * k && x <= y && dsc[x] > 0.f && dsc[y] > 0.f;
            src[u] = partial + (use[u] ? (int64_t)x * kmax + y : 0);
            acc[u] = 0.f;
        }
        int q = 0;
        for (; q + 4 <= splits; q += 4) {
            float v[8][4];
#pragma unroll
            for (int u = 0; u < 8; u++)
#pragma unroll
                for (int t = 0; t < 4; t++) v[u][t] = use[u] ? src[u][(q + t) * slice] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] += (v[u][0] + v[u][1]) + (v[u][2] + v[u][3]);
        }
        for (; q < splits; q++)
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] += use[u] ? src[u][q * slice] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = base + u * CQ_NT + tid;
            const int x = idx / k, y = idx - (idx / k) * k;
            if (idx >= k * k || x > y) continue;
            const float v = use[u] ? acc[u] / dsc[x] / dsc[y] : 0.f;
            Gs[x * ldg + y] = v;
            const float ev = v - (x == y ? 1.f : 0.f);
            defect += (x == y ? 1.0 : 2.0) * (double)(ev * ev);
        }
    }
    defect = warp_sum(defect);
    if (lane == 0) red[warp] = defect;
    if (Rprev != nullptr)
        for (int base = 0; base < k * k; base += 8 * CQ_NT) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int idx = base + u * CQ_NT + tid;
                const int i = idx / k, c = idx - (idx / k) * k;
                v[u] = idx < k * k ? Rprev[(int64_t)i * ldr + c] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int idx = base + u * CQ_NT + tid;
                const int i = idx / k, c = idx - (idx / k) * k;
                if (idx < k * k) Ps[i * ldg + c] = v[u];
            }
        }
    __syncthreads();
    if (tid == 0 && well_out != nullptr) {
        double tot = 0.0;
        for (int q = 0; q < CQ_NT / 32; q++) tot += red[q];
        *well_out = tot <= 0.25 ? 1 : 0;
    }

    const int y = tid & 63, q = tid >> 6, x0 = 16 * q;
    float S[16];
#pragma unroll
    for (int t = 0; t < 16; t++) S[t] = (y < k && x0 + t <= y) ? Gs[(x0 + t) * ldg + y] : 0.f;
    if (q == 0) {
        const float r0 = y < k ? S[0] : 0.f;
        rowf[y] = r0;
        rowg[y] = y > 0 ? r0 : 0.f;
        if (y == 0) rinv[0] = !(r0 > tol) ? 0.f : __frcp_rn(r0);
    }
    for (int j = 0; j < k; j++) {
        __syncthreads();
        const int b = j & 1;
        if (x0 + 15 > j && x0 < k) {
            const float inv = rinv[b];
            const float f = y == j ? 1.f : rowf[b * 64 + y];
            const float cf = f * inv;
            // rows (j, xmax] of this column change; none for columns >= k
            const int xmax = y >= k ? j : (y <= j ? k - 1 : y);
            const float4 *g4 = reinterpret_cast<const float4 *>(rowg + b * 64 + x0);
            float g[16];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float4 v = g4[u];
                g[4 * u] = v.x;
                g[4 * u + 1] = v.y;
                g[4 * u + 2] = v.z;
                g[4 * u + 3] = v.w;
            }
#pragma unroll
            for (int t = 0; t < 16; t++)
                if (x0 + t <= xmax) S[t] = fmaf(-cf, g[t], S[t]);
        }
        // publish row j + 1 (the owner of its diagonal: the pivot's reciprocal;
        // the pivot itself is kept and its square root taken after the loop).
        // S[jn - x0] by independent selects summed in a tree (exact: all but
        // one are zero), in asm the compiler cannot turn into an indexed
        // (local-memory) load, which would take S out of registers
        const int jn = j + 1;
        if (jn < k && (jn >> 4) == q) {
            float sel[16];
#pragma unroll
            for (int t = 0; t < 16; t++)
                asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, %3;\n\tselp.f32 %0, %1, 0f00000000, p;\n\t}"
                    : "=f"(sel[t])
                    : "f"(S[t]), "r"(x0 + t), "r"(jn));
#pragma unroll
            for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                for (int t = 0; t < w; t++) sel[t] += sel[t + w];
            const float pub = y >= k ? 0.f : sel[0];
            rowf[(b ^ 1) * 64 + y] = pub;
            rowg[(b ^ 1) * 64 + y] = y > jn ? pub : 0.f;
            if (y == jn) {
                const bool dj = !(pub > tol);
                rinv[b ^ 1] = dj ? 0.f : __frcp_rn(pub);
                piv[jn] = dj ? 0.f : pub;
            }
        }
    }
    if (q == 0 && y == 0) piv[0] = rinv[0] > 0.f ? S[0] : 0.f;
    __syncthreads();
    for (int c = tid; c < k; c += CQ_NT) piv[c] = sqrtf(piv[c]);
    // the columns back to shared memory (each thread its own quarter)
    if (y < k) {
#pragma unroll
        for (int t = 0; t < 16; t++)
            if (x0 + t < k) Gs[(x0 + t) * ldg + y] = S[t];
    }
    __syncthreads();
    // undo the equilibration (as in chol_body): R = P U D, R^{-1} = D^{-1} W P^{-1}
    for (int idx = tid; idx < k * k; idx += CQ_NT) {
        const int yy = idx / k, x = idx - (idx / k) * k;  // column yy of S, row x
        const float px = piv[x], dy = dsc[yy], sx = Gs[x * ldg + yy];
        if (x < yy) {
            const float rv = sx * (px > 0.f ? 1.f / px : 0.f) * dy;
            R[(int64_t)x * ldr + yy] = rv;
            R[(int64_t)yy * ldr + x] = 0.f;
            Rinv[(int64_t)yy * ldr + x] = 0.f;
            if (Rprev != nullptr) Rtot[(int64_t)yy * ldr + x] = 0.f;
        } else if (x == yy) {
            R[(int64_t)x * ldr + x] = px * dy;
            Rinv[(int64_t)x * ldr + x] = (px > 0.f && dy > 0.f) ? 1.f / px / dy : 0.f;
        } else {
            Rinv[(int64_t)yy * ldr + x] = (px > 0.f && dy > 0.f) ? sx / px / dy : 0.f;
        }
    }
    if (Rprev == nullptr) return;
    __syncthreads();
    // R (upper) into Gs for Rtot = R Rprev
    for (int idx = tid; idx < k * k; idx += CQ_NT) {
        const int x = idx / k, yy = idx - (idx / k) * k;
        if (yy < x) continue;
        const float px = piv[x], dy = dsc[yy];
        Gs[x * ldg + yy] = x == yy ? px * dy : Gs[x * ldg + yy] * (px > 0.f ? 1.f / px : 0.f) * dy;
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += CQ_NT) {
        const int x = idx / k, yy = idx - (idx / k) * k;
        if (yy < x) continue;
        float s = 0.f;
        for (int p = x; p <= yy; p++) s = fmaf(Gs[x * ldg + p], Ps[p * ldg + yy], s);
        Rtot[(int64_t)x * ldr + yy] = s;
    }
}

// ---------------------------------------------------------------------------
// The same factorisation in fp32 by 16-column block rows (k <= 128)
// ---------------------------------------------------------------------------
// Right-looking and blocked.  Block row J (rows c0 .. c0 + 15, c0 = 16 J) is
// eliminated by one warp in registers: lane l holds columns c0 + l + 32 s
// (s < SL) of those 16 rows, so a step j of the block takes the pivot from
// lane j by a shuffle, scales the lane's own entries of row j into u_j
// (U[j][y] = S[j][y] / p_j) and updates rows x > j of the block with the
// entries S[j][c0 + x] of lanes x: no barrier inside the block.  The 16
// finished rows (S and U) go to shared memory, and the whole CTA applies
// them to the trailing upper triangle in one rank-16 update
// (S[x][y] -= sum_j S[j][x] U[j][y], 4 x 4 register tiles), one barrier.
// W = U^{-1} (unit upper triangular) follows by block back substitution: each
// diagonal block inverted by its own warp, then the off-diagonal blocks block
// row by block row from the bottom, W_IJ = -W_II sum_{I<L<=J} U_IL W_LJ.  A
// pivot that is not positive (or below eps^2) drops its column: its U row
// is e_j and it updates nothing, as in the unblocked forms.  Same outputs,
// equilibration, pivot rule and well-conditioning test as chol_body; the
// rounding order differs.
constexpr int CB_NT = 256;

__host__ __device__ inline int cb_ld(int kmax) { return (kmax + 4 + 3) / 4 * 4; }

size_t chol_blk_smem(int kmax)
{
    const size_t ld = cb_ld(kmax);
    // Gs, Us, Ws (kmax x ld each), the block-row scratch (16 x ld), scales, pivots
    return (3 * (size_t)kmax * ld + 16 * ld + 2 * (size_t)kmax + 8) * sizeof(float) + 64;
}

// 1/p for a normal positive p: the hardware estimate and one Newton step
__device__ __forceinline__ float rcp_nr(float p)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
    return fmaf(r, fmaf(-p, r, 1.f), r);
}

// block row J of S (rows c0 .. c0 + nr - 1 of the trailing upper triangle in
// Gs) eliminated by one warp; its rows of S and U written back to Gs and Us,
// the pivots to piv (0 = dropped)
template <int SL>
__device__ __forceinline__ void cb_block_row(float *Gs, float *Us, float *piv, int ld, int k, int c0, float tol)
{
    const int lane = threadIdx.x & 31;
    float a[SL][16];
#pragma unroll
    for (int s = 0; s < SL; s++) {
        const int y = c0 + lane + 32 * s;
#pragma unroll
        for (int x = 0; x < 16; x++) a[s][x] = (y < k && c0 + x <= y) ? Gs[(c0 + x) * ld + y] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) {
        if (c0 + j >= k) break;  // uniform over the warp
        const float p = __shfl_sync(0xffffffffu, a[0][j], j);
        const bool drop = !(p > tol);
        const float inv = drop ? 0.f : rcp_nr(p);
        float u[SL];
#pragma unroll
        for (int s = 0; s < SL; s++) {
            u[s] = a[s][j] * inv;
            const int y = c0 + lane + 32 * s;
            if (y < k) {
                Gs[(c0 + j) * ld + y] = a[s][j];
                Us[(c0 + j) * ld + y] = y > c0 + j ? u[s] : (y == c0 + j ? 1.f : 0.f);
            }
        }
        if (lane == 0) piv[c0 + j] = drop ? 0.f : p;
        // rows x > j of the block: S[x][y] -= S[j][x] u_j[y] (positions below
        // the diagonal of the block are never read)
#pragma unroll
        for (int x = j + 1; x < 16; x++) {
            const float v = __shfl_sync(0xffffffffu, a[0][j], x);
#pragma unroll
            for (int s = 0; s < SL; s++) a[s][x] = fmaf(-v, u[s], a[s][x]);
        }
    }
}

template <int NT>
__device__ void chol_s_body(const float *__restrict__ partial, int splits, int kmax, int k, float *__restrict__ R,
                            float *__restrict__ Rinv, const float *__restrict__ Rprev, float *__restrict__ Rtot,
                            int ldr, int *well_out, unsigned char *smraw, double *red);

// (widths k <= 32 take the compact unblocked form below, chol_s_body:
// measured faster there, 27.7 -> 26.5 ms per video solve at k = 15, and
// slower at k = 60, where the blocked form's four block rows win)
__global__ void __launch_bounds__(CB_NT, 1) chol_blk_kernel(const float *__restrict__ partial, int splits, int kmax,
                                                             const int *kdyn, float *__restrict__ R,
                                                             float *__restrict__ Rinv, const float *__restrict__ Rprev,
                                                             float *__restrict__ Rtot, int ldr, int *well_out,
                                                             const int *skip_in, int *stats)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CB_NT / 32];
    const int k = *kdyn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (skip_in != nullptr && *skip_in) {
        for (int idx = tid; idx < k * k; idx += CB_NT) {
            const int i = idx / k, c = idx % k;
            R[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            Rinv[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            if (Rtot != nullptr) Rtot[(int64_t)i * ldr + c] = Rprev[(int64_t)i * ldr + c];
        }
        return;
    }
    if (stats != nullptr && tid == 0) atomicAdd(stats, 1);
    if (k <= 32) {
        chol_s_body<CB_NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, smraw, red);
        return;
    }
    const int ld = cb_ld(kmax);
    float *Gs = reinterpret_cast<float *>(smraw);  // S (upper); later R
    float *Us = Gs + (size_t)kmax * ld;            // U (unit upper); later R for Rtot
    float *Ws = Us + (size_t)kmax * ld;            // W = U^{-1}; later Rprev
    float *Ts = Ws + (size_t)kmax * ld;            // 16 x ld: sum_L U_IL W_LJ of one block row
    float *dsc = Ts + 16 * ld;                     // column scales
    float *piv = dsc + kmax;                       // pivots (0 = dropped); later their square roots
    const int64_t slice = (int64_t)kmax * kmax;
    const float tol = FLT_EPSILON * FLT_EPSILON;

    // column scales, the equilibrated Gram matrix (upper) and its distance from I
    for (int c = tid; c < k; c += CB_NT) {
        const float g = chol_gram_entry(partial, splits, slice, kmax, c, c);
        dsc[c] = (g > 0.f && isfinite(g)) ? sqrtf(g) : 0.f;
    }
    __syncthreads();
    double defect = 0.0;
    for (int base = 0; base < k * k; base += 8 * CB_NT) {
        float acc[8];
        const float *src[8];
        bool use[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = base + u * CB_NT + tid;
            const int x = idx / k, y = idx - (idx / k) * k;
            use[u] = idx < k * k && x <= y && dsc[x] > 0.f && dsc[y] > 0.f;
            src[u] = partial + (use[u] ? (int64_t)x * kmax + y : 0);
            acc[u] = 0.f;
        }
        int q = 0;
        for (; q + 4 <= splits; q += 4) {
            float v[8][4];
#pragma unroll
            for (int u = 0; u < 8; u++)
#pragma unroll
                for (int t = 0; t < 4; t++) v[u][t] = use[u] ? src[u][(q + t) * slice] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] += (v[u][0] + v[u][1]) + (v[u][2] + v[u][3]);
        }
        for (; q < splits; q++)
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] += use[u] ? src[u][q * slice] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int idx = base + u * CB_NT + tid;
            const int x = idx / k, y = idx - (idx / k) * k;
            if (idx >= k * k || x > y) continue;
            const float v = use[u] ? acc[u] / dsc[x] / dsc[y] : 0.f;
            Gs[x * ld + y] = v;
            const float ev = v - (x == y ? 1.f : 0.f);
            defect += (x == y ? 1.0 : 2.0) * (double)(ev * ev);
        }
    }
    defect = warp_sum(defect);
    if (lane == 0) red[warp] = defect;
    __syncthreads();
    if (tid == 0 && well_out != nullptr) {
        double tot = 0.0;
        for (int q = 0; q < CB_NT / 32; q++) tot += red[q];
        *well_out = tot <= 0.25 ? 1 : 0;
    }

    // elimination, block row by block row
    const int nb = (k + 15) >> 4;
    for (int J = 0; J < nb; J++) {
        const int c0 = 16 * J;
        if (warp == 0) {
            if (k - c0 <= 64)
                cb_block_row<2>(Gs, Us, piv, ld, k, c0, tol);
            else
                cb_block_row<4>(Gs, Us, piv, ld, k, c0, tol);
        }
        __syncthreads();
        const int t0 = c0 + 16;
        if (t0 >= k) break;
        // trailing update of the upper triangle, 4 x 4 tiles (xb <= yb)
        const int jn = 16;
        const int nt4 = (k - t0 + 3) >> 2;
        const int ntile = nt4 * (nt4 + 1) / 2;
        for (int e = tid; e < ntile; e += CB_NT) {
            int xb = 0, rem = e;
            while (rem >= nt4 - xb) {
                rem -= nt4 - xb;
                xb++;
            }
            const int yb = xb + rem;
            const int x = t0 + 4 * xb, y = t0 + 4 * yb;
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const float4 g = *reinterpret_cast<const float4 *>(Gs + (x + a) * ld + y);
                acc[a][0] = g.x;
                acc[a][1] = g.y;
                acc[a][2] = g.z;
                acc[a][3] = g.w;
            }
#pragma unroll 4
            for (int j = 0; j < jn; j++) {
                const float4 sx = *reinterpret_cast<const float4 *>(Gs + (c0 + j) * ld + x);
                const float4 uy = *reinterpret_cast<const float4 *>(Us + (c0 + j) * ld + y);
                const float sv[4] = {sx.x, sx.y, sx.z, sx.w}, uv[4] = {uy.x, uy.y, uy.z, uy.w};
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = fmaf(-sv[a], uv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; a++)
                *reinterpret_cast<float4 *>(Gs + (x + a) * ld + y) =
                    make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        }
        __syncthreads();
    }

    // W = U^{-1}: the diagonal blocks (warp J inverts block J, lane y its
    // column), zero below them
    for (int J = warp; J < nb; J += CB_NT / 32) {
        const int c0 = 16 * J, nr = min(16, k - c0);
        if (lane < nr) {
            const int y = c0 + lane;
            for (int i = lane + 1; i < nr; i++) Ws[(c0 + i) * ld + y] = 0.f;
            Ws[y * ld + y] = 1.f;
            for (int i = lane - 1; i >= 0; i--) {
                float sacc = 0.f;
                for (int c = i + 1; c <= lane; c++) sacc = fmaf(Us[(c0 + i) * ld + c0 + c], Ws[(c0 + c) * ld + y], sacc);
                Ws[(c0 + i) * ld + y] = -sacc;
            }
        }
    }
    __syncthreads();
    // off-diagonal blocks, block row I from the bottom: T = sum_{L > I} U_IL W_L,
    // then W_I = -W_II T (columns beyond block I)
    for (int I = nb - 2; I >= 0; I--) {
        const int i0 = 16 * I, t0 = i0 + 16, nc = k - t0;
        for (int e = tid; e < 16 * nc; e += CB_NT) {
            const int i = e / nc, y = t0 + (e - (e / nc) * nc);
            float sacc = 0.f;
            for (int c = t0; c <= y; c++) sacc = fmaf(Us[(i0 + i) * ld + c], Ws[c * ld + y], sacc);
            Ts[i * ld + y] = sacc;
        }
        __syncthreads();
        for (int e = tid; e < 16 * nc; e += CB_NT) {
            const int i = e / nc, y = t0 + (e - (e / nc) * nc);
            float sacc = 0.f;
            for (int c = i; c < 16; c++) sacc = fmaf(Ws[(i0 + i) * ld + i0 + c], Ts[c * ld + y], sacc);
            Ws[(i0 + i) * ld + y] = -sacc;
        }
        __syncthreads();
    }
    for (int c = tid; c < k; c += CB_NT) piv[c] = sqrtf(piv[c]);
    __syncthreads();

    // undo the equilibration: R = P U D (row x of P U is S[x][x:] / P_x), R^{-1} = D^{-1} W P^{-1}
    for (int idx = tid; idx < k * k; idx += CB_NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        const float px = piv[x], py = piv[y];
        float rv = 0.f, ri = 0.f;
        if (x < y) {
            rv = px > 0.f ? Gs[x * ld + y] / px * dsc[y] : 0.f;
            ri = (py > 0.f && dsc[x] > 0.f) ? Ws[x * ld + y] / py / dsc[x] : 0.f;
        } else if (x == y) {
            rv = px * dsc[x];
            ri = (px > 0.f && dsc[x] > 0.f) ? 1.f / px / dsc[x] : 0.f;
        }
        R[(int64_t)x * ldr + y] = rv;
        Rinv[(int64_t)x * ldr + y] = ri;
        if (Rprev != nullptr && x <= y) Us[x * ld + y] = rv;
    }
    if (Rprev == nullptr) return;
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += CB_NT) {
        const int i = idx / k, c = idx - (idx / k) * k;
        Ws[i * ld + c] = Rprev[(int64_t)i * ldr + c];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += CB_NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        float sacc = 0.f;
        if (x <= y)
            for (int p = x; p <= y; p++) sacc = fmaf(Us[x * ld + p], Ws[p * ld + y], sacc);
        Rtot[(int64_t)x * ldr + y] = sacc;
    }
}

// ---------------------------------------------------------------------------
// The same factorisation in fp32 with compact code (k <= 128)
// ---------------------------------------------------------------------------
// A one-CTA kernel runs most of its instructions once per launch, so each
// launch fetches its whole code from L2 (the kernels above unroll their
// register tiles into 167-665 KB of code, and a capture of the blocked one
// stalls on instruction fetch more than on anything else).  This form keeps
// S in shared memory and every loop rolled: the same right-looking
// elimination as chol_body (G in the upper triangle, W^T in the strict lower
// one, step j updating S[x][y] -= S[j][x] c_y / p_j for x > j and y <= j or
// y >= x, c_y = 1 at y = j and S[j][y] otherwise), warp w taking rows
// j + 1 + w, j + 1 + w + 16, ... and its lanes the columns, one barrier per
// step.  Same outputs, equilibration, pivot rule and well-conditioning test.
constexpr int CS_NT = 512;

size_t chol_s_smem(int kmax)
{
    // S (kmax x (kmax + 1)), Rprev staged for Rtot (same), scales, pivots
    return (size_t)(2 * kmax * (kmax + 1) + 2 * kmax + 8) * sizeof(float) + 64;
}

template <int NT>
__device__ void chol_s_body(const float *__restrict__ partial, int splits, int kmax, int k, float *__restrict__ R,
                            float *__restrict__ Rinv, const float *__restrict__ Rprev, float *__restrict__ Rtot,
                            int ldr, int *well_out, unsigned char *smraw, double *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ld = kmax + 1;
    float *S = reinterpret_cast<float *>(smraw);
    float *P = S + (size_t)kmax * ld;  // Rprev, then R for Rtot
    float *dsc = P + (size_t)kmax * ld;
    float *piv = dsc + kmax;
    const int64_t slice = (int64_t)kmax * kmax;
    const float tol = FLT_EPSILON * FLT_EPSILON;

    for (int c = tid; c < k; c += NT) {
        const float g = chol_gram_entry(partial, splits, slice, kmax, c, c);
        dsc[c] = (g > 0.f && isfinite(g)) ? sqrtf(g) : 0.f;
    }
    __syncthreads();
    // the equilibrated Gram matrix (upper; W^T = 0 below) and its distance from I
    double defect = 0.0;
    for (int idx = tid; idx < k * k; idx += NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        float v = 0.f;
        if (x <= y && dsc[x] > 0.f && dsc[y] > 0.f) {
            v = chol_gram_entry(partial, splits, slice, kmax, x, y) / dsc[x] / dsc[y];
            const float ev = v - (x == y ? 1.f : 0.f);
            defect += (x == y ? 1.0 : 2.0) * (double)(ev * ev);
        }
        S[x * ld + y] = v;
        if (Rprev != nullptr) P[x * ld + y] = Rprev[(int64_t)x * ldr + y];
    }
    defect = warp_sum(defect);
    if (lane == 0) red[warp] = defect;
    __syncthreads();
    if (tid == 0 && well_out != nullptr) {
        double tot = 0.0;
        for (int q = 0; q < NT / 32; q++) tot += red[q];
        *well_out = tot <= 0.25 ? 1 : 0;
    }

#pragma unroll 1
    for (int j = 0; j < k; j++) {
        const float p = S[j * ld + j];
        const bool drop = !(p > tol);
        if (tid == 0) piv[j] = drop ? 0.f : p;
        if (!drop) {
            const float inv = rcp_nr(p);
#pragma unroll 1
            for (int x = j + 1 + warp; x < k; x += NT / 32) {
                const float gx = S[j * ld + x] * inv;  // G[j][x] / p_j
#pragma unroll 1
                for (int y = lane; y < k; y += 32) {
                    if (y > j && y < x) continue;
                    const float cy = y == j ? 1.f : S[j * ld + y];
                    S[x * ld + y] = fmaf(-gx, cy, S[x * ld + y]);
                }
            }
        }
        __syncthreads();
    }
    for (int c = tid; c < k; c += NT) piv[c] = sqrtf(piv[c]);
    __syncthreads();

    // undo the equilibration: R = P U D (row x of P U is S[x][x:] / P_x),
    // R^{-1} = D^{-1} W P^{-1} with W[y][x] = S[x][y] below the diagonal
    for (int idx = tid; idx < k * k; idx += NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        const float px = piv[x], py = piv[y];
        float rv = 0.f, ri = 0.f;
        if (x < y) {
            rv = px > 0.f ? S[x * ld + y] * rcp_nr(px) * dsc[y] : 0.f;
            ri = (py > 0.f && dsc[x] > 0.f) ? S[y * ld + x] * rcp_nr(py) * rcp_nr(dsc[x]) : 0.f;
        } else if (x == y) {
            rv = px * dsc[x];
            ri = (px > 0.f && dsc[x] > 0.f) ? rcp_nr(px * dsc[x]) : 0.f;
        }
        R[(int64_t)x * ldr + y] = rv;
        Rinv[(int64_t)x * ldr + y] = ri;
    }
    if (Rprev == nullptr) return;
    __syncthreads();
    // R (upper) over the factorised S, for Rtot = R Rprev
    for (int idx = tid; idx < k * k; idx += NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        if (y < x) continue;
        const float px = piv[x];
        S[x * ld + y] = x == y ? px * dsc[x] : (px > 0.f ? S[x * ld + y] * rcp_nr(px) * dsc[y] : 0.f);
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += NT) {
        const int x = idx / k, y = idx - (idx / k) * k;
        float sacc = 0.f;
        if (x <= y)
            for (int q = x; q <= y; q++) sacc = fmaf(S[x * ld + q], P[q * ld + y], sacc);
        Rtot[(int64_t)x * ldr + y] = sacc;
    }
}

__global__ void __launch_bounds__(CS_NT, 1) chol_s_kernel(const float *__restrict__ partial, int splits, int kmax,
                                                           const int *kdyn, float *__restrict__ R,
                                                           float *__restrict__ Rinv, const float *__restrict__ Rprev,
                                                           float *__restrict__ Rtot, int ldr, int *well_out,
                                                           const int *skip_in, int *stats)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CS_NT / 32];
    const int k = *kdyn;
    const int tid = threadIdx.x;
    if (skip_in != nullptr && *skip_in) {
        for (int idx = tid; idx < k * k; idx += CS_NT) {
            const int i = idx / k, c = idx % k;
            R[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            Rinv[(int64_t)i * ldr + c] = (i == c) ? 1.f : 0.f;
            if (Rtot != nullptr) Rtot[(int64_t)i * ldr + c] = Rprev[(int64_t)i * ldr + c];
        }
        return;
    }
    if (stats != nullptr && tid == 0) atomicAdd(stats, 1);
    chol_s_body<CS_NT>(partial, splits, kmax, k, R, Rinv, Rprev, Rtot, ldr, well_out, smraw, red);
}

// ---------------------------------------------------------------------------
// CholeskyQR2 of a tall block in one thread-block cluster
// ---------------------------------------------------------------------------
// The two CholeskyQR passes (Gram, Cholesky, Q = X R^{-1}, twice) as one
// launch of a cluster of CQR_CL CTAs: every CTA takes a contiguous range of
// rows; the partial Gram matrices meet in distributed shared memory and are
// summed in rank order (each CTA sums one share of the entries); CTA 0 runs the
// equilibrated Cholesky (chol_body, the single-CTA factorisation above) and
// every CTA then forms its rows of Q.  The second pass runs only when the first
// found the equilibrated Gram matrix further than 0.5 from the identity (the
// flag is uniform over the cluster); otherwise Q = Q1 and R = R1 exactly, as
// in the multi-launch form.  fp32 only (k <= small_kmax<float>()).
constexpr int CQR_NT = CHOL_NT;

constexpr int CQR_CH = 64;  // rows of a staged chunk

// rows [c0, c0 + nr) of X (ld ldx, a multiple of 4), columns [0, k4), into the
// chunk buffer (ld k4 = round4(k)) with 16-byte loads
template <typename T>
__device__ __forceinline__ void cqr_load_chunk(const T *__restrict__ X, int64_t ldx, int c0, int nr, int k4, T *ch)
{
    const int q4 = k4 / 4;
    for (int e = threadIdx.x; e < nr * q4; e += CQR_NT) {
        const int r = e / q4, q = e - r * q4;
        *reinterpret_cast<float4 *>(ch + r * k4 + 4 * q) =
            *reinterpret_cast<const float4 *>(X + (int64_t)(c0 + r) * ldx + 4 * q);
    }
}

// Gp (k x k, ld k, upper 4 x 4 tiles; the rest zero) = X[r0:r1]^T X[r0:r1].
// Rows come through the chunk buffer; thread t takes tile t % T of the T upper
// tiles and the chunk rows g, g + G, ... (g = t / T, G = 512 / T groups); the
// groups' tiles are summed in order.  scratch: 512 x 16, ch: CQR_CH x round4(k).
template <typename T>
__device__ void cqr_gram(const T *__restrict__ X, int64_t ldx, int r0, int r1, int k, T *Gp, T *scratch, T *ch)
{
    const int tid = threadIdx.x;
    const int nb = (k + 3) / 4, ntile = nb * (nb + 1) / 2, k4 = 4 * nb;
    const int groups = max(1, CQR_NT / ntile);
    for (int e = tid; e < k * k; e += CQR_NT) Gp[e] = T(0);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = T(0);
    int bi = 0, bj = 0;
    const bool act = tid < ntile * groups;
    const int tile = tid % ntile, g = tid / ntile;
    {
        // tile -> (bi, bj) with bi <= bj, row by row of the upper block triangle
        int t = tile;
        while (t >= nb - bi) {
            t -= nb - bi;
            bi++;
        }
        bj = bi + t;
    }
    for (int c0 = r0; c0 < r1; c0 += CQR_CH) {
        const int nr = min(CQR_CH, r1 - c0);
        cqr_load_chunk<T>(X, ldx, c0, nr, k4, ch);
        __syncthreads();
        if (act) {
            for (int r = g; r < nr; r += groups) {
                const float4 u4 = *reinterpret_cast<const float4 *>(ch + r * k4 + 4 * bi);
                const float4 v4 = *reinterpret_cast<const float4 *>(ch + r * k4 + 4 * bj);
                const T u[4] = {u4.x, u4.y, u4.z, u4.w}, v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = fma(u[a], v[b], acc[a][b]);
            }
        }
        __syncthreads();
    }
    if (act) {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) scratch[(size_t)tid * 16 + a * 4 + b] = acc[a][b];
    }
    __syncthreads();
    for (int e = tid; e < ntile * 16; e += CQR_NT) {
        const int tl = e / 16, a = (e / 4) % 4, b = e % 4;
        T s = T(0);
        for (int q = 0; q < groups; q++) s += scratch[(size_t)(q * ntile + tl) * 16 + a * 4 + b];
        int t = tl, i = 0;
        while (t >= nb - i) {
            t -= nb - i;
            i++;
        }
        const int x = 4 * i + a, y = 4 * (i + t) + b;
        if (x < k && y < k) Gp[x * k + y] = s;
    }
    __syncthreads();
}

// Y[r0:r1] (ld ldy) = X[r0:r1] B with B (k x k) staged in shared memory with
// ld round4(k) and zero beyond k; X rows through the chunk buffer
template <typename T>
__device__ void cqr_apply(const T *__restrict__ X, int64_t ldx, int r0, int r1, int k, const T *Bs,
                          T *__restrict__ Y, int64_t ldy, T *ch)
{
    const int k4 = (k + 3) / 4 * 4, nc = k4 / 4;
    for (int c0 = r0; c0 < r1; c0 += CQR_CH) {
        const int nr = min(CQR_CH, r1 - c0);
        cqr_load_chunk<T>(X, ldx, c0, nr, k4, ch);
        __syncthreads();
        for (int tsk = threadIdx.x; tsk < nr * nc; tsk += CQR_NT) {
            const int r = tsk / nc, c = 4 * (tsk - (tsk / nc) * nc);
            const T *xr = ch + r * k4;
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = 0; i < k; i++) {
                const T xv = xr[i];
                const float4 b = *reinterpret_cast<const float4 *>(Bs + i * k4 + c);
                o.x = fma(xv, b.x, o.x);
                o.y = fma(xv, b.y, o.y);
                o.z = fma(xv, b.z, o.z);
                o.w = fma(xv, b.w, o.w);
            }
            T *yr = Y + (int64_t)(c0 + r) * ldy + c;
            if (c + 3 < k) {
                *reinterpret_cast<float4 *>(yr) = o;
            } else {
                yr[0] = o.x;
                if (c + 1 < k) yr[1] = o.y;
                if (c + 2 < k) yr[2] = o.z;
            }
        }
        __syncthreads();
    }
}

// the cluster's partial Gram matrices summed in rank order into G (global, ld ldg);
// CTA `rank` sums entries rank, rank + CL, ...
template <typename T>
__device__ void cqr_reduce(cg::cluster_group &cluster, T *Gp, int k, T *__restrict__ G, int ldg)
{
    const int cl = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    for (int e = rank * CQR_NT + threadIdx.x; e < k * k; e += cl * CQR_NT) {
        T s = T(0);
        for (int q = 0; q < cl; q++) s += cluster.map_shared_rank(Gp, q)[e];
        G[(int64_t)(e / k) * ldg + e % k] = s;
    }
}

// B (k x k, ld ldb) into shared memory with ld round4(k), zero-padded
template <typename T>
__device__ void cqr_stage(const T *__restrict__ B, int ldb, int k, T *Bs)
{
    const int k4 = (k + 3) / 4 * 4;
    for (int e = threadIdx.x; e < k * k4; e += CQR_NT) {
        const int i = e / k4, c = e - i * k4;
        Bs[e] = c < k ? B[(int64_t)i * ldb + c] : T(0);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void cqr_chol(const T *G, int KM, int k, T *R, T *Rinv, const T *Rprev, T *Rtot,
                                         int *well, T *ws, double *red)
{
    if (k <= 64)
        chol_body<T, 16, 4, 2>(G, 1, KM, k, R, Rinv, Rprev, Rtot, KM, well, ws, red);
    else
        chol_body<T, 16, 8, 4>(G, 1, KM, k, R, Rinv, Rprev, Rtot, KM, well, ws, red);
}

// X (rows x k, ld KM) -> Q (rows x k, ld KM) with orthonormal columns and, if
// Rout is given, X = Q Rout (k x k, ld KM); Q1, G, R1, R1i, R2, R2i: workspace
// (rows x KM and KM x KM, ld KM); well: the first pass's flag; stats: count of
// factorisations run.
template <typename T>
__global__ void __launch_bounds__(CQR_NT, 1)
    cholqr2_cluster_kernel(int rows, const T *__restrict__ X, T *__restrict__ Q, T *__restrict__ Q1, int KM,
                           const int *kdyn, T *G, T *R1, T *R1i, T *R2, T *R2i, T *Rout, int *well, int *stats,
                           int gp_off)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CQR_NT / 32];
    cg::cluster_group cluster = cg::this_cluster();
    const int cl = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const int k = *kdyn;
    if (k < 1) return;  // uniform over the cluster
    // Cholesky workspace; outside the factorisations it holds the Gram scratch
    // (512 x 16) and the chunk of staged rows (CQR_CH x round4(k))
    T *ws = reinterpret_cast<T *>(smraw);
    T *ch = ws + CQR_NT * 16;
    T *Gp = reinterpret_cast<T *>(smraw + gp_off);  // this CTA's partial Gram matrix (k x k), or a staged factor
    const int rpc = (rows + cl - 1) / cl;
    const int r0 = min(rows, rank * rpc), r1 = min(rows, r0 + rpc);

    // pass 1: Gram of X, Cholesky on CTA 0
    cqr_gram<T>(X, KM, r0, r1, k, Gp, ws, ch);
    cluster.sync();
    cqr_reduce<T>(cluster, Gp, k, G, KM);
    __threadfence();
    cluster.sync();
    if (rank == 0) {
        if (stats != nullptr && threadIdx.x == 0) atomicAdd(stats, 1);
        cqr_chol<T>(G, KM, k, R1, R1i, nullptr, nullptr, well, ws, red);
        __threadfence();
    }
    cluster.sync();
    const bool skip2 = *reinterpret_cast<volatile int *>(well) != 0;
    cqr_stage<T>(R1i, KM, k, Gp);
    cqr_apply<T>(X, KM, r0, r1, k, Gp, skip2 ? Q : Q1, KM, ch);
    if (skip2) {
        // second pass not needed: Q = Q1, R = R1
        if (Rout != nullptr && rank == 0)
            for (int e = threadIdx.x; e < k * k; e += CQR_NT)
                Rout[(int64_t)(e / k) * KM + e % k] = R1[(int64_t)(e / k) * KM + e % k];
        return;
    }
    __syncthreads();  // this CTA's rows of Q1 are written (and re-read below)

    // pass 2: Gram of Q1, Cholesky on CTA 0 (Rout = R2 R1)
    cqr_gram<T>(Q1, KM, r0, r1, k, Gp, ws, ch);
    cluster.sync();
    cqr_reduce<T>(cluster, Gp, k, G, KM);
    __threadfence();
    cluster.sync();
    if (rank == 0) {
        if (stats != nullptr && threadIdx.x == 0) atomicAdd(stats, 1);
        cqr_chol<T>(G, KM, k, R2, R2i, Rout != nullptr ? R1 : nullptr, Rout, nullptr, ws, red);
        __threadfence();
    }
    cluster.sync();
    cqr_stage<T>(R2i, KM, k, Gp);
    cqr_apply<T>(Q1, KM, r0, r1, k, Gp, Q, KM, ch);
}

// ---------------------------------------------------------------------------
// Gram matrix of a tall block by row ranges, loading only the live columns
// ---------------------------------------------------------------------------
// CTA b takes a contiguous range of rows of X (rows x k, ld KM) and writes
// X[r0:r1]^T X[r0:r1] (upper 4 x 4 tiles, zero below) as slice b of part (ld
// KM, slices KM x KM apart), which the Cholesky kernels sum in CTA order.  The
// rows come through shared memory 64 at a time, round4(k) columns each, so a
// narrow block (k = 15 on a 128-wide workspace) costs what its live columns
// cost.  fp32.
template <typename T>
__global__ void __launch_bounds__(CQR_NT) gram_rows_kernel(int rows, const T *__restrict__ X, int KM, const int *kdyn,
                                                            T *part)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = *kdyn;
    if (k < 1) return;
    const int nb = (int)gridDim.x, b = (int)blockIdx.x;
    const int rpc = (rows + nb - 1) / nb;
    const int r0 = min(rows, b * rpc), r1 = min(rows, r0 + rpc);
    const int k4 = (k + 3) / 4 * 4;
    T *scratch = reinterpret_cast<T *>(smraw);  // 512 x 16
    T *ch = scratch + CQR_NT * 16;              // CQR_CH x k4
    T *Gs = ch + CQR_CH * k4;                   // k x k
    cqr_gram<T>(X, KM, r0, r1, k, Gs, scratch, ch);
    T *slice = part + (int64_t)b * KM * KM;
    for (int e = threadIdx.x; e < k * k; e += CQR_NT) slice[(int64_t)(e / k) * KM + e % k] = Gs[e];
}


// ---------------------------------------------------------------------------
// The second CholeskyQR pass in one launch that returns at once when skipped
// ---------------------------------------------------------------------------
// After a first pass over X (rows x k, ld KM) that left Rt = R1, Rti = R1^{-1}
// (k x k, ld KM) and the well-conditioning flag.  When *well is set every CTA
// returns at once: the steady state then costs one launch instead of the
// three kernels of the multi-launch pass that each start only to find the
// flag.  Otherwise CTA b forms its rows of Q1 = X R1^{-1} (into the workspace
// Q1) and their Gram partial, written as slice b of Gp (ld KM); the last CTA
// to finish (a ticket counter, which it resets) sums the slices in CTA order
// into G, factorises it (chol_body: R2, R2^{-1}) and updates Rt <- R2 Rt and
// Rti <- Rti R2^{-1} in place.  Q = X Rti is left to the caller.  fp32.
template <typename T>
__global__ void __launch_bounds__(CQR_NT, 1)
    cqr_pass2_kernel(int rows, const T *__restrict__ X, T *Q1, int KM, const int *kdyn, T *Rt, T *Rti,
                     const int *well, T *Gp, T *G, T *R2, T *R2i, unsigned *ticket, int *stats, int gp_off)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[CQR_NT / 32];
    __shared__ int s_last;
    pdl_enter();
    if (*well) return;
    const int k = *kdyn;
    if (k < 1) return;
    T *ws = reinterpret_cast<T *>(smraw);  // Cholesky workspace, or the Gram scratch (512 x 16) and a row chunk
    T *ch = ws + CQR_NT * 16;
    T *Bs = reinterpret_cast<T *>(smraw + gp_off);  // R1^{-1} staged, then this CTA's Gram partial
    const int nb = (int)gridDim.x, b = (int)blockIdx.x, tid = threadIdx.x;
    const int rpc = (rows + nb - 1) / nb;
    const int r0 = min(rows, b * rpc), r1 = min(rows, r0 + rpc);

    cqr_stage<T>(Rti, KM, k, Bs);
    cqr_apply<T>(X, KM, r0, r1, k, Bs, Q1, KM, ch);
    __syncthreads();  // Bs is reused and this CTA's rows of Q1 are read back
    cqr_gram<T>(Q1, KM, r0, r1, k, Bs, ws, ch);
    T *slice = Gp + (int64_t)b * KM * KM;
    for (int e = tid; e < k * k; e += CQR_NT) slice[(int64_t)(e / k) * KM + e % k] = Bs[e];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(ticket, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid == 0) {
        *ticket = 0u;
        if (stats != nullptr) atomicAdd(stats, 1);
    }
    // the slices summed in CTA order (L2-coherent loads: other CTAs wrote them)
    for (int e = tid; e < k * k; e += CQR_NT) {
        const int64_t off = (int64_t)(e / k) * KM + e % k;
        T sacc = T(0);
        for (int q = 0; q < nb; q++) sacc += __ldcg(Gp + (int64_t)q * KM * KM + off);
        G[off] = sacc;
    }
    __threadfence();
    __syncthreads();
    cqr_chol<T>(G, KM, k, R2, R2i, Rt, Rt, nullptr, ws, red);
    __threadfence();
    __syncthreads();
    // Rti <- Rti R2^{-1} (both upper triangular), staged in shared memory
    T *A = ws, *Bm = Bs;
    for (int e = tid; e < k * k; e += CQR_NT) {
        const int64_t off = (int64_t)(e / k) * KM + e % k;
        A[e] = __ldcg(Rti + off);
        Bm[e] = __ldcg(R2i + off);
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += CQR_NT) {
        const int x = e / k, y = e - (e / k) * k;
        T sacc = T(0);
        if (x <= y)
            for (int p = x; p <= y; p++) sacc = fma(A[x * k + p], Bm[p * k + y], sacc);
        Rti[(int64_t)x * KM + y] = sacc;
    }
}

// ---------------------------------------------------------------------------
// one-sided Jacobi SVD of C = Rz^T (k x k): C = Ut diag(sig) Wt^T
// ---------------------------------------------------------------------------
constexpr int JAC_NT = 512;

__host__ __device__ constexpr int jac_ld(int k) { return (k + 31) / 32 * 32 + 8; }

// TPP consecutive lanes share one column pair (16 lanes for k <= 64, so the
// 32 pairs of a round fill the 512 threads; 8 lanes and up to 64 pairs for
// k <= 128); each lane keeps its EL elements of the two columns in registers
// between the dot product and the rotation.
template <typename T, int EL, int TPP>
__device__ __forceinline__ void jacobi_body(const T *__restrict__ Rz, int ldr, int k, T *__restrict__ Ut,
                                            T *__restrict__ Wt, T *__restrict__ sig, const Ctrl *ctrl, int *stats,
                                            T *__restrict__ Us, Ctrl *svt, T *sm, T *wmax, T *amax_p,
                                            int check = 0)
{
    // columns 8 banks apart (ld = 8 mod 32): with 8 lanes per pair the four
    // pairs a warp serves read 32 distinct banks
    const int ld = jac_ld(k);
    const int N = k + (k & 1);
    T *X = sm;          // X[c * ld + i]: column c of C
    T *V = X + k * ld;
    T *sv = V + k * ld; // squared column norms, then singular values
    int *pos = reinterpret_cast<int *>(sv + k);
    const int tid = threadIdx.x, nt = JAC_NT, lane = tid & 31, warp = tid >> 5;
    const T th2 = ctrl != nullptr ? T(ctrl->theta_L) * T(ctrl->theta_L) : T(-1);
    const int slot = tid / TPP, sub = tid % TPP, nslot = JAC_NT / TPP;
    const unsigned gmask = TPP == 32 ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));

    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        X[c * ld + i] = Rz[(int64_t)c * ldr + i];  // column c of Rz^T = row c of Rz
        V[c * ld + i] = (c == i) ? T(1) : T(0);
    }
    __syncthreads();

    // a pair is rotated when |x_p . x_q| exceeds the rounding bound of the
    // group dot product (k/TPP terms per lane in two chains + a shuffle tree)
    const T tol = T(2) * T((k + TPP - 1) / TPP + 4) * eps_of<T>();
    // columns whose norm is below the rounding noise of the largest one carry
    // no information; rotating them against large columns only moves noise
    const T negl = (T(4) * T(k) * eps_of<T>()) * (T(4) * T(k) * eps_of<T>());
    // a sweep whose largest rotated |g|/sqrt(ab) is delta leaves an
    // off-orthogonality of order delta^2 (Jacobi converges quadratically), so
    // a further sweep would only make rounding-level rotations.  While the
    // continuation weight is still above its final value the iterate moves
    // far more per iteration than an off-orthogonality of 1e-4 (the subspace
    // step itself is inexact), so the sweeps stop at delta <= 1e-2 there; at
    // the final weight (and in residual checks) they stop at 1e-4.
    const bool cont = ctrl != nullptr && ctrl->mu_k > ctrl->mu_bar * (1.0 + 1e-9);
    const T stop = cont ? T(1e-2) : min(sqrt(tol), T(1e-4));
    int sweeps = 0;
    for (int sweep = 0; sweep < 30; sweep++) {
        sweeps++;
        // exact squared norms at the start of each sweep; rotations then
        // update them by a' = a - t g, b' = b + t g (Rutishauser)
        for (int c = slot; c < k; c += nslot) {
            T s = T(0);
#pragma unroll
            for (int e = 0; e < EL; e++) {
                const int i = sub + TPP * e;
                if (i < k) s = fma(X[c * ld + i], X[c * ld + i], s);
            }
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
            if (sub == 0) sv[c] = s;
        }
        T mymax = T(0);  // largest rotated |g|/sqrt(ab) of this thread's pairs in the sweep
        __syncthreads();
        if (warp == 0) {
            T v = T(0);
            for (int c = lane; c < k; c += 32) v = max(v, sv[c]);
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) *amax_p = v;
        }
        __syncthreads();
        const T small = negl * *amax_p;
        // round-robin (circle) schedule: slot 0 holds column 0, slot s > 0
        // holds column 1 + (s - 1 + round) mod (N - 1); slot t meets N-1-t.
        // Every slot holds at most one pair (N / 2 <= 64); p and q advance by
        // one place per round.
        const int pr = slot;
        const bool has_pair = pr < N / 2;
        int p = pr == 0 ? 0 : 1 + (pr - 1) % (N - 1);
        int q = has_pair ? 1 + (N - 2 - pr) % (N - 1) : 0;
        // only the warps that hold pairs take part in the rounds; they meet
        // at a named barrier of their own
        const int act = min(JAC_NT, ((N / 2) * TPP + 31) & ~31);
        for (int round = 0; round < N - 1 && tid < act; round++) {
            if (has_pair && p < k && q < k) do {
                T *xp = X + p * ld, *xq = X + q * ld;
                const T a = sv[p], b = sv[q];
                T u[EL], w[EL];
#pragma unroll
                for (int e = 0; e < EL; e++) {
                    const int i = sub + TPP * e;
                    u[e] = i < k ? xp[i] : T(0);
                    w[e] = i < k ? xq[i] : T(0);
                }
                T g0 = T(0), g1 = T(0);
#pragma unroll
                for (int e = 0; e < EL; e += 2) {
                    g0 = fma(u[e], w[e], g0);
                    if (e + 1 < EL) g1 = fma(u[e + 1], w[e + 1], g1);
                }
                T g = g0 + g1;
#pragma unroll
                for (int o = TPP / 2; o > 0; o >>= 1) g += __shfl_xor_sync(gmask, g, o);
                if (!(a > small) || !(b > small)) break;
                if (a + b <= th2) break;
                const T rel = fabs(g) * rsqrt_of(a) * rsqrt_of(b);
                if (!(rel > tol)) break;
                // t = sign(z) / (|z| + sqrt(1 + z^2)) with z = (b - a) / (2 g),
                // multiplied through by |2 g|; the root is only a rotation
                // angle, so a rounding-level error in it costs nothing: the
                // applied rotation is orthogonal through cs and sn below
                const T e_ = b - a, f = T(2) * g;
                const T h2 = e_ * e_ + f * f;  // > 0: f != 0 here
                const T hyp = h2 * rsqrt_of(h2);
                T tt;
                if (hyp < T(1e37)) {  // finite, and in the fast quotient's range
                    tt = fast_div(f, e_ + copysign(hyp, e_));
                } else {
                    const T zeta = e_ / f, az = fabs(zeta);
                    tt = az > T(1e15) ? T(0.5) / zeta
                                      : (zeta >= T(0) ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
                }
                const T cs = rsqrt_nr(T(1) + tt * tt), sn = cs * tt;
                T *vp = V + p * ld, *vq = V + q * ld;
#pragma unroll
                for (int e = 0; e < EL; e++) {
                    const int i = sub + TPP * e;
                    if (i < k) {
                        xp[i] = cs * u[e] - sn * w[e];
                        xq[i] = sn * u[e] + cs * w[e];
                        const T vu = vp[i], vw = vq[i];
                        vp[i] = cs * vu - sn * vw;
                        vq[i] = sn * vu + cs * vw;
                    }
                }
                __syncwarp(gmask);
                if (sub == 0) {
                    sv[p] = max(a - tt * g, T(0));
                    sv[q] = b + tt * g;
                }
                mymax = max(mymax, rel);
            } while (false);
            asm volatile("bar.sync 1, %0;" ::"r"(act) : "memory");
            if (pr != 0) p = p == N - 1 ? 1 : p + 1;
            q = q == N - 1 ? 1 : q + 1;
        }
        // no rotation (largest 0) or only rotations below the stopping level
        for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
        if (lane == 0) wmax[warp] = mymax;
        __syncthreads();
        T gmax = T(0);
        for (int w = 0; w < JAC_NT / 32; w++) gmax = max(gmax, wmax[w]);
        const int done = !(gmax > stop);
        __syncthreads();
        if (done) break;
        if (check) {
            // every pair's off-orthogonality after this sweep, in one pass
            // (warp w rows p = w, w + 16, ..., lanes the partners q > p),
            // with the rotation's own skip rules; below stop / 10 the call
            // ends instead of running a sweep to confirm it
            T cmax = T(0);
            for (int p = warp; p < k; p += JAC_NT / 32) {
                const T a = sv[p];
                if (!(a > small)) continue;
                for (int q = p + 1 + lane; q < k; q += 32) {
                    const T b = sv[q];
                    if (!(b > small) || a + b <= th2) continue;
                    T g = T(0);
                    for (int i = 0; i < k; i++) g = fma(X[p * ld + i], X[q * ld + i], g);
                    cmax = max(cmax, fabs(g) * rsqrt_of(a) * rsqrt_of(b));
                }
            }
            for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
            if (lane == 0) wmax[warp] = cmax;
            __syncthreads();
            T call = T(0);
            for (int w = 0; w < JAC_NT / 32; w++) call = max(call, wmax[w]);
            __syncthreads();
            if (!(call > T(0.1) * stop)) break;
        }
    }
    if (stats != nullptr && tid == 0) {
        atomicAdd(stats, 1);
        atomicAdd(stats + 1, sweeps);
    }

    for (int c = slot; c < k; c += nslot) {
        T s = T(0);
#pragma unroll
        for (int e = 0; e < EL; e++) {
            const int i = sub + TPP * e;
            if (i < k) s = fma(X[c * ld + i], X[c * ld + i], s);
        }
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (sub == 0) sv[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int p = 0;
        for (int c2 = 0; c2 < k; c2++) p += (sv[c2] > sv[c]) || (sv[c2] == sv[c] && c2 < c);
        pos[c] = p;
        sig[p] = sv[c];
    }
    // fused SVT: r = number of singular values above the threshold (the
    // first r after sorting)
    const T thL = Us != nullptr ? T(svt->theta_L) : T(0);
    const int r = __syncthreads_count(Us != nullptr && tid < k && sv[tid] > thL);
    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        int p = pos[c];
        T s = sv[c];
        const T uu = s > T(0) ? X[c * ld + i] / s : T(0);
        Ut[(int64_t)i * ldr + p] = uu;
        Wt[(int64_t)i * ldr + p] = V[c * ld + i];
        if (Us != nullptr) Us[(int64_t)i * ldr + p] = p < r ? uu * (s - thL) : T(0);
    }
    if (Us != nullptr && tid == 0) {
        svt->r_new = r;
        int kn = r + svt->oversample;
        if (kn < 1) kn = 1;
        if (kn > svt->kcap) kn = svt->kcap;
        if (r >= k && k < svt->kcap) svt->flags |= 1;
        svt->k_next = kn;
    }
}

// one-sided Jacobi SVD of C = Rz^T (k x k): C = Ut diag(sig) Wt^T.
// When ctrl is given, pairs whose squared norms sum to at most theta_L^2 are
// not rotated: rotations preserve a + b, so neither column can end above the
// SVT threshold and their mixing cannot change the thresholded result.
// stats (optional): stats[0] counts the calls, stats[1] their sweeps.
// Us (optional, with svt): the SVT on the factors fused into the epilogue, as
// svt_small_kernel computes it for svt->theta_L (same arithmetic).
template <typename T, int NARROW = 0>
__global__ void __launch_bounds__(JAC_NT) jacobi_kernel(const T *__restrict__ Rz, int ldr, const int *kdyn,
                                                        T *__restrict__ Ut, T *__restrict__ Wt, T *__restrict__ sig,
                                                        const Ctrl *ctrl, int *stats, T *__restrict__ Us,
                                                        Ctrl *svt, int check)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T wmax[JAC_NT / 32];  // per-warp largest |g|/sqrt(ab) rotated in the sweep
    __shared__ T amax;
    const int k = *kdyn;
    T *sm = reinterpret_cast<T *>(smraw);
    // k <= 64: 16 lanes per column pair (32 pairs fill the 512 threads), or 8
    // (NARROW: half the warps in the rounds, a shorter shuffle tree); else 8
    if (k <= 64) {
        if constexpr (NARROW)
            jacobi_body<T, 8, 8>(Rz, ldr, k, Ut, Wt, sig, ctrl, stats, Us, svt, sm, wmax, &amax, check);
        else
            jacobi_body<T, 4, 16>(Rz, ldr, k, Ut, Wt, sig, ctrl, stats, Us, svt, sm, wmax, &amax, check);
    } else {
        jacobi_body<T, 16, 8>(Rz, ldr, k, Ut, Wt, sig, ctrl, stats, Us, svt, sm, wmax, &amax, check);
    }
}

// ---------------------------------------------------------------------------
// SVT on the factors + subspace width for the next iteration
// ---------------------------------------------------------------------------
template <typename T>
__global__ void svt_small_kernel(const T *__restrict__ Ut, const T *__restrict__ sig, int ldr, Ctrl *ctrl,
                                 T *__restrict__ Us, double *sig64)
{
    __shared__ int s_r;
    const int k = ctrl->k;
    const T th = T(ctrl->theta_L);
    if (threadIdx.x == 0) s_r = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (sig[c] > th) atomicAdd(&s_r, 1);
        if (sig64) sig64[c] = (double)sig[c];
    }
    __syncthreads();
    const int r = s_r;  // sig is sorted, so the kept values are the first r
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        int i = idx / k, c = idx % k;
        Us[(int64_t)i * ldr + c] = c < r ? Ut[(int64_t)i * ldr + c] * (sig[c] - th) : T(0);
    }
    if (threadIdx.x == 0) {
        ctrl->r_new = r;
        int kn = r + ctrl->oversample;
        if (kn < 1) kn = 1;
        if (kn > ctrl->kcap) kn = ctrl->kcap;
        if (r >= k && k < ctrl->kcap) ctrl->flags |= 1;
        ctrl->k_next = kn;
    }
}

// Random start columns of the subspace block: columns [k, k_next) and the
// columns whose singular value came out exactly zero (dropped directions).
template <typename T>
__global__ void fill_random_kernel(T *Omega, int64_t ldo, int rows, const Ctrl *ctrl, int all_cols,
                                   const T *__restrict__ sig, int kmax, uint64_t salt)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kmax) return;
    int kc = all_cols ? 0 : ctrl->k;
    int kn = all_cols ? ctrl->k : ctrl->k_next;
    if (c >= kn) return;
    bool fill = (c >= kc) || (sig != nullptr && sig[c] == T(0));
    if (!fill) return;
    uint64_t key = ctrl->seed * 0x9E3779B97F4A7C15ull + salt * 0xD1B54A32D192ED03ull + (uint64_t)ctrl->iter * 7919ull;
    for (int j = blockIdx.y; j < rows; j += gridDim.y)  // rows beyond the 65535 grid rows loop
        Omega[(int64_t)j * ldo + c] = T(hash_uniform(key ^ ((uint64_t)j * 1000003ull + (uint64_t)c * 0x100000001B3ull)));
}

// fill_random_kernel on Omega (rows_o rows) and prolong_kernel from Omega
// into B (n rows) in one launch: the prolongation reads the columns c < r_new,
// whose singular values are above the threshold and so are never refilled
template <typename T>
__global__ void fill_prolong_kernel(T *Omega, int64_t ldo, int rows_o, const Ctrl *ctrl, const T *__restrict__ sig,
                                    int kmax, uint64_t salt, int n, T *__restrict__ B, int64_t ldb, TransferDev<T> tr)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kmax) return;
    const int r = ctrl->r_new, kc = ctrl->k, kn = ctrl->k_next;
    const bool fill = c < kn && ((c >= kc) || (sig != nullptr && sig[c] == T(0)));
    const uint64_t key =
        ctrl->seed * 0x9E3779B97F4A7C15ull + salt * 0xD1B54A32D192ED03ull + (uint64_t)ctrl->iter * 7919ull;
    const int rows = max(n, rows_o);
    for (int j = blockIdx.y; j < rows; j += gridDim.y) {  // rows beyond the 65535 grid rows loop
        if (j < n) {
            T v = T(0);
            if (c < r) {
                const int a = tr.j0[j];
                v = tr.w0[j] * Omega[(int64_t)a * ldo + c];
                if (a + 1 < tr.nh && tr.w1[j] != T(0)) v = fma(tr.w1[j], Omega[(int64_t)(a + 1) * ldo + c], v);
            }
            B[(int64_t)j * ldb + c] = v;
        }
        if (j < rows_o && fill)
            Omega[(int64_t)j * ldo + c] =
                T(hash_uniform(key ^ ((uint64_t)j * 1000003ull + (uint64_t)c * 0x100000001B3ull)));
    }
}

__global__ void ctrl_begin_kernel(Ctrl *c)
{
    double mu = c->mu0 * c->eta_k;  // eta_k = eta^iter, kept by ctrl_end_kernel
    if (mu < c->mu_bar) mu = c->mu_bar;
    double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * c->t * c->t));
    c->mu_k = mu;
    c->t_next = t1;
    c->beta = (c->t - 1.0) / t1;
    c->theta_L = c->tau * mu;
    c->theta_S = c->tau * c->lam * mu;
}

__global__ void ctrl_take_width_kernel(Ctrl *c) { c->k = c->k_next; }

// residual check at weight mu_c: thresholds of the check, and a width of at
// least rank(L_k) + p so that the fine SVT is not truncated
__global__ void ctrl_set_check_kernel(Ctrl *chk, const Ctrl *it, double mu_c)
{
    chk->mu_bar = mu_c;
    chk->mu_k = mu_c;
    chk->theta_L = chk->tau * mu_c;
    chk->theta_S = chk->tau * chk->lam * mu_c;
    int k = max(chk->k_next, it->rk + chk->oversample);
    chk->k_next = min(k, chk->kcap);  // columns [k, k_next) get random vectors, then k = k_next
}

__global__ void ctrl_end_kernel(Ctrl *c)
{
    pdl_enter();
    c->t = c->t_next;
    c->rp = c->rk;
    c->rk = c->r_new;
    c->k = c->k_next;
    c->iter += 1;
    c->eta_k *= c->eta;
}

// threads of the Cholesky kernel: fp32 1024 (more warps hide the latency of
// each elimination step), fp64 512 (register budget)
template <typename T>
constexpr int chol_nt()
{
    return sizeof(T) == 4 ? 1024 : 512;
}

template <typename T>
size_t chol_smem(int kmax)
{
    // d, piv, two rows of S with their pivot reciprocals; R and Rprev for Rtot
    return (size_t)(4 * kmax + 2) * sizeof(T) + (size_t)2 * kmax * (kmax + 1) * sizeof(T) + 16;
}

template <typename T>
size_t jacobi_smem(int kmax)
{
    return (size_t)2 * kmax * jac_ld(kmax) * sizeof(T) + kmax * sizeof(T) + kmax * sizeof(int) + 16;
}

template <typename T>
void ensure_small_attrs()
{
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(chol_kernel<T, chol_nt<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)chol_smem<T>(small_kmax<T>()));
    cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem<T>(small_kmax<T>()));
    cudaFuncSetAttribute(jacobi_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem<T>(small_kmax<T>()));
    if (std::is_same<T, float>::value) {
        cudaFuncSetAttribute(chol_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_q_smem(small_kmax<float>()));
        cudaFuncSetAttribute(chol_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(chol_blk_smem(small_kmax<float>()), chol_s_smem(small_kmax<float>())));
        cudaFuncSetAttribute(chol_s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_s_smem(small_kmax<float>()));
    }
    done = true;
}

}  // namespace

template <typename T>
void launch_chol(const T *partialG, int splits, int kmax, const int *kdyn, T *R, T *Rinv, const T *Rprev, T *Rtot,
                 int ldr, int *well_out, const int *skip_in, cudaStream_t st, int *stats, int form)
{
    ensure_small_attrs<T>();
    CPCP_COUNT_LAUNCH();
    if constexpr (std::is_same<T, float>::value) {
        if (kmax <= small_kmax<float>() && form == 2) {
            chol_s_kernel<<<1, CS_NT, chol_s_smem(kmax), st>>>(partialG, splits, kmax, kdyn, R, Rinv, Rprev, Rtot,
                                                              ldr, well_out, skip_in, stats);
            return;
        }
        if (kmax <= small_kmax<float>() && form == 0) {
            launch_pdl(chol_blk_kernel, dim3(1), dim3(CB_NT), std::max(chol_blk_smem(kmax), chol_s_smem(kmax)), st,
                       partialG, splits, kmax, kdyn, R, Rinv, Rprev, Rtot, ldr, well_out, skip_in, stats);
            return;
        }
        if (kmax <= small_kmax<float>()) {
            chol_q_kernel<<<1, CQ_NT, chol_q_smem(kmax), st>>>(partialG, splits, kmax, kdyn, R, Rinv, Rprev, Rtot, ldr,
                                                              well_out, skip_in, stats);
            return;
        }
    }
    chol_kernel<T, chol_nt<T>()><<<1, chol_nt<T>(), chol_smem<T>(kmax), st>>>(partialG, splits, kmax, kdyn, R, Rinv,
                                                                            Rprev, Rtot, ldr,
                                                          well_out, skip_in, stats);
}

bool launch_cholqr2_cluster(int rows, const float *X, float *Q, float *Q1, int KM, const int *kdyn, float *G,
                            float *R1, float *R1i, float *R2, float *R2i, float *Rout, int *well, int *stats,
                            cudaStream_t st)
{
    // a cluster of 16 CTAs (non-portable size) where the device accepts it, else 8
    static int attr = 0;  // 0: not set, 1: set, -1: the kernel cannot be launched
    static int cl_max = 16;
    if (KM > small_kmax<float>() || rows < 1) return false;
    // Cholesky workspace (it also holds the Gram scratch of 512 4 x 4 register
    // tiles), then one k x k partial Gram matrix
    const int kx = small_kmax<float>();
    const size_t ws = std::max(chol_smem<float>(kx), (size_t)(CQR_NT * 16 + CQR_CH * kx) * sizeof(float));
    const int gp_off = (int)((ws + 255) / 256 * 256);
    const size_t smem = (size_t)gp_off + (size_t)kx * kx * sizeof(float);
    if (attr == 0) {
        attr = 1;
        if (cudaFuncSetAttribute(cholqr2_cluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            attr = -1;
        if (cudaFuncSetAttribute(cholqr2_cluster_kernel<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            cl_max = 8;
        cudaGetLastError();
    }
    if (attr < 0) return false;
    for (;;) {
        const int cl = std::min(cl_max, std::max(1, rows / 16));
        int c = 1;
        while (c * 2 <= cl) c *= 2;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(CQR_NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CPCP_COUNT_LAUNCH();
        const cudaError_t e = cudaLaunchKernelEx(&cfg, cholqr2_cluster_kernel<float>, rows, X, Q, Q1, KM, kdyn, G,
                                                 R1, R1i, R2, R2i, Rout, well, stats, gp_off);
        if (e == cudaSuccess) return true;
        cudaGetLastError();
        --g_kernel_launches;
        if (c <= 8) {
            attr = -1;  // not launchable here: the caller uses the multi-launch form from now on
            return false;
        }
        cl_max = 8;
    }
}

int launch_gram_rows(int rows, const float *X, int KM, const int *kdyn, float *part, cudaStream_t st)
{
    // up to 16 slices of at least 128 rows (the Cholesky kernels read every
    // slice of every entry, so more slices cost more there than they save here)
    const int nb = std::max(1, std::min(16, (rows + 127) / 128));
    const size_t smem = (size_t)(CQR_NT * 16 + CQR_CH * KM + KM * KM) * sizeof(float);
    static size_t attr = 0;
    if (attr < smem) {
        cudaFuncSetAttribute(gram_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    CPCP_COUNT_LAUNCH();
    launch_pdl(gram_rows_kernel<float>, dim3(nb), dim3(CQR_NT), smem, st, rows, X, KM, kdyn, part);
    return nb;
}

void launch_cqr_pass2(int rows, const float *X, float *Q1, int KM, const int *kdyn, float *Rt, float *Rti,
                      const int *well, float *Gp, float *G, float *R2, float *R2i, unsigned *ticket, int *stats,
                      cudaStream_t st)
{
    // the layout of the cluster kernel: Cholesky workspace (which also holds
    // the Gram scratch and a row chunk), then a k x k staging area
    const int kx = small_kmax<float>();
    const size_t ws = std::max(chol_smem<float>(kx), (size_t)(CQR_NT * 16 + CQR_CH * kx) * sizeof(float));
    const int gp_off = (int)((ws + 255) / 256 * 256);
    const size_t smem = (size_t)gp_off + (size_t)kx * kx * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cqr_pass2_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    // up to 16 CTAs of at least 128 rows each (the partial slices fit the
    // workspace's 64)
    const int nb = std::max(1, std::min(16, (rows + 127) / 128));
    CPCP_COUNT_LAUNCH();
    launch_pdl(cqr_pass2_kernel<float>, dim3(nb), dim3(CQR_NT), smem, st, rows, X, Q1, KM, kdyn, Rt, Rti, well, Gp,
               G, R2, R2i, ticket, stats, gp_off);
}

template <typename T>
void launch_jacobi(const T *Rz, int ldr, const int *kdyn, T *Ut, T *Wt, T *sig, int kmax, const Ctrl *ctrl,
                   cudaStream_t st, int *stats, T *Us, Ctrl *svt, int lanes, int check)
{
    ensure_small_attrs<T>();
    CPCP_COUNT_LAUNCH();
    if (lanes == 8)
        launch_pdl(jacobi_kernel<T, 1>, dim3(1), dim3(JAC_NT), jacobi_smem<T>(kmax), st, Rz, ldr, kdyn, Ut, Wt, sig,
                   ctrl, stats, Us, svt, check);
    else
        launch_pdl(jacobi_kernel<T, 0>, dim3(1), dim3(JAC_NT), jacobi_smem<T>(kmax), st, Rz, ldr, kdyn, Ut, Wt, sig,
                   ctrl, stats, Us, svt, check);
}

template <typename T>
void launch_svt_small(const T *Ut, const T *sig, int ldr, Ctrl *ctrl, T *Us, double *sig64, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    svt_small_kernel<T><<<1, 256, 0, st>>>(Ut, sig, ldr, ctrl, Us, sig64);
}

template <typename T>
void launch_fill_random(T *Omega, int64_t ldo, int rows, const Ctrl *ctrl, int all_cols, const T *sig, int kmax,
                        uint64_t salt, cudaStream_t st)
{
    dim3 grid((kmax + 63) / 64, std::min(rows, 65535));
    CPCP_COUNT_LAUNCH();
    fill_random_kernel<T><<<grid, 64, 0, st>>>(Omega, ldo, rows, ctrl, all_cols, sig, kmax, salt);
}

template <typename T>
void launch_fill_prolong(T *Omega, int64_t ldo, int rows_o, const Ctrl *ctrl, const T *sig, int kmax, uint64_t salt,
                         int n, T *B, int64_t ldb, const TransferDev<T> &tr, cudaStream_t st)
{
    dim3 grid((kmax + 63) / 64, std::min(std::max(rows_o, n), 65535));
    CPCP_COUNT_LAUNCH();
    fill_prolong_kernel<T><<<grid, 64, 0, st>>>(Omega, ldo, rows_o, ctrl, sig, kmax, salt, n, B, ldb, tr);
}

void launch_ctrl_begin(Ctrl *c, cudaStream_t st) { CPCP_COUNT_LAUNCH(); ctrl_begin_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_end(Ctrl *c, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    launch_pdl(ctrl_end_kernel, dim3(1), dim3(1), 0, st, c);
}
void launch_ctrl_take_width(Ctrl *c, cudaStream_t st) { CPCP_COUNT_LAUNCH(); ctrl_take_width_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_set_check(Ctrl *chk, const Ctrl *it, double mu_c, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    ctrl_set_check_kernel<<<1, 1, 0, st>>>(chk, it, mu_c);
}

int small_kmax_f32() { return small_kmax<float>(); }
int small_kmax_f64() { return small_kmax<double>(); }

#define INST(T)                                                                                                      \
    template void launch_chol<T>(const T *, int, int, const int *, T *, T *, const T *, T *, int, int *, const int *, \
                                 cudaStream_t, int *, int);                                                          \
    template void launch_jacobi<T>(const T *, int, const int *, T *, T *, T *, int, const Ctrl *, cudaStream_t,       \
                                   int *, T *, Ctrl *, int, int);                                                    \
    template void launch_svt_small<T>(const T *, const T *, int, Ctrl *, T *, double *, cudaStream_t);               \
    template void launch_fill_random<T>(T *, int64_t, int, const Ctrl *, int, const T *, int, uint64_t, cudaStream_t); \
    template void launch_fill_prolong<T>(T *, int64_t, int, const Ctrl *, const T *, int, uint64_t, int, T *, int64_t, \
                                         const TransferDev<T> &, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
