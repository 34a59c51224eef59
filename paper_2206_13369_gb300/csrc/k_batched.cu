// k_batched.cu -- many independent CPCP instances in one persistent launch.
//
// Each CTA takes the next instance from a device work queue (ordered by
// decreasing size on the host, so the longest solves start first) and runs
// the whole multilevel solve on it: the accelerated proximal-gradient
// iteration with continuation (Sec. 2.3), the coarse step of Alg. 4 (restrict
// M, subspace-iteration SVD and SVT on the coarse model, prolong), the same
// level-switching rule and the same fine residual checks as the single-instance
// solver.  Every stage is a CTA-scope device function; CTAs never wait on one
// another.
//
// Layout: the instance's iterates live in a device arena, oriented so that
// m >= n.  L_k and L_{k-1} are kept dense (m x n), so the elementwise pass
// needs no rank-dependent reconstruction; the SVT writes L_{k+1} = A B^T with
// one CTA contraction.  All contractions go through one tiled CTA GEMM with
// generic strides (64 x 64 or 128 x 32 tiles, register micro-tiles).
//
// Arithmetic: fp32 storage and contractions; block sums in fp64 with a fixed
// order; the residual check computes the gradient with error-free sums and
// rebuilds SVT(M) with compensated (Dot2) products, as the single-instance
// check does, so that its noise stays well below the tolerance.
#include <cfloat>

#include "../../include/cpcp.h"
#include "common.cuh"

namespace cpcp {

namespace {

constexpr int KB = BATCH_KB;
constexpr int NMAX = BATCH_NMAX;
constexpr int RB = 8;     // rows per chunk of the elementwise passes
constexpr int PB = 16;    // panel width of the blocked Cholesky and inverse
constexpr int TPP = 8;    // lanes per column pair in Jacobi
constexpr int TK = 32;    // K step of the tiled CTA GEMM
constexpr int CB = 64;    // columns per block of the compensated factor passes
constexpr int RBC = 32;   // rows per chunk of the compensated factor passes
constexpr float TAU = 0.5f;

constexpr int U_FLOATS = 2 * RB * NMAX;                        // pass tiles (aliased with the k x k work)
constexpr int SMALL_FLOATS = 2 * KB * (KB + 1) + (KB / PB) * PB * PB + 3 * KB;
static_assert(SMALL_FLOATS <= U_FLOATS, "k x k work must fit the pass tiles");
static_assert(2 * CB * (KB + 1) + 2 * RBC * KB <= U_FLOATS, "factor staging must fit the pass tiles");
constexpr int GW_FLOATS = TK * 128 + TK * 64;  // tiled GEMM staging (largest tile pair)
constexpr int AROW_FLOATS = RB * KB;
constexpr size_t DSMEM_BYTES = sizeof(float) * (U_FLOATS + GW_FLOATS + AROW_FLOATS);

struct Sm {
    float *tile;   // 2 x RB x NMAX: pass tiles
    float *small;  // k x k work (chol, Jacobi); aliases tile
    float *gw;     // GEMM staging
    float *arow;   // RB x KB rows of a factor
    int wide;      // CTA GEMM tiles for N > 32: 0 = 64 x 64, 1 = 128 x 64 (BatchOpts::tile)
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float rnd(uint64_t seed, uint64_t salt, int iter, int j, int c)
{
    const uint64_t key = seed * 0x9E3779B97F4A7C15ull + salt * 0xD1B54A32D192ED03ull + (uint64_t)iter * 7919ull;
    return (float)hash_uniform(key ^ ((uint64_t)j * 1000003ull + (uint64_t)c * 0x100000001B3ull));
}

// Sum of a and b over the CTA, the same fixed order in every thread; every
// thread returns the totals.
template <int NT>
__device__ void block_sum2(double &a, double &b, double *red)
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    double x = 0.0, y = 0.0;
    for (int i = 0; i < NT / 32; i++) {
        x += red[2 * i];
        y += red[2 * i + 1];
    }
    a = x;
    b = y;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// CTA GEMM: C[i][j] = sum_k A(i,k) B(k,j), A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj], C row-major (ldc).  Generic pointers (global or
// shared).  Ends with a barrier, so C is visible to the whole CTA.
// ---------------------------------------------------------------------------
template <int NT, int TM, int TN>
__device__ __noinline__ void gemm_tiles(int M, int N, int K, const float *A, int64_t sai, int64_t sak, const float *B, int64_t sbk,
                           int64_t sbj, float *C, int64_t ldc, float *gw)
{
    constexpr int NR = TN / 16;
    constexpr int MR = TM * TN / NT / NR;
    static_assert(MR * NR * NT == TM * TN && (TM / MR) * 16 == NT, "thread tiling");
    constexpr int LA = TM * TK / NT, LB = TN * TK / NT;  // tile elements each thread stages
    static_assert(LA * NT == TM * TK && LB * NT == TN * TK, "staging");
    float *As = gw;            // [TK][TM]
    float *Bs = gw + TK * TM;  // [TK][TN]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    float ra[LA], rb[LB];
    // the next K step of A and B goes to registers while the current one is
    // multiplied out of shared memory
    auto fetch = [&](int i0, int j0, int k0) {
#pragma unroll
        for (int q = 0; q < LA; q++) {
            const int e = tid + q * NT;
            int i, kk;
            if (sak == 1) {
                i = e / TK;
                kk = e % TK;
            } else {
                i = e % TM;
                kk = e / TM;
            }
            ra[q] = (i0 + i < M && k0 + kk < K) ? A[(int64_t)(i0 + i) * sai + (int64_t)(k0 + kk) * sak] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < LB; q++) {
            const int e = tid + q * NT;
            int j, kk;
            if (sbj == 1) {
                j = e % TN;
                kk = e / TN;
            } else {
                j = e / TK;
                kk = e % TK;
            }
            rb[q] = (j0 + j < N && k0 + kk < K) ? B[(int64_t)(k0 + kk) * sbk + (int64_t)(j0 + j) * sbj] : 0.f;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < LA; q++) {
            const int e = tid + q * NT;
            const int i = sak == 1 ? e / TK : e % TM, kk = sak == 1 ? e % TK : e / TM;
            As[kk * TM + i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < LB; q++) {
            const int e = tid + q * NT;
            const int j = sbj == 1 ? e % TN : e / TK, kk = sbj == 1 ? e / TN : e % TK;
            Bs[kk * TN + j] = rb[q];
        }
    };
    for (int i0 = 0; i0 < M; i0 += TM) {
        for (int j0 = 0; j0 < N; j0 += TN) {
            float acc[MR][NR];
#pragma unroll
            for (int r = 0; r < MR; r++)
#pragma unroll
                for (int c = 0; c < NR; c++) acc[r][c] = 0.f;
            if (K > 0) {
                fetch(i0, j0, 0);
                stage();
            }
            __syncthreads();
            for (int k0 = 0; k0 < K; k0 += TK) {
                const bool more = k0 + TK < K;
                if (more) fetch(i0, j0, k0 + TK);
                // the chunk's TK terms are summed apart and then added to the
                // total: rounding error ~ (sqrt(TK) + sqrt(K / TK)) eps instead
                // of sqrt(K) eps for one running sum
                float part[MR][NR];
#pragma unroll
                for (int r = 0; r < MR; r++)
#pragma unroll
                    for (int c = 0; c < NR; c++) part[r][c] = 0.f;
#pragma unroll 8
                for (int kk = 0; kk < TK; kk++) {
                    float a[MR], b[NR];
#pragma unroll
                    for (int r = 0; r < MR; r++) a[r] = As[kk * TM + ty * MR + r];
#pragma unroll
                    for (int c = 0; c < NR; c++) b[c] = Bs[kk * TN + tx * NR + c];
#pragma unroll
                    for (int r = 0; r < MR; r++)
#pragma unroll
                        for (int c = 0; c < NR; c++) part[r][c] = fmaf(a[r], b[c], part[r][c]);
                }
#pragma unroll
                for (int r = 0; r < MR; r++)
#pragma unroll
                    for (int c = 0; c < NR; c++) acc[r][c] += part[r][c];
                __syncthreads();
                if (more) stage();
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < MR; r++) {
                const int i = i0 + ty * MR + r;
                if (i >= M) continue;
#pragma unroll
                for (int c = 0; c < NR; c++) {
                    const int j = j0 + tx * NR + c;
                    if (j < N) C[(int64_t)i * ldc + j] = acc[r][c];
                }
            }
        }
    }
    __syncthreads();
}

// C[i][j] = sum_{kk < K} A[kk * lda + i] B[kk * ldb + j] for i < M, j < N <= 64
// (long K: Gram matrices X^T X and M^T Q).  Thread groups split K; each thread
// owns one row i of C and 16 columns at a time; group partials are added in a
// fixed order through shared memory.  B rows must be 16-byte aligned.
template <int NT>
__device__ __noinline__ void gemm_tn_longk(int M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb,
                              float *C, int64_t ldc, const Sm &sm)
{
    const int tid = threadIdx.x;
    const int Mc = (M + 31) / 32 * 32;
    const int tpg = Mc < NT ? Mc : NT;
    int G = NT / tpg;
    G = max(1, min(G, U_FLOATS / (16 * max(M, 1))));
    const int g = tid / tpg, li = tid % tpg;
    const bool active = g < G;
    const int k0 = active ? (int)((int64_t)K * g / G) : 0, k1 = active ? (int)((int64_t)K * (g + 1) / G) : 0;
    float *part = sm.tile;  // G x M x 16
    for (int jb = 0; jb < N; jb += 16) {
        for (int i = li; i < M; i += tpg) {
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; c++) acc[c] = 0.f;
            if (active) {
                // blocks of 32 terms summed apart, then added to the total
                for (int kb = k0; kb < k1; kb += 32) {
                    const int ke = min(k1, kb + 32);
                    float part[16];
#pragma unroll
                    for (int c = 0; c < 16; c++) part[c] = 0.f;
#pragma unroll 4
                    for (int kk = kb; kk < ke; kk++) {
                        const float a = A[(int64_t)kk * lda + i];
                        const float4 *bp = reinterpret_cast<const float4 *>(B + (int64_t)kk * ldb + jb);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const float4 b = bp[q];
                            part[4 * q] = fmaf(a, b.x, part[4 * q]);
                            part[4 * q + 1] = fmaf(a, b.y, part[4 * q + 1]);
                            part[4 * q + 2] = fmaf(a, b.z, part[4 * q + 2]);
                            part[4 * q + 3] = fmaf(a, b.w, part[4 * q + 3]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 16; c++) acc[c] += part[c];
                }
            }
            if (G == 1) {
                for (int c = 0; c < 16 && jb + c < N; c++) C[(int64_t)i * ldc + jb + c] = acc[c];
            } else if (active) {
#pragma unroll
                for (int c = 0; c < 16; c++) part[((int64_t)g * M + i) * 16 + c] = acc[c];
            }
        }
        if (G > 1) {
            __syncthreads();
            for (int e = tid; e < M * 16; e += NT) {
                const int i = e / 16, c = e % 16;
                if (jb + c >= N) continue;
                float s = 0.f;
                for (int q = 0; q < G; q++) s += part[((int64_t)q * M + i) * 16 + c];
                C[(int64_t)i * ldc + jb + c] = s;
            }
        }
        __syncthreads();
    }
}

template <int NT>
__device__ void cta_gemm(int M, int N, int K, const float *A, int64_t sai, int64_t sak, const float *B, int64_t sbk,
                         int64_t sbj, float *C, int64_t ldc, const Sm &sm)
{
    // output tiles (register tiles with NT = 512 / 256): 128 x 32 (4 x 2 / 8 x 2)
    // for N <= 32; for wider N 64 x 64 (2 x 4 / 4 x 4) or 128 x 64 (4 x 4 / 8 x 4),
    // which the autotuner of the launch picks
    if (N <= 32)
        gemm_tiles<NT, 128, 32>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, sm.gw);
    else if (sm.wide && M > 64)
        gemm_tiles<NT, 128, 64>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, sm.gw);
    else
        gemm_tiles<NT, 64, 64>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, sm.gw);
}

// ---------------------------------------------------------------------------
// Cholesky pass of CholeskyQR on the k x k Gram matrix Gin (ld KB), copied to
// sm.small:
// column-equilibrated blocked Cholesky R^T R = G and the blocked inverse,
// written to Rg and Rig (ld KB).  A non-positive pivot drops its column (zero
// row of R, zero column of R^{-1}).  Returns 1 when the equilibrated Gram
// matrix is within 0.5 of the identity (one pass suffices).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __noinline__ int chol_b(int k, const float *Gin, const Sm &sm, float *Rg, float *Rig, double *red)
{
    __shared__ int s_well;
    constexpr int nw = NT / 32;
    const int kp = (k + PB - 1) / PB * PB, ld = kp + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *G = sm.small;
    float *Ri = G + kp * ld;
    float *Tb = Ri + kp * ld;
    float *d = Tb + (kp / PB) * PB * PB;
    float *diag = d + kp;
    int *drop = reinterpret_cast<int *>(diag + kp);

    for (int idx = tid; idx < kp * kp; idx += NT) {
        const int p = idx / kp, c = idx % kp;
        G[p * ld + c] = (p < k && c < k) ? Gin[p * KB + c] : ((p == c) ? 1.f : 0.f);
    }
    __syncthreads();
    for (int p = tid; p < kp; p += NT) {
        const float g = G[p * ld + p];
        d[p] = (p < k && g > 0.f && isfinite(g)) ? sqrtf(g) : 0.f;
    }
    __syncthreads();
    double defect = 0.0, dummy = 0.0;
    for (int idx = tid; idx < k * k; idx += NT) {
        const int p = idx / k, c = idx % k;
        const float dp = d[p], dc = d[c];
        const float v = (dp > 0.f && dc > 0.f) ? G[p * ld + c] / dp / dc : 0.f;
        G[p * ld + c] = v;
        const float e = v - (p == c ? 1.f : 0.f);
        defect += (double)(e * e);
    }
    block_sum2<NT>(defect, dummy, red);
    if (tid == 0) s_well = defect <= 0.25 ? 1 : 0;

    const float tol = FLT_EPSILON * FLT_EPSILON;
    for (int p0 = 0; p0 < kp; p0 += PB) {
        if (warp == 0) {
            for (int jj = 0; jj < PB; jj++) {
                const int j = p0 + jj;
                const float piv = G[j * ld + j];
                const bool dj = !(piv > tol);
                const float sq = dj ? 0.f : sqrtf(piv);
                const float inv = dj ? 0.f : 1.f / sq;
                __syncwarp();
                if (lane > jj && lane < PB) G[j * ld + p0 + lane] *= inv;
                if (lane == 0) {
                    diag[j] = sq;
                    drop[j] = dj;
                }
                __syncwarp();
                if (lane > jj && lane < PB) {
                    const int b = p0 + lane;
                    const float gjb = G[j * ld + b];
                    for (int a = j + 1; a <= b; a++) G[a * ld + b] -= G[j * ld + a] * gjb;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int c = p0 + PB + tid; c < kp; c += NT) {
            for (int i = 0; i < PB; i++) {
                const int row = p0 + i;
                float s = G[row * ld + c];
                for (int l = 0; l < i; l++) s -= G[(p0 + l) * ld + row] * G[(p0 + l) * ld + c];
                G[row * ld + c] = drop[row] ? 0.f : s / diag[row];
            }
        }
        __syncthreads();
        for (int a = p0 + PB + warp; a < kp; a += nw) {
            float gl[PB];
#pragma unroll
            for (int l = 0; l < PB; l++) gl[l] = G[(p0 + l) * ld + a];
            for (int b = a + lane; b < kp; b += 32) {
                float s = 0.f;
#pragma unroll
                for (int l = 0; l < PB; l++) s = fmaf(gl[l], G[(p0 + l) * ld + b], s);
                G[a * ld + b] -= s;
            }
        }
        __syncthreads();
    }

    const int nb = kp / PB;
    auto rh = [&](int i, int c) -> float {
        if (c < i) return 0.f;
        if (c == i) return drop[i] ? 1.f : diag[i];
        return G[i * ld + c];
    };
    for (int t = tid; t < nb * PB; t += NT) {
        const int b = t / PB, cc = t % PB, base = b * PB;
        for (int i = PB - 1; i >= 0; i--) {
            float v = (i == cc) ? 1.f : 0.f;
            if (i < cc)
                for (int p = i + 1; p <= cc; p++) v -= rh(base + i, base + p) * Ri[(base + p) * ld + base + cc];
            Ri[(base + i) * ld + base + cc] = (i <= cc) ? v / rh(base + i, base + i) : 0.f;
        }
    }
    for (int idx = tid; idx < kp * kp; idx += NT) {
        const int i = idx / kp, c = idx % kp;
        if (i / PB > c / PB) Ri[i * ld + c] = 0.f;
    }
    __syncthreads();
    for (int dd = 1; dd < nb; dd++) {
        const int nblk = nb - dd;
        for (int e = tid; e < nblk * PB * PB; e += NT) {
            const int bi = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int i0 = bi * PB, j0 = (bi + dd) * PB;
            float s = 0.f;
            for (int l = i0 + PB; l < j0 + PB; l++) s = fmaf(rh(i0 + rr, l), Ri[l * ld + j0 + cc], s);
            Tb[e] = s;
        }
        __syncthreads();
        for (int e = tid; e < nblk * PB * PB; e += NT) {
            const int bi = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int i0 = bi * PB, j0 = (bi + dd) * PB;
            float s = 0.f;
            for (int p = rr; p < PB; p++) s = fmaf(Ri[(i0 + rr) * ld + i0 + p], Tb[bi * PB * PB + p * PB + cc], s);
            Ri[(i0 + rr) * ld + j0 + cc] = -s;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < k * k; idx += NT) {
        const int i = idx / k, c = idx % k;
        float rv = 0.f, iv = 0.f;
        if (c >= i && !drop[i]) rv = (c == i ? diag[i] : G[i * ld + c]) * d[c];
        if (c >= i && !drop[c] && d[i] > 0.f) iv = Ri[i * ld + c] / d[i];
        Rg[i * KB + c] = rv;
        Rig[i * KB + c] = iv;
    }
    __syncthreads();
    return s_well;
}

// CholeskyQR2 of X (rows x k, ld KB): Q = X R^{-1}; Rout (optional) = R.
template <int NT>
__device__ void orth_b(const BatchInst &I, int rows, int k, const float *X, float *Q, float *Rout, const Sm &sm,
                       double *red)
{
    // the Gram matrices go through I.Us, which is free until the SVT
    gemm_tn_longk<NT>(k, k, rows, X, KB, X, KB, I.Us, KB, sm);
    const int well = chol_b<NT>(k, I.Us, sm, I.R1, I.R1i, red);
    if (well) {
        cta_gemm<NT>(rows, k, k, X, KB, 1, I.R1i, KB, 1, Q, KB, sm);
        if (Rout) {
            for (int idx = threadIdx.x; idx < k * k; idx += NT) Rout[(idx / k) * KB + idx % k] = I.R1[(idx / k) * KB + idx % k];
            __syncthreads();
        }
        return;
    }
    cta_gemm<NT>(rows, k, k, X, KB, 1, I.R1i, KB, 1, I.Q1, KB, sm);
    gemm_tn_longk<NT>(k, k, rows, I.Q1, KB, I.Q1, KB, I.Us, KB, sm);
    chol_b<NT>(k, I.Us, sm, I.R2, I.R2i, red);
    cta_gemm<NT>(rows, k, k, I.Q1, KB, 1, I.R2i, KB, 1, Q, KB, sm);
    if (Rout) cta_gemm<NT>(k, k, k, I.R2, KB, 1, I.R1, KB, 1, Rout, KB, sm);
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD of C = Rz^T (k x k): C = Ut diag(sig) Wt^T, sig sorted
// descending (round-robin pairs, Rutishauser norm updates, the stopping rule
// of the single-instance kernel).  Pairs with a + b <= th2 are not rotated.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __noinline__ void jacobi_b(int k, const float *Rz, float *Ut, float *Wt, float *sig, float th2, const Sm &sm)
{
    __shared__ int rot_count;
    __shared__ unsigned long long gmax_bits;
    __shared__ float amax;
    const int ld = k + 1, N = k + (k & 1);
    float *X = sm.small;
    float *V = X + k * ld;
    float *sv = V + k * ld;
    int *pos = reinterpret_cast<int *>(sv + k);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = tid / TPP, sub = tid % TPP;
    constexpr int nslot = NT / TPP;
    const unsigned gmask = 0xFFu << (lane & ~(TPP - 1));

    for (int idx = tid; idx < k * k; idx += NT) {
        const int c = idx / k, i = idx % k;
        X[c * ld + i] = Rz[c * KB + i];
        V[c * ld + i] = (c == i) ? 1.f : 0.f;
    }
    __syncthreads();
    const float tol = 2.f * (float)((k + TPP - 1) / TPP + 4) * FLT_EPSILON;
    const float negl = (4.f * (float)k * FLT_EPSILON) * (4.f * (float)k * FLT_EPSILON);
    const float stop = fminf(sqrtf(tol), 1e-4f);
    for (int sweep = 0; sweep < 30; sweep++) {
        for (int c = slot; c < k; c += nslot) {
            float s = 0.f;
            for (int i = sub; i < k; i += TPP) s = fmaf(X[c * ld + i], X[c * ld + i], s);
            for (int o = TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
            if (sub == 0) sv[c] = s;
        }
        if (tid == 0) {
            rot_count = 0;
            gmax_bits = 0ull;
        }
        __syncthreads();
        if (warp == 0) {
            float v = 0.f;
            for (int c = lane; c < k; c += 32) v = fmaxf(v, sv[c]);
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) amax = v;
        }
        __syncthreads();
        const float small = negl * amax;
        for (int round = 0; round < N - 1; round++) {
            for (int pr = slot; pr < N / 2; pr += nslot) {
                const int p = pr == 0 ? 0 : 1 + (pr - 1 + round) % (N - 1);
                const int q = 1 + (N - 2 - pr + round) % (N - 1);
                if (p >= k || q >= k) continue;
                float *xp = X + p * ld, *xq = X + q * ld;
                float g = 0.f;
                for (int i = sub; i < k; i += TPP) g = fmaf(xp[i], xq[i], g);
                for (int o = TPP / 2; o > 0; o >>= 1) g += __shfl_xor_sync(gmask, g, o);
                const float a = sv[p], b = sv[q];
                if (!(a > small) || !(b > small)) continue;
                if (a + b <= th2) continue;
                const float rel = fabsf(g) / (sqrtf(a) * sqrtf(b));
                if (!(rel > tol)) continue;
                const float zeta = (b - a) / (2.f * g);
                const float az = fabsf(zeta);
                const float tt = az > 1e15f ? 0.5f / zeta : (zeta >= 0.f ? 1.f : -1.f) / (az + sqrtf(1.f + zeta * zeta));
                const float cs = 1.f / sqrtf(1.f + tt * tt), sn = cs * tt;
                float *vp = V + p * ld, *vq = V + q * ld;
                for (int i = sub; i < k; i += TPP) {
                    float u = xp[i], v = xq[i];
                    xp[i] = cs * u - sn * v;
                    xq[i] = sn * u + cs * v;
                    u = vp[i];
                    v = vq[i];
                    vp[i] = cs * u - sn * v;
                    vq[i] = sn * u + cs * v;
                }
                __syncwarp(gmask);
                if (sub == 0) {
                    sv[p] = fmaxf(a - tt * g, 0.f);
                    sv[q] = b + tt * g;
                    atomicAdd(&rot_count, 1);
                    atomicMax(&gmax_bits, (unsigned long long)__double_as_longlong((double)rel));
                }
            }
            __syncthreads();
        }
        const int done = (rot_count == 0) || (__longlong_as_double((long long)gmax_bits) <= (double)stop);
        __syncthreads();
        if (done) break;
    }
    for (int c = slot; c < k; c += nslot) {
        float s = 0.f;
        for (int i = sub; i < k; i += TPP) s = fmaf(X[c * ld + i], X[c * ld + i], s);
        for (int o = TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (sub == 0) sv[c] = sqrtf(s);
    }
    __syncthreads();
    for (int c = tid; c < k; c += NT) {
        int p = 0;
        for (int c2 = 0; c2 < k; c2++) p += (sv[c2] > sv[c]) || (sv[c2] == sv[c] && c2 < c);
        pos[c] = p;
        sig[p] = sv[c];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += NT) {
        const int c = idx / k, i = idx % k;
        const int p = pos[c];
        const float s = sv[c];
        Ut[i * KB + p] = s > 0.f ? X[c * ld + i] / s : 0.f;
        Wt[i * KB + p] = V[c * ld + i];
    }
    __syncthreads();
}

// Rank-k SVD of Mx (rows x nc, ld ldx) by q range passes from Om (nc x k):
// Mx ~ (Qy Ut) diag(sig) (Qz Wt)^T, left in the instance's arena.
template <int NT>
__device__ void svd_b(const BatchInst &I, int rows, int nc, const float *Mx, int64_t ldx, const float *Om, int k,
                      int q, float th2, const Sm &sm, double *red, long long *cyc)
{
    const float *om = Om;
    long long c0 = clock64(), c1;
    for (int s = 0; s < q; s++) {
        cta_gemm<NT>(rows, k, nc, Mx, ldx, 1, om, KB, 1, I.Y, KB, sm);
        c1 = clock64();
        cyc[0] += c1 - c0;
        orth_b<NT>(I, rows, k, I.Y, I.Qy, nullptr, sm, red);
        c0 = clock64();
        cyc[1] += c0 - c1;
        gemm_tn_longk<NT>(nc, k, rows, Mx, ldx, I.Qy, KB, I.Z, KB, sm);
        c1 = clock64();
        cyc[0] += c1 - c0;
        orth_b<NT>(I, nc, k, I.Z, I.Qz, I.Rz, sm, red);
        c0 = clock64();
        cyc[1] += c0 - c1;
        om = I.Qz;
    }
    jacobi_b<NT>(k, I.Rz, I.Ut, I.Wt, I.sig, th2, sm);
    cyc[2] += clock64() - c0;
}

// number of singular values above theta (sig sorted descending)
__device__ __forceinline__ int count_above(const float *sig, int k, float theta)
{
    int r = 0;
    while (r < k && sig[r] > theta) r++;
    return r;
}

// Us = Ut diag(sig - theta) on the first r columns, zero beyond
template <int NT>
__device__ void svt_scale(const BatchInst &I, int k, int r, float theta)
{
    for (int idx = threadIdx.x; idx < k * k; idx += NT) {
        const int i = idx / k, c = idx % k;
        I.Us[i * KB + c] = c < r ? I.Ut[i * KB + c] * (I.sig[c] - theta) : 0.f;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// elementwise passes (thread = column, RB rows per chunk)
// ---------------------------------------------------------------------------
struct Oriented {
    const float *D;
    int64_t ldd;
    const uint32_t *Q;
    int64_t ldq;
};

__device__ __forceinline__ bool observed(const Oriented &o, int i, int j)
{
    return o.Q == nullptr || ((o.Q[(int64_t)i * o.ldq + (j >> 5)] >> (j & 31)) & 1u);
}

// One iteration's pass at `level`: S_{k+1} = shrink(S^ - tau G, thS) into
// S[nxt]; M = L^ - tau G (level 0) or M_H = (L^ - tau G) R (level > 0).  With
// want_g also the sums ||G||^2 and ||G R||^2 (returned in gg).
template <int NT>
__device__ __noinline__ void pass_step(const BatchInst &I, const Oriented &od, int level, int cur, float beta, float thS,
                          bool want_g, const Sm &sm, double *red, double *gg)
{
    const int m = I.m, n = I.n, nxt = cur ^ 1;
    const int64_t ld = I.ld;
    const float *Lk = I.L[cur], *Lp = I.L[nxt], *Sk = I.S[cur];
    float *Sn = I.S[nxt];
    float *Mt = sm.tile, *Gt = sm.tile + RB * NMAX;
    const int nh = I.nh[level];
    double gsq = 0.0, ghsq = 0.0;
    for (int i0 = 0; i0 < m; i0 += RB) {
        for (int j = threadIdx.x; j < n; j += NT) {
            // every load of the chunk is issued before any store (the stores
            // could alias them, which would serialise one memory round trip
            // per row)
            float lk[RB], lp[RB], sk[RB], sp[RB], dv[RB];
            bool obs[RB];
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const int i = min(i0 + r, m - 1);
                const int64_t o = (int64_t)i * ld + j;
                obs[r] = observed(od, i, j);
                lk[r] = Lk[o];
                lp[r] = Lp[o];
                sk[r] = Sk[o];
                sp[r] = Sn[o];
                dv[r] = od.D[(int64_t)i * od.ldd + j];  // used only where observed
            }
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const int i = i0 + r;
                if (i >= m) break;
                const int64_t o = (int64_t)i * ld + j;
                const float lh = lk[r] + beta * (lk[r] - lp[r]), sh = sk[r] + beta * (sk[r] - sp[r]);
                const float g = obs[r] ? lh + sh - dv[r] : 0.f;
                Sn[o] = obs[r] ? shrink(sh - TAU * g, thS) : 0.f;
                const float mv = lh - TAU * g;
                if (level == 0) {
                    I.M[o] = mv;
                } else {
                    Mt[r * NMAX + j] = mv;
                    if (want_g) {
                        Gt[r * NMAX + j] = g;
                        gsq += (double)g * (double)g;
                    }
                }
            }
        }
        if (level > 0) {
            __syncthreads();
            const int *j0 = I.j0[level], *clo = I.clo[level], *chi = I.chi[level];
            const float *w0 = I.w0[level], *w1 = I.w1[level];
            for (int e = threadIdx.x; e < RB * nh; e += NT) {
                const int r = e / nh, c = e % nh, i = i0 + r;
                if (i >= m) continue;
                float s = 0.f, sg = 0.f;
                for (int j = clo[c]; j <= chi[c]; j++) {
                    const float w = (j0[j] == c) ? w0[j] : ((j0[j] + 1 == c) ? w1[j] : 0.f);
                    s = fmaf(Mt[r * NMAX + j], w, s);
                    if (want_g) sg = fmaf(Gt[r * NMAX + j], w, sg);
                }
                I.MH[(int64_t)i * I.ldh + c] = s;
                if (want_g) ghsq += (double)sg * (double)sg;
            }
            __syncthreads();
        }
    }
    block_sum2<NT>(gsq, ghsq, red);
    gg[0] = gsq;
    gg[1] = ghsq;
}

// Dot2 (Ogita, Rump, Oishi 2005) of a[0:r] . b[0:r]: the sum is hi + lo with
// about twice the working precision
__device__ __forceinline__ void dot2(const float *a, const float *b, int r, float &hi, float &lo)
{
    float s = 0.f, comp = 0.f;
    for (int c = 0; c < r; c++) {
        const float p = a[c] * b[c];
        const float pe = fmaf(a[c], b[c], -p);
        float t, te;
        two_sum(s, p, t, te);
        s = t;
        comp += te + pe;
    }
    hi = s;
    lo = comp;
}

enum { F_CHECK = 0, F_DIFF = 1, F_RECON = 2 };

// Passes over L_k = A[:, :r1] B[:, :r1]^T rebuilt from the SVT factors with
// compensated products (the residual is certified for this iterate, so the
// fp32 rounding of the dense L used by the iteration does not enter it).
//   F_CHECK  M = L_k - tau G and sum ||S_k - shrink(S_k - tau G, thS)||^2,
//            G = P_Q[L_k + S_k - D] formed with error-free sums
//   F_DIFF   sum ||L_k - Ac[:, :r2] Bc[:, :r2]^T||^2
//   F_RECON  L[cur] = L_k
// Column blocks of CB columns with the B rows staged once, row chunks of RBC
// with the A rows staged (both in shared memory).
template <int NT, int MODE>
__device__ __noinline__ double factor_pass(const BatchInst &I, const Oriented &od, int cur, int r1, int r2, float thS,
                              const Sm &sm, double *red)
{
    constexpr int G = NT / CB, RPT = RBC / G;
    static_assert(G * CB == NT && RPT * G == RBC, "factor pass tiling");
    constexpr int LDB = KB + 1;
    float *B1s = sm.small, *B2s = B1s + CB * LDB, *A1s = B2s + CB * LDB, *A2s = A1s + RBC * KB;
    const int m = I.m, n = I.n, jl = threadIdx.x % CB, rg = threadIdx.x / CB;
    double acc = 0.0, dummy = 0.0;
    for (int jb = 0; jb < n; jb += CB) {
        for (int e = threadIdx.x; e < CB * KB; e += NT) {
            const int jj = e / KB, c = e % KB, j = jb + jj;
            B1s[jj * LDB + c] = (j < n && c < r1) ? I.B[(int64_t)j * KB + c] : 0.f;
            if (MODE == F_DIFF) B2s[jj * LDB + c] = (j < n && c < r2) ? I.Bc[(int64_t)j * KB + c] : 0.f;
        }
        for (int i0 = 0; i0 < m; i0 += RBC) {
            for (int e = threadIdx.x; e < RBC * KB; e += NT) {
                const int rr = e / KB, c = e % KB, i = i0 + rr;
                A1s[e] = (i < m && c < r1) ? I.A[(int64_t)i * KB + c] : 0.f;
                if (MODE == F_DIFF) A2s[e] = (i < m && c < r2) ? I.Ac[(int64_t)i * KB + c] : 0.f;
            }
            __syncthreads();
            const int j = jb + jl;
            if (j < n) {
                float skv[RPT], dvv[RPT];
                bool obv[RPT];
                if (MODE == F_CHECK) {
#pragma unroll
                    for (int t = 0; t < RPT; t++) {
                        const int i = min(i0 + rg + G * t, m - 1);
                        skv[t] = I.S[cur][(int64_t)i * I.ld + j];
                        dvv[t] = od.D[(int64_t)i * od.ldd + j];  // used only where observed
                        obv[t] = observed(od, i, j);
                    }
                }
#pragma unroll
                for (int t = 0; t < RPT; t++) {
                    const int rr = rg + G * t, i = i0 + rr;
                    if (i >= m) break;
                    float h1, l1;
                    dot2(A1s + rr * KB, B1s + jl * LDB, r1, h1, l1);
                    const int64_t o = (int64_t)i * I.ld + j;
                    if (MODE == F_RECON) {
                        I.L[cur][o] = h1 + l1;
                    } else if (MODE == F_DIFF) {
                        float h2, l2;
                        dot2(A2s + rr * KB, B2s + jl * LDB, r2, h2, l2);
                        const double dl = ((double)h1 + (double)l1) - ((double)h2 + (double)l2);
                        acc += dl * dl;
                    } else {
                        const float sk = skv[t];
                        float g = 0.f;
                        if (obv[t]) {
                            float s1, e1, s2, e2;
                            two_sum(h1, sk, s1, e1);
                            two_sum(s1, -dvv[t], s2, e2);
                            g = s2 + ((e1 + e2) + l1);
                            const float x = sk - TAU * g;
                            // S - shrink(x): sk when x shrinks to zero, else tau g + thS sign(x)
                            const float ds = fabsf(x) > thS ? TAU * g + copysignf(thS, x) : sk;
                            acc += (double)ds * (double)ds;
                        }
                        I.M[o] = (h1 + l1) - TAU * g;
                    }
                }
            }
            __syncthreads();
        }
    }
    block_sum2<NT>(acc, dummy, red);
    return acc;
}

// ||P_Q D||^2 and the count of non-finite observed entries; M = tau P_Q D
template <int NT>
__device__ void pass_init(const BatchInst &I, const Oriented &od, double *red, double *out)
{
    double sq = 0.0, nf = 0.0;
    for (int i = 0; i < I.m; i++) {
        for (int j = threadIdx.x; j < I.n; j += NT) {
            float v = 0.f;
            if (observed(od, i, j)) {
                v = od.D[(int64_t)i * od.ldd + j];
                if (isfinite(v))
                    sq += (double)v * (double)v;
                else {
                    nf += 1.0;
                    v = 0.f;
                }
            }
            I.M[(int64_t)i * I.ld + j] = TAU * v;
        }
    }
    block_sum2<NT>(sq, nf, red);
    out[0] = sq;
    out[1] = nf;
}

template <int NT>
__device__ void fill_zero(float *X, int rows, int cols, int64_t ld)
{
    for (int i = 0; i < rows; i++)
        for (int j = threadIdx.x; j < cols; j += NT) X[(int64_t)i * ld + j] = 0.f;
}

// Om columns [c0, c1) random; with sig, also the columns c < c0 whose
// singular value is zero
template <int NT>
__device__ void fill_random_cols(float *Om, int rows, int c0, int c1, const float *sig, uint64_t seed, uint64_t salt,
                                 int iter)
{
    for (int idx = threadIdx.x; idx < rows * c1; idx += NT) {
        const int j = idx / c1, c = idx % c1;
        if (c >= c0 || (sig != nullptr && sig[c] == 0.f)) Om[(int64_t)j * KB + c] = rnd(seed, salt, iter, j, c);
    }
    __syncthreads();
}

// B (n x k) = R V (V: nh x k) for the transfer of `level`; level 0 copies
template <int NT>
__device__ void prolong_b(const BatchInst &I, int level, const float *V, float *Bout, int k)
{
    const int n = I.n, nh = I.nh[level];
    for (int idx = threadIdx.x; idx < n * k; idx += NT) {
        const int j = idx / k, c = idx % k;
        float v;
        if (level == 0) {
            v = V[(int64_t)j * KB + c];
        } else {
            const int a = I.j0[level][j];
            v = I.w0[level][j] * V[(int64_t)a * KB + c];
            if (a + 1 < nh) v = fmaf(I.w1[level][j], V[(int64_t)(a + 1) * KB + c], v);
        }
        Bout[(int64_t)j * KB + c] = v;
    }
    __syncthreads();
}

// Om (nh x r) = R^T B for the transfer of `level` (restriction of the right factor)
template <int NT>
__device__ void restrict_rows_b(const BatchInst &I, int level, const float *Bf, float *Om, int r)
{
    const int nh = I.nh[level];
    for (int idx = threadIdx.x; idx < nh * r; idx += NT) {
        const int c = idx / r, cc = idx % r;
        float s = 0.f;
        if (level == 0) {
            s = Bf[(int64_t)c * KB + cc];
        } else {
            const int *j0 = I.j0[level];
            for (int j = I.clo[level][c]; j <= I.chi[level][c]; j++) {
                const float w = (j0[j] == c) ? I.w0[level][j] : ((j0[j] + 1 == c) ? I.w1[level][j] : 0.f);
                s = fmaf(w, Bf[(int64_t)j * KB + cc], s);
            }
        }
        Om[(int64_t)c * KB + cc] = s;
    }
    __syncthreads();
}

// oriented copies of D and Q for an instance solved transposed
template <int NT>
__device__ void orient_in(const BatchInst &I, const Sm &sm)
{
    // user D is n x m (rows x cols); Dw[i][j] = D[j][i], i < m, j < n
    float *t = sm.tile;  // 32 x 33
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int bi = 0; bi < I.m; bi += 32)
        for (int bj = 0; bj < I.n; bj += 32) {
            for (int r = ty; r < 32; r += NT / 32) {
                const int uj = bj + r, ui = bi + tx;  // user row uj, user col ui
                t[r * 33 + tx] = (uj < I.n && ui < I.m) ? I.D[(int64_t)uj * I.ldd + ui] : 0.f;
            }
            __syncthreads();
            for (int r = ty; r < 32; r += NT / 32) {
                const int i = bi + r, j = bj + tx;
                if (i < I.m && j < I.n) I.Dw[(int64_t)i * I.ld + j] = t[tx * 33 + r];
            }
            __syncthreads();
        }
    if (I.Q != nullptr) {
        const int words = (I.n + 31) / 32;
        for (int idx = threadIdx.x; idx < I.m * words; idx += NT) {
            const int i = idx / words, w = idx % words;
            uint32_t bits = 0u;
            for (int b = 0; b < 32; b++) {
                const int j = w * 32 + b;
                if (j < I.n && ((I.Q[(int64_t)j * I.ldq + (i >> 5)] >> (i & 31)) & 1u)) bits |= 1u << b;
            }
            I.Qw[(int64_t)i * I.ldqw + w] = bits;
        }
    }
    __syncthreads();
}

// copy an oriented m x n array to a user output (transposed when trans)
template <int NT>
__device__ void orient_out(const BatchInst &I, const float *X, float *out, int64_t ldo, const Sm &sm)
{
    if (!I.trans) {
        for (int i = 0; i < I.m; i++)
            for (int j = threadIdx.x; j < I.n; j += NT) out[(int64_t)i * ldo + j] = X[(int64_t)i * I.ld + j];
        __syncthreads();
        return;
    }
    float *t = sm.tile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int bi = 0; bi < I.m; bi += 32)
        for (int bj = 0; bj < I.n; bj += 32) {
            for (int r = ty; r < 32; r += NT / 32) {
                const int i = bi + r, j = bj + tx;
                t[r * 33 + tx] = (i < I.m && j < I.n) ? X[(int64_t)i * I.ld + j] : 0.f;
            }
            __syncthreads();
            for (int r = ty; r < 32; r += NT / 32) {
                const int uj = bj + r, ui = bi + tx;  // user element (uj, ui) = oriented (ui, uj)
                if (uj < I.n && ui < I.m) out[(int64_t)uj * ldo + ui] = t[tx * 33 + r];
            }
            __syncthreads();
        }
}

// ---------------------------------------------------------------------------
// one instance, start to finish
// ---------------------------------------------------------------------------
template <int NT>
__device__ void solve_instance(const BatchInst &I, BatchResult *res, const BatchOpts &o, const Sm &sm, double *red)
{
    const int m = I.m, n = I.n, H = I.levels - 1;
    if (I.trans) orient_in<NT>(I, sm);
    Oriented od;
    od.D = I.trans ? I.Dw : I.D;
    od.ldd = I.trans ? I.ld : I.ldd;
    od.Q = I.trans ? I.Qw : I.Q;
    od.ldq = I.trans ? I.ldqw : I.ldq;
    const int kcap0 = min(n, KB);
    auto kcap = [&](int lv) { return min(I.nh[lv], KB); };

    double init[2];
    pass_init<NT>(I, od, red, init);
    BatchResult out;
    memset(&out, 0, sizeof(out));
    const double pqd = sqrt(init[0]);
    out.pqd = pqd;
    if (init[1] > 0.0 || !(pqd > 0.0)) {
        out.status = init[1] > 0.0 ? CPCP_ERR_NONFINITE_INPUT : CPCP_ERR_INVALID_ARG;
        if (threadIdx.x == 0) *res = out;
        return;
    }
    // mu_0 = ||P_Q D||_2, from a few power steps on M = tau P_Q D
    const int k0 = min(o.p, kcap0);
    fill_random_cols<NT>(I.Omf, n, 0, k0, nullptr, o.seed, 0x30ull, 0);
    long long scratch[4] = {0, 0, 0, 0};
    svd_b<NT>(I, m, n, I.M, I.ld, I.Omf, k0, 4, -1.f, sm, red, scratch);
    const double mu0 = I.sig[0] > 0.f ? (double)I.sig[0] / TAU : I.mu;
    out.mu0 = mu0;

    // start state: L = S = 0 in both slots, coarsest level
    for (int s = 0; s < 2; s++) {
        fill_zero<NT>(I.L[s], m, n, I.ld);
        fill_zero<NT>(I.S[s], m, n, I.ld);
    }
    int level = H;
    int k = min(o.p, kcap(level));
    int kc = min(o.p, kcap0);  // width of the check's fine SVD
    fill_random_cols<NT>(I.Om, I.nh[level], 0, k, nullptr, o.seed, 0x11ull, 0);
    fill_random_cols<NT>(I.Omf, n, 0, kc, nullptr, o.seed, 0x12ull, 0);

    const double mu = I.mu, lam = I.lam;
    double t = 1.0, rel = INFINITY, prev = INFINITY;
    int cur = 0, rk = 0, iter = 0, checks = 0;
    int level_start = 0;  // iteration at which the current level began
    int status = CPCP_ERR_NOT_CONVERGED;
    while (iter < o.max_iter) {
        const double mu_k = fmax(mu0 * pow(o.eta, (double)iter), mu);
        const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const float beta = (float)((t - 1.0) / t1);
        const float thL = (float)(0.5 * mu_k), thS = (float)(0.5 * lam * mu_k);
        const bool decide = (iter + 1) % o.check_every == 0;
        const bool early = o.early != 0 && level > 0 && iter == level_start;
        const bool want_g = (decide || early) && level > 0;
        double gg[2];
        long long c0 = clock64();
        pass_step<NT>(I, od, level, cur, beta, thS, want_g, sm, red, gg);
        long long c1 = clock64();
        out.cycles[level > 0 ? 0 : 1] += c1 - c0;
        const int nxt = cur ^ 1;
        const int nh = I.nh[level];
        const float *Mx = level > 0 ? I.MH : I.M;
        const int64_t ldx = level > 0 ? I.ldh : I.ld;
        svd_b<NT>(I, m, nh, Mx, ldx, I.Om, k, o.q, thL * thL, sm, red, out.svt_cycles);
        const long long cf = clock64();
        const int r = count_above(I.sig, k, thL);
        svt_scale<NT>(I, k, r, thL);
        cta_gemm<NT>(m, k, k, I.Qy, KB, 1, I.Us, KB, 1, I.A, KB, sm);   // A = Qy Us
        cta_gemm<NT>(nh, k, k, I.Qz, KB, 1, I.Wt, KB, 1, I.Z, KB, sm);  // V = Qz Wt (into Z)
        prolong_b<NT>(I, level, I.Z, I.B, k);                            // B = R V
        cta_gemm<NT>(m, n, r, I.A, KB, 1, I.B, 1, KB, I.L[nxt], I.ld, sm);  // L_{k+1} = A B^T
        // next subspace: V, grown to rank + p; zero-sigma and new columns random
        const int kn = max(1, min(r + o.p, kcap(level)));
        for (int idx = threadIdx.x; idx < nh * k; idx += NT) I.Om[(idx / k) * KB + idx % k] = I.Z[(idx / k) * KB + idx % k];
        __syncthreads();
        fill_random_cols<NT>(I.Om, nh, k, max(k, kn), I.sig, o.seed, 0x57E9ull, iter);
        const long long ce = clock64();
        out.cycles[2] += ce - c1;
        out.svt_cycles[3] += ce - cf;
        k = kn;
        rk = r;
        t = t1;
        cur = nxt;
        iter++;
        if (level < BATCH_LEVELS) out.level_iters[level]++;
        if (!decide && !early) continue;

        const bool at_final = !(mu_k > mu);
        bool finer = false;
        if (level > 0 && gg[0] > 0.0 && sqrt(fmax(gg[1], 0.0)) < I.kappa[level] * sqrt(gg[0])) finer = true;
        if (decide && !finer && at_final) {
            // fine residual check at (L_k, S_k)
            c0 = clock64();
            const float thLb = (float)(0.5 * mu), thSb = (float)(0.5 * lam * mu);
            const double s_part = factor_pass<NT, F_CHECK>(I, od, cur, rk, 0, thSb, sm, red);
            const int kce = min(kcap0, max(kc, rk + o.p));
            fill_random_cols<NT>(I.Omf, n, kc, kce, nullptr, o.seed, 0xC4ECull, iter);
            svd_b<NT>(I, m, n, I.M, I.ld, I.Omf, kce, o.qc, thLb * thLb, sm, red, scratch);
            const int rc = count_above(I.sig, kce, thLb);
            const bool saturated = rc >= kce && kce < kcap0;
            svt_scale<NT>(I, kce, rc, thLb);
            cta_gemm<NT>(m, kce, kce, I.Qy, KB, 1, I.Us, KB, 1, I.Ac, KB, sm);  // Ac = Qy Us
            cta_gemm<NT>(n, kce, kce, I.Qz, KB, 1, I.Wt, KB, 1, I.Bc, KB, sm);  // Bc = Qz Wt
            for (int idx = threadIdx.x; idx < n * kce; idx += NT)
                I.Omf[(idx / kce) * KB + idx % kce] = I.Bc[(idx / kce) * KB + idx % kce];
            __syncthreads();
            kc = saturated ? min(kcap0, 2 * kce) : min(kcap0, max(rc + o.p, 1));
            if (saturated) {
                rel = INFINITY;
            } else {
                const double l_part = factor_pass<NT, F_DIFF>(I, od, cur, rk, rc, 0.f, sm, red);
                rel = sqrt(fmax(s_part + l_part, 0.0)) / (double)TAU / pqd;
            }
            checks++;
            out.cycles[3] += clock64() - c0;
            if (rel <= o.tol) {
                status = CPCP_OK;
                break;
            }
            if (level > 0 && rel > o.ratio * prev) finer = true;
            prev = rel;
        }
        if (finer) {
            // one level finer: momentum restarts, the subspace is warm-started
            // from the restriction of the current right factor
            level--;
            level_start = iter;
            prev = INFINITY;
            t = 1.0;
            const int kl = min(kcap(level), max(rk + o.p, 1));
            restrict_rows_b<NT>(I, level, I.B, I.Om, rk);
            fill_random_cols<NT>(I.Om, I.nh[level], rk, kl, nullptr, o.seed, 0x77ull + level, iter);
            k = kl;
        }
    }
    out.status = status;
    out.iters = iter;
    out.checks = checks;
    out.rank = rk;
    out.final_level = level;
    out.relkkt = rel;
    if (I.Lout) {
        // the returned L is the iterate the residual was certified for
        if (iter > 0) factor_pass<NT, F_RECON>(I, od, cur, rk, 0, 0.f, sm, red);
        orient_out<NT>(I, I.L[cur], I.Lout, I.ldl, sm);
    }
    if (I.Sout) orient_out<NT>(I, I.S[cur], I.Sout, I.lds, sm);
    if (threadIdx.x == 0) *res = out;
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
    batched_kernel(const BatchInst *__restrict__ inst, BatchResult *res, const int *__restrict__ order, int count,
                   int *next, BatchOpts o)
{
    extern __shared__ float4 dsm4[];
    __shared__ BatchInst I;
    __shared__ double red[2 * (NT / 32)];
    __shared__ int s_w;
    float *dsm = reinterpret_cast<float *>(dsm4);
    Sm sm;
    sm.tile = dsm;
    sm.small = dsm;
    sm.gw = dsm + U_FLOATS;
    sm.arow = sm.gw + GW_FLOATS;
    sm.wide = o.tile;
    static_assert(sizeof(BatchInst) % 4 == 0, "descriptor copy");
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= count) return;
        const int id = order[w];
        const int *src = reinterpret_cast<const int *>(inst + id);
        int *dst = reinterpret_cast<int *>(&I);
        for (int i = threadIdx.x; i < (int)(sizeof(BatchInst) / 4); i += NT) dst[i] = src[i];
        __syncthreads();
        solve_instance<NT>(I, res + id, o, sm, red);
        __syncthreads();
    }
}

template <int NT>
int grid_for()
{
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(batched_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DSMEM_BYTES);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<NT>, NT, DSMEM_BYTES);
        cudaGetLastError();
        g = max(1, sms) * max(1, occ);
    }
    return g;
}

}  // namespace

int batched_grid(int nt) { return nt == 256 ? grid_for<256>() : grid_for<512>(); }

cudaError_t launch_batched(const BatchInst *inst, BatchResult *res, const int *order, int count, int *next,
                           const BatchOpts &o, int nt, cudaStream_t st)
{
    const int grid = std::min(count, batched_grid(nt));
    CPCP_COUNT_LAUNCH();
    if (nt == 256)
        batched_kernel<256><<<grid, 256, DSMEM_BYTES, st>>>(inst, res, order, count, next, o);
    else
        batched_kernel<512><<<grid, 512, DSMEM_BYTES, st>>>(inst, res, order, count, next, o);
    return cudaGetLastError();
}

}  // namespace cpcp
