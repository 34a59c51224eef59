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

#include "common.cuh"

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

// ---------------------------------------------------------------------------
// Cholesky pass of CholeskyQR
// ---------------------------------------------------------------------------
constexpr int CHOL_NT = 512;
constexpr int PB = 16;  // panel / block width of the blocked factorisation and inverse

// Gram reduction + equilibrated Cholesky R = chol(X^T X) (upper) and its
// inverse.  well_out (optional): set to 1 when the equilibrated Gram matrix is
// within 0.5 of the identity in Frobenius norm: X D^{-1} is then well enough
// conditioned (kappa^2 <= 3) that one CholeskyQR pass is accurate to a few
// units of rounding and a second pass can be skipped.  skip_in (optional):
// when *skip_in is set this pass is not needed; R = I, Rinv = I, Rtot = Rprev.
// Rtot = R Rprev when Rprev is given.  A column whose pivot is not positive is
// dropped: zero row in R, zero column in Rinv (zero column of Q).
template <typename T>
__global__ void __launch_bounds__(CHOL_NT) chol_kernel(const T *__restrict__ partial, int splits, int kmax,
                                                       const int *kdyn, T *__restrict__ R, T *__restrict__ Rinv,
                                                       const T *__restrict__ Rprev, T *__restrict__ Rtot, int ldr,
                                                       int *well_out, const int *skip_in)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = *kdyn;
    const int kp = (k + PB - 1) / PB * PB;
    const int ld = kp + 1;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (skip_in != nullptr && *skip_in) {
        for (int idx = tid; idx < k * k; idx += nt) {
            int i = idx / k, c = idx % k;
            R[(int64_t)i * ldr + c] = (i == c) ? T(1) : T(0);
            Rinv[(int64_t)i * ldr + c] = (i == c) ? T(1) : T(0);
            if (Rtot != nullptr) Rtot[(int64_t)i * ldr + c] = Rprev[(int64_t)i * ldr + c];
        }
        return;
    }
    T *G = reinterpret_cast<T *>(smraw);  // kp x ld: equilibrated Gram -> upper factor
    T *Ri = G + kp * ld;                  // kp x ld: inverse of the factor
    T *P = Ri + kp * ld;                  // k x ld: Rprev
    T *Tb = P + k * ld;                   // temporary blocks of the inverse
    T *d = Tb + (kp / PB) * PB * PB;      // column scales
    T *diag = d + kp;                     // diagonal of the factor
    int *drop = reinterpret_cast<int *>(diag + kp);
    __shared__ double red[CHOL_NT / 32];

    // Gram matrix from the row-split partial sums, in a fixed order (four
    // independent chains keep several loads in flight); padding = identity
    const int64_t slice = (int64_t)kmax * kmax;
    for (int idx = tid; idx < kp * kp; idx += nt) {
        int p = idx / kp, c = idx % kp;
        T v = (p == c) ? T(1) : T(0);
        if (p < k && c < k) {
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
            v = (s0 + s1) + (s2 + s3);
            if (Rprev != nullptr) P[p * ld + c] = Rprev[(int64_t)p * ldr + c];
        }
        G[p * ld + c] = v;
    }
    __syncthreads();
    for (int p = tid; p < kp; p += nt) {
        T g = G[p * ld + p];
        d[p] = (p < k && g > T(0) && isfinite(g)) ? sqrt(g) : T(0);
    }
    __syncthreads();
    double defect = 0.0;
    for (int idx = tid; idx < k * k; idx += nt) {
        int p = idx / k, c = idx % k;
        T dp = d[p], dc = d[c];
        T v = (dp > T(0) && dc > T(0)) ? G[p * ld + c] / dp / dc : T(0);
        G[p * ld + c] = v;
        T e = v - (p == c ? T(1) : T(0));
        defect += (double)(e * e);
    }
    defect = warp_sum(defect);
    if (lane == 0) red[warp] = defect;
    __syncthreads();
    if (tid == 0 && well_out != nullptr) {
        double tot = 0.0;
        for (int w = 0; w < nw; w++) tot += red[w];
        *well_out = tot <= 0.25 ? 1 : 0;
    }

    // blocked right-looking Cholesky (upper): per panel of PB columns, warp 0
    // factors the diagonal block, the panel rows right of it are solved
    // (one thread per column), and the trailing matrix gets a rank-PB update.
    // Only a non-positive (or denormal) pivot drops a column; a tiny positive
    // pivot gives a noise direction that the next CholeskyQR pass cleans up.
    const T tol = eps_of<T>() * eps_of<T>();
    for (int p0 = 0; p0 < kp; p0 += PB) {
        if (warp == 0) {
            for (int jj = 0; jj < PB; jj++) {
                const int j = p0 + jj;
                const T piv = G[j * ld + j];
                const bool dj = !(piv > tol);
                const T sq = dj ? T(0) : sqrt(piv);
                const T inv = dj ? T(0) : T(1) / sq;
                __syncwarp();
                if (lane > jj && lane < PB) G[j * ld + p0 + lane] *= inv;
                if (lane == 0) {
                    diag[j] = sq;
                    drop[j] = dj;
                }
                __syncwarp();
                // rank-1 update of the rest of the diagonal block; lane = column
                if (lane > jj && lane < PB) {
                    const int b = p0 + lane;
                    const T gjb = G[j * ld + b];
                    for (int a = j + 1; a <= b; a++) G[a * ld + b] -= G[j * ld + a] * gjb;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // panel rows: solve Rd^T Y = G[p0:p0+PB, c] for the columns c right of the block
        for (int c = p0 + PB + tid; c < kp; c += nt) {
            for (int i = 0; i < PB; i++) {
                const int row = p0 + i;
                T s = G[row * ld + c];
                for (int l = 0; l < i; l++) s -= G[(p0 + l) * ld + row] * G[(p0 + l) * ld + c];
                G[row * ld + c] = drop[row] ? T(0) : s / diag[row];
            }
        }
        __syncthreads();
        // trailing update, upper triangle: warp per row, lanes over columns
        for (int a = p0 + PB + warp; a < kp; a += nw) {
            T gl[PB];
#pragma unroll
            for (int l = 0; l < PB; l++) gl[l] = G[(p0 + l) * ld + a];
            for (int b = a + lane; b < kp; b += 32) {
                T s = T(0);
#pragma unroll
                for (int l = 0; l < PB; l++) s = fma(gl[l], G[(p0 + l) * ld + b], s);
                G[a * ld + b] -= s;
            }
        }
        __syncthreads();
    }

    // blocked inverse of Rh (the factor with dropped diagonals set to one):
    // diagonal blocks by back substitution (one thread per column), then the
    // block superdiagonals d = 1, 2, ...: X_ij = -X_ii (sum_l Rh_il X_lj)
    const int nb = kp / PB;
    auto rh = [&](int i, int c) -> T {
        if (c < i) return T(0);
        if (c == i) return drop[i] ? T(1) : diag[i];
        return G[i * ld + c];
    };
    for (int t = tid; t < nb * PB; t += nt) {
        const int b = t / PB, cc = t % PB, base = b * PB;
        for (int i = PB - 1; i >= 0; i--) {
            T v = (i == cc) ? T(1) : T(0);
            if (i < cc) {
                for (int p = i + 1; p <= cc; p++) v -= rh(base + i, base + p) * Ri[(base + p) * ld + base + cc];
            }
            Ri[(base + i) * ld + base + cc] = (i <= cc) ? v / rh(base + i, base + i) : T(0);
        }
    }
    for (int idx = tid; idx < kp * kp; idx += nt) {  // below the block diagonal
        int i = idx / kp, c = idx % kp;
        if (i / PB > c / PB) Ri[i * ld + c] = T(0);
    }
    __syncthreads();
    for (int dd = 1; dd < nb; dd++) {
        const int nblk = nb - dd;
        for (int e = tid; e < nblk * PB * PB; e += nt) {
            const int bi = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int i0 = bi * PB, j0 = (bi + dd) * PB;
            T s = T(0);
            for (int l = i0 + PB; l < j0 + PB; l++) s = fma(rh(i0 + rr, l), Ri[l * ld + j0 + cc], s);
            Tb[e] = s;
        }
        __syncthreads();
        for (int e = tid; e < nblk * PB * PB; e += nt) {
            const int bi = e / (PB * PB), rr = (e / PB) % PB, cc = e % PB;
            const int i0 = bi * PB, j0 = (bi + dd) * PB;
            T s = T(0);
            for (int p = rr; p < PB; p++) s = fma(Ri[(i0 + rr) * ld + i0 + p], Tb[bi * PB * PB + p * PB + cc], s);
            Ri[(i0 + rr) * ld + j0 + cc] = -s;
        }
        __syncthreads();
    }

    // undo the equilibration: R = Rt D, R^{-1} = D^{-1} Rt^{-1} (dropped
    // columns zero); Rtot = R Rprev
    for (int idx = tid; idx < k * k; idx += nt) {
        int i = idx / k, c = idx % k;
        T rv = T(0), iv = T(0);
        if (c >= i && !drop[i]) rv = (c == i ? diag[i] : G[i * ld + c]) * d[c];
        if (c >= i && !drop[c] && d[i] > T(0)) iv = Ri[i * ld + c] / d[i];
        R[(int64_t)i * ldr + c] = rv;
        Rinv[(int64_t)i * ldr + c] = iv;
        if (Rprev != nullptr) {
            T s = T(0);
            if (c >= i && !drop[i])
                for (int p = i; p <= c; p++) s = fma((p == i ? diag[i] : G[i * ld + p]) * d[p], P[p * ld + c], s);
            Rtot[(int64_t)i * ldr + c] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// one-sided Jacobi SVD of C = Rz^T (k x k): C = Ut diag(sig) Wt^T
// ---------------------------------------------------------------------------
constexpr int JAC_NT = 256, JAC_TPP = 8;

// When ctrl is given, pairs whose squared norms sum to at most theta_L^2 are
// not rotated: rotations preserve a + b, so neither column can end above the
// SVT threshold and their mixing cannot change the thresholded result.
template <typename T>
__global__ void __launch_bounds__(JAC_NT) jacobi_kernel(const T *__restrict__ Rz, int ldr, const int *kdyn,
                                                        T *__restrict__ Ut, T *__restrict__ Wt, T *__restrict__ sig,
                                                        const Ctrl *ctrl)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = *kdyn;
    const int ld = k + 1;
    const int N = k + (k & 1);
    T *X = reinterpret_cast<T *>(smraw);  // X[c * ld + i]: column c of C
    T *V = X + k * ld;
    T *sv = V + k * ld;                   // squared column norms, then singular values
    int *pos = reinterpret_cast<int *>(sv + k);
    __shared__ int rot_count;
    __shared__ unsigned long long gmax_bits;  // largest |g|/sqrt(ab) rotated in the sweep
    __shared__ T amax;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const T th2 = ctrl != nullptr ? T(ctrl->theta_L) * T(ctrl->theta_L) : T(-1);
    // JAC_TPP consecutive lanes share one column pair
    const int slot = tid / JAC_TPP, sub = tid % JAC_TPP, nslot = JAC_NT / JAC_TPP;
    const unsigned gmask = 0xFFu << (lane & ~(JAC_TPP - 1));

    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        X[c * ld + i] = Rz[(int64_t)c * ldr + i];  // column c of Rz^T = row c of Rz
        V[c * ld + i] = (c == i) ? T(1) : T(0);
    }
    __syncthreads();

    // a pair is rotated when |x_p . x_q| exceeds the rounding bound of the
    // group dot product (k/8 sequential terms per lane + a 3-level tree)
    const T tol = T(2) * T((k + JAC_TPP - 1) / JAC_TPP + 4) * eps_of<T>();
    // columns whose norm is below the rounding noise of the largest one carry
    // no information; rotating them against large columns only moves noise
    const T negl = (T(4) * T(k) * eps_of<T>()) * (T(4) * T(k) * eps_of<T>());
    // a sweep whose largest rotated |g|/sqrt(ab) is delta leaves an
    // off-orthogonality of order delta^2 (Jacobi converges quadratically), so
    // a further sweep would only make rounding-level rotations
    const T stop = min(sqrt(tol), T(1e-4));
    for (int sweep = 0; sweep < 30; sweep++) {
        // exact squared norms at the start of each sweep; rotations then
        // update them by a' = a - t g, b' = b + t g (Rutishauser)
        for (int c = slot; c < k; c += nslot) {
            T s = T(0);
            for (int i = sub; i < k; i += JAC_TPP) s = fma(X[c * ld + i], X[c * ld + i], s);
            for (int o = JAC_TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
            if (sub == 0) sv[c] = s;
        }
        if (tid == 0) {
            rot_count = 0;
            gmax_bits = 0ull;
        }
        __syncthreads();
        if (warp == 0) {
            T v = T(0);
            for (int c = lane; c < k; c += 32) v = max(v, sv[c]);
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) amax = v;
        }
        __syncthreads();
        const T small = negl * amax;
        for (int round = 0; round < N - 1; round++) {
            // round-robin (circle) schedule: slot 0 holds column 0, slot s > 0
            // holds column 1 + (s - 1 + round) mod (N - 1); slot t meets N-1-t
            for (int pr = slot; pr < N / 2; pr += nslot) {
                const int p = pr == 0 ? 0 : 1 + (pr - 1 + round) % (N - 1);
                const int q = 1 + (N - 2 - pr + round) % (N - 1);
                if (p >= k || q >= k) continue;
                T *xp = X + p * ld, *xq = X + q * ld;
                T g = T(0);
                for (int i = sub; i < k; i += JAC_TPP) g = fma(xp[i], xq[i], g);
                for (int o = JAC_TPP / 2; o > 0; o >>= 1) g += __shfl_xor_sync(gmask, g, o);
                const T a = sv[p], b = sv[q];
                if (!(a > small) || !(b > small)) continue;
                if (a + b <= th2) continue;
                const T rel = fabs(g) / (sqrt(a) * sqrt(b));
                if (!(rel > tol)) continue;
                T zeta = (b - a) / (T(2) * g);
                // t = sign(z) / (|z| + sqrt(1 + z^2)), or 1/(2 z) where z^2 would overflow
                T az = fabs(zeta);
                T tt = az > T(1e15) ? T(0.5) / zeta
                                    : (zeta >= T(0) ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
                T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
                T *vp = V + p * ld, *vq = V + q * ld;
                for (int i = sub; i < k; i += JAC_TPP) {
                    T u = xp[i], v = xq[i];
                    xp[i] = cs * u - sn * v;
                    xq[i] = sn * u + cs * v;
                    u = vp[i];
                    v = vq[i];
                    vp[i] = cs * u - sn * v;
                    vq[i] = sn * u + cs * v;
                }
                __syncwarp(gmask);
                if (sub == 0) {
                    sv[p] = max(a - tt * g, T(0));
                    sv[q] = b + tt * g;
                    atomicAdd(&rot_count, 1);
                    atomicMax(&gmax_bits, (unsigned long long)__double_as_longlong((double)rel));
                }
            }
            __syncthreads();
        }
        int done = (rot_count == 0) || (__longlong_as_double((long long)gmax_bits) <= (double)stop);
        __syncthreads();
        if (done) break;
    }

    for (int c = slot; c < k; c += nslot) {
        T s = T(0);
        for (int i = sub; i < k; i += JAC_TPP) s = fma(X[c * ld + i], X[c * ld + i], s);
        for (int o = JAC_TPP / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (sub == 0) sv[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int p = 0;
        for (int c2 = 0; c2 < k; c2++) p += (sv[c2] > sv[c]) || (sv[c2] == sv[c] && c2 < c);
        pos[c] = p;
        sig[p] = sv[c];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        int p = pos[c];
        T s = sv[c];
        Ut[(int64_t)i * ldr + p] = s > T(0) ? X[c * ld + i] / s : T(0);
        Wt[(int64_t)i * ldr + p] = V[c * ld + i];
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
    int j = blockIdx.y;
    if (j >= rows || c >= kmax) return;
    int kc = all_cols ? 0 : ctrl->k;
    int kn = all_cols ? ctrl->k : ctrl->k_next;
    if (c >= kn) return;
    bool fill = (c >= kc) || (sig != nullptr && sig[c] == T(0));
    if (!fill) return;
    uint64_t key = ctrl->seed * 0x9E3779B97F4A7C15ull + salt * 0xD1B54A32D192ED03ull + (uint64_t)ctrl->iter * 7919ull;
    Omega[(int64_t)j * ldo + c] = T(hash_uniform(key ^ ((uint64_t)j * 1000003ull + (uint64_t)c * 0x100000001B3ull)));
}

__global__ void ctrl_begin_kernel(Ctrl *c)
{
    double mu = c->mu0 * pow(c->eta, (double)c->iter);
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
    c->t = c->t_next;
    c->rp = c->rk;
    c->rk = c->r_new;
    c->k = c->k_next;
    c->iter += 1;
}

template <typename T>
size_t chol_smem(int kmax)
{
    const int kp = (kmax + PB - 1) / PB * PB;
    return (size_t)(2 * kp + kmax) * (kp + 1) * sizeof(T) + (size_t)kp * PB * sizeof(T) + 2 * kp * sizeof(T) +
           kp * sizeof(int) + 16;
}

template <typename T>
size_t jacobi_smem(int kmax)
{
    return (size_t)2 * kmax * (kmax + 1) * sizeof(T) + kmax * sizeof(T) + kmax * sizeof(int) + 16;
}

template <typename T>
void ensure_small_attrs()
{
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)chol_smem<T>(small_kmax<T>()));
    cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem<T>(small_kmax<T>()));
    done = true;
}

}  // namespace

template <typename T>
void launch_chol(const T *partialG, int splits, int kmax, const int *kdyn, T *R, T *Rinv, const T *Rprev, T *Rtot,
                 int ldr, int *well_out, const int *skip_in, cudaStream_t st)
{
    ensure_small_attrs<T>();
    CPCP_COUNT_LAUNCH();
    chol_kernel<T><<<1, CHOL_NT, chol_smem<T>(kmax), st>>>(partialG, splits, kmax, kdyn, R, Rinv, Rprev, Rtot, ldr,
                                                          well_out, skip_in);
}

template <typename T>
void launch_jacobi(const T *Rz, int ldr, const int *kdyn, T *Ut, T *Wt, T *sig, int kmax, const Ctrl *ctrl,
                   cudaStream_t st)
{
    ensure_small_attrs<T>();
    CPCP_COUNT_LAUNCH();
    jacobi_kernel<T><<<1, JAC_NT, jacobi_smem<T>(kmax), st>>>(Rz, ldr, kdyn, Ut, Wt, sig, ctrl);
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
    dim3 grid((kmax + 63) / 64, rows);
    CPCP_COUNT_LAUNCH();
    fill_random_kernel<T><<<grid, 64, 0, st>>>(Omega, ldo, rows, ctrl, all_cols, sig, kmax, salt);
}

void launch_ctrl_begin(Ctrl *c, cudaStream_t st) { CPCP_COUNT_LAUNCH(); ctrl_begin_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_end(Ctrl *c, cudaStream_t st) { CPCP_COUNT_LAUNCH(); ctrl_end_kernel<<<1, 1, 0, st>>>(c); }
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
                                 cudaStream_t);                                                                      \
    template void launch_jacobi<T>(const T *, int, const int *, T *, T *, T *, int, const Ctrl *, cudaStream_t);      \
    template void launch_svt_small<T>(const T *, const T *, int, Ctrl *, T *, double *, cudaStream_t);               \
    template void launch_fill_random<T>(T *, int64_t, int, const Ctrl *, int, const T *, int, uint64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
