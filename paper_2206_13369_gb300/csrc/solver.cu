// solver.cu -- host driver of the multilevel accelerated proximal-gradient
// solver for eq. (cpcp), and the C ABI declared in include/cpcp.h.
//
// One iteration (all device work, no host round trip):
//   ctrl_begin   momentum weight beta_k, continuation weight mu_k, thresholds
//   step pass    Lhat, Shat, G = P_Q[Lhat + Shat - D] (eq. (cpcp-grad-LS)),
//                S_{k+1} = shrink(Shat - G/2) (Alg. 3), M = Lhat - G/2 and
//                its restriction M_H = M R (Sec. 3.1; Alg. 4 restriction)
//   coarse SVD   subspace iteration on M_H: Y = M_H Omega, CholeskyQR2,
//                Z = M_H^T Q, CholeskyQR2 (Z = Qz Rz), Jacobi SVD of Rz^T
//   SVT          sigma > mu_k/2 kept (Sec. 3.2 coarse minimiser):
//                A = Qy Ut diag(sigma - mu_k/2), V = Qz Wt
//   prolong      B = R V, so L_{k+1} = A B^T = L_H R^T (Alg. 4 prolongation)
//   ctrl_end     rotate ranks, t_k, width
// Every `check_every` iterations once mu_k has reached mu, the fine-level
// gradient-mapping residual is evaluated (one scalar read back to the host),
// and the host decides to stop or to move one level finer.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/cpcp.h"
#include "common.cuh"

using namespace cpcp;

unsigned long long cpcp::g_kernel_launches = 0;
thread_local int cpcp::g_pdl = 0;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// The last unrolled (differentiable) run: its constants and where its
// checkpoints and inputs live (handle workspace), for cpcp_backward.
struct UnrollRec {
    bool valid = false;
    int m = 0, n = 0, K = 0, T = 0, halvings = 0, q = 0;
    int64_t ld = 0, ldq = 0;
    double lam = 0, mu = 0, rho = 0, eta = 0;
    const float *D = nullptr;     // copy of D (m x ld)
    const uint32_t *Q = nullptr;  // copy of the mask or nullptr
    float *ck = nullptr;          // checkpoints: per index 4 arrays m x ld (L_k, L_{k-1}, S_k, S_{k-1})
};

// Captured graph of the last batched solve (persistent launch + read-back of
// the per-instance reports), replayed while the call signature is unchanged.
struct BatchGraph {
    uint64_t sig = 0;
    int nt = 0, tile = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cpcp::BatchResult *host_res = nullptr;  // pinned
    int host_cap = 0;
    cudaStream_t stream = nullptr;          // private non-blocking stream (capturable)
};

}  // namespace

// CUDA-event timing of the solver phases (cpcp_options.profile)
struct PhaseTimer {
    struct Pair {
        cudaEvent_t a, b;
        int phase, level;
        bool spec;  // an iteration run while a residual check decides whether it counts
    };
    // phases 0-3: CPCP_PHASE_*; with profile >= 2 also the SVT phase of the
    // iterations split into 4: products with M, 5: CholeskyQR, 6: core Jacobi SVD,
    // 7: factor products and the next start block (DETAIL_* below)
    static constexpr int NPH = 8;
    std::vector<cudaEvent_t> pool;
    std::vector<Pair> pending;
    double ms[NPH] = {0, 0, 0, 0, 0, 0, 0, 0};
    int count[NPH] = {0, 0, 0, 0, 0, 0, 0, 0};
    // device time of the iterations (pass and SVT phases) by level
    double lvl_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int level = 0;      // level of the intervals opened next
    bool spec = false;  // the intervals opened next belong to speculative iterations
    bool on = false;
    bool detail = false;   // profile >= 2
    bool in_iter = false;  // inside an iteration's SVT phase (not a residual check)
    cudaStream_t st = nullptr;

    // a sub-interval of an iteration's SVT phase (profile >= 2 only)
    int open_sub(int phase) { return (detail && in_iter) ? open(phase) : -1; }

    cudaEvent_t take()
    {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    // returns an open interval; close() records its end
    int open(int phase)
    {
        if (!on) return -1;
        Pair p{take(), take(), phase, level, spec};
        cudaEventRecord(p.a, st);
        pending.push_back(p);
        return (int)pending.size() - 1;
    }
    void close(int idx)
    {
        if (idx >= 0) cudaEventRecord(pending[idx].b, st);
    }
    // after a stream synchronisation, with no interval open: fold the finished
    // intervals into the totals; those of speculative iterations wait for
    // keep_spec() or drop_spec()
    void harvest()
    {
        std::vector<Pair> keep;
        for (auto &p : pending) {
            if (p.spec) {
                keep.push_back(p);
                continue;
            }
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.phase] += t;
                count[p.phase]++;
                if (p.phase <= CPCP_PHASE_SVT && p.level >= 0 && p.level < 8) lvl_ms[p.level] += t;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.swap(keep);
    }
    // the speculative iterations count: their intervals are folded like others
    void keep_spec()
    {
        for (auto &p : pending) p.spec = false;
    }
    // the speculative iterations are discarded (their stream has been
    // synchronised): their intervals are dropped
    void drop_spec()
    {
        std::vector<Pair> keep;
        for (auto &p : pending) {
            if (p.spec) {
                pool.push_back(p.a);
                pool.push_back(p.b);
            } else {
                keep.push_back(p);
            }
        }
        pending.swap(keep);
    }
    void reset(bool enable, cudaStream_t s, bool sub = false)
    {
        harvest();
        for (int i = 0; i < NPH; i++) {
            ms[i] = 0;
            count[i] = 0;
        }
        for (int i = 0; i < 8; i++) lvl_ms[i] = 0;
        level = 0;
        drop_spec();
        spec = false;
        on = enable;
        detail = enable && sub;
        in_iter = false;
        st = s;
    }
    ~PhaseTimer()
    {
        for (auto e : pool) cudaEventDestroy(e);
        for (auto &p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    }
};

struct cpcp_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    cpcp_options opt{};
    std::string err;
    std::map<std::string, DevBuf> bufs;
    PhaseTimer timer;
    BatchGraph batch;
    std::map<uint64_t, std::pair<int, int>> batch_tuned;  // signature -> measured best (CTA size, GEMM tiles)
    UnrollRec unroll;
    // private non-blocking stream of the graph-replayed solve (the caller's
    // stream may be the legacy default stream, which cannot be captured) and
    // the two events that order it after and before the caller's stream
    cudaStream_t solve_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // second private stream on which the fine residual check runs while the
    // solve stream computes the next iterations, the event that orders it after
    // the snapshot of the checked iterate, and pinned host memory for its results
    cudaStream_t check_stream = nullptr;
    cudaEvent_t ev_snap = nullptr;
    void *check_host = nullptr;
    // second stream of an iteration's subspace SVD (the products off its
    // critical path) and the events that fork and join it
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_aux[8] = {};
    // transfer tables already uploaded to this handle's workspace, by
    // (operator, n, halvings, element size): built once, reused by every call
    struct TransferCache {
        int nh = 0;
        double kappa = 0.0;
        void *p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    };
    std::map<std::string, TransferCache> tcache;
};

namespace {

enum { DETAIL_PROD_M = 4, DETAIL_CHOLQR = 5, DETAIL_JACOBI = 6, DETAIL_FACTORS = 7 };

struct CpcpError {
    cpcp_status st;
    std::string msg;
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            throw CpcpError{CPCP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};    \
    } while (0)

void *ws_get(cpcp_context *h, const std::string &name, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    DevBuf &b = h->bufs[name];
    if (b.cap < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw CpcpError{CPCP_ERR_NOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes for " +
                                                name + " failed: " + cudaGetErrorString(e)};
        }
        b.cap = bytes;
    }
    return b.p;
}

template <typename T>
T *wsT(cpcp_context *h, const std::string &name, size_t elems)
{
    return reinterpret_cast<T *>(ws_get(h, name, elems * sizeof(T)));
}

inline int64_t round4(int64_t x) { return (x + 3) / 4 * 4; }
inline int round16(int x) { return (x + 15) / 16 * 16; }

// ---------------------------------------------------------------------------
// transfer operator (host construction, fp64)
// ---------------------------------------------------------------------------

// Largest eigenvalue of the symmetric tridiagonal matrix (d, e) by Sturm
// bisection (count of eigenvalues below x from the LDL^T pivots).
double tridiag_max_eig(const std::vector<double> &d, const std::vector<double> &e)
{
    const int n = (int)d.size();
    double lo = -1e300, hi = -1e300;
    for (int i = 0; i < n; i++) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        hi = std::max(hi, d[i] + r);
        lo = std::max(lo, d[i]);  // lambda_max >= max diagonal entry
    }
    auto below = [&](double x) {
        int cnt = 0;
        double q = d[0] - x;
        if (q < 0) cnt++;
        for (int i = 1; i < n; i++) {
            double qq = q == 0.0 ? 1e-300 : q;
            q = d[i] - x - e[i - 1] * e[i - 1] / qq;
            if (q < 0) cnt++;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-16 * std::fabs(hi); it++) {
        double mid = 0.5 * (lo + hi);
        if (below(mid) == n)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

struct HostTransfer {
    int n = 0, nh = 0, halvings = 0, max_span = 0;
    double scale = 1.0;
    double kappa = 0.0;  // threshold of the coarse-gradient test
    std::vector<int> j0, clo, chi;
    std::vector<double> w0, w1;
};

// One level of eq. (Rx) in the reading fixed by its worked example (Sec. 3.1):
// for even size row 1 = e_1, row 2j = e_j, row 2j+1 = (e_j + e_{j+1})/2; for
// odd size row 2j-1 = e_j, row 2j = (e_j + e_{j+1})/2 (1-based indices).
// Returns up to two (coarse index, weight) entries of fine row x (0-based).
int level_row(int size, int x, int *cols, double *ws)
{
    const int I = x + 1;
    if (size % 2 == 0) {
        if (I == 1) {
            cols[0] = 0;
            ws[0] = 1.0;
            return 1;
        }
        if (I % 2 == 0) {
            cols[0] = I / 2 - 1;
            ws[0] = 1.0;
            return 1;
        }
        int j = (I - 1) / 2;
        cols[0] = j - 1;
        ws[0] = 0.5;
        cols[1] = j;
        ws[1] = 0.5;
        return 2;
    }
    if (I % 2 == 1) {
        cols[0] = (I + 1) / 2 - 1;
        ws[0] = 1.0;
        return 1;
    }
    int j = I / 2;
    cols[0] = j - 1;
    ws[0] = 0.5;
    cols[1] = j;
    ws[1] = 0.5;
    return 2;
}

HostTransfer build_transfer(int n, int halvings)
{
    HostTransfer t;
    t.n = n;
    t.halvings = halvings;
    // sparse rows of the running product, at most 4 entries before merging
    std::vector<std::vector<std::pair<int, double>>> rows(n);
    for (int j = 0; j < n; j++) rows[j] = {{j, 1.0}};
    int cur = n;
    for (int h = 0; h < halvings; h++) {
        for (int j = 0; j < n; j++) {
            std::vector<std::pair<int, double>> out;
            for (auto &e : rows[j]) {
                int cols[2];
                double ws[2];
                int cnt = level_row(cur, e.first, cols, ws);
                for (int u = 0; u < cnt; u++) {
                    bool merged = false;
                    for (auto &o : out)
                        if (o.first == cols[u]) {
                            o.second += e.second * ws[u];
                            merged = true;
                        }
                    if (!merged) out.push_back({cols[u], e.second * ws[u]});
                }
            }
            std::vector<std::pair<int, double>> nz;
            for (auto &o : out)
                if (o.second != 0.0) nz.push_back(o);
            std::sort(nz.begin(), nz.end());
            rows[j] = nz;
        }
        cur = (cur + 1) / 2;
    }
    t.nh = cur;
    t.j0.assign(n, 0);
    t.w0.assign(n, 0.0);
    t.w1.assign(n, 0.0);
    t.clo.assign(cur, n);
    t.chi.assign(cur, -1);
    for (int j = 0; j < n; j++) {
        auto &r = rows[j];
        if (r.empty() || r.size() > 2 || (r.size() == 2 && r[1].first != r[0].first + 1))
            throw CpcpError{CPCP_ERR_NUMERIC, "composite transfer operator is not banded"};
        t.j0[j] = r[0].first;
        t.w0[j] = r[0].second;
        if (r.size() == 2) t.w1[j] = r[1].second;
        for (auto &e : r) {
            t.clo[e.first] = std::min(t.clo[e.first], j);
            t.chi[e.first] = std::max(t.chi[e.first], j);
        }
    }
    // R^T R is tridiagonal: diagonal d_c = sum_j R_jc^2, off e_c = sum_j R_jc R_j,c+1
    std::vector<double> d(cur, 0.0), e(cur > 1 ? cur - 1 : 1, 0.0);
    for (int j = 0; j < n; j++) {
        d[t.j0[j]] += t.w0[j] * t.w0[j];
        if (t.w1[j] != 0.0) {
            d[t.j0[j] + 1] += t.w1[j] * t.w1[j];
            e[t.j0[j]] += t.w0[j] * t.w1[j];
        }
    }
    double lmax = tridiag_max_eig(d, e);
    t.scale = 1.0 / std::sqrt(lmax);
    for (int j = 0; j < n; j++) {
        t.w0[j] *= t.scale;
        t.w1[j] *= t.scale;
    }
    for (int c = 0; c < cur; c++) t.max_span = std::max(t.max_span, t.chi[c] - t.clo[c] + 1);
    // coarse-gradient threshold: geometric mean of the share ||g R|| / ||g|| that
    // white noise keeps on average (||R||_F / sqrt(n)) and that a row constant
    // along the columns keeps (||1^T R|| / sqrt(n))
    double fro2 = 0.0, cs2 = 0.0;
    std::vector<double> cs(cur, 0.0);
    for (int j = 0; j < n; j++) {
        fro2 += t.w0[j] * t.w0[j] + t.w1[j] * t.w1[j];
        cs[t.j0[j]] += t.w0[j];
        if (t.w1[j] != 0.0) cs[t.j0[j] + 1] += t.w1[j];
    }
    for (int c = 0; c < cur; c++) cs2 += cs[c] * cs[c];
    t.kappa = std::sqrt(std::sqrt(fro2 / n) * std::sqrt(cs2 / n));
    return t;
}

int coarse_dim(int n, int halvings)
{
    for (int h = 0; h < halvings; h++) n = (n + 1) / 2;
    return n;
}

template <typename T>
TransferDev<T> upload_transfer(cpcp_context *h, int n, int halvings, const std::string &tag)
{
    // the tables depend on (n, halvings, T) only: each set lives in workspace
    // buffers of its own and is uploaded once per handle
    (void)tag;
    const std::string pre = "tr" + std::to_string(halvings) + "_n" + std::to_string(n) + "_" +
                            std::to_string(sizeof(T)) + "_";
    auto hit = h->tcache.find(pre);
    if (hit != h->tcache.end()) {
        TransferDev<T> d;
        d.n = n;
        d.nh = hit->second.nh;
        d.kappa = hit->second.kappa;
        d.j0 = static_cast<const int *>(hit->second.p[0]);
        d.w0 = static_cast<const T *>(hit->second.p[1]);
        d.w1 = static_cast<const T *>(hit->second.p[2]);
        d.clo = static_cast<const int *>(hit->second.p[3]);
        d.chi = static_cast<const int *>(hit->second.p[4]);
        return d;
    }
    HostTransfer t;
    if (halvings == 0) {
        t.n = n;
        t.nh = n;
        t.j0.resize(n);
        t.w0.assign(n, 1.0);
        t.w1.assign(n, 0.0);
        t.clo.resize(n);
        t.chi.resize(n);
        for (int j = 0; j < n; j++) t.j0[j] = t.clo[j] = t.chi[j] = j;
        t.max_span = 1;
    } else {
        t = build_transfer(n, halvings);
    }
    if (t.max_span > 64)
        throw CpcpError{CPCP_ERR_INVALID_ARG, "too many levels for the restriction tile (support wider than 64)"};
    int *j0 = wsT<int>(h, pre + "j0", n), *clo = wsT<int>(h, pre + "clo", t.nh), *chi = wsT<int>(h, pre + "chi", t.nh);
    T *w0 = wsT<T>(h, pre + "w0", n), *w1 = wsT<T>(h, pre + "w1", n);
    std::vector<T> w0t(t.w0.begin(), t.w0.end()), w1t(t.w1.begin(), t.w1.end());
    CK(cudaMemcpyAsync(j0, t.j0.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(clo, t.clo.data(), sizeof(int) * t.nh, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(chi, t.chi.data(), sizeof(int) * t.nh, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(w0, w0t.data(), sizeof(T) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(w1, w1t.data(), sizeof(T) * n, cudaMemcpyHostToDevice, h->stream));
    // the host vectors must outlive the asynchronous copies
    CK(cudaStreamSynchronize(h->stream));
    TransferDev<T> d;
    d.n = n;
    d.nh = t.nh;
    d.kappa = t.kappa;
    d.j0 = j0;
    d.w0 = w0;
    d.w1 = w1;
    d.clo = clo;
    d.chi = chi;
    cpcp_context::TransferCache c;
    c.nh = t.nh;
    c.kappa = t.kappa;
    c.p[0] = j0;
    c.p[1] = w0;
    c.p[2] = w1;
    c.p[3] = clo;
    c.p[4] = chi;
    h->tcache[pre] = c;
    return d;
}

// Orthonormal basis of the range of the composite R (the unit-norm scaled one)
// for `halvings` halvings: R C^{-1} with R^T R = C^T C.  R^T R is tridiagonal
// (diagonal sum_j R_jc^2, off-diagonal sum_j R_jc R_j,c+1: each row of R has
// two adjacent nonzeros at most), so C is upper bidiagonal (diagonal cd,
// super-diagonal ce, uploaded as T).  kappa: the coarse-gradient threshold of
// build_transfer for R C^{-1}, whose squared Frobenius norm is n_H and whose
// column sums are 1^T R C^{-1} (the recurrence x C = 1^T R).
template <typename T>
struct OrthTransfer {
    T *cd = nullptr, *ce = nullptr;
    double kappa = 0.0;
};

// Host part of OrthTransfer: cd, ce (n_H each) and kappa for `halvings`
// halvings of n.
double orth_factor(int n, int halvings, std::vector<double> &cd, std::vector<double> &ce)
{
    const HostTransfer ht = build_transfer(n, halvings);
    const int nh = ht.nh;
    std::vector<double> dg(nh, 0.0), of(nh, 0.0), cs(nh, 0.0);
    for (int j = 0; j < n; j++) {
        dg[ht.j0[j]] += ht.w0[j] * ht.w0[j];
        cs[ht.j0[j]] += ht.w0[j];
        if (ht.w1[j] != 0.0) {
            dg[ht.j0[j] + 1] += ht.w1[j] * ht.w1[j];
            of[ht.j0[j]] += ht.w0[j] * ht.w1[j];
            cs[ht.j0[j] + 1] += ht.w1[j];
        }
    }
    cd.assign(nh, 0.0);
    ce.assign(nh, 0.0);
    double prev = 0.0;
    for (int c = 0; c < nh; c++) {
        const double v = dg[c] - prev * prev;
        if (!(v > 0.0)) throw CpcpError{CPCP_ERR_NUMERIC, "R^T R is not positive definite"};
        cd[c] = std::sqrt(v);
        prev = c + 1 < nh ? of[c] / cd[c] : 0.0;
        ce[c] = prev;
    }
    double x = 0.0, cs2 = 0.0;
    for (int c = 0; c < nh; c++) {
        x = (cs[c] - (c > 0 ? x * ce[c - 1] : 0.0)) / cd[c];
        cs2 += x * x;
    }
    return std::sqrt(std::sqrt((double)nh / n) * std::sqrt(cs2 / n));
}

template <typename T>
OrthTransfer<T> upload_orth(cpcp_context *h, int n, int halvings, const std::string &tag)
{
    // uploaded once per handle, like the transfer tables
    (void)tag;
    const std::string pre = "orth" + std::to_string(halvings) + "_n" + std::to_string(n) + "_" +
                            std::to_string(sizeof(T)) + "_";
    OrthTransfer<T> o;
    auto hit = h->tcache.find(pre);
    if (hit != h->tcache.end()) {
        o.kappa = hit->second.kappa;
        o.cd = static_cast<T *>(hit->second.p[0]);
        o.ce = static_cast<T *>(hit->second.p[1]);
        return o;
    }
    std::vector<double> cdd, ced;
    o.kappa = orth_factor(n, halvings, cdd, ced);
    const int nh = (int)cdd.size();
    std::vector<T> cd(cdd.begin(), cdd.end()), ce(ced.begin(), ced.end());
    o.cd = wsT<T>(h, pre + "cd", nh);
    o.ce = wsT<T>(h, pre + "ce", nh);
    CK(cudaMemcpyAsync(o.cd, cd.data(), sizeof(T) * nh, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(o.ce, ce.data(), sizeof(T) * nh, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // the host vectors must outlive the copies
    cpcp_context::TransferCache c;
    c.nh = nh;
    c.kappa = o.kappa;
    c.p[0] = o.cd;
    c.p[1] = o.ce;
    h->tcache[pre] = c;
    return o;
}

// ---------------------------------------------------------------------------
// subspace-iteration SVD
// ---------------------------------------------------------------------------

template <typename T>
struct SvdWork {
    int KM;     // padded maximum width (leading dimension of k-wide buffers)
    int kcap;   // maximum live width
    T *Y, *Q1, *Qy, *Z, *Qz;
    T *Gpart, *Zpart, *Ypart;
    T *R1, *R1i, *R2, *R2i, *Rz, *Ut, *Wt, *Us, *sig;
    // the iteration's SVD with two streams: Z' = M^T Y, Rz^{-1}, the Gram
    // matrix of the second CholeskyQR pass, and its zeroed ticket counter
    T *Zp = nullptr, *Rzi = nullptr, *G2 = nullptr;
    unsigned *ticket = nullptr;
    double *sig64;
    int *well;  // per orthogonalisation: 1 when the second CholeskyQR pass is skipped
    // mixed precision: BF16 copies of M (m x nc) and M^T, and of the thin
    // operand (Omega^T or Q^T, round16(KM) rows); error flag of the
    // tensor-core kernels' bounded waits
    __nv_bfloat16 *Mb = nullptr, *Mt = nullptr, *Bt = nullptr;
    int *err = nullptr;
    // optional counters: Jacobi calls, Jacobi sweeps, Cholesky factorisations
    int *stats = nullptr;
    // fp32: the products with M on the tensor cores (options.products_tc)
    bool tc = false;
    // fp32: Gram matrices by row ranges (options.gram_form 0)
    bool gram_rows = false;
};

template <typename T>
SvdWork<T> svd_work(cpcp_context *h, const std::string &tag, int m, int ncols, int kcap)
{
    SvdWork<T> w;
    w.kcap = kcap;
    w.KM = (int)round4(kcap);
    size_t KM = w.KM;
    int rows = std::max(m, ncols);
    w.Y = wsT<T>(h, tag + "Y", (size_t)m * KM);
    w.Q1 = wsT<T>(h, tag + "Q1", (size_t)rows * KM);
    w.Qy = wsT<T>(h, tag + "Qy", (size_t)m * KM);
    w.Z = wsT<T>(h, tag + "Z", (size_t)ncols * KM);
    w.Qz = wsT<T>(h, tag + "Qz", (size_t)ncols * KM);
    w.Gpart = wsT<T>(h, tag + "Gpart", (size_t)64 * KM * KM);
    w.Zpart = wsT<T>(h, tag + "Zpart", (size_t)64 * ncols * KM);
    w.Ypart = wsT<T>(h, tag + "Ypart", (size_t)16 * m * KM);
    w.R1 = wsT<T>(h, tag + "R1", KM * KM);
    w.R1i = wsT<T>(h, tag + "R1i", KM * KM);
    w.R2 = wsT<T>(h, tag + "R2", KM * KM);
    w.R2i = wsT<T>(h, tag + "R2i", KM * KM);
    w.well = wsT<int>(h, tag + "well", 4);
    w.Rz = wsT<T>(h, tag + "Rz", KM * KM);
    w.Ut = wsT<T>(h, tag + "Ut", KM * KM);
    w.Wt = wsT<T>(h, tag + "Wt", KM * KM);
    w.Us = wsT<T>(h, tag + "Us", KM * KM);
    w.sig = wsT<T>(h, tag + "sig", KM);
    w.sig64 = wsT<double>(h, tag + "sig64", KM);
    if (std::is_same<T, float>::value) {
        w.Zp = wsT<T>(h, tag + "Zp", (size_t)ncols * KM);
        w.Rzi = wsT<T>(h, tag + "Rzi", KM * KM);
        w.G2 = wsT<T>(h, tag + "G2", KM * KM);
        w.ticket = wsT<unsigned>(h, tag + "ticket", 4);
        CK(cudaMemsetAsync(w.ticket, 0, 4 * sizeof(unsigned), h->stream));
    }
    // bounded-wait error flag of the tensor-core kernels (shared, cleared per solve)
    w.err = wsT<int>(h, "umma_err", 1);
    const int ptc = h->opt.products_tc;
    w.tc = std::is_same<T, float>::value && KM <= 128 && (ptc == 1 || (ptc == 0 && m >= 4096));
    w.gram_rows = std::is_same<T, float>::value && KM <= 128 && h->opt.gram_form == 0;
    return w;
}

// BF16 buffers of the mixed-precision contractions for matrices up to m x ncols
template <typename T>
void svd_work_bf16(cpcp_context *h, SvdWork<T> &w, const std::string &tag, int m, int ncols)
{
    const size_t kpm = umma_pad_k(m), kpn = umma_pad_k(ncols);
    w.Mb = wsT<__nv_bfloat16>(h, tag + "Mb", (size_t)umma_pad_rows(m) * kpn);
    w.Mt = wsT<__nv_bfloat16>(h, tag + "Mt", (size_t)umma_pad_rows(ncols) * kpm);
    w.Bt = wsT<__nv_bfloat16>(h, tag + "Bt", (size_t)round16(w.KM) * std::max(kpm, kpn));
    w.err = wsT<int>(h, "umma_err", 1);
}

// the bounded-wait error flag of the tensor-core kernels an SVD workspace uses:
// cleared before a call's first launch, read after its last
void tc_err_clear(const int *err, cudaStream_t st) { CK(cudaMemsetAsync(const_cast<int *>(err), 0, sizeof(int), st)); }
void tc_err_check(const int *err, cudaStream_t st)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (e) throw CpcpError{CPCP_ERR_TIMEOUT, "a bounded wait of a tensor-core kernel expired"};
}

// products of the subspace SVD: the cluster-reduced tall-skinny kernels, or the
// plain tiled ones when an operand is not 16-byte aligned
template <typename T>
void prod_nn_small(int rows, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc, const int *kdyn,
                   int kmax, cudaStream_t st, const int *skip = nullptr)
{
    // C (rows x k) = A (rows x k) B (k x k); skip: B is the identity
    if (!launch_ts_nn<T>(rows, 0, A, lda, B, ldb, C, ldc, kdyn, kdyn, kmax, kmax, skip, st))
        launch_gemm_nn<T>(rows, 0, A, lda, B, ldb, C, ldc, kdyn, kdyn, kmax, st);
}

template <typename T>
void prod_y(SvdWork<T> &w, int m, int nc, const T *Mx, int64_t ldx, const T *Om, const int *kdyn, cudaStream_t st)
{
    // Y = M Omega (m x k), K = nc long: fp32 on the tensor cores (three-part
    // TF32 split, split-K partials summed in a fixed order) where the operands
    // meet the TMA rules, else the cluster-reduced SIMT kernel
    if constexpr (std::is_same<T, float>::value) {
        if (w.tc) {
            const int sp = launch_prod_tc(0, m, nc, Mx, ldx, Om, w.KM, w.KM, kdyn, w.Ypart, w.KM, (int64_t)m * w.KM,
                                          16, w.err, st);
            if (sp > 0) {
                launch_reduce_partial<float>(w.Ypart, sp, m, w.KM, w.Y, w.KM, nullptr, kdyn, st);
                return;
            }
        }
    }
    if (!launch_ts_nn<T>(m, nc, Mx, ldx, Om, w.KM, w.Y, w.KM, nullptr, kdyn, nc, w.KM, nullptr, st))
        launch_gemm_nn_splitk<T>(m, nc, Mx, ldx, Om, w.KM, w.Y, w.KM, w.Ypart, kdyn, w.KM, st);
}

template <typename T>
void prod_z(SvdWork<T> &w, int m, int nc, const T *Mx, int64_t ldx, const T *Q, int64_t ldq, const int *kdyn,
            cudaStream_t st, T *out = nullptr, int max_ctas = 0)
{
    // Z = M^T Q (nc x k), K = m long (tensor cores as for Y), into w.Z or out;
    // max_ctas > 0 caps the tensor-core grid (a product beside other kernels)
    T *Zo = out != nullptr ? out : w.Z;
    if constexpr (std::is_same<T, float>::value) {
        if (w.tc && ldq == w.KM) {
            const int sp = launch_prod_tc(1, nc, m, Mx, ldx, Q, ldq, w.KM, kdyn, w.Zpart, w.KM, (int64_t)nc * w.KM,
                                          64, w.err, st, max_ctas);
            if (sp > 0) {
                launch_reduce_partial<float>(w.Zpart, sp, nc, w.KM, Zo, w.KM, nullptr, kdyn, st);
                return;
            }
        }
    }
    if (!launch_ts_tn<T>(nc, m, Mx, ldx, Q, ldq, Zo, w.KM, kdyn, w.KM, st)) {
        const int sp = launch_gemm_tn_partial<T>(m, nc, Mx, ldx, Q, ldq, w.Zpart, kdyn, w.KM, nc, st, nullptr);
        launch_reduce_partial<T>(w.Zpart, sp, nc, w.KM, Zo, w.KM, nullptr, kdyn, st);
    }
}

template <typename T>
int prod_gram(SvdWork<T> &w, int rows, const T *X, const int *kdyn, const int *skip, cudaStream_t st)
{
    // fp32 blocks of at least 4096 rows: by row ranges through shared memory,
    // live columns only (gram_form 0), where X is 16-byte aligned; else the
    // tiled cluster-reduced kernel.  (Measured: 19200 x 15 and 65536 x 18
    // gain, e.g. 67.5 -> 62.8 ms per hyperspectral solve; 2000 x 60 loses
    // 1.2 ms per solve, its Cholesky then summing 16 slices instead of 4.)
    if constexpr (std::is_same<T, float>::value) {
        if (skip == nullptr && w.gram_rows && rows >= 4096 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
            w.KM % 4 == 0)
            return launch_gram_rows(rows, X, w.KM, kdyn, w.Gpart, st);
    }
    const int g = launch_ts_gram<T>(rows, X, w.KM, w.Gpart, kdyn, w.KM, skip, st);
    if (g >= 0) return g;
    return launch_gemm_tn_partial<T>(rows, -1, X, w.KM, X, w.KM, w.Gpart, kdyn, w.KM, w.KM, st, skip);
}

// CholeskyQR2 of X (rows x k): Q = X R^{-1}; if Rout != nullptr it receives
// R = R2 R1.  The second pass is skipped on the device when the first one
// found X nearly orthogonal after column equilibration (the warm-started
// steady state), since it would then leave Q unchanged to rounding.
template <typename T>
void orth_impl(cpcp_context *h, SvdWork<T> &w, int rows, const T *X, T *Q, T *Rout, const int *kdyn, int slot);

template <typename T>
void orth(cpcp_context *h, SvdWork<T> &w, int rows, const T *X, T *Q, T *Rout, const int *kdyn, int slot)
{
    const int tq = h->timer.open_sub(DETAIL_CHOLQR);
    orth_impl<T>(h, w, rows, X, Q, Rout, kdyn, slot);
    h->timer.close(tq);
}

template <typename T>
void orth_impl(cpcp_context *h, SvdWork<T> &w, int rows, const T *X, T *Q, T *Rout, const int *kdyn, int slot)
{
    cudaStream_t st = h->stream;
    const int KM = w.KM;
    int *well = w.well + slot;
    if constexpr (std::is_same<T, float>::value) {
        // both passes in one thread-block cluster launch where available
        if (h->opt.cholqr_fused != 0 &&
            launch_cholqr2_cluster(rows, X, Q, w.Q1, KM, kdyn, w.Gpart, w.R1, w.R1i, w.R2, w.R2i, Rout, well,
                                   w.stats ? w.stats + 2 : nullptr, st))
            return;
    }
    int sp = prod_gram<T>(w, rows, X, kdyn, nullptr, st);
    launch_chol<T>(w.Gpart, sp, KM, kdyn, w.R1, w.R1i, nullptr, nullptr, KM, well, nullptr, st,
                   w.stats ? w.stats + 2 : nullptr, h->opt.chol_form);
    prod_nn_small<T>(rows, X, KM, w.R1i, KM, w.Q1, KM, kdyn, KM, st);
    // second pass; when skipped its factor is the identity and Q = Q1 exactly
    sp = prod_gram<T>(w, rows, w.Q1, kdyn, well, st);
    launch_chol<T>(w.Gpart, sp, KM, kdyn, w.R2, w.R2i, Rout ? w.R1 : nullptr, Rout, KM, nullptr, well, st,
                   w.stats ? w.stats + 2 : nullptr, h->opt.chol_form);
    prod_nn_small<T>(rows, w.Q1, KM, w.R2i, KM, Q, KM, kdyn, KM, st, well);
}

// Second stream of an iteration's subspace SVD, created on first use; with
// kernel-family timing (profile 2) everything stays in order on the solve
// stream, so that each family's events bracket its own kernels only.
cudaStream_t iter_aux(cpcp_context *h)
{
    if (h->timer.detail) return h->stream;
    if (!h->aux_stream) {
        CK(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
        for (auto &e : h->ev_aux) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return h->aux_stream;
}

// orders the work queued next on `to` after the work queued so far on `from`
// (nothing on one stream); slot: which of the handle's events carries it
void order_after(cpcp_context *h, cudaStream_t to, cudaStream_t from, int slot)
{
    if (to == from) return;
    CK(cudaEventRecord(h->ev_aux[slot], from));
    CK(cudaStreamWaitEvent(to, h->ev_aux[slot], 0));
}

// CholeskyQR2 of X (rows x k) as its triangular factors only: Rt = R (X = Q R)
// and Rti = R^{-1}; Q = X Rti is left to the caller.  The second pass is one
// launch that returns at once when the first found X nearly orthogonal after
// equilibration.  fp32.
void orth_factor_only(cpcp_context *h, SvdWork<float> &w, int rows, const float *X, float *Rt, float *Rti,
                      const int *kdyn, int slot)
{
    cudaStream_t st = h->stream;
    const int KM = w.KM;
    int *well = w.well + slot;
    int *stats = w.stats ? w.stats + 2 : nullptr;
    const int sp = prod_gram<float>(w, rows, X, kdyn, nullptr, st);
    launch_chol<float>(w.Gpart, sp, KM, kdyn, Rt, Rti, nullptr, nullptr, KM, well, nullptr, st, stats,
                       h->opt.chol_form);
    launch_cqr_pass2(rows, X, w.Q1, KM, kdyn, Rt, Rti, well, w.Gpart, w.G2, w.R2, w.R2i, w.ticket, stats, st);
}

// Whether Z' = M^T Y leaves room beside it on its usual grid.  On the tensor
// cores it is sized to about one CTA per SM, and where that fills three
// quarters of the GPU or more the kernels beside it push it into a second
// wave (measured on the 19200 x 400 video shape: 31.2 against 27.8 ms per
// solve with the SVD in order); its grid is then capped (zp_ctas), which
// measured 22.6 against 26.5 ms.
bool two_stream_fits(const SvdWork<float> &w, int nc, int m)
{
    if (!w.tc) return true;
    return 4 * prod_tc_ctas(nc, m, 64) < 3 * gpu_sm_count();
}

// the CTA budget of Z' on the tensor cores beside the other stream's chain:
// where its usual grid would fill three quarters of the SMs or more, three
// quarters of them, so that the chain's kernels find free SMs
int zp_ctas(const SvdWork<float> &w, int nc, int m)
{
    if (!w.tc || two_stream_fits(w, nc, m)) return 0;
    return 3 * gpu_sm_count() / 4 - 1;
}

// The subspace SVD of one iteration (one range pass, fp32) on two streams.
// With Q_Y = Y R_Y^{-1} the CholeskyQR2 of Y = M Omega, Z = M^T Q_Y equals
// (M^T Y) R_Y^{-1}, so Z' = M^T Y starts on the second stream as soon as Y
// exists and runs beside the Gram matrix and the factorisations of Y; the
// solve stream then needs only the k-wide product Z = Z' R_Y^{-1}.  Q_Y and
// Q_Z = Z R_Z^{-1}, needed only for the new factors, are formed on the second
// stream beside the factorisation of Z and the core Jacobi SVD.  Leaves the
// same outputs as subspace_svd (Qy, Qz, Ut, Wt, sig, the fused SVT) with
// Qy and Qz complete once the second stream has been joined (events 3, 6).
// The rounding differs from forming Q_Y first by a factor of the condition
// number of Y after column equilibration (near 1 in the warm-started steady
// state: the second CholeskyQR pass is then skipped).
void subspace_svd_iter(cpcp_context *h, SvdWork<float> &w, int m, int nc, const float *Mx, int64_t ldx,
                       const float *Omega, const int *kdyn, const Ctrl *jac_ctrl, float *Us, Ctrl *svt)
{
    cudaStream_t st = h->stream, ax = iter_aux(h);
    // svd_serial 2: only Z' on the second stream; the Q products in order
    cudaStream_t aq = h->opt.svd_serial == 2 ? st : ax;
    const int KM = w.KM;
    int tp = h->timer.open_sub(DETAIL_PROD_M);
    prod_y<float>(w, m, nc, Mx, ldx, Omega, kdyn, st);
    h->timer.close(tp);
    order_after(h, ax, st, 0);
    // (the sub-interval timers only open with profile = 2, where ax is the solve stream)
    tp = h->timer.open_sub(DETAIL_PROD_M);
    prod_z<float>(w, m, nc, Mx, ldx, w.Y, KM, kdyn, ax, w.Zp, ax != st ? zp_ctas(w, nc, m) : 0);  // Z' = M^T Y
    h->timer.close(tp);
    if (ax != st) CK(cudaEventRecord(h->ev_aux[1], ax));
    // programmatic dependent launch where a kernel follows a kernel of the
    // solve stream (not after a cross-stream wait; not while kernel families
    // are timed, whose events bracket single kernels)
    const bool pdl = h->opt.pdl_off == 0 && !h->timer.detail;
    int tq = h->timer.open_sub(DETAIL_CHOLQR);
    {
        PdlScope ps(pdl);
        orth_factor_only(h, w, m, w.Y, w.R1, w.R1i, kdyn, 0);
    }
    h->timer.close(tq);
    order_after(h, aq, st, 2);
    tq = h->timer.open_sub(DETAIL_CHOLQR);
    prod_nn_small<float>(m, w.Y, KM, w.R1i, KM, w.Qy, KM, kdyn, KM, aq);  // Q_Y
    h->timer.close(tq);
    if (aq != st) CK(cudaEventRecord(h->ev_aux[3], aq));
    if (ax != st) CK(cudaStreamWaitEvent(st, h->ev_aux[1], 0));
    tq = h->timer.open_sub(DETAIL_CHOLQR);
    prod_nn_small<float>(nc, w.Zp, KM, w.R1i, KM, w.Z, KM, kdyn, KM, st);  // Z = Z' R_Y^{-1}
    h->timer.close(tq);
    tq = h->timer.open_sub(DETAIL_CHOLQR);
    {
        PdlScope ps(pdl);
        orth_factor_only(h, w, nc, w.Z, w.Rz, w.Rzi, kdyn, 1);
    }
    h->timer.close(tq);
    order_after(h, aq, st, 4);
    tq = h->timer.open_sub(DETAIL_CHOLQR);
    prod_nn_small<float>(nc, w.Z, KM, w.Rzi, KM, w.Qz, KM, kdyn, KM, aq);  // Q_Z
    h->timer.close(tq);
    const int tj = h->timer.open_sub(DETAIL_JACOBI);
    {
        PdlScope ps(pdl && aq != st);  // (with Q_Z in order, the Jacobi follows it)
        launch_jacobi<float>(w.Rz, KM, kdyn, w.Ut, w.Wt, w.sig, w.kcap, jac_ctrl, st, w.stats, Us, svt,
                             h->opt.jacobi_lanes == 8 ? 8 : 16, h->timer.in_iter ? h->opt.jacobi_check : 0);
    }
    h->timer.close(tj);
}

// The subspace SVD below with both contractions with M on the tensor cores:
// M is rounded to BF16 once (kept as M and M^T, K-major both), each power
// step rounds the thin operand (Omega, then Q) and forms Y = M Omega and
// Z = M^T Q with fp32 accumulation.  Orthogonalisation and the core SVD stay
// fp32.
void subspace_svd_bf16(cpcp_context *h, SvdWork<float> &w, int m, int nc, const float *Mx, int64_t ldx,
                       const float *Omega, int q, const int *kdyn, const Ctrl *jac_ctrl, float *Us, Ctrl *svt)
{
    cudaStream_t st = h->stream;
    const int KM = w.KM, NB = round16(KM);
    const int mp = umma_pad_rows(m), ncp = umma_pad_rows(nc), kpm = umma_pad_k(m), kpn = umma_pad_k(nc);
    int tp = h->timer.open_sub(DETAIL_PROD_M);
    launch_bf16_pair(m, nc, Mx, ldx, w.Mb, mp, kpn, w.Mt, ncp, kpm, st);
    h->timer.close(tp);
    const float *Om = Omega;
    for (int s = 0; s < q; s++) {
        tp = h->timer.open_sub(DETAIL_PROD_M);
        launch_bf16_pair(nc, KM, Om, KM, nullptr, 0, 0, w.Bt, NB, kpn, st);
        int sp = launch_umma_tn(m, mp, kpn, w.Mb, kpn, w.Bt, NB, kpn, NB, kdyn, w.Ypart, KM, 16, w.err, st);
        if (sp < 0) throw CpcpError{CPCP_ERR_CUDA, "could not encode the TMA tensor maps"};
        launch_reduce_partial<float>(w.Ypart, sp, m, KM, w.Y, KM, nullptr, kdyn, st);
        h->timer.close(tp);
        orth<float>(h, w, m, w.Y, w.Qy, nullptr, kdyn, 0);
        tp = h->timer.open_sub(DETAIL_PROD_M);
        launch_bf16_pair(m, KM, w.Qy, KM, nullptr, 0, 0, w.Bt, NB, kpm, st);
        sp = launch_umma_tn(nc, ncp, kpm, w.Mt, kpm, w.Bt, NB, kpm, NB, kdyn, w.Zpart, KM, 64, w.err, st);
        if (sp < 0) throw CpcpError{CPCP_ERR_CUDA, "could not encode the TMA tensor maps"};
        launch_reduce_partial<float>(w.Zpart, sp, nc, KM, w.Z, KM, nullptr, kdyn, st);
        h->timer.close(tp);
        orth<float>(h, w, nc, w.Z, w.Qz, w.Rz, kdyn, 1);
        Om = w.Qz;
    }
    const int tj = h->timer.open_sub(DETAIL_JACOBI);
    launch_jacobi<float>(w.Rz, KM, kdyn, w.Ut, w.Wt, w.sig, w.kcap, jac_ctrl, st, w.stats, Us, svt,
                     h->opt.jacobi_lanes == 8 ? 8 : 16,
                     h->timer.in_iter ? h->opt.jacobi_check : 0);
    h->timer.close(tj);
}

// Rank-k SVD of Mx (m x nc, ld ldx): q range passes from Omega (nc x k).
// Leaves Qy (m x k), Qz (nc x k), Ut, Wt (k x k), sig (k) with
// Mx ~ (Qy Ut) diag(sig) (Qz Wt)^T.  bf16: the contractions with Mx on the
// tensor cores (fp32 data only; svd_work_bf16 must have sized the buffers).
// Us, svt (optional): the SVT on the factors (launch_svt_small for svt) fused
// into the core SVD.
template <typename T>
void subspace_svd(cpcp_context *h, SvdWork<T> &w, int m, int nc, const T *Mx, int64_t ldx, const T *Omega,
                  int q, const int *kdyn, const Ctrl *jac_ctrl, bool bf16 = false, T *Us = nullptr,
                  Ctrl *svt = nullptr)
{
    if constexpr (std::is_same<T, float>::value) {
        if (bf16) {
            subspace_svd_bf16(h, w, m, nc, Mx, ldx, Omega, q, kdyn, jac_ctrl, Us, svt);
            return;
        }
    }
    cudaStream_t st = h->stream;
    const int KM = w.KM;
    const T *Om = Omega;
    for (int s = 0; s < q; s++) {
        int tp = h->timer.open_sub(DETAIL_PROD_M);
        prod_y<T>(w, m, nc, Mx, ldx, Om, kdyn, st);
        h->timer.close(tp);
        orth<T>(h, w, m, w.Y, w.Qy, nullptr, kdyn, 0);
        tp = h->timer.open_sub(DETAIL_PROD_M);
        prod_z<T>(w, m, nc, Mx, ldx, w.Qy, KM, kdyn, st);
        h->timer.close(tp);
        orth<T>(h, w, nc, w.Z, w.Qz, w.Rz, kdyn, 1);
        Om = w.Qz;
    }
    const int tj = h->timer.open_sub(DETAIL_JACOBI);
    launch_jacobi<T>(w.Rz, KM, kdyn, w.Ut, w.Wt, w.sig, w.kcap, jac_ctrl, st, w.stats, Us, svt,
                     h->opt.jacobi_lanes == 8 ? 8 : 16,
                     h->timer.in_iter ? h->opt.jacobi_check : 0);
    h->timer.close(tj);
}

template <typename T>
int kmax_small();
template <>
int kmax_small<float>()
{
    return small_kmax_f32();
}
template <>
int kmax_small<double>()
{
    return small_kmax_f64();
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------

struct Opts {
    int max_iter, check_every, k_max, p, q, qc, start_level, precision, tc_pass, graphs, transfer;
    bool early_test;
    double eta, mu0, ratio, refine_at;
    uint64_t seed;
};

Opts resolve(const cpcp_options &o)
{
    Opts r;
    r.max_iter = o.max_iter > 0 ? o.max_iter : 5000;
    r.check_every = o.check_every > 0 ? o.check_every : 10;
    r.eta = o.eta > 0 ? o.eta : 0.9;
    r.mu0 = o.mu0;
    r.ratio = o.switch_ratio > 0 ? o.switch_ratio : 0.9;
    r.k_max = o.k_max > 0 ? o.k_max : 256;
    r.p = o.oversample > 0 ? o.oversample : 10;
    r.q = o.power_iters > 0 ? o.power_iters : 1;
    r.qc = o.check_power_iters > 0 ? o.check_power_iters : 2;
    r.start_level = o.start_level;
    r.precision = o.precision;
    r.tc_pass = o.pass_simt == 0;
    r.graphs = o.plain_launches == 0;
    r.transfer = o.transfer;
    r.early_test = o.early_test >= 0;
    r.refine_at = o.refine_at > 0 ? o.refine_at : 1e-3;
    r.seed = o.seed ? o.seed : 1;
    return r;
}

template <typename T>
struct SolveState {
    int m, n, ldS, KM, kcap0;
    const T *D;
    int64_t ldd;
    const uint32_t *Q;
    int64_t ldq;
    T *S[2], *A[2], *B[2];
    T *M, *MH, *GH;
    int64_t ldMH;
    T *Om, *Omf, *Ac, *Bc;
    Ctrl *ctrl, *cchk;
    double *partial, *sums;
    // overlapped fine checks: the snapshot of the checked iterate (S, A, B and
    // the control block) and the check's own M and partial sums
    T *Ssnap = nullptr, *Asnap = nullptr, *Bsnap = nullptr, *Mc = nullptr;
    Ctrl *csnap = nullptr;
    double *partial_c = nullptr, *sums_c = nullptr;
    int partial_blocks;
    bool bf16;  // contractions of the iteration's SVD in BF16 (mixed precision, before refinement)
    int *tc_err = nullptr;  // set: the fine pass runs on the tensor cores (its bounded-wait error flag)
    // orthonormal-basis transfer on the coarse levels (option transfer = 1): per level the
    // bidiagonal factor and level-test threshold, and a coarse n_H x KM scratch for C^{-1} V
    bool orth = false;
    std::vector<OrthTransfer<T>> ot;
    T *Vp = nullptr;
    std::vector<TransferDev<T>> tr;
};

template <typename T>
PassArgs<T> base_args(SolveState<T> &s)
{
    PassArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.m = s.m;
    a.n = s.n;
    a.D = s.D;
    a.ldd = s.ldd;
    a.Q = s.Q;
    a.ldq = s.ldq;
    a.lds = s.ldS;
    a.ldso = s.ldS;
    a.ldfa = s.KM;
    a.ldfb = s.KM;
    a.ldfap = s.KM;
    a.ldfbp = s.KM;
    a.ctrl = s.ctrl;
    a.ldm = s.ldS;
    a.M = s.M;
    a.partial = s.partial;
    return a;
}

// Where a fine residual check reads the checked iterate and writes its
// scratch: the solve's live buffers (a check run in order), or a snapshot of
// the iterate with scratch of its own (a check run on the second stream while
// the next iterations are computed).  host: pinned memory for the results
// (six sums, then the check's control block).
template <typename T>
struct CheckSrc {
    const T *S, *A, *B;
    const Ctrl *it;  // the iteration's control block at the checked iterate (its rank rk)
    T *M;
    double *partial, *sums;
    double *host;
};

double *check_host(cpcp_context *h)
{
    if (!h->check_host) CK(cudaMallocHost(&h->check_host, 64 + sizeof(Ctrl)));
    return static_cast<double *>(h->check_host);
}

// Fine-level residual at (L_k, S_k) = (A B^T, S) of src for the weight mu_c:
// the launches, on h->stream, ending with the copy of the results to
// src.host.
template <typename T>
void check_launch(cpcp_context *h, SolveState<T> &s, SvdWork<T> &wf, const CheckSrc<T> &src, const Opts &o,
                  double mu_c)
{
    cudaStream_t st = h->stream;
    int tmr = h->timer.open(CPCP_PHASE_CHECK);
    launch_ctrl_set_check(s.cchk, src.it, mu_c, st);
    PassArgs<T> a = base_args(s);
    a.ctrl = s.cchk;
    a.M = src.M;
    a.partial = src.partial;
    a.Sk = src.S;
    a.Ak = src.A;
    a.Bk = src.B;
    a.rk = &src.it->rk;
    int nb = launch_check_pass<T>(a, st);
    launch_sum_partials(src.partial, nb, 3, src.sums, st);
    // fine SVT of M = L - tau G with width kf, warm-started from the last check
    launch_fill_random<T>(s.Omf, s.KM, s.n, s.cchk, 0, wf.sig, s.KM, 0xC4ECull, st);
    launch_ctrl_take_width(s.cchk, st);
    subspace_svd<T>(h, wf, s.m, s.n, src.M, s.ldS, s.Omf, o.qc, &s.cchk->k, s.cchk, false, wf.Us, s.cchk);
    prod_nn_small<T>(s.m, wf.Qy, wf.KM, wf.Us, wf.KM, s.Ac, s.KM, &s.cchk->k, wf.KM, st);
    prod_nn_small<T>(s.n, wf.Qz, wf.KM, wf.Wt, wf.KM, s.Omf, s.KM, &s.cchk->k, wf.KM, st);
    launch_prolong<T>(s.n, s.Omf, s.KM, s.Bc, s.KM, s.tr[0], &s.cchk->r_new, s.KM, st);
    PassArgs<T> b = base_args(s);
    b.ctrl = s.cchk;
    b.M = src.M;
    b.partial = src.partial;
    b.Ak = src.A;
    b.Bk = src.B;
    b.Ap = s.Ac;
    b.Bp = s.Bc;
    b.rk = &src.it->rk;
    b.rp = &s.cchk->r_new;
    nb = launch_diff_pass<T>(b, st);
    launch_sum_partials(src.partial, nb, 3, src.sums + 3, st);
    h->timer.close(tmr);
    CK(cudaMemcpyAsync(src.host, src.sums, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(src.host + 8, s.cchk, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
}

// The check's results once stream `st` (the one check_launch used) has run
// them: rel-KKT (or +inf when the fine SVT width was insufficient), the next
// check's width, the S part of the residual and the rank of the check's SVT.
template <typename T>
double check_finish(cpcp_context *h, SolveState<T> &s, const CheckSrc<T> &src, const Opts &o, double pqd, int *kf,
                    double *s_part_out, int *rank_out, cudaStream_t st)
{
    CK(cudaStreamSynchronize(st));
    h->timer.harvest();
    double sums[6];
    Ctrl cc;
    memcpy(sums, src.host, sizeof(sums));
    memcpy(&cc, src.host + 8, sizeof(Ctrl));
    *s_part_out = sums[0];
    int kcur = cc.k;
    int r = cc.r_new;
    bool saturated = (r >= kcur) && (kcur < s.kcap0);
    // width for the next check: rank + oversampling, doubled if saturated;
    // columns [kcur, want) get random vectors before the next check
    int want = saturated ? std::min(s.kcap0, 2 * kcur) : std::min(s.kcap0, std::max(r + o.p, 1));
    *kf = want;
    Ctrl upd = cc;
    upd.k = kcur;
    upd.k_next = want;
    CK(cudaMemcpyAsync(s.cchk, &upd, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    *rank_out = r;
    if (saturated) return INFINITY;
    double tau = 0.5;
    return std::sqrt(std::max(sums[0] + sums[3], 0.0)) / tau / pqd;
}

// Fine-level residual at (L_k, S_k) = (A[cur] B[cur]^T, S[cur]), in order on
// the solve's stream.
template <typename T>
double fine_check(cpcp_context *h, SolveState<T> &s, SvdWork<T> &wf, int cur, const Opts &o, double pqd,
                  double mu_c, int *kf, double *s_part_out, int *rank_out)
{
    const CheckSrc<T> src{s.S[cur], s.A[cur], s.B[cur], s.ctrl, s.M, s.partial, s.sums, check_host(h)};
    check_launch<T>(h, s, wf, src, o, mu_c);
    return check_finish<T>(h, s, src, o, pqd, kf, s_part_out, rank_out, h->stream);
}

// One iteration.  With want_g on a coarse level the pass also restricts the
// gradient; s.sums[8] then holds ||G||_F^2 and s.sums[11] ||G R||_F^2.
template <typename T>
// part 0: the whole iteration; 1: the schedule update and the fused pass
// only; 2: the rest (subspace SVD, SVT, new factors, schedule end), which the
// caller times itself (part 2 is what the solver replays as a CUDA graph).
void one_iteration(cpcp_context *h, SolveState<T> &s, SvdWork<T> &w, int level, int cur, const Opts &o,
                   bool want_g, int part = 0)
{
    cudaStream_t st = h->stream;
    const int nxt = cur ^ 1;
    const TransferDev<T> &tr = s.tr[level];
    const T *Mx = level > 0 ? s.MH : s.M;
    const int64_t ldx = level > 0 ? s.ldMH : s.ldS;
    if (part != 2) {
    launch_ctrl_begin(s.ctrl, st);
    PassArgs<T> a = base_args(s);
    a.Sk = s.S[cur];
    a.Sp = s.S[nxt];
    a.Sout = s.S[nxt];
    a.Ak = s.A[cur];
    a.Bk = s.B[cur];
    a.Ap = s.A[nxt];
    a.Bp = s.B[nxt];
    a.rk = &s.ctrl->rk;
    a.rp = &s.ctrl->rp;
    if (level > 0) {
        CK(cudaMemsetAsync(s.MH, 0, sizeof(T) * (size_t)s.m * s.ldMH, st));
        a.M = nullptr;
        a.MH = s.MH;
        a.ldh = s.ldMH;
        a.tr = tr;
        if (want_g) {
            CK(cudaMemsetAsync(s.GH, 0, sizeof(T) * (size_t)s.m * s.ldMH, st));
            a.GH = s.GH;
        }
        int tp = h->timer.open(CPCP_PHASE_PASS_COARSE);
        int nb = launch_step_pass<T>(a, true, st);
        // orthonormal basis of the coarse range: M_H C^{-1}
        if (s.orth) launch_bidiag_right_solve<T>(s.m, tr.nh, s.MH, s.ldMH, s.ot[level].cd, s.ot[level].ce, st);
        h->timer.close(tp);
        if (want_g) {
            launch_sum_partials(s.partial, nb, 3, s.sums + 8, st);
            if (s.orth) launch_bidiag_right_solve<T>(s.m, tr.nh, s.GH, s.ldMH, s.ot[level].cd, s.ot[level].ce, st);
            int nq = launch_sumsq<T>(s.m, tr.nh, s.GH, s.ldMH, s.partial, st);
            launch_sum_partials(s.partial, nq, 1, s.sums + 11, st);
        }
    } else {
        int tp = h->timer.open(CPCP_PHASE_PASS_FINE);
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (s.tc_err != nullptr) done = launch_pass_tc(a, s.tc_err, st);
        }
        if (!done) launch_step_pass<T>(a, false, st);
        h->timer.close(tp);
    }
    }
    if (part == 1) return;
    const int ts = part == 0 ? h->timer.open(CPCP_PHASE_SVT) : -1;
    h->timer.in_iter = true;
    bool two = false;
    if constexpr (std::is_same<T, float>::value)
        two = !s.bf16 && o.q == 1 && h->opt.svd_serial != 1 && w.KM <= kmax_small<float>();
    if constexpr (std::is_same<T, float>::value) {
        if (two) subspace_svd_iter(h, w, s.m, tr.nh, Mx, ldx, s.Om, &s.ctrl->k, s.ctrl, w.Us, s.ctrl);
    }
    // (programmatic dependent launch stays with the two-stream form: in the
    // in-order form it made the 4-level video solve 3.6 ms slower, 93.2 ->
    // 96.8 ms, its waiting CTAs holding SMs that the other streams' kernels use)
    if (!two) subspace_svd<T>(h, w, s.m, tr.nh, Mx, ldx, s.Om, o.q, &s.ctrl->k, s.ctrl, s.bf16, w.Us, s.ctrl);
    const int tf = h->timer.open_sub(DETAIL_FACTORS);
    h->timer.in_iter = false;
    // new factors into the "previous" slot (its old content was consumed
    // above); with the two-stream SVD, A = Q_Y U_s on the solve stream beside
    // the next start block V = Q_Z W_t on the second one
    if (two) {
        cudaStream_t ax = h->opt.svd_serial == 2 ? st : iter_aux(h);
        order_after(h, ax, st, 5);
        if (ax != st) CK(cudaStreamWaitEvent(st, h->ev_aux[3], 0));
        prod_nn_small<T>(s.m, w.Qy, w.KM, w.Us, w.KM, s.A[nxt], s.KM, &s.ctrl->k, w.KM, st);
        prod_nn_small<T>(tr.nh, w.Qz, w.KM, w.Wt, w.KM, s.Om, s.KM, &s.ctrl->k, w.KM, ax);
        order_after(h, st, ax, 6);
    } else {
        prod_nn_small<T>(s.m, w.Qy, w.KM, w.Us, w.KM, s.A[nxt], s.KM, &s.ctrl->k, w.KM, st);
        prod_nn_small<T>(tr.nh, w.Qz, w.KM, w.Wt, w.KM, s.Om, s.KM, &s.ctrl->k, w.KM, st);
    }
    if (s.orth && level > 0) {
        // B = R C^{-1} V; the next start block keeps V (random columns into Vp are unused)
        launch_bidiag_left_solve<T>(tr.nh, s.Om, s.KM, &s.ctrl->k, s.KM, s.ot[level].cd, s.ot[level].ce, s.Vp, s.KM,
                                    st);
        launch_fill_prolong<T>(s.Vp, s.KM, tr.nh, s.ctrl, w.sig, s.KM, 0x57E9ull, s.n, s.B[nxt], s.KM, tr, st);
        launch_fill_random<T>(s.Om, s.KM, tr.nh, s.ctrl, 0, w.sig, s.KM, 0x57EBull, st);
    } else {
        launch_fill_prolong<T>(s.Om, s.KM, tr.nh, s.ctrl, w.sig, s.KM, 0x57E9ull, s.n, s.B[nxt], s.KM, tr, st);
    }
    h->timer.close(tf);
    h->timer.close(ts);
    {
        PdlScope ps(two && h->opt.pdl_off == 0 && !h->timer.detail);
        launch_ctrl_end(s.ctrl, st);
    }
}

// Runs the solve on the handle's private stream: ordered after the work the
// caller queued on its stream, and the caller's stream waits for the solve
// (on every exit path).
struct PrivateStream {
    cpcp_context *h;
    cudaStream_t user;
    bool on = false;
    PrivateStream(cpcp_context *h_, bool use) : h(h_), user(h_->stream)
    {
        if (!use) return;
        if (!h->solve_stream) CK(cudaStreamCreateWithFlags(&h->solve_stream, cudaStreamNonBlocking));
        if (!h->ev_in) CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
        if (!h->ev_out) CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
        CK(cudaEventRecord(h->ev_in, user));
        CK(cudaStreamWaitEvent(h->solve_stream, h->ev_in, 0));
        h->stream = h->solve_stream;
        on = true;
    }
    ~PrivateStream()
    {
        if (!on) return;
        cudaEventRecord(h->ev_out, h->solve_stream);
        cudaStreamWaitEvent(user, h->ev_out, 0);
        h->stream = user;
    }
};

// One iteration's kernels as an instantiated CUDA graph (per level and buffer
// parity); destroyed with the solve.
struct IterGraph {
    bool seen = false;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;
};

struct IterGraphs {
    IterGraph g[8][2];  // level, buffer parity
    ~IterGraphs()
    {
        for (auto &row : g)
            for (auto &x : row)
                if (x.exec) cudaGraphExecDestroy(x.exec);
    }
};

template <typename T>
cpcp_status solve_core(cpcp_context *h, int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq,
                       double lam, double mu, int levels, double tol, T *L_out, int64_t ldl, T *S_out, int64_t lds,
                       cpcp_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    const Opts o = resolve(h->opt);
    // iterations without a level decision replay a CUDA graph of their kernels
    // (captured the second time the same level and buffer parity come up,
    // once every workspace buffer exists); the kernels read the iteration's
    // scalars (weights, widths, ranks) from the device control block
    // (profile >= 2 times kernel families inside the iteration: plain launches)
    const bool use_graphs = o.graphs && h->opt.profile < 2;
    PrivateStream ps(h, use_graphs);
    cudaStream_t st = h->stream;
    const int H = levels - 1;
    h->timer.reset(h->opt.profile != 0, st, h->opt.profile >= 2);
    if (std::is_same<T, float>::value) iter_aux(h);  // created before any stream capture
    const unsigned long long launches0 = g_kernel_launches;
    SolveState<T> s;
    s.m = m;
    s.n = n;
    s.D = D;
    s.ldd = ldd;
    s.Q = Q;
    s.ldq = ldq;
    s.ldS = round4(n);
    s.kcap0 = std::min({o.k_max, kmax_small<T>(), n});
    s.KM = (int)round4(s.kcap0);
    const size_t mn = (size_t)m * s.ldS;
    for (int i = 0; i < 2; i++) {
        s.S[i] = wsT<T>(h, "S" + std::to_string(i), mn);
        s.A[i] = wsT<T>(h, "A" + std::to_string(i), (size_t)m * s.KM);
        s.B[i] = wsT<T>(h, "B" + std::to_string(i), (size_t)n * s.KM);
    }
    s.M = wsT<T>(h, "M", mn);
    s.tr.clear();
    for (int lv = 0; lv <= H; lv++) s.tr.push_back(upload_transfer<T>(h, n, lv, "solve"));
    int nh1 = H >= 1 ? s.tr[1].nh : 1;
    s.ldMH = round4(nh1);
    s.MH = wsT<T>(h, "MH", (size_t)m * s.ldMH);
    s.GH = wsT<T>(h, "GH", (size_t)m * s.ldMH);
    s.orth = H > 0 && o.transfer == 1;
    s.ot.clear();
    if (s.orth) {
        s.ot.emplace_back();  // level 0: no transfer
        for (int lv = 1; lv <= H; lv++) s.ot.push_back(upload_orth<T>(h, n, lv, "solve_o" + std::to_string(lv)));
        s.Vp = wsT<T>(h, "Vp", (size_t)nh1 * s.KM);
    }
    s.Om = wsT<T>(h, "Om", (size_t)n * s.KM);
    s.Omf = wsT<T>(h, "Omf", (size_t)n * s.KM);
    s.Ac = wsT<T>(h, "Ac", (size_t)m * s.KM);
    s.Bc = wsT<T>(h, "Bc", (size_t)n * s.KM);
    s.ctrl = wsT<Ctrl>(h, "ctrl", 1);
    s.cchk = wsT<Ctrl>(h, "cchk", 1);
    s.partial_blocks = ((n + 63) / 64) * ((m + 63) / 64);
    s.partial = wsT<double>(h, "partial", (size_t)std::max(s.partial_blocks * 3, 512));
    s.sums = wsT<double>(h, "sums", 16);
    const bool overlap = use_graphs && h->opt.check_serial == 0;
    if (overlap) {
        s.Ssnap = wsT<T>(h, "Ssnap", mn);
        s.Asnap = wsT<T>(h, "Asnap", (size_t)m * s.KM);
        s.Bsnap = wsT<T>(h, "Bsnap", (size_t)n * s.KM);
        s.Mc = wsT<T>(h, "Mc", mn);
        s.csnap = wsT<Ctrl>(h, "csnap", 1);
        s.partial_c = wsT<double>(h, "partial_c", (size_t)std::max(s.partial_blocks * 3, 512));
        s.sums_c = wsT<double>(h, "sums_c", 16);
        if (!h->check_stream) {
            // lowest priority: the iterations' latency chain goes first
            int least = 0, greatest = 0;
            CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            CK(cudaStreamCreateWithPriority(&h->check_stream, cudaStreamNonBlocking, least));
        }
        if (!h->ev_snap) CK(cudaEventCreateWithFlags(&h->ev_snap, cudaEventDisableTiming));
    }
    SvdWork<T> w = svd_work<T>(h, "it_", m, n, s.kcap0);
    SvdWork<T> wf = svd_work<T>(h, "ck_", m, n, s.kcap0);
    w.stats = wf.stats = wsT<int>(h, "svd_stats", 4);
    CK(cudaMemsetAsync(w.stats, 0, sizeof(int) * 4, st));
    s.bf16 = o.precision == 1;
    if (s.bf16) svd_work_bf16<T>(h, w, "it_", m, n);
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    if (std::is_same<T, float>::value && o.tc_pass) {
        s.tc_err = wsT<int>(h, "tc_err", 1);
        CK(cudaMemsetAsync(s.tc_err, 0, sizeof(int), st));
    }

    // control blocks
    Ctrl c0;
    memset(&c0, 0, sizeof(c0));
    c0.eta_k = 1.0;
    c0.tau = 0.5;
    c0.lam = lam;
    c0.mu_bar = mu;
    c0.eta = o.eta;
    c0.t = 1.0;
    c0.oversample = o.p;
    c0.seed = o.seed;
    Ctrl cc = c0;
    cc.theta_L = 0.5 * mu;
    cc.k = std::min(s.kcap0, 8);
    cc.k_next = cc.k;
    cc.kcap = s.kcap0;
    cc.mu_k = mu;
    CK(cudaMemcpyAsync(s.cchk, &cc, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));

    // norms of P_Q D, finiteness, and mu_0 = ||P_Q D||_2 estimate (fine SVD of tau P_Q D)
    PassArgs<T> a0 = base_args(s);
    int nb = launch_check_pass<T>(a0, st);
    launch_sum_partials(s.partial, nb, 3, s.sums, st);
    double sums0[3];
    CK(cudaMemcpyAsync(sums0, s.sums, sizeof(sums0), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (sums0[2] > 0) throw CpcpError{CPCP_ERR_NONFINITE_INPUT, "non-finite value in an observed entry of D"};
    const double pqd = std::sqrt(sums0[1]);
    if (!(pqd > 0)) throw CpcpError{CPCP_ERR_INVALID_ARG, "P_Q[D] is zero"};
    double mu0 = o.mu0;
    if (!(mu0 > 0)) {
        launch_fill_random<T>(s.Omf, s.KM, n, s.cchk, 1, nullptr, s.KM, 0x30ull, st);
        subspace_svd<T>(h, wf, m, n, s.M, s.ldS, s.Omf, 4, &s.cchk->k, nullptr);
        T sig0;
        CK(cudaMemcpyAsync(&sig0, wf.sig, sizeof(T), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        mu0 = (double)sig0 / 0.5;
    }
    // start state
    // start_level 0 (default) = coarsest; s > 0 starts at min(s, levels) - 1 halvings
    int level = o.start_level > 0 ? std::min(o.start_level - 1, H) : H;
    c0.mu0 = mu0;
    c0.k = std::min(o.p, std::min(s.kcap0, s.tr[level].nh));
    c0.k_next = c0.k;
    c0.kcap = std::min(s.kcap0, s.tr[level].nh);
    CK(cudaMemcpyAsync(s.ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    cc.k = std::min(s.kcap0, o.p);
    cc.k_next = cc.k;
    CK(cudaMemcpyAsync(s.cchk, &cc, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(s.S[0], 0, sizeof(T) * mn, st));
    CK(cudaMemsetAsync(s.S[1], 0, sizeof(T) * mn, st));
    launch_fill_random<T>(s.Om, s.KM, s.tr[level].nh, s.ctrl, 1, nullptr, s.KM, 0x11ull, st);
    CK(cudaMemsetAsync(s.Omf, 0, sizeof(T) * (size_t)n * s.KM, st));
    CK(cudaMemsetAsync(wf.sig, 0, sizeof(T) * wf.KM, st));
    launch_fill_random<T>(s.Omf, s.KM, n, s.cchk, 1, nullptr, s.KM, 0x12ull, st);

    cpcp_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.mu0 = mu0;
    inf.pqd_fro = pqd;
    int cur = 0, iter = 0, checks = 0, kf = cc.k, rank = 0;
    int level_start = 0;  // iteration at which the current level began
    double rel = INFINITY, prev = INFINITY;
    double prev2 = INFINITY;  // the check before prev (on the same level), for the overlap's guess
    cpcp_status status = CPCP_ERR_NOT_CONVERGED;
    IterGraphs graphs;
    // one iteration at the current level and buffer parity: with graph replay
    // the schedule update and the fused pass are launched directly (the
    // profile's events bracket the pass) and the rest of the iteration is the
    // graph
    auto run_iteration = [&](bool want_g) {
        h->timer.level = level;
        if (use_graphs && !want_g && !s.bf16 && level < 8) {
            one_iteration<T>(h, s, w, level, cur, o, false, 1);
            IterGraph &G = graphs.g[level][cur];
            if (G.exec == nullptr && G.seen) {
                const unsigned long long l0 = g_kernel_launches;
                CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                cudaGraph_t graph = nullptr;
                try {
                    one_iteration<T>(h, s, w, level, cur, o, false, 2);
                } catch (...) {
                    cudaStreamEndCapture(st, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    throw;
                }
                CK(cudaStreamEndCapture(st, &graph));
                const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
                cudaGraphDestroy(graph);
                CK(ie);
                G.launches = g_kernel_launches - l0;
                g_kernel_launches = l0;
            }
            const int ts = h->timer.open(CPCP_PHASE_SVT);
            if (G.exec != nullptr) {
                CK(cudaGraphLaunch(G.exec, st));
                g_kernel_launches += G.launches;
            } else {
                G.seen = true;
                one_iteration<T>(h, s, w, level, cur, o, false, 2);
            }
            h->timer.close(ts);
        } else {
            one_iteration<T>(h, s, w, level, cur, o, want_g);
        }
        cur ^= 1;
    };
    for (iter = 0; iter < o.max_iter;) {
        // every check_every iterations: a level decision (coarse levels) and,
        // once the weight is final, the fine residual check; with the early
        // test also the coarse-gradient test at a coarse level's first iteration
        const bool decide = (iter + 1) % o.check_every == 0;
        const bool early = o.early_test && level > 0 && iter == level_start;
        const bool want_g = (decide || early) && level > 0;
        run_iteration(want_g);
        if (level < 8) inf.level_iters[level]++;
        if (s.bf16) inf.bf16_iters++;
        iter++;
        if (!decide && !early) continue;
        // weight of the iteration just done: mu_k = max(mu0 eta^k, mu)
        const double mu_k = std::max(mu0 * std::pow(o.eta, (double)(iter - 1)), mu);
        const bool at_final = !(mu_k > mu);
        bool finer = false;
        if (level > 0) {
            // coarse-gradient test: keep the coarse model while G R carries at
            // least kappa of ||G||
            double g2[4];
            CK(cudaMemcpyAsync(g2, s.sums + 8, sizeof(g2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            const double kap = s.orth ? s.ot[level].kappa : s.tr[level].kappa;
            if (g2[0] > 0.0 && std::sqrt(std::max(g2[3], 0.0)) < kap * std::sqrt(g2[0])) finer = true;
        }
        if (decide && !finer && at_final) {
            double spart;
            // on the fine level the check can only stop the solve or let it go
            // on: it then runs on the check stream, from a snapshot of the
            // iterate, while the solve stream computes the next iterations
            // (none of them a decision point), which count only if it goes on
            const bool ovl = overlap && level == 0 && !s.bf16;
            int nspec = 0;
            const int cur_k = cur;
            if (ovl) {
                // iterations computed meanwhile: five while the last two checks'
                // rate says this one will not stop the solve, else one (the ones
                // computed beside the stopping check are dropped, and the result
                // waits for them).  The count changes no result.
                const bool hist = std::isfinite(prev) && std::isfinite(prev2) && prev2 > 0.0;
                const int want = (hist && prev * (prev / prev2) <= tol) ? 1 : 5;
                nspec = std::min({want, o.check_every - 1, o.max_iter - iter});
                CK(cudaMemcpyAsync(s.Ssnap, s.S[cur], sizeof(T) * (size_t)m * s.ldS, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(s.Asnap, s.A[cur], sizeof(T) * (size_t)m * s.KM, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(s.Bsnap, s.B[cur], sizeof(T) * (size_t)n * s.KM, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(s.csnap, s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, st));
                CK(cudaEventRecord(h->ev_snap, st));
                CK(cudaStreamWaitEvent(h->check_stream, h->ev_snap, 0));
                const CheckSrc<T> src{s.Ssnap, s.Asnap, s.Bsnap, s.csnap, s.Mc, s.partial_c, s.sums_c, check_host(h)};
                h->stream = h->check_stream;
                h->timer.st = h->check_stream;
                try {
                    check_launch<T>(h, s, wf, src, o, mu);
                } catch (...) {
                    h->stream = st;
                    h->timer.st = st;
                    throw;
                }
                h->stream = st;
                h->timer.st = st;
                h->timer.spec = true;
                for (int i = 0; i < nspec; i++) run_iteration(false);
                h->timer.spec = false;
                rel = check_finish<T>(h, s, src, o, pqd, &kf, &spart, &rank, h->check_stream);
            } else {
                rel = fine_check<T>(h, s, wf, cur, o, pqd, mu, &kf, &spart, &rank);
            }
            if (h->opt.trace && checks < h->opt.trace_cap) h->opt.trace[checks] = rel;
            checks++;
            if (rel <= tol) {
                status = CPCP_OK;
                if (ovl) {
                    // the checked iterate is the result: drop the iterations
                    // computed meanwhile and put it back in its slot
                    CK(cudaStreamSynchronize(st));
                    h->timer.drop_spec();
                    cur = cur_k;
                    CK(cudaMemcpyAsync(s.S[cur], s.Ssnap, sizeof(T) * (size_t)m * s.ldS, cudaMemcpyDeviceToDevice,
                                       st));
                    CK(cudaMemcpyAsync(s.A[cur], s.Asnap, sizeof(T) * (size_t)m * s.KM, cudaMemcpyDeviceToDevice, st));
                    CK(cudaMemcpyAsync(s.B[cur], s.Bsnap, sizeof(T) * (size_t)n * s.KM, cudaMemcpyDeviceToDevice, st));
                    CK(cudaMemcpyAsync(s.ctrl, s.csnap, sizeof(Ctrl), cudaMemcpyDeviceToDevice, st));
                }
                break;
            }
            if (ovl) {
                h->timer.keep_spec();
                inf.level_iters[0] += nspec;
                iter += nspec;
            }
            if (level > 0 && rel > o.ratio * prev) finer = true;
            prev2 = prev;
            prev = rel;
            if (s.bf16 && rel <= o.refine_at) {
                // mixed precision: fp32 contractions from here on, momentum restarts
                s.bf16 = false;
                if (!finer) {
                    Ctrl c;
                    CK(cudaMemcpyAsync(&c, s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                    c.t = 1.0;
                    CK(cudaMemcpyAsync(s.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
                }
            }
        }
        if (finer) {
            // move one level finer: restart momentum, warm-start the subspace
            // from the restriction of the current right factor
            level--;
            level_start = iter;
            prev = INFINITY;
            prev2 = INFINITY;
            Ctrl cur_c;
            CK(cudaMemcpyAsync(&cur_c, s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            cur_c.t = 1.0;
            cur_c.kcap = std::min(s.kcap0, s.tr[level].nh);
            cur_c.k = std::min(cur_c.kcap, std::max(cur_c.rk + o.p, 1));
            cur_c.k_next = cur_c.k;
            CK(cudaMemcpyAsync(s.ctrl, &cur_c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
            launch_restrict_rows<T>(s.B[cur], s.KM, s.Om, s.KM, s.tr[level], &s.ctrl->rk, s.KM, st);
            // columns beyond the rank get random vectors
            Ctrl tmp = cur_c;
            tmp.k = std::max(cur_c.rk, 0);
            tmp.k_next = cur_c.k;
            Ctrl *ctmp = wsT<Ctrl>(h, "ctmp", 1);
            CK(cudaMemcpyAsync(ctmp, &tmp, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
            launch_fill_random<T>(s.Om, s.KM, s.tr[level].nh, ctmp, 0, nullptr, s.KM, 0x77ull + level, st);
            CK(cudaStreamSynchronize(st));
        }
    }
    inf.iters = iter;
    inf.final_level = level;
    inf.checks = checks;
    inf.relkkt = rel;
    Ctrl fin;
    CK(cudaMemcpyAsync(&fin, s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    int stats[4];
    CK(cudaMemcpyAsync(stats, w.stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    int umma_err = 0, tc_err = 0;
    if (w.err) CK(cudaMemcpyAsync(&umma_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (s.tc_err) CK(cudaMemcpyAsync(&tc_err, s.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (umma_err || tc_err) throw CpcpError{CPCP_ERR_TIMEOUT, "a bounded wait of the tensor-core kernel expired"};
    inf.rank = fin.rk;
    inf.jacobi_calls = stats[0];
    inf.jacobi_sweeps = stats[1];
    inf.chol_factors = stats[2];
    // outputs
    if (S_out) {
        CK(cudaMemcpy2DAsync(S_out, sizeof(T) * lds, s.S[cur], sizeof(T) * s.ldS, sizeof(T) * n, m,
                             cudaMemcpyDeviceToDevice, st));
    }
    if (L_out) {
        PassArgs<T> r = base_args(s);
        r.Ak = s.A[cur];
        r.Bk = s.B[cur];
        r.rk = &s.ctrl->rk;
        r.M = L_out;
        r.ldm = ldl;
        launch_reconstruct<T>(r, st);
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    inf.status = status;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.launches = (long long)(g_kernel_launches - launches0);
    h->timer.harvest();
    for (int i = 0; i < CPCP_NUM_PHASES; i++) {
        inf.phase_ms[i] = h->timer.ms[i];
        inf.phase_count[i] = h->timer.count[i];
        inf.svt_detail_ms[i] = h->timer.ms[DETAIL_PROD_M + i];
    }
    for (int i = 0; i < 8; i++) inf.level_ms[i] = h->timer.lvl_ms[i];
    if (info) *info = inf;
    return status;
}

bool is_device_ptr(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// IALM (Alg. 1) / ML-IALM (Alg. 4) for PCP on device buffers, n <= m; see
// cpcp_ialm.  The low-rank step is the CPCP path's: M (or its restriction
// M R) -> warm-started subspace SVD with the SVT fused into its core SVD ->
// factors A = U diag(sigma - 1/mu)_+ and B = R V -> L = A B^T.
template <typename T>
cpcp_status ialm_core(cpcp_context *h, int m, int n, const T *D, int64_t ldd, double lam, int levels, double mu0,
                      double rho, int max_iter, double tol, T *L_out, int64_t ldl, T *S_out, int64_t lds,
                      double *fg, cpcp_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    const unsigned long long launches0 = g_kernel_launches;
    cudaStream_t st = h->stream;
    const Opts o = resolve(h->opt);
    const int H = levels - 1;
    const int64_t ldS = round4(n);
    const int kcap0 = std::min({o.k_max, kmax_small<T>(), n});
    const int KM = (int)round4(kcap0);
    const size_t mn = (size_t)m * ldS;
    T *S = wsT<T>(h, "ia_S", mn), *Y = wsT<T>(h, "ia_Y", mn), *M = wsT<T>(h, "ia_M", mn), *L = wsT<T>(h, "ia_L", mn);
    TransferDev<T> tr = upload_transfer<T>(h, n, H, "ialm");
    const int nh = tr.nh;
    const int64_t ldh = round4(nh);
    T *MH = H > 0 ? wsT<T>(h, "ia_MH", (size_t)m * ldh) : nullptr;
    T *A = wsT<T>(h, "ia_A", (size_t)m * KM), *B = wsT<T>(h, "ia_B", (size_t)n * KM);
    T *Om = wsT<T>(h, "ia_Om", (size_t)n * KM);
    Ctrl *ctrl = wsT<Ctrl>(h, "ia_ctrl", 1);
    const int nblk = ialm_blocks();
    double *partial = wsT<double>(h, "ia_partial", (size_t)std::max(nblk, 1024));
    double *sums = wsT<double>(h, "ia_sums", 4);
    SvdWork<T> w = svd_work<T>(h, "ia_svd_", m, n, kcap0);  // own tags: "ia_Y" is the multiplier
    tc_err_clear(w.err, h->stream);
    // orthonormal-basis transfer (option): R C^{-1} with R^T R = C^T C
    const bool orth = H > 0 && o.transfer == 1;
    T *Cd = nullptr, *Ce = nullptr, *Vp = nullptr;
    if (orth) {
        const OrthTransfer<T> ot = upload_orth<T>(h, n, H, "ia");
        Cd = ot.cd;
        Ce = ot.ce;
        Vp = wsT<T>(h, "ia_Vp", (size_t)nh * KM);
    }

    // ||D||_F, and ||D||_2 for the default mu0 (subspace SVD of D, 4 passes)
    const int nq = launch_sumsq<T>(m, n, D, ldd, partial, st);
    launch_sum_partials(partial, nq, 1, sums, st);
    double d2 = 0.0;
    CK(cudaMemcpyAsync(&d2, sums, sizeof(double), cudaMemcpyDeviceToHost, st));
    Ctrl c0;
    memset(&c0, 0, sizeof(c0));
    c0.eta_k = 1.0;
    c0.tau = 1.0;
    c0.lam = lam;
    c0.mu_bar = INFINITY;  // the core SVD's sweeps always stop at the strict level
    c0.seed = o.seed;
    c0.oversample = o.p;
    c0.kcap = std::min(kcap0, nh);
    c0.k = std::min(c0.kcap, 8);
    c0.k_next = c0.k;
    CK(cudaStreamSynchronize(st));
    const double nD = std::sqrt(d2);
    if (!(nD > 0) || !std::isfinite(nD)) throw CpcpError{CPCP_ERR_INVALID_ARG, "D is zero or not finite"};
    if (!(mu0 > 0)) {
        // ||D||_2: block of 16, 8 passes (the top value converges like
        // (sigma_17 / sigma_1)^16)
        Ctrl ce = c0;
        ce.k = std::min(kcap0, 16);
        ce.k_next = ce.k;
        CK(cudaMemcpyAsync(ctrl, &ce, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        launch_fill_random<T>(Om, KM, n, ctrl, 1, nullptr, KM, 0x1A10ull, st);
        subspace_svd<T>(h, w, m, n, D, ldd, Om, 8, &ctrl->k, nullptr);
        T s0;
        CK(cudaMemcpyAsync(&s0, w.sig, sizeof(T), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        mu0 = 1.25 / (double)s0;
    }
    c0.k = std::min(c0.kcap, o.p);
    c0.k_next = c0.k;
    CK(cudaMemcpyAsync(ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(S, 0, sizeof(T) * mn, st));
    CK(cudaMemsetAsync(Y, 0, sizeof(T) * mn, st));
    launch_fill_random<T>(Om, KM, nh, ctrl, 1, nullptr, KM, 0x1A11ull, st);

    PassArgs<T> rc;
    memset(&rc, 0, sizeof(rc));
    rc.m = m;
    rc.n = n;
    rc.Ak = A;
    rc.Bk = B;
    rc.ldfa = KM;
    rc.ldfb = KM;
    rc.ldfap = KM;
    rc.ldfbp = KM;
    rc.rk = &ctrl->r_new;
    rc.ctrl = ctrl;
    rc.M = L;
    rc.ldm = ldS;

    cpcp_status status = CPCP_ERR_NOT_CONVERGED;
    double mu = mu0, gap = INFINITY;
    int k = 0;
    for (k = 0; k < max_iter;) {
        launch_ialm_ctrl(ctrl, mu, 0, st);
        launch_ialm_m<T>(m, n, D, ldd, S, Y, ldS, mu, M, ldS, st);
        const T *Mx = M;
        int64_t ldx = ldS;
        if (H > 0) {
            launch_restrict<T>(m, n, M, ldS, MH, ldh, tr, st);
            if (orth) launch_bidiag_right_solve<T>(m, nh, MH, ldh, Cd, Ce, st);  // M R C^{-1}
            Mx = MH;
            ldx = ldh;
        }
        // the SVT must be complete: an SVT truncated at the subspace width
        // leaves D - L - S large, which the multiplier step then amplifies by
        // the growing mu_k.  While every value of the width is above the
        // threshold, widen (new random columns) and redo (the r = k rule).
        for (;;) {
            subspace_svd<T>(h, w, m, nh, Mx, ldx, Om, std::max(o.q, 2), &ctrl->k, ctrl, false, w.Us, ctrl);
            Ctrl cw;
            CK(cudaMemcpyAsync(&cw, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (cw.r_new < cw.k || cw.k >= cw.kcap) break;
            Ctrl wide = cw;
            wide.k_next = std::min(cw.kcap, 2 * cw.k);
            CK(cudaMemcpyAsync(ctrl, &wide, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
            prod_nn_small<T>(nh, w.Qz, KM, w.Wt, KM, Om, KM, &ctrl->k, KM, st);  // the subspace found so far
            launch_fill_random<T>(Om, KM, nh, ctrl, 0, nullptr, KM, 0x1A13ull + (uint64_t)cw.k, st);
            wide.k = wide.k_next;
            CK(cudaMemcpyAsync(ctrl, &wide, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        }
        prod_nn_small<T>(m, w.Qy, KM, w.Us, KM, A, KM, &ctrl->k, KM, st);
        prod_nn_small<T>(nh, w.Qz, KM, w.Wt, KM, Om, KM, &ctrl->k, KM, st);
        if (orth) {
            // B = R C^{-1} V; the next start block keeps V (random columns
            // into Vp are unused)
            launch_bidiag_left_solve<T>(nh, Om, KM, &ctrl->k, KM, Cd, Ce, Vp, KM, st);
            launch_fill_prolong<T>(Vp, KM, nh, ctrl, w.sig, KM, 0x1A12ull, n, B, KM, tr, st);
            launch_fill_random<T>(Om, KM, nh, ctrl, 0, w.sig, KM, 0x1A14ull, st);
        } else {
            launch_fill_prolong<T>(Om, KM, nh, ctrl, w.sig, KM, 0x1A12ull, n, B, KM, tr, st);
        }
        launch_reconstruct<T>(rc, st);
        launch_ialm_update<T>(m, n, D, ldd, L, ldS, S, Y, ldS, lam, mu, partial, st);
        launch_sum_partials(partial, nblk, 1, sums, st);
        launch_ialm_ctrl(ctrl, mu, 1, st);
        double e2 = 0.0;
        CK(cudaMemcpyAsync(&e2, sums, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        gap = std::sqrt(e2) / nD;
        if (fg) fg[k] = gap;
        mu = rho > 1.0 ? mu * rho : mu0 * (double)(k + 2);
        k++;
        if (!std::isfinite(gap)) {
            status = CPCP_ERR_NUMERIC;
            break;
        }
        if (gap <= tol) {
            status = CPCP_OK;
            break;
        }
    }
    Ctrl fin;
    CK(cudaMemcpyAsync(&fin, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    if (S_out)
        CK(cudaMemcpy2DAsync(S_out, sizeof(T) * lds, S, sizeof(T) * ldS, sizeof(T) * n, m, cudaMemcpyDeviceToDevice,
                             st));
    if (L_out)
        CK(cudaMemcpy2DAsync(L_out, sizeof(T) * ldl, L, sizeof(T) * ldS, sizeof(T) * n, m, cudaMemcpyDeviceToDevice,
                             st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    tc_err_check(w.err, st);
    if (info) {
        cpcp_info inf;
        memset(&inf, 0, sizeof(inf));
        inf.status = status;
        inf.iters = k;
        inf.level_iters[std::min(H, 7)] = k;
        inf.final_level = H;
        inf.rank = fin.rk;
        inf.relkkt = gap;
        inf.mu0 = mu0;
        inf.pqd_fro = nD;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        inf.launches = (long long)(g_kernel_launches - launches0);
        *info = inf;
    }
    return status;
}

// FW-T (Alg. 3) / ML-FWT (Alg. 6) for eq. (cpcp) on device buffers; see
// cpcp_fwt.  The m x n passes and the scalars (t_L, t_S, U_L, U_S, the LMOs'
// vertices, the line search, the stop test) in k_fwt.cu, in device memory
// (FwScal); the top singular pair of G (or of G R) from the warm-started
// subspace SVD of the CPCP path.  An iteration is a fixed sequence of launches
// with no host round trip: it is captured once as a CUDA graph and replayed,
// and the host reads the stop state every check_every iterations (kernels of
// iterations after the stop return at once).
template <typename T>
cpcp_status fwt_core(cpcp_context *h, int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq,
                     double lam, double mu, int levels, int max_iter, double tol, T *L_out, int64_t ldl, T *S_out,
                     int64_t lds, double *ftrace, cpcp_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    const unsigned long long launches0 = g_kernel_launches;
    const Opts o = resolve(h->opt);
    // graph replay runs on the handle's private stream (the caller's may be the
    // legacy default stream, which cannot be captured)
    PrivateStream ps(h, o.graphs);
    cudaStream_t st = h->stream;
    const int H = levels - 1;
    const int64_t ld = round4(n);
    TransferDev<T> tr = upload_transfer<T>(h, n, H, "fwt");
    const int nh = tr.nh;
    const int64_t ldh = round4(nh);
    const int kcap0 = std::min({o.k_max, kmax_small<T>(), nh, m});
    const int KM = (int)round4(kcap0);
    const size_t mn = (size_t)m * ld;
    T *L = wsT<T>(h, "fw_L", mn), *S = wsT<T>(h, "fw_S", mn), *G = wsT<T>(h, "fw_G", mn);
    T *GR = H > 0 ? wsT<T>(h, "fw_GR", (size_t)m * ldh) : nullptr;
    T *Om = wsT<T>(h, "fw_Om", (size_t)nh * KM), *Ub = wsT<T>(h, "fw_U", (size_t)m * KM);
    T *Vb = wsT<T>(h, "fw_V", (size_t)nh * KM), *Vf = H > 0 ? wsT<T>(h, "fw_Vf", (size_t)n * KM) : nullptr;
    Ctrl *ctrl = wsT<Ctrl>(h, "fw_ctrl", 1);
    const int nb = fwt_blocks();
    double *partial = wsT<double>(h, "fw_partial", (size_t)nb * 5), *amv = wsT<double>(h, "fw_amv", nb);
    int64_t *ami = wsT<int64_t>(h, "fw_ami", nb);
    SvdWork<T> w = svd_work<T>(h, "fw_svd_", m, n, kcap0);
    tc_err_clear(w.err, h->stream);
    // orthonormal-basis transfer (option): the coarse LMO on G R C^{-1}, lifted by R C^{-1}
    const bool orth = H > 0 && o.transfer == 1;
    OrthTransfer<T> ot;
    T *Vp = nullptr;
    if (orth) {
        ot = upload_orth<T>(h, n, H, "fw");
        Vp = wsT<T>(h, "fw_Vp", (size_t)nh * KM);
    }
    FwScal *sc = wsT<FwScal>(h, "fw_scal", 1);
    double *trace = wsT<double>(h, "fw_trace", (size_t)max_iter);
    const double lamL = mu, lamS = lam * mu;
    {
        FwScal s0;
        memset(&s0, 0, sizeof(s0));
        s0.lamL = lamL;
        s0.lamS = lamS;
        s0.tol = tol;
        s0.margin = sizeof(T) == 4 ? 1e-5 : 1e-12;
        CK(cudaMemcpyAsync(sc, &s0, sizeof(FwScal), cudaMemcpyHostToDevice, st));
    }

    Ctrl c0;
    memset(&c0, 0, sizeof(c0));
    c0.kcap = kcap0;
    c0.k = std::min(kcap0, std::max(2, o.p));  // block width p (oversample): the LMO needs the top pair only
    c0.k_next = c0.k;
    c0.seed = o.seed;
    c0.oversample = o.p;
    CK(cudaMemcpyAsync(ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(L, 0, sizeof(T) * mn, st));
    CK(cudaMemsetAsync(S, 0, sizeof(T) * mn, st));
    launch_fill_random<T>(Om, KM, nh, ctrl, 1, nullptr, KM, 0xF3A1ull, st);
    launch_fwt_grad<T>(m, n, D, ldd, Q, ldq, L, S, ld, G, partial, amv, ami, st);
    launch_fwt_first(sc, partial, amv, ami, st);
    // one iteration: the LMO of the nuclear ball (top singular pair of G, or of
    // G R lifted by R) and of the l1 ball (from the device argmax), the line
    // search, the update with the thresholding step, the scalars
    auto iteration = [&]() {
        const T *Mx = G;
        int64_t ldx = ld;
        if (H > 0) {
            launch_restrict<T>(m, n, G, ld, GR, ldh, tr, st);
            if (orth) launch_bidiag_right_solve<T>(m, nh, GR, ldh, ot.cd, ot.ce, st);
            Mx = GR;
            ldx = ldh;
        }
        subspace_svd<T>(h, w, m, nh, Mx, ldx, Om, o.q, &ctrl->k, nullptr);
        prod_nn_small<T>(m, w.Qy, KM, w.Ut, KM, Ub, KM, &ctrl->k, KM, st);
        prod_nn_small<T>(nh, w.Qz, KM, w.Wt, KM, Vb, KM, &ctrl->k, KM, st);
        CK(cudaMemcpyAsync(Om, Vb, sizeof(T) * (size_t)nh * KM, cudaMemcpyDeviceToDevice, st));  // warm start
        const T *vv = Vb;
        if (H > 0) {
            const T *vsrc = Vb;
            if (orth) {
                launch_bidiag_left_solve<T>(nh, Vb, KM, &ctrl->k, KM, ot.cd, ot.ce, Vp, KM, st);
                vsrc = Vp;
            }
            launch_prolong<T>(n, vsrc, KM, Vf, KM, tr, &ctrl->k, KM, st);
            vv = Vf;
        }
        launch_fwt_lmo<T>(sc, w.sig, G, ld, m, n, st);
        launch_fwt_coef<T>(m, n, Q, ldq, L, S, G, ld, Ub, KM, vv, KM, sc, partial, st);
        launch_fwt_ls(sc, partial, st);
        launch_fwt_update<T>(m, n, D, ldd, Q, ldq, L, S, G, ld, Ub, KM, vv, KM, sc, partial, amv, ami, st);
        launch_fwt_post(sc, partial, amv, ami, trace, st);
    };
    // the first iteration launched directly (every workspace buffer then exists),
    // the rest replayed from a graph of one iteration
    cudaGraphExec_t gexec = nullptr;
    unsigned long long glaunches = 0;
    struct GraphGuard {
        cudaGraphExec_t &e;
        ~GraphGuard()
        {
            if (e) cudaGraphExecDestroy(e);
        }
    } gguard{gexec};
    const bool graphs = o.graphs;
    FwScal fin;
    int launched = 0;
    const int batch = std::max(1, o.check_every);
    for (;;) {
        const int todo = std::min(batch, max_iter - launched);
        for (int b = 0; b < todo; b++, launched++) {
            if (launched == 0 || !graphs) {
                iteration();
                continue;
            }
            if (gexec == nullptr) {
                const unsigned long long l0 = g_kernel_launches;
                CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                cudaGraph_t graph = nullptr;
                try {
                    iteration();
                } catch (...) {
                    cudaStreamEndCapture(st, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    throw;
                }
                CK(cudaStreamEndCapture(st, &graph));
                const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
                cudaGraphDestroy(graph);
                CK(ie);
                glaunches = g_kernel_launches - l0;
                g_kernel_launches = l0;
            }
            CK(cudaGraphLaunch(gexec, st));
            g_kernel_launches += glaunches;
        }
        CK(cudaMemcpyAsync(&fin, sc, sizeof(FwScal), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (fin.done != 0 || launched >= max_iter) break;
    }
    const int k = fin.iters;
    const cpcp_status status = fin.done == 1 ? CPCP_OK : (fin.done == 2 ? CPCP_ERR_NUMERIC : CPCP_ERR_NOT_CONVERGED);
    const double rel = fin.rel, f = fin.f;
    if (ftrace && k > 0) CK(cudaMemcpyAsync(ftrace, trace, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    if (L_out)
        CK(cudaMemcpy2DAsync(L_out, sizeof(T) * ldl, L, sizeof(T) * ld, sizeof(T) * n, m, cudaMemcpyDeviceToDevice,
                             st));
    if (S_out)
        CK(cudaMemcpy2DAsync(S_out, sizeof(T) * lds, S, sizeof(T) * ld, sizeof(T) * n, m, cudaMemcpyDeviceToDevice,
                             st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    tc_err_check(w.err, st);
    if (info) {
        cpcp_info inf;
        memset(&inf, 0, sizeof(inf));
        inf.status = status;
        inf.iters = k;
        inf.level_iters[std::min(H, 7)] = k;
        inf.final_level = H;
        inf.relkkt = rel;
        inf.mu0 = f;  // the epigraph objective at the last iterate
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        inf.launches = (long long)(g_kernel_launches - launches0);
        *info = inf;
    }
    return status;
}

template <typename T>
cpcp_status ialm_dispatch(cpcp_context *h, int m, int n, const void *Dv, int64_t ldd, double lam, int levels,
                          double mu0, double rho, int max_iter, double tol, void *Lv, int64_t ldl, void *Sv,
                          int64_t lds, double *fg, cpcp_info *info)
{
    cudaStream_t st = h->stream;
    const T *D = static_cast<const T *>(Dv);
    T *L = static_cast<T *>(Lv), *S = static_cast<T *>(Sv);
    if (!is_device_ptr(Dv)) {
        T *Dd = wsT<T>(h, "stage_D", (size_t)m * n);
        CK(cudaMemcpy2DAsync(Dd, sizeof(T) * n, D, sizeof(T) * ldd, sizeof(T) * n, m, cudaMemcpyHostToDevice, st));
        T *Ld = L ? wsT<T>(h, "stage_L", (size_t)m * n) : nullptr;
        T *Sd = S ? wsT<T>(h, "stage_S", (size_t)m * n) : nullptr;
        cpcp_status r = ialm_core<T>(h, m, n, Dd, n, lam, levels, mu0, rho, max_iter, tol, Ld, n, Sd, n, fg, info);
        if (L)
            CK(cudaMemcpy2DAsync(L, sizeof(T) * ldl, Ld, sizeof(T) * n, sizeof(T) * n, m, cudaMemcpyDeviceToHost,
                                 st));
        if (S)
            CK(cudaMemcpy2DAsync(S, sizeof(T) * lds, Sd, sizeof(T) * n, sizeof(T) * n, m, cudaMemcpyDeviceToHost,
                                 st));
        CK(cudaStreamSynchronize(st));
        return r;
    }
    return ialm_core<T>(h, m, n, D, ldd, lam, levels, mu0, rho, max_iter, tol, L, ldl, S, lds, fg, info);
}

template <typename T>
cpcp_status solve_dispatch(cpcp_context *h, int m, int n, const void *Dv, int64_t ldd, const uint32_t *Q,
                           int64_t ldq, double lam, double mu, int levels, double tol, void *Lv, int64_t ldl,
                           void *Sv, int64_t lds, cpcp_info *info)
{
    cudaStream_t st = h->stream;
    const T *D = static_cast<const T *>(Dv);
    T *L = static_cast<T *>(Lv), *S = static_cast<T *>(Sv);
    bool host = !is_device_ptr(Dv);
    if (host) {
        // stage host buffers through device memory
        T *Dd = wsT<T>(h, "stage_D", (size_t)m * n);
        CK(cudaMemcpy2DAsync(Dd, sizeof(T) * n, D, sizeof(T) * ldd, sizeof(T) * n, m, cudaMemcpyHostToDevice, st));
        const uint32_t *Qd = nullptr;
        if (Q) {
            uint32_t *q = wsT<uint32_t>(h, "stage_Q", (size_t)m * ldq);
            CK(cudaMemcpyAsync(q, Q, sizeof(uint32_t) * m * ldq, cudaMemcpyHostToDevice, st));
            Qd = q;
        }
        T *Ld = L ? wsT<T>(h, "stage_L", (size_t)m * n) : nullptr;
        T *Sd = S ? wsT<T>(h, "stage_S", (size_t)m * n) : nullptr;
        cpcp_status r = solve_dispatch<T>(h, m, n, Dd, n, Qd, ldq, lam, mu, levels, tol, Ld, n, Sd, n, info);
        if (L)
            CK(cudaMemcpy2DAsync(L, sizeof(T) * ldl, Ld, sizeof(T) * n, sizeof(T) * n, m, cudaMemcpyDeviceToHost,
                                 st));
        if (S)
            CK(cudaMemcpy2DAsync(S, sizeof(T) * lds, Sd, sizeof(T) * n, sizeof(T) * n, m, cudaMemcpyDeviceToHost,
                                 st));
        CK(cudaStreamSynchronize(st));
        return r;
    }
    if (n > m) {
        // solve the transposed problem (PCP/CPCP are transpose invariant)
        T *Dt = wsT<T>(h, "tr_D", (size_t)n * m);
        launch_transpose<T>(m, n, D, ldd, Dt, m, st);
        uint32_t *Qt = nullptr;
        int64_t ldqt = (m + 31) / 32;
        if (Q) {
            Qt = wsT<uint32_t>(h, "tr_Q", (size_t)n * ldqt);
            launch_transpose_mask(m, n, Q, ldq, Qt, ldqt, st);
        }
        T *Lt = L ? wsT<T>(h, "tr_L", (size_t)n * m) : nullptr;
        T *St = S ? wsT<T>(h, "tr_S", (size_t)n * m) : nullptr;
        cpcp_status r = solve_core<T>(h, n, m, Dt, m, Qt, ldqt, lam, mu, levels, tol, Lt, m, St, m, info);
        if (L) launch_transpose<T>(n, m, Lt, m, L, ldl, st);
        if (S) launch_transpose<T>(n, m, St, m, S, lds, st);
        CK(cudaStreamSynchronize(st));
        return r;
    }
    return solve_core<T>(h, m, n, D, ldd, Q, ldq, lam, mu, levels, tol, L, ldl, S, lds, info);
}

// ---------------------------------------------------------------------------
// single step / standalone operators
// ---------------------------------------------------------------------------

template <typename T>
cpcp_status step_impl(cpcp_context *h, int m, int n, const void *Dv, int64_t ldd, const uint32_t *Q, int64_t ldq,
                      double lam, double mu_k, double beta, int halvings, const void *Skv, const void *Spv,
                      int64_t lds_in, const void *Akv, int64_t lda, const void *Bkv, int64_t ldb, int r_k,
                      const void *Apv, int64_t ldap, const void *Bpv, int64_t ldbp, int r_p, int k, int q,
                      const void *Om0, int64_t ldo,
                      void *Soutv, int64_t lds, void *Aov, int64_t ldao, void *Bov, int64_t ldbo, int *r_out,
                      double *sigma_out)
{
    cudaStream_t st = h->stream;
    TransferDev<T> tr = upload_transfer<T>(h, n, halvings, "step");
    const int nh = tr.nh;
    if (k < 1 || k > nh || k > kmax_small<T>())
        throw CpcpError{CPCP_ERR_INVALID_ARG, "k must satisfy 1 <= k <= min(n_H, " +
                                                  std::to_string(kmax_small<T>()) + ")"};
    SvdWork<T> w = svd_work<T>(h, "st_", m, n, k);
    tc_err_clear(w.err, h->stream);
    const int KM = w.KM;
    Ctrl c;
    memset(&c, 0, sizeof(c));
    c.tau = 0.5;
    c.lam = lam;
    c.mu_bar = mu_k;
    c.mu_k = mu_k;
    c.beta = beta;
    c.theta_L = 0.5 * mu_k;
    c.theta_S = 0.5 * lam * mu_k;
    c.rk = r_k;
    c.rp = r_p;
    c.k = k;
    c.k_next = k;
    c.kcap = k;
    c.seed = h->opt.seed ? h->opt.seed : 1;
    Ctrl *cd = wsT<Ctrl>(h, "st_ctrl", 1);
    CK(cudaMemcpyAsync(cd, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    PassArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.m = m;
    a.n = n;
    a.D = static_cast<const T *>(Dv);
    a.ldd = ldd;
    a.Q = Q;
    a.ldq = ldq;
    a.Sk = static_cast<const T *>(Skv);
    a.Sp = static_cast<const T *>(Spv);
    a.lds = lds_in;
    a.Sout = static_cast<T *>(Soutv);
    a.ldso = lds;
    a.Ak = static_cast<const T *>(Akv);
    a.Bk = static_cast<const T *>(Bkv);
    a.Ap = static_cast<const T *>(Apv);
    a.Bp = static_cast<const T *>(Bpv);
    a.ldfa = lda;
    a.ldfb = ldb;
    a.ldfap = ldap;
    a.ldfbp = ldbp;
    a.rk = &cd->rk;
    a.rp = &cd->rp;
    a.ctrl = cd;
    const T *Mx;
    int64_t ldx;
    int *tc_err = nullptr;
    if (halvings > 0) {
        int64_t ldh = round4(nh);
        T *MH = wsT<T>(h, "st_MH", (size_t)m * ldh);
        CK(cudaMemsetAsync(MH, 0, sizeof(T) * (size_t)m * ldh, st));
        a.MH = MH;
        a.ldh = ldh;
        a.tr = tr;
        launch_step_pass<T>(a, true, st);
        Mx = MH;
        ldx = ldh;
    } else {
        int64_t ldm = round4(n);
        T *M = wsT<T>(h, "st_M", (size_t)m * ldm);
        a.M = M;
        a.ldm = ldm;
        // fp32: the tensor-core fine pass where the operands meet its TMA rules
        // (as in cpcp_solve), else the SIMT pass
        bool tc = false;
        if constexpr (std::is_same<T, float>::value) {
            if (!h->opt.pass_simt) {
                tc_err = wsT<int>(h, "st_tc_err", 1);
                CK(cudaMemsetAsync(tc_err, 0, sizeof(int), st));
                tc = launch_pass_tc(a, tc_err, st);
            }
        }
        if (!tc) launch_step_pass<T>(a, false, st);
        Mx = M;
        ldx = ldm;
    }
    T *Om = wsT<T>(h, "st_Om", (size_t)nh * KM);
    if (Om0) {
        CK(cudaMemcpy2DAsync(Om, sizeof(T) * KM, Om0, sizeof(T) * ldo, sizeof(T) * k, nh, cudaMemcpyDefault, st));
    } else {
        launch_fill_random<T>(Om, KM, nh, cd, 1, nullptr, KM, 0x51ull, st);
    }
    subspace_svd<T>(h, w, m, nh, Mx, ldx, Om, q, &cd->k, nullptr);
    launch_svt_small<T>(w.Ut, w.sig, KM, cd, w.Us, w.sig64, st);
    launch_gemm_nn<T>(m, 0, w.Qy, KM, w.Us, KM, static_cast<T *>(Aov), ldao, &cd->k, &cd->k, KM, st);
    T *V = wsT<T>(h, "st_V", (size_t)nh * KM);
    launch_gemm_nn<T>(nh, 0, w.Qz, KM, w.Wt, KM, V, KM, &cd->k, &cd->k, KM, st);
    launch_prolong<T>(n, V, KM, static_cast<T *>(Bov), ldbo, tr, &cd->r_new, k, st);
    Ctrl out;
    CK(cudaMemcpyAsync(&out, cd, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    if (sigma_out) CK(cudaMemcpyAsync(sigma_out, w.sig64, sizeof(double) * k, cudaMemcpyDefault, st));
    int tc_flag = 0;
    if (tc_err) CK(cudaMemcpyAsync(&tc_flag, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (tc_flag) throw CpcpError{CPCP_ERR_TIMEOUT, "a bounded wait of the tensor-core pass expired"};
    tc_err_check(w.err, st);
    if (r_out) *r_out = out.r_new;
    return CPCP_OK;
}

template <typename T>
cpcp_status svd_impl(cpcp_context *h, int m, int n, const void *Mv, int64_t ldm, int k, int q, const void *Om0,
                     int64_t ldo, void *Uv, int64_t ldu, void *Vv, int64_t ldv, double *sigma)
{
    cudaStream_t st = h->stream;
    if (k < 1 || k > n || k > kmax_small<T>())
        throw CpcpError{CPCP_ERR_INVALID_ARG, "k must satisfy 1 <= k <= min(n, " +
                                                  std::to_string(kmax_small<T>()) + ")"};
    SvdWork<T> w = svd_work<T>(h, "sv_", m, n, k);
    tc_err_clear(w.err, h->stream);
    const int KM = w.KM;
    const bool bf16 = std::is_same<T, float>::value && h->opt.precision == 1;
    if (bf16) {
        svd_work_bf16<T>(h, w, "sv_", m, n);
        CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    }
    Ctrl c;
    memset(&c, 0, sizeof(c));
    c.k = k;
    c.k_next = k;
    c.kcap = k;
    c.seed = h->opt.seed ? h->opt.seed : 1;
    Ctrl *cd = wsT<Ctrl>(h, "sv_ctrl", 1);
    CK(cudaMemcpyAsync(cd, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    T *Om = wsT<T>(h, "sv_Om", (size_t)n * KM);
    if (Om0)
        CK(cudaMemcpy2DAsync(Om, sizeof(T) * KM, Om0, sizeof(T) * ldo, sizeof(T) * k, n, cudaMemcpyDefault, st));
    else
        launch_fill_random<T>(Om, KM, n, cd, 1, nullptr, KM, 0x5Dull, st);
    subspace_svd<T>(h, w, m, n, static_cast<const T *>(Mv), ldm, Om, q, &cd->k, nullptr, bf16);
    launch_gemm_nn<T>(m, 0, w.Qy, KM, w.Ut, KM, static_cast<T *>(Uv), ldu, &cd->k, &cd->k, KM, st);
    launch_gemm_nn<T>(n, 0, w.Qz, KM, w.Wt, KM, static_cast<T *>(Vv), ldv, &cd->k, &cd->k, KM, st);
    // singular values as doubles
    std::vector<T> sh(k);
    CK(cudaMemcpyAsync(sh.data(), w.sig, sizeof(T) * k, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    std::vector<double> sd(sh.begin(), sh.end());
    CK(cudaMemcpy(sigma, sd.data(), sizeof(double) * k, cudaMemcpyDefault));
    tc_err_check(w.err, st);
    return CPCP_OK;
}

cpcp_status gemm_bf16_impl(cpcp_context *h, int rows, int K, int N, const float *A, int64_t lda, const float *B,
                           int64_t ldb, float *C, int64_t ldc)
{
    cudaStream_t st = h->stream;
    const int rp = umma_pad_rows(rows), kp = umma_pad_k(K), NB = round16(N), ldp = (int)round4(N);
    __nv_bfloat16 *Ab = wsT<__nv_bfloat16>(h, "gb_A", (size_t)rp * kp);
    __nv_bfloat16 *Bb = wsT<__nv_bfloat16>(h, "gb_B", (size_t)NB * kp);
    float *part = wsT<float>(h, "gb_part", (size_t)64 * rows * ldp);
    int *kd = wsT<int>(h, "gb_k", 1);
    int *err = wsT<int>(h, "umma_err", 1);
    CK(cudaMemcpyAsync(kd, &N, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    launch_bf16_pair(rows, K, A, lda, Ab, rp, kp, nullptr, 0, 0, st);
    launch_bf16_pair(N, K, B, ldb, Bb, NB, kp, nullptr, 0, 0, st);
    int sp = launch_umma_tn(rows, rp, kp, Ab, kp, Bb, NB, kp, NB, kd, part, ldp, 64, err, st);
    if (sp < 0) throw CpcpError{CPCP_ERR_CUDA, "could not encode the TMA tensor maps"};
    launch_reduce_partial<float>(part, sp, rows, ldp, C, ldc, nullptr, kd, st);
    int e = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (e) throw CpcpError{CPCP_ERR_TIMEOUT, "a bounded wait of the tensor-core kernel expired"};
    return CPCP_OK;
}

// ---------------------------------------------------------------------------
// batched solve (host side): validation, arena layout, transfer tables,
// descriptors, the captured graph and the CTA-size autotuner
// ---------------------------------------------------------------------------

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

struct BatchLayout {
    std::vector<BatchInst> inst;
    std::vector<int> order;
    size_t arena_floats = 0;
};

cpcp_status batched_impl(cpcp_context *h, int count, const cpcp_problem *P, double tol, cpcp_info *infos)
{
    auto t0 = std::chrono::steady_clock::now();
    const unsigned long long launches0 = g_kernel_launches;
    const Opts o = resolve(h->opt);
    const int KB = BATCH_KB;
    if (count < 1 || !P) throw CpcpError{CPCP_ERR_INVALID_ARG, "count must be >= 1 and probs non-NULL"};
    if (!(tol > 0)) throw CpcpError{CPCP_ERR_INVALID_ARG, "tol must be positive"};

    // validation and oriented sizes
    std::vector<BatchInst> inst(count);
    std::map<std::pair<int, int>, HostTransfer> tables;
    for (int i = 0; i < count; i++) {
        const cpcp_problem &q = P[i];
        const std::string who = "instance " + std::to_string(i) + ": ";
        if (q.m < 1 || q.n < 1 || !q.D || q.ldd < q.n || (q.L && q.ldl < q.n) || (q.S && q.lds < q.n))
            throw CpcpError{CPCP_ERR_INVALID_ARG, who + "bad sizes, D or leading dimension"};
        if (q.Q && q.ldq < (q.n + 31) / 32) throw CpcpError{CPCP_ERR_INVALID_ARG, who + "ldq < ceil(n/32)"};
        if (!(q.lambda > 0) || !(q.mu > 0)) throw CpcpError{CPCP_ERR_INVALID_ARG, who + "lambda and mu must be positive"};
        if (q.levels < 1 || q.levels > BATCH_LEVELS)
            throw CpcpError{CPCP_ERR_INVALID_ARG, who + "levels must be in [1, 4] for the batched solve"};
        BatchInst &b = inst[i];
        memset(&b, 0, sizeof(b));
        b.trans = q.n > q.m ? 1 : 0;
        b.m = std::max(q.m, q.n);
        b.n = std::min(q.m, q.n);
        if (b.n > BATCH_NMAX) throw CpcpError{CPCP_ERR_INVALID_ARG, who + "min(m, n) exceeds 1024"};
        b.levels = q.levels;
        for (int lv = 0; lv < BATCH_LEVELS; lv++) b.nh[lv] = coarse_dim(b.n, std::min(lv, q.levels - 1));
        if (q.levels > 1 && 2 * b.nh[q.levels - 1] > b.m + 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, who + "coarse width exceeds (m+1)/2 (Assumption 2)"};
        for (int lv = 1; lv < q.levels; lv++) {
            auto key = std::make_pair(b.n, lv);
            if (!tables.count(key)) tables[key] = build_transfer(b.n, lv);
            b.kappa[lv] = tables[key].kappa;
        }
        b.D = q.D;
        b.ldd = q.ldd;
        b.Q = q.Q;
        b.ldq = q.ldq;
        b.Lout = q.L;
        b.ldl = q.ldl;
        b.Sout = q.S;
        b.lds = q.lds;
        b.lam = q.lambda;
        b.mu = q.mu;
    }
    // transfer tables in one device buffer: per (n, h) j0, clo, chi (int) and w0, w1 (float)
    size_t tab_words = 0;
    std::map<std::pair<int, int>, size_t> tab_off;
    for (auto &kv : tables) {
        tab_off[kv.first] = tab_words;
        const HostTransfer &t = kv.second;
        tab_words += (size_t)3 * t.n + 2 * (size_t)t.nh;
        tab_words = (tab_words + 63) / 64 * 64;
    }
    std::vector<uint32_t> tab_host(std::max<size_t>(tab_words, 64), 0u);
    for (auto &kv : tables) {
        const HostTransfer &t = kv.second;
        uint32_t *w = tab_host.data() + tab_off[kv.first];
        for (int j = 0; j < t.n; j++) {
            w[j] = (uint32_t)t.j0[j];
            float f0 = (float)t.w0[j], f1 = (float)t.w1[j];
            memcpy(&w[t.n + j], &f0, 4);
            memcpy(&w[2 * t.n + j], &f1, 4);
        }
        for (int c = 0; c < t.nh; c++) {
            w[3 * t.n + c] = (uint32_t)t.clo[c];
            w[3 * t.n + t.nh + c] = (uint32_t)t.chi[c];
        }
    }
    uint32_t *tab_dev = wsT<uint32_t>(h, "bt_tables", tab_host.size());

    // arena layout (floats, every array 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t floats) {
        size_t o0 = off;
        off += (floats + 63) / 64 * 64;
        return o0;
    };
    struct Offs {
        size_t Dw, Qw, S0, S1, L0, L1, M, MH, A, B, Ac, Bc, Om, Omf, Y, Qy, Q1, Z, Qz, R[8], sig;
    };
    std::vector<Offs> offs(count);
    for (int i = 0; i < count; i++) {
        BatchInst &b = inst[i];
        Offs &f = offs[i];
        b.ld = round4(b.n);
        b.ldh = b.levels > 1 ? round4(b.nh[1]) : 4;
        b.ldqw = (b.n + 31) / 32;
        const size_t mn = (size_t)b.m * b.ld;
        f.Dw = b.trans ? take(mn) : 0;
        f.Qw = (b.trans && b.Q) ? take((size_t)b.m * b.ldqw) : 0;
        f.S0 = take(mn);
        f.S1 = take(mn);
        f.L0 = take(mn);
        f.L1 = take(mn);
        f.M = take(mn);
        f.MH = b.levels > 1 ? take((size_t)b.m * b.ldh) : 0;
        f.A = take((size_t)b.m * KB);
        f.Ac = take((size_t)b.m * KB);
        f.Y = take((size_t)b.m * KB);
        f.Qy = take((size_t)b.m * KB);
        f.Q1 = take((size_t)b.m * KB);
        f.B = take((size_t)b.n * KB);
        f.Bc = take((size_t)b.n * KB);
        f.Om = take((size_t)b.n * KB);
        f.Omf = take((size_t)b.n * KB);
        f.Z = take((size_t)b.n * KB);
        f.Qz = take((size_t)b.n * KB);
        for (int r = 0; r < 8; r++) f.R[r] = take((size_t)KB * KB);
        f.sig = take(KB);
    }
    float *arena = wsT<float>(h, "bt_arena", off);
    for (int i = 0; i < count; i++) {
        BatchInst &b = inst[i];
        const Offs &f = offs[i];
        b.Dw = b.trans ? arena + f.Dw : nullptr;
        b.Qw = (b.trans && b.Q) ? reinterpret_cast<uint32_t *>(arena + f.Qw) : nullptr;
        b.S[0] = arena + f.S0;
        b.S[1] = arena + f.S1;
        b.L[0] = arena + f.L0;
        b.L[1] = arena + f.L1;
        b.M = arena + f.M;
        b.MH = b.levels > 1 ? arena + f.MH : nullptr;
        b.A = arena + f.A;
        b.Ac = arena + f.Ac;
        b.Y = arena + f.Y;
        b.Qy = arena + f.Qy;
        b.Q1 = arena + f.Q1;
        b.B = arena + f.B;
        b.Bc = arena + f.Bc;
        b.Om = arena + f.Om;
        b.Omf = arena + f.Omf;
        b.Z = arena + f.Z;
        b.Qz = arena + f.Qz;
        float **R[8] = {&b.R1, &b.R1i, &b.R2, &b.R2i, &b.Rz, &b.Ut, &b.Wt, &b.Us};
        for (int r = 0; r < 8; r++) *R[r] = arena + f.R[r];
        b.sig = arena + f.sig;
        for (int lv = 1; lv < b.levels; lv++) {
            const HostTransfer &t = tables[std::make_pair(b.n, lv)];
            uint32_t *w = tab_dev + tab_off[std::make_pair(b.n, lv)];
            b.j0[lv] = reinterpret_cast<const int *>(w);
            b.w0[lv] = reinterpret_cast<const float *>(w + t.n);
            b.w1[lv] = reinterpret_cast<const float *>(w + 2 * t.n);
            b.clo[lv] = reinterpret_cast<const int *>(w + 3 * t.n);
            b.chi[lv] = reinterpret_cast<const int *>(w + 3 * t.n + t.nh);
        }
    }
    // largest instances first
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)inst[a].m * inst[a].n > (double)inst[b].m * inst[b].n;
    });

    BatchOpts bo;
    memset(&bo, 0, sizeof(bo));  // hashed below, padding included
    bo.max_iter = o.max_iter;
    bo.early = o.early_test ? 1 : 0;
    bo.check_every = o.check_every;
    bo.p = std::min(o.p, BATCH_KB);
    bo.q = o.q;
    bo.qc = o.qc;
    bo.eta = o.eta;
    bo.ratio = o.ratio;
    bo.tol = tol;
    bo.seed = o.seed;

    BatchInst *inst_dev = wsT<BatchInst>(h, "bt_inst", count);
    BatchResult *res_dev = wsT<BatchResult>(h, "bt_res", count);
    int *order_dev = wsT<int>(h, "bt_order", count);
    int *next_dev = wsT<int>(h, "bt_next", 1);

    BatchGraph &g = h->batch;
    if (!g.stream) CK(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    cudaStream_t bs = g.stream;
    // inputs were produced on the caller's stream
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpyAsync(tab_dev, tab_host.data(), sizeof(uint32_t) * tab_host.size(), cudaMemcpyHostToDevice, bs));
    CK(cudaMemcpyAsync(inst_dev, inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, bs));
    CK(cudaMemcpyAsync(order_dev, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, bs));
    CK(cudaStreamSynchronize(bs));

    // Shape signature (sizes, levels, masks present, tolerance, options): the
    // key of the tuned CTA size.  The graph signature adds the handle's own
    // device buffers the captured launch reads; user pointers are not part of
    // either, since the descriptors are uploaded before every launch.
    uint64_t sig = fnv1a(&count, sizeof(count));
    for (int i = 0; i < count; i++) {
        const int key[4] = {P[i].m, P[i].n, P[i].levels, P[i].Q != nullptr};
        sig = fnv1a(key, sizeof(key), sig);
    }
    sig = fnv1a(&tol, sizeof(tol), sig);
    sig = fnv1a(&bo, sizeof(bo), sig);
    uint64_t gsig = fnv1a(&arena, sizeof(arena), sig);
    const void *bufs[4] = {inst_dev, res_dev, order_dev, next_dev};
    gsig = fnv1a(bufs, sizeof(bufs), gsig);

    // launch configuration: CTA size (256 or 512 threads) and the CTA GEMM's
    // output tiles for wide products (64 x 64 or 128 x 64): the user's CTA size,
    // else the tuned pair for this batch signature if one was measured, else
    // (on the first call with batch_autotune) every pair timed and the fastest
    // kept, else 512 threads with 64 x 64 tiles
    int nt = h->opt.batch_threads;
    int tile = 0;
    if (nt != 0 && nt != 256 && nt != 512) throw CpcpError{CPCP_ERR_INVALID_ARG, "batch_threads must be 0, 256 or 512"};
    if (nt == 0) {
        auto it = h->batch_tuned.find(sig);
        if (it != h->batch_tuned.end()) {
            nt = it->second.first;
            tile = it->second.second;
        } else if (h->opt.batch_autotune) {
            float best = 0.f;
            for (int cand : {256, 512}) {
                for (int tl : {0, 1}) {
                    BatchOpts bt = bo;
                    bt.tile = tl;
                    cudaEvent_t e0, e1;
                    CK(cudaEventCreate(&e0));
                    CK(cudaEventCreate(&e1));
                    CK(cudaMemsetAsync(next_dev, 0, sizeof(int), bs));
                    CK(cudaEventRecord(e0, bs));
                    CK(launch_batched(inst_dev, res_dev, order_dev, count, next_dev, bt, cand, bs));
                    CK(cudaEventRecord(e1, bs));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    if (nt == 0 || ms < best) {
                        best = ms;
                        nt = cand;
                        tile = tl;
                    }
                }
            }
            h->batch_tuned[sig] = {nt, tile};
        } else {
            nt = 512;
        }
    }
    bo.tile = tile;

    if (g.host_cap < count) {
        if (g.host_res) cudaFreeHost(g.host_res);
        g.host_res = nullptr;
        g.host_cap = 0;
        CK(cudaMallocHost(&g.host_res, sizeof(BatchResult) * count));
        g.host_cap = count;
        g.sig = 0;  // the captured copy targets the old buffer
    }
    if (!(g.exec && g.sig == gsig && g.nt == nt && g.tile == tile)) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g.exec = nullptr;
        g.graph = nullptr;
        g.sig = 0;
        CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(next_dev, 0, sizeof(int), bs);
        cudaError_t e2 = launch_batched(inst_dev, res_dev, order_dev, count, next_dev, bo, nt, bs);
        cudaError_t e3 = cudaMemcpyAsync(g.host_res, res_dev, sizeof(BatchResult) * count, cudaMemcpyDeviceToHost, bs);
        cudaGraph_t graph = nullptr;
        cudaError_t e4 = cudaStreamEndCapture(bs, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw CpcpError{CPCP_ERR_CUDA, "capture of the batched launch failed"};
        }
        g.graph = graph;
        CK(cudaGraphInstantiate(&g.exec, g.graph, 0));
        g.sig = gsig;
        g.nt = nt;
        g.tile = tile;
    } else {
        CPCP_COUNT_LAUNCH();  // the replayed persistent kernel
    }
    CK(cudaGraphLaunch(g.exec, bs));
    CK(cudaStreamSynchronize(bs));
    CK(cudaGetLastError());

    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const long long launches = (long long)(g_kernel_launches - launches0);
    int khz = 0;
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, h->device));
    bool any_nf = false, any_nc = false, any_bad = false;
    for (int i = 0; i < count; i++) {
        const BatchResult &r = g.host_res[i];
        any_bad |= r.status == CPCP_ERR_INVALID_ARG;
        any_nf |= r.status == CPCP_ERR_NONFINITE_INPUT;
        any_nc |= r.status == CPCP_ERR_NOT_CONVERGED;
        if (infos) {
            cpcp_info &f = infos[i];
            memset(&f, 0, sizeof(f));
            f.status = r.status;
            f.iters = r.iters;
            for (int lv = 0; lv < BATCH_LEVELS; lv++) f.level_iters[lv] = r.level_iters[lv];
            f.final_level = r.final_level;
            f.rank = r.rank;
            f.checks = r.checks;
            f.relkkt = r.relkkt;
            f.mu0 = r.mu0;
            f.pqd_fro = r.pqd;
            f.seconds = secs;
            f.launches = launches;
            f.batch_threads = nt;
            f.batch_tile = tile;
            // per-instance device time by phase, from the SM cycle counter at the nominal clock
            for (int ph = 0; ph < 4; ph++) {
                f.phase_ms[ph] = khz > 0 ? (double)r.cycles[ph] / khz : 0.0;
                f.phase_count[ph] = 0;
                f.svt_detail_ms[ph] = khz > 0 ? (double)r.svt_cycles[ph] / khz : 0.0;
            }
        }
    }
    if (any_bad) return CPCP_ERR_INVALID_ARG;
    if (any_nf) return CPCP_ERR_NONFINITE_INPUT;
    if (any_nc) return CPCP_ERR_NOT_CONVERGED;
    return CPCP_OK;
}

// ---------------------------------------------------------------------------
// unrolled (differentiable) program: recording forward and reverse sweep
// ---------------------------------------------------------------------------

struct UnrollWork {
    float *XL, *MH, *Y, *Bf, *X, *Vc, *gMH;
    double *nrm;
    int *pos, *err;
    void *gs;
};

UnrollWork unroll_work(cpcp_context *h, int m, int64_t ld, int q)
{
    UnrollWork w;
    w.XL = wsT<float>(h, "ur_XL", (size_t)m * ld);
    w.MH = wsT<float>(h, "ur_MH", (size_t)m * q);
    w.Y = wsT<float>(h, "ur_Y", (size_t)m * q);
    w.gMH = wsT<float>(h, "ur_gMH", (size_t)m * q);
    w.Bf = wsT<float>(h, "ur_Bf", (size_t)q * q);
    w.X = wsT<float>(h, "ur_X", (size_t)q * m);
    w.Vc = wsT<float>(h, "ur_Vc", (size_t)q * q);
    w.nrm = wsT<double>(h, "ur_nrm", q);
    w.pos = wsT<int>(h, "ur_pos", q);
    w.err = wsT<int>(h, "ur_err", 1);
    w.gs = ws_get(h, "ur_gs", full_svd_sync_bytes());
    return w;
}

// momentum weights beta_k and continuation weights mu_k (and d mu_k / d mu)
void unroll_schedule(const UnrollRec &r, std::vector<double> &beta, std::vector<double> &mus, std::vector<double> &dmus)
{
    beta.resize(r.K);
    mus.resize(r.K);
    dmus.resize(r.K);
    double t = 1.0;
    for (int k = 0; k < r.K; k++) {
        const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        beta[k] = (t - 1.0) / t1;
        t = t1;
        dmus[k] = std::max(r.rho * std::pow(r.eta, (double)k), 1.0);
        mus[k] = r.mu * dmus[k];
    }
}

// One step: (L_k, L_p, S_k, S_p) -> (Lout, Sout); leaves the exact SVD of the
// step's M_H in (U, sig, V).
void unroll_step(cpcp_context *h, const UnrollRec &r, const TransferDev<float> &tr, UnrollWork &w, double beta,
                 double mu_k, const float *Lk, const float *Lp, const float *Sk, const float *Sp, float *Lout,
                 float *Sout, float *U, double *sig, float *V)
{
    cudaStream_t st = h->stream;
    const int m = r.m, n = r.n, q = r.q;
    const double thL = 0.5 * mu_k;
    const float thS = (float)(0.5 * r.lam * mu_k);
    launch_unroll_step(m, n, r.D, r.ld, r.Q, r.ldq, Lk, Lp, Sk, Sp, r.ld, (float)beta, thS, Sout, w.XL, st);
    const float *M = w.XL;
    int64_t ldm = r.ld;
    if (r.halvings > 0) {
        launch_restrict<float>(m, n, w.XL, r.ld, w.MH, q, tr, st);
        M = w.MH;
        ldm = q;
    }
    if (launch_full_svd(m, q, M, ldm, U, q, V, q, sig, w.X, w.Vc, w.nrm, w.pos, w.gs, w.err, st) < 0)
        throw CpcpError{CPCP_ERR_CUDA, std::string("full SVD launch failed: ") + cudaGetErrorString(cudaGetLastError())};
    launch_svt_right(q, sig, V, q, thL, w.Bf, q, st);
    if (r.halvings > 0) {
        launch_gemm_nn<float>(m, q, U, q, w.Bf, q, w.Y, q, nullptr, nullptr, q, st);
        launch_row_prolong(m, n, q, w.Y, q, tr, Lout, r.ld, st);
    } else {
        launch_gemm_nn<float>(m, q, U, q, w.Bf, q, Lout, r.ld, nullptr, nullptr, q, st);
    }
}

void check_unroll_err(cpcp_context *h, UnrollWork &w)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaGetLastError());
    if (e) throw CpcpError{CPCP_ERR_TIMEOUT, "a bounded grid barrier of the SVD expired"};
}

cpcp_status unroll_forward(cpcp_context *h, int m, int n, const float *D, int64_t ldd, const uint32_t *Q, int64_t ldq,
                           double lam, double mu, int levels, float *L_out, int64_t ldl, float *S_out, int64_t lds,
                           cpcp_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    const unsigned long long launches0 = g_kernel_launches;
    cudaStream_t st = h->stream;
    UnrollRec &r = h->unroll;
    r.valid = false;
    if (n > m) throw CpcpError{CPCP_ERR_INVALID_ARG, "the unrolled program needs n <= m"};
    if (!(h->opt.rho > 0)) throw CpcpError{CPCP_ERR_INVALID_ARG, "the unrolled program needs options.rho > 0"};
    r.m = m;
    r.n = n;
    r.K = h->opt.unroll;
    r.T = h->opt.ckpt_every > 0 ? h->opt.ckpt_every : 10;
    r.halvings = levels - 1;
    r.q = coarse_dim(n, r.halvings);
    r.ld = round4(n);
    r.lam = lam;
    r.mu = mu;
    r.rho = h->opt.rho;
    r.eta = h->opt.eta > 0 ? h->opt.eta : 0.9;
    if (r.q > 1024) throw CpcpError{CPCP_ERR_INVALID_ARG, "the unrolled program needs n_H <= 1024"};
    const size_t mn = (size_t)m * r.ld;
    float *Dc = wsT<float>(h, "ur_D", mn);
    CK(cudaMemcpy2DAsync(Dc, sizeof(float) * r.ld, D, sizeof(float) * ldd, sizeof(float) * n, m, cudaMemcpyDefault, st));
    r.D = Dc;
    r.Q = nullptr;
    r.ldq = (n + 31) / 32;
    if (Q) {
        uint32_t *Qc = wsT<uint32_t>(h, "ur_Q", (size_t)m * r.ldq);
        CK(cudaMemcpy2DAsync(Qc, sizeof(uint32_t) * r.ldq, Q, sizeof(uint32_t) * ldq, sizeof(uint32_t) * r.ldq, m,
                             cudaMemcpyDefault, st));
        r.Q = Qc;
    }
    const int nck = (r.K + r.T - 1) / r.T;
    r.ck = wsT<float>(h, "ur_ck", (size_t)nck * 4 * mn);
    TransferDev<float> tr = upload_transfer<float>(h, n, r.halvings, "ur");
    UnrollWork w = unroll_work(h, m, r.ld, r.q);
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    float *L[2] = {wsT<float>(h, "ur_L0", mn), wsT<float>(h, "ur_L1", mn)};
    float *S[2] = {wsT<float>(h, "ur_S0", mn), wsT<float>(h, "ur_S1", mn)};
    float *U = wsT<float>(h, "ur_U", (size_t)m * r.q), *V = wsT<float>(h, "ur_V", (size_t)r.q * r.q);
    double *sig = wsT<double>(h, "ur_sig", r.q);
    for (int i = 0; i < 2; i++) {
        CK(cudaMemsetAsync(L[i], 0, sizeof(float) * mn, st));
        CK(cudaMemsetAsync(S[i], 0, sizeof(float) * mn, st));
    }
    std::vector<double> beta, mus, dmus;
    unroll_schedule(r, beta, mus, dmus);
    int cur = 0;  // L[cur] = L_k, L[cur ^ 1] = L_{k-1}
    for (int k = 0; k < r.K; k++) {
        if (k % r.T == 0) {
            float *c = r.ck + (size_t)(k / r.T) * 4 * mn;
            CK(cudaMemcpyAsync(c, L[cur], sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c + mn, L[cur ^ 1], sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c + 2 * mn, S[cur], sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c + 3 * mn, S[cur ^ 1], sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        }
        unroll_step(h, r, tr, w, beta[k], mus[k], L[cur], L[cur ^ 1], S[cur], S[cur ^ 1], L[cur ^ 1], S[cur ^ 1], U,
                    sig, V);
        cur ^= 1;
    }
    if (L_out)
        CK(cudaMemcpy2DAsync(L_out, sizeof(float) * ldl, L[cur], sizeof(float) * r.ld, sizeof(float) * n, m,
                             cudaMemcpyDefault, st));
    if (S_out)
        CK(cudaMemcpy2DAsync(S_out, sizeof(float) * lds, S[cur], sizeof(float) * r.ld, sizeof(float) * n, m,
                             cudaMemcpyDefault, st));
    check_unroll_err(h, w);
    r.valid = true;
    if (info) {
        cpcp_info inf;
        memset(&inf, 0, sizeof(inf));
        inf.status = CPCP_OK;
        inf.iters = r.K;
        inf.level_iters[std::min(r.halvings, 7)] = r.K;
        inf.final_level = r.halvings;
        inf.mu0 = mus.empty() ? mu : mus[0];
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        inf.launches = (long long)(g_kernel_launches - launches0);
        *info = inf;
    }
    return CPCP_OK;
}

cpcp_status unroll_backward(cpcp_context *h, const float *dL, int64_t ldgl, const float *dS, int64_t ldgs, float *dD,
                            int64_t ldgd, double *dlambda, double *dmu)
{
    cudaStream_t st = h->stream;
    const UnrollRec &r = h->unroll;
    if (!r.valid) throw CpcpError{CPCP_ERR_INVALID_ARG, "no unrolled run recorded on this handle"};
    const int m = r.m, n = r.n, q = r.q, T = r.T;
    const size_t mn = (size_t)m * r.ld, mq = (size_t)m * q, qq = (size_t)q * q;
    TransferDev<float> tr = upload_transfer<float>(h, n, r.halvings, "ur");
    UnrollWork w = unroll_work(h, m, r.ld, q);
    CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    std::vector<double> beta, mus, dmus;
    unroll_schedule(r, beta, mus, dmus);
    // segment states (T + 2 of each) and the segment's SVDs
    float *Ls = wsT<float>(h, "ub_Ls", (size_t)(T + 2) * mn), *Ss = wsT<float>(h, "ub_Ss", (size_t)(T + 2) * mn);
    float *Us = wsT<float>(h, "ub_U", (size_t)T * mq), *Vs = wsT<float>(h, "ub_V", (size_t)T * qq);
    double *sigs = wsT<double>(h, "ub_sig", (size_t)T * q);
    // adjoint recursion and dD in fp64; gL32 is the fp32 copy of gLn for the contractions
    double *gLn = wsT<double>(h, "ub_gLn", mn), *gSn = wsT<double>(h, "ub_gSn", mn);
    double *gLp = wsT<double>(h, "ub_gLp", mn), *gSp = wsT<double>(h, "ub_gSp", mn);
    double *dD64 = wsT<double>(h, "ub_dD", mn);
    float *gL32 = wsT<float>(h, "ub_gL32", mn), *gXL = wsT<float>(h, "ub_gXL", mn);
    float *gY = wsT<float>(h, "ub_gY", mq), *P = wsT<float>(h, "ub_P", mq), *Tm = wsT<float>(h, "ub_T", mq);
    float *W = wsT<float>(h, "ub_W", mq), *Z = wsT<float>(h, "ub_Z", mq);
    float *A = wsT<float>(h, "ub_A", qq), *B = wsT<float>(h, "ub_B", qq), *Vt = wsT<float>(h, "ub_Vt", qq);
    float *part = wsT<float>(h, "ub_part", (size_t)64 * qq);
    double *gthL = wsT<double>(h, "ub_gthL", 256), *gthS = wsT<double>(h, "ub_gthS", 2048);
    double *scal = wsT<double>(h, "ub_scal", 2);
    CK(cudaMemcpy2DAsync(gL32, sizeof(float) * r.ld, dL, sizeof(float) * ldgl, sizeof(float) * n, m,
                         cudaMemcpyDefault, st));
    launch_widen(m, n, gL32, r.ld, gLn, r.ld, st);
    if (dS) {
        float *tmp = wsT<float>(h, "ub_dS", mn);
        CK(cudaMemcpy2DAsync(tmp, sizeof(float) * r.ld, dS, sizeof(float) * ldgs, sizeof(float) * n, m,
                             cudaMemcpyDefault, st));
        launch_widen(m, n, tmp, r.ld, gSn, r.ld, st);
    } else {
        CK(cudaMemsetAsync(gSn, 0, sizeof(double) * mn, st));
    }
    CK(cudaMemsetAsync(gLp, 0, sizeof(double) * mn, st));
    CK(cudaMemsetAsync(gSp, 0, sizeof(double) * mn, st));
    CK(cudaMemsetAsync(dD64, 0, sizeof(double) * mn, st));
    CK(cudaMemsetAsync(scal, 0, sizeof(double) * 2, st));
    const int nck = (r.K + T - 1) / T;
    for (int c = nck - 1; c >= 0; c--) {
        const int k0 = c * T, k1 = std::min(r.K, k0 + T);
        // states of the segment: Ls[j] = L_{k0 - 1 + j}
        const float *ck = r.ck + (size_t)c * 4 * mn;
        CK(cudaMemcpyAsync(Ls + mn, ck, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(Ls, ck + mn, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(Ss + mn, ck + 2 * mn, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(Ss, ck + 3 * mn, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        for (int k = k0; k < k1; k++) {
            const int j = k - k0;
            unroll_step(h, r, tr, w, beta[k], mus[k], Ls + (j + 1) * mn, Ls + j * mn, Ss + (j + 1) * mn, Ss + j * mn,
                        Ls + (j + 2) * mn, Ss + (j + 2) * mn, Us + j * mq, sigs + (size_t)j * q, Vs + j * qq);
        }
        for (int k = k1 - 1; k >= k0; k--) {
            const int j = k - k0;
            const float *U = Us + j * mq, *V = Vs + j * qq;
            const double *sg = sigs + (size_t)j * q;
            const double thL = 0.5 * mus[k];
            const float thS = (float)(0.5 * r.lam * mus[k]);
            // gY = gL_{k+1} R
            const float *gy = gL32;
            int64_t ldy = r.ld;
            if (r.halvings > 0) {
                launch_restrict<float>(m, n, gL32, r.ld, gY, q, tr, st);
                gy = gY;
                ldy = q;
            }
            // SVT adjoint on the exact SVD: A = U^T gY V, B, gM = [U B + (gY V - U A) diag(f/s)] V^T
            launch_gemm_nn<float>(m, q, gy, ldy, V, q, P, q, nullptr, nullptr, q, st);
            const int sp = launch_gemm_tn_partial<float>(m, q, U, q, P, q, part, nullptr, q, q, st, nullptr);
            launch_reduce_partial<float>(part, sp, q, q, A, q, nullptr, nullptr, st);
            const int nb = launch_svt_adjoint_core(q, A, q, sg, thL, B, q, gthL, st);
            launch_gemm_nn<float>(m, q, U, q, B, q, Tm, q, nullptr, nullptr, q, st);
            launch_gemm_nn<float>(m, q, U, q, A, q, W, q, nullptr, nullptr, q, st);
            launch_svt_adjoint_combine(m, q, Tm, P, W, q, sg, thL, Z, st);
            launch_transpose<float>(q, q, V, q, Vt, q, st);
            if (r.halvings > 0) {
                launch_gemm_nn<float>(m, q, Z, q, Vt, q, w.gMH, q, nullptr, nullptr, q, st);
                launch_row_prolong(m, n, q, w.gMH, q, tr, gXL, r.ld, st);
            } else {
                launch_gemm_nn<float>(m, q, Z, q, Vt, q, gXL, r.ld, nullptr, nullptr, q, st);
            }
            const int ns = launch_unroll_adjoint(m, n, r.D, r.ld, r.Q, r.ldq, Ls + (j + 1) * mn, Ls + j * mn,
                                                 Ss + (j + 1) * mn, Ss + j * mn, r.ld, beta[k], thS, gXL, gLn, gSn,
                                                 gLp, gSp, dD64, gL32, gthS, st);
            launch_unroll_scalars(gthL, nb, gthS, ns, r.lam, mus[k], dmus[k], scal, st);
        }
    }
    launch_narrow(m, n, dD64, r.ld, dD, ldgd, st);
    double sc[2];
    CK(cudaMemcpyAsync(sc, scal, sizeof(sc), cudaMemcpyDeviceToHost, st));
    check_unroll_err(h, w);
    if (dlambda) *dlambda = sc[0];
    if (dmu) *dmu = sc[1];
    return CPCP_OK;
}

template <typename F>
cpcp_status guarded(cpcp_context *h, F &&f)
{
    try {
        if (h) {
            h->err.clear();
            CK(cudaSetDevice(h->device));
        }
        return f();
    } catch (const CpcpError &e) {
        if (h) h->err = e.msg;
        return e.st;
    } catch (const std::exception &e) {
        if (h) h->err = e.what();
        return CPCP_ERR_NOMEM;
    }
}

bool bad_dtype(cpcp_dtype dt) { return dt != CPCP_F32 && dt != CPCP_F64; }

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char *cpcp_status_string(cpcp_status s)
{
    switch (s) {
    case CPCP_OK: return "ok";
    case CPCP_ERR_INVALID_ARG: return "invalid argument";
    case CPCP_ERR_NONFINITE_INPUT: return "non-finite observed input";
    case CPCP_ERR_CUDA: return "CUDA error";
    case CPCP_ERR_NOMEM: return "out of device memory";
    case CPCP_ERR_NOT_CONVERGED: return "not converged (iteration cap)";
    case CPCP_ERR_TIMEOUT: return "bounded device wait expired";
    case CPCP_ERR_NUMERIC: return "numerical breakdown";
    }
    return "unknown status";
}

const char *cpcp_last_error(cpcp_handle h) { return h ? h->err.c_str() : ""; }

cpcp_status cpcp_create(cpcp_handle *out, int device, void *stream, const cpcp_options *opt)
{
    if (!out) return CPCP_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return CPCP_ERR_CUDA;
    }
    if (device < 0 || device >= count) return CPCP_ERR_INVALID_ARG;
    cpcp_context *h = new (std::nothrow) cpcp_context();
    if (!h) return CPCP_ERR_NOMEM;
    h->device = device;
    h->stream = static_cast<cudaStream_t>(stream);
    if (opt) h->opt = *opt;
    *out = h;
    return CPCP_OK;
}

void cpcp_destroy(cpcp_handle h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->batch.stream) cudaStreamSynchronize(h->batch.stream);
    if (h->batch.exec) cudaGraphExecDestroy(h->batch.exec);
    if (h->batch.graph) cudaGraphDestroy(h->batch.graph);
    if (h->batch.host_res) cudaFreeHost(h->batch.host_res);
    if (h->batch.stream) cudaStreamDestroy(h->batch.stream);
    if (h->solve_stream) {
        cudaStreamSynchronize(h->solve_stream);
        cudaStreamDestroy(h->solve_stream);
    }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->check_stream) {
        cudaStreamSynchronize(h->check_stream);
        cudaStreamDestroy(h->check_stream);
    }
    if (h->ev_snap) cudaEventDestroy(h->ev_snap);
    if (h->aux_stream) {
        cudaStreamSynchronize(h->aux_stream);
        cudaStreamDestroy(h->aux_stream);
    }
    for (auto e : h->ev_aux)
        if (e) cudaEventDestroy(e);
    if (h->check_host) cudaFreeHost(h->check_host);
    for (auto &kv : h->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    delete h;
}

cpcp_status cpcp_transfer_orth(int n, int halvings, double *cd, double *ce, double *kappa)
{
    if (n < 1 || halvings < 1 || halvings > 5) return CPCP_ERR_INVALID_ARG;
    try {
        std::vector<double> a, b;
        const double k = orth_factor(n, halvings, a, b);
        if (cd) std::copy(a.begin(), a.end(), cd);
        if (ce) std::copy(b.begin(), b.end(), ce);
        if (kappa) *kappa = k;
        return CPCP_OK;
    } catch (const CpcpError &e) {
        return e.st;
    }
}

cpcp_status cpcp_transfer_info(int n, int halvings, double *scale, int *nh)
{
    if (n < 1 || halvings < 0 || halvings > 5) return CPCP_ERR_INVALID_ARG;
    try {
        if (halvings == 0) {
            if (scale) *scale = 1.0;
            if (nh) *nh = n;
            return CPCP_OK;
        }
        HostTransfer t = build_transfer(n, halvings);
        if (scale) *scale = t.scale;
        if (nh) *nh = t.nh;
        return CPCP_OK;
    } catch (const CpcpError &e) {
        return e.st;
    }
}

cpcp_status cpcp_solve(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, const uint32_t *Q,
                       int64_t ldq, double lambda, double mu, int levels, double tol, void *L_out, int64_t ldl,
                       void *S_out, int64_t lds, cpcp_info *info)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (m < 1 || n < 1 || !D || bad_dtype(dt)) throw CpcpError{CPCP_ERR_INVALID_ARG, "bad sizes, D or dtype"};
        if (!(lambda > 0) || !(mu > 0) || !(tol > 0))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "lambda, mu and tol must be positive"};
        if (levels < 1 || levels > 6) throw CpcpError{CPCP_ERR_INVALID_ARG, "levels must be in [1, 6]"};
        if (h->opt.precision < 0 || h->opt.precision > 1 || (h->opt.precision == 1 && dt != CPCP_F32))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "precision must be 0, or 1 (mixed) with CPCP_F32"};
        if (ldd < n || (L_out && ldl < n) || (S_out && lds < n))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "leading dimension smaller than n"};
        if (Q && ldq < (n + 31) / 32) throw CpcpError{CPCP_ERR_INVALID_ARG, "ldq < ceil(n/32)"};
        int mm = std::max(m, n), nn = std::min(m, n);
        int nh = coarse_dim(nn, levels - 1);
        if (nh < 1) throw CpcpError{CPCP_ERR_INVALID_ARG, "coarse width below 1"};
        if (levels > 1 && 2 * nh > mm + 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "coarse width exceeds (m+1)/2 (Assumption 2)"};
        if (h->opt.transfer != 0 && h->opt.transfer != 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "transfer must be 0 or 1"};
        if (h->opt.subspace_mode != 0)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "subspace_mode must be 0"};
        if (h->opt.early_test < -1 || h->opt.early_test > 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "early_test must be -1, 0 or 1"};
        if (h->opt.products_tc < -1 || h->opt.products_tc > 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "products_tc must be -1, 0 or 1"};
        if (h->opt.chol_form < 0 || h->opt.chol_form > 2)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "chol_form must be 0, 1 or 2"};
        if (h->opt.svd_serial < 0 || h->opt.svd_serial > 2)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "svd_serial must be 0, 1 or 2"};
        if (h->opt.gram_form < 0 || h->opt.gram_form > 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "gram_form must be 0 or 1"};
        if (h->opt.jacobi_lanes != 0 && h->opt.jacobi_lanes != 8 && h->opt.jacobi_lanes != 16)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "jacobi_lanes must be 0, 8 or 16"};
        if (h->opt.jacobi_check < 0 || h->opt.jacobi_check > 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "jacobi_check must be 0 or 1"};
        if (h->opt.pdl_off < 0 || h->opt.pdl_off > 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "pdl_off must be 0 or 1"};
        if (h->opt.unroll > 0) {
            if (dt != CPCP_F32) throw CpcpError{CPCP_ERR_INVALID_ARG, "the unrolled program is fp32"};
            if (h->opt.transfer == 1)
                throw CpcpError{CPCP_ERR_INVALID_ARG, "the unrolled program takes the unit-norm R (transfer = 0)"};
            return unroll_forward(h, m, n, static_cast<const float *>(D), ldd, Q, ldq, lambda, mu, levels,
                                  static_cast<float *>(L_out), ldl, static_cast<float *>(S_out), lds, info);
        }
        if (dt == CPCP_F32)
            return solve_dispatch<float>(h, m, n, D, ldd, Q, ldq, lambda, mu, levels, tol, L_out, ldl, S_out, lds,
                                         info);
        return solve_dispatch<double>(h, m, n, D, ldd, Q, ldq, lambda, mu, levels, tol, L_out, ldl, S_out, lds,
                                      info);
    });
}

cpcp_status cpcp_ialm(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, double lambda,
                      int levels, double mu0, double rho, int max_iter, double tol, void *L_out, int64_t ldl,
                      void *S_out, int64_t lds, double *fg, cpcp_info *info)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (n < 1 || m < n || !D || bad_dtype(dt)) throw CpcpError{CPCP_ERR_INVALID_ARG, "need 1 <= n <= m, D, dtype"};
        if (!(lambda > 0) || !(tol > 0) || max_iter < 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "lambda and tol must be positive, max_iter >= 1"};
        if (levels < 1 || levels > 6) throw CpcpError{CPCP_ERR_INVALID_ARG, "levels must be in [1, 6]"};
        if (h->opt.transfer != 0 && h->opt.transfer != 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "transfer must be 0 or 1"};
        if (ldd < n || (L_out && ldl < n) || (S_out && lds < n))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "leading dimension smaller than n"};
        const int nh = coarse_dim(n, levels - 1);
        if (nh < 1) throw CpcpError{CPCP_ERR_INVALID_ARG, "coarse width below 1"};
        if (levels > 1 && 2 * nh > m + 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "coarse width exceeds (m+1)/2 (Assumption 2)"};
        if (dt == CPCP_F32)
            return ialm_dispatch<float>(h, m, n, D, ldd, lambda, levels, mu0, rho, max_iter, tol, L_out, ldl, S_out,
                                        lds, fg, info);
        return ialm_dispatch<double>(h, m, n, D, ldd, lambda, levels, mu0, rho, max_iter, tol, L_out, ldl, S_out, lds,
                                     fg, info);
    });
}

cpcp_status cpcp_fwt(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, const uint32_t *Q,
                     int64_t ldq, double lambda, double mu, int levels, int max_iter, double tol, void *L_out,
                     int64_t ldl, void *S_out, int64_t lds, double *ftrace, cpcp_info *info)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (m < 1 || n < 1 || !D || bad_dtype(dt)) throw CpcpError{CPCP_ERR_INVALID_ARG, "need m, n >= 1, D, dtype"};
        if (!(lambda > 0) || !(mu > 0) || !(tol >= 0) || max_iter < 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "lambda and mu must be positive, tol >= 0, max_iter >= 1"};
        if (levels < 1 || levels > 6) throw CpcpError{CPCP_ERR_INVALID_ARG, "levels must be in [1, 6]"};
        if (ldd < n || (L_out && ldl < n) || (S_out && lds < n) || (Q && ldq < (n + 31) / 32))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "leading dimension too small"};
        if (coarse_dim(n, levels - 1) < 1) throw CpcpError{CPCP_ERR_INVALID_ARG, "coarse width below 1"};
        if (h->opt.transfer != 0 && h->opt.transfer != 1)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "transfer must be 0 or 1"};
        if (!is_device_ptr(D) || (Q && !is_device_ptr(Q)) || (L_out && !is_device_ptr(L_out)) ||
            (S_out && !is_device_ptr(S_out)))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "cpcp_fwt takes device buffers"};
        if (dt == CPCP_F32)
            return fwt_core<float>(h, m, n, static_cast<const float *>(D), ldd, Q, ldq, lambda, mu, levels, max_iter,
                                   tol, static_cast<float *>(L_out), ldl, static_cast<float *>(S_out), lds, ftrace,
                                   info);
        return fwt_core<double>(h, m, n, static_cast<const double *>(D), ldd, Q, ldq, lambda, mu, levels, max_iter,
                                tol, static_cast<double *>(L_out), ldl, static_cast<double *>(S_out), lds, ftrace,
                                info);
    });
}

cpcp_status cpcp_step(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd, const uint32_t *Q,
                      int64_t ldq, double lambda, double mu_k, double beta, int halvings, const void *S_k,
                      const void *S_p, int64_t lds_in, const void *A_k, int64_t lda, const void *B_k, int64_t ldb,
                      int r_k, const void *A_p, int64_t ldap, const void *B_p, int64_t ldbp, int r_p, int k, int q,
                      const void *Omega0, int64_t ldo, void *S_out, int64_t lds, void *A_out, int64_t ldao,
                      void *B_out, int64_t ldbo, int *r_out, double *sigma_out)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (m < 1 || n < 1 || n > m || !D || !S_k || !S_out || !A_out || !B_out || bad_dtype(dt))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad sizes or NULL buffer (cpcp_step needs n <= m)"};
        if (!(lambda > 0) || !(mu_k > 0) || beta < 0 || halvings < 0 || halvings > 5 || q < 1 || r_k < 0 ||
            r_p < 0 || (r_k > 0 && (!A_k || !B_k)) || (r_p > 0 && (!A_p || !B_p)) || (beta > 0 && !S_p))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad step parameters"};
        if (dt == CPCP_F32)
            return step_impl<float>(h, m, n, D, ldd, Q, ldq, lambda, mu_k, beta, halvings, S_k, S_p, lds_in, A_k,
                                    lda, B_k, ldb, r_k, A_p, ldap, B_p, ldbp, r_p, k, q, Omega0, ldo, S_out, lds,
                                    A_out, ldao, B_out, ldbo, r_out, sigma_out);
        return step_impl<double>(h, m, n, D, ldd, Q, ldq, lambda, mu_k, beta, halvings, S_k, S_p, lds_in, A_k, lda,
                                 B_k, ldb, r_k, A_p, ldap, B_p, ldbp, r_p, k, q, Omega0, ldo, S_out, lds, A_out,
                                 ldao, B_out, ldbo, r_out, sigma_out);
    });
}

cpcp_status cpcp_restrict(cpcp_handle h, int m, int n, int halvings, cpcp_dtype dt, const void *M, int64_t ldm,
                          void *MH, int64_t ldh)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (m < 1 || n < 1 || halvings < 0 || halvings > 5 || !M || !MH || bad_dtype(dt))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad restrict arguments"};
        if (dt == CPCP_F32) {
            TransferDev<float> tr = upload_transfer<float>(h, n, halvings, "op");
            launch_restrict<float>(m, n, static_cast<const float *>(M), ldm, static_cast<float *>(MH), ldh, tr,
                                   h->stream);
        } else {
            TransferDev<double> tr = upload_transfer<double>(h, n, halvings, "op");
            launch_restrict<double>(m, n, static_cast<const double *>(M), ldm, static_cast<double *>(MH), ldh, tr,
                                    h->stream);
        }
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaGetLastError());
        return CPCP_OK;
    });
}

cpcp_status cpcp_prolong(cpcp_handle h, int n, int halvings, int r, cpcp_dtype dt, const void *V, int64_t ldv,
                         void *B, int64_t ldb)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (n < 1 || r < 1 || halvings < 0 || halvings > 5 || !V || !B || bad_dtype(dt) || ldb < r)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad prolong arguments"};
        if (dt == CPCP_F32) {
            TransferDev<float> tr = upload_transfer<float>(h, n, halvings, "op");
            launch_prolong<float>(n, static_cast<const float *>(V), ldv, static_cast<float *>(B), ldb, tr, nullptr,
                                  r, h->stream);
        } else {
            TransferDev<double> tr = upload_transfer<double>(h, n, halvings, "op");
            launch_prolong<double>(n, static_cast<const double *>(V), ldv, static_cast<double *>(B), ldb, tr, nullptr,
                                   r, h->stream);
        }
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaGetLastError());
        return CPCP_OK;
    });
}

cpcp_status cpcp_svd(cpcp_handle h, int m, int n, cpcp_dtype dt, const void *M, int64_t ldm, int k, int q,
                     const void *Omega0, int64_t ldo, void *U, int64_t ldu, void *V, int64_t ldv, double *sigma)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (m < 1 || n < 1 || n > m || !M || !U || !V || !sigma || q < 1 || bad_dtype(dt))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad svd arguments (needs m >= n)"};
        if (h->opt.precision < 0 || h->opt.precision > 1 || (h->opt.precision == 1 && dt != CPCP_F32))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "precision must be 0, or 1 (mixed) with CPCP_F32"};
        if (dt == CPCP_F32) return svd_impl<float>(h, m, n, M, ldm, k, q, Omega0, ldo, U, ldu, V, ldv, sigma);
        return svd_impl<double>(h, m, n, M, ldm, k, q, Omega0, ldo, U, ldu, V, ldv, sigma);
    });
}

cpcp_status cpcp_backward(cpcp_handle h, const float *dL, int64_t ldgl, const float *dS, int64_t ldgs, float *dD,
                          int64_t ldgd, double *dlambda, double *dmu)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (!dL || !dD || ldgl < h->unroll.n || ldgd < h->unroll.n || (dS && ldgs < h->unroll.n))
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad backward arguments"};
        return unroll_backward(h, dL, ldgl, dS, ldgs, dD, ldgd, dlambda, dmu);
    });
}

cpcp_status cpcp_solve_batched(cpcp_handle h, int count, const cpcp_problem *probs, double tol, cpcp_info *infos)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (h->opt.transfer != 0)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "the batched solve takes the unit-norm R (transfer = 0)"};
        return batched_impl(h, count, probs, tol, infos);
    });
}

cpcp_status cpcp_gemm_bf16(cpcp_handle h, int rows, int K, int N, const float *A, int64_t lda, const float *B,
                           int64_t ldb, float *C, int64_t ldc)
{
    if (!h) return CPCP_ERR_INVALID_ARG;
    return guarded(h, [&]() -> cpcp_status {
        if (rows < 1 || K < 1 || N < 1 || N > 256 || !A || !B || !C || lda < K || ldb < K || ldc < N)
            throw CpcpError{CPCP_ERR_INVALID_ARG, "bad gemm_bf16 arguments (1 <= N <= 256)"};
        return gemm_bf16_impl(h, rows, K, N, A, lda, B, ldb, C, ldc);
    });
}

}  // extern "C"
