// Active-set solve of the weight problem (Sec. 2.3) for libraries with many
// more orbits than constraints.
//
// The non-negative least-squares minimiser keeps only a part of the N orbits
// (about rank(U), more with the regulariser), so instead of iterating on all
// of them this follows the Lawson-Hanson active-set method on a passive set F:
// solve the unconstrained problem on F, keep the iterate feasible and its
// objective non-increasing, and add the orbits that violate the KKT conditions
// (negative gradient g_i > tol at w_i = 0).  Two changes make it fit a
// hundred-thousand-orbit library: violators enter in blocks of the strongest
// (largest g_i / |u~_i|), and when the solution on F has negative weights the
// projection max(x, 0) is taken whenever it lowers the objective, so that many
// orbits can leave in one step; the classical step back to the first zero is
// the fallback that keeps the method monotone.
//
// Each reduced problem (U~_F^T U~_F + 2 lambda/N I) x = q_F is solved on the
// GPU by preconditioned conjugate gradients whose products use the stored
// matrix with FP64 accumulation.  The preconditioner is the Cholesky factor of
// the Jacobi-scaled Gram of the factored set P0, formed on the tensor cores
// (BF16 hi + lo split, FP32 accumulation), factored in FP32 with its triangular
// inverse kept explicitly.  The solve accepts any F inside P0: the orbits of P0
// outside F are masked and the preconditioner is corrected to the exact
// inverse on F (block inverse of P0's).  A pivoting step whose passive set
// stays inside P0 (a few orbits masked) reuses the factor, one that adds a few
// orbits extends it by bordering, and any other refactors on its own passive
// set.  The gradient over all N orbits is recomputed in FP64 after every step.
#include "sw_linalg.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

namespace sw {

namespace {

#define AS_CUDA(ctx, expr, what)                                   \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return (ctx)->cuda_fail(e_, what);  \
    } while (0)
#define AS_TRY(expr)                 \
    do {                             \
        sw_status s_ = (expr);       \
        if (s_ != SW_OK) return s_;  \
    } while (0)

__global__ void k_as_chi2_finish(const double* __restrict__ in3, double lam_over_n, double* __restrict__ out3)
{
    out3[0] = in3[0];
    out3[1] = in3[1];
    out3[2] = lam_over_n * in3[2];
}

inline int64_t pad64(int64_t n) { return (n + 63) / 64 * 64; }

// ---- preconditioned conjugate gradients on (G_P + mu I) x = q_P, all in FP64.
// cg[0], cg[2]: r.z of the two most recent iterations (ping-pong, slot `old` /
// `fresh`), cg[1]: p.Ap, cg[3]: max|r| (bits of a non-negative double).
constexpr int CG_THREADS = 256;

__device__ inline double block_sum(double v)
{
    __shared__ double part[CG_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < CG_THREADS / 32 ? part[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double block_max(double v)
{
    __shared__ double part[CG_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < CG_THREADS / 32 ? part[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// out += sum_i a_i (b_i + mu c_i)
__global__ void k_cg_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                         const double* __restrict__ c, double mu, double* __restrict__ out)
{
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)CG_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_THREADS)
        s += a[i] * (b[i] + (c ? mu * c[i] : 0.0));
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// x += alpha p, r -= alpha m (Ap + mu p) with alpha = cg[old] / cg[1]; cg[3] = max|r|.
// m (nullable) masks the orbits of the factored set that are not in the passive set.
__global__ void k_cg_step(int64_t n, const double* __restrict__ cg, int old, const double* __restrict__ p,
                          const double* __restrict__ Ap, double mu, const double* __restrict__ m,
                          double* __restrict__ x, double* __restrict__ r, unsigned long long* __restrict__ rmax)
{
    const double alpha = cg[old] / cg[1];
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)CG_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_THREADS) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * (m ? m[i] : 1.0) * (Ap[i] + mu * p[i]);
        r[i] = ri;
        mx = fmax(mx, fabs(ri));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomicMax(rmax, (unsigned long long)__double_as_longlong(mx));
}

// p = z + beta p with beta = cg[fresh] / cg[old] (beta = 0 on the first step)
__global__ void k_cg_dir(int64_t n, const double* __restrict__ cg, int fresh, int old, bool first,
                         const double* __restrict__ z, double* __restrict__ p)
{
    const double beta = first ? 0.0 : cg[fresh] / cg[old];
    for (int64_t i = blockIdx.x * (int64_t)CG_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_THREADS)
        p[i] = z[i] + beta * p[i];
}

// r = m (q - g - mu x); max|r|
__global__ void k_cg_residual(int64_t n, const double* __restrict__ q, const double* __restrict__ g,
                              const double* __restrict__ x, double mu, const double* __restrict__ m,
                              double* __restrict__ r, unsigned long long* __restrict__ rmax)
{
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)CG_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_THREADS) {
        const double ri = (m ? m[i] : 1.0) * (q[i] - g[i] - mu * x[i]);
        r[i] = ri;
        mx = fmax(mx, fabs(ri));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomicMax(rmax, (unsigned long long)__double_as_longlong(mx));
}

// z = m z
__global__ void k_cg_mask(int64_t n, const double* __restrict__ m, double* __restrict__ z)
{
    for (int64_t i = blockIdx.x * (int64_t)CG_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_THREADS)
        z[i] *= m[i];
}

// XdT[k][i] = X[i][dpos[k]]: the columns of the factor's inverse at the masked orbits, as rows
template <typename GT>
__global__ void k_gather_xcols(const GT* __restrict__ X, int64_t ldx, int64_t K, const int64_t* __restrict__ dpos,
                               int64_t nD, GT* __restrict__ XdT, int64_t ldt)
{
    const int64_t n = nD * K;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / K, i = t - k * K;
        XdT[(size_t)k * ldt + i] = X[(size_t)i * ldx + dpos[k]];
    }
}

// W = H^-1 for a symmetric positive definite n x n matrix H (row-major, lower triangle read), in
// FP64 on the host: H = C C^T (Cholesky-Crout), Ci = C^-1, W = Ci^T Ci.  false if a pivot is not
// positive.
bool spd_inverse(std::vector<double>& H, int64_t n, std::vector<double>& W)
{
    for (int64_t j = 0; j < n; ++j) {
        double* hj = &H[(size_t)j * n];
        double d = hj[j];
        for (int64_t k = 0; k < j; ++k) d -= hj[k] * hj[k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        hj[j] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            double* hi = &H[(size_t)i * n];
            double v = hi[j];
            for (int64_t k = 0; k < j; ++k) v -= hi[k] * hj[k];
            hi[j] = v / d;
        }
    }
    // Ci by forward substitution, one row at a time: Ci[i][j] = -(sum_{k=j}^{i-1} C[i][k] Ci[k][j]) / C[i][i]
    std::vector<double> Ci((size_t)n * n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const double* hi = &H[(size_t)i * n];
        double* ci = &Ci[(size_t)i * n];
        for (int64_t k = 0; k < i; ++k) {
            const double c = hi[k];
            const double* ck = &Ci[(size_t)k * n];
            for (int64_t j = 0; j <= k; ++j) ci[j] -= c * ck[j];
        }
        const double inv = 1.0 / hi[i];
        for (int64_t j = 0; j < i; ++j) ci[j] *= inv;
        ci[i] = inv;
    }
    W.assign((size_t)n * n, 0.0);
    for (int64_t k = 0; k < n; ++k) {   // W += Ci[k]^T Ci[k] over the rows of Ci
        const double* ck = &Ci[(size_t)k * n];
        for (int64_t i = 0; i <= k; ++i) {
            const double a = ck[i];
            if (a == 0.0) continue;
            double* wi = &W[(size_t)i * n];
            for (int64_t j = 0; j <= k; ++j) wi[j] += a * ck[j];
        }
    }
    return true;
}

inline int cg_blocks(const sw_ctx* ctx, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + CG_THREADS - 1) / CG_THREADS, (int64_t)ctx_sms(ctx) * 8));
}

struct Span {
    char* p;
    size_t used = 0;
    template <typename X>
    X* take(int64_t n)
    {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + (size_t)n * sizeof(X);
        return p ? reinterpret_cast<X*>(p + off) : nullptr;
    }
};

// device vectors of the active-set solve
template <typename GT>
struct AsVecs {
    double *inv_sig, *ys, *acc, *e, *xs;          // M
    double *q, *h, *w, *ute, *gneg;               // N
    double *qP, *sP, *x, *gP, *ridge;             // passive set (cap)
    double *r, *z, *p, *mask, *xa;                // conjugate gradients, passive mask, candidate (cap)
    int64_t* idx;
    GT *rs, *t1, *c;
    double* scal;                                 // chi[4], pgmax, bad, info, err, cg[8]
    size_t carve(char* base, int64_t M, int64_t N, int64_t cap)
    {
        Span s{base};
        inv_sig = s.take<double>(M); ys = s.take<double>(M); acc = s.take<double>(M); e = s.take<double>(M);
        xs = s.take<double>(M);
        q = s.take<double>(N); h = s.take<double>(N); w = s.take<double>(N); ute = s.take<double>(N);
        gneg = s.take<double>(N);
        qP = s.take<double>(cap); sP = s.take<double>(cap); x = s.take<double>(cap); gP = s.take<double>(cap);
        ridge = s.take<double>(cap); idx = s.take<int64_t>(cap);
        r = s.take<double>(cap); z = s.take<double>(cap); p = s.take<double>(cap);
        mask = s.take<double>(cap); xa = s.take<double>(cap);
        rs = s.take<GT>(cap); t1 = s.take<GT>(cap); c = s.take<GT>(cap);
        scal = s.take<double>(16);
        return s.used + 256;
    }
};

}  // namespace

template <typename T, typename AT, typename GT>
sw_status solve_active_set(sw_ctx* ctx, const sw_matrix* Um, const double* y_dev, const double* sig_dev, double lam,
                           double* w_dev, double* chi2_dev, AsWarm* warm)
{
    const int64_t M = Um->M, N = Um->N;
    const T* U = (const T*)Um->d;
    cudaStream_t st = ctx->stream;
    SolveWS& ws = ctx->solve_ws;
    const int64_t cap = std::min<int64_t>(N, std::max<int64_t>(2 * M, 4096));
    const int64_t ldA = pad64(M);
    const bool split = sizeof(AT) == 2;
    const double mu = 2.0 * lam / (double)N;
    const double floor_ridge = sizeof(GT) == 4 ? 1e-6 : 1e-11;   // keeps the factor definite; CG removes it

    AsVecs<GT> V{};
    AS_TRY(ctx->ensure(&ws.outer, &ws.outer_cap, V.carve(nullptr, M, N, cap), "active-set vectors"));
    V.carve((char*)ws.outer, M, N, cap);
    double* chi = V.scal;
    unsigned long long* pgmax = (unsigned long long*)(V.scal + 4);
    int* bad = (int*)(V.scal + 5);
    int* info = (int*)(V.scal + 6);
    int* gerr = (int*)(V.scal + 7);
    double* cg = V.scal + 8;
    unsigned long long* rmax = (unsigned long long*)(cg + 3);

    AS_CUDA(ctx, cudaMemsetAsync(V.scal, 0, 16 * sizeof(double), st), "memset");
    AS_CUDA(ctx, prep_data(ctx, M, sig_dev, y_dev, V.inv_sig, V.ys, bad), "prep data");
    AS_CUDA(ctx, ut_times_x<T>(ctx, U, M, N, V.ys, V.q), "q");
    AS_CUDA(ctx, colnorm2<T>(ctx, U, M, N, V.inv_sig, V.h), "column norms");
    std::vector<double> qh(N), hh(N), gh(N), zh(N, 0.0), xh;
    int badh = 0;
    AS_CUDA(ctx, cudaMemcpyAsync(qh.data(), V.q, N * sizeof(double), cudaMemcpyDeviceToHost, st), "q");
    AS_CUDA(ctx, cudaMemcpyAsync(hh.data(), V.h, N * sizeof(double), cudaMemcpyDeviceToHost, st), "h");
    AS_CUDA(ctx, cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
    AS_CUDA(ctx, cudaStreamSynchronize(st), "active set");
    if (badh) { set_error(ctx, "solve: errors must be positive and finite, data finite"); return SW_EINVAL; }
    double qmax = 0.0;
    for (int64_t i = 0; i < N; ++i) qmax = std::max(qmax, std::fabs(qh[i]));
    const double gtol = ctx->opt.kkt_tol * std::max(qmax, 1e-300);
    const double rtol = ctx->opt.as_cg_tol * gtol;

    // ---- factor of the passive Gram on a set P0 of orbits: gathered columns Uc,
    // scales s = h^-1/2, explicit inverse X of the Cholesky factor of S G~ S + R
    // (tensor-core Gram of the scaled columns)
    std::vector<int64_t> P0;
    std::vector<int64_t> pos(N, -1);
    int n_factor = 0, n_solves = 0, cg_total = 0;
    // the tensor-core factorisation wants 16-byte rows of G and X (TMA)
    const bool fact_tc = sizeof(GT) == 4 && ctx->opt.chol_tc && !ctx->opt.chol_coop && chol_tc_available();
    int64_t ldG = 0;   // leading dimension of the factored set's G and X
    // passive Grams kept between factorisations (tensor-core form): valid within this solve, and
    // across the warm-started solves of one bootstrap (same matrix and errors)
    const bool gcache = fact_tc && split;
    // bordering (tensor-core form): the factor's buffers keep room for as_border more orbits, so that a
    // passive set adding a few orbits to the factored set P0 extends P0's factor instead of refactoring
    const int64_t slack = gcache ? std::max(0, ctx->opt.as_border) : 0;
    bool p0_ok = false;            // ws.X holds the inverse factor of P0
    double fl_ok = floor_ridge;    // ridge floor of that factor
    int n_border = 0;
    // the masked orbits' correction prepared for the next solve (prepare_mask, below)
    constexpr int64_t kMaskExactMax = 384;
    constexpr double kMaskCond = 3e3;
    int64_t mk_n = 0, mk_ldT = 0;
    GT *mk_XdT = nullptr, *mk_W = nullptr, *mk_cD = nullptr, *mk_uD = nullptr;
    bool mk_ready = false;
    int n_mask_refused = 0;
    if (!(warm && warm->start) || (int64_t)ws.gc_pos.size() != N) {
        ws.gc_set.clear();
        ws.gc_pos.assign(N, -1);
    }
    auto factor = [&](const std::vector<int64_t>& S_in, bool& ok) -> sw_status {
        const int64_t nP = (int64_t)S_in.size();
        ldG = fact_tc ? (nP + slack + 3) / 4 * 4 : nP;
        const int64_t room = nP + slack;
        ok = false;
        p0_ok = false;
        mk_ready = false;
        // with a kept Gram: the orbits it holds first (in its order), whole tile rows of them
        // gathered from it, the rest (and the partial tile row) computed
        std::vector<int64_t> S;
        int64_t r0 = 0;
        if (gcache && !ws.gc_set.empty()) {
            S.reserve(nP);
            std::vector<std::pair<int64_t, int64_t>> kept;
            for (int64_t i : S_in)
                if (ws.gc_pos[i] >= 0) kept.push_back({ws.gc_pos[i], i});
            std::sort(kept.begin(), kept.end());
            for (auto& kv : kept) S.push_back(kv.second);
            for (int64_t i : S_in)
                if (ws.gc_pos[i] < 0) S.push_back(i);
            r0 = (int64_t)kept.size() / 128 * 128;
        } else {
            S = S_in;
        }
        for (int64_t i : P0) pos[i] = -1;
        P0 = S;
        for (int64_t k = 0; k < nP; ++k) pos[S[k]] = k;
        std::vector<double> sh(nP), rh(nP);
        // G doubles as the bordering's scratch (two slack x ldG and two slack x slack blocks)
        const size_t g_elems = std::max((size_t)nP * ldG, (size_t)slack * (2 * ldG + 2 * ((slack + 3) / 4 * 4)));
        AS_TRY(ctx->ensure(&ws.Uc, &ws.Uc_cap, (size_t)room * M * sizeof(T), "passive columns"));
        AS_TRY(ctx->ensure(&ws.A, &ws.A_cap, (size_t)room * ldA * sizeof(AT), "passive matrix"));
        if (split) AS_TRY(ctx->ensure(&ws.Alo, &ws.Alo_cap, (size_t)room * ldA * sizeof(AT), "passive matrix (lo)"));
        AS_TRY(ctx->ensure(&ws.G, &ws.G_cap, g_elems * sizeof(GT), "reduced Gram"));
        AS_TRY(ctx->ensure(&ws.X, &ws.X_cap, (size_t)room * ldG * sizeof(GT), "reduced inverse factor"));
        AS_TRY(ctx->ensure(&ws.D, &ws.D_cap, 64 * 64 * sizeof(GT), "block scratch"));
        T* Uc = (T*)ws.Uc;
        AT* A = (AT*)ws.A;
        AT* Alo = split ? (AT*)ws.Alo : nullptr;
        GT* G = (GT*)ws.G;
        for (int64_t k = 0; k < nP; ++k) sh[k] = 1.0 / std::sqrt(hh[S[k]] > 0.0 ? hh[S[k]] : 1.0);
        AS_CUDA(ctx, cudaMemcpyAsync(V.idx, S.data(), nP * sizeof(int64_t), cudaMemcpyHostToDevice, st), "idx");
        AS_CUDA(ctx, cudaMemcpyAsync(V.sP, sh.data(), nP * sizeof(double), cudaMemcpyHostToDevice, st), "scales");
        AS_CUDA(ctx, gather_cols<T>(ctx, U, M, V.idx, nP, Uc), "gather");
        AS_CUDA(ctx, (whiten<T, AT>(ctx, Uc, M, nP, V.inv_sig, V.sP, A, Alo, ldA, true)), "whiten");
        double fl = floor_ridge;
        int infoh = 1, gerrh = 0;
        float* Gn = nullptr;   // the new kept Gram
        if constexpr (sizeof(AT) == 2) {
            if (gcache) {
                const int nx = 1 - ws.gc_cur;
                AS_TRY(ctx->ensure(&ws.Gc[nx], &ws.Gc_cap[nx], (size_t)room * ldG * sizeof(float), "kept Gram"));
                Gn = (float*)ws.Gc[nx];
                if (r0 > 0) {
                    std::vector<int64_t> ci(r0);
                    for (int64_t k = 0; k < r0; ++k) ci[k] = ws.gc_pos[S[k]];
                    AS_TRY(ctx->ensure(&ws.gcidx, &ws.gcidx_cap, (size_t)r0 * sizeof(int64_t), "kept Gram index"));
                    AS_CUDA(ctx, cudaMemcpyAsync(ws.gcidx, ci.data(), r0 * sizeof(int64_t), cudaMemcpyHostToDevice, st),
                            "kept Gram index");
                    AS_CUDA(ctx, gather_gram(ctx, (const float*)ws.Gc[ws.gc_cur], ws.gc_ld, (const int64_t*)ws.gcidx, r0, Gn,
                                             ldG),
                            "kept Gram");
                    // the host index list must outlive its copy
                    AS_CUDA(ctx, cudaStreamSynchronize(st), "kept Gram");
                }
                AS_CUDA(ctx, gram_tc(ctx, A, Alo, nP, ldA, Gn, gerr, ldG, r0 / 128), "reduced Gram");
                for (int64_t i : ws.gc_set) ws.gc_pos[i] = -1;
                ws.gc_set = S;
                for (int64_t k = 0; k < nP; ++k) ws.gc_pos[S[k]] = k;
                ws.gc_cur = nx;
                ws.gc_ld = ldG;
            }
        }
        double fl_try = fl;
        for (int attempt = 0; attempt < 4 && infoh != 0; ++attempt, fl *= 100.0) {
            fl_try = fl;
            for (int64_t k = 0; k < nP; ++k) rh[k] = std::max(mu * sh[k] * sh[k], fl);
            AS_CUDA(ctx, cudaMemcpyAsync(V.ridge, rh.data(), nP * sizeof(double), cudaMemcpyHostToDevice, st), "ridge");
            AS_CUDA(ctx, cudaMemsetAsync(info, 0, sizeof(int), st), "memset");
            if constexpr (sizeof(AT) == 2) {
                if (Gn)
                    AS_CUDA(ctx, cudaMemcpyAsync(G, Gn, (size_t)nP * ldG * sizeof(float), cudaMemcpyDeviceToDevice, st),
                            "reduced Gram");
                else
                    AS_CUDA(ctx, gram_tc(ctx, A, Alo, nP, ldA, (float*)G, gerr, ldG), "reduced Gram");
            } else {
                AS_CUDA(ctx, (gemm<GT, true, true>(ctx, K_GRAM_SIMT, nP, nP, ldA, GT(1), (const GT*)A, ldA,
                                                   (const GT*)A, ldA, GT(0), G, ldG, 0)),
                        "reduced Gram");
            }
            AS_CUDA(ctx, shift_diag_vec<GT>(ctx, G, nP, ldG, V.ridge), "ridge");
            int* cerr = (int*)(V.scal + 12);
            AS_CUDA(ctx, cudaMemsetAsync(cerr, 0, sizeof(int), st), "memset");
            cudaError_t ce = ctx->opt.chol_coop ? cholesky_inverse_coop<GT>(ctx, G, (GT*)ws.X, nP, info, cerr)
                                                : cudaErrorNotSupported;
            // verbose > 2: the host's enqueue time of the factorisation against its time to completion
            const bool timed = ctx->opt.verbose > 2;
            if (timed) AS_CUDA(ctx, cudaStreamSynchronize(st), "reduced factor");
            const auto th0 = std::chrono::steady_clock::now();
            if constexpr (sizeof(GT) == 4) {
                if (ce == cudaErrorNotSupported && fact_tc)
                    ce = cholesky_inverse_tc(ctx, (float*)G, (float*)ws.X, nP, ldG, info, gerr, false);
            }
            const auto th1 = std::chrono::steady_clock::now();
            if (ce == cudaErrorNotSupported) {
                cudaGetLastError();
                ce = ldG == nP ? cholesky_inverse<GT>(ctx, G, (GT*)ws.X, (GT*)ws.D, nP, info) : cudaErrorInvalidValue;
            }
            AS_CUDA(ctx, ce, "reduced Cholesky");
            int cerrh = 0;
            AS_CUDA(ctx, cudaMemcpyAsync(&infoh, info, sizeof(int), cudaMemcpyDeviceToHost, st), "info");
            AS_CUDA(ctx, cudaMemcpyAsync(&gerrh, gerr, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
            AS_CUDA(ctx, cudaMemcpyAsync(&cerrh, cerr, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
            AS_CUDA(ctx, cudaStreamSynchronize(st), "reduced factor");
            if (timed)
                fprintf(stderr, "[sw]   factor K %lld: enqueued in %.2f ms, done in %.2f ms\n", (long long)nP,
                        std::chrono::duration<double, std::milli>(th1 - th0).count(),
                        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count());
            if (gerrh) { set_error(ctx, "solve: a tensor-core kernel (Gram or factor update) timed out"); return SW_ETIMEOUT; }
            if (cerrh) { set_error(ctx, "solve: a grid barrier of the Cholesky kernel timed out"); return SW_ETIMEOUT; }
        }
        ++n_factor;
        if (warm) ++warm->factorisations;
        if (infoh != 0) return SW_OK;   // ok = false
        ok = true;
        p0_ok = true;
        fl_ok = fl_try;
        return SW_OK;
    };

    // orbits the factor's buffers hold at leading dimension ldG
    auto room_of = [&]() -> int64_t {
        if (!ldG || !ws.X || !ws.Uc || !ws.A || !ws.Gc[ws.gc_cur]) return 0;
        int64_t r = (int64_t)(ws.X_cap / ((size_t)ldG * sizeof(GT)));
        r = std::min(r, (int64_t)(ws.Gc_cap[ws.gc_cur] / ((size_t)ldG * sizeof(float))));
        r = std::min(r, (int64_t)(ws.Uc_cap / ((size_t)M * sizeof(T))));
        r = std::min(r, (int64_t)(ws.A_cap / ((size_t)ldA * sizeof(AT))));
        if (split) r = std::min(r, ws.Alo ? (int64_t)(ws.Alo_cap / ((size_t)ldA * sizeof(AT))) : 0);
        return r;
    };

    // ---- bordering: P1 = (P0, E) from the factor of P0.  With A the scaled, shifted Gram and
    // X0 = L0^-1 (A_00 = L0 L0^T):  L_E0 = A_E0 X0^T,  L_EE L_EE^T = A_EE - L_E0 L_E0^T,  and the
    // new block row of the inverse  X_E0 = -X_EE L_E0 X0,  X_EE = L_EE^-1.  The rows of the kept
    // Gram for E come from the tensor-core Gram of the appended tile rows; the leading block of the
    // factor, and of everything indexed by P0, is unchanged.  ok = false if an entering orbit lies
    // nearly in the span of P0 (a diagonal of A_EE - L_E0 L_E0^T below 5e-4 of its own) or that
    // matrix is not positive definite in FP32 (the caller then refactors).
    auto border = [&](const std::vector<int64_t>& E, bool& ok) -> sw_status {
        ok = false;
        mk_ready = false;
        if constexpr (sizeof(AT) == 2 && sizeof(GT) == 4) {
            const int64_t K0 = (int64_t)P0.size(), nE = (int64_t)E.size(), K1 = K0 + nE;
            const int64_t ldS = (nE + 3) / 4 * 4;
            T* Uc = (T*)ws.Uc;
            AT* A = (AT*)ws.A;
            AT* Alo = (AT*)ws.Alo;
            float* Gk = (float*)ws.Gc[ws.gc_cur];
            float* X = (float*)ws.X;
            float* L21 = (float*)ws.G;   // scratch: the in-place factor is not needed after factoring
            float* Y = L21 + (size_t)nE * ldG;
            float* Sm = Y + (size_t)nE * ldG;
            float* X22 = Sm + (size_t)nE * ldS;
            std::vector<double> sh(nE), rh(nE);
            for (int64_t k = 0; k < nE; ++k) {
                sh[k] = 1.0 / std::sqrt(hh[E[k]] > 0.0 ? hh[E[k]] : 1.0);
                rh[k] = std::max(mu * sh[k] * sh[k], fl_ok);
            }
            AS_CUDA(ctx, cudaMemcpyAsync(V.idx + K0, E.data(), nE * sizeof(int64_t), cudaMemcpyHostToDevice, st), "idx");
            AS_CUDA(ctx, cudaMemcpyAsync(V.sP + K0, sh.data(), nE * sizeof(double), cudaMemcpyHostToDevice, st), "scales");
            AS_CUDA(ctx, cudaMemcpyAsync(V.ridge + K0, rh.data(), nE * sizeof(double), cudaMemcpyHostToDevice, st), "ridge");
            AS_CUDA(ctx, gather_cols<T>(ctx, U, M, V.idx + K0, nE, Uc + (size_t)K0 * M), "gather");
            AS_CUDA(ctx, (whiten<T, AT>(ctx, Uc + (size_t)K0 * M, M, nE, V.inv_sig, V.sP + K0, A + (size_t)K0 * ldA,
                                        Alo + (size_t)K0 * ldA, ldA, true)),
                    "whiten");
            // the kept Gram's tile rows from the one holding row K0 on (P0's rows there are recomputed)
            AS_CUDA(ctx, gram_tc(ctx, A, Alo, K1, ldA, Gk, gerr, ldG, K0 / 128), "reduced Gram");
            for (size_t k = (size_t)K0; k < ws.gc_set.size(); ++k) ws.gc_pos[ws.gc_set[k]] = -1;
            ws.gc_set.resize(K0);
            for (int64_t k = 0; k < nE; ++k) {
                P0.push_back(E[k]);
                pos[E[k]] = K0 + k;
                ws.gc_set.push_back(E[k]);
                ws.gc_pos[E[k]] = K0 + k;
            }
            AS_CUDA(ctx, cudaMemsetAsync(X + (size_t)K0 * ldG, 0, (size_t)nE * ldG * sizeof(float), st), "memset");
            AS_CUDA(ctx, cudaMemsetAsync(L21, 0, (size_t)2 * nE * ldG * sizeof(float), st), "memset");   // L21, Y
            // L_E0 = A_E0 X0^T (X0 lower triangular)
            AS_CUDA(ctx, (gemm_acc<float, true, true>(ctx, K_BORDER, nE, K0, K0, 1.f, Gk + (size_t)K0 * ldG, ldG, X,
                                                      ldG, L21, ldG)),
                    "border");
            // S = A_EE + R_E - L_E0 L_E0^T (lower triangle; the factorisation reads no other)
            AS_CUDA(ctx, cudaMemcpy2DAsync(Sm, ldS * sizeof(float), Gk + (size_t)K0 * ldG + K0, ldG * sizeof(float),
                                           nE * sizeof(float), nE, cudaMemcpyDeviceToDevice, st),
                    "border");
            AS_CUDA(ctx, shift_diag_vec<float>(ctx, Sm, nE, ldS, V.ridge + K0), "ridge");
            AS_CUDA(ctx, (gemm_acc<float, true, false>(ctx, K_BORDER, nE, nE, K0, -1.f, L21, ldG, L21, ldG, Sm, ldS)),
                    "border");
            // every entering orbit must keep kBorderCond of its (unit) scaled norm outside the span of P0:
            // nearer to it the Schur complement is within the FP32 factor's error of zero (refactor)
            {
                constexpr double kBorderCond = 5e-4;
                std::vector<float> sd(nE);
                AS_CUDA(ctx, cudaMemcpy2DAsync(sd.data(), sizeof(float), Sm, (ldS + 1) * sizeof(float), sizeof(float), nE,
                                               cudaMemcpyDeviceToHost, st),
                        "border");
                AS_CUDA(ctx, cudaStreamSynchronize(st), "border");
                double smin = HUGE_VAL;
                for (int64_t k = 0; k < nE; ++k) smin = std::min(smin, (double)sd[k] / (1.0 + rh[k]));
                if (ctx->opt.verbose > 1) fprintf(stderr, "[sw]   border: min Schur diagonal %.3g\n", smin);
                if (!(smin >= kBorderCond)) return SW_OK;
            }
            AS_CUDA(ctx, cudaMemsetAsync(info, 0, sizeof(int), st), "memset");
            AS_CUDA(ctx, cholesky_inverse_tc(ctx, Sm, X22, nE, ldS, info, gerr, false), "border");
            // X_E0 = -X_EE (L_E0 X0), X_EE
            AS_CUDA(ctx, (gemm_acc<float, false, true>(ctx, K_BORDER, nE, K0, K0, 1.f, L21, ldG, X, ldG, Y, ldG)),
                    "border");
            AS_CUDA(ctx, (gemm<float, false, false>(ctx, K_BORDER, nE, K0, nE, -1.f, X22, ldS, Y, ldG, 0.f,
                                                    X + (size_t)K0 * ldG, ldG, 0)),
                    "border");
            AS_CUDA(ctx, cudaMemcpy2DAsync(X + (size_t)K0 * ldG + K0, ldG * sizeof(float), X22, ldS * sizeof(float),
                                           nE * sizeof(float), nE, cudaMemcpyDeviceToDevice, st),
                    "border");
            int infoh = 1, gerrh = 0;
            AS_CUDA(ctx, cudaMemcpyAsync(&infoh, info, sizeof(int), cudaMemcpyDeviceToHost, st), "info");
            AS_CUDA(ctx, cudaMemcpyAsync(&gerrh, gerr, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
            AS_CUDA(ctx, cudaStreamSynchronize(st), "border");
            if (gerrh) { set_error(ctx, "solve: a tensor-core kernel (Gram or factor update) timed out"); return SW_ETIMEOUT; }
            ++n_border;
            ok = infoh == 0;
        }
        return SW_OK;
    };

    // a passive set that adds at most as_border orbits to the factored set, with at most as_mask of the
    // extended set masked, borders the factor; done = false leaves the refactoring to the caller
    auto try_border = [&](const std::vector<int64_t>& Fn, bool& done) -> sw_status {
        done = false;
        if (!slack || !p0_ok || P0.empty() || ws.gc_ld != ldG) return SW_OK;
        std::vector<int64_t> E;
        for (int64_t i : Fn)
            if (pos[i] < 0) E.push_back(i);
        const int64_t K0 = (int64_t)P0.size(), nE = (int64_t)E.size(), K1 = K0 + nE;
        if (nE == 0 || nE > slack || K1 > cap || K1 > ldG || K1 > room_of()) return SW_OK;
        if ((double)(K1 - (int64_t)Fn.size()) > ctx->opt.as_mask * (double)K1) return SW_OK;
        const int64_t ldS = (nE + 3) / 4 * 4;
        if ((size_t)nE * (2 * ldG + 2 * ldS) * sizeof(float) > ws.G_cap) return SW_OK;
        // the kept Gram must hold P0 in the factor's order
        if ((int64_t)ws.gc_set.size() < K0) return SW_OK;
        for (int64_t k = 0; k < K0; ++k)
            if (ws.gc_set[k] != P0[k]) return SW_OK;
        bool ok = false;
        AS_TRY(border(E, ok));
        if (ctx->opt.verbose > 1)
            fprintf(stderr, "[sw]   border: %lld orbits appended to %lld, %lld masked%s\n", (long long)nE,
                    (long long)K0, (long long)(K1 - (int64_t)Fn.size()), ok ? "" : " (ill-conditioned: refactor)");
        if (!ok) p0_ok = false;
        done = ok;
        return SW_OK;
    };

    // ---- correction of the masked orbits D = P0 \ F for the solve on F.  With H = A^-1 = X^T X for
    // the scaled, shifted Gram A of P0, the inverse of A_FF is (H - H_:D H_DD^-1 H_D:)_FF (block
    // inverse), so the preconditioner applies z = X^T (t - X_:D u), t = X r, u = H_DD^-1 (X_:D^T t):
    // exact on F up to the factor's rounding, where the masked form alone leaves |D| outlying
    // eigenvalues to the iteration.  H_DD = X_:D^T X_:D is inverted on the host in FP64.  ok = false
    // when the correction cannot be formed accurately: more than kMaskExactMax masked orbits, or a
    // masked orbit nearly in the span of the others (H_dd = 1 / its squared distance from them, in
    // units of its unit scaled norm, above kMaskCond: the factor's ~1e-4 relative error would then
    // dominate the correction).
    auto prepare_mask = [&](const std::vector<int64_t>& Fs, bool& ok) -> sw_status {
        ok = false;
        mk_ready = false;
        mk_n = 0;
        const int64_t nP = (int64_t)P0.size();
        const GT* X = (const GT*)ws.X;
        std::vector<char> inP(nP, 0);
        for (int64_t i : Fs) inP[pos[i]] = 1;
        std::vector<int64_t> dpos;
        for (int64_t k = 0; k < nP; ++k)
            if (!inP[k]) dpos.push_back(k);
        const int64_t nD = (int64_t)dpos.size();
        if (nD == 0) { ok = mk_ready = true; return SW_OK; }
        if (nD > kMaskExactMax) return SW_OK;
        const int64_t ldT = (nP + 3) / 4 * 4;
        Span sp{nullptr};
        sp.take<int64_t>(nD);
        sp.take<GT>(nD * ldT);
        sp.take<GT>(nD * nD);
        sp.take<GT>(nD * nD);
        sp.take<GT>(nD);
        sp.take<GT>(nD);
        AS_TRY(ctx->ensure(&ws.Mc, &ws.Mc_cap, sp.used + 256, "masked-orbit correction"));
        Span sm{(char*)ws.Mc};
        int64_t* dpos_d = sm.take<int64_t>(nD);
        GT* XdT = sm.take<GT>(nD * ldT);
        GT* Hd = sm.take<GT>(nD * nD);
        GT* Wd = sm.take<GT>(nD * nD);
        GT* cD = sm.take<GT>(nD);
        GT* uD = sm.take<GT>(nD);
        AS_CUDA(ctx, cudaMemcpyAsync(dpos_d, dpos.data(), nD * sizeof(int64_t), cudaMemcpyHostToDevice, st),
                "masked orbits");
        {
            LaunchTimer lt(ctx, K_PCG);
            k_gather_xcols<GT><<<(unsigned)std::min<int64_t>((nD * nP + 255) / 256, (int64_t)ctx_sms(ctx) * 16), 256,
                                 0, st>>>(X, ldG, nP, dpos_d, nD, XdT, ldT);
        }
        AS_CUDA(ctx, cudaGetLastError(), "masked orbits");
        AS_CUDA(ctx, cudaMemsetAsync(Hd, 0, (size_t)nD * nD * sizeof(GT), st), "memset");
        AS_CUDA(ctx, (gemm_acc<GT, true, false>(ctx, K_PCG, nD, nD, nP, GT(1), XdT, ldT, XdT, ldT, Hd, nD)),
                "masked orbits");
        std::vector<GT> hg((size_t)nD * nD);
        AS_CUDA(ctx, cudaMemcpyAsync(hg.data(), Hd, hg.size() * sizeof(GT), cudaMemcpyDeviceToHost, st),
                "masked orbits");
        AS_CUDA(ctx, cudaStreamSynchronize(st), "masked orbits");
        std::vector<double> H(hg.begin(), hg.end()), Wh;
        double hmax = 0.0;
        for (int64_t k = 0; k < nD; ++k) hmax = std::max(hmax, H[(size_t)k * nD + k]);
        if (ctx->opt.verbose > 1) fprintf(stderr, "[sw]   mask: %lld orbits, max H_dd %.3g\n", (long long)nD, hmax);
        if (!(hmax <= kMaskCond) || !spd_inverse(H, nD, Wh)) {
            ++n_mask_refused;
            return SW_OK;
        }
        std::vector<GT> wg(Wh.begin(), Wh.end());
        AS_CUDA(ctx, cudaMemcpyAsync(Wd, wg.data(), wg.size() * sizeof(GT), cudaMemcpyHostToDevice, st),
                "masked orbits");
        AS_CUDA(ctx, cudaStreamSynchronize(st), "masked orbits");
        mk_n = nD;
        mk_ldT = ldT;
        mk_XdT = XdT;
        mk_W = Wd;
        mk_cD = cD;
        mk_uD = uD;
        ok = mk_ready = true;
        return SW_OK;
    };

    // ---- (G_F + mu I) x = q_F for a passive set F inside P0, by preconditioned
    // conjugate gradients in the coordinates of P0 with the orbits outside F masked:
    // the preconditioner is the inverse on F obtained from the P0 factor (below).
    // Products use the stored matrix with FP64 accumulation.  Result in xh (P0 order,
    // zero outside F).
    auto solve_on = [&](const std::vector<int64_t>& F, bool& converged) -> sw_status {
        const int64_t nP = (int64_t)P0.size();
        const T* Uc = (const T*)ws.Uc;
        const GT* X = (const GT*)ws.X;
        converged = false;
        std::vector<double> mh(nP, 0.0);
        for (int64_t i : F) mh[pos[i]] = 1.0;
        AS_CUDA(ctx, cudaMemcpyAsync(V.mask, mh.data(), nP * sizeof(double), cudaMemcpyHostToDevice, st), "mask");
        AS_CUDA(ctx, gather_vec(ctx, V.q, V.idx, nP, V.qP), "q_P");
        const int nb = cg_blocks(ctx, nP);
        // the masked orbits' correction, when prepare_mask formed it for this passive set
        const int64_t nDc = mk_ready ? mk_n : 0, ldT = mk_ldT;
        GT *XdT = mk_XdT, *Wd = mk_W, *cD = mk_cD, *uD = mk_uD;
        mk_ready = false;
        auto precond = [&](const double* r, double* z) -> sw_status {   // z = m S X^T X S r (corrected)
            AS_CUDA(ctx, scale_to<GT>(ctx, nP, r, V.sP, V.rs), "precondition");
            AS_CUDA(ctx, (rowdot<GT, GT, GT, GT>(ctx, K_TRMV_L, X, nP, nP, ldG, V.rs, V.t1, 1.0, 0.0, true)),
                    "precondition");
            if (nDc) {
                AS_CUDA(ctx, (rowdot<GT, GT, GT, GT>(ctx, K_PCG, XdT, nDc, nP, ldT, V.t1, cD, 1.0, 0.0, false)),
                        "precondition");
                AS_CUDA(ctx, (rowdot<GT, GT, GT, GT>(ctx, K_PCG, Wd, nDc, nDc, nDc, cD, uD, 1.0, 0.0, false)),
                        "precondition");
                AS_CUDA(ctx, (colcomb<GT, GT, GT, GT>(ctx, K_PCG, XdT, nDc, nP, ldT, uD, V.t1, -1.0, false)),
                        "precondition");
            }
            AS_CUDA(ctx, cudaMemsetAsync(V.c, 0, nP * sizeof(GT), st), "memset");
            AS_CUDA(ctx, (colcomb<GT, GT, GT, GT>(ctx, K_TRMV_LT, X, nP, nP, ldG, V.t1, V.c, 1.0, true)),
                    "precondition");
            AS_CUDA(ctx, cudaMemsetAsync(z, 0, nP * sizeof(double), st), "memset");
            AS_CUDA(ctx, axpy_scaled<GT>(ctx, nP, V.c, V.sP, z), "precondition");
            {
                LaunchTimer lt(ctx, K_PCG);
                k_cg_mask<<<nb, CG_THREADS, 0, st>>>(nP, V.mask, z);
            }
            AS_CUDA(ctx, cudaGetLastError(), "precondition");
            return SW_OK;
        };
        auto apply_G = [&](const double* v, double* out) -> sw_status {   // out = U_P0^T W U_P0 v
            AS_CUDA(ctx, cudaMemsetAsync(V.acc, 0, M * sizeof(double), st), "memset");
            AS_CUDA(ctx, u_times_w<T>(ctx, Uc, M, nP, v, V.acc), "U_P v");
            AS_CUDA(ctx, weight_sq(ctx, M, V.acc, V.inv_sig, V.xs), "weights");
            AS_CUDA(ctx, ut_times_x<T>(ctx, Uc, M, nP, V.xs, out), "U_P^T");
            return SW_OK;
        };
        // warm start x = m P^-1 q, r = m (q - (G + mu) x)
        AS_TRY(precond(V.qP, V.x));
        AS_TRY(apply_G(V.x, V.gP));
        AS_CUDA(ctx, cudaMemsetAsync(cg, 0, 8 * sizeof(double), st), "memset");
        {
            LaunchTimer lt(ctx, K_PCG);
            k_cg_residual<<<nb, CG_THREADS, 0, st>>>(nP, V.qP, V.gP, V.x, mu, V.mask, V.r, rmax);
        }
        AS_CUDA(ctx, cudaGetLastError(), "residual");
        double rm = 0.0;
        int old = 0, fresh = 2, it = 0;
        for (;; ++it) {
            AS_CUDA(ctx, cudaMemcpyAsync(&rm, rmax, sizeof(double), cudaMemcpyDeviceToHost, st), "residual");
            AS_CUDA(ctx, cudaStreamSynchronize(st), "pcg");
            if (!(rm > rtol)) { converged = rm == rm; break; }
            if (it >= ctx->opt.as_cg_max) break;
            AS_TRY(precond(V.r, V.z));
            AS_CUDA(ctx, cudaMemsetAsync(cg + fresh, 0, sizeof(double), st), "memset");
            AS_CUDA(ctx, cudaMemsetAsync(cg + 1, 0, sizeof(double), st), "memset");
            AS_CUDA(ctx, cudaMemsetAsync(cg + 3, 0, sizeof(double), st), "memset");
            {
                LaunchTimer lt(ctx, K_PCG);
                k_cg_dot<<<nb, CG_THREADS, 0, st>>>(nP, V.r, V.z, nullptr, 0.0, cg + fresh);
                k_cg_dir<<<nb, CG_THREADS, 0, st>>>(nP, cg, fresh, old, it == 0, V.z, V.p);
            }
            AS_CUDA(ctx, cudaGetLastError(), "pcg");
            AS_TRY(apply_G(V.p, V.gP));
            {
                LaunchTimer lt(ctx, K_PCG);
                k_cg_dot<<<nb, CG_THREADS, 0, st>>>(nP, V.p, V.gP, V.p, mu, cg + 1);
                k_cg_step<<<nb, CG_THREADS, 0, st>>>(nP, cg, fresh, V.p, V.gP, mu, V.mask, V.x, V.r, rmax);
            }
            AS_CUDA(ctx, cudaGetLastError(), "pcg");
            std::swap(old, fresh);
        }
        cg_total += it;
        ++n_solves;
        if (ctx->opt.verbose > 1)
            fprintf(stderr, "[sw]   solve |F| %zu in |P0| %lld: max|r| %.3g (tolerance %.3g), %d steps\n", F.size(),
                    (long long)nP, rm, rtol, it);
        xh.resize(nP);
        AS_CUDA(ctx, cudaMemcpyAsync(xh.data(), V.x, nP * sizeof(double), cudaMemcpyDeviceToHost, st), "x");
        AS_CUDA(ctx, cudaStreamSynchronize(st), "reduced solve");
        for (double v : xh)
            if (!std::isfinite(v)) converged = false;
        return SW_OK;
    };

    // objective chi^2 + mu |w|^2 of weights w supported on P0 (device vector in P0 order)
    auto objective_P0 = [&](const double* wP, double& fval) -> sw_status {
        const int64_t nP = (int64_t)P0.size();
        double ch[4];
        AS_CUDA(ctx, cudaMemsetAsync(V.acc, 0, M * sizeof(double), st), "memset");
        AS_CUDA(ctx, u_times_w<T>(ctx, (const T*)ws.Uc, M, nP, wP, V.acc), "U_P w");
        AS_CUDA(ctx, residual(ctx, M, y_dev, V.acc, V.inv_sig, V.e, V.xs), "residual");
        AS_CUDA(ctx, cudaMemsetAsync(chi, 0, 4 * sizeof(double), st), "memset");
        AS_CUDA(ctx, chi2(ctx, M, Um->nd, V.e, nP, wP, chi), "chi2");
        AS_CUDA(ctx, cudaMemcpyAsync(ch, chi, 4 * sizeof(double), cudaMemcpyDeviceToHost, st), "chi2");
        AS_CUDA(ctx, cudaStreamSynchronize(st), "objective");
        fval = ch[0] + mu * ch[2];
        return SW_OK;
    };

    // exact state of zh over all N: negative gradient gh, projected gradient, chi^2.  With wP (the
    // device copy of zh on P0, in P0's order; zh zero outside P0) U w is formed from P0's gathered
    // columns instead of the whole matrix.
    double pg_rel = 1.0, chi_h[4] = {0, 0, 0, 0};
    auto evaluate = [&](const double* wP = nullptr) -> sw_status {
        AS_CUDA(ctx, cudaMemcpyAsync(V.w, zh.data(), N * sizeof(double), cudaMemcpyHostToDevice, st), "w");
        AS_CUDA(ctx, cudaMemsetAsync(V.acc, 0, M * sizeof(double), st), "memset");
        if (wP)
            AS_CUDA(ctx, u_times_w<T>(ctx, (const T*)ws.Uc, M, (int64_t)P0.size(), wP, V.acc), "U_P w");
        else
            AS_CUDA(ctx, u_times_w<T>(ctx, U, M, N, V.w, V.acc), "U w");
        AS_CUDA(ctx, residual(ctx, M, y_dev, V.acc, V.inv_sig, V.e, V.xs), "residual");
        AS_CUDA(ctx, ut_times_x<T>(ctx, U, M, N, V.xs, V.ute), "U^T e");
        AS_CUDA(ctx, cudaMemsetAsync(pgmax, 0, 8, st), "memset");
        AS_CUDA(ctx, kkt(ctx, N, V.ute, V.w, mu, V.gneg, pgmax), "KKT");
        AS_CUDA(ctx, cudaMemsetAsync(chi, 0, 4 * sizeof(double), st), "memset");
        AS_CUDA(ctx, chi2(ctx, M, Um->nd, V.e, N, V.w, chi), "chi2");
        unsigned long long pb = 0;
        AS_CUDA(ctx, cudaMemcpyAsync(&pb, pgmax, 8, cudaMemcpyDeviceToHost, st), "KKT");
        AS_CUDA(ctx, cudaMemcpyAsync(chi_h, chi, 4 * sizeof(double), cudaMemcpyDeviceToHost, st), "chi2");
        AS_CUDA(ctx, cudaMemcpyAsync(gh.data(), V.gneg, N * sizeof(double), cudaMemcpyDeviceToHost, st), "g");
        AS_CUDA(ctx, cudaStreamSynchronize(st), "evaluate");
        double pgv;
        memcpy(&pgv, &pb, 8);
        pg_rel = pgv / std::max(qmax, 1e-300);
        return SW_OK;
    };

    // ---- block principal pivoting (Portugal, Judice & Vicente 1994; Kim & Park 2011)
    // on the passive set F: solve on F, then move passive orbits with negative weight
    // out and KKT violators (g_i > tol at w_i = 0) in.  Entering is limited to the
    // max(as_block, as_grow |F|) strongest violators (largest g_i / |u~_i|).  While the number of
    // violations keeps falling, all of them are exchanged; after a step without a new
    // minimum only the most violating fraction is, halved at every such step (the
    // strongest first), which damps the cycling that a full exchange can fall into;
    // a fraction below one orbit exchanges the single worst violator.
    std::vector<char> inF(N, 0);
    std::vector<int64_t> F;
    std::vector<double> buf;
    bool failed = false, converged = false, evaluated = false;
    // candidate set C: the orbits with the largest q_i / |u~_i| first; pivoting runs on
    // C and C grows by the strongest violators outside it whenever F is optimal on C
    std::vector<char> inC(N, 0);
    int64_t nC = std::min<int64_t>(N, std::max<int64_t>(1, ctx->opt.as_candidates > 0 ? (int64_t)ctx->opt.as_candidates : 2 * M));
    if (warm && warm->start) nC = N;   // a warm start begins near the optimum: every orbit is a candidate
    {
        std::vector<std::pair<double, int64_t>> sc(N);
        for (int64_t i = 0; i < N; ++i) sc[i] = {hh[i] > 0.0 ? qh[i] / std::sqrt(hh[i]) : -1e300, i};
        std::partial_sort(sc.begin(), sc.begin() + nC, sc.end(),
                          [](const std::pair<double, int64_t>& a, const std::pair<double, int64_t>& b) {
                              return a.first > b.first;
                          });
        for (int64_t k = 0; k < nC; ++k) inC[sc[k].second] = 1;
    }
    int outer = 0;
    int64_t best_nv = N + 1;
    double frac = 1.0;
    const int64_t block = std::max<int64_t>(1, ctx->opt.as_block);
    // merit: objective of the projection max(x, 0) of each iterate; the best is kept
    std::vector<double> zbest(N, 0.0);
    double fproj = 0.0, fbest = 0.0;
    // reference of the damping test: the best objective since the candidate set last grew (a wider
    // candidate set starts from a worse passive set than the optimum on the narrower one)
    double fref = 0.0;
    {
        double f0 = 0.0;
        AS_TRY(evaluate());
        f0 = chi_h[0];
        fbest = fproj = fref = f0;
    }
    // the factor of P0 serves every passive set inside it (the orbits of P0 \ F masked)
    // (the recorded factor of a warm start serves every passive set inside it; another factor serves
    // those that mask at most as_mask of it)
    auto factored_covers = [&](const std::vector<int64_t>& S) {
        if (P0.empty() || !p0_ok) return false;
        for (int64_t i : S)
            if (pos[i] < 0) return false;
        if (warm && warm->have_factor) return true;
        return (double)((int64_t)P0.size() - (int64_t)S.size()) <= ctx->opt.as_mask * (double)P0.size();
    };
    if (warm && warm->start && (int64_t)warm->F0.size() == N && !warm->P0.empty()) {
        // begin from the recorded passive set, solved against this problem's data with the factor of
        // P0 (factored again when an earlier warm-started solve replaced it)
        bool have = warm->have_factor;
        if (have) {
            for (int64_t i : P0) pos[i] = -1;
            P0 = warm->P0;
            ldG = warm->ld;
            for (int64_t k = 0; k < (int64_t)P0.size(); ++k) pos[P0[k]] = k;
            p0_ok = true;
            fl_ok = warm->fl;
        } else {
            const std::vector<int64_t> S = warm->P0;
            AS_TRY(factor(S, have));
            warm->have_factor = have;
        }
        if (have)
            for (int64_t i = 0; i < N; ++i)
                if (warm->F0[i]) { inF[i] = 1; F.push_back(i); }
        if (!F.empty()) {
            bool conv = false, mok = false;
            AS_TRY(prepare_mask(F, mok));   // masked-only without it
            AS_TRY(solve_on(F, conv));
            std::fill(zh.begin(), zh.end(), 0.0);
            for (int64_t i : F) zh[i] = xh[pos[i]];
            buf.assign(P0.size(), 0.0);
            for (int64_t i : F) buf[pos[i]] = std::max(zh[i], 0.0);
            AS_CUDA(ctx, cudaMemcpyAsync(V.xa, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                    "x+");
            AS_TRY(objective_P0(V.xa, fproj));
            if (fproj < fbest) {
                fbest = fproj;
                for (int64_t i = 0; i < N; ++i) zbest[i] = std::max(zh[i], 0.0);
            }
            AS_TRY(evaluate(V.x));
            evaluated = true;
        }
    }
    // verbose > 2: wall time of each phase of a pivoting step (host decisions, factor, solve, objective,
    // evaluation), each phase ending at a synchronisation
    auto wall = [] { return std::chrono::steady_clock::now(); };
    auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    for (; outer < 1000000 && n_solves < ctx->opt.as_solves; ++outer) {
        const auto w0 = wall();
        auto w1 = w0, w2 = w0, w3 = w0, w4 = w0;
        std::vector<std::pair<double, int64_t>> neg, enter;   // (violation, orbit)
        bool widened = false;
        for (int64_t i : F)
            if (zh[i] < 0.0) neg.push_back({-zh[i] * std::sqrt(hh[i]), i});
        for (int64_t i = 0; i < N; ++i)
            if (inC[i] && !inF[i] && gh[i] > gtol && hh[i] > 0.0) enter.push_back({gh[i] / std::sqrt(hh[i]), i});
        if (neg.empty() && enter.empty() && nC < N) {
            // optimal on the candidate set C: widen C by the strongest violators outside it
            std::vector<std::pair<double, int64_t>> out;
            for (int64_t i = 0; i < N; ++i)
                if (!inC[i] && gh[i] > gtol && hh[i] > 0.0) out.push_back({gh[i] / std::sqrt(hh[i]), i});
            const int64_t kc = std::min<int64_t>((int64_t)out.size(), std::max<int64_t>(block, nC / 2));
            std::partial_sort(out.begin(), out.begin() + kc, out.end(),
                              [](const std::pair<double, int64_t>& a, const std::pair<double, int64_t>& b) {
                                  return a.first > b.first;
                              });
            for (int64_t k = 0; k < kc; ++k) {
                inC[out[k].second] = 1;
                enter.push_back(out[k]);
            }
            nC += kc;
            best_nv = N + 1;
            fref = HUGE_VAL;
            widened = kc > 0;
            frac = 1.0;
            if (ctx->opt.verbose && kc)
                fprintf(stderr, "[sw] candidate set widened by %lld to %lld orbits\n", (long long)kc, (long long)nC);
        }
        const int64_t nv = (int64_t)(neg.size() + enter.size());
        if (ctx->opt.verbose)
            fprintf(stderr,
                    "[sw] pivoting %d: |F| %zu solves %d cg %d negative %zu entering %zu fraction %.3g "
                    "objective+ %.10g\n",
                    outer, F.size(), n_solves, cg_total, neg.size(), enter.size(), frac, fproj);
        if (nv == 0) { converged = true; break; }
        const int64_t lim = std::max<int64_t>(block, (int64_t)(ctx->opt.as_grow * (double)F.size()));
        if (outer > 0) {
            // damped exchanges: halve the fraction when neither the objective nor the violation count
            // improved, and let it recover only gradually (x4 per improving step), so that a degenerate
            // problem does not alternate between full and damped exchanges
            if (fproj < fref * (1.0 - 1e-13) || nv < best_nv) frac = std::min(1.0, 4.0 * frac);
            else frac *= 0.5;
            best_nv = std::min(best_nv, nv);
            if (!widened) fref = std::min(fref, fproj);   // fproj is still the narrower set's
        }
        auto by_violation = [](const std::pair<double, int64_t>& a, const std::pair<double, int64_t>& b) {
            return a.first > b.first;
        };
        int64_t kn = (int64_t)std::ceil(frac * (double)neg.size());
        int64_t ke = std::min<int64_t>(lim, (int64_t)std::ceil(frac * (double)enter.size()));
        if (frac * (double)nv < 1.0) {   // single worst violator
            kn = ke = 0;
            if (!neg.empty() && (enter.empty() || *std::max_element(neg.begin(), neg.end()) >
                                                      *std::max_element(enter.begin(), enter.end())))
                kn = 1;
            else
                ke = 1;
        }
        ke = std::max<int64_t>(0, std::min<int64_t>(ke, cap - ((int64_t)F.size() - kn)));
        std::partial_sort(neg.begin(), neg.begin() + kn, neg.end(), by_violation);
        std::partial_sort(enter.begin(), enter.begin() + ke, enter.end(), by_violation);
        for (int64_t k = 0; k < kn; ++k) inF[neg[k].second] = 0;
        for (int64_t k = 0; k < ke; ++k) inF[enter[k].second] = 1;
        F.clear();
        for (int64_t i = 0; i < N; ++i)
            if (inF[i]) F.push_back(i);
        std::fill(zh.begin(), zh.end(), 0.0);
        bool solved = false;   // V.x holds zh on P0
        w1 = wall();
        if (!F.empty()) {
            bool ok = true, conv = false;
            // the factor of P0 serves F when it covers F and the masked orbits' correction can be formed
            // (a warm start's recorded factor also runs masked-only); else it is bordered by the entering
            // orbits; else F is factored.  A bordered factor keeps P0's factor as its leading block: a
            // warm start's recorded factor survives it.
            bool ready = false;
            if (factored_covers(F)) {
                bool mok = false;
                AS_TRY(prepare_mask(F, mok));
                ready = mok || (warm && warm->have_factor);
            }
            if (!ready) {
                bool bordered = false;
                AS_TRY(try_border(F, bordered));
                if (bordered) AS_TRY(prepare_mask(F, ready));
            }
            if (!ready) {
                AS_TRY(factor(F, ok));
                if (warm) warm->have_factor = false;   // P0 is now this passive set
            }
            if (!ok) { failed = true; break; }
            w2 = wall();
            AS_TRY(solve_on(F, conv));
            w3 = wall();
            solved = true;
            for (int64_t i : F) zh[i] = xh[pos[i]];
            buf.assign(P0.size(), 0.0);
            for (int64_t i : F) buf[pos[i]] = std::max(zh[i], 0.0);
            AS_CUDA(ctx, cudaMemcpyAsync(V.xa, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                    "x+");
            AS_TRY(objective_P0(V.xa, fproj));
            w4 = wall();
        } else {
            fproj = fbest;
        }
        if (fproj < fbest) {
            fbest = fproj;
            for (int64_t i = 0; i < N; ++i) zbest[i] = std::max(zh[i], 0.0);
        }
        AS_TRY(evaluate(solved ? V.x : nullptr));
        evaluated = true;
        if (ctx->opt.verbose > 2 && solved)
            fprintf(stderr, "[sw]   step %d (ms): host %.2f, factor %.2f, solve %.2f, objective %.2f, evaluation %.2f\n",
                    outer, ms(w0, w1), ms(w1, w2), ms(w2, w3), ms(w3, w4), ms(w4, wall()));
    }
    if (!converged) {   // return the best projected iterate
        zh = zbest;
        evaluated = false;
    }
    // the returned weights are the feasible part of the last iterate
    bool clipped = false;
    for (auto& v : zh)
        if (v < 0.0) { v = 0.0; clipped = true; }
    if (clipped) evaluated = false;
    if (!evaluated) AS_TRY(evaluate());
    const bool kkt_ok = pg_rel <= ctx->opt.kkt_tol;
    int64_t support = 0;
    for (int64_t i = 0; i < N; ++i) support += zh[i] > 0.0;
    if (warm && warm->record && kkt_ok && !failed) {
        // keep the passive set and weights, and factor P0 = the support plus the zero-weight orbits
        // nearest to entering (largest g_i / |u~_i|, all below the KKT tolerance)
        warm->F0.assign(N, 0);
        warm->w0 = zh;
        std::vector<int64_t> S;
        for (int64_t i = 0; i < N; ++i)
            if (zh[i] > 0.0) { warm->F0[i] = 1; S.push_back(i); }
        std::vector<std::pair<double, int64_t>> near;
        for (int64_t i = 0; i < N; ++i)
            if (!warm->F0[i] && hh[i] > 0.0) near.push_back({gh[i] / std::sqrt(hh[i]), i});
        const int64_t extra = std::min<int64_t>(
            (int64_t)near.size(),
            std::min<int64_t>(cap - (int64_t)S.size(), (int64_t)std::ceil(warm->p0_extra * (double)S.size())));
        if (extra > 0) {
            std::partial_sort(near.begin(), near.begin() + extra, near.end(),
                              [](const std::pair<double, int64_t>& a, const std::pair<double, int64_t>& b) {
                                  return a.first > b.first;
                              });
            for (int64_t k = 0; k < extra; ++k) S.push_back(near[k].second);
        }
        std::sort(S.begin(), S.end());
        bool ok = false;
        if (!S.empty()) AS_TRY(factor(S, ok));
        warm->P0 = P0;
        warm->ld = ldG;
        warm->fl = fl_ok;
        warm->have_factor = ok;
    }
    {
        LaunchTimer lt(ctx, K_CHI2);
        k_as_chi2_finish<<<1, 1, 0, st>>>(chi, lam / (double)N, chi2_dev);
    }
    AS_CUDA(ctx, cudaGetLastError(), "chi2");
    AS_CUDA(ctx, cudaMemcpyAsync(w_dev, V.w, N * sizeof(double), cudaMemcpyDeviceToDevice, st), "weights");
    AS_CUDA(ctx, cudaStreamSynchronize(st), "active set");
    ctx->solve_info[0] = cg_total;
    ctx->solve_info[1] = n_factor;
    ctx->solve_info[2] = pg_rel;
    ctx->solve_info[3] = N > M ? 1.0 : 0.0;
    ctx->solve_info[4] = n_solves;
    ctx->solve_info[5] = kkt_ok ? 1.0 : 0.0;
    ctx->solve_info[6] = outer + 1;
    ctx->solve_info[7] = (double)support;
    if (ctx->opt.verbose)
        fprintf(stderr,
                "[sw] active set done: support %lld solves %d factors %d borders %d (masks refused %d) cg %d "
                "pg_rel %.3g%s\n",
                (long long)support, n_solves, n_factor, n_border, n_mask_refused, cg_total, pg_rel,
                converged ? "" : " (stopped)");
    if (failed) {
        set_error(ctx, "solve: reduced Gram not positive definite after ridge retries (|F| %zu)", F.size());
        return SW_ENONCONV;
    }
    if (!kkt_ok) {
        set_error(ctx, "solve: active set stopped at projected gradient %.3g of max|q| after %d solves", pg_rel,
                  n_solves);
        return SW_ENONCONV;
    }
    return SW_OK;
}

namespace {
// y_b = y + sigma xi on the observed rows r >= nd; the 3-D density rows stay as they are (Sec. 2.4)
__global__ void k_boot_data(int64_t M, int64_t nd, const double* __restrict__ y, const double* __restrict__ sig,
                            const double* __restrict__ xi, double* __restrict__ yb)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (int64_t)gridDim.x * blockDim.x)
        yb[r] = r < nd ? y[r] : y[r] + sig[r] * xi[r];
}
}  // namespace

template <typename T, typename AT, typename GT>
sw_status solve_bootstrap(sw_ctx* ctx, const sw_matrix* Um, const double* y_dev, const double* sig_dev, double lam,
                          int64_t B, const double* xi_dev, double* w_dev, double* chi2b_dev)
{
    const int64_t M = Um->M, N = Um->N;
    cudaStream_t st = ctx->stream;
    SolveWS& ws = ctx->solve_ws;
    // scratch: realisation data yb (M), weights (N), 1/sigma (M), y/sigma^2 (M), U w (M), residuals (2 M),
    // chi^2 parts (4), flag
    const size_t need = (size_t)(6 * M + N + 8) * sizeof(double);
    AS_TRY(ctx->ensure(&ws.boot, &ws.boot_cap, need, "bootstrap vectors"));
    double* yb = (double*)ws.boot;
    double* wb = yb + M;
    double* inv_sig = wb + N;
    double* ys = inv_sig + M;
    double* acc = ys + M;
    double* e = acc + M;
    double* xs = e + M;
    double* chi = xs + M;
    int* bad = (int*)(chi + 4);
    AS_CUDA(ctx, cudaMemsetAsync(chi, 0, 8 * sizeof(double), st), "memset");
    AS_CUDA(ctx, prep_data(ctx, M, sig_dev, y_dev, inv_sig, ys, bad), "prep data");
    AsWarm warm;
    warm.p0_extra = ctx->opt.boot_p0_extra;
    warm.record = true;
    sw_status worst = solve_active_set<T, AT, GT>(ctx, Um, y_dev, sig_dev, lam, wb, chi, &warm);
    if (worst != SW_OK && worst != SW_ENONCONV) return worst;
    warm.record = false;
    warm.start = true;
    int64_t solves = 0, cg = 0;
    for (int64_t b = 0; b < B; ++b) {
        {
            LaunchTimer lt(ctx, K_MISC);
            k_boot_data<<<(unsigned)std::min<int64_t>((M + 255) / 256, 4096), 256, 0, st>>>(
                M, Um->nd, y_dev, sig_dev, xi_dev + (size_t)b * M, yb);
        }
        AS_CUDA(ctx, cudaGetLastError(), "bootstrap data");
        double* wout = w_dev ? w_dev + (size_t)b * N : wb;
        sw_status s = solve_active_set<T, AT, GT>(ctx, Um, yb, sig_dev, lam, wout, chi, &warm);
        if (s != SW_OK && s != SW_ENONCONV) return s;
        if (s == SW_ENONCONV) worst = SW_ENONCONV;
        solves += (int64_t)ctx->solve_info[4];
        cg += (int64_t)ctx->solve_info[0];
        // chi2_b: the observational chi^2 of w_b against the observed data
        AS_CUDA(ctx, cudaMemsetAsync(acc, 0, M * sizeof(double), st), "memset");
        AS_CUDA(ctx, u_times_w<T>(ctx, (const T*)Um->d, M, N, wout, acc), "U w_b");
        AS_CUDA(ctx, residual(ctx, M, y_dev, acc, inv_sig, e, xs), "residual");
        AS_CUDA(ctx, cudaMemsetAsync(chi, 0, 4 * sizeof(double), st), "memset");
        AS_CUDA(ctx, chi2(ctx, M, Um->nd, e, N, wout, chi), "chi2_b");
        AS_CUDA(ctx, cudaMemcpyAsync(chi2b_dev + b, chi + 1, sizeof(double), cudaMemcpyDeviceToDevice, st),
                "chi2_b");
    }
    AS_CUDA(ctx, cudaStreamSynchronize(st), "bootstrap");
    ctx->solve_info[4] = (double)solves;
    ctx->solve_info[1] = (double)warm.factorisations;
    ctx->solve_info[0] = (double)cg;
    return worst;
}

template sw_status solve_bootstrap<float, __nv_bfloat16, float>(sw_ctx*, const sw_matrix*, const double*,
                                                                 const double*, double, int64_t, const double*,
                                                                 double*, double*);
template sw_status solve_bootstrap<float, float, float>(sw_ctx*, const sw_matrix*, const double*, const double*,
                                                        double, int64_t, const double*, double*, double*);
template sw_status solve_bootstrap<double, double, double>(sw_ctx*, const sw_matrix*, const double*, const double*,
                                                           double, int64_t, const double*, double*, double*);

template sw_status solve_active_set<float, __nv_bfloat16, float>(sw_ctx*, const sw_matrix*, const double*,
                                                                  const double*, double, double*, double*, AsWarm*);
template sw_status solve_active_set<float, float, float>(sw_ctx*, const sw_matrix*, const double*, const double*,
                                                         double, double*, double*, AsWarm*);
template sw_status solve_active_set<double, double, double>(sw_ctx*, const sw_matrix*, const double*,
                                                            const double*, double, double*, double*, AsWarm*);

}  // namespace sw
