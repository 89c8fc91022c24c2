// Weight solve of arxiv 2607.00117 Sec. 2.3: minimise
//   1/2 ||(U w - y) / sigma||^2 + (lambda / N) ||w||^2  subject to w >= 0
// (the compact NNLS form of Eq. objective_function) by ADMM, as the paper
// does: an unconstrained quadratic solve, a clip to w >= 0, and a difference
// vector carried between iterations.
//
//   U~ = diag(1/sigma) U, h_i = ||U~ e_i||^2, K = min(M, N).
//   The ADMM penalty is per orbit, P = diag(rho h_i) (the scalar-penalty
//   ADMM on the Jacobi-equilibrated problem), so with
//   Lambda = (2 lambda/N) I + P and s = Lambda^{-1/2}, A = U~ diag(s) (BF16 in
//   the FP32 form, FP64 in the plain form):
//     orbit space (N <= M):      (H~ + P)^{-1} = diag(s) (A^T A + I)^{-1} diag(s)
//     constraint space (M < N):  (H~ + P)^{-1} = diag(s) (I - A^T (A A^T + I)^{-1} A) diag(s)
//   The K x K Gram + I is factored once (blocked Cholesky) and inverted
//   (X = L^{-1}); every iteration applies X^T X with two triangular
//   matrix-vector products (plus two products with A in constraint space).
//
// ADMM iteration, over-relaxed by alpha:
//   w = (H~ + P)^{-1} (q' + P (z - u)),  w^ = alpha w + (1 - alpha) z,
//   z = max(0, w^ + u),  u += w^ - z,   H~ = s^-1 A^T A s^-1 + (2 lambda/N) I.
//
// Refinement (FP64 residuals against the stored U): with the exact negative
// gradient g = U~^T (y~ - U~ w) - (2 lambda / N) w, the next ADMM run solves
// the Gram-precision problem with q' = H~ w + g, warm-started at z = w,
// u = P^{-1} g; its fixed point satisfies the exact KKT conditions.  Rounds
// stop when the projected gradient falls below kkt_tol * max |q| or chi^2
// stops changing (chi2_tol).  Directions with little curvature (the near-null
// space of U~, held only by the 2 lambda/N regulariser) converge slowly under
// any first-order method but barely move chi^2; when the KKT tolerance is not
// met, an active-set polish finishes the job exactly: Lawson-Hanson steps on
// the support with the reduced normal equations formed in FP64 from the
// stored matrix and solved by Cholesky (supports up to polish_max orbits).
#include "sw_linalg.cuh"

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <vector>

using namespace sw;

void SolveWS::release()
{
    void* bufs[] = {A, Alo, G, Gs, X, D, vec, R, H, Hi, pv, Uc, outer, boot, Gc[0], Gc[1], gcidx, Mc};
    for (void* b : bufs)
        if (b) cudaFree(b);
    *this = SolveWS();
}

namespace {

#define CUDA_TRY(ctx, expr, what)                                  \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return (ctx)->cuda_fail(e_, what);  \
    } while (0)
#define SW_TRY(expr)                 \
    do {                             \
        sw_status s_ = (expr);       \
        if (s_ != SW_OK) return s_;  \
    } while (0)

__global__ void k_absmax(int64_t n, const double* __restrict__ a, unsigned long long* out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_chi2_finish(const double* __restrict__ in3, double lam_over_n, double* __restrict__ out3)
{
    out3[0] = in3[0];
    out3[1] = in3[1];
    out3[2] = lam_over_n * in3[2];
}

struct Carve {
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

template <typename GT>
struct Vecs {
    double *inv_sig, *ys, *acc, *e, *xs, *q, *wd, *ute, *gneg, *chi, *trace, *h, *s64;
    unsigned long long *pgmax, *qmax;
    int *info, *bad, *err;
    unsigned* stats;
    GT *qp, *z, *u, *r, *wv, *v, *t, *t1, *t2, *t3, *tmpM, *wg, *sg, *rho_i, *dg, *zbest;
    double* y;
    double* sig;
    size_t carve(char* base, int64_t M, int64_t N, int64_t K)
    {
        Carve c{base};
        inv_sig = c.take<double>(M); ys = c.take<double>(M); acc = c.take<double>(M); e = c.take<double>(M);
        xs = c.take<double>(M); y = c.take<double>(M); sig = c.take<double>(M);
        q = c.take<double>(N); wd = c.take<double>(N); ute = c.take<double>(N); gneg = c.take<double>(N);
        h = c.take<double>(N); s64 = c.take<double>(N);
        chi = c.take<double>(4); trace = c.take<double>(1);
        pgmax = c.take<unsigned long long>(1); qmax = c.take<unsigned long long>(1);
        info = c.take<int>(1); bad = c.take<int>(1); err = c.take<int>(1);
        stats = c.take<unsigned>(4);
        qp = c.take<GT>(N); z = c.take<GT>(N); u = c.take<GT>(N); r = c.take<GT>(N); wv = c.take<GT>(N);
        v = c.take<GT>(N); t = c.take<GT>(N); wg = c.take<GT>(N);
        sg = c.take<GT>(N); rho_i = c.take<GT>(N); dg = c.take<GT>(N); zbest = c.take<GT>(N);
        t1 = c.take<GT>(K); t2 = c.take<GT>(K); t3 = c.take<GT>(K); tmpM = c.take<GT>(M);
        return c.used + 256;
    }
};

inline int64_t pad64(int64_t n) { return (n + 63) / 64 * 64; }

// The weight problem on an orbit-major matrix U (M rows, N orbits, the first
// nd rows being density cells).  n_reg is the orbit count of the regulariser
// (lambda / n_reg) ||w||^2 -- the full library size when U holds a working set.
struct Problem {
    const void* U;
    int64_t M, N, nd;
    double n_reg;
    bool force_orbit;
};

template <typename T, typename AT, typename GT>
sw_status solve_impl(sw_ctx* ctx, const Problem& pb, const double* y_dev, const double* sig_dev, double lam,
                     double* w_dev, double* chi2_dev, const double* w0 = nullptr)
{
    const int64_t M = pb.M, N = pb.N;
    const bool orbit = pb.force_orbit || N <= M;
    const int64_t K = orbit ? N : M;
    const int64_t ldA = orbit ? pad64(M) : pad64(N);
    const int64_t Arows = orbit ? N : M;
    const T* U = (const T*)pb.U;
    const bool split = sizeof(AT) == 2;   // BF16 operand stored as hi + lo halves
    cudaStream_t st = ctx->stream;
    SolveWS& ws = ctx->solve_ws;
    Vecs<GT> V{};
    size_t vec_bytes = V.carve(nullptr, M, N, K);
    SW_TRY(ctx->ensure(&ws.vec, &ws.vec_cap, vec_bytes, "solve vectors"));
    V.carve((char*)ws.vec, M, N, K);
    SW_TRY(ctx->ensure(&ws.A, &ws.A_cap, (size_t)Arows * ldA * sizeof(AT), "whitened matrix"));
    if (split) SW_TRY(ctx->ensure(&ws.Alo, &ws.Alo_cap, (size_t)Arows * ldA * sizeof(AT), "whitened matrix (lo)"));
    SW_TRY(ctx->ensure(&ws.G, &ws.G_cap, (size_t)K * K * sizeof(GT), "Gram"));
    SW_TRY(ctx->ensure(&ws.X, &ws.X_cap, (size_t)K * K * sizeof(GT), "inverse factor"));
    SW_TRY(ctx->ensure(&ws.D, &ws.D_cap, 64 * 64 * sizeof(GT), "block scratch"));
    AT* A = (AT*)ws.A;
    AT* Alo = split ? (AT*)ws.Alo : nullptr;
    GT* G = (GT*)ws.G;
    GT* X = (GT*)ws.X;
    GT* D = (GT*)ws.D;

    CUDA_TRY(ctx, cudaMemsetAsync(V.chi, 0, 256 * 3, st), "memset");  // chi, trace, pgmax, qmax, flags
    CUDA_TRY(ctx, cudaMemsetAsync(V.info, 0, sizeof(int), st), "memset");
    CUDA_TRY(ctx, cudaMemsetAsync(V.bad, 0, sizeof(int), st), "memset");
    CUDA_TRY(ctx, cudaMemsetAsync(V.err, 0, sizeof(int), st), "memset");
    CUDA_TRY(ctx, cudaMemsetAsync(V.trace, 0, sizeof(double), st), "memset");
    CUDA_TRY(ctx, cudaMemsetAsync(V.qmax, 0, sizeof(unsigned long long), st), "memset");
    // ---- data: 1/sigma and y/sigma^2; q = U~^T y~ exactly (FP64 accumulation)
    CUDA_TRY(ctx, prep_data(ctx, M, sig_dev, y_dev, V.inv_sig, V.ys, V.bad), "prep data");
    CUDA_TRY(ctx, ut_times_x<T>(ctx, U, M, N, V.ys, V.q), "q");
    {
        LaunchTimer lt(ctx, K_MISC);
        k_absmax<<<64, 256, 0, st>>>(N, V.q, V.qmax);
    }
    // ---- per-orbit ADMM penalty rho_i = rho ||U~ e_i||^2 and column scale
    // s_i = (2 lam/N + rho_i)^{-1/2}: with A = U~ diag(s) the ADMM matrix is
    // H~ + P = diag(1/s) (A^T A + I) diag(1/s) (orbit space) and, by Woodbury,
    // (H~ + P)^{-1} = diag(s) (I - A^T (A A^T + I)^{-1} A) diag(s) (constraint space).
    const double two_lam_n = 2.0 * lam / pb.n_reg;
    const double rho = orbit ? ctx->opt.admm_rho : ctx->opt.admm_rho_cs;
    CUDA_TRY(ctx, colnorm2<T>(ctx, U, M, N, V.inv_sig, V.h), "column norms");
    CUDA_TRY(ctx, admm_scales<GT>(ctx, N, V.h, two_lam_n, rho, 0.0, V.s64, V.sg, V.rho_i, V.dg), "scales");
    // ---- whitening, Gram, unit shift, Cholesky, inverse
    CUDA_TRY(ctx, (whiten<T, AT>(ctx, U, M, N, V.inv_sig, V.s64, A, Alo, ldA, orbit)), "whiten");
    if constexpr (sizeof(AT) == 2) {
        CUDA_TRY(ctx, gram_tc(ctx, A, Alo, K, ldA, (float*)G, V.err), "tensor-core Gram");
    } else {
        CUDA_TRY(ctx, (gemm<GT, true, true>(ctx, K_GRAM_SIMT, K, K, ldA, GT(1), (const GT*)A, ldA, (const GT*)A, ldA,
                                            GT(0), G, K, 0)),
                 "Gram");
    }
    double qmax_d = 0.0;
    int bad = 0, gerr = 0;
    unsigned long long qbits = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&qbits, V.qmax, 8, cudaMemcpyDeviceToHost, st), "qmax");
    CUDA_TRY(ctx, cudaMemcpyAsync(&bad, V.bad, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
    CUDA_TRY(ctx, cudaMemcpyAsync(&gerr, V.err, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "solve setup");
    memcpy(&qmax_d, &qbits, 8);
    if (bad) { set_error(ctx, "solve: errors must be positive and finite, data finite"); return SW_EINVAL; }
    if (gerr) { set_error(ctx, "solve: tensor-core Gram kernel timed out"); return SW_ETIMEOUT; }
    CUDA_TRY(ctx, shift_and_trace<GT>(ctx, G, K, nullptr, 1.0), "shift");
    // keep a symmetric copy of G + I: every ADMM step is refined against it, which makes
    // the step consistent with the Gram even where the FP32 factor is not accurate
    const int inner_refine = orbit ? ctx->opt.inner_refine : 0;
    GT* Gs = nullptr;
    if (inner_refine > 0) {
        SW_TRY(ctx->ensure(&ws.Gs, &ws.Gs_cap, (size_t)K * K * sizeof(GT), "Gram copy"));
        Gs = (GT*)ws.Gs;
        CUDA_TRY(ctx, symmetrize<GT>(ctx, G, K, Gs), "symmetrize");
    }
    CUDA_TRY(ctx, cholesky_inverse<GT>(ctx, G, X, D, K, V.info), "Cholesky and inverse");
    int info = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&info, V.info, sizeof(int), cudaMemcpyDeviceToHost, st), "info");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "factorisation");
    if (info) { set_error(ctx, "solve: shifted Gram not positive definite at pivot %d", info - 1); return SW_ENONCONV; }

    // ---- ADMM: apply the inverse to the scaled right-hand side rs
    auto apply = [&](const GT* rs) -> cudaError_t {
        cudaError_t e;
        if (orbit) {   // y = (G + I)^{-1} rs by X^T X and refinement against G + I, w = s o y
            if ((e = rowdot<GT, GT, GT, GT>(ctx, K_TRMV_L, X, K, K, K, rs, V.t1, 1.0, 0.0, true))) return e;
            if ((e = cudaMemsetAsync(V.wv, 0, K * sizeof(GT), st))) return e;
            if ((e = colcomb<GT, GT, GT, GT>(ctx, K_TRMV_LT, X, K, K, K, V.t1, V.wv, 1.0, true))) return e;
            for (int k = 0; k < inner_refine; ++k) {
                if ((e = cudaMemcpyAsync(V.t2, rs, K * sizeof(GT), cudaMemcpyDeviceToDevice, st))) return e;
                if ((e = rowdot<GT, GT, GT, double>(ctx, K_GEMV_N, Gs, K, K, K, V.wv, V.t2, -1.0, 1.0, false)))
                    return e;
                if ((e = rowdot<GT, GT, GT, GT>(ctx, K_TRMV_L, X, K, K, K, V.t2, V.t1, 1.0, 0.0, true))) return e;
                if ((e = colcomb<GT, GT, GT, GT>(ctx, K_TRMV_LT, X, K, K, K, V.t1, V.wv, 1.0, true))) return e;
            }
            return cudaSuccess;
        }
        // v = A^T X^T X A rs, w = s o (rs - v)
        if ((e = rowdot<AT, GT, GT, GT>(ctx, K_GEMV_N, A, M, N, ldA, rs, V.t1, 1.0, 0.0, false, Alo))) return e;
        if ((e = rowdot<GT, GT, GT, GT>(ctx, K_TRMV_L, X, K, K, K, V.t1, V.t2, 1.0, 0.0, true))) return e;
        if ((e = cudaMemsetAsync(V.t3, 0, K * sizeof(GT), st))) return e;
        if ((e = colcomb<GT, GT, GT, GT>(ctx, K_TRMV_LT, X, K, K, K, V.t2, V.t3, 1.0, true))) return e;
        if ((e = cudaMemsetAsync(V.v, 0, N * sizeof(GT), st))) return e;
        return colcomb<AT, GT, GT, GT>(ctx, K_GEMV_T, A, M, N, ldA, V.t3, V.v, 1.0, false, Alo);
    };
    int total_iter = 0;
    auto run_admm = [&](bool& converged) -> sw_status {
        converged = false;
        std::vector<double> hist;
        CUDA_TRY(ctx, admm_init<GT>(ctx, N, V.qp, V.z, V.u, V.sg, V.rho_i, V.r), "ADMM init");
        for (int it = 1; it <= ctx->opt.admm_max_iter; ++it) {
            CUDA_TRY(ctx, apply(V.r), "ADMM solve");
            const bool check = (it % ctx->opt.check_every) == 0 || it == ctx->opt.admm_max_iter;
            if (check) CUDA_TRY(ctx, cudaMemsetAsync(V.stats, 0, 4 * sizeof(unsigned), st), "memset");
            CUDA_TRY(ctx, admm_update<GT>(ctx, N, orbit ? V.wv : nullptr, orbit ? nullptr : V.v, V.sg, V.rho_i, V.dg,
                                          V.qp, ctx->opt.admm_alpha, V.r, V.z, V.u, check ? V.stats : nullptr),
                     "ADMM update");
            ++total_iter;
            if (check) {
                unsigned sv[4];
                CUDA_TRY(ctx, cudaMemcpyAsync(sv, V.stats, sizeof(sv), cudaMemcpyDeviceToHost, st), "stats");
                CUDA_TRY(ctx, cudaStreamSynchronize(st), "ADMM");
                float pr, du, zm;
                memcpy(&pr, &sv[0], 4); memcpy(&du, &sv[1], 4); memcpy(&zm, &sv[2], 4);
                const double scale = ctx->opt.admm_tol * std::max(1.0, (double)zm);
                if (!std::isfinite(pr) || !std::isfinite(zm)) { set_error(ctx, "ADMM diverged"); return SW_ENONCONV; }
                if (pr <= scale && du <= scale) { converged = true; break; }
                // stagnation: the residual has not halved over the last 5 checks
                const double res = std::max((double)pr, (double)du);
                hist.push_back(res);
                if (hist.size() > 5 && res > 0.5 * hist[hist.size() - 6]) break;
            }
        }
        return SW_OK;
    };
    // first run: q' = q, z = u = 0
    CUDA_TRY(ctx, (convert<double, GT>(ctx, N, V.q, V.qp)), "q'");
    if (w0) CUDA_TRY(ctx, (convert<double, GT>(ctx, N, w0, V.z)), "warm start");   // w0 may alias w_dev
    else CUDA_TRY(ctx, cudaMemsetAsync(V.z, 0, N * sizeof(GT), st), "memset");
    CUDA_TRY(ctx, cudaMemsetAsync(V.u, 0, N * sizeof(GT), st), "memset");
    bool conv = false;
    SW_TRY(run_admm(conv));

    // ---- exact state of an iterate held in V.wd: e = (y - U w)/sigma, U~^T e,
    // negative gradient g, projected-gradient norm and chi^2 parts (all FP64)
    auto evaluate = [&](double& pg_rel_out, double chi[3]) -> sw_status {
        CUDA_TRY(ctx, cudaMemsetAsync(V.acc, 0, M * sizeof(double), st), "memset");
        CUDA_TRY(ctx, u_times_w<T>(ctx, U, M, N, V.wd, V.acc), "U w");
        CUDA_TRY(ctx, residual(ctx, M, y_dev, V.acc, V.inv_sig, V.e, V.xs), "residual");
        CUDA_TRY(ctx, ut_times_x<T>(ctx, U, M, N, V.xs, V.ute), "U^T e");
        CUDA_TRY(ctx, cudaMemsetAsync(V.pgmax, 0, 8, st), "memset");
        CUDA_TRY(ctx, kkt(ctx, N, V.ute, V.wd, two_lam_n, V.gneg, V.pgmax), "KKT");
        CUDA_TRY(ctx, cudaMemsetAsync(V.chi, 0, 4 * sizeof(double), st), "memset");
        CUDA_TRY(ctx, chi2(ctx, M, pb.nd, V.e, N, V.wd, V.chi), "chi2");
        unsigned long long pb = 0;
        double c3[4];
        CUDA_TRY(ctx, cudaMemcpyAsync(&pb, V.pgmax, 8, cudaMemcpyDeviceToHost, st), "KKT");
        CUDA_TRY(ctx, cudaMemcpyAsync(c3, V.chi, 4 * sizeof(double), cudaMemcpyDeviceToHost, st), "chi2");
        CUDA_TRY(ctx, cudaStreamSynchronize(st), "KKT");
        double pg;
        memcpy(&pg, &pb, 8);
        pg_rel_out = pg / std::max(qmax_d, 1e-300);
        chi[0] = c3[0]; chi[1] = c3[1]; chi[2] = c3[2];
        return SW_OK;
    };

    // ---- refinement with FP64 residuals from the stored matrix
    int rounds = 0, polish_iters = 0;
    double pg_rel = 0.0, chi[3] = {0, 0, 0}, chi_prev = -1.0;
    bool kkt_ok = false, chi_stable = false;
    double f_best = 1e300;
    for (;;) {
        CUDA_TRY(ctx, (convert<GT, double>(ctx, N, V.z, V.wd)), "w");
        SW_TRY(evaluate(pg_rel, chi));
        const double f = 0.5 * chi[0] + lam / pb.n_reg * chi[2];   // the exact objective Q(w)
        if (ctx->opt.verbose)
            fprintf(stderr, "[sw]   core round %d: N %lld K %lld chi2 %.9g Q %.9g pg_rel %.3g admm %d\n", rounds,
                    (long long)N, (long long)K, chi[0], f, pg_rel, total_iter);
        if (pg_rel <= ctx->opt.kkt_tol) { kkt_ok = true; break; }
        if (!(f <= f_best)) {
            // a refinement round that raises the exact objective means the Gram-precision
            // problem is too far from the exact one here: return to the best iterate and stop
            CUDA_TRY(ctx, cudaMemcpyAsync(V.z, V.zbest, N * sizeof(GT), cudaMemcpyDeviceToDevice, st), "revert");
            CUDA_TRY(ctx, (convert<GT, double>(ctx, N, V.z, V.wd)), "w");
            SW_TRY(evaluate(pg_rel, chi));
            break;
        }
        f_best = f;
        CUDA_TRY(ctx, cudaMemcpyAsync(V.zbest, V.z, N * sizeof(GT), cudaMemcpyDeviceToDevice, st), "best");
        if (chi_prev >= 0.0 && std::fabs(chi[0] - chi_prev) <= ctx->opt.chi2_tol * std::max(chi[0], 1e-300)) {
            chi_stable = true;
            break;
        }
        chi_prev = chi[0];
        if (rounds >= ctx->opt.refine_max) break;
        ++rounds;
        // q' = H~_data w + U~^T e, with H~_data w = (A^T A (w / s)) / s in the Gram precision
        CUDA_TRY(ctx, div_to<GT>(ctx, N, V.wd, V.s64, V.wg), "w / s");
        if (orbit) {
            CUDA_TRY(ctx, cudaMemsetAsync(V.tmpM, 0, M * sizeof(GT), st), "memset");
            CUDA_TRY(ctx, (colcomb<AT, GT, GT, GT>(ctx, K_GEMV_T, A, N, M, ldA, V.wg, V.tmpM, 1.0, false, Alo)), "A w");
            CUDA_TRY(ctx, (rowdot<AT, GT, GT, GT>(ctx, K_GEMV_N, A, N, M, ldA, V.tmpM, V.t, 1.0, 0.0, false, Alo)), "A^T A w");
        } else {
            CUDA_TRY(ctx, (rowdot<AT, GT, GT, GT>(ctx, K_GEMV_N, A, M, N, ldA, V.wg, V.tmpM, 1.0, 0.0, false, Alo)), "A w");
            CUDA_TRY(ctx, cudaMemsetAsync(V.t, 0, N * sizeof(GT), st), "memset");
            CUDA_TRY(ctx, (colcomb<AT, GT, GT, GT>(ctx, K_GEMV_T, A, M, N, ldA, V.tmpM, V.t, 1.0, false, Alo)), "A^T A w");
        }
        CUDA_TRY(ctx, refine_rhs<GT>(ctx, N, V.t, V.gneg, V.wd, V.s64, two_lam_n, V.rho_i, V.qp, V.z, V.u),
                 "refine rhs");
        SW_TRY(run_admm(conv));
    }

    // ---- active-set polish (Lawson-Hanson steps on the support, FP64): the
    // reduced normal equations (U~_P^T U~_P + 2 lambda/N I) x = q_P are formed
    // from the stored matrix and solved by Cholesky; infeasible solutions step
    // back to the boundary and drop variables; KKT violators join the support.
    if (!kkt_ok && ctx->opt.polish_max > 0) {
        std::vector<double> zh(N), xh, gh(N);
        CUDA_TRY(ctx, cudaMemcpyAsync(zh.data(), V.wd, N * sizeof(double), cudaMemcpyDeviceToHost, st), "polish");
        CUDA_TRY(ctx, cudaStreamSynchronize(st), "polish");
        std::vector<char> inP(N, 0);
        for (int64_t i = 0; i < N; ++i) inP[i] = zh[i] > 0.0;
        const double gtol = ctx->opt.kkt_tol * qmax_d;
        bool single_add = false, failed = false, polished_stable = false;
        std::vector<double> last_z;
        for (int outer = 0; outer < 64 && !failed; ++outer) {
            for (int inner = 0; inner < 200 && polish_iters < ctx->opt.polish_solves; ++inner) {
                std::vector<int64_t> P;
                for (int64_t i = 0; i < N; ++i)
                    if (inP[i]) P.push_back(i);
                const int64_t nP = (int64_t)P.size();
                if (nP == 0) break;
                if (nP > ctx->opt.polish_max) { failed = true; break; }
                SW_TRY(ctx->ensure(&ws.R, &ws.R_cap, (size_t)nP * M * sizeof(double), "polish rows"));
                SW_TRY(ctx->ensure(&ws.H, &ws.H_cap, (size_t)nP * nP * sizeof(double), "polish matrix"));
                SW_TRY(ctx->ensure(&ws.Hi, &ws.Hi_cap, (size_t)nP * nP * sizeof(double), "polish inverse"));
                SW_TRY(ctx->ensure(&ws.pv, &ws.pv_cap, (size_t)nP * (8 + 3 * 8) + 64 * 64 * 8 + 1024, "polish vectors"));
                int64_t* didx = (int64_t*)ws.pv;
                double* qP = (double*)(didx + nP);
                double* tP = qP + nP;
                double* xP = tP + nP;
                double* Dd = xP + nP;
                double* R = (double*)ws.R;
                double* Hm = (double*)ws.H;
                double* Hi = (double*)ws.Hi;
                CUDA_TRY(ctx, cudaMemcpyAsync(didx, P.data(), nP * sizeof(int64_t), cudaMemcpyHostToDevice, st), "idx");
                CUDA_TRY(ctx, cudaMemsetAsync(V.info, 0, sizeof(int), st), "memset");
                CUDA_TRY(ctx, gather_rows<T>(ctx, U, M, didx, nP, V.inv_sig, R), "gather");
                CUDA_TRY(ctx, (gemm<double, true, true>(ctx, K_GRAM_SIMT, nP, nP, M, 1.0, R, M, R, M, 0.0, Hm, nP, 0)),
                         "reduced Gram");
                // lambda = 0 leaves the reduced system singular when the support exceeds the rank;
                // a ridge of 1e-11 of the mean diagonal keeps it factorable (no effect on chi^2 at FP64)
                CUDA_TRY(ctx, cudaMemsetAsync(V.trace, 0, sizeof(double), st), "memset");
                CUDA_TRY(ctx, shift_and_trace<double>(ctx, Hm, nP, V.trace, 0.0), "trace");
                double trH = 0.0;
                CUDA_TRY(ctx, cudaMemcpyAsync(&trH, V.trace, sizeof(double), cudaMemcpyDeviceToHost, st), "trace");
                CUDA_TRY(ctx, cudaStreamSynchronize(st), "trace");
                const double ridge = std::max(two_lam_n, 1e-11 * trH / (double)nP);
                CUDA_TRY(ctx, shift_and_trace<double>(ctx, Hm, nP, nullptr, ridge), "shift");
                CUDA_TRY(ctx, cholesky_inverse<double>(ctx, Hm, Hi, Dd, nP, V.info), "reduced Cholesky");
                CUDA_TRY(ctx, gather_vec(ctx, V.q, didx, nP, qP), "q_P");
                CUDA_TRY(ctx, (rowdot<double, double, double, double>(ctx, K_TRMV_L, Hi, nP, nP, nP, qP, tP, 1.0, 0.0,
                                                                      true)), "solve");
                CUDA_TRY(ctx, cudaMemsetAsync(xP, 0, nP * sizeof(double), st), "memset");
                CUDA_TRY(ctx, (colcomb<double, double, double, double>(ctx, K_TRMV_LT, Hi, nP, nP, nP, tP, xP, 1.0,
                                                                       true)), "solve");
                xh.resize(nP);
                int info = 0;
                CUDA_TRY(ctx, cudaMemcpyAsync(xh.data(), xP, nP * sizeof(double), cudaMemcpyDeviceToHost, st), "x");
                CUDA_TRY(ctx, cudaMemcpyAsync(&info, V.info, sizeof(int), cudaMemcpyDeviceToHost, st), "info");
                CUDA_TRY(ctx, cudaStreamSynchronize(st), "polish");
                ++polish_iters;
                if (info) { failed = true; break; }
                double alpha = 1.0;
                bool feasible = true;
                for (int64_t k = 0; k < nP; ++k) {
                    if (!(xh[k] > 0.0)) {
                        feasible = false;
                        const double zk = zh[P[k]];
                        const double a = zk > 0.0 ? zk / (zk - xh[k]) : 0.0;
                        alpha = std::min(alpha, a);
                    }
                }
                if (feasible) {
                    for (int64_t k = 0; k < nP; ++k) zh[P[k]] = xh[k];
                    break;
                }
                for (int64_t k = 0; k < nP; ++k) {
                    double& zk = zh[P[k]];
                    zk = zk + alpha * (xh[k] - zk);
                    if (!(zk > 1e-300) || !(xh[k] > 0.0 || zk > 0.0)) { zk = 0.0; }
                    if (zk <= 0.0) inP[P[k]] = 0;
                }
            }
            if (failed) break;
            for (int64_t i = 0; i < N; ++i)
                if (!inP[i]) zh[i] = 0.0;
            CUDA_TRY(ctx, cudaMemcpyAsync(V.wd, zh.data(), N * sizeof(double), cudaMemcpyHostToDevice, st), "w");
            const double chi_before = chi[0];
            SW_TRY(evaluate(pg_rel, chi));
            if (pg_rel <= ctx->opt.kkt_tol) { kkt_ok = true; break; }
            if (std::fabs(chi[0] - chi_before) <= ctx->opt.chi2_tol * std::max(chi[0], 1e-300) && outer > 0) {
                polished_stable = true;
                break;
            }
            if (polish_iters >= ctx->opt.polish_solves) break;
            // KKT violators: g_i = -grad_i > tol at w_i = 0
            CUDA_TRY(ctx, cudaMemcpyAsync(gh.data(), V.gneg, N * sizeof(double), cudaMemcpyDeviceToHost, st), "g");
            CUDA_TRY(ctx, cudaStreamSynchronize(st), "g");
            const bool stalled = !last_z.empty() && last_z == zh;
            if (stalled) single_add = true;
            last_z = zh;
            int64_t best = -1;
            int added = 0;
            for (int64_t i = 0; i < N; ++i) {
                if (inP[i] || !(gh[i] > gtol)) continue;
                if (single_add) {
                    if (best < 0 || gh[i] > gh[best]) best = i;
                } else {
                    inP[i] = 1;
                    ++added;
                }
            }
            if (single_add && best >= 0) { inP[best] = 1; ++added; }
            if (!added) break;
        }
        // keep the polished iterate unless the polish gave up part-way
        if (polished_stable) chi_stable = true;
        if (!kkt_ok && (failed || !polished_stable)) {
            CUDA_TRY(ctx, (convert<GT, double>(ctx, N, V.z, V.wd)), "w");
            SW_TRY(evaluate(pg_rel, chi));
        }
    }
    // ---- outputs: chi^2 parts of the final weights, weights
    {
        LaunchTimer lt(ctx, K_CHI2);
        k_chi2_finish<<<1, 1, 0, st>>>(V.chi, lam / pb.n_reg, chi2_dev);
    }
    CUDA_TRY(ctx, cudaGetLastError(), "chi2");
    CUDA_TRY(ctx, cudaMemcpyAsync(w_dev, V.wd, N * sizeof(double), cudaMemcpyDeviceToDevice, st), "weights");
    ctx->solve_info[0] = total_iter;
    ctx->solve_info[1] = rounds;
    ctx->solve_info[2] = pg_rel;
    ctx->solve_info[3] = N > M ? 1.0 : 0.0;
    ctx->solve_info[4] = polish_iters;
    ctx->solve_info[6] = 0.0;
    ctx->solve_info[7] = 0.0;
    ctx->solve_info[5] = kkt_ok ? 1.0 : 0.0;
    if (!kkt_ok && !chi_stable) {
        set_error(ctx, "solve: neither the KKT tolerance (projected gradient %.3g of max|q|) nor a stable chi^2 was "
                       "reached after %d refinement rounds", pg_rel, rounds);
        return SW_ENONCONV;
    }
    return SW_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Working set for N > M.  The non-negative minimiser has at most about rank(U)
// = M positive weights (exactly so at lambda = 0), so the orbit-space solve --
// free of the digit cancellation of the Woodbury form -- runs on a working set
// C of ws_factor * M orbits: first the orbits best correlated with the data
// (q_i / ||U~ e_i||), then, round by round, the support of the last solution
// plus the strongest violators of the exact KKT conditions over all N orbits
// (negative gradient g_i > kkt_tol max|q| at w_i = 0).  The solution is exact
// when no orbit outside C violates the conditions.
// ---------------------------------------------------------------------------
template <typename T, typename AT, typename GT>
static sw_status solve_working_set(sw_ctx* ctx, const sw_matrix* Um, const double* y_dev, const double* sig_dev,
                                   double lam, double* w_dev, double* chi2_dev)
{
    const int64_t M = Um->M, N = Um->N;
    const T* U = (const T*)Um->d;
    cudaStream_t st = ctx->stream;
    SolveWS& ws = ctx->solve_ws;
    int64_t nC = std::min<int64_t>(N, (int64_t)std::ceil(ctx->opt.ws_factor * (double)M));
    const int64_t nC_max = std::min<int64_t>(N, 3 * nC);
    // outer vectors: inv_sig, ys, acc, e, xs (M); q, h, w, ute, gneg (N); wC (nC_max); idx; scalars
    Carve c{nullptr};
    auto carve = [&](char* base, double** o) {
        c = Carve{base};
        for (int k = 0; k < 5; ++k) o[k] = c.take<double>(M);
        for (int k = 5; k < 10; ++k) o[k] = c.take<double>(N);
        o[10] = c.take<double>(nC_max);
        o[11] = (double*)c.take<int64_t>(nC_max);
        o[12] = c.take<double>(8);
        return c.used + 256;
    };
    double* o[13];
    const size_t need = carve(nullptr, o);
    SW_TRY(ctx->ensure(&ws.outer, &ws.outer_cap, need, "working-set vectors"));
    carve((char*)ws.outer, o);
    double *inv_sig = o[0], *ys = o[1], *acc = o[2], *e = o[3], *xs = o[4];
    double *q = o[5], *h = o[6], *w = o[7], *ute = o[8], *gneg = o[9], *wC = o[10], *scal = o[12];
    int64_t* didx = (int64_t*)o[11];
    int* bad = (int*)(scal + 4);
    unsigned long long* pgmax = (unsigned long long*)(scal + 5);
    unsigned long long* qmax = (unsigned long long*)(scal + 6);
    const double two_lam_n = 2.0 * lam / (double)N;

    CUDA_TRY(ctx, cudaMemsetAsync(scal, 0, 8 * sizeof(double), st), "memset");
    CUDA_TRY(ctx, prep_data(ctx, M, sig_dev, y_dev, inv_sig, ys, bad), "prep data");
    CUDA_TRY(ctx, ut_times_x<T>(ctx, U, M, N, ys, q), "q");
    CUDA_TRY(ctx, colnorm2<T>(ctx, U, M, N, inv_sig, h), "column norms");
    {
        LaunchTimer lt(ctx, K_MISC);
        k_absmax<<<64, 256, 0, st>>>(N, q, qmax);
    }
    std::vector<double> qh(N), hh(N), gh(N), wh(nC_max);
    int badh = 0;
    unsigned long long qb = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(qh.data(), q, N * sizeof(double), cudaMemcpyDeviceToHost, st), "q");
    CUDA_TRY(ctx, cudaMemcpyAsync(hh.data(), h, N * sizeof(double), cudaMemcpyDeviceToHost, st), "h");
    CUDA_TRY(ctx, cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
    CUDA_TRY(ctx, cudaMemcpyAsync(&qb, qmax, 8, cudaMemcpyDeviceToHost, st), "qmax");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "working set");
    if (badh) { set_error(ctx, "solve: errors must be positive and finite, data finite"); return SW_EINVAL; }
    double qmax_d;
    memcpy(&qmax_d, &qb, 8);
    const double gtol = ctx->opt.kkt_tol * std::max(qmax_d, 1e-300);

    // initial working set: best correlated orbits
    std::vector<int64_t> order(N);
    for (int64_t i = 0; i < N; ++i) order[i] = i;
    auto score = [&](int64_t i, const std::vector<double>& g) {
        return hh[i] > 0.0 ? g[i] / std::sqrt(hh[i]) : -1e300;
    };
    std::partial_sort(order.begin(), order.begin() + nC, order.end(),
                      [&](int64_t a, int64_t b) { return score(a, qh) > score(b, qh); });
    std::vector<int64_t> C(order.begin(), order.begin() + nC);
    std::vector<char> inC(N, 0);

    sw_status core = SW_OK;
    double pg_rel = 0.0, chi_prev = -1.0, chi_now = 0.0;
    bool done = false;
    int rounds = 0;
    double inner_info[6] = {0, 0, 0, 0, 0, 0};
    for (; rounds < ctx->opt.ws_rounds && !done; ++rounds) {
        std::sort(C.begin(), C.end());
        nC = (int64_t)C.size();
        std::fill(inC.begin(), inC.end(), 0);
        for (int64_t i : C) inC[i] = 1;
        SW_TRY(ctx->ensure(&ws.Uc, &ws.Uc_cap, (size_t)nC * M * sizeof(T), "working-set columns"));
        CUDA_TRY(ctx, cudaMemcpyAsync(didx, C.data(), nC * sizeof(int64_t), cudaMemcpyHostToDevice, st), "idx");
        CUDA_TRY(ctx, gather_cols<T>(ctx, U, M, didx, nC, (T*)ws.Uc), "gather");
        Problem pb{ws.Uc, M, nC, Um->nd, (double)N, true};
        if (rounds > 0) CUDA_TRY(ctx, gather_vec(ctx, w, didx, nC, wC), "warm start");
        core = solve_impl<T, AT, GT>(ctx, pb, y_dev, sig_dev, lam, wC, scal, rounds > 0 ? wC : nullptr);
        if (core != SW_OK && core != SW_ENONCONV) return core;
        for (int k = 0; k < 6; ++k) inner_info[k] += (k == 2 || k == 3 || k == 5) ? 0.0 : ctx->solve_info[k];
        inner_info[2] = ctx->solve_info[2];
        // exact state over all N orbits
        CUDA_TRY(ctx, cudaMemsetAsync(w, 0, N * sizeof(double), st), "memset");
        CUDA_TRY(ctx, scatter_vec(ctx, wC, didx, nC, w), "scatter");
        CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, M * sizeof(double), st), "memset");
        CUDA_TRY(ctx, u_times_w<T>(ctx, U, M, N, w, acc), "U w");
        CUDA_TRY(ctx, residual(ctx, M, y_dev, acc, inv_sig, e, xs), "residual");
        CUDA_TRY(ctx, ut_times_x<T>(ctx, U, M, N, xs, ute), "U^T e");
        CUDA_TRY(ctx, cudaMemsetAsync(pgmax, 0, 8, st), "memset");
        CUDA_TRY(ctx, kkt(ctx, N, ute, w, two_lam_n, gneg, pgmax), "KKT");
        unsigned long long pb_bits = 0;
        double chi_dev[3];
        CUDA_TRY(ctx, cudaMemcpyAsync(&pb_bits, pgmax, 8, cudaMemcpyDeviceToHost, st), "KKT");
        CUDA_TRY(ctx, cudaMemcpyAsync(chi_dev, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "chi2");
        CUDA_TRY(ctx, cudaMemcpyAsync(gh.data(), gneg, N * sizeof(double), cudaMemcpyDeviceToHost, st), "g");
        CUDA_TRY(ctx, cudaMemcpyAsync(wh.data(), wC, nC * sizeof(double), cudaMemcpyDeviceToHost, st), "w");
        CUDA_TRY(ctx, cudaStreamSynchronize(st), "working set");
        double pg;
        memcpy(&pg, &pb_bits, 8);
        pg_rel = pg / std::max(qmax_d, 1e-300);
        chi_now = chi_dev[0];
        if (ctx->opt.verbose) {
            int64_t nsup = 0, nviol = 0, nposq = 0;
            for (int64_t k = 0; k < nC; ++k) nsup += wh[k] > 0.0;
            for (int64_t i = 0; i < N; ++i) { nviol += (!inC[i] && gh[i] > gtol); nposq += qh[i] > gtol; }
            fprintf(stderr, "[sw] ws round %d: |C| %lld core %d chi2 %.9g pg_rel %.3g support %lld violators %lld "
                            "q>tol %lld inner admm %g refine %g polish %g\n", rounds, (long long)nC, (int)core,
                    chi_now, pg_rel, (long long)nsup, (long long)nviol, (long long)nposq, ctx->solve_info[0],
                    ctx->solve_info[1], ctx->solve_info[4]);
        }
        // violators outside C, strongest first
        std::vector<int64_t> viol;
        for (int64_t i = 0; i < N; ++i)
            if (!inC[i] && gh[i] > gtol) viol.push_back(i);
        if (viol.empty() || pg_rel <= ctx->opt.kkt_tol) { done = true; break; }
        if (chi_prev >= 0.0 && std::fabs(chi_now - chi_prev) <= ctx->opt.chi2_tol * std::max(chi_now, 1e-300)) {
            done = true;
            break;
        }
        chi_prev = chi_now;
        std::sort(viol.begin(), viol.end(), [&](int64_t a, int64_t b) { return score(a, gh) > score(b, gh); });
        std::vector<int64_t> next;
        for (int64_t k = 0; k < nC; ++k)
            if (wh[k] > 0.0) next.push_back(C[k]);
        const int64_t cap = std::min<int64_t>(nC_max, std::max<int64_t>((int64_t)C.size(),
                                                                       (int64_t)(next.size() + viol.size())));
        for (size_t k = 0; k < viol.size() && (int64_t)next.size() < cap; ++k) next.push_back(viol[k]);
        // keep the size: refill with the previous zero-weight members
        for (int64_t k = 0; k < nC && (int64_t)next.size() < (int64_t)C.size(); ++k)
            if (!(wh[k] > 0.0)) next.push_back(C[k]);
        C.swap(next);
    }
    // outputs: the full weight vector and the chi^2 parts of the final state
    double* chi = scal;   // [total, obs, reg] from the last core solve equal the exact values over all N
    CUDA_TRY(ctx, cudaMemsetAsync(chi, 0, 4 * sizeof(double), st), "memset");
    CUDA_TRY(ctx, chi2(ctx, M, Um->nd, e, N, w, chi), "chi2");
    {
        LaunchTimer lt(ctx, K_CHI2);
        k_chi2_finish<<<1, 1, 0, st>>>(chi, lam / (double)N, chi2_dev);
    }
    CUDA_TRY(ctx, cudaGetLastError(), "chi2");
    CUDA_TRY(ctx, cudaMemcpyAsync(w_dev, w, N * sizeof(double), cudaMemcpyDeviceToDevice, st), "weights");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "working set");
    ctx->solve_info[0] = inner_info[0];
    ctx->solve_info[1] = inner_info[1];
    ctx->solve_info[2] = pg_rel;
    ctx->solve_info[3] = 1.0;
    ctx->solve_info[4] = inner_info[4];
    ctx->solve_info[5] = pg_rel <= ctx->opt.kkt_tol ? 1.0 : 0.0;
    ctx->solve_info[6] = rounds + (done ? 0 : 0);
    ctx->solve_info[7] = (double)C.size();
    if (!done) {
        set_error(ctx, "solve: working set did not settle in %d rounds (projected gradient %.3g of max|q|)", rounds,
                  pg_rel);
        return SW_ENONCONV;
    }
    return (core == SW_ENONCONV && pg_rel > ctx->opt.kkt_tol) ? SW_ENONCONV : SW_OK;
}

static sw_status solve_dispatch(sw_ctx* ctx, const sw_matrix* U, const double* y_dev, const double* sig_dev,
                                double lam, double* w_dev, double* chi2_dev)
{
    // orbits outnumber constraints: moderate N -> orbit space on all orbits (exact through the
    // polish); large N -> working set; working_set = 0 -> the constraint-space (Woodbury) form
    const bool many = U->N > U->M;
    const bool direct = many && ctx->opt.working_set && U->N <= ctx->opt.orbit_direct_max;
    const bool ws = many && ctx->opt.working_set && !direct;
    const Problem pb{U->d, U->M, U->N, U->nd, (double)U->N, direct};
    // solver: 1 active set, 2 ADMM (the paper's, with refinement and polish), 0 (auto) the active
    // set whenever its reduced systems stay definite (lambda > 0, or no more orbits than rows) and for
    // large libraries, ADMM otherwise
    const bool active = ctx->opt.solver == 1 ||
                        (ctx->opt.solver == 0 && (lam > 0.0 || !many || (ws && ctx->opt.large_solver == 0)));
    if (active) {
        if (U->elem == 8) return solve_active_set<double, double, double>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev);
        if (ctx->opt.gram_tc && gram_tc_available())
            return solve_active_set<float, __nv_bfloat16, float>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev);
        return solve_active_set<float, float, float>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev);
    }
    if (U->elem == 8) {
        return ws ? solve_working_set<double, double, double>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev)
                  : solve_impl<double, double, double>(ctx, pb, y_dev, sig_dev, lam, w_dev, chi2_dev);
    }
    if (ctx->opt.gram_tc && gram_tc_available())
        return ws ? solve_working_set<float, __nv_bfloat16, float>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev)
                  : solve_impl<float, __nv_bfloat16, float>(ctx, pb, y_dev, sig_dev, lam, w_dev, chi2_dev);
    return ws ? solve_working_set<float, float, float>(ctx, U, y_dev, sig_dev, lam, w_dev, chi2_dev)
              : solve_impl<float, float, float>(ctx, pb, y_dev, sig_dev, lam, w_dev, chi2_dev);
}

static sw_status check_solve_args(sw_ctx* ctx, const sw_matrix* U, const void* a, const void* b, double lam,
                                  const void* w, const void* c)
{
    if (!ctx) return SW_EINVAL;
    ctx->err.clear();
    if (!U || !a || !b || !w || !c) { set_error(ctx, "solve: NULL argument"); return SW_EINVAL; }
    if (U->ctx != ctx) { set_error(ctx, "solve: matrix belongs to another context"); return SW_EINVAL; }
    if (!(lam >= 0.0) || !std::isfinite(lam)) { set_error(ctx, "solve: lambda must be finite and >= 0"); return SW_EINVAL; }
    if (U->M <= 0 || U->N <= 0) { set_error(ctx, "solve: empty matrix"); return SW_EINVAL; }
    return SW_OK;
}

extern "C" sw_status sw_solve_weights_device(sw_ctx* ctx, const sw_matrix* U, const double* data_dev,
                                             const double* errors_dev, double lambda, double* weights_dev,
                                             double* chi2_dev)
{
    SW_TRY(check_solve_args(ctx, U, data_dev, errors_dev, lambda, weights_dev, chi2_dev));
    cudaSetDevice(ctx->device);
    return solve_dispatch(ctx, U, data_dev, errors_dev, lambda, weights_dev, chi2_dev);
}

extern "C" sw_status sw_solve_weights(sw_ctx* ctx, const sw_matrix* U, const double* data, const double* errors,
                                      double lambda, double* weights_out, double* chi2_out)
{
    SW_TRY(check_solve_args(ctx, U, data, errors, lambda, weights_out, chi2_out));
    cudaSetDevice(ctx->device);
    const int64_t M = U->M, N = U->N;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (2 * M + N + 4) * sizeof(double));
    if (e != cudaSuccess) { cudaGetLastError(); return ctx->cuda_fail(e, "solve staging"); }
    double *dy = buf, *ds = buf + M, *dw = buf + 2 * M, *dc = buf + 2 * M + N;
    sw_status s = SW_OK;
    if ((e = cudaMemcpyAsync(dy, data, M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ds, errors, M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream))) {
        s = ctx->cuda_fail(e, "data upload");
    } else {
        s = solve_dispatch(ctx, U, dy, ds, lambda, dw, dc);
        if (s == SW_OK || s == SW_ENONCONV) {
            cudaError_t e2;
            if ((e2 = cudaMemcpyAsync(weights_out, dw, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
                (e2 = cudaMemcpyAsync(chi2_out, dc, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
                (e2 = cudaStreamSynchronize(ctx->stream)))
                s = ctx->cuda_fail(e2, "result download");
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    return s;
}

extern "C" sw_status sw_solve_bootstrap(sw_ctx* ctx, const sw_matrix* U, const double* data, const double* errors,
                                        double lambda, int64_t n_boot, const double* xi, double* weights_out,
                                        double* chi2_b_out, double* chi2_model_out)
{
    SW_TRY(check_solve_args(ctx, U, data, errors, lambda, chi2_b_out, chi2_model_out));
    if (n_boot < 1 || !xi) { set_error(ctx, "sw_solve_bootstrap: n_boot >= 1 and the draws xi are required"); return SW_EINVAL; }
    if (!(lambda > 0.0) && U->N > U->M) {
        set_error(ctx, "sw_solve_bootstrap: the warm-started active set needs lambda > 0 or no more orbits than rows");
        return SW_EINVAL;
    }
    cudaSetDevice(ctx->device);
    const int64_t M = U->M, N = U->N, B = n_boot;
    double* buf = nullptr;
    const size_t nbuf = (size_t)(2 * M + B * M + (weights_out ? B * N : 0) + B);
    cudaError_t e = cudaMalloc(&buf, nbuf * sizeof(double));
    if (e != cudaSuccess) { cudaGetLastError(); return ctx->cuda_fail(e, "bootstrap staging"); }
    double *dy = buf, *ds = buf + M, *dxi = buf + 2 * M, *dw = weights_out ? dxi + B * M : nullptr;
    double* dc = dxi + B * M + (weights_out ? B * N : 0);
    sw_status s = SW_OK;
    if ((e = cudaMemcpyAsync(dy, data, M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ds, errors, M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(dxi, xi, (size_t)B * M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream))) {
        s = ctx->cuda_fail(e, "bootstrap upload");
    } else {
        if (U->elem == 8)
            s = solve_bootstrap<double, double, double>(ctx, U, dy, ds, lambda, B, dxi, dw, dc);
        else if (ctx->opt.gram_tc && gram_tc_available())
            s = solve_bootstrap<float, __nv_bfloat16, float>(ctx, U, dy, ds, lambda, B, dxi, dw, dc);
        else
            s = solve_bootstrap<float, float, float>(ctx, U, dy, ds, lambda, B, dxi, dw, dc);
        if (s == SW_OK || s == SW_ENONCONV) {
            cudaError_t e2;
            if ((e2 = cudaMemcpyAsync(chi2_b_out, dc, B * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
                (weights_out && (e2 = cudaMemcpyAsync(weights_out, dw, (size_t)B * N * sizeof(double),
                                                      cudaMemcpyDeviceToHost, ctx->stream))) ||
                (e2 = cudaStreamSynchronize(ctx->stream))) {
                s = ctx->cuda_fail(e2, "bootstrap download");
            } else {
                // marginalised chi^2 over the realisations: -2 ln of the bootstrap-averaged likelihood
                // exp(-chi2_b / 2), taken relative to the smallest chi2_b so nothing over- or underflows
                double cmin = chi2_b_out[0];
                for (int64_t b = 1; b < B; ++b) cmin = std::min(cmin, chi2_b_out[b]);
                double sum = 0.0;
                for (int64_t b = 0; b < B; ++b) sum += std::exp(-0.5 * (chi2_b_out[b] - cmin));
                *chi2_model_out = cmin - 2.0 * std::log(sum / (double)B);
            }
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    return s;
}

extern "C" sw_status sw_solve_info(sw_ctx* ctx, double* out8)
{
    if (!ctx || !out8) return SW_EINVAL;
    for (int k = 0; k < 8; ++k) out8[k] = ctx->solve_info[k];
    return SW_OK;
}

extern "C" sw_status sw_matrix_apply(const sw_matrix* U, const double* w, double* y_out)
{
    if (!U || !w || !y_out || U->ctx->destroyed) return SW_EINVAL;
    sw_ctx* ctx = U->ctx;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (U->N + U->M) * sizeof(double));
    if (e != cudaSuccess) { cudaGetLastError(); return ctx->cuda_fail(e, "apply buffers"); }
    sw_status s = SW_OK;
    if ((e = cudaMemcpyAsync(buf, w, U->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemsetAsync(buf + U->N, 0, U->M * sizeof(double), ctx->stream)) ||
        (e = (U->elem == 8 ? u_times_w<double>(ctx, (const double*)U->d, U->M, U->N, buf, buf + U->N)
                           : u_times_w<float>(ctx, (const float*)U->d, U->M, U->N, buf, buf + U->N))) ||
        (e = cudaMemcpyAsync(y_out, buf + U->N, U->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        s = ctx->cuda_fail(e, "matrix apply");
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    return s;
}

extern "C" sw_status sw_factor_preconditioner(sw_ctx* ctx, const float* gram, int64_t K, int mode, float* L_out,
                                              float* X_out, int* info_out)
{
    CHECK_CTX(ctx);
    if (!gram || !L_out || !X_out || !info_out || K <= 0 || K > 65536 || (mode != 0 && mode != 1)) {
        set_error(ctx, "sw_factor_preconditioner: bad arguments");
        return SW_EINVAL;
    }
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    if (mode == 0 && !chol_tc_available()) {
        set_error(ctx, "sw_factor_preconditioner: the tensor-map encoder is unavailable");
        return SW_ECUDA;
    }
    const int64_t ld = mode == 0 ? (K + 3) / 4 * 4 : K;
    cudaStream_t st = ctx->stream;
    float *G = nullptr, *X = nullptr, *D = nullptr;
    int* flags = nullptr;
    sw_status s = SW_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&G, (size_t)K * ld * sizeof(float))) || (e = cudaMalloc(&X, (size_t)K * ld * sizeof(float))) ||
        (e = cudaMalloc(&D, 64 * 64 * sizeof(float))) || (e = cudaMalloc(&flags, 2 * sizeof(int)))) {
        cudaGetLastError();
        s = ctx->cuda_fail(e, "factor buffers");
    }
    int fh[2] = {0, 0};
    if (s == SW_OK) {
        if ((e = cudaMemcpy2DAsync(G, ld * sizeof(float), gram, K * sizeof(float), K * sizeof(float), K,
                                   cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st)) ||
            (e = mode == 0 ? cholesky_inverse_tc(ctx, G, X, K, ld, flags, flags + 1)
                           : cholesky_inverse<float>(ctx, G, X, D, K, flags)) ||
            (e = cudaMemcpy2DAsync(L_out, K * sizeof(float), G, ld * sizeof(float), K * sizeof(float), K,
                                   cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpy2DAsync(X_out, K * sizeof(float), X, ld * sizeof(float), K * sizeof(float), K,
                                   cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(fh, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            s = ctx->cuda_fail(e, "preconditioner factorisation");
    }
    cudaStreamSynchronize(st);
    cudaFree(G);
    cudaFree(X);
    cudaFree(D);
    cudaFree(flags);
    if (s == SW_OK && fh[1]) {
        set_error(ctx, "sw_factor_preconditioner: a tensor-core update timed out");
        s = SW_ETIMEOUT;
    }
    *info_out = fh[0];
    return s;
}
