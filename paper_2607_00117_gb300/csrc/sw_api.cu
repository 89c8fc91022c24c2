// C-ABI of libsw: context, potential set-up, orbit-library integration,
// projection to the orbit matrix, and diagnostics.  The weight solve lives in
// sw_solve.cu.
#include "sw_api_internal.cuh"

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

namespace sw {

const char* kKernelNames[K_COUNT] = {
    "ics_to_soa", "orbit_project_bin", "orbit_drift", "zero_flagged", "finalize_columns", "trajectory",
    "potential_eval", "whiten", "gram_tcgen05", "gram_simt", "shift_diag", "diag_factor_inverse", "panel_gemm",
    "syrk_update", "inverse_block_row", "trinv_update", "gemv_n", "gemv_t", "trmv_l", "trmv_lt", "admm_update",
    "residual", "gradient", "chi2", "misc", "batch_orbit_bin", "mlp_fwd", "mlp_bwd", "adam", "reduce_gh", "pcg", "bundle", "cholesky_inverse",
    "syrk_update_tcgen05", "trinv_update_tcgen05", "factor_border"};

void set_error(sw_ctx* ctx, const char* fmt, ...)
{
    if (!ctx) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
}

cudaStream_t ctx_stream(sw_ctx* ctx) { return ctx->stream; }
int ctx_sms(const sw_ctx* ctx) { return ctx->n_sm; }

LaunchTimer::LaunchTimer(sw_ctx* c, int kid) : LaunchTimer(c, kid, c ? c->stream : nullptr) {}

LaunchTimer::LaunchTimer(sw_ctx* c, int kid, cudaStream_t s) : ctx(c), id(kid), on(c && c->prof), st(s)
{
    if (!ctx) return;
    ctx->launches++;
    ctx->k_launch[id]++;
    if (on) {
        cudaEvent_t a = ctx->take_event(), b = ctx->take_event();
        cudaEventRecord(a, st);
        ctx->recs.push_back({id, a, b});
    }
}

LaunchTimer::~LaunchTimer()
{
    if (on) cudaEventRecord(ctx->recs.back().b, st);
}

}  // namespace sw

using namespace sw;

cudaEvent_t sw_ctx::take_event()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void sw_ctx::harvest()
{
    if (recs.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto& r : recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) k_ms[r.id] += ms;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

sw_status sw_ctx::cuda_fail(cudaError_t e, const char* what)
{
    set_error(this, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA;
}

sw_status sw_ctx::ensure(void** p, size_t* cap, size_t need, const char* what)
{
    if (*cap >= need && *p) return SW_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (need == 0) return SW_OK;
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error(this, "cudaMalloc(%zu bytes) for %s failed: %s", need, what, cudaGetErrorString(e));
        return SW_ENOMEM;
    }
    ++n_alloc;
    *cap = need;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Every entry point starts by clearing any stale, non-sticky runtime error so
// that a later cudaGetLastError() reports only errors of this call.
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

extern "C" sw_status sw_create(sw_ctx** out, int device, sw_precision prec, void* cuda_stream)
{
    if (!out) return SW_EINVAL;
    *out = nullptr;
    if (prec != SW_FP64_PLAIN && prec != SW_FP32_KAHAN) return SW_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SW_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SW_ECUDA;
    sw_ctx* c = new sw_ctx();
    c->device = device;
    c->prec = prec;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->n_sm < 1) {
        cudaGetLastError();
        c->n_sm = 1;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SW_ECUDA;
        }
        c->own_stream = true;
    }
    c->opt.ej_every = prec == SW_FP64_PLAIN ? 1 : 8;
    if (cudaMalloc(&c->d_stats, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return SW_ENOMEM;
    }
    *out = c;
    return SW_OK;
}

static void ctx_release(sw_ctx* ctx)
{
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->harvest();
    void* bufs[] = {ctx->d_soa, ctx->d_cs, ctx->d_aos, ctx->d_drift, ctx->d_status, ctx->d_stats, ctx->d_ghtab,
                    ctx->d_mlp, ctx->d_split, ctx->d_chol, ctx->d_ttotal, ctx->d_chol_tc, ctx->d_cut,
                    ctx->d_invsig_f};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (auto& b : ctx->mat_cache) cudaFree(b.first);
    ctx->mat_cache.clear();
    if (ctx->d_ghw) cudaFree(ctx->d_ghw);
    ctx->d_ghw = nullptr;
    ctx->d_soa = ctx->d_cs = ctx->d_ghtab = ctx->d_mlp = ctx->d_split = ctx->d_chol = nullptr;
    ctx->d_ttotal = ctx->d_chol_tc = ctx->d_cut = ctx->d_invsig_f = nullptr;
    ctx->d_aos = ctx->d_drift = nullptr;
    ctx->d_status = nullptr;
    ctx->d_stats = nullptr;
    ctx->solve_ws.release();
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    ctx->pool.clear();
    for (cudaEvent_t e : ctx->dep_events) cudaEventDestroy(e);
    ctx->dep_events.clear();
    if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
    ctx->stream2 = nullptr;
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    ctx->stream = nullptr;
    cudaGetLastError();
}

// Matrices still alive keep the (released) context object until the last one
// is freed, so freeing in either order is safe.
extern "C" sw_status sw_destroy(sw_ctx* ctx)
{
    if (!ctx || ctx->destroyed) return SW_OK;
    ctx_release(ctx);
    ctx->destroyed = true;
    if (ctx->live_matrices == 0) delete ctx;
    return SW_OK;
}

extern "C" const char* sw_last_error(const sw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------
// Potential (Sec. 3.2): NFW (M200, c, H0) -> (M_DM, R_s) with Delta = 200,
// rho_crit = 3 H^2 / (8 pi G) and M_DM = M200 / [ln(1+c) - c/(1+c)].
// ---------------------------------------------------------------------------
static bool pos_finite(double x) { return std::isfinite(x) && x > 0.0; }

namespace sw {

sw_status check_potential(sw_ctx* ctx, const sw_potential_params* p)
{
    if (!p) { set_error(ctx, "sw_set_potential: params is NULL"); return SW_EINVAL; }
    if (p->disc_M != 0.0 && !(pos_finite(p->disc_M) && pos_finite(p->disc_a) && pos_finite(p->disc_b))) {
        set_error(ctx, "sw_set_potential: disc mass and scales must be positive and finite");
        return SW_EINVAL;
    }
    if (p->halo_M200 != 0.0 && !(pos_finite(p->halo_M200) && pos_finite(p->halo_c) && pos_finite(p->H0))) {
        set_error(ctx, "sw_set_potential: halo M200, c and H0 must be positive and finite");
        return SW_EINVAL;
    }
    if (p->bar_kind != 0 && p->bar_kind != 1) {
        set_error(ctx, "sw_set_potential: bar_kind must be 0 (Long-Murali) or 1 (Dehnen-Aly T3 + V4)");
        return SW_EINVAL;
    }
    if (p->bar_M != 0.0 && p->bar_kind == 0 &&
        !(pos_finite(p->bar_M) && pos_finite(p->bar_L) && pos_finite(p->bar_b) && pos_finite(p->bar_c))) {
        set_error(ctx, "sw_set_potential: bar mass, half-length and scales must be positive and finite");
        return SW_EINVAL;
    }
    if (p->bar_M != 0.0 && p->bar_kind == 1 &&
        !(pos_finite(p->bar_M) && pos_finite(p->bar_L) && pos_finite(p->disc_b))) {
        set_error(ctx, "sw_set_potential: the paper's bar needs a positive mass, half-length and disc height");
        return SW_EINVAL;
    }
    if (p->test_kind < 0 || p->test_kind > 2 || (p->test_kind == 2 && !pos_finite(p->test_a)) ||
        (p->test_kind != 0 && !(std::isfinite(p->test_M) && p->test_M >= 0.0))) {
        set_error(ctx, "sw_set_potential: bad test potential");
        return SW_EINVAL;
    }
    return SW_OK;
}

// NFW from (M200, c, H0) (Sec. 2.1): rho_crit = 3 H0^2 / (8 pi G), R200 from M200 = 200 rho_crit
// (4 pi / 3) R200^3, R_s = R200 / c, M_DM = M200 / [ln(1 + c) - c / (1 + c)].
void halo_constants(const sw_potential_params& p, double& Mdm, double& rs)
{
    Mdm = 0.0;
    rs = 1.0;
    if (p.halo_M200 > 0.0) {
        const double pi = 3.14159265358979323846;
        double H = p.H0 / 1000.0;
        double rho_c = 3.0 * H * H / (8.0 * pi * SW_G);
        double Rv = cbrt(3.0 * p.halo_M200 / (4.0 * pi * 200.0 * rho_c));
        rs = Rv / p.halo_c;
        Mdm = p.halo_M200 / (log(1.0 + p.halo_c) - p.halo_c / (1.0 + p.halo_c));
    }
}

}  // namespace sw

extern "C" sw_status sw_set_potential(sw_ctx* ctx, const sw_potential_params* p)
{
    CHECK_CTX(ctx);
    SW_TRY(check_potential(ctx, p));
    ctx->pot = *p;
    halo_constants(*p, ctx->Mdm, ctx->rs);
    ctx->has_pot = true;
    return SW_OK;
}

// Positive nodes and weights of the 8-point Gauss-Legendre rule on [-1, 1]: the roots of the
// Legendre polynomial P_8 by Newton's method from the asymptotic first guesses, weights
// 2 / ((1 - x^2) P_8'(x)^2) (Abramowitz & Stegun 25.4.29).
static void gauss_legendre8(double x[4], double w[4])
{
    const int n = 8;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n / 2; ++k) {
        double t = std::cos(pi * (k + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 60; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2 * j - 1) * t * p1 - (j - 1) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double step = p1 / dp;
            t -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        x[k] = t;
        w[k] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

template <typename T>
FieldT<T> make_field_from(const sw_potential_params& p, double Mdm, double rs)
{
    FieldT<T> f{};
    f.has_disc = p.disc_M > 0.0;
    f.gm_disc = (T)(SW_G * p.disc_M);
    f.disc_a = (T)p.disc_a;
    f.disc_b2 = (T)(p.disc_b * p.disc_b);
    f.has_halo = Mdm > 0.0;
    f.gm_halo = (T)(SW_G * Mdm);
    f.halo_rs = (T)rs;
    f.halo_inv_rs = (T)(1.0 / rs);
    f.has_bar = p.bar_M > 0.0;
    f.k_bar = p.bar_M > 0.0 ? (T)(SW_G * p.bar_M / (2.0 * p.bar_L)) : T(0);
    f.bar_L = (T)p.bar_L;
    f.bar_a = (T)p.bar_b;
    f.bar_b2 = (T)(p.bar_c * p.bar_c);
    f.test_kind = p.test_kind;
    f.gm_test = (T)(SW_G * p.test_M);
    f.test_a2 = (T)(p.test_a * p.test_a);
    f.bar_kind = p.bar_kind;
    if (p.bar_kind == 1 && p.bar_M > 0.0) {
        // the paper's bar (Sec. 2.1.2): T3 (eta = 1, a = L_b / 5, b = b_d, L = L_b) + V4 (eta = 0,
        // a = b = 0.5 kpc, L = 0.1 kpc), equal halves of M_b
        f.da_gm1 = (T)(SW_G * 0.5 * p.bar_M);
        f.da_a1 = (T)(p.bar_L / 5.0);
        f.da_b1sq = (T)(p.disc_b * p.disc_b);
        f.da_L1 = (T)p.bar_L;
        f.da_gm2 = (T)(SW_G * 0.5 * p.bar_M);
        f.da_a2 = (T)0.5;
        f.da_b2sq = (T)0.25;
        f.da_L2 = (T)0.1;
        double gx[4], gw[4];
        gauss_legendre8(gx, gw);
        for (int k = 0; k < 4; ++k) {
            f.gl_x[k] = (T)gx[k];
            f.gl_w[k] = (T)gw[k];
        }
    }
    return f;
}

template <typename T>
FieldT<T> make_field(const sw_ctx* ctx)
{
    return make_field_from<T>(ctx->pot, ctx->Mdm, ctx->rs);
}
template FieldT<float> make_field_from<float>(const sw_potential_params&, double, double);
template FieldT<double> make_field_from<double>(const sw_potential_params&, double, double);

// rows of the SoA orbit state: 6, plus 6 rounding residuals in FP32
template <typename T>
static constexpr int soa_rows() { return sizeof(T) == 4 ? 12 : 6; }

// cos / sin of Omega_p * (n dt), n = 0..nsteps, in FP64 on the host.
template <typename T>
void cs_table(std::vector<T>& out, double omega, double dt, int64_t nsteps)
{
    out.resize(2 * (nsteps + 1));
    for (int64_t n = 0; n <= nsteps; ++n) {
        double th = omega * ((double)n * dt);
        out[2 * n] = (T)cos(th);
        out[2 * n + 1] = (T)sin(th);
    }
}

template <typename T>
static sw_status upload_library(sw_ctx* ctx, const double* ics_dev_aos, int64_t n, double omega, double dt,
                                int64_t nsteps)
{
    SW_TRY(ctx->ensure(&ctx->d_soa, &ctx->soa_cap, (size_t)soa_rows<T>() * n * sizeof(T), "orbit state"));
    CUDA_TRY(ctx, launch_ics_to_soa<T>(ctx, ics_dev_aos, n, (T*)ctx->d_soa, n), "ics_to_soa");
    std::vector<T> cs;
    cs_table<T>(cs, omega, dt, nsteps);
    SW_TRY(ctx->ensure(&ctx->d_cs, &ctx->cs_cap, cs.size() * sizeof(T), "cos/sin table"));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_cs, cs.data(), cs.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream),
             "cos/sin upload");
    // the host vector dies at return: make the copy complete first
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cos/sin upload");
    ctx->n_orb = n;
    ctx->omega = omega;
    ctx->dt = dt;
    ctx->nsteps = nsteps;
    ctx->has_lib = true;
    return SW_OK;
}

template <typename T>
static ModelT<T> base_model(sw_ctx* ctx)
{
    ModelT<T> m{};
    m.f = make_field<T>(ctx);
    m.dt = (T)ctx->dt;
    m.half_dt = (T)(0.5 * ctx->dt);
    m.omega = (T)ctx->omega;
    m.cs = (const T*)ctx->d_cs;
    m.n_orb = ctx->n_orb;
    m.orbit_base = 0;
    return m;
}

template <typename T>
static sw_status drift_pass(sw_ctx* ctx, double* drift_dev, uint8_t* status_dev)
{
    ModelT<T> m = base_model<T>(ctx);
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_stats, 0, 4 * sizeof(unsigned long long), ctx->stream), "memset");
    CUDA_TRY(ctx, launch_orbit_drift<T>(ctx, m, (const T*)ctx->d_soa, ctx->n_orb, ctx->nsteps, 1, drift_dev,
                                        status_dev, ctx->d_stats),
             "orbit drift kernel");
    return SW_OK;
}

static sw_status check_lib_args(sw_ctx* ctx, int64_t n_orb, double omega, double dt, int64_t nsteps)
{
    if (!ctx->has_pot) { set_error(ctx, "set the potential first"); return SW_ESTATE; }
    if (n_orb <= 0 || nsteps <= 0 || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(omega)) {
        set_error(ctx, "integrate: need n_orb > 0, nsteps > 0, finite dt > 0 and finite omega_p");
        return SW_EINVAL;
    }
    if (nsteps > (int64_t)1 << 28) { set_error(ctx, "integrate: nsteps too large"); return SW_EINVAL; }
    return SW_OK;
}

extern "C" sw_status sw_integrate_library_device(sw_ctx* ctx, const double* ics_dev, int64_t n_orb, double omega_p,
                                                 double dt, int64_t nsteps, double* drift_dev, uint8_t* status_dev)
{
    CHECK_CTX(ctx);
    if (!ics_dev) { set_error(ctx, "ics is NULL"); return SW_EINVAL; }
    SW_TRY(check_lib_args(ctx, n_orb, omega_p, dt, nsteps));
    cudaSetDevice(ctx->device);
    if (ctx->prec == SW_FP64_PLAIN) {
        SW_TRY(upload_library<double>(ctx, ics_dev, n_orb, omega_p, dt, nsteps));
        if (drift_dev || status_dev) SW_TRY(drift_pass<double>(ctx, drift_dev, status_dev));
    } else {
        SW_TRY(upload_library<float>(ctx, ics_dev, n_orb, omega_p, dt, nsteps));
        if (drift_dev || status_dev) SW_TRY(drift_pass<float>(ctx, drift_dev, status_dev));
    }
    return SW_OK;
}

extern "C" sw_status sw_integrate_library(sw_ctx* ctx, const double* ics, int64_t n_orb, double omega_p, double dt,
                                          int64_t nsteps, double* drift_out, uint8_t* status_out)
{
    CHECK_CTX(ctx);
    if (!ics) { set_error(ctx, "ics is NULL"); return SW_EINVAL; }
    SW_TRY(check_lib_args(ctx, n_orb, omega_p, dt, nsteps));
    cudaSetDevice(ctx->device);
    SW_TRY(ctx->ensure((void**)&ctx->d_aos, &ctx->aos_cap, (size_t)6 * n_orb * sizeof(double), "ic staging"));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_aos, ics, (size_t)6 * n_orb * sizeof(double), cudaMemcpyHostToDevice,
                                  ctx->stream),
             "ic upload");
    double* dd = nullptr;
    uint8_t* ds = nullptr;
    if (drift_out || status_out) {
        SW_TRY(ctx->ensure_stats(n_orb));
        dd = ctx->d_drift;
        ds = ctx->d_status;
    }
    SW_TRY(sw_integrate_library_device(ctx, ctx->d_aos, n_orb, omega_p, dt, nsteps, dd, ds));
    if (drift_out)
        CUDA_TRY(ctx, cudaMemcpyAsync(drift_out, dd, n_orb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                 "drift download");
    if (status_out)
        CUDA_TRY(ctx, cudaMemcpyAsync(status_out, ds, n_orb, cudaMemcpyDeviceToHost, ctx->stream), "status download");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "integrate");
    return SW_OK;
}

sw_status sw_ctx::ensure_stats(int64_t n)
{
    SW_TRY(ensure((void**)&d_drift, &drift_cap, n * sizeof(double), "drift"));
    SW_TRY(ensure((void**)&d_status, &status_cap, (size_t)n, "status"));
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Projection (Sec. 2.2.3-2.2.4)
// ---------------------------------------------------------------------------
static void euler_matrix(double a, double b, double g, double R[9])
{
    double A[9] = {cos(a), -sin(a), 0, sin(a), cos(a), 0, 0, 0, 1};
    double B[9] = {1, 0, 0, 0, cos(b), -sin(b), 0, sin(b), cos(b)};
    double C[9] = {cos(g), -sin(g), 0, sin(g), cos(g), 0, 0, 0, 1};
    double T_[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += B[3 * i + k] * A[3 * k + j];
            T_[3 * i + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += C[3 * i + k] * T_[3 * k + j];
            R[3 * i + j] = s;
        }
}

template <typename T>
GridT<T> make_grid(double incl, double pa, double bar_angle, const sw_pixel_grid* pix, const sw_vbins* vb,
                   const sw_density_grid* dens, int gh, int mirror4)
{
    GridT<T> g{};
    double R[9];
    euler_matrix(bar_angle, incl, pa, R);
    for (int k = 0; k < 9; ++k) g.R[k] = (T)R[k];
    g.nx = pix->nx; g.ny = pix->ny;
    g.x0 = (T)pix->x0; g.y0 = (T)pix->y0; g.dx = (T)pix->dx; g.dy = (T)pix->dy;
    g.inv_dx = (T)(1.0 / pix->dx); g.inv_dy = (T)(1.0 / pix->dy);
    g.nv = gh ? 0 : vb->nv;
    g.v0 = gh ? T(0) : (T)vb->v0; g.dv = gh ? T(1) : (T)vb->dv; g.inv_dv = gh ? T(1) : (T)(1.0 / vb->dv);
    g.nR = dens->nR; g.nphi = dens->nphi; g.nz = dens->nz;
    double dR = dens->Rmax / dens->nR, dphi = 2.0 * 3.14159265358979323846 / dens->nphi,
           dz = (dens->zmax - dens->zmin) / dens->nz;
    g.dR = (T)dR; g.inv_dR = (T)(1.0 / dR); g.dphi = (T)dphi; g.inv_dphi = (T)(1.0 / dphi);
    g.zmin = (T)dens->zmin; g.dz = (T)dz; g.inv_dz = (T)(1.0 / dz);
    g.gh = gh;
    g.ncopy = mirror4 ? 4 : 1;
    // the copies (-x, -y, +-z) project to (-X, -Y, -V) of the (x, y, -+z) copies: with grids symmetric
    // about 0 their bins are the reflected ones
    auto centred = [](double lo, int n, double w) { return std::fabs(lo + 0.5 * n * w) <= 1e-12 * (std::fabs(lo) + w); };
    g.sym = centred(pix->x0, pix->nx, pix->dx) && centred(pix->y0, pix->ny, pix->dy) &&
            (gh || centred(vb->v0, vb->nv, vb->dv));
    g.nd = (int64_t)dens->nR * dens->nphi * dens->nz;
    g.npix = (int64_t)pix->nx * pix->ny;
    g.M = g.nd + g.npix + (gh ? 4 * g.npix : g.npix * g.nv);
    return g;
}

template void cs_table<float>(std::vector<float>&, double, double, int64_t);
template void cs_table<double>(std::vector<double>&, double, double, int64_t);
template GridT<float> make_grid<float>(double, double, double, const sw_pixel_grid*, const sw_vbins*,
                                       const sw_density_grid*, int, int);
template GridT<double> make_grid<double>(double, double, double, const sw_pixel_grid*, const sw_vbins*,
                                         const sw_density_grid*, int, int);

// Matrix buffers: a freed matrix's buffer is kept by its context and handed to the next matrix
// whose size it covers with at most 1/8 to spare; a failed allocation first returns the kept
// buffers to the driver and tries again.
static cudaError_t matrix_alloc(sw_ctx* ctx, void** d, size_t bytes)
{
    for (size_t k = 0; k < ctx->mat_cache.size(); ++k) {
        const size_t have = ctx->mat_cache[k].second;
        if (have >= bytes && have - bytes <= bytes / 8) {
            *d = ctx->mat_cache[k].first;
            ctx->mat_cache.erase(ctx->mat_cache.begin() + k);
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(d, bytes);
    if (e != cudaSuccess && !ctx->mat_cache.empty()) {
        cudaGetLastError();
        for (auto& b : ctx->mat_cache) cudaFree(b.first);
        ctx->mat_cache.clear();
        e = cudaMalloc(d, bytes);
    }
    return e;
}

static void matrix_release(sw_ctx* ctx, void* d, size_t bytes)
{
    if (!d) return;
    if (ctx->destroyed || !ctx->opt.matrix_cache) {
        cudaFree(d);
        return;
    }
    ctx->mat_cache.emplace_back(d, bytes);
    while (ctx->mat_cache.size() > 4) {   // the oldest goes back first
        cudaFree(ctx->mat_cache.front().first);
        ctx->mat_cache.erase(ctx->mat_cache.begin());
    }
}

static size_t matrix_bytes(const sw_matrix* U) { return (size_t)U->M * (size_t)U->N * (size_t)U->elem; }

template <typename T>
static sw_status project_impl(sw_ctx* ctx, const GridT<T>& g, const double* gh_v0_s, sw_matrix** U_out)
{
    const int64_t Norb = ctx->n_orb, M = g.M;
    const int nb = ctx->opt.project_bundle;   // orbits per column (bundles accumulated at bin time)
    if (nb > 1 && (Norb % nb != 0 || ctx->opt.integrator != 0)) {
        set_error(ctx, "sw_project: project_bundle %d needs the kick-drift-kick integrator and must divide the %lld orbits",
                  nb, (long long)Norb);
        return SW_EINVAL;
    }
    const int64_t N = nb > 1 ? Norb / nb : Norb;   // columns
    sw_matrix* U = new sw_matrix();
    U->ctx = ctx;
    U->M = M; U->N = N; U->nd = g.nd; U->npix = g.npix; U->nkin = M - g.nd - g.npix;
    U->gh = g.gh; U->elem = sizeof(T); U->nsteps = ctx->nsteps; U->ncopy = g.ncopy;
    U->device = ctx->device;
    U->nv = g.nv; U->v0 = (double)g.v0; U->dv = (double)g.dv;
    size_t bytes = (size_t)M * (size_t)N * sizeof(T);
    cudaError_t e = matrix_alloc(ctx, &U->d, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete U;
        set_error(ctx, "cudaMalloc(%zu bytes) for the orbit matrix failed: %s", bytes, cudaGetErrorString(e));
        return SW_ENOMEM;
    }
    auto fail = [&](sw_status s) { matrix_release(ctx, U->d, bytes); delete U; return s; };
    if ((e = cudaMemsetAsync(U->d, 0, bytes, ctx->stream)) != cudaSuccess) return fail(ctx->cuda_fail(e, "memset U"));
    ModelT<T> m = base_model<T>(ctx);
    m.g = g;
    m.U = U->d;
    m.ldu = M;
    m.bundle = nb > 1 ? nb : 1;
    if (g.gh) {
        // per-pixel (v0, 1/s) table in the working precision
        std::vector<T> tab(2 * g.npix);
        for (int64_t p = 0; p < g.npix; ++p) {
            double s = gh_v0_s[2 * p + 1];
            if (!(s > 0.0) || !std::isfinite(s) || !std::isfinite(gh_v0_s[2 * p])) {
                set_error(ctx, "sw_project: GH reference (v0, s) of pixel %lld is invalid", (long long)p);
                return fail(SW_EINVAL);
            }
            tab[2 * p] = (T)gh_v0_s[2 * p];
            tab[2 * p + 1] = (T)(1.0 / s);
        }
        sw_status s = ctx->ensure(&ctx->d_ghtab, &ctx->ghtab_cap, tab.size() * sizeof(T), "GH table");
        if (s != SW_OK) return fail(s);
        if ((e = cudaMemcpyAsync(ctx->d_ghtab, tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice,
                                 ctx->stream)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "GH table upload"));
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx->cuda_fail(e, "GH table"));
        m.gh_v0s = (const T*)ctx->d_ghtab;
    }
    sw_status s = ctx->ensure_stats(Norb);
    if (s != SW_OK) return fail(s);
    if ((e = cudaMemsetAsync(ctx->d_stats, 0, 4 * sizeof(unsigned long long), ctx->stream)) != cudaSuccess)
        return fail(ctx->cuda_fail(e, "memset"));
    if (ctx->opt.integrator == 1) {
        // the paper's adaptive Bogacki-Shampine integrator in the bar frame, step-weighted samples
        s = ctx->ensure(&ctx->d_ttotal, &ctx->ttotal_cap, (size_t)N * sizeof(double), "integration times");
        if (s != SW_OK) return fail(s);
        if ((e = launch_orbit_bin_bs3<T>(ctx, m, (const T*)ctx->d_soa, N, ctx->nsteps, ctx->opt.ej_every,
                                         ctx->opt.bs3_rtol, ctx->d_drift, ctx->d_status, (double*)ctx->d_ttotal,
                                         ctx->d_stats)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "orbit kernel (adaptive)"));
        if ((e = launch_zero_flagged<T>(ctx, U->d, M, N, ctx->d_status)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "zero flagged"));
        if ((e = launch_finalize_w<T>(ctx, U->d, M, N, (const double*)ctx->d_ttotal, g.ncopy)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "finalize"));
    } else {
        if ((e = launch_orbit_bin<T>(ctx, m, (const T*)ctx->d_soa, Norb, ctx->nsteps, ctx->opt.ej_every,
                                     ctx->d_drift, ctx->d_status, ctx->d_stats)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "orbit kernel"));
        if (nb > 1) {
            // a realisation cut by the quality test contributes a zero column to its bundle's mean:
            // integrate the (rare) cut orbits again and subtract their counts, which restores the
            // bundle's integer counts exactly (GH sums to rounding)
            unsigned long long st[4];
            if ((e = cudaMemcpyAsync(st, ctx->d_stats, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream)) ||
                (e = cudaStreamSynchronize(ctx->stream)))
                return fail(ctx->cuda_fail(e, "orbit statistics"));
            if (st[1] + st[2] > 0) {
                std::vector<uint8_t> sh(Norb);
                if ((e = cudaMemcpyAsync(sh.data(), ctx->d_status, Norb, cudaMemcpyDeviceToHost, ctx->stream)) ||
                    (e = cudaStreamSynchronize(ctx->stream)))
                    return fail(ctx->cuda_fail(e, "orbit status"));
                std::vector<int64_t> cut;
                for (int64_t i = 0; i < Norb; ++i)
                    if (sh[i] != ST_OK) cut.push_back(i);
                s = ctx->ensure(&ctx->d_cut, &ctx->cut_cap, cut.size() * sizeof(int64_t), "cut orbits");
                if (s != SW_OK) return fail(s);
                if ((e = cudaMemcpyAsync(ctx->d_cut, cut.data(), cut.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                         ctx->stream)))
                    return fail(ctx->cuda_fail(e, "cut orbits"));
                ModelT<T> mc = m;
                mc.sign = -1;
                mc.orbit_list = (const int64_t*)ctx->d_cut;
                mc.n_orb = (int64_t)cut.size();
                if ((e = launch_orbit_bin<T>(ctx, mc, (const T*)ctx->d_soa, Norb, ctx->nsteps, ctx->opt.ej_every,
                                             nullptr, nullptr, nullptr)) ||
                    (e = cudaStreamSynchronize(ctx->stream)))   // the host list dies at return
                    return fail(ctx->cuda_fail(e, "orbit kernel (cut realisations)"));
            }
        } else if ((e = launch_zero_flagged<T>(ctx, U->d, M, N, ctx->d_status)) != cudaSuccess) {
            return fail(ctx->cuda_fail(e, "zero flagged"));
        }
        const int64_t count_rows = g.gh ? g.nd + g.npix : M;
        const double norm = 1.0 / ((double)g.ncopy * (double)ctx->nsteps * (double)(nb > 1 ? nb : 1));
        if ((e = launch_finalize<T>(ctx, U->d, M, N, count_rows, norm)) != cudaSuccess)
            return fail(ctx->cuda_fail(e, "finalize"));
    }
    ctx->last_proj_n = Norb;
    ctx->live_matrices++;
    *U_out = U;
    return SW_OK;
}

extern "C" sw_status sw_project(sw_ctx* ctx, double incl, double pa, double bar_angle, const sw_pixel_grid* pix,
                                const sw_vbins* vb, const sw_density_grid* dens, const double* gh_v0_s, int mirror4,
                                sw_matrix** U_out)
{
    CHECK_CTX(ctx);
    if (!U_out || !pix || !dens || (!gh_v0_s && !vb)) { set_error(ctx, "sw_project: NULL argument"); return SW_EINVAL; }
    *U_out = nullptr;
    if (!ctx->has_lib) { set_error(ctx, "sw_project: integrate a library first"); return SW_ESTATE; }
    if (!(std::isfinite(incl) && std::isfinite(pa) && std::isfinite(bar_angle))) {
        set_error(ctx, "sw_project: non-finite angle");
        return SW_EINVAL;
    }
    if (pix->nx <= 0 || pix->ny <= 0 || !pos_finite(pix->dx) || !pos_finite(pix->dy) || !std::isfinite(pix->x0) ||
        !std::isfinite(pix->y0) || dens->nR <= 0 || dens->nphi <= 0 || dens->nz <= 0 || !pos_finite(dens->Rmax) ||
        !(dens->zmax > dens->zmin) || !std::isfinite(dens->zmin) || !std::isfinite(dens->zmax) ||
        (!gh_v0_s && (vb->nv <= 0 || !pos_finite(vb->dv) || !std::isfinite(vb->v0)))) {
        set_error(ctx, "sw_project: invalid grid");
        return SW_EINVAL;
    }
    const int gh = gh_v0_s != nullptr;
    int64_t nd = (int64_t)dens->nR * dens->nphi * dens->nz, np = (int64_t)pix->nx * pix->ny;
    int64_t M = nd + np + (gh ? 4 * np : np * (int64_t)vb->nv);
    if (M >= ((int64_t)1 << 31) / 2) { set_error(ctx, "sw_project: too many rows (%lld)", (long long)M); return SW_EINVAL; }
    cudaSetDevice(ctx->device);
    if (ctx->prec == SW_FP64_PLAIN)
        return project_impl<double>(ctx, make_grid<double>(incl, pa, bar_angle, pix, vb, dens, gh, mirror4), gh_v0_s,
                                    U_out);
    return project_impl<float>(ctx, make_grid<float>(incl, pa, bar_angle, pix, vb, dens, gh, mirror4), gh_v0_s, U_out);
}

extern "C" sw_status sw_project_stats(sw_ctx* ctx, double* drift_out, uint8_t* status_out)
{
    CHECK_CTX(ctx);
    if (ctx->last_proj_n <= 0 || !ctx->d_drift) { set_error(ctx, "no projection yet"); return SW_ESTATE; }
    int64_t n = ctx->last_proj_n;
    if (drift_out)
        CUDA_TRY(ctx, cudaMemcpyAsync(drift_out, ctx->d_drift, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                 "drift download");
    if (status_out)
        CUDA_TRY(ctx, cudaMemcpyAsync(status_out, ctx->d_status, n, cudaMemcpyDeviceToHost, ctx->stream),
                 "status download");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "project stats");
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Histogram rows -> Gauss-Hermite rows
// ---------------------------------------------------------------------------
static double gh_weight(int m, double w)
{
    const double pi = 3.14159265358979323846;
    double e = 2.0 * sqrt(pi) * exp(-0.5 * w * w) / sqrt(2.0 * pi);
    switch (m) {
    case 1: return e * sqrt(2.0) * w;
    case 2: return e * (2.0 * w * w - 1.0) / sqrt(2.0);
    case 3: return e * (2.0 * w * w * w - 3.0 * w) / sqrt(3.0);
    default: return e * (4.0 * w * w * w * w - 12.0 * w * w + 3.0) / sqrt(24.0);
    }
}

template <typename T>
static sw_status reduce_gh_impl(sw_ctx* ctx, const sw_matrix* Uh, const double* v0s, sw_matrix** out)
{
    const int64_t npix = Uh->npix, nd = Uh->nd, N = Uh->N;
    const int nv = Uh->nv;
    const int64_t Mg = nd + npix * 5;
    std::vector<T> W((size_t)npix * nv * 4);
    for (int64_t p = 0; p < npix; ++p) {
        const double v0 = v0s[2 * p], sg = v0s[2 * p + 1];
        if (!(sg > 0.0) || !std::isfinite(sg) || !std::isfinite(v0)) {
            set_error(ctx, "sw_reduce_gh: GH reference (v0, s) of pixel %lld is invalid", (long long)p);
            return SW_EINVAL;
        }
        for (int k = 0; k < nv; ++k) {
            const double w = (Uh->v0 + (k + 0.5) * Uh->dv - v0) / sg;
            for (int m = 1; m <= 4; ++m) W[((size_t)p * nv + k) * 4 + (m - 1)] = (T)gh_weight(m, w);
        }
    }
    void* dW = nullptr;
    sw_matrix* G = new sw_matrix(*Uh);
    G->d = nullptr;
    G->M = Mg; G->nkin = 4 * npix; G->gh = 1;
    cudaError_t e;
    const size_t gbytes = (size_t)Mg * N * sizeof(T);
    if (ctx->ensure(&ctx->d_ghw, &ctx->ghw_cap, W.size() * sizeof(T), "GH weights") != SW_OK) {
        delete G;
        return SW_ENOMEM;
    }
    dW = ctx->d_ghw;
    if ((e = matrix_alloc(ctx, &G->d, gbytes))) {
        cudaGetLastError();
        delete G;
        set_error(ctx, "sw_reduce_gh: allocation failed");
        return SW_ENOMEM;
    }
    if ((e = cudaMemcpyAsync(dW, W.data(), W.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = launch_reduce_gh<T>(ctx, Uh->d, Uh->M, N, nd, npix, nv, dW, G->d, Mg)) ||
        (e = cudaStreamSynchronize(ctx->stream))) {
        matrix_release(ctx, G->d, gbytes); delete G;
        return ctx->cuda_fail(e, "reduce GH");
    }
    ctx->live_matrices++;
    *out = G;
    return SW_OK;
}

extern "C" sw_status sw_reduce_gh(sw_ctx* ctx, const sw_matrix* U_hist, const double* gh_v0_s, sw_matrix** U_gh_out)
{
    CHECK_CTX(ctx);
    if (!U_hist || !gh_v0_s || !U_gh_out) { set_error(ctx, "sw_reduce_gh: NULL argument"); return SW_EINVAL; }
    *U_gh_out = nullptr;
    if (U_hist->ctx != ctx || U_hist->gh || U_hist->nv <= 0) {
        set_error(ctx, "sw_reduce_gh: needs a velocity-histogram matrix of this context");
        return SW_EINVAL;
    }
    return U_hist->elem == 8 ? reduce_gh_impl<double>(ctx, U_hist, gh_v0_s, U_gh_out)
                             : reduce_gh_impl<float>(ctx, U_hist, gh_v0_s, U_gh_out);
}

extern "C" sw_status sw_bundle(sw_ctx* ctx, const sw_matrix* U, int64_t n, sw_matrix** U_out)
{
    CHECK_CTX(ctx);
    if (!U || !U_out) { set_error(ctx, "sw_bundle: NULL argument"); return SW_EINVAL; }
    *U_out = nullptr;
    if (U->ctx != ctx) { set_error(ctx, "sw_bundle: matrix belongs to another context"); return SW_EINVAL; }
    if (n < 1 || U->N % n != 0) {
        set_error(ctx, "sw_bundle: bundle size %lld must divide the orbit count %lld", (long long)n, (long long)U->N);
        return SW_EINVAL;
    }
    sw_matrix* B = new sw_matrix(*U);
    B->d = nullptr;
    B->N = U->N / n;
    const size_t bytes = (size_t)U->M * (size_t)B->N * (size_t)U->elem;
    cudaError_t e = matrix_alloc(ctx, &B->d, bytes);
    if (e) {
        cudaGetLastError();
        delete B;
        set_error(ctx, "sw_bundle: allocation failed");
        return SW_ENOMEM;
    }
    e = U->elem == 8 ? launch_bundle<double>(ctx, U->d, U->M, B->N, (int)n, B->d)
                     : launch_bundle<float>(ctx, U->d, U->M, B->N, (int)n, B->d);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) {
        matrix_release(ctx, B->d, bytes);
        delete B;
        return ctx->cuda_fail(e, "bundle");
    }
    ctx->live_matrices++;
    *U_out = B;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Matrix access
// ---------------------------------------------------------------------------
extern "C" sw_status sw_matrix_shape(const sw_matrix* U, int64_t* M, int64_t* N, int64_t* blocks3)
{
    if (!U) return SW_EINVAL;
    if (M) *M = U->M;
    if (N) *N = U->N;
    if (blocks3) { blocks3[0] = U->nd; blocks3[1] = U->npix; blocks3[2] = U->nkin; }
    return SW_OK;
}

extern "C" sw_status sw_matrix_copy(const sw_matrix* U, double* host_out)
{
    if (!U || !host_out || U->ctx->destroyed) return SW_EINVAL;
    sw_ctx* ctx = U->ctx;
    cudaGetLastError();
    cudaSetDevice(ctx->device);
    size_t n = (size_t)U->M * (size_t)U->N;
    if (U->elem == 8) {
        CUDA_TRY(ctx, cudaMemcpyAsync(host_out, U->d, n * 8, cudaMemcpyDeviceToHost, ctx->stream), "U download");
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "U download");
    } else {
        std::vector<float> tmp(n);
        CUDA_TRY(ctx, cudaMemcpyAsync(tmp.data(), U->d, n * 4, cudaMemcpyDeviceToHost, ctx->stream), "U download");
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "U download");
        for (size_t k = 0; k < n; ++k) host_out[k] = tmp[k];
    }
    return SW_OK;
}

extern "C" sw_status sw_matrix_free(sw_matrix* U)
{
    if (!U) return SW_OK;
    if (U->borrowed) return SW_EINVAL;   // owned by its batch
    sw_ctx* ctx = U->ctx;
    cudaSetDevice(U->device);
    if (!ctx->destroyed) {
        cudaStreamSynchronize(ctx->stream);
        ctx->solve_ws.forget_matrix(U);
    } else {
        cudaDeviceSynchronize();
    }
    matrix_release(ctx, U->d, matrix_bytes(U));
    cudaGetLastError();
    delete U;
    if (--ctx->live_matrices == 0 && ctx->destroyed) delete ctx;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Test hooks
// ---------------------------------------------------------------------------
template <typename T>
static sw_status trajectory_impl(sw_ctx* ctx, const double* ics, int64_t n, double omega, double dt, int64_t nsteps,
                                 double* out)
{
    double* d_aos = nullptr;
    T* d_soa = nullptr;
    T* d_cs = nullptr;
    double* d_out = nullptr;
    size_t out_n = (size_t)n * (nsteps + 1) * 6;
    std::vector<T> cs;
    cs_table<T>(cs, omega, dt, nsteps);
    cudaError_t e = cudaSuccess;
    sw_status st = SW_OK;
    if ((e = cudaMalloc(&d_aos, 6 * n * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&d_soa, soa_rows<T>() * n * sizeof(T))) != cudaSuccess ||
        (e = cudaMalloc(&d_cs, cs.size() * sizeof(T))) != cudaSuccess ||
        (e = cudaMalloc(&d_out, out_n * sizeof(double))) != cudaSuccess) {
        st = ctx->cuda_fail(e, "trajectory buffers");
    } else {
        ModelT<T> m = base_model<T>(ctx);
        m.dt = (T)dt; m.half_dt = (T)(0.5 * dt); m.omega = (T)omega; m.cs = d_cs; m.n_orb = n;
        if ((e = cudaMemcpyAsync(d_aos, ics, 6 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
            (e = cudaMemcpyAsync(d_cs, cs.data(), cs.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream)) ||
            (e = launch_ics_to_soa<T>(ctx, d_aos, n, d_soa, n)) ||
            (e = launch_trajectory<T>(ctx, m, d_soa, n, n, nsteps, d_out)) ||
            (e = cudaMemcpyAsync(out, d_out, out_n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaStreamSynchronize(ctx->stream)))
            st = ctx->cuda_fail(e, "trajectory");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(d_aos); cudaFree(d_soa); cudaFree(d_cs); cudaFree(d_out);
    return st;
}

extern "C" sw_status sw_trajectory(sw_ctx* ctx, const double* ics, int64_t n, double omega_p, double dt,
                                   int64_t nsteps, double* out)
{
    CHECK_CTX(ctx);
    if (!ics || !out || n <= 0 || nsteps < 0 || !(dt > 0)) { set_error(ctx, "sw_trajectory: bad arguments"); return SW_EINVAL; }
    if (!ctx->has_pot) { set_error(ctx, "set the potential first"); return SW_ESTATE; }
    cudaSetDevice(ctx->device);
    return ctx->prec == SW_FP64_PLAIN ? trajectory_impl<double>(ctx, ics, n, omega_p, dt, nsteps, out)
                                      : trajectory_impl<float>(ctx, ics, n, omega_p, dt, nsteps, out);
}

template <typename T>
static sw_status poteval_impl(sw_ctx* ctx, const double* xyz, int64_t n, double* phi, double* acc)
{
    double *dx = nullptr, *dp = nullptr, *da = nullptr;
    cudaError_t e;
    sw_status st = SW_OK;
    if ((e = cudaMalloc(&dx, 3 * n * sizeof(double))) || (e = cudaMalloc(&dp, n * sizeof(double))) ||
        (e = cudaMalloc(&da, 3 * n * sizeof(double)))) {
        st = ctx->cuda_fail(e, "potential buffers");
    } else if ((e = cudaMemcpyAsync(dx, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
               (e = launch_poteval<T>(ctx, make_field<T>(ctx), dx, n, dp, da)) ||
               (e = cudaMemcpyAsync(phi, dp, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
               (e = cudaMemcpyAsync(acc, da, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
               (e = cudaStreamSynchronize(ctx->stream))) {
        st = ctx->cuda_fail(e, "potential eval");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(dx); cudaFree(dp); cudaFree(da);
    return st;
}

extern "C" sw_status sw_potential_eval(sw_ctx* ctx, const double* xyz, int64_t n, double* phi_out, double* acc_out)
{
    CHECK_CTX(ctx);
    if (!xyz || !phi_out || !acc_out || n <= 0) { set_error(ctx, "sw_potential_eval: bad arguments"); return SW_EINVAL; }
    if (!ctx->has_pot) { set_error(ctx, "set the potential first"); return SW_ESTATE; }
    cudaSetDevice(ctx->device);
    return ctx->prec == SW_FP64_PLAIN ? poteval_impl<double>(ctx, xyz, n, phi_out, acc_out)
                                      : poteval_impl<float>(ctx, xyz, n, phi_out, acc_out);
}

// ---------------------------------------------------------------------------
// Profiling
// ---------------------------------------------------------------------------
extern "C" sw_status sw_set_profiling(sw_ctx* ctx, int enable)
{
    CHECK_CTX(ctx);
    ctx->prof = enable != 0;
    return SW_OK;
}

extern "C" int sw_kernel_count(void) { return K_COUNT; }

extern "C" sw_status sw_kernel_stats(sw_ctx* ctx, int k, const char** name, int64_t* launches, double* total_ms)
{
    CHECK_CTX(ctx);
    if (k < 0 || k >= K_COUNT) return SW_EINVAL;
    ctx->harvest();
    if (name) *name = kKernelNames[k];
    if (launches) *launches = ctx->k_launch[k];
    if (total_ms) *total_ms = ctx->k_ms[k];
    return SW_OK;
}

namespace sw {
const int kKernelWorkKind[K_COUNT] = {
    W_BYTES /*ics_soa*/, W_ORBIT_STEPS /*orbit_bin*/, W_ORBIT_STEPS /*orbit_drift*/, W_BYTES /*zero_flagged*/,
    W_BYTES /*finalize*/, W_NONE /*trajectory*/, W_NONE /*poteval*/, W_BYTES /*whiten*/, W_FLOP_TENSOR /*gram_tc*/,
    W_FLOP_SIMT /*gram_simt*/, W_NONE /*shift*/, W_FLOP_SIMT /*potrf_diag*/, W_FLOP_SIMT /*trsm_panel*/,
    W_FLOP_SIMT /*syrk_update*/, W_FLOP_SIMT /*trinv_diag*/, W_FLOP_SIMT /*trinv_update*/, W_BYTES /*gemv_n*/,
    W_BYTES /*gemv_t*/, W_BYTES /*trmv_l*/, W_BYTES /*trmv_lt*/, W_NONE /*admm_update*/, W_BYTES /*residual*/,
    W_BYTES /*gradient*/, W_NONE /*chi2*/, W_NONE /*misc*/, W_ORBIT_STEPS /*batch_orbit*/, W_FLOP_SIMT /*mlp_fwd*/,
    W_FLOP_SIMT /*mlp_bwd*/, W_NONE /*adam*/, W_BYTES /*reduce_gh*/, W_NONE /*pcg*/, W_BYTES /*bundle*/,
    W_FLOP_SIMT /*cholesky_inverse*/, W_FLOP_TENSOR /*syrk_tc*/, W_FLOP_TENSOR /*trinv_tc*/,
    W_FLOP_SIMT /*border*/};

void add_work(sw_ctx* ctx, int kid, double units)
{
    if (ctx && ctx->prof && kid >= 0 && kid < K_COUNT) ctx->k_work[kid] += units;
}
}  // namespace sw

extern "C" sw_status sw_kernel_work(sw_ctx* ctx, int k, double* work, int* kind)
{
    if (!ctx || k < 0 || k >= K_COUNT) return SW_EINVAL;
    if (work) *work = ctx->k_work[k];
    if (kind) *kind = kKernelWorkKind[k];
    return SW_OK;
}

extern "C" sw_status sw_reset_stats(sw_ctx* ctx)
{
    CHECK_CTX(ctx);
    ctx->harvest();
    for (int k = 0; k < K_COUNT; ++k) { ctx->k_launch[k] = 0; ctx->k_ms[k] = 0.0; ctx->k_work[k] = 0.0; }
    return SW_OK;
}

extern "C" int64_t sw_launch_count(const sw_ctx* ctx) { return ctx ? ctx->launches : 0; }
extern "C" int64_t sw_alloc_count(const sw_ctx* ctx) { return ctx ? ctx->n_alloc : -1; }

extern "C" sw_status sw_set_option(sw_ctx* ctx, const char* key, double value)
{
    CHECK_CTX(ctx);
    if (!key) return SW_EINVAL;
    if (!strcmp(key, "ej_every")) {
        if (!(value >= 1 && value <= 1e6)) return SW_EINVAL;
        ctx->opt.ej_every = (int)value;
    } else if (!strcmp(key, "admm_max_iter")) {
        if (!(value >= 1)) return SW_EINVAL;
        ctx->opt.admm_max_iter = (int)value;
    } else if (!strcmp(key, "admm_tol")) {
        if (!(value > 0)) return SW_EINVAL;
        ctx->opt.admm_tol = value;
    } else if (!strcmp(key, "refine_max")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.refine_max = (int)value;
    } else if (!strcmp(key, "kkt_tol")) {
        if (!(value > 0)) return SW_EINVAL;
        ctx->opt.kkt_tol = value;
    } else if (!strcmp(key, "check_every")) {
        if (!(value >= 1)) return SW_EINVAL;
        ctx->opt.check_every = (int)value;
    } else if (!strcmp(key, "admm_rho")) {
        if (!(value > 0)) return SW_EINVAL;
        ctx->opt.admm_rho = value;
    } else if (!strcmp(key, "admm_rho_cspace")) {
        if (!(value > 0)) return SW_EINVAL;
        ctx->opt.admm_rho_cs = value;
    } else if (!strcmp(key, "admm_alpha")) {
        if (!(value > 0 && value < 2)) return SW_EINVAL;
        ctx->opt.admm_alpha = value;
    } else if (!strcmp(key, "chi2_tol")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.chi2_tol = value;
    } else if (!strcmp(key, "polish_solves")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.polish_solves = (int)value;
    } else if (!strcmp(key, "polish_max")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.polish_max = (int)value;
    } else if (!strcmp(key, "large_solver")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.large_solver = (int)value;
    } else if (!strcmp(key, "as_block")) {
        if (!(value >= 1)) return SW_EINVAL;
        ctx->opt.as_block = (int)value;
    } else if (!strcmp(key, "as_candidates")) {
        if (!(value >= 0.0)) return SW_EINVAL;
        ctx->opt.as_candidates = value;
    } else if (!strcmp(key, "solver")) {
        if (!(value == 0 || value == 1 || value == 2)) return SW_EINVAL;
        ctx->opt.solver = (int)value;
    } else if (!strcmp(key, "chol_coop")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_coop = (int)value;
    } else if (!strcmp(key, "matrix_cache")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.matrix_cache = (int)value;
        if (!value) {
            cudaSetDevice(ctx->device);
            for (auto& b : ctx->mat_cache) cudaFree(b.first);
            ctx->mat_cache.clear();
        }
    } else if (!strcmp(key, "project_bundle")) {
        if (!(value >= 1.0 && value <= 1024.0 && value == std::floor(value))) return SW_EINVAL;
        ctx->opt.project_bundle = (int)value;
    } else if (!strcmp(key, "as_border")) {
        if (!(value >= 0 && value <= 4096 && value == std::floor(value))) return SW_EINVAL;
        ctx->opt.as_border = (int)value;
    } else if (!strcmp(key, "as_mask")) {
        if (!(value >= 0.0 && value <= 1.0)) return SW_EINVAL;
        ctx->opt.as_mask = value;
    } else if (!strcmp(key, "boot_p0_extra")) {
        if (!(value >= 0.0 && value <= 4.0)) return SW_EINVAL;
        ctx->opt.boot_p0_extra = value;
    } else if (!strcmp(key, "chol_panel_tc")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_panel_tc = (int)value;
    } else if (!strcmp(key, "chol_super")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_super = (int)value;
    } else if (!strcmp(key, "chol_pdl")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_pdl = (int)value;
    } else if (!strcmp(key, "chol_reserve_sms")) {
        if (!(value >= 0 && value <= 128 && value == std::floor(value))) return SW_EINVAL;
        ctx->opt.chol_reserve_sms = (int)value;
    } else if (!strcmp(key, "chol_lookahead")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_lookahead = (int)value;
    } else if (!strcmp(key, "chol_tc")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.chol_tc = (int)value;
    } else if (!strcmp(key, "integrator")) {
        if (!(value == 0 || value == 1)) return SW_EINVAL;
        ctx->opt.integrator = (int)value;
    } else if (!strcmp(key, "bs3_rtol")) {
        if (!(value > 0.0 && value < 1.0)) return SW_EINVAL;
        ctx->opt.bs3_rtol = value;
    } else if (!strcmp(key, "as_grow")) {
        if (!(value >= 0.0)) return SW_EINVAL;
        ctx->opt.as_grow = value;
    } else if (!strcmp(key, "as_cg_tol")) {
        if (!(value > 0.0)) return SW_EINVAL;
        ctx->opt.as_cg_tol = value;
    } else if (!strcmp(key, "as_cg_max")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.as_cg_max = (int)value;
    } else if (!strcmp(key, "as_solves")) {
        if (!(value >= 1)) return SW_EINVAL;
        ctx->opt.as_solves = (int)value;
    } else if (!strcmp(key, "inner_refine")) {
        if (!(value >= 0 && value <= 8)) return SW_EINVAL;
        ctx->opt.inner_refine = (int)value;
    } else if (!strcmp(key, "verbose")) {
        ctx->opt.verbose = (int)value;
    } else if (!strcmp(key, "working_set")) {
        ctx->opt.working_set = value != 0;
    } else if (!strcmp(key, "orbit_direct_max")) {
        if (!(value >= 0)) return SW_EINVAL;
        ctx->opt.orbit_direct_max = (int64_t)value;
    } else if (!strcmp(key, "ws_factor")) {
        if (!(value > 0)) return SW_EINVAL;
        ctx->opt.ws_factor = value;
    } else if (!strcmp(key, "ws_rounds")) {
        if (!(value >= 1)) return SW_EINVAL;
        ctx->opt.ws_rounds = (int)value;
    } else if (!strcmp(key, "gram_tensor_cores")) {
        ctx->opt.gram_tc = value != 0;
    } else {
        set_error(ctx, "unknown option '%s'", key);
        return SW_EINVAL;
    }
    return SW_OK;
}
