// Batched model construction: many trial potentials (each with its own orbit
// count, pattern speed and viewing angles, one shared observation grid) built in
// one persistent launch that is captured once in a CUDA graph and replayed.
//
// The paper evaluates one model at a time inside its MCMC (Sec. 3.2) and
// batches only the bootstrap NNLS solves of one model (Sec. 2.4).  Here every
// model's orbit state sits in one SoA array, every model's matrix in one
// column block of a single allocation, and a work queue of (model, orbit tile)
// items lets CTAs that finish a short model move on to the next, so uneven
// orbit counts do not leave SMs idle.  The launch shape (threads per CTA and
// CTAs in the persistent grid) is chosen by timing short probe runs of the
// actual models on the first run.
#include "sw_common.cuh"
#include "sw_api_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

using namespace sw;

struct sw_batch {
    sw_ctx* ctx = nullptr;
    int n_models = 0;
    int64_t nsteps = 0, ntot = 0, M = 0, npix = 0, nd = 0;
    int gh = 0, mirror4 = 1, elem = 4;
    sw_pixel_grid pix{};
    sw_vbins vb{};
    sw_density_grid dens{};
    std::vector<int64_t> n_orb, col_off;
    void *U = nullptr, *soa = nullptr, *cs = nullptr, *ghtab = nullptr, *models = nullptr;
    int2* items = nullptr;
    int* next = nullptr;
    double* drift = nullptr;
    uint8_t* status = nullptr;
    int n_items = 0;
    std::vector<sw_matrix> views;
    bool models_set = false, tuned = false, have_graph = false;
    int threads = 128, grid = 0, ej_every = 8;   // grid: set from the device's SM count at creation
    int pot = 0;                                  // 1: every model is disc + halo + Long-Murali bar (FP32 kernel)
    std::vector<double> tune_ms;   // per candidate, in candidate order
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kThreads[3] = {64, 128, 256};
constexpr int kCtasPerSm[4] = {1, 2, 4, 8};

void free_batch(sw_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void* bufs[] = {b->U, b->soa, b->cs, b->ghtab, b->models, b->items, b->next, b->drift, b->status};
    for (void* p : bufs)
        if (p) cudaFree(p);
    cudaGetLastError();
}

sw_status build_items(sw_batch* b, int threads)
{
    std::vector<int2> it;
    for (int k = 0; k < b->n_models; ++k)
        for (int64_t f = 0; f < b->n_orb[k]; f += threads) it.push_back(make_int2(k, (int)f));
    if (b->items) cudaFree(b->items);
    b->items = nullptr;
    cudaError_t e = cudaMalloc(&b->items, std::max<size_t>(1, it.size()) * sizeof(int2));
    if (!e) e = cudaMemcpyAsync(b->items, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice, b->ctx->stream);
    if (!e) e = cudaStreamSynchronize(b->ctx->stream);
    if (e) return b->ctx->cuda_fail(e, "batch work items");
    b->n_items = (int)it.size();
    return SW_OK;
}

// the work of one run, enqueued on the context stream (also what the graph holds)
template <typename T>
cudaError_t enqueue(sw_batch* b, int64_t nsteps)
{
    sw_ctx* ctx = b->ctx;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(b->U, 0, (size_t)b->M * b->ntot * sizeof(T), st);
    if (!e) e = cudaMemsetAsync(b->next, 0, sizeof(int), st);
    if (!e)
        e = launch_batch_orbit_bin<T>(st, b->threads, b->grid, b->gh, b->pot, (const ModelT<T>*)b->models, b->items,
                                      b->n_items, b->next, (const T*)b->soa, b->ntot, nsteps, b->ej_every, b->drift,
                                      b->status);
    if (!e) e = launch_zero_flagged<T>(ctx, b->U, b->M, b->ntot, b->status);
    const int64_t count_rows = b->gh ? b->nd + b->npix : b->M;
    const double norm = 1.0 / ((b->mirror4 ? 4.0 : 1.0) * (double)b->nsteps);
    if (!e) e = launch_finalize<T>(ctx, b->U, b->M, b->ntot, count_rows, norm);
    return e;
}

template <typename T>
sw_status autotune(sw_batch* b)
{
    sw_ctx* ctx = b->ctx;
    const int64_t probe = std::min<int64_t>(b->nsteps, 128);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = ctx->prof;
    ctx->prof = false;
    double best = 1e300;
    const int sms = ctx_sms(ctx);
    int best_t = 128, best_g = sms * 2;
    b->tune_ms.clear();
    sw_status s = SW_OK;
    for (int t : kThreads) {
        if ((s = build_items(b, t)) != SW_OK) break;
        for (int c : kCtasPerSm) {
            b->threads = t;
            b->grid = sms * c * (128 / t > 0 ? 128 / t : 1);
            if (b->grid < 1) b->grid = 1;
            cudaEventRecord(e0, ctx->stream);
            cudaError_t e = enqueue<T>(b, probe);
            cudaEventRecord(e1, ctx->stream);
            if (!e) e = cudaEventSynchronize(e1);
            if (e) { s = ctx->cuda_fail(e, "batch autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            b->tune_ms.push_back(ms);
            if (ms < best) { best = ms; best_t = t; best_g = b->grid; }
        }
        if (s != SW_OK) break;
    }
    ctx->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SW_OK) return s;
    b->threads = best_t;
    b->grid = best_g;
    b->tuned = true;
    return build_items(b, best_t);
}

template <typename T>
sw_status run_impl(sw_batch* b)
{
    sw_ctx* ctx = b->ctx;
    if (!b->tuned) {
        sw_status s = autotune<T>(b);
        if (s != SW_OK) return s;
    }
    if (!b->have_graph) {
        const bool prof = ctx->prof;
        ctx->prof = false;
        cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            cudaError_t ee = enqueue<T>(b, b->nsteps);
            e = cudaStreamEndCapture(ctx->stream, &b->graph);
            if (ee) e = ee;
        }
        if (!e) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        ctx->prof = prof;
        if (e) {   // capture unavailable on this stream: launch the same work directly
            cudaGetLastError();
            if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
            b->exec = nullptr;
        } else {
            b->have_graph = true;
        }
    }
    cudaError_t e;
    {
        LaunchTimer lt(ctx, K_BATCH_ORBIT);
        add_work(ctx, K_BATCH_ORBIT, (double)b->ntot * (double)b->nsteps);
        if (b->have_graph) {
            e = cudaGraphLaunch(b->exec, ctx->stream);
        } else {
            const bool prof = ctx->prof;
            ctx->prof = false;
            e = enqueue<T>(b, b->nsteps);
            ctx->prof = prof;
        }
    }
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return ctx->cuda_fail(e, "batched model construction");
    return SW_OK;
}

template <typename T>
sw_status set_models_impl(sw_batch* b, const sw_potential_params* pots, const double* omega_p, const double* angles,
                          double dt, const double* ics, const double* gh_v0_s)
{
    sw_ctx* ctx = b->ctx;
    const int K = b->n_models;
    std::vector<ModelT<T>> ms(K);
    std::vector<T> cs_all((size_t)K * 2 * (b->nsteps + 1));
    std::vector<T> tab(b->gh ? (size_t)K * b->npix * 2 : 0);
    for (int k = 0; k < K; ++k) {
        sw_status s = check_potential(ctx, &pots[k]);
        if (s != SW_OK) return s;
        if (!std::isfinite(omega_p[k]) || !std::isfinite(angles[3 * k]) || !std::isfinite(angles[3 * k + 1]) ||
            !std::isfinite(angles[3 * k + 2])) {
            set_error(ctx, "sw_batch_set_models: model %d has a non-finite pattern speed or angle", k);
            return SW_EINVAL;
        }
        double Mdm, rs;
        halo_constants(pots[k], Mdm, rs);
        ModelT<T>& m = ms[k];
        m = ModelT<T>{};
        m.f = make_field_from<T>(pots[k], Mdm, rs);
        m.g = make_grid<T>(angles[3 * k], angles[3 * k + 1], angles[3 * k + 2], &b->pix, b->gh ? nullptr : &b->vb,
                           &b->dens, b->gh, b->mirror4);
        m.dt = (T)dt;
        m.half_dt = (T)(0.5 * dt);
        m.omega = (T)omega_p[k];
        std::vector<T> cs;
        cs_table<T>(cs, omega_p[k], dt, b->nsteps);
        std::copy(cs.begin(), cs.end(), cs_all.begin() + (size_t)k * 2 * (b->nsteps + 1));
        m.cs = (const T*)b->cs + (size_t)k * 2 * (b->nsteps + 1);
        if (b->gh) {
            for (int64_t p = 0; p < b->npix; ++p) {
                const double v0 = gh_v0_s[((size_t)k * b->npix + p) * 2], sg = gh_v0_s[((size_t)k * b->npix + p) * 2 + 1];
                if (!(sg > 0.0) || !std::isfinite(sg) || !std::isfinite(v0)) {
                    set_error(ctx, "sw_batch_set_models: GH reference of model %d pixel %lld is invalid", k,
                              (long long)p);
                    return SW_EINVAL;
                }
                tab[((size_t)k * b->npix + p) * 2] = (T)v0;
                tab[((size_t)k * b->npix + p) * 2 + 1] = (T)(1.0 / sg);
            }
            m.gh_v0s = (const T*)b->ghtab + (size_t)k * b->npix * 2;
        }
        m.U = (char*)b->U + (size_t)b->col_off[k] * b->M * sizeof(T);
        m.n_orb = b->n_orb[k];
        m.orbit_base = b->col_off[k];
        m.ldu = b->M;
    }
    for (int64_t i = 0; i < 6 * b->ntot; ++i)
        if (!std::isfinite(ics[i])) {
            set_error(ctx, "sw_batch_set_models: non-finite initial condition");
            return SW_EINVAL;
        }
    cudaStream_t st = ctx->stream;
    double* aos = nullptr;
    cudaError_t e = cudaMalloc(&aos, (size_t)b->ntot * 6 * sizeof(double));
    if (!e) e = cudaMemcpyAsync(aos, ics, (size_t)b->ntot * 6 * sizeof(double), cudaMemcpyHostToDevice, st);
    if (!e) e = launch_ics_to_soa<T>(ctx, aos, b->ntot, (T*)b->soa, b->ntot);
    if (!e) e = cudaMemcpyAsync(b->cs, cs_all.data(), cs_all.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (!e && b->gh) e = cudaMemcpyAsync(b->ghtab, tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b->models, ms.data(), ms.size() * sizeof(ModelT<T>), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (aos) cudaFree(aos);
    if (e) return ctx->cuda_fail(e, "batch model upload");
    // the kernel's potential layout: a captured graph holds the kernel of the layout it was captured with
    int pot = sizeof(T) == 4 ? 1 : 0;
    for (int k = 0; k < K && pot; ++k) {
        const FieldT<T>& f = ms[k].f;
        if (!(f.has_disc && f.has_halo && f.has_bar && f.bar_kind == 0 && f.test_kind == 0)) pot = 0;
    }
    if (pot != b->pot && b->have_graph) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        b->have_graph = false;
    }
    b->pot = pot;
    b->models_set = true;
    return SW_OK;
}

}  // namespace

extern "C" sw_status sw_batch_create(sw_ctx* ctx, int n_models, const int64_t* n_orb, int64_t nsteps,
                                     const sw_pixel_grid* pix, const sw_vbins* vb, const sw_density_grid* dens,
                                     int gh, int mirror4, sw_batch** out)
{
    CHECK_CTX(ctx);
    if (!out || !n_orb || !pix || !dens || (!gh && !vb) || n_models < 1 || nsteps < 1) {
        set_error(ctx, "sw_batch_create: NULL argument, no models or no steps");
        return SW_EINVAL;
    }
    *out = nullptr;
    if (ctx->opt.integrator != 0) {
        set_error(ctx, "sw_batch_create: the batched launch integrates with kick-drift-kick only (option integrator = 0)");
        return SW_EINVAL;
    }
    if (pix->nx <= 0 || pix->ny <= 0 || !(pix->dx > 0) || !(pix->dy > 0) || dens->nR <= 0 || dens->nphi <= 0 ||
        dens->nz <= 0 || !(dens->Rmax > 0) || !(dens->zmax > dens->zmin) ||
        (!gh && (vb->nv <= 0 || !(vb->dv > 0)))) {
        set_error(ctx, "sw_batch_create: invalid grid");
        return SW_EINVAL;
    }
    sw_batch* b = new sw_batch();
    b->ctx = ctx;
    b->grid = ctx_sms(ctx) * 4;
    b->n_models = n_models;
    b->nsteps = nsteps;
    b->gh = gh != 0;
    b->mirror4 = mirror4 != 0;
    b->elem = ctx->prec == SW_FP64_PLAIN ? 8 : 4;
    b->pix = *pix;
    if (vb) b->vb = *vb;
    b->dens = *dens;
    b->ej_every = ctx->opt.ej_every;
    b->nd = (int64_t)dens->nR * dens->nphi * dens->nz;
    b->npix = (int64_t)pix->nx * pix->ny;
    b->M = b->nd + b->npix + (b->gh ? 4 * b->npix : b->npix * (int64_t)vb->nv);
    b->n_orb.assign(n_orb, n_orb + n_models);
    for (int k = 0; k < n_models; ++k) {
        if (n_orb[k] < 1 || n_orb[k] > ((int64_t)1 << 30)) {
            delete b;
            set_error(ctx, "sw_batch_create: model %d has %lld orbits", k, (long long)n_orb[k]);
            return SW_EINVAL;
        }
        b->col_off.push_back(b->ntot);
        b->ntot += n_orb[k];
    }
    const size_t T = b->elem, rows = T == 4 ? 12 : 6;
    cudaError_t e = cudaMalloc(&b->U, (size_t)b->M * b->ntot * T);
    if (!e) e = cudaMalloc(&b->soa, rows * b->ntot * T);
    if (!e) e = cudaMalloc(&b->cs, (size_t)n_models * 2 * (nsteps + 1) * T);
    if (!e) e = cudaMalloc(&b->ghtab, std::max<size_t>(1, (size_t)n_models * b->npix * 2 * T));
    if (!e) e = cudaMalloc(&b->models, (size_t)n_models * (T == 4 ? sizeof(ModelT<float>) : sizeof(ModelT<double>)));
    if (!e) e = cudaMalloc(&b->next, sizeof(int));
    if (!e) e = cudaMalloc(&b->drift, (size_t)b->ntot * sizeof(double));
    if (!e) e = cudaMalloc(&b->status, (size_t)b->ntot);
    if (e) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        set_error(ctx, "sw_batch_create: device allocation failed");
        return SW_ENOMEM;
    }
    b->views.resize(n_models);
    for (int k = 0; k < n_models; ++k) {
        sw_matrix& v = b->views[k];
        v.ctx = ctx;
        v.M = b->M; v.N = n_orb[k]; v.nd = b->nd; v.npix = b->npix; v.nkin = b->M - b->nd - b->npix;
        v.gh = b->gh; v.elem = (int)T; v.ncopy = b->mirror4 ? 4 : 1; v.device = ctx->device; v.nsteps = nsteps;
        v.nv = b->gh ? 0 : vb->nv; v.v0 = b->gh ? 0.0 : vb->v0; v.dv = b->gh ? 1.0 : vb->dv;
        v.d = (char*)b->U + (size_t)b->col_off[k] * b->M * T;
        v.borrowed = true;
    }
    sw_status s = build_items(b, b->threads);
    if (s != SW_OK) { free_batch(b); delete b; return s; }
    ctx->live_matrices++;   // the batch keeps its context alive like a matrix does
    *out = b;
    return SW_OK;
}

extern "C" sw_status sw_batch_set_models(sw_batch* b, const sw_potential_params* pots, const double* omega_p,
                                         const double* angles, double dt, const double* ics, const double* gh_v0_s)
{
    if (!b) return SW_EINVAL;
    sw_ctx* ctx = b->ctx;
    CHECK_CTX(ctx);
    if (!pots || !omega_p || !angles || !ics || (b->gh && !gh_v0_s) || !(dt > 0) || !std::isfinite(dt)) {
        set_error(ctx, "sw_batch_set_models: NULL argument or bad dt");
        return SW_EINVAL;
    }
    return b->elem == 8 ? set_models_impl<double>(b, pots, omega_p, angles, dt, ics, gh_v0_s)
                        : set_models_impl<float>(b, pots, omega_p, angles, dt, ics, gh_v0_s);
}

extern "C" sw_status sw_batch_run(sw_batch* b)
{
    if (!b) return SW_EINVAL;
    sw_ctx* ctx = b->ctx;
    CHECK_CTX(ctx);
    if (!b->models_set) { set_error(ctx, "sw_batch_run: set the models first"); return SW_ESTATE; }
    if (ctx->opt.integrator != 0) {
        set_error(ctx, "sw_batch_run: the batched launch integrates with kick-drift-kick only (option integrator = 0)");
        return SW_EINVAL;
    }
    for (auto& v : b->views) ctx->solve_ws.forget_matrix(&v);
    return b->elem == 8 ? run_impl<double>(b) : run_impl<float>(b);
}

extern "C" sw_status sw_batch_matrix(sw_batch* b, int k, sw_matrix** view)
{
    if (!b || !view || k < 0 || k >= b->n_models) return SW_EINVAL;
    *view = &b->views[k];
    return SW_OK;
}

extern "C" sw_status sw_batch_stats(sw_batch* b, double* drift_out, uint8_t* status_out)
{
    if (!b) return SW_EINVAL;
    sw_ctx* ctx = b->ctx;
    CHECK_CTX(ctx);
    cudaError_t e = cudaSuccess;
    if (drift_out) e = cudaMemcpyAsync(drift_out, b->drift, b->ntot * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (!e && status_out) e = cudaMemcpyAsync(status_out, b->status, b->ntot, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    return e ? ctx->cuda_fail(e, "batch stats") : SW_OK;
}

extern "C" sw_status sw_batch_info(const sw_batch* b, int64_t* info4, double* tune_ms12)
{
    if (!b || !info4) return SW_EINVAL;
    info4[0] = b->threads;
    info4[1] = b->grid;
    info4[2] = b->tuned ? 1 : 0;
    info4[3] = b->have_graph ? 1 : 0;
    if (tune_ms12)
        for (int i = 0; i < 12; ++i) tune_ms12[i] = i < (int)b->tune_ms.size() ? b->tune_ms[i] : -1.0;
    return SW_OK;
}

extern "C" sw_status sw_batch_destroy(sw_batch* b)
{
    if (!b) return SW_OK;
    if (!b->ctx->destroyed) {
        cudaSetDevice(b->ctx->device);
        cudaStreamSynchronize(b->ctx->stream);
        for (auto& v : b->views) b->ctx->solve_ws.forget_matrix(&v);
    }
    sw_ctx* ctx = b->ctx;
    if (ctx->destroyed) cudaSetDevice(ctx->device);
    free_batch(b);
    delete b;
    if (--ctx->live_matrices == 0 && ctx->destroyed) delete ctx;
    return SW_OK;
}
