// Context and matrix objects behind the opaque C-ABI handles (internal).
#pragma once
#include "sw_common.cuh"

#include <string>
#include <vector>

struct sw_matrix;

namespace sw {

struct Options {
    int ej_every = 1;            // Jacobi-energy check interval (steps) in the projection pass
    int admm_max_iter = 400;     // ADMM iteration cap per run
    double admm_tol = 1e-6;      // ADMM stop: ||w-z||inf, rho||z-z_prev||inf <= tol * max(1, ||z||inf)
    int refine_max = 8;          // refinement rounds with FP64 residuals
    double kkt_tol = 1e-9;       // KKT stop: ||P(grad)||inf <= kkt_tol * max|q|
    int check_every = 20;        // ADMM iterations between host convergence checks
    double admm_rho = 0.01;      // ADMM penalty relative to each orbit's Gram diagonal (orbit space)
    double admm_rho_cs = 1.0;    // the same in constraint space (the Woodbury form cancels digits for small rho)
    double admm_alpha = 1.6;     // over-relaxation
    double chi2_tol = 1e-6;      // refinement also stops once chi^2 changes by less than this (relative)
    int64_t orbit_direct_max = 8192;  // N > M up to this size: orbit space on all orbits
    int polish_max = 2048;       // largest support solved exactly by the active-set polish (0: off)
    int polish_solves = 400;     // cap on reduced solves per polish
    bool working_set = true;     // N > M: orbit-space solves on a working set instead of the Woodbury form
    double ws_factor = 0.6;      // initial working-set size in units of M
    int ws_rounds = 6;           // working-set exchange rounds
    int verbose = 0;        // solver progress on stderr
    int inner_refine = 1;        // refinement steps of each ADMM linear solve against the kept Gram
    int large_solver = 0;        // N > orbit_direct_max: 0 block active set, 1 ADMM working set
    int as_block = 1024;         // active set: violators entering per pivoting step
    double as_candidates = 0;    // active set: initial candidate-set size (0: 2 M)
    double as_grow = 0.0;        // active set: at most max(as_block, as_grow |F|) orbits enter per step
    int solver = 0;              // 0 auto, 1 active set, 2 ADMM (see solve_dispatch)
    int chol_coop = 0;           // Cholesky + inverse in one cooperative launch (0: per-step launches)
    int chol_tc = 1;             // FP32 Cholesky + inverse with tcgen05 trailing updates (0: SIMT, 64-wide)
    int chol_lookahead = 1;      // tensor-core factorisation: bulk updates on a second stream (1) or in line (0)
    int chol_reserve_sms = 8;    // tensor-core factorisation: SMs the bulk updates leave to the next steps' chain
    double boot_p0_extra = 0.0;  // bootstrap: factored set = the plain solve's support plus this fraction of near-active orbits
    int chol_pdl = 1;            // tensor-core factorisation: panel launched programmatically behind its diagonal block
    int chol_panel_tc = 0;       // tensor-core factorisation: panels on the tensor cores (BF16 hi + lo split) or FP32 SIMT
    int chol_super = 1;          // tensor-core factorisation: 256-wide super-steps (rank-256 bulk updates) or 128-wide steps
    int project_bundle = 1;      // orbits per column of sw_project's matrix (bundles accumulated at bin time)
    int matrix_cache = 1;        // keep freed matrix buffers for reuse by the next matrices of this context
    int integrator = 0;          // 0: kick-drift-kick at fixed dt; 1: adaptive Bogacki-Shampine 3(2) in the bar frame
    double bs3_rtol = 1e-4;      // relative tolerance of the adaptive integrator
    int as_cg_max = 200;         // active set: conjugate-gradient steps per reduced solve
    int as_border = 256;         // active set: at most this many entering orbits appended to the factor (0: refactor)
    double as_mask = 0.02;       // active set: largest fraction of the factored set masked before refactoring
    double as_cg_tol = 0.05;     // active set: CG stops at max|r| <= as_cg_tol * kkt_tol * max|q|
    int as_solves = 400;         // active set: cap on reduced solves
    bool gram_tc = true;         // tcgen05 BF16 Gram (FP32 path); false: SIMT FP32 Gram
};

// Device workspace of the weight solve, sized for the largest problem seen.
struct SolveWS {
    void* A = nullptr; size_t A_cap = 0;          // whitened matrix (BF16 or FP64), K-major for the Gram
    void* Alo = nullptr; size_t Alo_cap = 0;      // BF16 rounding residual of A (hi/lo split)
    void* Uc = nullptr; size_t Uc_cap = 0;        // working-set columns of U
    void* outer = nullptr; size_t outer_cap = 0;  // working-set driver vectors
    void* G = nullptr; size_t G_cap = 0;          // K x K Gram, Cholesky factor in place
    void* Gs = nullptr; size_t Gs_cap = 0;        // symmetric copy of Gram + I (step refinement)
    void* X = nullptr; size_t X_cap = 0;          // K x K inverse of the Cholesky factor
    void* D = nullptr; size_t D_cap = 0;          // nb x nb diagonal-block scratch
    void* vec = nullptr; size_t vec_cap = 0;      // vectors
    void* R = nullptr; size_t R_cap = 0;          // polish: gathered whitened rows (FP64)
    void* H = nullptr; size_t H_cap = 0;          // polish: reduced normal matrix (FP64)
    void* Hi = nullptr; size_t Hi_cap = 0;        // polish: inverse of its Cholesky factor
    void* pv = nullptr; size_t pv_cap = 0;        // polish: index list and vectors
    void* boot = nullptr; size_t boot_cap = 0;    // bootstrap solves: realisation data and vectors
    // the last passive Gram of the active set (scaled, before the ridge), kept so that the next
    // passive set recomputes only the tile rows of its entering orbits: two buffers (the last and
    // the next), the orbits in the last one's order and each orbit's position in it
    void* Gc[2] = {nullptr, nullptr}; size_t Gc_cap[2] = {0, 0};
    void* gcidx = nullptr; size_t gcidx_cap = 0;
    void* Mc = nullptr; size_t Mc_cap = 0;        // correction of the masked orbits: X's columns, H_DD^-1
    int gc_cur = 0;
    int64_t gc_ld = 0;
    std::vector<int64_t> gc_set, gc_pos;
    const sw_matrix* A_of = nullptr;              // which matrix A was built from
    void release();
    void forget_matrix(const sw_matrix* U) { if (A_of == U) A_of = nullptr; gc_set.clear(); }
};

struct LaunchRec {
    int id;
    cudaEvent_t a, b;
};

}  // namespace sw

struct sw_ctx {
    int device = 0;
    int n_sm = 1;                  // streaming multiprocessors of the device (queried at creation)
    int64_t n_alloc = 0;           // device allocations made by ensure() since creation
    sw_precision prec = SW_FP32_KAHAN;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    sw::Options opt;
    // potential
    sw_potential_params pot{};
    bool has_pot = false;
    double Mdm = 0.0, rs = 1.0;
    // orbit library
    int64_t n_orb = 0, nsteps = 0;
    double omega = 0.0, dt = 0.0;
    bool has_lib = false;
    void* d_soa = nullptr; size_t soa_cap = 0;
    void* d_cs = nullptr; size_t cs_cap = 0;
    double* d_aos = nullptr; size_t aos_cap = 0;
    double* d_drift = nullptr; size_t drift_cap = 0;
    uint8_t* d_status = nullptr; size_t status_cap = 0;
    unsigned long long* d_stats = nullptr;
    void* d_ghtab = nullptr; size_t ghtab_cap = 0;
    int64_t last_proj_n = 0;
    void* d_mlp = nullptr; size_t mlp_cap = 0;   // MLP activations
    void* d_split = nullptr; size_t split_cap = 0;   // FP64 vectors split into float hi + lo
    void* d_chol = nullptr; size_t chol_cap = 0;     // cooperative Cholesky: diagonal inverses, barrier
    void* d_chol_tc = nullptr; size_t chol_tc_cap = 0;   // tensor-core Cholesky: diagonal inverse, BF16 panels
    void* d_cut = nullptr; size_t cut_cap = 0;           // bundled projection: indices of cut realisations
    void* d_invsig_f = nullptr; size_t invsig_f_cap = 0; // whitening: 1/sigma in FP32
    // device buffers of freed matrices, kept for the next matrices (the orbit matrix of a model is
    // rebuilt at the same size for every model: a cudaMalloc / cudaFree of gigabytes per model avoided)
    std::vector<std::pair<void*, size_t>> mat_cache;
    void* d_ghw = nullptr; size_t ghw_cap = 0;            // GH weights of sw_reduce_gh
    void* d_ttotal = nullptr; size_t ttotal_cap = 0;   // per-orbit integration time (adaptive integrator)
    // solve
    sw::SolveWS solve_ws;
    double solve_info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // lifetime: matrices keep their context alive until the last one is freed
    int64_t live_matrices = 0;
    bool destroyed = false;
    // second stream (the factorisation's bulk updates) and dependency events between the two
    cudaStream_t stream2 = nullptr;
    std::vector<cudaEvent_t> dep_events;
    // profiling
    bool prof = false;
    std::vector<sw::LaunchRec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches = 0;
    int64_t k_launch[sw::K_COUNT] = {};
    double k_ms[sw::K_COUNT] = {};
    double k_work[sw::K_COUNT] = {};

    cudaEvent_t take_event();
    void harvest();
    sw_status cuda_fail(cudaError_t e, const char* what);
    sw_status ensure(void** p, size_t* cap, size_t need, const char* what);
    sw_status ensure_stats(int64_t n);
};

struct sw_matrix {
    sw_ctx* ctx = nullptr;
    int64_t M = 0, N = 0, nd = 0, npix = 0, nkin = 0;
    int gh = 0, elem = 4, ncopy = 4, device = 0;
    int64_t nsteps = 0;
    int nv = 0;            // velocity bins of a histogram matrix (0 in GH mode)
    double v0 = 0.0, dv = 1.0;
    void* d = nullptr;   // orbit-major: column i at d + i * M
    bool borrowed = false; // a view into a batch's storage: freed with the batch, not by sw_matrix_free
};

extern "C" sw_status sw_set_option(sw_ctx* ctx, const char* key, double value);

// shared by the single-model and batched paths (sw_api.cu)
namespace sw {
sw_status check_potential(sw_ctx* ctx, const sw_potential_params* p);
void halo_constants(const sw_potential_params& p, double& Mdm, double& rs);
}  // namespace sw
template <typename T>
sw::FieldT<T> make_field_from(const sw_potential_params& p, double Mdm, double rs);
template <typename T>
void cs_table(std::vector<T>& out, double omega, double dt, int64_t nsteps);
template <typename T>
sw::GridT<T> make_grid(double incl, double pa, double bar_angle, const sw_pixel_grid* pix, const sw_vbins* vb,
                       const sw_density_grid* dens, int gh, int mirror4);

// Entry-point prologue: reject a NULL or destroyed context, clear the last error
// message, select the context's device and drop a stale CUDA error.
#define CHECK_CTX(ctx)                                       \
    do {                                                     \
        if (!(ctx) || (ctx)->destroyed) return SW_EINVAL;    \
        (ctx)->err.clear();                                  \
        cudaSetDevice((ctx)->device);                        \
        cudaGetLastError();                                  \
    } while (0)
