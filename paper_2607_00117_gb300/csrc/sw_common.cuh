// Internal declarations shared by the libsw translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#include "../../include/sw.h"

#define SW_G 4.300917e-6

namespace sw {

// ---------------------------------------------------------------------------
// Potential constants, converted to the working precision T on the host.
// Disc: Miyamoto-Nagai; halo: NFW; bar: needle-convolved MN (n = 1, eta = 0);
// test: point mass (kind 1) or Plummer (kind 2).
// ---------------------------------------------------------------------------
template <typename T>
struct FieldT {
    T gm_disc, disc_a, disc_b2;
    T gm_halo, halo_rs, halo_inv_rs;
    T k_bar, bar_L, bar_a, bar_b2;     // k_bar = G M / (2 L)
    T gm_test, test_a2;
    // the paper's bar (bar_kind 1): T3 long bar (G M_1, a_1, b_1^2, L_1) and V4 bulge (G M_2, a_2, b_2^2,
    // L_2), and the 8-point Gauss-Legendre rule on [-1, 1] (positive nodes and their weights) used for
    // the V4 needle integrals
    T da_gm1, da_a1, da_b1sq, da_L1;
    T da_gm2, da_a2, da_b2sq, da_L2;
    T gl_x[4], gl_w[4];
    int test_kind;
    int has_disc, has_halo, has_bar;
    int bar_kind;                      // 0 Long-Murali needle (n = 1, eta = 0); 1 Dehnen-Aly T3 + V4
};

// Observation geometry: Euler matrix rows and bin grids.
template <typename T>
struct GridT {
    T R[9];                            // Rz(gamma) Rx(beta) Rz(alpha), row-major
    T x0, y0, inv_dx, inv_dy, dx, dy;
    T v0, inv_dv, dv;
    T dR, inv_dR, inv_dphi, dphi, zmin, inv_dz, dz;
    int nx, ny, nv, nR, nphi, nz;
    int gh, ncopy;
    int sym;                           // pixel and velocity grids symmetric about 0 (mirror copies by reflection)
    int64_t nd, npix, M;               // rows: density, pixel mass, kinematic block starts at nd + npix
};

// Per-model launch constants of the orbit kernel.
template <typename T>
struct ModelT {
    FieldT<T> f;
    GridT<T> g;
    T dt, half_dt, omega;
    const T* cs;                       // (nsteps + 1) x 2 : cos, sin of Omega_p * n * dt
    const T* gh_v0s;                   // npix x 2 (v0, s), GH mode only
    void* U;                           // orbit-major M x N column block of this model
    int64_t n_orb;
    int64_t orbit_base;                // first orbit of this model in the state arrays
    int64_t ldu;                       // column stride of U (rows)
    // orbit bundles accumulated at bin time: orbit i adds into column i / bundle (bundle <= 1: column i)
    int bundle;
    // sign < 0: subtract the orbits' counts (removes realisations cut by the quality test from a
    // bundled column); orbit_list (nullable): thread k integrates orbit orbit_list[k]
    int sign;
    const int64_t* orbit_list;
};

// Per-orbit status codes (mirrors SW_ORBIT_*).
enum { ST_OK = 0, ST_DRIFT = 1, ST_NONFINITE = 2 };

// Host-side helpers implemented in sw_api.cu.
void set_error(sw_ctx* ctx, const char* fmt, ...);

// Kernel-launch registry for per-kernel CUDA-event timing and launch counting.
enum KernelId {
    K_ICS_SOA = 0, K_ORBIT_BIN, K_ORBIT_DRIFT, K_ZERO_FLAGGED, K_FINALIZE, K_TRAJ, K_POTEVAL,
    K_WHITEN, K_GRAM_TC, K_GRAM_SIMT, K_SHIFT, K_POTRF_DIAG, K_TRSM_PANEL, K_SYRK_UPDATE,
    K_TRINV_DIAG, K_TRINV_UPDATE, K_GEMV_N, K_GEMV_T, K_TRMV_L, K_TRMV_LT, K_ADMM_UPDATE,
    K_RESID, K_GRAD, K_CHI2, K_MISC, K_BATCH_ORBIT, K_MLP_FWD, K_MLP_BWD, K_ADAM, K_REDUCE_GH, K_PCG, K_BUNDLE, K_CHOL_COOP,
    K_SYRK_TC, K_TRINV_TC, K_BORDER, K_COUNT
};
extern const char* kKernelNames[K_COUNT];

struct LaunchTimer {
    sw_ctx* ctx; int id; bool on; cudaStream_t st;
    LaunchTimer(sw_ctx* c, int kid);                    // on the context's stream
    LaunchTimer(sw_ctx* c, int kid, cudaStream_t s);    // on another stream of the context
    ~LaunchTimer();
};

cudaStream_t ctx_stream(sw_ctx* ctx);
// streaming multiprocessors of the context's device
int ctx_sms(const sw_ctx* ctx);

// Algorithmic work of a launch, accumulated per kernel for the roofline: FLOPs for the
// dense factorisation and Gram kernels, HBM bytes for the streaming kernels, orbit-steps
// for the orbit kernels (kind per kernel in kKernelWorkKind).
void add_work(sw_ctx* ctx, int kid, double units);
enum WorkKind { W_NONE = 0, W_FLOP_SIMT = 1, W_FLOP_TENSOR = 2, W_BYTES = 3, W_ORBIT_STEPS = 4 };
extern const int kKernelWorkKind[K_COUNT];

// ---- orbit kernels (k_orbit.cu)
template <typename T>
cudaError_t launch_ics_to_soa(sw_ctx* ctx, const double* ics_dev_aos, int64_t n, T* soa, int64_t ld);
template <typename T>
cudaError_t launch_orbit_bin(sw_ctx* ctx, const ModelT<T>& m, const T* soa, int64_t ld, int64_t nsteps,
                             int ej_every, double* drift, uint8_t* status, unsigned long long* stats);
template <typename T>
cudaError_t launch_orbit_drift(sw_ctx* ctx, const ModelT<T>& m, const T* soa, int64_t ld, int64_t nsteps,
                               int ej_every, double* drift, uint8_t* status, unsigned long long* stats);
template <typename T>
cudaError_t launch_zero_flagged(sw_ctx* ctx, void* U, int64_t M, int64_t N, const uint8_t* status);
template <typename T>
cudaError_t launch_finalize(sw_ctx* ctx, void* U, int64_t M, int64_t N, int64_t count_rows, double norm);
// the paper's adaptive integrator: step-weighted columns and the per-orbit integration time
template <typename T>
cudaError_t launch_orbit_bin_bs3(sw_ctx* ctx, const ModelT<T>& m, const T* soa, int64_t ld, int64_t nsteps,
                                 int ej_every, double rtol, double* drift, uint8_t* status, double* t_total,
                                 unsigned long long* stats);
template <typename T>
cudaError_t launch_finalize_w(sw_ctx* ctx, void* U, int64_t M, int64_t N, const double* t_total, int ncopy);
template <typename T>
cudaError_t launch_trajectory(sw_ctx* ctx, const ModelT<T>& m, const T* soa, int64_t ld, int64_t n,
                              int64_t nsteps, double* out);
template <typename T>
cudaError_t launch_poteval(sw_ctx* ctx, const FieldT<T>& f, const double* xyz, int64_t n, double* phi,
                           double* acc);
template <typename T>
cudaError_t launch_reduce_gh(sw_ctx* ctx, const void* Uh, int64_t Mh, int64_t N, int64_t nd, int64_t npix, int nv,
                             const void* W, void* Ug, int64_t Mg);
template <typename T>
cudaError_t launch_bundle(sw_ctx* ctx, const void* U, int64_t M, int64_t Nb, int n, void* out);
// persistent multi-model launch: threads per CTA in {64, 128, 256}, grid CTAs; pot = 1 (FP32 only) when
// every model is disc + halo + Long-Murali bar with no test fixture
template <typename T>
cudaError_t launch_batch_orbit_bin(cudaStream_t st, int threads, int grid, int gh, int pot, const ModelT<T>* models,
                                   const int2* items, int n_items, int* next, const T* soa, int64_t ld,
                                   int64_t nsteps, int ej_every, double* drift, uint8_t* status);

}  // namespace sw
