// Internal declarations of the weight-solve kernels (k_linalg.cu, k_gram_tc.cu).
#pragma once
#include "sw_api_internal.cuh"

#include <vector>

namespace sw {

template <typename T, typename AT>
cudaError_t whiten(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* inv_sig, const double* cs, AT* A,
                   AT* Alo, int64_t ldA, bool orbit_space);
template <typename T>
cudaError_t colnorm2(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* inv_sig, double* h);
template <typename GT>
cudaError_t admm_scales(sw_ctx* ctx, int64_t N, const double* h, double two_lam_n, double rho, double floor_,
                        double* s64, GT* s, GT* rho_i, GT* d);
template <typename GT>
cudaError_t div_to(sw_ctx* ctx, int64_t n, const double* a, const double* b, GT* out);
template <typename T, bool BT, bool LOWER>
cudaError_t gemm(sw_ctx* ctx, int kid, int64_t m, int64_t n, int64_t k, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, int64_t diag_off);
// C[m x n] += alpha A op(B), the contraction split into slices accumulated by atomics (C initialised
// by the caller); TRI: B lower triangular, only its triangle contracted (BT: B n x k, row c holding
// k <= c; else B k x n, column c holding k >= c)
template <typename T, bool BT, bool TRI>
cudaError_t gemm_acc(sw_ctx* ctx, int kid, int64_t m, int64_t n, int64_t k, T alpha, const T* A, int64_t lda,
                     const T* B, int64_t ldb, T* C, int64_t ldc);
// Cholesky (in place) and the explicit inverse X = L^{-1} in one cooperative launch (k_chol.cu);
// cudaErrorNotSupported when the device cannot launch it; *d_err != 0 if a barrier wait ran out
template <typename T>
cudaError_t cholesky_inverse_coop(sw_ctx* ctx, T* G, T* X, int64_t K, int* d_info, int* d_err);
// Cholesky (in place) and the explicit inverse X = L^{-1} by per-step launches (D unused)
template <typename T>
cudaError_t cholesky_inverse(sw_ctx* ctx, T* G, T* X, T* D, int64_t K, int* d_info);
// FP32 Cholesky (in place) and X = L^{-1} in 128-wide steps with the trailing and inverse updates on
// the tensor cores (k_chol_tc.cu); cudaErrorNotSupported without the tensor-map encoder; *d_err != 0 if
// a bounded wait of a tensor-core kernel ran out
// G and X are K x K with leading dimension ld, a multiple of 4 (16-byte rows for the TMA).  Without
// keep_L the diagonal blocks of L are not written back (G then holds only the panels below them).
cudaError_t cholesky_inverse_tc(sw_ctx* ctx, float* G, float* X, int64_t K, int64_t ld, int* d_info, int* d_err,
                                bool keep_L = true);
bool chol_tc_available();
template <typename T>
cudaError_t symmetrize(sw_ctx* ctx, const T* G, int64_t K, T* S);
template <typename T>
cudaError_t shift_diag_vec(sw_ctx* ctx, T* G, int64_t K, int64_t ld, const double* d);
template <typename GT>
cudaError_t scale_to(sw_ctx* ctx, int64_t n, const double* a, const double* s, GT* out);
template <typename GT>
cudaError_t as_residual(sw_ctx* ctx, int64_t n, const double* q, const double* g, const double* x, double mu,
                        const double* s, GT* rs);
template <typename GT>
cudaError_t axpy_scaled(sw_ctx* ctx, int64_t n, const GT* c, const double* s, double* x);
cudaError_t weight_sq(sw_ctx* ctx, int64_t m, const double* acc, const double* inv_sig, double* xs);
template <typename T>
cudaError_t shift_and_trace(sw_ctx* ctx, T* G, int64_t K, double* d_trace, double shift);
// A2 (nullable, same layout): the operand is A + A2 (the lo half of a split matrix)
template <typename AT, typename XT, typename YT, typename ACC>
cudaError_t rowdot(sw_ctx* ctx, int kid, const AT* A, int64_t rows, int64_t cols, int64_t lda, const XT* x, YT* y,
                   double alpha, double beta, bool lower, const AT* A2 = nullptr);
template <typename AT, typename XT, typename YT, typename ACC>
cudaError_t colcomb(sw_ctx* ctx, int kid, const AT* A, int64_t rows, int64_t cols, int64_t lda, const XT* x, YT* y,
                    double alpha, bool lower, const AT* A2 = nullptr);
template <typename GT>
cudaError_t admm_update(sw_ctx* ctx, int64_t N, const GT* y, const GT* v, const GT* s, const GT* rho_i, const GT* d,
                        const GT* qp, double alpha, GT* rs, GT* z, GT* u, unsigned* stats);
template <typename GT>
cudaError_t admm_init(sw_ctx* ctx, int64_t N, const GT* qp, const GT* z, const GT* u, const GT* s, const GT* rho_i,
                      GT* rs);
template <typename T>
cudaError_t u_times_w(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* w, double* acc);
// U w for an FP32 matrix with the float hi + lo halves of w staged in caller-provided buffers
// (N floats each): no workspace of the context is touched or allocated
cudaError_t u_times_w_presplit(sw_ctx* ctx, const float* U, int64_t M, int64_t N, const double* w, float* wh,
                               float* wl, double* acc);
cudaError_t residual(sw_ctx* ctx, int64_t M, const double* y, const double* acc, const double* inv_sig, double* e,
                     double* xs);
template <typename T>
cudaError_t ut_times_x(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* xs, double* out);
cudaError_t kkt(sw_ctx* ctx, int64_t N, const double* ute, const double* w, double two_lam_n, double* gneg,
                unsigned long long* pgmax);
cudaError_t chi2(sw_ctx* ctx, int64_t M, int64_t nd, const double* e, int64_t N, const double* w, double* out3);
cudaError_t prep_data(sw_ctx* ctx, int64_t M, const double* sigma, const double* y, double* inv_sig, double* ys,
                      int* bad);
template <typename A, typename B>
cudaError_t convert(sw_ctx* ctx, int64_t n, const A* a, B* b);
template <typename GT>
cudaError_t refine_rhs(sw_ctx* ctx, int64_t N, const GT* t, const double* gneg, const double* w, const double* s64,
                       double two_lam_n, const GT* rho_i, GT* qp, GT* z, GT* u);

template <typename T>
cudaError_t gather_rows(sw_ctx* ctx, const T* U, int64_t M, const int64_t* idx, int64_t nP, const double* inv_sig,
                        double* R);
cudaError_t gather_vec(sw_ctx* ctx, const double* a, const int64_t* idx, int64_t n, double* out);
template <typename T>
cudaError_t gather_cols(sw_ctx* ctx, const T* U, int64_t M, const int64_t* idx, int64_t n, T* Uc);
cudaError_t scatter_vec(sw_ctx* ctx, const double* a, const int64_t* idx, int64_t n, double* out);

// Warm start of the active-set solve across related problems (the bootstrap realisations of one
// matrix, Sec. 2.4): `record` keeps the final passive set and weights of a solve and factors a
// superset P0 of its passive set (the passive set plus the zero-weight orbits nearest to entering);
// `start` begins a later solve from that passive set and those weights and reuses the factor of P0
// for every passive set inside it.
struct AsWarm {
    bool record = false, start = false;
    std::vector<char> F0;        // passive set of the recorded solve (N flags)
    std::vector<double> w0;      // its weights (N)
    std::vector<int64_t> P0;     // the factored set, in the order of its factor
    int64_t ld = 0;              // leading dimension of its G and X
    double fl = 0.0;             // ridge floor of its factor
    bool have_factor = false;
    double p0_extra = 0.0;       // P0 = F0 plus up to this fraction of |F0| near-active orbits
    int64_t factorisations = 0;  // factorisations made by the solves of this warm start
};

// block active-set solve (sw_active_set.cu)
template <typename T, typename AT, typename GT>
sw_status solve_active_set(sw_ctx* ctx, const sw_matrix* U, const double* y_dev, const double* sig_dev, double lam,
                           double* w_dev, double* chi2_dev, AsWarm* warm = nullptr);
// B bootstrap realisations of the data (Sec. 2.4): y_b = y + sigma xi_b on the observed rows (the
// density rows unchanged), one active-set solve each, warm-started from the solve on y; chi2_b is
// the observational chi^2 of w_b against y (xi_dev: B x M device, w_dev: B x N device or NULL,
// chi2b_dev: B device)
template <typename T, typename AT, typename GT>
sw_status solve_bootstrap(sw_ctx* ctx, const sw_matrix* U, const double* y_dev, const double* sig_dev, double lam,
                          int64_t B, const double* xi_dev, double* w_dev, double* chi2b_dev);

// tcgen05 Gram (k_gram_tc.cu): C (K x K, FP32, row-major, lower tiles) = A A^T with A
// K x ldA BF16 row-major (ldA a multiple of 64, columns beyond the data zero).  With
// A_lo non-NULL the operand is A + A_lo and the three leading products of the split
// are accumulated.  d_err receives a non-zero code if a bounded wait ran out.  row_tile0 > 0
// computes only the tile rows from row_tile0 on (rows 128 row_tile0 .. K - 1 of the lower part).
cudaError_t gram_tc(sw_ctx* ctx, const __nv_bfloat16* A, const __nv_bfloat16* A_lo, int64_t K, int64_t ldA, float* C,
                    int* d_err, int64_t ldc = 0, int64_t row_tile0 = 0);
// G[a][b] = Gc[cidx[a]][cidx[b]] (Gc lower-triangular, read symmetrically) for b <= a < r0
cudaError_t gather_gram(sw_ctx* ctx, const float* Gc, int64_t ldc, const int64_t* cidx, int64_t r0, float* G,
                        int64_t ldG);
bool gram_tc_available();

}  // namespace sw
