// Dense linear algebra of the weight solve (arxiv 2607.00117 Sec. 2.3):
// whitening, blocked Cholesky of the shifted Gram, explicit inverse of the
// Cholesky factor, HBM-bound matrix-vector products, the fused ADMM update,
// and FP64 residual / gradient / chi^2 passes over the stored orbit matrix.
#include "sw_linalg.cuh"

namespace sw {

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
template <typename AT> __device__ __forceinline__ AT to_a(float v);
template <> __device__ __forceinline__ __nv_bfloat16 to_a<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float to_a<float>(float v) { return v; }
template <typename AT> __device__ __forceinline__ AT to_a_d(double v);
template <> __device__ __forceinline__ double to_a_d<double>(double v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_a_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <> __device__ __forceinline__ float to_a_d<float>(double v) { return (float)v; }

__device__ __forceinline__ float from_a(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from_a(float v) { return v; }
__device__ __forceinline__ double from_a(double v) { return v; }

// ---------------------------------------------------------------------------
// Whitening: A~ = diag(1/sigma) U diag(cs) (cs: per-orbit column scale),
// written K-major for the Gram.
// Orbit space: A[i * ldA + r] (rows are orbits, contraction over constraints).
// Constraint space: A[r * ldA + i] (rows are constraints, contraction over orbits).
// Padding columns up to ldA are zero.
// ---------------------------------------------------------------------------
// hi/lo split: lo (nullable) receives the rounding residual of the value in hi
template <typename AT>
__device__ __forceinline__ void store_split(AT* hi, AT* lo, size_t k, double v)
{
    const AT h = to_a_d<AT>(v);
    hi[k] = h;
    if (lo) lo[k] = to_a_d<AT>(v - (double)from_a(h));
}

template <typename T, typename AT>
__global__ void k_whiten_orbit(const T* __restrict__ U, int64_t M, int64_t N, const double* __restrict__ inv_sig,
                               const double* __restrict__ cs, AT* __restrict__ A, AT* __restrict__ Alo, int64_t ldA)
{
    for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
        const T* col = U + (size_t)i * M;
        const double c = cs[i];
        for (int64_t r = threadIdx.x; r < ldA; r += blockDim.x)
            store_split(A, Alo, (size_t)i * ldA + r, r < M ? (double)col[r] * inv_sig[r] * c : 0.0);
    }
}

// FP32 matrix -> BF16 hi + lo halves, orbit space, in FP32 arithmetic (the split keeps ~16 bits, so
// FP32 products lose nothing; FP64 arithmetic here would make the pass FP64-bound on this part).
// inv_sig_f: 1/sigma in FP32.  Each thread handles pairs of rows (one 4-byte BF16x2 store per half).
__global__ void k_whiten_orbit_f32(const float* __restrict__ U, int64_t M, int64_t N,
                                   const float* __restrict__ inv_sig_f, const double* __restrict__ cs,
                                   __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ Alo, int64_t ldA)
{
    for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
        const float* col = U + (size_t)i * M;
        const float c = (float)cs[i];
        __nv_bfloat162* a2 = reinterpret_cast<__nv_bfloat162*>(A + (size_t)i * ldA);
        __nv_bfloat162* l2 = reinterpret_cast<__nv_bfloat162*>(Alo + (size_t)i * ldA);
        for (int64_t p = threadIdx.x; 2 * p < ldA; p += blockDim.x) {
            const int64_t r = 2 * p;
            const float v0 = r < M ? col[r] * inv_sig_f[r] * c : 0.f;
            const float v1 = r + 1 < M ? col[r + 1] * inv_sig_f[r + 1] * c : 0.f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            a2[p] = h;
            if (Alo) l2[p] = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
        }
    }
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

template <typename T, typename AT>
__global__ void k_whiten_transpose(const T* __restrict__ U, int64_t M, int64_t N, const double* __restrict__ inv_sig,
                                   const double* __restrict__ cs, AT* __restrict__ A, AT* __restrict__ Alo,
                                   int64_t ldA)
{
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        int64_t i = i0 + k, r = r0 + tx;
        tile[k][tx] = (i < N && r < M) ? (double)U[(size_t)i * M + r] * inv_sig[r] * cs[i] : 0.0;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        int64_t r = r0 + k, i = i0 + tx;
        if (r < M && i < ldA) store_split(A, Alo, (size_t)r * ldA + i, tile[tx][k]);
    }
}

// ---------------------------------------------------------------------------
// Split-contraction SIMT GEMM for short, wide products: C[m x n] += alpha A op(B),
// A row-major m x k; BT: B is n x k row-major (A B^T), else k x n row-major (A B).
// The contraction is cut into slices of kchunk (blockIdx.z) accumulated into C by
// atomics, so that a product with few rows still fills the GPU.  TRI: B is lower
// triangular, and each 64-column tile of C contracts only over B's triangle
// (BT: row c of B holds entries k <= c; else column c of B holds entries k >= c).
// ---------------------------------------------------------------------------
template <typename T, bool BT, bool TRI>
__global__ void __launch_bounds__(256) k_gemm_acc(int64_t m, int64_t n, int64_t k, T alpha, const T* __restrict__ A,
                                                  int64_t lda, const T* __restrict__ B, int64_t ldb, T* __restrict__ C,
                                                  int64_t ldc, int64_t kchunk)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    const int64_t bm = (int64_t)blockIdx.y * BM, bn = (int64_t)blockIdx.x * BN;
    int64_t klo = 0, khi = k;
    if (TRI) {
        if (BT) khi = bn + BN < k ? bn + BN : k;
        else klo = bn;
    }
    const int64_t k0 = klo + (int64_t)blockIdx.z * kchunk;
    const int64_t k1 = k0 + kchunk < khi ? k0 + kchunk : khi;
    if (k0 >= k1) return;
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int64_t kb = k0; kb < k1; kb += BK) {
        {
            const int r = t >> 2, kq = (t & 3) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t gr = bm + r, gk = kb + kq + q;
                As[kq + q][r] = (gr < m && gk < k1) ? A[(size_t)gr * lda + gk] : T(0);
            }
        }
        if (BT) {
            const int r = t >> 2, kq = (t & 3) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t gc = bn + r, gk = kb + kq + q;
                Bs[kq + q][r] = (gc < n && gk < k1) ? B[(size_t)gc * ldb + gk] : T(0);
            }
        } else {
            const int kk = t >> 4, cq = (t & 15) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t gc = bn + cq + q, gk = kb + kk;
                Bs[kk][cq + q] = (gc < n && gk < k1) ? B[(size_t)gk * ldb + gc] : T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = bm + ty * 4 + i;
        if (gr >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gc = bn + tx * 4 + j;
            if (gc < n) atomicAdd(C + (size_t)gr * ldc + gc, alpha * acc[i][j]);
        }
    }
}

// ---------------------------------------------------------------------------
// SIMT GEMM: C[m x n] = beta C + alpha A op(B); A row-major m x k; BT: B is
// n x k row-major (C = A B^T), else k x n row-major (C = A B).  LOWER skips
// 64 x 64 tiles that lie strictly above the diagonal of the global matrix
// (global row - global col = tile row - tile col + diag_off).
// ---------------------------------------------------------------------------
template <typename T, bool BT, bool LOWER>
__global__ void __launch_bounds__(256) k_gemm(int64_t m, int64_t n, int64_t k, T alpha, const T* __restrict__ A,
                                              int64_t lda, const T* __restrict__ B, int64_t ldb, T beta,
                                              T* __restrict__ C, int64_t ldc, int64_t diag_off)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    const int64_t bm = (int64_t)blockIdx.y * BM, bn = (int64_t)blockIdx.x * BN;
    if (LOWER && bm + BM - 1 + diag_off < bn) return;
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int64_t k0 = 0; k0 < k; k0 += BK) {
        {   // A tile: 64 rows x 16 k; thread -> row t/4, k (t%4)*4 .. +4
            int r = t >> 2, kq = (t & 3) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int64_t gr = bm + r, gk = k0 + kq + q;
                As[kq + q][r] = (gr < m && gk < k) ? A[(size_t)gr * lda + gk] : T(0);
            }
        }
        if (BT) {
            int r = t >> 2, kq = (t & 3) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int64_t gc = bn + r, gk = k0 + kq + q;
                Bs[kq + q][r] = (gc < n && gk < k) ? B[(size_t)gc * ldb + gk] : T(0);
            }
        } else {
            int kk = t >> 4, cq = (t & 15) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int64_t gc = bn + cq + q, gk = k0 + kk;
                Bs[kk][cq + q] = (gc < n && gk < k) ? B[(size_t)gk * ldb + gc] : T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gr = bm + ty * 4 + i;
        if (gr >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gc = bn + tx * 4 + j;
            if (gc >= n) continue;
            T* c = C + (size_t)gr * ldc + gc;
            *c = (beta == T(0) ? T(0) : beta * *c) + alpha * acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// Cholesky pieces (block size NB = 64).
// ---------------------------------------------------------------------------
constexpr int NB = 64;

// The diagonal block's factor and its inverse in one CTA of 256 threads.  Cholesky: four
// threads per row, each row's update split over the four by column, every thread computing
// the pivot itself, two barriers per column step.  Then D = L_kk^{-1} by forward
// substitution with four lanes of one warp per column (the
// columns are independent; each column's dot products are split over its four lanes and
// combined by shuffles).  L_kk goes back to G, D (NB x NB, zero outside bs) to D.  (A
// register-resident variant with fully unrolled loops measured slower: its code no longer
// fits the instruction cache.)
template <typename T>
__global__ void __launch_bounds__(256) k_diag_factor_inv(T* __restrict__ G, int64_t ld, int64_t j0, int bs,
                                                         T* __restrict__ D, int* info)
{
    extern __shared__ unsigned char smraw[];
    T (*a)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smraw);
    T (*x)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smraw + sizeof(T) * NB * (NB + 1));
    const int t = threadIdx.x, row = t & (NB - 1), q = t >> 6;
    for (int e = t; e < NB * NB; e += 256) {
        int i = e / NB, j = e % NB;
        a[i][j] = (i < bs && j <= i) ? G[(size_t)(j0 + i) * ld + j0 + j] : T(0);
        x[i][j] = T(0);
    }
    __syncthreads();
    for (int j = 0; j < bs; ++j) {
        T d = a[j][j];
        if (!(d > T(0))) {
            if (t == 0 && info) atomicCAS(info, 0, (int)(j0 + j + 1));
            d = T(1e-30);
        }
        d = sqrt(d);
        if (q == 0 && row > j && row < bs) a[row][j] /= d;
        __syncthreads();
        if (row > j && row < bs) {
            const T aij = a[row][j];
            for (int l = j + 1 + q; l <= row; l += 4) a[row][l] -= aij * a[l][j];
        }
        if (t == 0) a[j][j] = d;
        __syncthreads();
    }
    // inverse: lanes 4c .. 4c + 3 own column c
    const int col = t >> 2, part = t & 3;
    if (part == 0 && col < bs) x[col][col] = T(1) / a[col][col];
    __syncwarp();
    for (int i = 1; i < bs; ++i) {
        T s = T(0);
        if (i > col)
            for (int l = col + part; l < i; l += 4) s += a[i][l] * x[l][col];
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (part == 0 && i > col && col < bs) x[i][col] = -s / a[i][i];
        __syncwarp();
    }
    __syncthreads();
    for (int e = t; e < NB * NB; e += 256) {
        int i = e / NB, j = e % NB;
        if (i < bs && j <= i) G[(size_t)(j0 + i) * ld + j0 + j] = a[i][j];
        D[e] = x[i][j];
    }
}

// Block row k of X (rows j0..j0+bs, columns 0..ncols): X_k <- D X_k.
template <typename T>
__global__ void __launch_bounds__(64) k_trmm_diag(T* __restrict__ X, int64_t ld, int64_t j0, int bs, int64_t ncols,
                                                  const T* __restrict__ D)
{
    extern __shared__ unsigned char smraw[];
    T (*Dm)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smraw);
    T (*S)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smraw + sizeof(T) * NB * (NB + 1));
    const int t = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * NB;
    for (int e = t; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        Dm[i][j] = D[e];
        int64_t gc = c0 + j;
        S[i][j] = (i < bs && gc < ncols) ? X[(size_t)(j0 + i) * ld + gc] : T(0);
    }
    __syncthreads();
    // thread t owns column t of the slab (S is a private copy, so writing X is safe)
    const int64_t gc = c0 + t;
    if (gc >= ncols) return;
    T col[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) col[l] = S[l][t];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i >= bs) break;
        T s = T(0);
#pragma unroll
        for (int l = 0; l <= i; ++l) s += Dm[i][l] * col[l];
        X[(size_t)(j0 + i) * ld + gc] = s;
    }
}

template <typename T>
__global__ void k_set_identity(T* __restrict__ X, int64_t K)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += (int64_t)gridDim.x * blockDim.x)
        X[e] = (e / K == e % K) ? T(1) : T(0);
}

template <typename T>
__global__ void k_shift_diag(T* __restrict__ G, int64_t K, double shift)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x)
        G[(size_t)i * K + i] += (T)shift;
}

// G_ii += d_i (per-variable ridge)
template <typename T>
__global__ void k_shift_diag_vec(T* __restrict__ G, int64_t K, int64_t ld, const double* __restrict__ d)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x)
        G[(size_t)i * ld + i] += (T)d[i];
}

// Active-set reduced solve helpers: out_k = s_k * a_k (to working precision), and
// r_k = q_k - g_k - mu x_k (FP64), optionally scaled by s_k into working precision.
template <typename GT>
__global__ void k_scale_to(int64_t n, const double* __restrict__ a, const double* __restrict__ s, GT* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (GT)(a[i] * s[i]);
}

template <typename GT>
__global__ void k_as_residual(int64_t n, const double* __restrict__ q, const double* __restrict__ g,
                              const double* __restrict__ x, double mu, const double* __restrict__ s,
                              GT* __restrict__ rs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rs[i] = (GT)((q[i] - g[i] - mu * x[i]) * s[i]);
}

// x_k += s_k * c_k
template <typename GT>
__global__ void k_axpy_scaled(int64_t n, const GT* __restrict__ c, const double* __restrict__ s, double* __restrict__ x)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)c[i] * s[i];
}

// xs_r = acc_r * inv_sig_r^2
__global__ void k_weight_sq(int64_t m, const double* __restrict__ acc, const double* __restrict__ inv_sig,
                            double* __restrict__ xs)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        xs[r] = acc[r] * inv_sig[r] * inv_sig[r];
}

// S = G with the lower triangle mirrored to the upper one (full symmetric copy)
template <typename T>
__global__ void k_symmetrize(const T* __restrict__ G, int64_t K, T* __restrict__ S)
{
    __shared__ T tile[32][33];
    const int64_t bi = blockIdx.y, bj = blockIdx.x;   // tile (bi, bj) of S, 32 x 32
    const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8
    if (bi >= bj) {
        for (int k = ty; k < 32; k += 8) {
            int64_t r = bi * 32 + k, c = bj * 32 + tx;
            if (r < K && c < K) S[(size_t)r * K + c] = (r >= c) ? G[(size_t)r * K + c] : G[(size_t)c * K + r];
        }
    } else {   // upper tile: transpose of the lower tile (bj, bi)
        for (int k = ty; k < 32; k += 8) {
            int64_t r = bj * 32 + k, c = bi * 32 + tx;
            tile[k][tx] = (r < K && c < K) ? G[(size_t)r * K + c] : T(0);
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {
            int64_t r = bi * 32 + k, c = bj * 32 + tx;
            if (r < K && c < K) S[(size_t)r * K + c] = tile[tx][k];
        }
    }
}

template <typename T>
__global__ void k_trace(const T* __restrict__ G, int64_t K, double* out)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)G[(size_t)i * K + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// ---------------------------------------------------------------------------
// Matrix-vector products on row-major A (rows x cols, leading dim lda).
// rowdot: y[r] = alpha * sum_c A[r, c] x[c] + beta * y[r]   (one warp per row)
// colcomb: y[c] += alpha * sum_r A[r, c] x[r]               (threads over
//          columns, blockIdx.y splits the rows; partial sums by atomics)
// lower: only c <= r contributes.
// ---------------------------------------------------------------------------
template <typename AT, typename XT, typename YT, typename ACC>
__global__ void __launch_bounds__(256) k_rowdot(const AT* __restrict__ A, const AT* __restrict__ A2, int64_t rows,
                                                int64_t cols, int64_t lda, const XT* __restrict__ x,
                                                YT* __restrict__ y, double alpha, double beta, int lower)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarp) {
        const AT* a = A + (size_t)r * lda;
        const int64_t n = lower ? (r + 1 < cols ? r + 1 : cols) : cols;
        ACC s = ACC(0);
        if constexpr (sizeof(AT) == 2) {
            const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(a);
            const __nv_bfloat162* b2 = A2 ? reinterpret_cast<const __nv_bfloat162*>(A2 + (size_t)r * lda) : nullptr;
            const int64_t n2 = n >> 1;
            for (int64_t c = lane; c < n2; c += 32) {
                float2 v = __bfloat1622float2(a2[c]);
                if (b2) {
                    const float2 l = __bfloat1622float2(b2[c]);
                    v.x += l.x;
                    v.y += l.y;
                }
                s += (ACC)v.x * (ACC)x[2 * c] + (ACC)v.y * (ACC)x[2 * c + 1];
            }
            if ((n & 1) && lane == 0)
                s += ((ACC)from_a(a[n - 1]) + (A2 ? (ACC)from_a(A2[(size_t)r * lda + n - 1]) : ACC(0))) *
                     (ACC)x[n - 1];
        } else {
            for (int64_t c = lane; c < n; c += 32) s += (ACC)from_a(a[c]) * (ACC)x[c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[r] = (YT)(alpha * (double)s + (beta == 0.0 ? 0.0 : beta * (double)y[r]));
    }
}

template <typename AT, typename XT, typename YT, typename ACC>
__global__ void __launch_bounds__(256) k_colcomb(const AT* __restrict__ A, const AT* __restrict__ A2, int64_t rows,
                                                 int64_t cols, int64_t lda, const XT* __restrict__ x,
                                                 YT* __restrict__ y, double alpha, int64_t rows_per_split, int lower)
{
    const int64_t c2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // column pair index
    const int64_t c = 2 * c2;
    if (c >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    int64_t r1 = r0 + rows_per_split;
    if (r1 > rows) r1 = rows;
    int64_t rs = r0;
    if (lower && rs < c) rs = c;
    ACC s0 = ACC(0), s1 = ACC(0);
    const bool two = c + 1 < cols;
    for (int64_t r = rs; r < r1; ++r) {
        const AT* a = A + (size_t)r * lda + c;
        ACC xr = (ACC)x[r];
        if constexpr (sizeof(AT) == 2) {
            const AT* b = A2 ? A2 + (size_t)r * lda + c : nullptr;
            if (two) {
                float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(a));
                if (b) {
                    const float2 l = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(b));
                    v.x += l.x;
                    v.y += l.y;
                }
                s0 += (ACC)v.x * xr;
                s1 += (ACC)v.y * xr;
            } else {
                s0 += ((ACC)from_a(a[0]) + (b ? (ACC)from_a(b[0]) : ACC(0))) * xr;
            }
        } else {
            s0 += (ACC)from_a(a[0]) * xr;
            if (two && (!lower || r >= c + 1)) s1 += (ACC)from_a(a[1]) * xr;
        }
    }
    if (r1 > rs) {
        atomicAdd(&y[c], (YT)(alpha * (double)s0));
        if (two) atomicAdd(&y[c + 1], (YT)(alpha * (double)s1));
    }
}

// ---------------------------------------------------------------------------
// ADMM (Sec. 2.3) with a per-orbit penalty P = diag(rho_i): the quadratic step
// w = (H~ + P)^{-1} (q' + P (z - u)) is applied as w = s o y with
// s = (2 lam/N + rho_i)^{-1/2} (see sw_solve.cu), then, over-relaxed by alpha,
// z = max(0, alpha w + (1 - alpha) z + u), u += alpha w + (1 - alpha) z_old - z,
// and the next scaled right-hand side rs = s o (q' + P (z - u)).
// Constraint space passes v and forms y = rs - v.
// stats (nullable): max |w - z| d, max |z - z_prev| d, max z d (float bits),
// with d_i = ||column i of U~||, i.e. in units of the equilibrated problem.
// ---------------------------------------------------------------------------
template <typename GT>
__global__ void k_admm_update(int64_t N, const GT* __restrict__ y, const GT* __restrict__ v,
                              const GT* __restrict__ sc, const GT* __restrict__ rho_i, const GT* __restrict__ d,
                              const GT* __restrict__ qp, GT alpha, GT* __restrict__ rs, GT* __restrict__ z,
                              GT* __restrict__ u, unsigned* stats)
{
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const GT si = sc[i];
        const GT w = v ? si * (rs[i] - v[i]) : si * y[i];
        const GT zo = z[i], uo = u[i];
        const GT wh = alpha * w + (GT(1) - alpha) * zo;
        GT zn = wh + uo;
        zn = zn > GT(0) ? zn : GT(0);
        const GT un = uo + wh - zn;
        z[i] = zn;
        u[i] = un;
        rs[i] = si * (qp[i] + rho_i[i] * (zn - un));
        const GT di = d[i];
        m0 = fmaxf(m0, (float)(fabs((double)(w - zn)) * (double)di));
        m1 = fmaxf(m1, (float)(fabs((double)(zn - zo)) * (double)di));
        m2 = fmaxf(m2, (float)((double)zn * (double)di));
    }
    if (!stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(stats + 0, __float_as_uint(m0));
        atomicMax(stats + 1, __float_as_uint(m1));
        atomicMax(stats + 2, __float_as_uint(m2));
    }
}

// rs = s o (q' + P (z - u)) (initialisation)
template <typename GT>
__global__ void k_admm_init(int64_t N, const GT* __restrict__ qp, const GT* __restrict__ z, const GT* __restrict__ u,
                            const GT* __restrict__ sc, const GT* __restrict__ rho_i, GT* __restrict__ rs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        rs[i] = sc[i] * (qp[i] + rho_i[i] * (z[i] - u[i]));
}

// Per-orbit ADMM scaling from the exact column norms h_i = ||U~ e_i||^2:
// rho_i = rho h_i, Lambda_i = 2 lam/N + rho_i (floored), s_i = Lambda_i^{-1/2}.
template <typename GT>
__global__ void k_admm_scales(int64_t N, const double* __restrict__ h, double two_lam_n, double rho, double floor_,
                              double* __restrict__ s64, GT* __restrict__ s, GT* __restrict__ rho_i, GT* __restrict__ d)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double hi = h[i];
        double lam_i = two_lam_n + rho * hi;
        if (!(lam_i > floor_)) lam_i = 1.0;   // an empty orbit with lambda = 0: its column is zero
        double si = 1.0 / sqrt(lam_i);
        s64[i] = si;
        s[i] = (GT)si;
        rho_i[i] = (GT)(rho * hi);
        d[i] = (GT)sqrt(hi);
    }
}

// ---------------------------------------------------------------------------
// FP64 passes over the stored orbit matrix (orbit-major, column i at U + i M).
// ---------------------------------------------------------------------------
// acc[r] += sum_i U[i, r] w[i]   (threads over rows r, blockIdx.y splits orbits)
template <typename T>
__global__ void __launch_bounds__(256) k_u_times_w(const T* __restrict__ U, int64_t M, int64_t N,
                                                   const double* __restrict__ w, double* __restrict__ acc,
                                                   int64_t orbits_per_split)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int64_t i0 = (int64_t)blockIdx.y * orbits_per_split;
    int64_t i1 = i0 + orbits_per_split;
    if (i1 > N) i1 = N;
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
        double wi = w[i];
        if (wi != 0.0) s += (double)U[(size_t)i * M + r] * wi;
    }
    if (i1 > i0) atomicAdd(acc + r, s);
}

// ---- double-float products for FP32 matrices.  GB300's FP64 pipe is a small
// fraction of its FP32 rate, so the products of the stored FP32 matrix with FP64
// vectors are formed in float-float arithmetic (Dekker 1971; Knuth's two-sum): the
// vector is split once into float hi + lo, each product u x_hi is made exact by an
// FMA residual, and the running sum keeps its own rounding error; about 2^-44
// relative per term, far below the solver's tolerances.
__global__ void k_split_ff(int64_t n, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float h = (float)v;
        hi[i] = h;
        lo[i] = (float)(v - (double)h);
    }
}

struct FF {
    float h, l;
};


// Running double-float sum: s.h keeps the rounded sum, s.l the exact rounding errors of its
// additions (two-sum) and the low parts of the products; ff_renorm folds s.l back (fast two-sum,
// |s.l| << |s.h|) every few terms, so that s.l stays ~2^-24 of the sum and its own rounding
// ~2^-48.
__device__ __forceinline__ void ff_acc(FF& s, float u, float xh, float xl)
{
    const float ph = u * xh;
    const float pl = fmaf(u, xl, fmaf(u, xh, -ph));
    const float t = s.h + ph;
    const float bb = t - s.h;
    s.l += ((s.h - (t - bb)) + (ph - bb)) + pl;
    s.h = t;
}

__device__ __forceinline__ void ff_renorm(FF& s)
{
    const float t = s.h + s.l;
    s.l -= t - s.h;
    s.h = t;
}

__device__ __forceinline__ double ff_value(const FF& s) { return (double)s.h + (double)s.l; }

// acc[r] += sum_i U[i, r] w[i] with w split into (wh, wl); zero weights skipped.  VEC: each thread
// owns four consecutive rows (16-byte loads; M a multiple of 4 and U 16-byte aligned), four
// orbits in flight
template <bool VEC>
__global__ void __launch_bounds__(256) k_u_times_w_ff(const float* __restrict__ U, int64_t M, int64_t N,
                                                      const float* __restrict__ wh, const float* __restrict__ wl,
                                                      double* __restrict__ acc, int64_t orbits_per_split)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * (VEC ? 4 : 1);
    if (r >= M) return;
    const int64_t i0 = (int64_t)blockIdx.y * orbits_per_split;
    int64_t i1 = i0 + orbits_per_split;
    if (i1 > N) i1 = N;
    if (i1 <= i0) return;
    if constexpr (VEC) {
        FF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int64_t i = i0;
        for (; i + 4 <= i1; i += 4) {
            float4 u[4];
            float h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = wh[i + q];
                l[q] = wl[i + q];
                u[q] = h[q] != 0.f ? *reinterpret_cast<const float4*>(U + (size_t)(i + q) * M + r)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ff_acc(s[0], u[q].x, h[q], l[q]);
                ff_acc(s[1], u[q].y, h[q], l[q]);
                ff_acc(s[2], u[q].z, h[q], l[q]);
                ff_acc(s[3], u[q].w, h[q], l[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) ff_renorm(s[q]);
        }
        for (; i < i1; ++i) {
            const float h = wh[i];
            if (h == 0.f) continue;
            const float4 u = *reinterpret_cast<const float4*>(U + (size_t)i * M + r);
            const float l = wl[i];
            ff_acc(s[0], u.x, h, l); ff_acc(s[1], u.y, h, l); ff_acc(s[2], u.z, h, l); ff_acc(s[3], u.w, h, l);
#pragma unroll
            for (int q = 0; q < 4; ++q) ff_renorm(s[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(acc + r + q, ff_value(s[q]));
    } else {
        // four independent double-float sums keep four loads in flight per thread
        FF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int64_t i = i0;
        for (; i + 4 <= i1; i += 4) {
            float u[4], h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = wh[i + q];
                l[q] = wl[i + q];
                u[q] = h[q] != 0.f ? U[(size_t)(i + q) * M + r] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ff_acc(s[q], u[q], h[q], l[q]);
                ff_renorm(s[q]);
            }
        }
        for (; i < i1; ++i) {
            const float h = wh[i];
            if (h != 0.f) {
                ff_acc(s[0], U[(size_t)i * M + r], h, wl[i]);
                ff_renorm(s[0]);
            }
        }
        atomicAdd(acc + r, (ff_value(s[0]) + ff_value(s[1])) + (ff_value(s[2]) + ff_value(s[3])));
    }
}

// out[i] = sum_r U[i, r] x[r] with x split into (xh, xl); one warp per orbit
__global__ void __launch_bounds__(256) k_ut_times_x_ff(const float* __restrict__ U, int64_t M, int64_t N,
                                                       const float* __restrict__ xh, const float* __restrict__ xl,
                                                       double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < N; i += nwarp) {
        const float* col = U + (size_t)i * M;
        FF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int64_t r = lane;
        for (; r + 96 < M; r += 128) {
            float u[4], h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u[q] = col[r + 32 * q];
                h[q] = xh[r + 32 * q];
                l[q] = xl[r + 32 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ff_acc(s[q], u[q], h[q], l[q]);
                ff_renorm(s[q]);
            }
        }
        for (; r < M; r += 32) {
            ff_acc(s[0], col[r], xh[r], xl[r]);
            ff_renorm(s[0]);
        }
        double d = (ff_value(s[0]) + ff_value(s[1])) + (ff_value(s[2]) + ff_value(s[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) out[i] = d;
    }
}

// The same with x staged in shared memory once per CTA (one persistent 1024-thread CTA per SM) and
// each lane streaming four consecutive rows of its orbit's column per 16-byte load, four loads in
// flight; M a multiple of 4, U 16-byte aligned, 8 M bytes of shared memory
constexpr int UTX_THREADS = 1024;
__global__ void __launch_bounds__(UTX_THREADS, 1) k_ut_times_x_ff_sm(const float* __restrict__ U, int64_t M, int64_t N,
                                                                     const float* __restrict__ xh,
                                                                     const float* __restrict__ xl,
                                                                     double* __restrict__ out)
{
    extern __shared__ float4 utx_sm[];
    float4* Xh = utx_sm;
    float4* Xl = utx_sm + M / 4;
    for (int64_t e = threadIdx.x; e < M / 4; e += UTX_THREADS) {
        Xh[e] = reinterpret_cast<const float4*>(xh)[e];
        Xl[e] = reinterpret_cast<const float4*>(xl)[e];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * (UTX_THREADS / 32);
    for (int64_t i = (int64_t)blockIdx.x * (UTX_THREADS / 32) + (threadIdx.x >> 5); i < N; i += nwarp) {
        const float4* col = reinterpret_cast<const float4*>(U + (size_t)i * M);
        FF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int64_t c = lane;   // 16-byte chunk of the column
        const int64_t nch = M / 4;
        for (; c + 96 < nch; c += 128) {
            float4 u[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) u[q] = col[c + 32 * q];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 h = Xh[c + 32 * q], l = Xl[c + 32 * q];
                ff_acc(s[0], u[q].x, h.x, l.x);
                ff_acc(s[1], u[q].y, h.y, l.y);
                ff_acc(s[2], u[q].z, h.z, l.z);
                ff_acc(s[3], u[q].w, h.w, l.w);
            }
            // four terms per sum between renormalisations (as in k_u_times_w_ff): s.l stays within
            // a few units of the last place of s.h
#pragma unroll
            for (int k = 0; k < 4; ++k) ff_renorm(s[k]);
        }
        for (; c < nch; c += 32) {
            const float4 u = col[c], h = Xh[c], l = Xl[c];
            ff_acc(s[0], u.x, h.x, l.x);
            ff_acc(s[1], u.y, h.y, l.y);
            ff_acc(s[2], u.z, h.z, l.z);
            ff_acc(s[3], u.w, h.w, l.w);
#pragma unroll
            for (int k = 0; k < 4; ++k) ff_renorm(s[k]);
        }
        double d = (ff_value(s[0]) + ff_value(s[1])) + (ff_value(s[2]) + ff_value(s[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) out[i] = d;
    }
}

// e[r] = (y[r] - acc[r]) * inv_sig[r]; also xs[r] = e[r] * inv_sig[r].
__global__ void k_residual(int64_t M, const double* __restrict__ y, const double* __restrict__ acc,
                           const double* __restrict__ inv_sig, double* __restrict__ e, double* __restrict__ xs)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (int64_t)gridDim.x * blockDim.x) {
        double v = (y[r] - acc[r]) * inv_sig[r];
        e[r] = v;
        xs[r] = v * inv_sig[r];
    }
}

// out[i] = sum_r U[i, r] xs[r]  (one warp per orbit)
template <typename T>
__global__ void __launch_bounds__(256) k_ut_times_x(const T* __restrict__ U, int64_t M, int64_t N,
                                                    const double* __restrict__ xs, double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < N; i += nwarp) {
        const T* col = U + (size_t)i * M;
        double s = 0.0;
        for (int64_t r = lane; r < M; r += 32) s += (double)col[r] * xs[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
}

// h[i] = sum_r (U[i, r] inv_sig[r])^2  (one warp per orbit)
template <typename T>
__global__ void __launch_bounds__(256) k_colnorm2(const T* __restrict__ U, int64_t M, int64_t N,
                                                  const double* __restrict__ inv_sig, double* __restrict__ h)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < N; i += nwarp) {
        const T* col = U + (size_t)i * M;
        double s = 0.0;
        if constexpr (sizeof(T) == 4) {
            // FP32 products, each lane's sum in FP32 (a few hundred terms, ~1e-6 relative: the norms set
            // the Jacobi scaling and the ranking of violators), the warp's total in FP64
            float sf = 0.f;
            for (int64_t r = lane; r < M; r += 32) {
                const float v = col[r] * (float)inv_sig[r];
                sf = fmaf(v, v, sf);
            }
            s = (double)sf;
        } else {
            for (int64_t r = lane; r < M; r += 32) {
                double v = (double)col[r] * inv_sig[r];
                s += v * v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) h[i] = s;
    }
}

// KKT of min 1/2 w^T H w - q^T w, w >= 0 with the exact gradient
// grad = H w - q = -(U~^T e) + (2 lam / N) w  (e = y~ - U~ w):
// projected gradient pg = grad where w > 0, min(grad, 0) where w = 0.
// out: g_neg[i] = U~^T e - (2 lam/N) w (the negative gradient) and atomic max |pg| (float bits)
__global__ void k_kkt(int64_t N, const double* __restrict__ ute, const double* __restrict__ w, double two_lam_n,
                      double* __restrict__ gneg, unsigned long long* pgmax)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double g = ute[i] - two_lam_n * w[i];
        gneg[i] = g;
        double grad = -g;
        double pg = w[i] > 0.0 ? grad : fmin(grad, 0.0);
        m = fmax(m, fabs(pg));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(pgmax, (unsigned long long)__double_as_longlong(m));
}

// chi2 parts: [sum e^2, sum_{r >= nd} e^2] and reg sum w^2
__global__ void k_chi2(int64_t M, int64_t nd, const double* __restrict__ e, int64_t N, const double* __restrict__ w,
                       double* __restrict__ out3)
{
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (int64_t)gridDim.x * blockDim.x) {
        double v = e[r] * e[r];
        a += v;
        if (r >= nd) b += v;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        c += w[i] * w[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out3 + 0, a);
        atomicAdd(out3 + 1, b);
        atomicAdd(out3 + 2, c);
    }
}

// inv_sig = 1/sigma, yt = y / sigma (both FP64); flags a non-positive sigma.
__global__ void k_prep_data(int64_t M, const double* __restrict__ sigma, const double* __restrict__ y,
                            double* __restrict__ inv_sig, double* __restrict__ ys, int* bad)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (int64_t)gridDim.x * blockDim.x) {
        double s = sigma[r];
        if (!(s > 0.0) || !isfinite(s) || !isfinite(y[r])) { atomicExch(bad, 1); s = 1.0; }
        inv_sig[r] = 1.0 / s;
        ys[r] = y[r] / s * (1.0 / s);   // y / sigma^2, the weight of U in q = U~^T y~
    }
}

// elementwise helpers
template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* __restrict__ a, B* __restrict__ b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (B)a[i];
}

// q' = t / s + g + (2 lam / N) w with t = A^T A (w / s) the Gram-precision
// product of the column-scaled matrix; warm start z = w, u = P^{-1} g.
template <typename GT>
__global__ void k_refine_rhs(int64_t N, const GT* __restrict__ t, const double* __restrict__ gneg,
                             const double* __restrict__ w, const double* __restrict__ s64, double two_lam_n,
                             const GT* __restrict__ rho_i, GT* __restrict__ qp, GT* __restrict__ z, GT* __restrict__ u)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        qp[i] = (GT)((double)t[i] / s64[i] + gneg[i] + two_lam_n * w[i]);
        z[i] = (GT)w[i];
        const double ri = (double)rho_i[i];
        u[i] = (GT)(ri > 0.0 ? gneg[i] / ri : 0.0);
    }
}

// out = a / b elementwise (double in, GT out)
template <typename GT>
__global__ void k_div_to(int64_t n, const double* __restrict__ a, const double* __restrict__ b, GT* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (GT)(a[i] / b[i]);
}

// R[k, r] = U[idx[k], r] * inv_sig[r]  (rows of the whitened matrix, FP64)
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ U, int64_t M, const int64_t* __restrict__ idx, int64_t nP,
                              const double* __restrict__ inv_sig, double* __restrict__ R)
{
    for (int64_t k = blockIdx.x; k < nP; k += gridDim.x) {
        const T* col = U + (size_t)idx[k] * M;
        double* row = R + (size_t)k * M;
        for (int64_t r = threadIdx.x; r < M; r += blockDim.x) row[r] = (double)col[r] * inv_sig[r];
    }
}

// Uc[k, :] = U[idx[k], :] (orbit columns of the stored matrix, unchanged)
template <typename T>
__global__ void k_gather_cols(const T* __restrict__ U, int64_t M, const int64_t* __restrict__ idx, int64_t n,
                              T* __restrict__ Uc)
{
    for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
        const T* src = U + (size_t)idx[k] * M;
        T* dst = Uc + (size_t)k * M;
        for (int64_t r = threadIdx.x; r < M; r += blockDim.x) dst[r] = src[r];
    }
}

// out[idx[k]] = a[k]
__global__ void k_scatter_vec(const double* __restrict__ a, const int64_t* __restrict__ idx, int64_t n,
                              double* __restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[idx[k]] = a[k];
}

__global__ void k_gather_vec(const double* __restrict__ a, const int64_t* __restrict__ idx, int64_t n,
                             double* __restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = a[idx[k]];
}

// ===========================================================================
// host launchers
// ===========================================================================
static inline unsigned cap_grid(int64_t n, int b, int64_t cap = 1 << 20)
{
    int64_t g = (n + b - 1) / b;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

template <typename T, typename AT>
cudaError_t whiten(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* inv_sig, const double* cs, AT* A,
                   AT* Alo, int64_t ldA, bool orbit_space)
{
    LaunchTimer lt(ctx, K_WHITEN);
    add_work(ctx, K_WHITEN, (double)M * N * (sizeof(T) + (Alo ? 2.0 : 1.0) * sizeof(AT)));
    if constexpr (sizeof(T) == 4 && sizeof(AT) == 2) {
        if (orbit_space && (ldA & 1) == 0) {
            // 1/sigma in FP32 once per call (M values), then the FP32 pass
            if (ctx->ensure(&ctx->d_invsig_f, &ctx->invsig_f_cap, (size_t)M * sizeof(float), "1/sigma (FP32)") !=
                SW_OK)
                return cudaErrorMemoryAllocation;
            float* isf = (float*)ctx->d_invsig_f;
            k_to_float<<<cap_grid(M, 256, 1024), 256, 0, ctx_stream(ctx)>>>(M, inv_sig, isf);
            k_whiten_orbit_f32<<<cap_grid(N, 1, 65536), 256, 0, ctx_stream(ctx)>>>(U, M, N, isf, cs, A, Alo, ldA);
            return cudaGetLastError();
        }
    }
    if (orbit_space) {
        k_whiten_orbit<T, AT><<<cap_grid(N, 1, 65536), 256, 0, ctx_stream(ctx)>>>(U, M, N, inv_sig, cs, A, Alo, ldA);
    } else {
        dim3 grid((unsigned)((ldA + 31) / 32), (unsigned)((M + 31) / 32));
        k_whiten_transpose<T, AT><<<grid, dim3(32, 8), 0, ctx_stream(ctx)>>>(U, M, N, inv_sig, cs, A, Alo, ldA);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t colnorm2(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* inv_sig, double* h)
{
    LaunchTimer lt(ctx, K_MISC);
    k_colnorm2<T><<<cap_grid(N * 32, 256, ctx_sms(ctx) * 64), 256, 0, ctx_stream(ctx)>>>(U, M, N, inv_sig, h);
    return cudaGetLastError();
}

template <typename GT>
cudaError_t admm_scales(sw_ctx* ctx, int64_t N, const double* h, double two_lam_n, double rho, double floor_,
                        double* s64, GT* s, GT* rho_i, GT* d)
{
    LaunchTimer lt(ctx, K_MISC);
    k_admm_scales<GT><<<cap_grid(N, 256, 4096), 256, 0, ctx_stream(ctx)>>>(N, h, two_lam_n, rho, floor_, s64, s,
                                                                           rho_i, d);
    return cudaGetLastError();
}

template <typename GT>
cudaError_t div_to(sw_ctx* ctx, int64_t n, const double* a, const double* b, GT* out)
{
    LaunchTimer lt(ctx, K_MISC);
    k_div_to<GT><<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, a, b, out);
    return cudaGetLastError();
}

template <typename T, bool BT, bool LOWER>
cudaError_t gemm(sw_ctx* ctx, int kid, int64_t m, int64_t n, int64_t k, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, int64_t diag_off)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, kid);
    add_work(ctx, kid, LOWER ? (double)m * (double)(n + 1) * (double)k : 2.0 * (double)m * (double)n * (double)k);
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 63) / 64));
    k_gemm<T, BT, LOWER><<<grid, 256, 0, ctx_stream(ctx)>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, diag_off);
    return cudaGetLastError();
}

template <typename T, bool BT, bool TRI>
cudaError_t gemm_acc(sw_ctx* ctx, int kid, int64_t m, int64_t n, int64_t k, T alpha, const T* A, int64_t lda,
                     const T* B, int64_t ldb, T* C, int64_t ldc)
{
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, kid);
    add_work(ctx, kid, (TRI ? 1.0 : 2.0) * (double)m * (double)n * (double)k);
    const int64_t gx = (n + 63) / 64, gy = (m + 63) / 64;
    // about four CTAs per SM over the tiles; slices of at least 256 (a multiple of 16)
    const int64_t want = std::max<int64_t>(1, (int64_t)ctx_sms(ctx) * 4 / std::max<int64_t>(1, gx * gy));
    int64_t kchunk = std::max<int64_t>(256, (k + want - 1) / want);
    kchunk = (kchunk + 15) / 16 * 16;
    const int64_t gz = (k + kchunk - 1) / kchunk;
    if (gz > 65535) return cudaErrorInvalidValue;
    k_gemm_acc<T, BT, TRI><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), 256, 0, ctx_stream(ctx)>>>(
        m, n, k, alpha, A, lda, B, ldb, C, ldc, kchunk);
    return cudaGetLastError();
}

template <typename T>
static size_t smem2() { return 2 * sizeof(T) * NB * (NB + 1); }

// Cholesky factor L of G (in place, lower) and X = L^{-1}.  Per 64-wide step: one CTA
// factors the diagonal block and inverts it (D_k = L_kk^{-1}); the panel below becomes
// P = A D_k^T, a plain GEMM over all rows instead of a row-by-row substitution; then the
// trailing update.  The inverse X is then built by block rows from the kept D_k.
template <typename T>
cudaError_t cholesky_inverse(sw_ctx* ctx, T* G, T* X, T* D, int64_t K, int* d_info)
{
    (void)D;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_diag_factor_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<T>());
        cudaFuncSetAttribute(k_trmm_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<T>());
        attr_set = true;
    }
    if (K <= 0) return cudaSuccess;
    cudaStream_t st = ctx_stream(ctx);
    const int64_t nb = (K + NB - 1) / NB;
    const size_t dbytes = (size_t)nb * NB * NB * sizeof(T), pbytes = (size_t)K * NB * sizeof(T);
    if (ctx->ensure(&ctx->d_chol, &ctx->chol_cap, dbytes + pbytes + 256, "factor scratch") != SW_OK)
        return cudaErrorMemoryAllocation;
    T* Dall = (T*)ctx->d_chol;
    T* P = (T*)((char*)ctx->d_chol + ((dbytes + 255) & ~(size_t)255));
    cudaError_t e;
    for (int64_t jb = 0; jb < nb; ++jb) {
        const int64_t j0 = jb * NB;
        const int bs = (int)(K - j0 < NB ? K - j0 : NB);
        T* Dk = Dall + (size_t)jb * NB * NB;
        {
            LaunchTimer lt(ctx, K_POTRF_DIAG);
            add_work(ctx, K_POTRF_DIAG, 2.0 * (double)bs * bs * bs / 3.0);
            k_diag_factor_inv<T><<<1, 256, smem2<T>(), st>>>(G, K, j0, bs, Dk, d_info);
        }
        if ((e = cudaGetLastError())) return e;
        const int64_t r0 = j0 + bs;
        if (r0 < K) {
            e = gemm<T, true, false>(ctx, K_TRSM_PANEL, K - r0, bs, bs, T(1), G + (size_t)r0 * K + j0, K, Dk, NB, T(0),
                                     P, NB, 0);
            if (!e) e = cudaMemcpy2DAsync(G + (size_t)r0 * K + j0, K * sizeof(T), P, NB * sizeof(T), bs * sizeof(T),
                                          K - r0, cudaMemcpyDeviceToDevice, st);
            if (!e)
                e = gemm<T, true, true>(ctx, K_SYRK_UPDATE, K - r0, K - r0, bs, T(-1), G + (size_t)r0 * K + j0, K,
                                        G + (size_t)r0 * K + j0, K, T(1), G + (size_t)r0 * K + r0, K, 0);
            if (e) return e;
        }
    }
    {
        LaunchTimer lt(ctx, K_MISC);
        k_set_identity<T><<<cap_grid(K * K, 256, 65536), 256, 0, st>>>(X, K);
    }
    for (int64_t jb = 0; jb < nb; ++jb) {
        const int64_t j0 = jb * NB;
        const int bs = (int)(K - j0 < NB ? K - j0 : NB);
        const int64_t ncols = j0 + bs;
        {
            LaunchTimer lt(ctx, K_TRINV_DIAG);
            add_work(ctx, K_TRINV_DIAG, 2.0 * (double)bs * bs * (double)ncols);
            k_trmm_diag<T><<<(unsigned)((ncols + NB - 1) / NB), 64, smem2<T>(), st>>>(X, K, j0, bs, ncols,
                                                                                    Dall + (size_t)jb * NB * NB);
        }
        const int64_t r0 = j0 + bs;
        if (r0 < K) {
            e = gemm<T, false, false>(ctx, K_TRINV_UPDATE, K - r0, ncols, bs, T(-1), G + (size_t)r0 * K + j0, K,
                                      X + (size_t)j0 * K, K, T(1), X + (size_t)r0 * K, K, 0);
            if (e) return e;
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t shift_and_trace(sw_ctx* ctx, T* G, int64_t K, double* d_trace, double shift)
{
    LaunchTimer lt(ctx, K_SHIFT);
    if (d_trace) k_trace<T><<<cap_grid(K, 256, 1024), 256, 0, ctx_stream(ctx)>>>(G, K, d_trace);
    else k_shift_diag<T><<<cap_grid(K, 256, 1024), 256, 0, ctx_stream(ctx)>>>(G, K, shift);
    return cudaGetLastError();
}

template <typename T>
cudaError_t shift_diag_vec(sw_ctx* ctx, T* G, int64_t K, int64_t ld, const double* d)
{
    LaunchTimer lt(ctx, K_SHIFT);
    k_shift_diag_vec<T><<<cap_grid(K, 256, 1024), 256, 0, ctx_stream(ctx)>>>(G, K, ld, d);
    return cudaGetLastError();
}
template cudaError_t shift_diag_vec<float>(sw_ctx*, float*, int64_t, int64_t, const double*);
template cudaError_t shift_diag_vec<double>(sw_ctx*, double*, int64_t, int64_t, const double*);

template <typename GT>
cudaError_t scale_to(sw_ctx* ctx, int64_t n, const double* a, const double* s, GT* out)
{
    LaunchTimer lt(ctx, K_MISC);
    k_scale_to<GT><<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, a, s, out);
    return cudaGetLastError();
}
template <typename GT>
cudaError_t as_residual(sw_ctx* ctx, int64_t n, const double* q, const double* g, const double* x, double mu,
                        const double* s, GT* rs)
{
    LaunchTimer lt(ctx, K_RESID);
    k_as_residual<GT><<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, q, g, x, mu, s, rs);
    return cudaGetLastError();
}
template <typename GT>
cudaError_t axpy_scaled(sw_ctx* ctx, int64_t n, const GT* c, const double* s, double* x)
{
    LaunchTimer lt(ctx, K_MISC);
    k_axpy_scaled<GT><<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, c, s, x);
    return cudaGetLastError();
}
cudaError_t weight_sq(sw_ctx* ctx, int64_t m, const double* acc, const double* inv_sig, double* xs)
{
    LaunchTimer lt(ctx, K_RESID);
    k_weight_sq<<<cap_grid(m, 256, 4096), 256, 0, ctx_stream(ctx)>>>(m, acc, inv_sig, xs);
    return cudaGetLastError();
}
template cudaError_t scale_to<float>(sw_ctx*, int64_t, const double*, const double*, float*);
template cudaError_t scale_to<double>(sw_ctx*, int64_t, const double*, const double*, double*);
template cudaError_t as_residual<float>(sw_ctx*, int64_t, const double*, const double*, const double*, double,
                                        const double*, float*);
template cudaError_t as_residual<double>(sw_ctx*, int64_t, const double*, const double*, const double*, double,
                                         const double*, double*);
template cudaError_t axpy_scaled<float>(sw_ctx*, int64_t, const float*, const double*, double*);
template cudaError_t axpy_scaled<double>(sw_ctx*, int64_t, const double*, const double*, double*);

template <typename T>
cudaError_t symmetrize(sw_ctx* ctx, const T* G, int64_t K, T* S)
{
    LaunchTimer lt(ctx, K_MISC);
    dim3 grid((unsigned)((K + 31) / 32), (unsigned)((K + 31) / 32));
    k_symmetrize<T><<<grid, dim3(32, 8), 0, ctx_stream(ctx)>>>(G, K, S);
    return cudaGetLastError();
}
template cudaError_t symmetrize<float>(sw_ctx*, const float*, int64_t, float*);
template cudaError_t symmetrize<double>(sw_ctx*, const double*, int64_t, double*);

template <typename AT, typename XT, typename YT, typename ACC>
cudaError_t rowdot(sw_ctx* ctx, int kid, const AT* A, int64_t rows, int64_t cols, int64_t lda, const XT* x, YT* y,
                   double alpha, double beta, bool lower, const AT* A2)
{
    if (rows <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, kid);
    add_work(ctx, kid, (double)rows * cols * sizeof(AT) * (lower ? 0.5 : 1.0) * (A2 ? 2.0 : 1.0));
    k_rowdot<AT, XT, YT, ACC><<<cap_grid(rows * 32, 256, ctx_sms(ctx) * 64), 256, 0, ctx_stream(ctx)>>>(
        A, A2, rows, cols, lda, x, y, alpha, beta, lower);
    return cudaGetLastError();
}

// y must be pre-initialised (it is accumulated into)
template <typename AT, typename XT, typename YT, typename ACC>
cudaError_t colcomb(sw_ctx* ctx, int kid, const AT* A, int64_t rows, int64_t cols, int64_t lda, const XT* x, YT* y,
                    double alpha, bool lower, const AT* A2)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, kid);
    add_work(ctx, kid, (double)rows * cols * sizeof(AT) * (lower ? 0.5 : 1.0) * (A2 ? 2.0 : 1.0));
    int64_t pairs = (cols + 1) / 2;
    unsigned gx = (unsigned)((pairs + 255) / 256);
    // enough blocks to fill the GPU several times over, rows split evenly
    int64_t want = (ctx_sms(ctx) * 16 + gx - 1) / gx;
    if (want < 1) want = 1;
    int64_t rps = (rows + want - 1) / want;
    if (rps < 32) rps = 32;
    unsigned gy = (unsigned)((rows + rps - 1) / rps);
    k_colcomb<AT, XT, YT, ACC><<<dim3(gx, gy), 256, 0, ctx_stream(ctx)>>>(A, A2, rows, cols, lda, x, y, alpha, rps,
                                                                          lower);
    return cudaGetLastError();
}

template <typename GT>
cudaError_t admm_update(sw_ctx* ctx, int64_t N, const GT* y, const GT* v, const GT* s, const GT* rho_i, const GT* d,
                        const GT* qp, double alpha, GT* rs, GT* z, GT* u, unsigned* stats)
{
    LaunchTimer lt(ctx, K_ADMM_UPDATE);
    k_admm_update<GT><<<cap_grid(N, 256, ctx_sms(ctx) * 8), 256, 0, ctx_stream(ctx)>>>(N, y, v, s, rho_i, d, qp, (GT)alpha,
                                                                              rs, z, u, stats);
    return cudaGetLastError();
}

template <typename GT>
cudaError_t admm_init(sw_ctx* ctx, int64_t N, const GT* qp, const GT* z, const GT* u, const GT* s, const GT* rho_i,
                      GT* rs)
{
    LaunchTimer lt(ctx, K_MISC);
    k_admm_init<GT><<<cap_grid(N, 256, ctx_sms(ctx) * 8), 256, 0, ctx_stream(ctx)>>>(N, qp, z, u, s, rho_i, rs);
    return cudaGetLastError();
}

static cudaError_t split_ff(sw_ctx* ctx, const double* x, int64_t n, float** hi, float** lo)
{
    if (ctx->ensure(&ctx->d_split, &ctx->split_cap, (size_t)2 * n * sizeof(float), "split vector") != SW_OK)
        return cudaErrorMemoryAllocation;
    *hi = (float*)ctx->d_split;
    *lo = *hi + n;
    k_split_ff<<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, x, *hi, *lo);
    return cudaGetLastError();
}

// U w for an FP32 matrix with w already split: rows in 16-byte groups when the columns allow it
static void launch_u_times_w_ff(sw_ctx* ctx, const float* U, int64_t M, int64_t N, const float* wh, const float* wl,
                                double* acc)
{
    const bool vec = M % 4 == 0 && ((uintptr_t)U & 15) == 0;
    const int64_t rows_per_cta = vec ? 1024 : 256;
    const unsigned gx = (unsigned)((M + rows_per_cta - 1) / rows_per_cta);
    int64_t want = (ctx_sms(ctx) * 16 + gx - 1) / gx;
    if (want < 1) want = 1;
    int64_t ops = (N + want - 1) / want;
    if (ops < 16) ops = 16;
    const unsigned gy = (unsigned)((N + ops - 1) / ops);
    if (vec) k_u_times_w_ff<true><<<dim3(gx, gy), 256, 0, ctx_stream(ctx)>>>(U, M, N, wh, wl, acc, ops);
    else k_u_times_w_ff<false><<<dim3(gx, gy), 256, 0, ctx_stream(ctx)>>>(U, M, N, wh, wl, acc, ops);
}

template <typename T>
cudaError_t u_times_w(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* w, double* acc)
{
    LaunchTimer lt(ctx, K_RESID);
    add_work(ctx, K_RESID, (double)M * N * sizeof(T) + 8.0 * (N + 2.0 * M));
    unsigned gx = (unsigned)((M + 255) / 256);
    int64_t want = (ctx_sms(ctx) * 16 + gx - 1) / gx;
    if (want < 1) want = 1;
    int64_t ops = (N + want - 1) / want;
    if (ops < 16) ops = 16;
    unsigned gy = (unsigned)((N + ops - 1) / ops);
    if constexpr (sizeof(T) == 4) {
        float *wh, *wl;
        cudaError_t e = split_ff(ctx, w, N, &wh, &wl);
        if (e) return e;
        launch_u_times_w_ff(ctx, U, M, N, wh, wl, acc);
    } else {
        k_u_times_w<T><<<dim3(gx, gy), 256, 0, ctx_stream(ctx)>>>(U, M, N, w, acc, ops);
    }
    return cudaGetLastError();
}

cudaError_t u_times_w_presplit(sw_ctx* ctx, const float* U, int64_t M, int64_t N, const double* w, float* wh,
                               float* wl, double* acc)
{
    LaunchTimer lt(ctx, K_RESID);
    add_work(ctx, K_RESID, (double)M * N * sizeof(float) + 8.0 * (N + 2.0 * M));
    k_split_ff<<<cap_grid(N, 256, 4096), 256, 0, ctx_stream(ctx)>>>(N, w, wh, wl);
    launch_u_times_w_ff(ctx, U, M, N, wh, wl, acc);
    return cudaGetLastError();
}

cudaError_t residual(sw_ctx* ctx, int64_t M, const double* y, const double* acc, const double* inv_sig, double* e,
                     double* xs)
{
    LaunchTimer lt(ctx, K_RESID);
    k_residual<<<cap_grid(M, 256, 4096), 256, 0, ctx_stream(ctx)>>>(M, y, acc, inv_sig, e, xs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t ut_times_x(sw_ctx* ctx, const T* U, int64_t M, int64_t N, const double* xs, double* out)
{
    LaunchTimer lt(ctx, K_GRAD);
    add_work(ctx, K_GRAD, (double)M * N * sizeof(T) + 8.0 * (N + M));
    if constexpr (sizeof(T) == 4) {
        float *xh, *xl;
        cudaError_t e = split_ff(ctx, xs, M, &xh, &xl);
        if (e) return e;
        const size_t smem = (size_t)M * 2 * sizeof(float);
        const bool vec = M % 4 == 0 && ((uintptr_t)U & 15) == 0 && ((uintptr_t)xh & 15) == 0 &&
                         ((uintptr_t)xl & 15) == 0 && smem <= 200 * 1024;
        static size_t smem_set = 0;
        if (vec && smem > smem_set) {
            if (cudaFuncSetAttribute(k_ut_times_x_ff_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                cudaSuccess)
                smem_set = 200 * 1024;
            else
                cudaGetLastError();
        }
        if (vec && smem <= smem_set)
            k_ut_times_x_ff_sm<<<(unsigned)std::min<int64_t>(ctx_sms(ctx), (N + 31) / 32), UTX_THREADS, smem,
                                 ctx_stream(ctx)>>>(U, M, N, xh, xl, out);
        else
            k_ut_times_x_ff<<<cap_grid(N * 32, 256, ctx_sms(ctx) * 64), 256, 0, ctx_stream(ctx)>>>(U, M, N, xh, xl, out);
    } else {
        k_ut_times_x<T><<<cap_grid(N * 32, 256, ctx_sms(ctx) * 64), 256, 0, ctx_stream(ctx)>>>(U, M, N, xs, out);
    }
    return cudaGetLastError();
}

cudaError_t kkt(sw_ctx* ctx, int64_t N, const double* ute, const double* w, double two_lam_n, double* gneg,
                unsigned long long* pgmax)
{
    LaunchTimer lt(ctx, K_GRAD);
    k_kkt<<<cap_grid(N, 256, 4096), 256, 0, ctx_stream(ctx)>>>(N, ute, w, two_lam_n, gneg, pgmax);
    return cudaGetLastError();
}

cudaError_t chi2(sw_ctx* ctx, int64_t M, int64_t nd, const double* e, int64_t N, const double* w, double* out3)
{
    LaunchTimer lt(ctx, K_CHI2);
    int64_t mx = M > N ? M : N;
    k_chi2<<<cap_grid(mx, 256, 4096), 256, 0, ctx_stream(ctx)>>>(M, nd, e, N, w, out3);
    return cudaGetLastError();
}

cudaError_t prep_data(sw_ctx* ctx, int64_t M, const double* sigma, const double* y, double* inv_sig, double* ys,
                      int* bad)
{
    LaunchTimer lt(ctx, K_MISC);
    k_prep_data<<<cap_grid(M, 256, 4096), 256, 0, ctx_stream(ctx)>>>(M, sigma, y, inv_sig, ys, bad);
    return cudaGetLastError();
}

template <typename A, typename B>
cudaError_t convert(sw_ctx* ctx, int64_t n, const A* a, B* b)
{
    LaunchTimer lt(ctx, K_MISC);
    k_convert<A, B><<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(n, a, b);
    return cudaGetLastError();
}

template <typename GT>
cudaError_t refine_rhs(sw_ctx* ctx, int64_t N, const GT* t, const double* gneg, const double* w, const double* s64,
                       double two_lam_n, const GT* rho_i, GT* qp, GT* z, GT* u)
{
    LaunchTimer lt(ctx, K_MISC);
    k_refine_rhs<GT><<<cap_grid(N, 256, 4096), 256, 0, ctx_stream(ctx)>>>(N, t, gneg, w, s64, two_lam_n, rho_i, qp, z,
                                                                          u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_rows(sw_ctx* ctx, const T* U, int64_t M, const int64_t* idx, int64_t nP, const double* inv_sig,
                        double* R)
{
    if (nP <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, K_MISC);
    k_gather_rows<T><<<cap_grid(nP, 1, 65536), 256, 0, ctx_stream(ctx)>>>(U, M, idx, nP, inv_sig, R);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_cols(sw_ctx* ctx, const T* U, int64_t M, const int64_t* idx, int64_t n, T* Uc)
{
    if (n <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, K_MISC);
    k_gather_cols<T><<<cap_grid(n, 1, 65536), 256, 0, ctx_stream(ctx)>>>(U, M, idx, n, Uc);
    return cudaGetLastError();
}
template cudaError_t gather_cols<float>(sw_ctx*, const float*, int64_t, const int64_t*, int64_t, float*);
template cudaError_t gather_cols<double>(sw_ctx*, const double*, int64_t, const int64_t*, int64_t, double*);

cudaError_t scatter_vec(sw_ctx* ctx, const double* a, const int64_t* idx, int64_t n, double* out)
{
    if (n <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, K_MISC);
    k_scatter_vec<<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(a, idx, n, out);
    return cudaGetLastError();
}

cudaError_t gather_vec(sw_ctx* ctx, const double* a, const int64_t* idx, int64_t n, double* out)
{
    if (n <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, K_MISC);
    k_gather_vec<<<cap_grid(n, 256, 4096), 256, 0, ctx_stream(ctx)>>>(a, idx, n, out);
    return cudaGetLastError();
}

// ---- explicit instantiations -------------------------------------------------
template cudaError_t gather_rows<float>(sw_ctx*, const float*, int64_t, const int64_t*, int64_t, const double*,
                                        double*);
template cudaError_t gather_rows<double>(sw_ctx*, const double*, int64_t, const int64_t*, int64_t, const double*,
                                         double*);
#define SW_WH(T, AT) \
    template cudaError_t whiten<T, AT>(sw_ctx*, const T*, int64_t, int64_t, const double*, const double*, AT*, AT*, \
                                       int64_t, bool);
SW_WH(float, __nv_bfloat16)
SW_WH(float, float)
SW_WH(double, double)
template cudaError_t gemm<float, true, true>(sw_ctx*, int, int64_t, int64_t, int64_t, float, const float*, int64_t,
                                             const float*, int64_t, float, float*, int64_t, int64_t);
template cudaError_t gemm_acc<float, true, true>(sw_ctx*, int, int64_t, int64_t, int64_t, float, const float*,
                                                 int64_t, const float*, int64_t, float*, int64_t);
template cudaError_t gemm_acc<float, false, true>(sw_ctx*, int, int64_t, int64_t, int64_t, float, const float*,
                                                  int64_t, const float*, int64_t, float*, int64_t);
template cudaError_t gemm_acc<float, true, false>(sw_ctx*, int, int64_t, int64_t, int64_t, float, const float*,
                                                  int64_t, const float*, int64_t, float*, int64_t);
template cudaError_t gemm_acc<double, true, false>(sw_ctx*, int, int64_t, int64_t, int64_t, double,
                                                   const double*, int64_t, const double*, int64_t, double*, int64_t);
template cudaError_t gemm<float, false, false>(sw_ctx*, int, int64_t, int64_t, int64_t, float, const float*, int64_t,
                                               const float*, int64_t, float, float*, int64_t, int64_t);
template cudaError_t gemm<double, true, true>(sw_ctx*, int, int64_t, int64_t, int64_t, double, const double*,
                                              int64_t, const double*, int64_t, double, double*, int64_t, int64_t);
template cudaError_t cholesky_inverse<float>(sw_ctx*, float*, float*, float*, int64_t, int*);
template cudaError_t cholesky_inverse<double>(sw_ctx*, double*, double*, double*, int64_t, int*);
template cudaError_t shift_and_trace<float>(sw_ctx*, float*, int64_t, double*, double);
template cudaError_t shift_and_trace<double>(sw_ctx*, double*, int64_t, double*, double);
template cudaError_t rowdot<__nv_bfloat16, float, float, float>(sw_ctx*, int, const __nv_bfloat16*, int64_t, int64_t,
                                                               int64_t, const float*, float*, double, double, bool, const __nv_bfloat16*);
template cudaError_t colcomb<__nv_bfloat16, float, float, float>(sw_ctx*, int, const __nv_bfloat16*, int64_t,
                                                                int64_t, int64_t, const float*, float*, double, bool, const __nv_bfloat16*);
template cudaError_t rowdot<float, float, float, float>(sw_ctx*, int, const float*, int64_t, int64_t, int64_t,
                                                       const float*, float*, double, double, bool, const float*);
template cudaError_t rowdot<float, float, float, double>(sw_ctx*, int, const float*, int64_t, int64_t, int64_t,
                                                        const float*, float*, double, double, bool, const float*);
template cudaError_t colcomb<float, float, float, float>(sw_ctx*, int, const float*, int64_t, int64_t, int64_t,
                                                        const float*, float*, double, bool, const float*);
template cudaError_t rowdot<double, double, double, double>(sw_ctx*, int, const double*, int64_t, int64_t, int64_t,
                                                           const double*, double*, double, double, bool,
                                                           const double*);
template cudaError_t colcomb<double, double, double, double>(sw_ctx*, int, const double*, int64_t, int64_t, int64_t,
                                                            const double*, double*, double, bool, const double*);
#define SW_GT(GT)                                                                                                  \
    template cudaError_t admm_update<GT>(sw_ctx*, int64_t, const GT*, const GT*, const GT*, const GT*, const GT*,   \
                                         const GT*, double, GT*, GT*, GT*, unsigned*);                             \
    template cudaError_t admm_init<GT>(sw_ctx*, int64_t, const GT*, const GT*, const GT*, const GT*, const GT*, GT*); \
    template cudaError_t admm_scales<GT>(sw_ctx*, int64_t, const double*, double, double, double, double*, GT*, GT*, \
                                         GT*);                                                                     \
    template cudaError_t refine_rhs<GT>(sw_ctx*, int64_t, const GT*, const double*, const double*, const double*,   \
                                        double, const GT*, GT*, GT*, GT*);                                         \
    template cudaError_t div_to<GT>(sw_ctx*, int64_t, const double*, const double*, GT*);
SW_GT(float)
SW_GT(double)
template cudaError_t u_times_w<float>(sw_ctx*, const float*, int64_t, int64_t, const double*, double*);
template cudaError_t u_times_w<double>(sw_ctx*, const double*, int64_t, int64_t, const double*, double*);
template cudaError_t ut_times_x<float>(sw_ctx*, const float*, int64_t, int64_t, const double*, double*);
template cudaError_t ut_times_x<double>(sw_ctx*, const double*, int64_t, int64_t, const double*, double*);
template cudaError_t colnorm2<float>(sw_ctx*, const float*, int64_t, int64_t, const double*, double*);
template cudaError_t colnorm2<double>(sw_ctx*, const double*, int64_t, int64_t, const double*, double*);
template cudaError_t convert<double, float>(sw_ctx*, int64_t, const double*, float*);
template cudaError_t convert<float, double>(sw_ctx*, int64_t, const float*, double*);
template cudaError_t convert<double, double>(sw_ctx*, int64_t, const double*, double*);

}  // namespace sw
