// Cholesky factor and its explicit inverse in one cooperative launch.
//
// The blocked right-looking factorisation with 64-wide panels is a chain of
// K/64 steps; launching three kernels per step makes the host's launch rate
// and the single-CTA diagonal kernels the critical path.  Here one launch
// with every CTA resident walks the whole chain, separated by a grid barrier:
//
//   factor: for block column j: the panel below the diagonal block is
//           multiplied by D_j = L_jj^{-1} (tiles over all CTAs); then the
//           trailing lower tiles are updated, C -= P_i P_k^T, while CTA 0 first
//           updates and factors the next diagonal block (potrf and its inverse
//           D_{j+1}) so that the next panel step can start at once;
//   inverse: X = L^{-1} by block rows: X_k <- D_k X_k, then
//           X_i <- X_i - L_ik X_k for the rows below (tiles over all CTAs).
//
// The grid barrier is a sense-reversing counter whose waits are bounded by a
// global-timer deadline; on a timeout the kernel records an error and every CTA
// returns at its next barrier.
#include "sw_common.cuh"
#include "sw_api_internal.cuh"

#include <algorithm>

namespace sw {
namespace {

constexpr int TB = 64;           // tile / panel width
constexpr int THR = 256;         // threads per CTA
constexpr int LD = TB + 1;       // shared-memory row stride (no bank conflicts)

struct GridBar {
    unsigned count;
    unsigned gen;
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// all CTAs meet here; false once any wait has run out (then every CTA returns)
__device__ bool grid_barrier(GridBar* bar, int* err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &bar->gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const unsigned long long deadline = now_ns() + 2000000000ull;   // 2 s
            while (*vgen == g) {
                if (*(volatile int*)err || now_ns() > deadline) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = *(volatile int*)err == 0;
    }
    __syncthreads();
    return ok;
}

// load a TB x TB tile (rows r0.., cols c0..) of a row-major matrix into s, zero outside
// [0, nr) x [0, nc) of the tile and, when lower, above the diagonal of the global matrix
template <typename T>
__device__ __forceinline__ void load_tile(T (*s)[LD], const T* __restrict__ M, int64_t ld, int64_t r0, int64_t c0,
                                          int nr, int nc)
{
    for (int e = threadIdx.x; e < TB * TB; e += THR) {
        const int i = e / TB, j = e % TB;
        s[i][j] = (i < nr && j < nc) ? __ldcg(M + (size_t)(r0 + i) * ld + c0 + j) : T(0);
    }
}

// acc (4 x 4 per thread) = A B^T (transB) or A B over the shared tiles
template <typename T, bool TRANSB>
__device__ __forceinline__ void tile_mma(const T (*A)[LD], const T (*B)[LD], T acc[4][4])
{
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll 4
    for (int k = 0; k < TB; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[ty * 4 + i][k];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = TRANSB ? B[tx * 4 + j][k] : B[k][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
}

// diagonal block j0 (bs x bs): Cholesky in place in G and its inverse into D (TB x TB)
template <typename T>
__device__ void factor_diag(T* __restrict__ G, int64_t K, int64_t j0, int bs, T* __restrict__ D, int* info,
                            T (*a)[LD], T (*x)[LD])
{
    const int t = threadIdx.x;
    for (int e = t; e < TB * TB; e += THR) {
        const int i = e / TB, j = e % TB;
        a[i][j] = (i < bs && j <= i) ? __ldcg(G + (size_t)(j0 + i) * K + j0 + j) : T(0);
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
        if (t > j && t < bs) a[t][j] /= d;
        __syncthreads();
        if (t == j) a[j][j] = d;
        if (t > j && t < bs) {
            const T aij = a[t][j];
            for (int l = j + 1; l <= t; ++l) a[t][l] -= aij * a[l][j];
        }
        __syncthreads();
    }
    // inverse by forward substitution, thread t < bs owns column t
    if (t < bs) {
        x[t][t] = T(1) / a[t][t];
        for (int i = t + 1; i < bs; ++i) {
            T s = T(0);
            for (int l = t; l < i; ++l) s += a[i][l] * x[l][t];
            x[i][t] = -s / a[i][i];
        }
    }
    __syncthreads();
    for (int e = t; e < TB * TB; e += THR) {
        const int i = e / TB, j = e % TB;
        if (i < bs && j <= i) G[(size_t)(j0 + i) * K + j0 + j] = a[i][j];
        D[e] = x[i][j];
    }
    __syncthreads();
}

// lower-triangular tile index p -> (ti, tk), tk <= ti, counting from (0, 0)
__device__ __forceinline__ void tri_index(int64_t p, int64_t& ti, int64_t& tk)
{
    int64_t r = (int64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > p) --r;
    while ((r + 1) * (r + 2) / 2 <= p) ++r;
    ti = r;
    tk = p - r * (r + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(THR) k_chol_inverse(T* __restrict__ G, T* __restrict__ X, int64_t K,
                                                      T* __restrict__ Dall, int* info, GridBar* bar, int* err)
{
    extern __shared__ unsigned char smraw[];
    T (*A)[LD] = reinterpret_cast<T (*)[LD]>(smraw);
    T (*B)[LD] = reinterpret_cast<T (*)[LD]>(smraw + sizeof(T) * TB * LD);
    const int64_t nb = (K + TB - 1) / TB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    auto width = [&](int64_t b) { return (int)std::min<int64_t>(TB, K - b * TB); };

    // X = identity
    for (int64_t e = (int64_t)blockIdx.x * THR + threadIdx.x; e < K * K; e += (int64_t)gridDim.x * THR)
        X[e] = (e / K == e % K) ? T(1) : T(0);
    if (blockIdx.x == 0) factor_diag<T>(G, K, 0, width(0), Dall, info, A, B);
    if (!grid_barrier(bar, err)) return;

    for (int64_t jb = 0; jb < nb; ++jb) {
        const int64_t j0 = jb * TB;
        const int bs = width(jb);
        const T* D = Dall + (size_t)jb * TB * TB;
        // panel: P_i = A_ij D_j^T for the tiles below the diagonal block
        for (int64_t ib = jb + 1 + blockIdx.x; ib < nb; ib += gridDim.x) {
            const int rs = width(ib);
            load_tile<T>(A, G, K, ib * TB, j0, rs, bs);
            for (int e = threadIdx.x; e < TB * TB; e += THR) B[e / TB][e % TB] = __ldcg(D + e);
            __syncthreads();
            T acc[4][4] = {};
            tile_mma<T, true>(A, B, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = ty * 4 + i, c = tx * 4 + j;
                    if (r < rs && c < bs) G[(size_t)(ib * TB + r) * K + j0 + c] = acc[i][j];
                }
            __syncthreads();
        }
        if (!grid_barrier(bar, err)) return;
        // trailing update of the lower tiles (ti, tk), jb < tk <= ti; CTA 0 takes the
        // next diagonal tile first and factors it
        const int64_t m = nb - jb - 1;
        if (m > 0) {
            const int64_t ntiles = m * (m + 1) / 2;
            for (int64_t p = blockIdx.x; p < ntiles; p += gridDim.x) {
                int64_t ti, tk;
                tri_index(p, ti, tk);
                ti += jb + 1;
                tk += jb + 1;
                const int rs = width(ti), cs = width(tk);
                load_tile<T>(A, G, K, ti * TB, j0, rs, bs);
                load_tile<T>(B, G, K, tk * TB, j0, cs, bs);
                __syncthreads();
                T acc[4][4] = {};
                tile_mma<T, true>(A, B, acc);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int r = ty * 4 + i, c = tx * 4 + j;
                        if (r < rs && c < cs && (ti != tk || c <= r)) {
                            T* g = G + (size_t)(ti * TB + r) * K + tk * TB + c;
                            *g = __ldcg(g) - acc[i][j];
                        }
                    }
                __syncthreads();
                if (p == 0)   // tile (jb+1, jb+1) is complete: factor it now
                    factor_diag<T>(G, K, (jb + 1) * TB, width(jb + 1), Dall + (size_t)(jb + 1) * TB * TB, info, A, B);
            }
        }
        if (!grid_barrier(bar, err)) return;
    }

    // inverse by block rows
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * TB;
        const int bs = width(kb);
        const int64_t ncols = k0 + bs, nct = (ncols + TB - 1) / TB;
        const T* D = Dall + (size_t)kb * TB * TB;
        // X_k <- D_k X_k (block row k, columns 0..ncols)
        for (int64_t cb = blockIdx.x; cb < nct; cb += gridDim.x) {
            const int cs = (int)std::min<int64_t>(TB, ncols - cb * TB);
            for (int e = threadIdx.x; e < TB * TB; e += THR) A[e / TB][e % TB] = __ldcg(D + e);
            load_tile<T>(B, X, K, k0, cb * TB, bs, cs);
            __syncthreads();
            T acc[4][4] = {};
            tile_mma<T, false>(A, B, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = ty * 4 + i, c = tx * 4 + j;
                    if (r < bs && c < cs) X[(size_t)(k0 + r) * K + cb * TB + c] = acc[i][j];
                }
            __syncthreads();
        }
        if (!grid_barrier(bar, err)) return;
        // X_i -= L_ik X_k for block rows i > k
        const int64_t mrows = nb - kb - 1;
        const int64_t ntiles = mrows * nct;
        for (int64_t p = blockIdx.x; p < ntiles; p += gridDim.x) {
            const int64_t ib = kb + 1 + p / nct, cb = p % nct;
            const int rs = width(ib), cs = (int)std::min<int64_t>(TB, ncols - cb * TB);
            load_tile<T>(A, G, K, ib * TB, k0, rs, bs);
            load_tile<T>(B, X, K, k0, cb * TB, bs, cs);
            __syncthreads();
            T acc[4][4] = {};
            tile_mma<T, false>(A, B, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = ty * 4 + i, c = tx * 4 + j;
                    if (r < rs && c < cs) {
                        T* xp = X + (size_t)(ib * TB + r) * K + cb * TB + c;
                        *xp = __ldcg(xp) - acc[i][j];
                    }
                }
            __syncthreads();
        }
        if (!grid_barrier(bar, err)) return;
    }
}

}  // namespace

// One cooperative launch: L (in place in G's lower triangle) and X = L^{-1}.  Returns
// cudaErrorNotSupported when the device cannot launch it cooperatively (the caller then
// uses the multi-launch path); *d_err != 0 after the launch means a barrier wait ran out.
template <typename T>
cudaError_t cholesky_inverse_coop(sw_ctx* ctx, T* G, T* X, int64_t K, int* d_info, int* d_err)
{
    if (K <= 0) return cudaSuccess;
    static int grid = 0;
    const size_t smem = 2 * sizeof(T) * TB * LD;
    if (grid == 0) {
        int dev = 0, coop = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (!coop) { grid = -1; return cudaErrorNotSupported; }
        cudaFuncSetAttribute(k_chol_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_inverse<T>, THR, smem);
        if (per < 1) { grid = -1; return cudaErrorNotSupported; }
        grid = std::min(per, 2) * sms;
    }
    if (grid < 0) return cudaErrorNotSupported;
    const int64_t nb = (K + TB - 1) / TB;
    // scratch: the diagonal inverses (nb x TB x TB) and the barrier
    size_t need = (size_t)nb * TB * TB * sizeof(T) + 256;
    if (ctx->ensure(&ctx->d_chol, &ctx->chol_cap, need, "Cholesky scratch") != SW_OK) return cudaErrorMemoryAllocation;
    T* Dall = (T*)ctx->d_chol;
    GridBar* bar = (GridBar*)((char*)ctx->d_chol + (size_t)nb * TB * TB * sizeof(T));
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx->stream);
    if (e) return e;
    LaunchTimer lt(ctx, K_CHOL_COOP);
    add_work(ctx, K_CHOL_COOP, 2.0 * (double)K * K * K / 3.0);
    void* args[] = {&G, &X, &K, &Dall, &d_info, &bar, &d_err};
    return cudaLaunchCooperativeKernel((const void*)k_chol_inverse<T>, dim3(grid), dim3(THR), args, smem, ctx->stream);
}

template cudaError_t cholesky_inverse_coop<float>(sw_ctx*, float*, float*, int64_t, int*, int*);
template cudaError_t cholesky_inverse_coop<double>(sw_ctx*, double*, double*, int64_t, int*, int*);

}  // namespace sw
