// Learned chi^2 emulator: a fully connected network n_in -> width (x n_hidden,
// SiLU) -> 1, trained by mean-squared error with Adam (Kingma & Ba 2015), all in
// hand-written kernels.  The paper runs its MCMC on the exact chi^2 (Sec. 3.2,
// 1.3 s per evaluation) and names differentiable surrogates as the way to cheaper
// likelihoods (Sec. 5.3); here the network screens MCMC proposals before the
// exact model judges them (delayed acceptance, Christen & Fox 2005).
//
// Parameters are one FP32 array: for each layer l, W_l (out x in, row-major)
// followed by b_l (out).  Activations of a batch live in a context scratch
// buffer: for each hidden layer the pre-activation Z_l and the output H_l
// (batch x width, row-major), then the network output.
#include "sw_common.cuh"
#include "sw_api_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace sw {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ float ld_round(float v, bool bf16)
{
    return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// C[m, n] (row-major, ldc) = sum_k A(m, k) B(k, n) (+ C when accumulate), with
// A(m, k) = A[m sam + k sak] and B(k, n) = B[k sbk + n sbn]: one kernel serves the
// forward (X W^T), weight-gradient (D^T H) and input-gradient (D W) products.
// 256 threads, 64 x 64 tile, 4 x 4 outputs per thread.  With bf16 set, both
// operands are rounded to BF16 as they are loaded (FP32 accumulation).
__global__ void __launch_bounds__(256) k_mlp_gemm(int M, int N, int K, const float* __restrict__ A, int64_t sam,
                                                  int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbn,
                                                  float* __restrict__ C, int64_t ldc, bool accumulate, bool bf16)
{
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int mm = e / TK, kk = e % TK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? ld_round(A[(int64_t)m * sam + (int64_t)k * sak], bf16) : 0.f;
        }
        for (int e = threadIdx.x; e < TN * TK; e += 256) {
            const int kk = e / TN, nn = e % TN;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < K) ? ld_round(B[(int64_t)k * sbk + (int64_t)n * sbn], bf16) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float* c = C + (int64_t)m * ldc + n;
            *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
    }
}

__device__ __forceinline__ float sigm(float a) { return 1.f / (1.f + __expf(-a)); }

// Z += b (per column); H = silu(Z) = Z sigma(Z) when act, else H = Z
__global__ void k_mlp_bias_act(int64_t rows, int cols, const float* __restrict__ b, float* __restrict__ Z,
                               float* __restrict__ H, bool act)
{
    const int64_t n = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[e] + b[e % cols];
        Z[e] = z;
        H[e] = act ? z * sigm(z) : z;
    }
}

// D = 2 / B (out - t); loss += sum (out - t)^2
__global__ void k_mlp_mse(int64_t B, const float* __restrict__ out, const float* __restrict__ t,
                          float* __restrict__ D, double* __restrict__ loss)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = out[i] - t[i];
        D[i] = 2.f / (float)B * r;
        s += (double)r * r;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// D *= silu'(Z) = sigma(Z) (1 + Z (1 - sigma(Z)))
__global__ void k_mlp_silu_bwd(int64_t n, const float* __restrict__ Z, float* __restrict__ D)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[e], s = sigm(z);
        D[e] *= s * (1.f + z * (1.f - s));
    }
}

// g[c] = sum_r D[r, c] (one warp per column)
__global__ void k_mlp_colsum(int64_t rows, int cols, const float* __restrict__ D, float* __restrict__ g)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x & 31;
    if (warp >= cols) return;
    float s = 0.f;
    for (int64_t r = lane; r < rows; r += 32) s += D[r * cols + warp];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[warp] = s;
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

inline int grid_for(const sw_ctx* ctx, int64_t n, int threads = 256)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)ctx_sms(ctx) * 8));
}

struct Net {
    int n_in, width, n_hidden;
    int layers() const { return n_hidden + 1; }
    int in(int l) const { return l == 0 ? n_in : width; }
    int out(int l) const { return l == n_hidden ? 1 : width; }
    int64_t w_off(int l) const
    {
        int64_t o = 0;
        for (int k = 0; k < l; ++k) o += (int64_t)out(k) * in(k) + out(k);
        return o;
    }
    int64_t count() const { return w_off(layers()); }
};

bool valid(const Net& n) { return n.n_in >= 1 && n.width >= 1 && n.n_hidden >= 1 && n.n_in <= 4096 && n.width <= 8192; }

cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B,
                 int64_t sbk, int64_t sbn, float* C, int64_t ldc, bool acc, bool bf16)
{
    dim3 g((N + TN - 1) / TN, (M + TM - 1) / TM);
    k_mlp_gemm<<<g, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, acc, bf16);
    return cudaGetLastError();
}

// forward pass; activations in the scratch: Z_l, H_l for hidden l, then the output.
// Returns the output pointer.
cudaError_t forward(sw_ctx* ctx, const Net& n, const float* P, const float* X, int64_t Bn, bool bf16, float* ws,
                    float** out)
{
    cudaStream_t st = ctx->stream;
    const float* h = X;
    float* z = ws;
    for (int l = 0; l < n.layers(); ++l) {
        const int in = n.in(l), o = n.out(l);
        const float* W = P + n.w_off(l);
        const float* b = W + (int64_t)o * in;
        float* Z = z;
        float* H = (l < n.n_hidden) ? z + Bn * o : z;
        cudaError_t e;
        {
            LaunchTimer lt(ctx, K_MLP_FWD);
            e = gemm(st, (int)Bn, o, in, h, in, 1, W, 1, in, Z, o, false, bf16);
            if (!e) {
                k_mlp_bias_act<<<grid_for(ctx, Bn * o), 256, 0, st>>>(Bn, o, b, Z, H, l < n.n_hidden);
                e = cudaGetLastError();
            }
        }
        if (e) return e;
        h = H;
        z = (l < n.n_hidden) ? z + 2 * Bn * o : z;
    }
    *out = const_cast<float*>(h);
    return cudaSuccess;
}

size_t scratch_floats(const Net& n, int64_t Bn) { return (size_t)Bn * (2 * n.width * n.n_hidden + 1 + 2 * n.width); }

}  // namespace
}  // namespace sw

using namespace sw;

extern "C" int64_t sw_mlp_param_count(int n_in, int width, int n_hidden)
{
    Net n{n_in, width, n_hidden};
    return valid(n) ? n.count() : -1;
}

extern "C" sw_status sw_mlp_forward(sw_ctx* ctx, int n_in, int width, int n_hidden, const float* params_dev,
                                    const float* x_dev, int64_t batch, int bf16, float* out_dev)
{
    CHECK_CTX(ctx);
    Net n{n_in, width, n_hidden};
    if (!valid(n) || batch < 0 || !params_dev || !out_dev || (batch > 0 && !x_dev)) {
        set_error(ctx, "sw_mlp_forward: invalid network shape or NULL argument");
        return SW_EINVAL;
    }
    if (batch == 0) return SW_OK;
    sw_status s = ctx->ensure(&ctx->d_mlp, &ctx->mlp_cap, scratch_floats(n, batch) * sizeof(float), "MLP scratch");
    if (s != SW_OK) return s;
    float* out = nullptr;
    cudaError_t e = forward(ctx, n, params_dev, x_dev, batch, bf16 != 0, (float*)ctx->d_mlp, &out);
    if (!e) e = cudaMemcpyAsync(out_dev, out, batch * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    return e ? ctx->cuda_fail(e, "MLP forward") : SW_OK;
}

extern "C" sw_status sw_mlp_loss_grad(sw_ctx* ctx, int n_in, int width, int n_hidden, const float* params_dev,
                                      const float* x_dev, const float* t_dev, int64_t batch, float* grad_dev,
                                      double* loss_out)
{
    CHECK_CTX(ctx);
    Net n{n_in, width, n_hidden};
    if (!valid(n) || batch < 1 || !params_dev || !x_dev || !t_dev || !grad_dev || !loss_out) {
        set_error(ctx, "sw_mlp_loss_grad: invalid network shape, empty batch or NULL argument");
        return SW_EINVAL;
    }
    const size_t need = scratch_floats(n, batch) * sizeof(float) + 64;
    sw_status s = ctx->ensure(&ctx->d_mlp, &ctx->mlp_cap, need, "MLP scratch");
    if (s != SW_OK) return s;
    cudaStream_t st = ctx->stream;
    float* ws = (float*)ctx->d_mlp;
    float* out = nullptr;
    cudaError_t e = forward(ctx, n, params_dev, x_dev, batch, false, ws, &out);
    // gradient buffers after the activations: D (batch x width) and its successor
    float* D = ws + (size_t)batch * (2 * n.width * n.n_hidden + 1);
    float* D2 = D + (size_t)batch * n.width;
    double* dloss = (double*)(D2 + (size_t)batch * n.width);
    dloss = (double*)(((uintptr_t)dloss + 15) & ~(uintptr_t)15);
    if (!e) e = cudaMemsetAsync(dloss, 0, sizeof(double), st);
    if (!e) {
        LaunchTimer lt(ctx, K_MLP_BWD);
        k_mlp_mse<<<grid_for(ctx, batch), 256, 0, st>>>(batch, out, t_dev, D, dloss);
        e = cudaGetLastError();
    }
    for (int l = n.layers() - 1; l >= 0 && !e; --l) {
        const int in = n.in(l), o = n.out(l);
        const float* W = params_dev + n.w_off(l);
        float* gW = grad_dev + n.w_off(l);
        float* gb = gW + (int64_t)o * in;
        // input of layer l: X or H_{l-1}
        const float* Hin = l == 0 ? x_dev : ws + (size_t)(l - 1) * 2 * batch * n.width + (size_t)batch * n.width;
        LaunchTimer lt(ctx, K_MLP_BWD);
        e = gemm(st, o, in, (int)batch, D, 1, o, Hin, in, 1, gW, in, false, false);
        if (!e) {
            k_mlp_colsum<<<(o * 32 + 255) / 256, 256, 0, st>>>(batch, o, D, gb);
            e = cudaGetLastError();
        }
        if (!e && l > 0) {
            const float* Zin = ws + (size_t)(l - 1) * 2 * batch * n.width;
            e = gemm(st, (int)batch, in, o, D, o, 1, W, in, 1, D2, in, false, false);
            if (!e) {
                k_mlp_silu_bwd<<<grid_for(ctx, batch * in), 256, 0, st>>>(batch * in, Zin, D2);
                e = cudaGetLastError();
            }
            std::swap(D, D2);
        }
    }
    double l2 = 0.0;
    if (!e) e = cudaMemcpyAsync(&l2, dloss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return ctx->cuda_fail(e, "MLP backward");
    *loss_out = l2 / (double)batch;
    return SW_OK;
}

extern "C" sw_status sw_mlp_adam(sw_ctx* ctx, int64_t n_params, float* params_dev, const float* grad_dev,
                                 float* m_dev, float* v_dev, int64_t step, double lr, double beta1, double beta2,
                                 double eps)
{
    CHECK_CTX(ctx);
    if (n_params < 1 || step < 1 || !params_dev || !grad_dev || !m_dev || !v_dev || !(lr > 0) ||
        !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) {
        set_error(ctx, "sw_mlp_adam: invalid argument");
        return SW_EINVAL;
    }
    const float c1 = (float)(1.0 - std::pow(beta1, (double)step)), c2 = (float)(1.0 - std::pow(beta2, (double)step));
    {
        LaunchTimer lt(ctx, K_ADAM);
        k_adam<<<grid_for(ctx, n_params), 256, 0, ctx->stream>>>(n_params, params_dev, grad_dev, m_dev, v_dev, (float)lr,
                                                            (float)beta1, (float)beta2, (float)eps, c1, c2);
    }
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    return e ? ctx->cuda_fail(e, "Adam") : SW_OK;
}
