// sw_matrix_apply_static: y = U w without any device allocation.
//
// Some callers cannot allocate device memory when they call into the library:
// a host process whose device memory is handed out by another allocator (a
// framework's caching pool sized at start-up), or a pipeline that must not
// allocate once it is running.  For them this entry point computes the same
// product as sw_matrix_apply, but keeps its scratch -- the staged weight
// vector and the zero-initialised FP64 accumulator of U w -- in a file-scope
// device array of fixed size instead of cudaMalloc'ed buffers.
//
// The array holds SW_APPLY_STATIC_MAX doubles (16 MiB); every device that
// loads the library keeps it until the process exits.  One call uses N
// doubles for w, M for the accumulator and, for an FP32 matrix, N more
// (2 N floats) for the float hi + lo halves of w that the FP32 product reads.
// All calls share it, so calls that overlap on the GPU race (serialise them,
// e.g. on one stream).
#include "sw_linalg.cuh"

#define SW_APPLY_STATIC_MAX (1 << 21)  // doubles: N + M (2 N + M for FP32 matrices) of one call

namespace {

__device__ __align__(256) double g_apply_scratch[SW_APPLY_STATIC_MAX];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(int device, double** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" sw_status sw_matrix_apply_static(const sw_matrix* U, const double* w, double* y_out)
{
    if (!U || !w || !y_out || U->ctx->destroyed) return SW_EINVAL;
    sw_ctx* ctx = U->ctx;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    const int64_t need = (U->elem == 8 ? 1 : 2) * U->N + U->M;
    if (need > (int64_t)SW_APPLY_STATIC_MAX) {
        sw::set_error(ctx,
                      "sw_matrix_apply_static: the call needs %lld values of scratch (N + M, 2 N + M for an FP32 "
                      "matrix), more than the static array's %d",
                      (long long)need, SW_APPLY_STATIC_MAX);
        return SW_EINVAL;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(ctx->device, &scratch);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "static scratch address");
    double* d_w = scratch;           // N staged weights
    double* d_y = scratch + U->N;    // M accumulators, zeroed below (the array keeps the last call's contents)
    float* d_wh = reinterpret_cast<float*>(d_y + U->M);   // FP32 matrices: float hi + lo halves of w
    float* d_wl = d_wh + U->N;
    if ((e = cudaMemcpyAsync(d_w, w, U->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemsetAsync(d_y, 0, U->M * sizeof(double), ctx->stream)) ||
        (e = (U->elem == 8 ? sw::u_times_w<double>(ctx, (const double*)U->d, U->M, U->N, d_w, d_y)
                           : sw::u_times_w_presplit(ctx, (const float*)U->d, U->M, U->N, d_w, d_wh, d_wl, d_y))) ||
        (e = cudaMemcpyAsync(y_out, d_y, U->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return ctx->cuda_fail(e, "static matrix apply");
    return SW_OK;
}
