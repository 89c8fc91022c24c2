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
// loads the library keeps it until the process exits.  All calls share it, so
// calls that overlap on the GPU race (serialise them, e.g. on one stream).
#include "sw_linalg.cuh"

#define SW_APPLY_STATIC_MAX (1 << 21)  // doubles: N + M of one call must not exceed this

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
    if (U->N + U->M > (int64_t)SW_APPLY_STATIC_MAX) {
        sw::set_error(ctx, "sw_matrix_apply_static: N + M = %lld exceeds the static scratch of %d values",
                      (long long)(U->N + U->M), SW_APPLY_STATIC_MAX);
        return SW_EINVAL;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(ctx->device, &scratch);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "static scratch address");
    double* d_w = scratch;           // N staged weights
    double* d_y = scratch + U->N;    // M accumulators, zeroed below (the array keeps the last call's contents)
    if ((e = cudaMemcpyAsync(d_w, w, U->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemsetAsync(d_y, 0, U->M * sizeof(double), ctx->stream)) ||
        (e = (U->elem == 8 ? sw::u_times_w<double>(ctx, (const double*)U->d, U->M, U->N, d_w, d_y)
                           : sw::u_times_w<float>(ctx, (const float*)U->d, U->M, U->N, d_w, d_y))) ||
        (e = cudaMemcpyAsync(y_out, d_y, U->M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return ctx->cuda_fail(e, "static matrix apply");
    return SW_OK;
}
