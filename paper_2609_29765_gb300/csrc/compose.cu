// compose.cu -- entry points composed from the others (host code only).
//  * stc_factorize_mixed: several patterns, each with its own batch of value sets,
//    factorized by one persistent launch in a single call: a group is created, run and
//    destroyed around the caller's buffers (the batching of Sec. 1 and 2 over uneven
//    patterns); the kernel is the replay kernel behind stc_factorize_group.
//  * stc_quad_backward: the gradient of the quadratic form x^T A x, the symmetric outer
//    product of x with itself.
#include <cuda_runtime.h>

#include "stc.h"

extern "C" int stc_factorize_mixed(int32_t nplans, const stc_plan* const* plans, const double* const* d_values,
                                   const int64_t* batch, void* const* d_factor, int32_t* const* d_info,
                                   void* stream) {
    if (!plans || !d_values || !batch || !d_factor || !d_info) return STC_ERR_INVALID_ARG;
    stc_group* g = nullptr;
    int rc = stc_group_create(nplans, plans, batch, &g);
    if (rc != STC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, stc_group_workspace_bytes(g), st) != cudaSuccess) {
        stc_group_destroy(g);
        return STC_ERR_OUT_OF_MEMORY;
    }
    rc = stc_factorize_group(g, d_values, d_factor, d_info, ws, stream);
    // waits for the launch and reads its status word (STC_OK or STC_ERR_TIMEOUT)
    const int status = rc != STC_OK ? rc : stc_sync_status(ws, stream);
    const bool freed = cudaFreeAsync(ws, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    stc_group_destroy(g);
    return status != STC_OK ? status : (freed ? STC_OK : STC_ERR_CUDA);
}

extern "C" int stc_quad_backward(const stc_plan* plan, int64_t batch, const double* d_x, const double* d_gout,
                                 double* d_gvalues, int accumulate, void* stream) {
    return stc_sym_outer_backward(plan, batch, d_x, d_x, d_gout, d_gvalues, accumulate, stream);
}
