// Element-wise entry point for the integer-pipe conversions of fp_convert.cuh,
// so that each can be checked against the hardware conversion on crafted bit
// patterns.  The kernels of the solve inline these functions; nothing on the
// solve path calls this entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp_convert.cuh"
#include "omm_internal.cuh"

namespace {

__global__ void convert_kernel(int op, int64_t n, const void *__restrict__ in, const int32_t *__restrict__ e,
                               void *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        switch (op) {
            case 0: ((float *)out)[i] = omm::sw_d2f(((const double *)in)[i]); break;
            case 1: ((double *)out)[i] = omm::sw_f2d(((const float *)in)[i]); break;
            case 2: ((double *)out)[i] = omm::sw_i64_scaled(((const int64_t *)in)[i], e[i]); break;
            default: ((double *)out)[i] = omm::sw_scale2(((const double *)in)[i], e[i]); break;
        }
    }
}

}  // namespace

extern "C" int omm_op_convert(int32_t op, int64_t n, const void *in, const int32_t *e, void *out, void *stream) {
    if (op < 0 || op > 3 || n < 0) {
        omm::set_error("omm_op_convert: op = %d (0..3), n = %lld (>= 0)", (int)op, (long long)n);
        return OMM_ERR_ARG;
    }
    if (n == 0) return OMM_OK;
    if (in == nullptr || out == nullptr || (op >= 2 && e == nullptr)) {
        omm::set_error("omm_op_convert: NULL array");
        return OMM_ERR_ARG;
    }
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    convert_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(op, n, in, e, out);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}
