// Read-bandwidth probe (no counterpart in the paper): the measured roof for
// a kernel whose working set stays in L2, such as the factored FP32
// coefficient set of the 192^3 workload (75 MB in the 129 MB L2).  One
// launch streams a device buffer `repeats` times with 16-byte loads that are
// cached in L2 only; after the first pass a buffer that fits in L2 is read
// from it.
#include "sfm_internal.h"

namespace {

__global__ void __launch_bounds__(256) read_probe_kernel(const float4* p, long long n4, int repeats,
                                                         float* sink) {
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < repeats; ++r) {
#pragma unroll 4
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(p + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    }
    if (acc == 1.25e30f) sink[0] = acc;   // never true for a zeroed buffer; keeps the loads
}

}  // namespace

extern "C" int sfm_probe_read_gbs(int device, size_t bytes, int repeats, double* gbs) {
    if (!gbs || bytes < 16 || repeats < 1) {
        sfm::set_global_error("sfm_probe_read_gbs: bad arguments");
        return SFM_ERR_ARG;
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        sfm::set_global_error("sfm_probe_read_gbs: no such device");
        return SFM_ERR_CUDA;
    }
    const long long n4 = (long long)(bytes / 16);
    float4* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&buf, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        const int grid = nsm * 8;
        read_probe_kernel<<<grid, 256>>>(buf, n4, 1, sink);   // warm-up: brings the buffer into L2
        cudaEventRecord(e0);
        read_probe_kernel<<<grid, 256>>>(buf, n4, repeats, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    cudaSetDevice(prev);
    if (e != cudaSuccess || !(ms > 0.f)) {
        sfm::set_global_error(std::string("sfm_probe_read_gbs: ") + cudaGetErrorString(e));
        return SFM_ERR_CUDA;
    }
    *gbs = (double)n4 * 16.0 * repeats / (ms * 1e-3) / 1e9;
    return SFM_OK;
}
