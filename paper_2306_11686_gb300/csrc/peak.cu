/*
 * gf_fp64_add_rate: the FP64 add throughput of this GPU, measured.
 *
 * The Jacobi sweep's arithmetic is bound by the FP64 pipe (GB300 retires
 * FP64 adds at a small fraction of its FP32 and integer rates), so its
 * roofline needs this pipe's peak.  Every thread runs eight independent
 * chains of correctly rounded FP64 adds (add.rn.f64), enough independent
 * work to keep the pipe busy at any latency; the kernel is timed with CUDA
 * events on the caller's stream.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "gf.h"

#define GF_PEAK_CHAINS 8

__device__ double gf_peak_sink;

__global__ void __launch_bounds__(256) fp64_add_chains(double inc, int64_t iters)
{
    double x[GF_PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < GF_PEAK_CHAINS; k++)
        x[k] = (double)threadIdx.x * 1e-3 + (double)k;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < GF_PEAK_CHAINS; k++)
            x[k] = __dadd_rn(x[k], inc);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < GF_PEAK_CHAINS; k++)
        s = __dadd_rn(s, x[k]);
    if (s == -1.0)          /* never true for these inputs; keeps the chains live */
        gf_peak_sink = s;
}

extern "C" GF_API int gf_fp64_add_rate(uint32_t blocks, int64_t iters, void *stream, float *ms, double *adds)
{
    if (!ms || !adds || iters < 1)
        return GF_EINVAL;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp64_add_chains, 256, 0) != cudaSuccess)
        return GF_ECUDA;
    const uint32_t grid = blocks ? blocks : (uint32_t)(sms * (occ > 0 ? occ : 1));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GF_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = GF_ECUDA;
    } else {
        const double inc = 1.0 / 1024.0;
        void *args[2] = {(void *)&inc, (void *)&iters};
        if (cudaLaunchKernel((const void *)fp64_add_chains, dim3(grid), dim3(256), args, 0, s) != cudaSuccess ||
            cudaEventRecord(e0, s) != cudaSuccess ||
            cudaLaunchKernel((const void *)fp64_add_chains, dim3(grid), dim3(256), args, 0, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            rc = GF_ECUDA;
        *adds = (double)grid * 256.0 * (double)iters * GF_PEAK_CHAINS;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    return rc;
}
