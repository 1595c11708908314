// Arithmetic-throughput probe of the GPU the library runs on: the measured
// denominators of the ALU rooflines (the FP64 dslash is bound by the FP64
// pipe on GB300, the double-float dslash by the FP32 pipe).
//
// Every thread runs NCHAIN independent fused multiply-add chains
// a <- a * b + c for ITERS iterations (no memory traffic inside the loop),
// so the kernel issues nothing but FMAs once the loop is unrolled; the
// chains are summed into one store per thread so the compiler keeps them.
// The grid is a whole number of waves: 8 blocks of 256 threads per SM.
#include "ctx.h"

namespace ov {

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAIN = 8;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) fma_peak_kernel(T b, T c, int iters, T* out)
{
    T a[PK_CHAIN];
#pragma unroll
    for (int j = 0; j < PK_CHAIN; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < PK_CHAIN; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PK_CHAIN; ++j) s += a[j];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

}  // namespace

}  // namespace ov

using namespace ov;

extern "C" int ov_measure_fma_peak(int prec, double* gflops, void* stream)
{
    if (!gflops || (prec != P_F64 && prec != P_F32)) return OV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return OV_ECUDA;
    const int blocks = sms * 8;
    const size_t n = (size_t)blocks * PK_THREADS;
    // FP64 is a small fraction of the FP32 rate on GB300: fewer iterations keep both near 20 ms
    const int iters = prec == P_F64 ? 64 : 2048;
    void* out = nullptr;
    if (cudaMalloc(&out, n * 8) != cudaSuccess) {
        cudaGetLastError();
        return OV_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = OV_OK;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) status = OV_ECUDA;
    for (int rep = 0; rep < 6 && status == OV_OK; ++rep) {  // the first launch warms up, best of the rest
        cudaEventRecord(e0, st);
        if (prec == P_F64)
            fma_peak_kernel<double><<<blocks, PK_THREADS, 0, st>>>(1.0000001, 1e-7, iters, (double*)out);
        else
            fma_peak_kernel<float><<<blocks, PK_THREADS, 0, st>>>(1.0000001f, 1e-7f, iters, (float*)out);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            status = OV_ECUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (status != OV_OK) return status;
    const double flops = 2.0 * (double)n * iters * 16 * PK_CHAIN;
    *gflops = flops / (best * 1e-3) / 1e9;
    return OV_OK;
}
