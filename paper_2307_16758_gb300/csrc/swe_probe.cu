// Arithmetic peak of this GPU: fused multiply-adds per second in FP32 or
// FP64, measured by a kernel of independent FMA chains.  It serves as the
// denominator of the arithmetic roofline of the FP64 path (which GB300's
// FP64 units bound) next to the HBM roofline of the FP32 path.  Not part of
// the paper's method.
#include <cuda_runtime.h>

#include <string>

#include "swe_async.cuh"
#include "swe_dev.h"

void swe_set_error(const std::string &msg);
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread (hides the FMA latency)
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;

// x <- x * a + b on kChains values per thread, `iters` times; |a| < 1 keeps
// them bounded.  The sum is stored so that the work cannot be removed.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fma_chains(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[(size_t)blockIdx.x * kBlock + threadIdx.x] = s;
}

template <typename T> int fma_peak(int iters, cudaStream_t s, double *flops_per_s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        swe_set_error("swe_fma_peak: no usable GPU");
        return SWE_ERR_CUDA;
    }
    const int grid = sms * kBlocksPerSm;
    T *out = (T *)dev_alloc(sizeof(T) * (size_t)grid * kBlock, s);
    if (!out) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma_chains<T><<<grid, kBlock, 0, s>>>(out, iters / 8 + 1, T(0.999), T(1e-3));     // warm-up
        e = cudaEventRecord(e0, s);
    }
    if (e == cudaSuccess) {
        k_fma_chains<T><<<grid, kBlock, 0, s>>>(out, iters, T(0.999), T(1e-3));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(out, s);
    if (e != cudaSuccess) {
        swe_set_error(std::string("swe_fma_peak: ") + cudaGetErrorString(e));
        return SWE_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * grid * kBlock;
    *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
    return SWE_OK;
}

// The bounded wait of the tile step's pipeline (mbar_wait) on an mbarrier
// whose phase completes only if `arrive` is set: with arrive = 0 nothing ever
// completes it, the wait must give up after `polls` polls, and the kernel
// reports that and returns like the tile step does.  Every thread of the
// block waits, as in the pipeline.
__global__ void k_wait_probe(uint32_t polls, int arrive, int *timed_out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        swe_dev::mbar_init(&bar);
        swe_dev::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && arrive) swe_dev::mbar_arrive(&bar);
    const bool ok = __syncthreads_and(swe_dev::mbar_wait(&bar, 0, polls));
    if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

}  // namespace

extern "C" int swe_probe_bounded_wait(uint32_t polls, int arrive, int *timed_out, void *stream)
{
    if (!timed_out || polls == 0 || polls > (1u << 22)) {
        swe_set_error("swe_probe_bounded_wait: bad argument");
        return SWE_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int *d = (int *)dev_alloc(sizeof(int), s);
    if (!d) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
    int h = -1;
    cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int), s);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 128, 0, s>>>(polls, arrive ? 1 : 0, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d, s);
    if (e != cudaSuccess) {
        swe_set_error(std::string("swe_probe_bounded_wait: ") + cudaGetErrorString(e));
        return SWE_ERR_CUDA;
    }
    *timed_out = h;
    return SWE_OK;
}

extern "C" int swe_fma_peak(int precision, int iters, void *stream, double *flops_per_s)
{
    if (!flops_per_s || iters < 1 || iters > (1 << 20) || (precision != SWE_FP32 && precision != SWE_FP64)) {
        swe_set_error("swe_fma_peak: bad argument");
        return SWE_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SWE_FP32 ? fma_peak<float>(iters, s, flops_per_s) : fma_peak<double>(iters, s, flops_per_s);
}
