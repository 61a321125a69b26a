// kernels_probe.cu -- throughput probes that measure the roofline denominators
// of this GPU in the same process as the benchmark: the FP32 and FP64 FMA
// rates of the CUDA cores (the pipes the gravity sum and the aggregate update
// use; nothing on the path is a dense contraction, so no tensor cores) and
// the HBM copy bandwidth (the contact pass's bound).
//
// FMA probes: every thread runs kChains independent chains a = a * b + c for
// `iters` rounds (2 flop per FMA, 4 per packed f32x2 FMA), so that each
// scheduler always has an independent FMA to issue; the grid is a whole
// number of waves (kProbeBlocksPerSM blocks of kProbeBlock threads per SM).
// The chains' sum is written only when it equals a value it cannot take, so
// the work is not removed and the sink is never written in practice.
// Copy probe: float4 grid-stride copy of `bytes` from src to dst; the rate is
// counted as bytes read plus bytes written.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "dem.h"

namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeBlocksPerSM = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeBlock) k_probe_fma32(int64_t iters, float b, float c, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345e-30f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeBlock) k_probe_fma32x2(int64_t iters, float b, float c, float *sink)
{
    unsigned long long a[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c), "f"(c));
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float lo = (float)(threadIdx.x + k), hi = (float)(threadIdx.x + 2 * k + 1);
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(lo), "f"(hi));
    }
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
        s += lo + hi;
    }
    if (s == -1.2345e-30f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeBlock) k_probe_fma64(int64_t iters, double b, double c, double *sink)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345e-300) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeBlock) k_probe_copy(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                                            int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * kProbeBlock;
    for (int64_t i = (int64_t)blockIdx.x * kProbeBlock + threadIdx.x; i < n; i += stride)
        __stcs(dst + i, __ldcs(src + i));
}

dem_status probe_fail(char *msg, size_t len, dem_status s, const char *what, cudaError_t e)
{
    if (msg && len) snprintf(msg, len, "%s: %s", what, e == cudaSuccess ? "invalid argument" : cudaGetErrorString(e));
    return s;
}

}  // namespace

extern "C" dem_status dem_probe_peak(int32_t kind, int64_t size, int32_t reps, const void *src, void *dst,
                                     void *cuda_stream, double *rate_out, double *ms_out, int32_t *sm_count_out,
                                     char *msg, size_t msg_len)
{
    if (msg && msg_len) msg[0] = 0;
    if (!rate_out || reps < 1 || size < 1 || !dst || kind < DEM_PROBE_FMA32 || kind > DEM_PROBE_COPY)
        return probe_fail(msg, msg_len, DEM_ERR_ARG, "dem_probe_peak", cudaSuccess);
    if (kind == DEM_PROBE_COPY &&
        (!src || (size & 15) || (((uintptr_t)src) & 15) || (((uintptr_t)dst) & 15)))
        return probe_fail(msg, msg_len, DEM_ERR_ARG, "dem_probe_peak (copy: 16-byte sizes and alignment)",
                          cudaSuccess);
    if (kind != DEM_PROBE_COPY && (((uintptr_t)dst) & 7))
        return probe_fail(msg, msg_len, DEM_ERR_ARG, "dem_probe_peak (sink not 8-byte aligned)", cudaSuccess);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return probe_fail(msg, msg_len, DEM_ERR_CUDA, "device query", e);
    if (sm_count_out) *sm_count_out = sms;
    const unsigned grid = (unsigned)(sms * kProbeBlocksPerSM);
    const double threads = (double)grid * kProbeBlock;
    cudaEvent_t ev[2];
    e = cudaEventCreate(&ev[0]);
    if (e != cudaSuccess) return probe_fail(msg, msg_len, DEM_ERR_CUDA, "cudaEventCreate", e);
    e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return probe_fail(msg, msg_len, DEM_ERR_CUDA, "cudaEventCreate", e);
    }
    double work = 0.0, best_ms = 0.0;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(ev[0], st);
        if (e != cudaSuccess) break;
        switch (kind) {
        case DEM_PROBE_FMA32:
            k_probe_fma32<<<grid, kProbeBlock, 0, st>>>(size, 0.999999f, 1e-7f, (float *)dst);
            work = threads * (double)size * 4.0 * kChains * 2.0;
            break;
        case DEM_PROBE_FMA32X2:
            k_probe_fma32x2<<<grid, kProbeBlock, 0, st>>>(size, 0.999999f, 1e-7f, (float *)dst);
            work = threads * (double)size * 4.0 * kChains * 4.0;
            break;
        case DEM_PROBE_FMA64:
            k_probe_fma64<<<grid, kProbeBlock, 0, st>>>(size, 0.9999999999, 1e-15, (double *)dst);
            work = threads * (double)size * 4.0 * kChains * 2.0;
            break;
        default: {
            const int64_t n = size / 16;
            k_probe_copy<<<grid * 2, kProbeBlock, 0, st>>>((const float4 *)src, (float4 *)dst, n);
            work = 2.0 * (double)size;
        }
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess && (r == 0 || ms < best_ms)) best_ms = ms;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return probe_fail(msg, msg_len, DEM_ERR_CUDA, "probe launch", e);
    *rate_out = best_ms > 0.0 ? work / (best_ms * 1e-3) : 0.0;
    if (ms_out) *ms_out = best_ms;
    return DEM_OK;
}
