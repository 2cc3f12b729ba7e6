// md_probe.cu -- measurement and test hooks of the library: the device's own
// ceilings for the force pass's roofline (FP32 and FP64 fused multiply-add
// throughput, random 16-byte gathers from an L2-resident array, a streaming
// copy through HBM), and the library's FP64 reciprocal / reciprocal square
// root evaluated on an array so that tests can hold them to an error bound.
// None of this is on the MD path; the paper has no counterpart.
#include <cuda_runtime.h>

#include <algorithm>

#include "md_common.cuh"
#include "md_kernels.h"

namespace md {
namespace {

// ---------------------------------------------------------- FMA ceilings --
// Each thread runs kChains independent multiply-add chains of kIters steps:
// enough independent work per warp to keep the pipe busy.  The chains'
// values are written only if they come out as an impossible sentinel, so
// the compiler must compute them but the store never happens.
constexpr int kChains = 8;
constexpr int kIters = 4096;

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, T *sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-12345.678) sink[threadIdx.x] = s;
}

// ------------------------------------------------------- gather ceiling --
// A streamed list of record indices (read once from HBM, 16-byte vector
// loads, evict-first) drives 16-byte gathers from a record array small enough
// to stay in L2: the access shape of the force pass's neighbour loop with no
// locality between the lanes of a warp.
__global__ void k_fill_indices(uint32_t *idx, long long m, uint32_t mask) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        // a 32-bit integer mix (multiply-xorshift) of the position
        uint32_t h = (uint32_t)i * 0x9E3779B9u;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        h *= 0xC2B2AE35u;
        h ^= h >> 16;
        idx[i] = h & mask;
    }
}

__global__ void k_fill_records(float4 *rec, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rec[i] = make_float4(0.25f * (i & 7), 0.5f * (i & 3), 0.125f * (i & 15), 1.0f);
}

__global__ void __launch_bounds__(256) k_gather_peak(const uint4 *idx4, long long m4, const float4 *rec,
                                                     float *sink) {
    float acc = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m4;
         k += (long long)gridDim.x * blockDim.x) {
        uint4 e;
        asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(e.x), "=r"(e.y), "=r"(e.z), "=r"(e.w)
                     : "l"(idx4 + k));
        const float4 r0 = __ldg(&rec[e.x]), r1 = __ldg(&rec[e.y]), r2 = __ldg(&rec[e.z]), r3 = __ldg(&rec[e.w]);
        acc += (r0.x + r0.y + r0.z) + (r1.x + r1.y + r1.z) + (r2.x + r2.y + r2.z) + (r3.x + r3.y + r3.z);
    }
    if (acc == -12345.678f) sink[threadIdx.x] = acc;
}

// ---------------------------------------------------------- HBM ceiling --
__global__ void __launch_bounds__(256) k_copy_peak(const float4 *a, float4 *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// ------------------------------------------------------------- FP64 math --
__global__ void k_fp64_math(int op, long long n, const double *x, double *y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = op == 0 ? rcp_newton(x[i]) : rsqrt_newton(x[i]);
}

// time `reps` runs of `launch` (after one untimed run) with CUDA events on s
template <class F>
cudaError_t time_ms(cudaStream_t s, int reps, F launch, float *ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    launch();
    e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) *ms /= (float)reps;
    return e;
}

}  // namespace
}  // namespace md

using namespace md;

extern "C" md_status md_probe_ceilings(void *stream, md_ceilings *out) {
    if (!out) {
        set_last_error("md_probe_ceilings: null argument");
        return MD_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("md_probe_ceilings: no CUDA device");
        return MD_ERR_CUDA;
    }
    const long long m = 64ll << 20;        // gathered indices (256 MB streamed)
    const int nrec = 1 << 20;              // 16 MB of records: L2-resident
    const long long ncopy = 32ll << 20;    // 512 MB copied per pass
    uint32_t *idx = nullptr;
    float4 *rec = nullptr, *ca = nullptr, *cb = nullptr;
    float *sinkf = nullptr;
    double *sinkd = nullptr;
    cudaError_t e = cudaMalloc(&idx, m * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&rec, nrec * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&ca, ncopy * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&cb, ncopy * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&sinkf, 256 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&sinkd, 256 * sizeof(double));
    auto cleanup = [&]() {
        cudaFree(idx); cudaFree(rec); cudaFree(ca); cudaFree(cb); cudaFree(sinkf); cudaFree(sinkd);
    };
    if (e != cudaSuccess) {
        cleanup();
        set_last_error("md_probe_ceilings: device allocation failed");
        return MD_ERR_OOM;
    }
    const dim3 grid((unsigned)(n_sm * 8)), blk(256);
    k_fill_indices<<<grid, blk, 0, s>>>(idx, m, (uint32_t)(nrec - 1));
    k_fill_records<<<(nrec + 255) / 256, 256, 0, s>>>(rec, nrec);
    e = cudaMemsetAsync(ca, 0, ncopy * sizeof(float4), s);
    float ms32 = 0.f, ms64 = 0.f, msg = 0.f, msc = 0.f;
    if (e == cudaSuccess)
        e = time_ms(s, 5, [&]() { k_fma_peak<float><<<grid, blk, 0, s>>>(1.0000001f, 1e-7f, sinkf); }, &ms32);
    const dim3 grid64((unsigned)n_sm), blk64(256);  // FP64 is slow on this GPU: a smaller grid suffices
    if (e == cudaSuccess)
        e = time_ms(s, 3, [&]() { k_fma_peak<double><<<grid64, blk64, 0, s>>>(1.0000000001, 1e-10, sinkd); }, &ms64);
    if (e == cudaSuccess)
        e = time_ms(s, 10, [&]() { k_gather_peak<<<grid, blk, 0, s>>>((const uint4 *)idx, m / 4, rec, sinkf); }, &msg);
    if (e == cudaSuccess)
        e = time_ms(s, 10, [&]() { k_copy_peak<<<grid, blk, 0, s>>>(ca, cb, ncopy); }, &msc);
    cleanup();
    if (e != cudaSuccess) {
        set_last_error("md_probe_ceilings: a probe kernel failed");
        return MD_ERR_CUDA;
    }
    const double thr32 = (double)grid.x * blk.x, thr64 = (double)grid64.x * blk64.x;
    out->fp32_fma_tflops = 2.0 * kChains * kIters * thr32 / (ms32 * 1e-3) / 1e12;
    out->fp64_fma_tflops = 2.0 * kChains * kIters * thr64 / (ms64 * 1e-3) / 1e12;
    out->l2_gather_gps = (double)m / (msg * 1e-3) / 1e9;
    out->l2_gather_gbs = 16.0 * (double)m / (msg * 1e-3) / 1e9;
    out->index_stream_gbs = 4.0 * (double)m / (msg * 1e-3) / 1e9;
    out->hbm_copy_gbs = 2.0 * 16.0 * (double)ncopy / (msc * 1e-3) / 1e9;
    return MD_OK;
}

extern "C" md_status md_probe_fp64_math(int32_t op, int64_t n, const double *x, double *y, void *stream) {
    if ((op != 0 && op != 1) || n < 0 || (n > 0 && (!x || !y))) {
        set_last_error("md_probe_fp64_math: bad argument");
        return MD_ERR_INVALID;
    }
    if (n == 0) return MD_OK;
    long long nn = n;
    void *args[] = {&op, &nn, (void *)&x, &y};
    const dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 4096));
    // the launch's own status, so that an error left pending elsewhere is not reported as ours
    if (cudaLaunchKernel((const void *)k_fp64_math, grid, dim3(256), args, 0, (cudaStream_t)stream) != cudaSuccess) {
        set_last_error("md_probe_fp64_math: kernel launch failed");
        return MD_ERR_CUDA;
    }
    return MD_OK;
}
