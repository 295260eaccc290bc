// probe.cu -- measured throughput of the SMs' L1 and L2 data paths for 16-byte loads and of their
// FP32 fused multiply-add pipes (not in the paper).
//
// With positions in cell order, neighbouring positions share most of the 64 stencil rows of
// Eq. (b-splineapproximation): the evaluation kernels find those rows in the SM's L1 cache or,
// failing that, in L2, and read HBM little more than once per row.  The rates that bound them
// are then how fast L1 and L2 return 16-byte loads.  This probe measures both with the load
// shape the evaluation kernels issue (16 bytes per lane, each warp instruction 512 contiguous
// bytes = four 128-byte lines): every SM runs two 1024-thread blocks, eight independent loads
// per thread in flight.
//   level 1: ld.global.nc over a 64 KB buffer that stays resident in every SM's L1;
//   level 2: ld.global.cg (cached in L2 only) over a 32 MB buffer that stays resident in L2,
//            each block sweeping its own 128 KB window per iteration so that all L2 slices of
//            both dies serve the SMs.
#include "qmcspl_internal.cuh"
#include "eval_common.cuh"

namespace qmcspl {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeBlocksPerSm = 2;
constexpr int kProbeUnroll = 8;          // independent loads per thread per iteration
constexpr int kProbeRuns = 5;
constexpr int kL1Vec = 4096;             // 16-byte vectors in the L1 working set: 64 KB
constexpr int kL1Iters = 4096;
constexpr int kL2Vec = 1 << 21;          // 16-byte vectors in the L2 working set: 32 MB
constexpr int kL2Iters = 512;

template <int LEVEL>
__device__ __forceinline__ uint4 probe_load(const uint4* p)
{
    uint4 v;
    if (LEVEL == 1)
        asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p));
    else
        asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p));
    return v;
}

// Iteration k of thread i reads, for u = 0 .. kProbeUnroll-1, vector
//   level 1: (i + 32 k + 1024 u)                      mod kL1Vec
//   level 2: (8192 (block + k) + i + 1024 u)          mod kL2Vec
// (the moduli are powers of two: every access stays in the buffer).  A warp's 32 lanes read
// 32 consecutive vectors, i.e. 512 contiguous bytes.
template <int LEVEL>
__global__ void __launch_bounds__(kProbeThreads) cache_probe_kernel(const uint4* __restrict__ buf,
                                                                     long long* cycles, uint4* sink)
{
    constexpr int mask = (LEVEL == 1 ? kL1Vec : kL2Vec) - 1;
    constexpr int iters = LEVEL == 1 ? kL1Iters : kL2Iters;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const long long t0 = clock64();
    for (int k = 0; k < iters; ++k) {
        const int base = LEVEL == 1 ? (int)threadIdx.x + 32 * k
                                    : kProbeThreads * kProbeUnroll * ((int)blockIdx.x + k) + (int)threadIdx.x;
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            const uint4 v = probe_load<LEVEL>(buf + ((base + u * kProbeThreads) & mask));
            acc.x ^= v.x;
            acc.y ^= v.y;
            acc.z ^= v.z;
            acc.w ^= v.w;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    // keeps the loads live; the buffer holds zeros, so this never holds
    if ((acc.x & acc.y & acc.z & acc.w) == 0xffffffffu) sink[blockIdx.x] = acc;
}

// FP32 multiply-add throughput: every thread runs kFmaChains independent chains of
// fma.rn.f32 (PACKED = false) or fma.rn.f32x2 (PACKED = true: two lanes of FP32 per
// instruction), kFmaIters steps each.  m and a come from the host so that nothing folds.
constexpr int kFmaChains = 8;
constexpr int kFmaIters = 4096;

template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float m, float a, long long* cycles, float* sink)
{
    __syncthreads();
    const long long t0 = clock64();
    float out = 0.f;
    if (PACKED) {
        f32x2 acc[kFmaChains];
        const f32x2 m2 = pack2(m, m), a2 = pack2(a, a);
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) acc[i] = pack2((float)(threadIdx.x + i), (float)i);
        for (int k = 0; k < kFmaIters; ++k) {
#pragma unroll
            for (int i = 0; i < kFmaChains; ++i) acc[i] = ffma2(acc[i], m2, a2);
        }
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) {
            float lo, hi;
            unpack2(acc[i], lo, hi);
            out += lo + hi;
        }
    } else {
        float acc[kFmaChains];
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) acc[i] = (float)(threadIdx.x + i);
        for (int k = 0; k < kFmaIters; ++k) {
#pragma unroll
            for (int i = 0; i < kFmaChains; ++i) asm("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[i]) : "f"(m), "f"(a));
        }
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) out += acc[i];
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    if (out == -1.0f) sink[blockIdx.x] = out;   // keeps the chains live; m = 1, a = 0 never gives -1
}

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_probe_fma(int packed, double* tflops, double* flops_per_clk, double* sm_mhz, void* stream)
{
    clear_error();
    if (packed != 0 && packed != 1) return set_error(QMCSPL_ERR_ARG, "qmcspl_probe_fma: packed must be 0 or 1");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    const int blocks = kProbeBlocksPerSm * sms;
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double best_ms = 0.0;
    long long best_cycles = 0;
    const int nc = blocks < 1024 ? blocks : 1024;
    long long c[1024];
    cudaError_t e = dev_malloc((void**)&sink, sizeof(float) * (size_t)blocks);
    if (e == cudaSuccess) e = dev_malloc((void**)&cyc, sizeof(long long) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    for (int run = 0; run <= kProbeRuns && e == cudaSuccess; ++run) {   // run 0 warms up
        e = cudaEventRecord(ev[0], st);
        if (e != cudaSuccess) break;
        if (packed) fma_probe_kernel<true><<<blocks, kProbeThreads, 0, st>>>(1.0f, 0.0f, cyc, sink);
        else fma_probe_kernel<false><<<blocks, kProbeThreads, 0, st>>>(1.0f, 0.0f, cyc, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaMemcpy(c, cyc, sizeof(long long) * (size_t)nc, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess || run == 0) continue;
        long long cmax = 0;
        for (int i = 0; i < nc; ++i) cmax = c[i] > cmax ? c[i] : cmax;
        if (best_ms == 0.0 || ms < best_ms) {
            best_ms = ms;
            best_cycles = cmax;
        }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (e != cudaSuccess) return cuda_error(e, "qmcspl_probe_fma");
    const double flops = (double)blocks * kProbeThreads * kFmaIters * kFmaChains * 2.0 * (packed ? 2.0 : 1.0);
    const double mhz = best_ms > 0.0 ? (double)best_cycles / (best_ms * 1e3) : 0.0;
    const double rate = best_ms > 0.0 ? flops / (best_ms * 1e-3) / 1e12 : 0.0;
    if (tflops) *tflops = rate;
    if (sm_mhz) *sm_mhz = mhz;
    if (flops_per_clk) *flops_per_clk = mhz > 0.0 ? rate * 1e12 / ((double)sms * mhz * 1e6) : 0.0;
    return QMCSPL_OK;
}

extern "C" int qmcspl_probe_cache(int level, double* gbs, double* bytes_per_clk, double* sm_mhz, void* stream)
{
    clear_error();
    if (level != 1 && level != 2) return set_error(QMCSPL_ERR_ARG, "qmcspl_probe_cache: level must be 1 or 2");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    const int blocks = kProbeBlocksPerSm * sms;
    const size_t nvec = level == 1 ? kL1Vec : kL2Vec;
    const int iters = level == 1 ? kL1Iters : kL2Iters;
    uint4* buf = nullptr;
    uint4* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double best_ms = 0.0;
    long long best_cycles = 0;
    const int nc = blocks < 1024 ? blocks : 1024;
    long long c[1024];
    cudaError_t e = dev_malloc((void**)&buf, sizeof(uint4) * nvec);
    if (e == cudaSuccess) e = dev_malloc((void**)&sink, sizeof(uint4) * (size_t)blocks);
    if (e == cudaSuccess) e = dev_malloc((void**)&cyc, sizeof(long long) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(uint4) * nvec, st);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    for (int run = 0; run <= kProbeRuns && e == cudaSuccess; ++run) {   // run 0 warms up
        e = cudaEventRecord(ev[0], st);
        if (e != cudaSuccess) break;
        if (level == 1) cache_probe_kernel<1><<<blocks, kProbeThreads, 0, st>>>(buf, cyc, sink);
        else cache_probe_kernel<2><<<blocks, kProbeThreads, 0, st>>>(buf, cyc, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaMemcpy(c, cyc, sizeof(long long) * (size_t)nc, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess || run == 0) continue;
        long long cmax = 0;
        for (int i = 0; i < nc; ++i) cmax = c[i] > cmax ? c[i] : cmax;
        if (best_ms == 0.0 || ms < best_ms) {
            best_ms = ms;
            best_cycles = cmax;
        }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (e != cudaSuccess) return cuda_error(e, "qmcspl_probe_cache");
    const double bytes = (double)blocks * kProbeThreads * iters * kProbeUnroll * 16.0;
    const double mhz = best_ms > 0.0 ? (double)best_cycles / (best_ms * 1e3) : 0.0;
    const double rate = best_ms > 0.0 ? bytes / (best_ms * 1e-3) / 1e9 : 0.0;
    if (gbs) *gbs = rate;
    if (sm_mhz) *sm_mhz = mhz;
    if (bytes_per_clk) *bytes_per_clk = mhz > 0.0 ? rate * 1e9 / ((double)sms * mhz * 1e6) : 0.0;
    return QMCSPL_OK;
}
