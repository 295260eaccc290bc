// probe.cu -- measured throughput of the SMs' L1 data path for 16-byte loads (not in the
// paper).
//
// With positions in cell order, neighbouring positions share most of the 64 stencil rows of
// Eq. (b-splineapproximation), and the evaluation kernels find those rows in the SM's L1
// cache; the rate that bounds them is then how fast the SMs return 16-byte loads from L1,
// not the HBM rate.  This probe measures that rate with the load the evaluation kernels
// issue (ld.global.nc of 16 bytes per lane, each warp instruction 512 contiguous bytes =
// four 128-byte wavefronts): every SM runs two 1024-thread blocks that sweep a 64 KB
// buffer (L1-resident after the first pass), eight independent loads per thread in flight.
#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeBlocksPerSm = 2;
constexpr int kProbeVec = 4096;          // 16-byte vectors in the working set: 64 KB
constexpr int kProbeUnroll = 8;          // independent loads per thread per iteration
constexpr int kProbeIters = 4096;
constexpr int kProbeRuns = 5;

__device__ __forceinline__ uint4 ld_nc16(const uint4* p)
{
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Each iteration reads kProbeUnroll vectors per thread, 1024 vectors apart, then moves the
// window by 32 vectors (512 bytes) so that successive iterations read different addresses.
// Indices are taken modulo kProbeVec (a power of two): every access stays in the buffer.
__global__ void __launch_bounds__(kProbeThreads) l1_probe_kernel(const uint4* __restrict__ buf,
                                                                  long long* cycles, uint4* sink)
{
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    int base = threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int k = 0; k < kProbeIters; ++k) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            const uint4 v = ld_nc16(buf + ((base + u * kProbeThreads) & (kProbeVec - 1)));
            acc.x ^= v.x;
            acc.y ^= v.y;
            acc.z ^= v.z;
            acc.w ^= v.w;
        }
        base = (base + 32) & (kProbeVec - 1);
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    // keeps the loads live; the buffer is filled so that this never holds
    if ((acc.x & acc.y & acc.z & acc.w) == 0xffffffffu) sink[blockIdx.x] = acc;
}

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_probe_l1(double* gbs, double* bytes_per_clk, double* sm_mhz, void* stream)
{
    clear_error();
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    const int blocks = kProbeBlocksPerSm * sms;
    uint4* buf = nullptr;
    uint4* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double best_ms = 0.0;
    long long best_cycles = 0;
    cudaError_t e = dev_malloc((void**)&buf, sizeof(uint4) * kProbeVec);
    if (e == cudaSuccess) e = dev_malloc((void**)&sink, sizeof(uint4) * (size_t)blocks);
    if (e == cudaSuccess) e = dev_malloc((void**)&cyc, sizeof(long long) * (size_t)blocks);
    // 0x00 bytes: the XOR of the loaded words stays 0, so the sink is never written
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(uint4) * kProbeVec, st);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    for (int run = 0; run <= kProbeRuns && e == cudaSuccess; ++run) {   // run 0 warms up
        e = cudaEventRecord(ev[0], st);
        if (e != cudaSuccess) break;
        l1_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(buf, cyc, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        long long c[1024];
        const int nc = blocks < 1024 ? blocks : 1024;
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
    if (e != cudaSuccess) return cuda_error(e, "qmcspl_probe_l1");
    const double bytes = (double)blocks * kProbeThreads * kProbeIters * kProbeUnroll * 16.0;
    const double mhz = best_ms > 0.0 ? (double)best_cycles / (best_ms * 1e3) : 0.0;
    const double rate = best_ms > 0.0 ? bytes / (best_ms * 1e-3) / 1e9 : 0.0;
    if (gbs) *gbs = rate;
    if (sm_mhz) *sm_mhz = mhz;
    if (bytes_per_clk) *bytes_per_clk = mhz > 0.0 ? rate * 1e9 / ((double)sms * mhz * 1e6) : 0.0;
    return QMCSPL_OK;
}
