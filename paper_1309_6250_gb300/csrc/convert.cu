// convert.cu -- 16-bit copies of float outputs for the host-buffer evaluation (not in the paper).
//
// qmcspl_eval_vgl_host_ex with a 16-bit output type converts each staged chunk of outputs on the
// device before the device-to-host copies, so that half the bytes cross the link.  Each value is
// rounded to the nearest bfloat16 or IEEE half, ties to even (half: values beyond its range become
// infinities, small ones subnormal).
#include <cuda_fp16.h>

#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

// Thread i converts the 8 consecutive floats 8i .. 8i + 7 (aligned 16-byte loads and store when
// the buffers allow), the last partial group element by element.
template <bool BF16>
__global__ void convert_outputs_kernel(const float* __restrict__ src, uint16_t* __restrict__ dst, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k = 8 * i;
    if (k >= n) return;
    auto cvt = [](float x) -> uint16_t {
        if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
        return __half_as_ushort(__float2half_rn(x));
    };
    const bool aligned = ((reinterpret_cast<uintptr_t>(src + k) | reinterpret_cast<uintptr_t>(dst + k)) & 15) == 0;
    if (k + 8 <= n && aligned) {
        const float4 a = reinterpret_cast<const float4*>(src + k)[0];
        const float4 b = reinterpret_cast<const float4*>(src + k)[1];
        uint4 o;
        o.x = cvt(a.x) | ((uint32_t)cvt(a.y) << 16);
        o.y = cvt(a.z) | ((uint32_t)cvt(a.w) << 16);
        o.z = cvt(b.x) | ((uint32_t)cvt(b.y) << 16);
        o.w = cvt(b.z) | ((uint32_t)cvt(b.w) << 16);
        *reinterpret_cast<uint4*>(dst + k) = o;
        return;
    }
    for (long long j = k; j < n && j < k + 8; ++j) dst[j] = cvt(src[j]);
}

}  // namespace

int launch_convert_outputs(const float* src, void* dst, long long n, bool to_bf16, cudaStream_t st)
{
    if (n <= 0) return QMCSPL_OK;
    const long long threads = (n + 7) / 8;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (to_bf16) convert_outputs_kernel<true><<<blocks, 256, 0, st>>>(src, static_cast<uint16_t*>(dst), n);
    else convert_outputs_kernel<false><<<blocks, 256, 0, st>>>(src, static_cast<uint16_t*>(dst), n);
    return cuda_error(cudaGetLastError(), "convert_outputs_kernel launch");
}

}  // namespace qmcspl
