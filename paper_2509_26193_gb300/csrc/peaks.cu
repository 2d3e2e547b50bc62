// Measurement probes for the roofline denominators of the search (no counterpart in
// the paper): the rates that bound a Barnes-Hut walk on this GPU, measured by
// kernels of this library instead of derived from unit counts and clocks.
//
//   kind 1  FP32 FMA issue: 16 independent FMA chains per thread (one FFMA each).
//   kind 2  special-function unit ex2 (ex2.approx.ftz.f32): 8 independent chains.
//   kind 3  L2 read bandwidth: float4 reads of a device buffer that fits in L2,
//           cached in L2 only (ld.global.cg), `iters` passes.
//   kind 4  packed FP32 FMA (fma.rn.f32x2): 8 independent chains of two lanes.
//
// The host times a launch with CUDA events; `ops` is the work of one launch (FMAs,
// ex2 evaluations, or bytes read). Every kernel stores a value that depends on all
// its arithmetic, so nothing is optimised away.
#include "internal.h"

namespace rl {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int64_t iters, float *out,
                                                                  int64_t out_len)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = 1.0f + 1e-3f * (float)(k + (tid & 7));
    const float b = 0.9999f, c = 1e-4f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    out[tid % out_len] = s;
}

__global__ void __launch_bounds__(kProbeThreads) ffma2_probe_kernel(int64_t iters, float *out,
                                                                    int64_t out_len)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long a[8];
    const float2 bb = make_float2(0.9999f, 0.9998f), cc = make_float2(1e-4f, 2e-4f);
    const unsigned long long b = *reinterpret_cast<const unsigned long long *>(&bb);
    const unsigned long long c = *reinterpret_cast<const unsigned long long *>(&cc);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 v = make_float2(1.0f + 1e-3f * (float)k, 1.0f + 1e-3f * (float)(tid & 7));
        a[k] = *reinterpret_cast<const unsigned long long *>(&v);
    }
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(b), "l"(c));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 v = *reinterpret_cast<const float2 *>(&a[k]);
        s += v.x + v.y;
    }
    out[tid % out_len] = s;
}

__global__ void __launch_bounds__(kProbeThreads) ex2_probe_kernel(int64_t iters, float *out,
                                                                  int64_t out_len)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1e-2f * (float)(k + (tid & 7));
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = ex2_approx(-a[k]); // stays in (0.5, 1]
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[tid % out_len] = s;
}

__global__ void __launch_bounds__(kProbeThreads) l2_probe_kernel(int64_t iters,
                                                                 const float4 *__restrict__ buf,
                                                                 int64_t n4, float *out)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float s = 0.0f;
    for (int64_t it = 0; it < iters; ++it) {
        // a different starting offset per pass so that no SM reads the same lines twice
        // in a row from its own L1 (the loads bypass L1 anyway)
        const int64_t shift = (it * 4099) % n4;
        for (int64_t k = tid; k < n4; k += stride) {
            int64_t j = k + shift;
            if (j >= n4) j -= n4;
            float4 v;
            asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "l"(buf + j));
            s += v.x + v.y + v.z + v.w;
        }
    }
    if (s == 1.2345f) out[0] = s; // never true for the buffers the host passes
}

} // namespace
} // namespace rl

extern "C" relearn_status relearn_peak_probe(int32_t kind, int64_t iters, float *buf,
                                             int64_t buf_len, int64_t *ops, void *stream)
{
    using namespace rl;
    if (iters < 1 || !buf || buf_len < 1 || !ops) return RELEARN_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RELEARN_ERR_CUDA;
    if (cudaPeekAtLastError() != cudaSuccess) return RELEARN_ERR_CUDA; // not ours to clear
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t grid = (int64_t)sms * kProbeBlocksPerSm;
    const int64_t threads = grid * kProbeThreads;
    switch (kind) {
    case 1:
        fma_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, st>>>(iters, buf, buf_len);
        *ops = threads * iters * 8 * 16;
        break;
    case 2:
        ex2_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, st>>>(iters, buf, buf_len);
        *ops = threads * iters * 8 * 8;
        break;
    case 3: {
        const int64_t n4 = buf_len / 4;
        if (n4 < 1 || (reinterpret_cast<uintptr_t>(buf) & 15)) return RELEARN_ERR_INVALID_ARG;
        l2_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, st>>>(
            iters, reinterpret_cast<const float4 *>(buf), n4, buf);
        *ops = iters * n4 * 16;
        break;
    }
    case 4:
        ffma2_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, st>>>(iters, buf, buf_len);
        *ops = threads * iters * 16 * 8 * 2; // FMAs (two per instruction)
        break;
    default:
        return RELEARN_ERR_INVALID_ARG;
    }
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RELEARN_OK : RELEARN_ERR_CUDA;
}
