// Throughput probes (no paper counterpart): the peaks that the roofline fractions of the
// ALU-bound kernels are quoted against, measured on the GPU at hand instead of derived from unit
// counts.  Each probe is one launch of independent dependency chains, enough warps per SM to keep
// the unit busy and a loop long enough that launch overhead is negligible; the caller times the
// launch with events on the same stream and divides the returned operation count by the time.
//   kind 0: binary32 fused multiply-add (FFMA), 2 flop each
//   kind 1: binary32 approximate base-2 logarithm (lg2.approx, the special-function unit the
//           near field's logarithms use), 1 operation each
//   kind 2: binary64 fused multiply-add (DFMA), 2 flop each
// The results are written to a device buffer the caller provides (so nothing is optimised away).
#include "common.cuh"

namespace fmm {
namespace {

constexpr int PROBE_TPB = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_TPB) k_probe_ffma(int iters, float* out)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    const float m = 0.999999f, b = 1e-7f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; c++) a[c] = fmaf(a[c], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += a[c];
    out[blockIdx.x * PROBE_TPB + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_TPB) k_probe_lg2(int iters, float* out)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) a[c] = 2.0f + 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; c++) {
                float r;
                asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
                a[c] = r + 2.0f;  // stays in [2, 4): lg2 in [1, 2)
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += a[c];
    out[blockIdx.x * PROBE_TPB + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_TPB) k_probe_dfma(int iters, float* out)
{
    double a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.9999999999, b = 1e-12;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; c++) a[c] = fma(a[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += a[c];
    out[blockIdx.x * PROBE_TPB + threadIdx.x] = (float)s;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" int fmm_probe_throughput(int kind, int iters, float* out, double* ops, void* stream)
{
    if (!out || !ops) return fail(FMM_ERR_ARG, "NULL argument");
    if (kind < 0 || kind > 2) return fail(FMM_ERR_ARG, "unknown probe %d", kind);
    if (iters < 1 || iters > (1 << 20)) return fail(FMM_ERR_ARG, "iterations %d outside [1, 2^20]", iters);
    int dev = 0, sms = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)(sms * PROBE_BLOCKS_PER_SM);
    cudaStream_t s = (cudaStream_t)stream;
    const double per_thread = (double)iters * 16 * PROBE_CHAINS;
    const double threads = (double)blocks * PROBE_TPB;
    if (kind == 0) {
        k_probe_ffma<<<blocks, PROBE_TPB, 0, s>>>(iters, out);
        *ops = 2.0 * per_thread * threads;
    } else if (kind == 1) {
        k_probe_lg2<<<blocks, PROBE_TPB, 0, s>>>(iters, out);
        *ops = per_thread * threads;
    } else {
        k_probe_dfma<<<blocks, PROBE_TPB, 0, s>>>(iters, out);
        *ops = 2.0 * per_thread * threads;
    }
    note_launch();
    FMM_LAUNCH_CHECK("throughput probe");
    return FMM_OK;
}

extern "C" int fmm_probe_blocks(void)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(FMM_ERR_CUDA, "device query");
    return sms * PROBE_BLOCKS_PER_SM;
}
