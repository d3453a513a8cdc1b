// Device-wide exclusive scan of int32 counts with a base offset read from device memory, used to
// turn per-box list lengths into CSR offsets without a host round trip.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int STPB = 256;
constexpr int SITEMS = 16;
constexpr int STILE = STPB * SITEMS;

__device__ __forceinline__ int64_t block_scan64(int64_t v, int64_t* tmp, int64_t& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) tmp[lane] = s;
    }
    __syncthreads();
    total = tmp[nw - 1];
    int64_t before = w ? tmp[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(STPB) k_tile_sums(const int32_t* __restrict__ in, int64_t m,
                                                    int64_t* __restrict__ sums)
{
    __shared__ int64_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * STILE + (int64_t)threadIdx.x * SITEMS;
    int64_t s = 0;
    for (int j = 0; j < SITEMS; j++)
        if (base + j < m) s += in[base + j];
    int64_t tot;
    block_scan64(s, tmp, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* sums, int64_t nt)
{
    __shared__ int64_t tmp[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < nt; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < nt ? sums[i] : 0;
        int64_t tot;
        int64_t e = block_scan64(v, tmp, tot);
        if (i < nt) sums[i] = carry + e;
        carry += tot;
    }
}

// out[i] = base + sum_{j<i} in[j], i = 0..m.  Values are clamped to INT32_MAX (the caller's
// capacity check then reports the overflow).
__global__ void __launch_bounds__(STPB) k_scan_down(const int32_t* __restrict__ in, int64_t m,
                                                    const int64_t* __restrict__ sums,
                                                    const int32_t* __restrict__ basep,
                                                    int32_t* __restrict__ out)
{
    __shared__ int64_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * STILE + (int64_t)threadIdx.x * SITEMS;
    int32_t v[SITEMS];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SITEMS; j++) {
        v[j] = (base + j < m) ? in[base + j] : 0;
        s += v[j];
    }
    int64_t tot;
    int64_t e = block_scan64(s, tmp, tot);
    int64_t run = (int64_t)basep[0] + sums[blockIdx.x] + e;
#pragma unroll
    for (int j = 0; j < SITEMS; j++) {
        if (base + j < m) {
            out[base + j] = (int32_t)min(run, (int64_t)INT32_MAX);
            run += v[j];
            if (base + j == m - 1) out[m] = (int32_t)min(run, (int64_t)INT32_MAX);
        }
    }
}

}  // namespace

int64_t scan_tmp_words(int64_t m) { return 2 * ((m + STILE - 1) / STILE) + 2; }

int scan_with_base(const int32_t* in, int64_t m, const int32_t* base, int32_t* out, uint32_t* tmp,
                   cudaStream_t s)
{
    if (m <= 0) return 0;
    int64_t nt = (m + STILE - 1) / STILE;
    int64_t* sums = (int64_t*)tmp;
    k_tile_sums<<<(unsigned)nt, STPB, 0, s>>>(in, m, sums); note_launch();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nt); note_launch();
    k_scan_down<<<(unsigned)nt, STPB, 0, s>>>(in, m, sums, base, out); note_launch();
    FMM_LAUNCH_CHECK("scan");
    return 0;
}

}  // namespace fmm
