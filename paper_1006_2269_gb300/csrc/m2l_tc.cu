// M2L on the tensor cores (binary32 path): the far-to-local shifts of Section 4 as one dense
// contraction over every weak pair of every level.
//
// With radius-scaled coefficients the shift of a multipole a~ (source box s, radius rho_s) to a
// local expansion b~ (target box t, radius rho_t), z0 = c_s - c_t, u = -2 rho_s / z0 and
// v = 2 rho_t / z0, is
//     b~_l = v^l * sum_k M'[l][k] x_k,   x_0 = a~_0,  x_k = a~_k u^k  (k >= 1),
//     b~_0 += a~_0 log|z0|,
// with the constant matrix M'[l][k] = C(l+k-1, k-1) / 2^(l+k) (k >= 1), M'[l][0] = -1/(l 2^l),
// M'[0][0] = 0: a diagonal pre-scaling, one constant matrix, a diagonal post-scaling -- the
// "constant transition matrix with pre- and post-scaling" of Section 4.  A tile of 128 weak
// pairs stacks the pre-scaled rows x into X[128][K] (real and imaginary parts separately) and the
// tensor cores form X M'^T; the pre- and post-scaling, the logarithm and the reduction into the
// target boxes stay on the SIMT units.
//
// Precision: tcgen05 multiplies tf32 operands (11 significant bits) and accumulates in binary32.
// Both operands are split into a tf32 high part and a tf32 low part (x = x_hi + x_lo to about
// 2^-22 relative; M' likewise) and three products are accumulated, X_hi M_hi + X_hi M_lo +
// X_lo M_hi: the dropped X_lo M_lo and the residuals are about 2^-22 of each term.
//
// Mechanics (sm_100-family tcgen05): 128 threads per CTA, one row (weak pair) per thread.  The
// operands live in shared memory in the canonical K-major layout without swizzle (8-row x 16-byte
// core matrices; K-adjacent core matrices 128 B apart, 8-row groups KC/4 x 128 B apart) and are
// described by 64-bit shared-memory descriptors.  One thread issues the MMAs (M = 128, N = 32,
// K = 8 per instruction) into two 32-column TMEM accumulators (real, imaginary), commits them to
// an mbarrier, and after the wait every warp reads its 32 TMEM lanes with tcgen05.ld.  Every wait
// is bounded: a wait that gives up sets the timeout bit of the status word, waits (bounded) for
// the MMAs in flight, frees the TMEM and returns.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int TC_ROWS = 128;  // weak pairs per tile = MMA M = threads per CTA
constexpr int TC_N = 32;      // output coefficients l (MMA N), P <= 32
constexpr int CORE = 128;     // bytes of one core matrix: 8 rows x 16 bytes
constexpr int TMEM_COLS = 64; // two 32-column binary32 accumulators
constexpr int64_t WAIT_LIMIT = int64_t(1) << 20;  // tries of a bounded wait (each may suspend briefly)

__constant__ float c_tc[2][TC_N][32];  // M' as tf32 high and low parts, zero-padded

template <int KC>
struct TcLayout {
    static constexpr int KG = KC / 4;           // core matrices along K
    static constexpr int LBO = CORE;            // K-adjacent core matrices
    static constexpr int SBO = CORE * KG;       // 8-row groups
    static constexpr int A_BYTES = TC_ROWS * KC * 4;
    static constexpr int B_BYTES = TC_N * KC * 4;
    static constexpr int OFF_BH = 0, OFF_BL = B_BYTES, OFF_A = 2 * B_BYTES;  // A: re_hi, re_lo, im_hi, im_lo
    static constexpr int OFF_MISC = OFF_A + 4 * A_BYTES;
    static constexpr int STG = 2 * KC + 1;      // staging row stride in floats (odd: no bank conflicts)
    static constexpr int STAGE_BYTES = TC_ROWS * STG * 4 + 2 * TC_ROWS * 4;  // reuses the A region
    static_assert(STAGE_BYTES <= 4 * A_BYTES, "staging must fit in the operand region");
    static constexpr int SMEM = OFF_MISC + 16 + 4 * TC_ROWS;
};

// byte offset of element (row r, column k) in the canonical K-major layout without swizzle
template <int KC>
__device__ __forceinline__ int kmaj(int r, int k)
{
    return (r & 7) * 16 + (k & 3) * 4 + (k >> 2) * TcLayout<KC>::LBO + (r >> 3) * TcLayout<KC>::SBO;
}

__device__ __forceinline__ float tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// x ~ hi + lo with both parts tf32 (11 significant bits, rounded to nearest): |x - hi - lo| is
// about 2^-23 |x|.  The MMA reads tf32 operands by dropping the low 13 bits, so both parts are
// rounded here.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo)
{
    hi = tf32(x);
    lo = tf32(x - hi);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets in
// 16-byte units, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (uint64_t(1) << 46);
}

// Instruction descriptor of kind::tf32: D binary32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12
// = 2), both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int64_t i = 0; i < WAIT_LIMIT; i++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void two_sum_f(float& hi, float& lo, float v)
{
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}


__device__ __forceinline__ unsigned lanemask_lt_()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int KC>
__global__ void __launch_bounds__(TC_ROWS, (KC <= 24 ? 4 : 3)) k_m2l_tc(Sched sc, const Inst* __restrict__ I,
                                                    const LInst* __restrict__ LIs, int P, int PS,
                                                    const int32_t* __restrict__ woff,
                                                    const int32_t* __restrict__ widx,
                                                    const int32_t* __restrict__ wtgt,
                                                    const float* __restrict__ chi, const float* __restrict__ clo,
                                                    const float* __restrict__ rad32,
                                                    const float2* __restrict__ Me, float* __restrict__ Le,
                                                    float* __restrict__ L0lo, int32_t* status)
{
    using Lay = TcLayout<KC>;
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int STG = Lay::STG;
    uint64_t* bar = (uint64_t*)(sm + Lay::OFF_MISC);
    uint32_t* tslot = (uint32_t*)(sm + Lay::OFF_MISC + 8);
    int* flag = (int*)(sm + Lay::OFF_MISC + 12);
    int* tgt_s = (int*)(sm + Lay::OFF_MISC + 16);
    float* stage = (float*)(sm + Lay::OFF_A);
    int* seg_start = (int*)(sm + Lay::OFF_A + TC_ROWS * STG * 4);  // after the staged rows
    int* seg_tgt = seg_start + TC_ROWS;
    __shared__ int wcnt[4];

    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    if (S.L < 1) return;  // CTA-uniform, before any TMEM is taken
    woff += S.o0;
    widx += TL.w0;
    wtgt += TL.w0;
    chi += 2 * S.b0;
    clo += 2 * S.b0;
    rad32 += S.b0;
    Me += S.b0 * PS;
    Le += 2 * S.b0 * PS;
    L0lo += S.b0;
    const int64_t e_begin = woff[1];
    const int64_t e_end = min((int64_t)woff[S.nbox], TL.wcap);
    const int64_t ntile = e_end > e_begin ? (e_end - e_begin + TC_ROWS - 1) / TC_ROWS : 0;

    // constant operand (both parts) and the barrier
    for (int e = t; e < TC_N * KC; e += TC_ROWS) {
        const int n = e / KC, k = e % KC;
        *(float*)(sm + Lay::OFF_BH + kmaj<KC>(n, k)) = c_tc[0][n][k];
        *(float*)(sm + Lay::OFF_BL + kmaj<KC>(n, k)) = c_tc[1][n][k];
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 1;
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t bar_a = smem_u32(bar);
    const uint32_t sbase = smem_u32(sm);
    uint32_t phase = 0;
    bool pending = false;  // an MMA batch committed but not yet observed complete

    // the inputs of row t are loaded one tile ahead, so their latency overlaps the MMAs, the
    // post-scaling and the reduction of the tile before
    int64_t cg = -1;
    float2 ha, hb, la, lb;
    float rs = 0.f, rt = 0.f;
    float4 av[KC / 2];
    auto fetch = [&](int64_t tl) {
        const int64_t e = e_begin + tl * TC_ROWS + t;
        cg = -1;
        if (tl < ntile && e < e_end) {
            cg = wtgt[e];
            const int64_t sg = weak_source(cg, widx[e]);
            ha = *(const float2*)(chi + 2 * sg);
            hb = *(const float2*)(chi + 2 * cg);
            la = *(const float2*)(clo + 2 * sg);
            lb = *(const float2*)(clo + 2 * cg);
            rs = rad32[sg];
            rt = rad32[cg];
            const float4* src = (const float4*)(Me + sg * PS);  // two coefficients per load
#pragma unroll
            for (int k2 = 0; k2 < KC / 2; k2++) av[k2] = 2 * k2 < P ? src[k2] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    fetch(z.rank);

    for (int64_t tile = z.rank; tile < ntile; tile += z.nb) {
        // ---- pre-scaling: row t of X ----
        const bool valid = cg >= 0;
        const int64_t g = cg;
        float vr = 0.f, vi = 0.f, logt = 0.f;
        float xr[KC], xi[KC];
#pragma unroll
        for (int k = 0; k < KC; k++) xr[k] = xi[k] = 0.f;
        if (valid) {
            const float z0r = (ha.x - hb.x) + (la.x - lb.x), z0i = (ha.y - hb.y) + (la.y - lb.y);
            const float r2 = z0r * z0r + z0i * z0i;
            const float ir2 = 1.f / r2;
            const float inr = z0r * ir2, ini = -z0i * ir2;  // 1 / z0
            const float us = -2.f * rs, vs = 2.f * rt;
            const float ur = inr * us, ui = ini * us;
            vr = inr * vs;
            vi = ini * vs;
            float ar[KC], ai[KC];
#pragma unroll
            for (int k2 = 0; k2 < KC / 2; k2++) {
                ar[2 * k2] = av[k2].x;
                ai[2 * k2] = av[k2].y;
                ar[2 * k2 + 1] = 2 * k2 + 1 < P ? av[k2].z : 0.f;
                ai[2 * k2 + 1] = 2 * k2 + 1 < P ? av[k2].w : 0.f;
            }
            const float a0 = ar[0];
            logt = a0 * 0.5f * logf(r2);
            xr[0] = a0;
            float pr = ur, pi = ui;
#pragma unroll
            for (int k = 1; k < KC; k++) {
                xr[k] = ar[k] * pr - ai[k] * pi;
                xi[k] = ar[k] * pi + ai[k] * pr;
                const float nr = pr * ur - pi * ui;
                pi = pr * ui + pi * ur;
                pr = nr;
            }
        }
        tgt_s[t] = valid ? (int)g : -1;
        // split into tf32 high and low parts, 16-byte stores of four K-adjacent values
#pragma unroll
        for (int kg = 0; kg < KC / 4; kg++) {
            float4 rh, rl, ih, il;
            float* prh = &rh.x;
            float* prl = &rl.x;
            float* pih = &ih.x;
            float* pil = &il.x;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                split_tf32(xr[4 * kg + j], prh[j], prl[j]);
                split_tf32(xi[4 * kg + j], pih[j], pil[j]);
            }
            const int off = kmaj<KC>(t, 4 * kg);
            *(float4*)(sm + Lay::OFF_A + 0 * Lay::A_BYTES + off) = rh;
            *(float4*)(sm + Lay::OFF_A + 1 * Lay::A_BYTES + off) = rl;
            *(float4*)(sm + Lay::OFF_A + 2 * Lay::A_BYTES + off) = ih;
            *(float4*)(sm + Lay::OFF_A + 3 * Lay::A_BYTES + off) = il;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // ---- the contraction: D_re = X_re M'^T, D_im = X_im M'^T (three split products each) ----
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int part = 0; part < 2; part++) {  // 0: real, 1: imaginary
                const uint32_t d = tmem + part * TC_N;
                const uint32_t ah = sbase + Lay::OFF_A + (2 * part) * Lay::A_BYTES;
                const uint32_t al = ah + Lay::A_BYTES;
                const uint32_t bh = sbase + Lay::OFF_BH, bl = sbase + Lay::OFF_BL;
#pragma unroll
                for (int ks = 0; ks < KC / 8; ks++) {
                    const uint32_t ko = ks * 2 * Lay::LBO;  // 8 tf32 = two core matrices along K
                    mma_tf32(d, sdesc(ah + ko, Lay::LBO, Lay::SBO), sdesc(bh + ko, Lay::LBO, Lay::SBO), ks > 0);
                    mma_tf32(d, sdesc(ah + ko, Lay::LBO, Lay::SBO), sdesc(bl + ko, Lay::LBO, Lay::SBO), 1);
                    mma_tf32(d, sdesc(al + ko, Lay::LBO, Lay::SBO), sdesc(bh + ko, Lay::LBO, Lay::SBO), 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                         : "memory");
        }
        pending = true;
        fetch(tile + z.nb);  // the next tile's inputs, while the MMAs run
        if (t == 0 && !mbar_wait(bar_a, phase)) {
            atomicOr(status, ST_TIMEOUT);
            *flag = 0;
        }
        __syncthreads();
        if (!*flag) break;
        pending = false;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- post-scaling: row t of the result, 16 coefficients at a time ----
        float* st = stage + t * STG;
        float pr = 1.f, pi = 0.f;
        const uint32_t row = (uint32_t)(32 * w) << 16;
#pragma unroll
        for (int h = 0; h < (KC + 15) / 16; h++) {
            float yr[16], yi[16];
            tmem_ld16(tmem + row + 16 * h, yr);
            tmem_ld16(tmem + row + TC_N + 16 * h, yi);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (valid) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int o = 16 * h + j;
                    if (o < P) {
                        const float br = pr * yr[j] - pi * yi[j], bi = pr * yi[j] + pi * yr[j];
                        if (o == 0) {
                            float hi = logt, lo = 0.f;
                            two_sum_f(hi, lo, br);
                            st[0] = hi;
                            st[1] = bi;
                            st[2 * KC] = lo;
                        } else {
                            st[2 * o] = br;
                            st[2 * o + 1] = bi;
                        }
                    }
                    const float nr = pr * vr - pi * vi;
                    pi = pr * vi + pi * vr;
                    pr = nr;
                }
            }
        }
        // ---- segments of equal target (targets are non-decreasing along the rows) ----
        // a segment also starts at every 32nd row, so that no reduction chain is longer than 32
        const bool head = valid && (t == 0 || tgt_s[t - 1] != (int)g || (t & 31) == 0);
        const unsigned bal = __ballot_sync(0xffffffffu, head);
        if (lane == 0) wcnt[w] = __popc(bal);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        int before = 0, nseg = 0;
        for (int ww = 0; ww < 4; ww++) {
            if (ww < w) before += wcnt[ww];
            nseg += wcnt[ww];
        }
        if (head) {
            const int s = before + __popc(bal & lanemask_lt_());
            seg_start[s] = t;
            seg_tgt[s] = (int)g;
        }
        const int nvalid = (int)min((int64_t)TC_ROWS, e_end - (e_begin + tile * TC_ROWS));
        __syncthreads();
        // ---- reduction: one (segment, coefficient part) per item; Re b_0 in float-float ----
        const int ncol = 2 * P;
        for (int item = t; item < nseg * ncol; item += TC_ROWS) {
            const int s = item / ncol, c = item - s * ncol;
            const int r0 = seg_start[s], r1 = s + 1 < nseg ? seg_start[s + 1] : nvalid;
            const int64_t gg = seg_tgt[s];
            if (c == 0) {
                float hi = 0.f, lo = 0.f;
                for (int r = r0; r < r1; r++) {
                    two_sum_f(hi, lo, stage[r * STG]);
                    lo += stage[r * STG + 2 * KC];
                }
                const float old = atomicAdd(&Le[gg * 2 * PS], hi);
                const float sum = old + hi;
                const float bb = sum - old;
                atomicAdd(&L0lo[gg], ((old - (sum - bb)) + (hi - bb)) + lo);
            } else {
                float a0 = 0.f, a1 = 0.f;
                int r = r0;
                for (; r + 1 < r1; r += 2) {
                    a0 += stage[r * STG + c];
                    a1 += stage[(r + 1) * STG + c];
                }
                if (r < r1) a0 += stage[r * STG + c];
                atomicAdd(&Le[gg * 2 * PS + c], a0 + a1);
            }
        }
        __syncthreads();
    }
    // ---- teardown: no MMA may be in flight when the TMEM is released ----
    if (pending && t == 0) mbar_wait(bar_a, phase);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// The bounded wait above on an mbarrier that nothing completes (it expects one arrival that
// never comes): the wait gives up after `limit` tries, records the timeout and the kernel
// returns.  One warp, no tensor memory, no MMA: it exercises only the give-up path.
__global__ void k_wait_selftest(int64_t limit, int32_t* status)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        bool ok = false;
        for (int64_t i = 0; i < limit && !ok; i++) {
            uint32_t r;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(r)
                : "r"(b), "r"(0u)
                : "memory");
            ok = r != 0;
        }
        if (!ok) atomicOr(status, ST_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b));
    }
}

std::mutex g_tc_mutex;
bool g_tc_ready[128] = {};

float tf32_host(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;  // nearest, ties away
    float r;
    memcpy(&r, &u, 4);
    return r;
}

int ensure_tc_tables()
{
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    if (dev < 0 || dev >= 128) return fail(FMM_ERR_ARG, "device ordinal %d out of range", dev);
    if (g_tc_ready[dev]) return 0;
    static double big[2 * TC_N + 2][2 * TC_N + 2];
    for (int i = 0; i < 2 * TC_N + 2; i++)
        for (int j = 0; j < 2 * TC_N + 2; j++)
            big[i][j] = j == 0 ? 1.0 : (i == 0 ? 0.0 : big[i - 1][j - 1] + big[i - 1][j]);
    static float tab[2][TC_N][32];
    for (int l = 0; l < TC_N; l++)
        for (int k = 0; k < 32; k++) {
            double v;
            if (k == 0)
                v = l == 0 ? 0.0 : -1.0 / ((double)l * ldexp(1.0, l));
            else
                v = ldexp(big[l + k - 1][k - 1], -(l + k));
            const float hi = tf32_host((float)v);
            tab[0][l][k] = hi;
            tab[1][l][k] = tf32_host((float)(v - (double)hi));
        }
    FMM_CUDA(cudaMemcpyToSymbol(c_tc, tab, sizeof(tab)));
    g_tc_ready[dev] = true;
    return 0;
}

template <int KC>
int launch(fmm_tree t, fmm_lists li, int P, int PS, const void* Me, void* Le, cudaStream_t s)
{
    using Lay = TcLayout<KC>;
    FMM_CUDA(cudaFuncSetAttribute(k_m2l_tc<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    k_m2l_tc<KC><<<t->s_m2l.blocks, TC_ROWS, Lay::SMEM, s>>>(
        t->s_m2l.d, t->dinst, li->dlinst, P, PS, li->woff, li->widx, li->wtgt, t->cen_hi, t->cen_lo, t->rad32,
        (const float2*)Me, (float*)Le, t->Lf0lo, t->status);
    note_launch();
    FMM_LAUNCH_CHECK("evaluate: M2L (tensor cores)");
    return 0;
}

}  // namespace

bool m2l_tc_supported(int P) { return P <= 32; }

int bounded_wait_selftest(int64_t limit, cudaStream_t s)
{
    int32_t* st = nullptr;
    if (cudaMalloc((void**)&st, 4) != cudaSuccess) return fail(FMM_ERR_OOM, "status word");
    int rc = FMM_OK;
    int32_t h = 0;
    if (cudaMemsetAsync(st, 0, 4, s) != cudaSuccess) rc = fail(FMM_ERR_CUDA, "memset");
    if (!rc) {
        k_wait_selftest<<<1, 32, 0, s>>>(limit, st);
        note_launch();
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(&h, st, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = fail(FMM_ERR_CUDA, "bounded-wait self-test");
    }
    cudaFree(st);
    if (rc) return rc;
    return (h & ST_TIMEOUT) ? fail(FMM_ERR_TIMEOUT, "the bounded wait gave up after %lld tries, as it should",
                                   (long long)limit)
                            : FMM_OK;
}

// Binary32 M2L over all weak pairs with the tensor cores; Me, Le: [nbox][PS] float2.
int m2l_tc(fmm_tree t, fmm_lists li, int P, int PS, const void* Me, void* Le, cudaStream_t s)
{
    int rc = ensure_tc_tables();
    if (rc) return rc;
    if (t->s_m2l.blocks == 0) return 0;
    if (P <= 8) return launch<8>(t, li, P, PS, Me, Le, s);
    if (P <= 16) return launch<16>(t, li, P, PS, Me, Le, s);
    if (P <= 24) return launch<24>(t, li, P, PS, Me, Le, s);
    return launch<32>(t, li, P, PS, Me, Le, s);
}

}  // namespace fmm
