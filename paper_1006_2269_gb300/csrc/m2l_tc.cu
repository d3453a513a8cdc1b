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
#include <climits>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int TC_ROWS = 128;  // weak pairs per tile = MMA M = threads per CTA
constexpr int TC_N = 32;      // output coefficients l (MMA N), P <= 32
constexpr int CORE = 128;     // bytes of one core matrix: 8 rows x 16 bytes
constexpr int TMEM_COLS = 128;  // two buffers of two 32-column binary32 accumulators
constexpr int64_t WAIT_LIMIT = int64_t(1) << 20;  // tries of a bounded wait (each may suspend briefly)
constexpr int TC_CHUNK_DEFAULT = 16;  // consecutive weak entries per row (tiles per chunk)

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
    static constexpr int SMEM = OFF_MISC + 16;
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// Columns [H, H + W) of this thread's TMEM row (real part at column l, imaginary at TC_N + l),
// post-scaled by (pr, pi) = (2v)^l and added to the running sums; Re b~_0 also takes the log term
// and is summed in float-float.  Every lane of the warp executes the loads.
template <int PI, bool EXACT, int H, int W>
__device__ __forceinline__ void post_scale(uint32_t trow, bool valid, int P, float2 (&acc)[PI], float& lo0,
                                           float& pr, float& pi, float vr, float vi, float logt)
{
    float yr[W], yi[W];
    if constexpr (W == 16) {
        tmem_ld16(trow + H, yr);
        tmem_ld16(trow + TC_N + H, yi);
    } else {
        tmem_ld8(trow + H, yr);
        tmem_ld8(trow + TC_N + H, yi);
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (!valid) return;
#pragma unroll
    for (int j = 0; j < W; j++) {
        const int o = H + j;
        if (o >= PI) break;
        if (EXACT || o < P) {
            if (o == 0) {
                two_sum_f(acc[0].x, lo0, logt);
                two_sum_f(acc[0].x, lo0, yr[0]);
                acc[0].y += yi[0];
            } else {
                acc[o].x += pr * yr[j] - pi * yi[j];
                acc[o].y += pr * yi[j] + pi * yr[j];
            }
        }
        const float nr = pr * vr - pi * vi;
        pi = pr * vi + pi * vr;
        pr = nr;
    }
}

// Largest box id g of the instance with woff[g] <= e (woff non-decreasing, woff[0] = 0 <= e <
// woff[nbox]): the target box of weak entry e.
__device__ __forceinline__ int64_t target_of(const int32_t* __restrict__ woff, int64_t nbox, int64_t e)
{
    int64_t lo = 0, hi = nbox;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(woff + mid) <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Target box of the first entry of every row of every chunk of the tensor-core M2L: rows start
// every T entries from the instance's first weak entry; row k's target goes to rowtgt[k] (k <
// wcap, since k T < wcap).  Same schedule as the M2L launch.
__global__ void k_row_targets(Sched sc, const Inst* __restrict__ I, const LInst* __restrict__ LIs, int T,
                              const int32_t* __restrict__ woff, int32_t* __restrict__ rowtgt)
{
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    if (S.L < 1) return;
    woff += S.o0;
    rowtgt += TL.w0;
    const int64_t e_begin = woff[1];
    const int64_t e_end = min((int64_t)woff[S.nbox], TL.wcap);
    const int64_t nrow = e_end > e_begin ? (e_end - e_begin + T - 1) / T : 0;
    for (int64_t k = (int64_t)z.rank * blockDim.x + threadIdx.x; k < nrow; k += (int64_t)z.nb * blockDim.x)
        rowtgt[k] = (int32_t)target_of(woff, S.nbox, e_begin + k * T);
}

// tf32 high part of a finite binary32 value: rounded to 11 significant bits, ties away from zero
// (the rounding of cvt.rna.tf32 for finite inputs, in two integer operations); x - hi is exact.
__device__ __forceinline__ float tf32_hi(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// Work decomposition.  A chunk is TC_ROWS x T consecutive weak entries (sorted by target).  Row r
// of the CTA owns the T consecutive entries [E0 + r T, E0 + (r + 1) T) and takes one of them per
// tile, so tile i stacks the entries E0 + r T + i of all rows.  Each row keeps the post-scaled
// contributions of its current target in registers and flushes them with vector atomics when the
// target changes: no cross-row reduction, one barrier per tile.  A row finds its first target in
// a table made just before (k_row_targets, one binary search in woff per row) and follows the CSR
// offsets from there, so no per-entry target array is read.  Loads run ahead of their use: the
// next entry's source coefficients and geometry during the MMAs and the epilogue of the current
// one, its source index one entry earlier still, the next chunk's first target and source index
// a chunk ahead.  EXACT: P == PI (no per-coefficient bounds).  PIPE: two TMEM accumulator buffers,
// the epilogue of tile i - 1 runs while the MMAs of tile i execute (two CTAs per SM); otherwise one
// buffer, each tile's epilogue right after its own MMAs (three CTAs per SM up to P = 21, whose
// interleaving hides the MMA latency instead).  Keeping the running sums in TMEM instead of
// registers (four CTAs per SM) measured slower.
template <int PI, bool EXACT, bool PIPE>
__global__ void __launch_bounds__(TC_ROWS, (PI <= 21 && !PIPE) ? 3 : 2) k_m2l_tc(Sched sc, const Inst* __restrict__ I,
                                                    const LInst* __restrict__ LIs, int Prt, int PS, int T, bool rdirect,
                                                    const int32_t* __restrict__ woff,
                                                    const int32_t* __restrict__ widx,
                                                    const int32_t* __restrict__ rowtgt,
                                                    const float* __restrict__ chi, const float* __restrict__ clo,
                                                    const float* __restrict__ rad32,
                                                    const float2* __restrict__ Me, float* __restrict__ Le,
                                                    float* __restrict__ L0lo, int32_t* status)
{
    constexpr int KC = (PI + 7) / 8 * 8;  // K padded to the MMA's 8
    constexpr int NV = (PI + 1) / 2;      // float4 loads of a source row (two coefficients each)
    const int P = EXACT ? PI : Prt;
    using Lay = TcLayout<KC>;
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t* bar = (uint64_t*)(sm + Lay::OFF_MISC);
    uint32_t* tslot = (uint32_t*)(sm + Lay::OFF_MISC + 8);

    const int t = threadIdx.x, w = t >> 5;
    const Slot z = slot_of(sc);
    const Inst S = I[z.i];
    const LInst TL = LIs[z.i];
    if (S.L < 1) return;  // CTA-uniform, before any TMEM is taken
    // instance offsets are added at each access instead of to the pointers, so that the pointers
    // stay kernel parameters (constant bank) and cost no registers
    const int b0 = (int)S.b0, w0 = (int)TL.w0;
    const int64_t o0 = S.o0;
#define WOFF(b) __ldg(woff + o0 + (b))
    const int nbox = (int)S.nbox;
    const int e_begin = WOFF(1);
    const int e_end = (int)min((int64_t)WOFF(nbox), TL.wcap);
    const int csize = TC_ROWS * T;
    const int nchunk = e_end > e_begin ? (e_end - e_begin + csize - 1) / csize : 0;
    if (z.rank >= nchunk) return;  // CTA-uniform

    // constant operand (both parts), the barrier, the accumulator columns
    for (int e = t; e < TC_N * KC; e += TC_ROWS) {
        const int n = e / KC, k = e % KC;
        *(float*)(sm + Lay::OFF_BH + kmaj<KC>(n, k)) = c_tc[0][n][k];
        *(float*)(sm + Lay::OFF_BL + kmaj<KC>(n, k)) = c_tc[1][n][k];
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
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
    const uint32_t trow = (uint32_t)(32 * w) << 16;  // this warp's TMEM lanes
    unsigned char* arow = sm + Lay::OFF_A + kmaj<KC>(t, 0);  // this row in the A operand
    uint32_t phase = 0;
    bool bad = false;      // a wait of this thread gave up: the CTA stops at the next barrier
    bool pending = false;  // thread 0: an MMA batch committed and not observed complete

    // the entry being prefetched: target g (woff[g + 1] = gend, woff[g + 2] = gend2), the source
    // index wn of the entry after it
    int g = 0, gend = 0, gend2 = 0, wn = 0;
    // prefetched inputs of the next entry (ng < 0: none)
    int ng = -1;
    float2 nha, nla, thb, tlb;
    float nrs = 0.f, trt = 0.f;
    float4 nav[NV];
    auto next_off = [&](int b) { return b + 2 <= nbox ? WOFF(b + 2) : INT_MAX; };
    auto set_target = [&](int b) {
        g = b;
        thb = __ldg((const float2*)(chi + 2 * (int64_t)(b0 + b)));
        tlb = __ldg((const float2*)(clo + 2 * (int64_t)(b0 + b)));
        trt = __ldg(rad32 + b0 + b);
    };
    auto fetch = [&](int e, int e1) {
        ng = -1;
        if (e >= e1) return;
        if (e >= gend) {  // the next target (boxes without entries are skipped)
            int b = g + 1, be = gend2;
            while (e >= be) be = WOFF((++b) + 1);
            set_target(b);
            gend = be;
            gend2 = next_off(b);
        }
        ng = g;
        const int sg = (int)weak_source(g, wn);
        if (e + 1 < e1) wn = __ldg(widx + w0 + e + 1);
        nha = __ldg((const float2*)(chi + 2 * (int64_t)(b0 + sg)));
        nla = __ldg((const float2*)(clo + 2 * (int64_t)(b0 + sg)));
        nrs = __ldg(rad32 + b0 + sg);
        const float4* src = (const float4*)(Me + (int64_t)(b0 + sg) * PS);
#pragma unroll
        for (int k2 = 0; k2 < NV; k2++)  // coefficients 2 k2, 2 k2 + 1 < PS (P rounded up to even)
            nav[k2] = (EXACT || 2 * k2 < P) ? __ldg(src + k2) : make_float4(0.f, 0.f, 0.f, 0.f);
    };

    // Re b~_0 of a flushed row goes out as an atomic addition whose returned old value gives the
    // rounding error of the stored sum; that correction is sent at the next flush (or at the end),
    // so the atomic's round trip overlaps the following tiles
    int pcur = -1;
    float pold = 0.f, phi_ = 0.f, plo = 0.f;
    auto complete = [&]() {
        if (pcur < 0) return;
        const float sum = pold + phi_;
        const float bb = sum - pold;
        atomicAdd(L0lo + b0 + pcur, ((pold - (sum - bb)) + (phi_ - bb)) + plo);
        pcur = -1;
    };
    // first target and source index of this row in the CTA's next chunk
    auto row_start = [&](int c) {  // first entry of this row in chunk c (e_end when beyond)
        return (int)min((int64_t)e_begin + (int64_t)c * csize + (int64_t)t * T, (int64_t)e_end);
    };
    int rt_next = 0, w_next = 0;
    auto row_ahead = [&](int c) {
        const int e = row_start(c);
        if (c < nchunk && e < e_end) {
            // row k's first target: the list's every-eighth table when T is a multiple of 8,
            // else the table made for this launch
            const int64_t k = (int64_t)c * TC_ROWS + t;
            rt_next = rdirect ? __ldg(rowtgt + (w0 >> 3) + ((k * T) >> 3)) : __ldg(rowtgt + w0 + k);
            w_next = __ldg(widx + w0 + e);
        }
    };
    int my0 = 0, my1 = 0;  // this row's entries in the chunk being fetched
    auto start_chunk = [&](int c) {
        my0 = row_start(c);
        my1 = (int)min((int64_t)my0 + T, (int64_t)e_end);
        if (my0 < my1) {
            set_target(rt_next);
            gend = WOFF(g + 1);
            gend2 = next_off(g);
            wn = w_next;
        }
        row_ahead(c + z.nb);
    };

    // the row's running sums for target `cur`: Re b~_0 in float-float (acc[0].x + lo0); they carry
    // over from tile to tile (and chunk to chunk) until the target changes
    int cur = -1;
    float2 acc[PI];
    float lo0 = 0.f;
#pragma unroll
    for (int j = 0; j < PI; j++) acc[j] = make_float2(0.f, 0.f);
    auto flush = [&]() {
        float* dst = Le + (int64_t)(b0 + cur) * 2 * PS;
        complete();
        pold = atomicAdd(dst, acc[0].x);  // Re b~_0 as hi/lo (exact two-sum, completed later)
        phi_ = acc[0].x;
        plo = lo0;
        pcur = cur;
        atomicAdd((float4*)dst, make_float4(0.f, acc[0].y, PI > 1 ? acc[1].x : 0.f, PI > 1 ? acc[1].y : 0.f));
#pragma unroll
        for (int j = 2; j < PI; j += 2)
            if (EXACT || j < P)
                atomicAdd((float4*)(dst + 2 * j),
                          make_float4(acc[j].x, acc[j].y, j + 1 < PI ? acc[j + 1].x : 0.f, j + 1 < PI ? acc[j + 1].y : 0.f));
    };
    // post-scaling of a finished tile (TMEM buffer at column `col`) into the running sums:
    // b~_l += (2v)^l (M' x)_l
    auto epilogue = [&](uint32_t col, bool valid, int pg, float vr, float vi, float logt) {
        if (valid && pg != cur) {
            if (cur >= 0) flush();
#pragma unroll
            for (int j = 0; j < PI; j++) acc[j] = make_float2(0.f, 0.f);
            lo0 = 0.f;
            cur = pg;
        }
        float pr = 1.f, pi = 0.f;
        const uint32_t ta = tmem + trow + col;
        // eight columns at a time (fewer live registers beside the prefetched next entry)
        post_scale<PI, EXACT, 0, 8>(ta, valid, P, acc, lo0, pr, pi, vr, vi, logt);
        if constexpr (KC >= 16) post_scale<PI, EXACT, 8, 8>(ta, valid, P, acc, lo0, pr, pi, vr, vi, logt);
        if constexpr (KC >= 24) post_scale<PI, EXACT, 16, 8>(ta, valid, P, acc, lo0, pr, pi, vr, vi, logt);
        if constexpr (KC >= 32) post_scale<PI, EXACT, 24, 8>(ta, valid, P, acc, lo0, pr, pi, vr, vi, logt);
    };

    // Loop over the tiles (chunk c, tile i) of this CTA.  PIPE: wait for the MMAs of the previous
    // tile, write this tile's rows, start the next entry's loads, barrier, one thread issues this
    // tile's MMAs into the other TMEM buffer, and meanwhile every row post-scales the previous
    // tile's results.  Otherwise: write the rows, start the loads, barrier, MMAs, wait, post-scale.
    int c = z.rank, i = 0;
    row_ahead(c);
    start_chunk(c);
    fetch(my0, my1);
    bool have_prev = false;  // a tile whose MMAs were issued and whose epilogue is still due
    bool dvalid = false;
    int dpg = -1;
    float dvr = 0.f, dvi = 0.f, dlogt = 0.f;
    uint32_t buf = 0;  // TMEM columns of this tile's accumulators: 0 or 2 * TC_N
    for (;;) {
        // ---- the previous tile's MMAs have finished: A is free, its accumulators are ready ----
        if (PIPE && have_prev) {
            if (!__all_sync(0xffffffffu, mbar_wait(bar_a, phase))) {  // warp-uniform outcome
                bad = true;
                if ((t & 31) == 0) atomicOr(status, ST_TIMEOUT);
            } else {
                if (t == 0) pending = false;
                phase ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
            }
        }
        // ---- pre-scaling: row t of X from the prefetched inputs (not after a wait gave up: the
        // tensor cores may still read A) ----
        const int pg = ng;
        const bool valid = pg >= 0;
        float vr = 0.f, vi = 0.f, logt = 0.f;
        if (!bad && valid) {
            const float z0r = (nha.x - thb.x) + (nla.x - tlb.x), z0i = (nha.y - thb.y) + (nla.y - tlb.y);
            const float r2 = z0r * z0r + z0i * z0i;
            const float ir2 = __frcp_rn(r2);
            const float inr = z0r * ir2, ini = -z0i * ir2;  // 1 / z0
            const float us = -2.f * nrs, vs = 2.f * trt;
            const float ur = inr * us, ui = ini * us;
            vr = inr * vs;
            vi = ini * vs;
            const float a0 = nav[0].x;
            logt = a0 * 0.5f * logf(r2);
            float xr[KC], xi[KC];
            xr[0] = a0;
            xi[0] = 0.f;
            float pr = ur, pi = ui;
#pragma unroll
            for (int k = 1; k < KC; k++) {
                if (k < PI && (EXACT || k < P)) {
                    const float4 q4 = nav[k >> 1];
                    const float ar = (k & 1) ? q4.z : q4.x, ai = (k & 1) ? q4.w : q4.y;
                    xr[k] = ar * pr - ai * pi;
                    xi[k] = ar * pi + ai * pr;
                    const float nr = pr * ur - pi * ui;
                    pi = pr * ui + pi * ur;
                    pr = nr;
                } else {
                    xr[k] = xi[k] = 0.f;
                }
            }
            // tf32 high part rounded to nearest; the low part keeps the rest (the MMA reads its
            // top 11 bits: about 2^-22 of x is lost)
#pragma unroll
            for (int kg = 0; kg < KC / 4; kg++) {
                float4 rh, rl, ih, il;
                float* prh = &rh.x;
                float* prl = &rl.x;
                float* pih = &ih.x;
                float* pil = &il.x;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    prh[j] = tf32_hi(xr[4 * kg + j]);
                    prl[j] = xr[4 * kg + j] - prh[j];
                    pih[j] = tf32_hi(xi[4 * kg + j]);
                    pil[j] = xi[4 * kg + j] - pih[j];
                }
                const int off = kg * Lay::LBO;
                *(float4*)(arow + 0 * Lay::A_BYTES + off) = rh;
                *(float4*)(arow + 1 * Lay::A_BYTES + off) = rl;
                *(float4*)(arow + 2 * Lay::A_BYTES + off) = ih;
                *(float4*)(arow + 3 * Lay::A_BYTES + off) = il;
            }
        } else if (!bad) {
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int kg = 0; kg < KC / 4; kg++)
#pragma unroll
                for (int a = 0; a < 4; a++) *(float4*)(arow + a * Lay::A_BYTES + kg * Lay::LBO) = z4;
        }
        // ---- the next entry (next tile of this chunk, or the first of the CTA's next chunk) ----
        int cn = c, in = i + 1;
        if (in == T) {
            cn = c + z.nb;
            in = 0;
        }
        if (!bad) {
            if (in == 0) {
                if (cn < nchunk) {
                    start_chunk(cn);
                    fetch(my0, my1);
                } else {
                    ng = -1;
                }
            } else {
                fetch(my0 + in, my1);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) {  // a wait gave up somewhere in the CTA: every thread stops
            bad = true;
            break;
        }
        // ---- this tile's contraction: D_re = X_re M'^T, D_im = X_im M'^T (three split products) ----
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int part = 0; part < 2; part++) {  // 0: real, 1: imaginary
                const uint32_t d = tmem + buf + part * TC_N;
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
            pending = true;
        }
        if constexpr (PIPE) {
            // ---- the previous tile's epilogue, while this tile's MMAs run ----
            if (have_prev) epilogue(buf ^ (2 * TC_N), dvalid, dpg, dvr, dvi, dlogt);
            have_prev = true;
            dvalid = valid;
            dpg = pg;
            dvr = vr;
            dvi = vi;
            dlogt = logt;
            buf ^= 2 * TC_N;
        } else {
            // ---- this tile's epilogue after its MMAs (warp-uniform wait outcome) ----
            if (!__all_sync(0xffffffffu, mbar_wait(bar_a, phase))) {
                bad = true;
                if ((t & 31) == 0) atomicOr(status, ST_TIMEOUT);
            } else {
                if (t == 0) pending = false;
                phase ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
                epilogue(0, valid, pg, vr, vi, logt);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        c = cn;
        i = in;
        if (c >= nchunk) {
            if (!PIPE && __syncthreads_or(bad)) bad = true;  // CTA-uniform before the drain
            break;
        }
    }
    // ---- drain: the last tile's MMAs and epilogue, the last flush ----
    if (!bad && have_prev) {
        if (__all_sync(0xffffffffu, mbar_wait(bar_a, phase))) {
            if (t == 0) pending = false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            epilogue(buf ^ (2 * TC_N), dvalid, dpg, dvr, dvi, dlogt);
        } else {
            bad = true;
            if ((t & 31) == 0) atomicOr(status, ST_TIMEOUT);
        }
    }
    if (!bad && cur >= 0) flush();
    complete();
    // ---- teardown: no MMA may be in flight when the TMEM is released ----
    if (pending && t == 0) mbar_wait(bar_a, phase);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}
#undef WOFF

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

template <int PI, bool EXACT, bool PIPE>
int launch3(fmm_tree t, fmm_lists li, int P, int PS, const void* Me, void* Le, cudaStream_t s)
{
    using Lay = TcLayout<(PI + 7) / 8 * 8>;
    FMM_CUDA(cudaFuncSetAttribute(k_m2l_tc<PI, EXACT, PIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    const int T = t->tune_m2l_chunk > 0 ? t->tune_m2l_chunk : TC_CHUNK_DEFAULT;
    const bool rdirect = T % 8 == 0;  // rows start at list rows of eight entries
    if (!rdirect) {
        k_row_targets<<<t->s_m2l.blocks, 256, 0, s>>>(t->s_m2l.d, t->dinst, li->dlinst, T, li->woff, li->rowtgt);
        note_launch();
    }
    k_m2l_tc<PI, EXACT, PIPE><<<t->s_m2l.blocks, TC_ROWS, Lay::SMEM, s>>>(
        t->s_m2l.d, t->dinst, li->dlinst, P, PS, T, rdirect, li->woff, li->widx, rdirect ? li->wrow : li->rowtgt,
        t->cen_hi, t->cen_lo, t->rad32,
        (const float2*)Me, (float*)Le, t->Lf0lo, t->status);
    note_launch();
    FMM_LAUNCH_CHECK("evaluate: M2L (tensor cores)");
    return 0;
}

// Accumulator stages: 2 (pipelined epilogue) or 1; 0 picks by order (2 from P = 22 on, where the
// register budget is two CTAs per SM anyway).
template <int PI, bool EXACT>
int launch(fmm_tree t, fmm_lists li, int P, int PS, const void* Me, void* Le, cudaStream_t s)
{
    const bool pipe = t->tune_m2l_stages == 2 || (t->tune_m2l_stages == 0 && P > 21);
    return pipe ? launch3<PI, EXACT, true>(t, li, P, PS, Me, Le, s) : launch3<PI, EXACT, false>(t, li, P, PS, Me, Le, s);
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
    // exact instantiations for the orders of the benchmark workloads (p = 16, 20, 30)
    if (P == 17) return launch<17, true>(t, li, P, PS, Me, Le, s);
    if (P == 21) return launch<21, true>(t, li, P, PS, Me, Le, s);
    if (P == 31) return launch<31, true>(t, li, P, PS, Me, Le, s);
    if (P <= 8) return launch<8, false>(t, li, P, PS, Me, Le, s);
    if (P <= 16) return launch<16, false>(t, li, P, PS, Me, Le, s);
    if (P <= 24) return launch<24, false>(t, li, P, PS, Me, Le, s);
    return launch<32, false>(t, li, P, PS, Me, Le, s);
}

}  // namespace fmm
