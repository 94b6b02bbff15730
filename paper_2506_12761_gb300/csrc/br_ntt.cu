// Blind rotation with the external product computed exactly by a two-prime
// number-theoretic transform (integer pipe only; no floating point).
//
// Per step i the product out_j = sum_r D_r(X) * BK_i[r][j](X) mod (X^N+1) is an
// integer polynomial whose coefficients are bounded by 6 * N * 64 * 2^32 <
// 2^50.6 in magnitude (digits |d| <= 64, key words < 2^32).  It is computed
// modulo p0 = 167772161 and p1 = 195198977 (both 1 mod 2N) with negacyclic
// NTTs, recombined by the Chinese remainder theorem into the exact signed
// integer (p0 * p1 > 2^54.8), and reduced mod 2^32: bit-identical to the
// dense contraction.
//
// Transform: Cooley-Tukey forward / Gentleman-Sande inverse with the powers of
// a primitive 2N-th root psi in bit-reversed order (the merged negacyclic
// form), Shoup multiplications with lazy reduction.  Both primes are below
// 2^32 / 22, so a forward value, which grows by less than 2p per stage from
// below 2p, stays below 22p < 2^32 through all ten stages with no reduction,
// six pointwise products (each below 2p) sum to less than 12p, and the
// inverse reduces only on every third stage.
// The pointwise products are Shoup multiplications by the transformed key,
// stored with N^-1 folded in and with each value's Shoup companion.
//
// Layout: one warp owns one bootstrap.  A 1024-point transform lives in the
// warp's registers, 32 points per lane; the five stages whose pairs lie in
// one lane run in registers, a 32x32 shared-memory transpose (16-byte rows
// XOR-swizzled) moves to the other lane grouping, and five more stages run in
// registers.  No block
// barrier is involved: each warp synchronises only itself.  Warp 0 also
// streams the transformed key in 16 KB chunks (one step, prime and row) into a
// ring with bulk asynchronous copies; full/empty mbarriers hand the chunks
// between warp 0 (which issues the copies) and all compute warps.
#include <algorithm>
#include <cstdio>
#include <utility>
#include <vector>

#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kShapes[5] = {6, 8, 9, 10, 12}; // compute warps = bootstraps per CTA, chosen per launch
constexpr int kMaxWarps = 12;
constexpr int kTwLane = 31 * 32;               // lane-dependent twiddles of one transform: 31 groups x 32 lanes
constexpr uint32_t kTmemCols = 512;            // per CTA: up to 3 warps share a 32-lane quarter, 112 columns each
constexpr uint32_t kTmemWarpCols = 112;        // per warp: 64 for the product mod p0, 48 for the packed digits
constexpr uint32_t kP[2] = {167772161u, 195198977u};   // p0 < p1 < 2^32 / 22: the bounds below rely on it
constexpr uint32_t kPmod32 = (uint32_t)(167772161ull * 195198977ull);   // p0 p1 mod 2^32
constexpr int kXch = 32 * 32;                  // transpose tile (16-byte chunks XOR-swizzled by row)
constexpr int kChunkWords = 4 * kN;            // one (step, prime, row): per output component the values and their Shoup companions, 16 KB
constexpr int kChunks = kn * 2 * kRows;        // consumed in this order: step, prime, row
constexpr size_t kBkNttWords = (size_t)kChunks * kChunkWords;
constexpr int kRing = 2;                       // ring slots of the key stream

// Twiddles psi^(+-brv(k)) with their Shoup companions floor(w * 2^32 / p) as
// (w, w') pairs: [prime][0 = forward, 1 = inverse][k].  Uniformly indexed
// stages read the constant bank (one 8-byte load per pair); lane-dependent
// stages read the shared-memory copy of gWL below.
__constant__ uint2 cWp[2][2][kN];
// The lane-dependent twiddles of the in-lane stages after (forward) or before
// (inverse) the transpose, as (w, w') pairs in [stage][group][lane] order so
// that a warp reads them from shared memory without bank conflicts.
__device__ uint2 gWL[2][2][kTwLane];
// The first two forward stages of a digit polynomial by lookups.  Stage 0
// multiplies digits d = b - 64 (b the packed byte) by its one twiddle
// psi^512; stage 1 multiplies d + psi^512 d' by psi^256 or psi^768, which by
// linearity (and psi^1024 = -1) is a sum of two lookups.  gTab[prime][0][b] =
// psi^512 d, [1][b] = psi^256 d, [2][b] = psi^768 d, all mod p.
__device__ uint32_t gTab[2][3][128];

struct PrimeConsts {
    uint32_t p[2];
    uint32_t scale[2];       // N^-1 mod p: folds the inverse scaling into the key
    uint32_t crt_inv;        // p0^-1 mod p1
    uint32_t crt_inv_s;      // its Shoup companion
};
__constant__ PrimeConsts cP;

template <int WARPS> struct __align__(128) Smem {
    uint32_t ring[kRing][kChunkWords];    // 2 x 16 KB: stream of the transformed key
    uint2 twl[2][2][kTwLane];             // 31 KB: lane-dependent twiddles [prime][direction]
    uint32_t tab[2][3][128];              // 3 KB: first-two-stage products of the digits, per prime
    uint32_t acc[WARPS][2 * kN];          // 8 KB per warp: ACC of its bootstrap
    uint32_t xch[WARPS][kXch];            // 4.1 KB per warp: transpose tile
    uint16_t abar[WARPS][kSlotWords];     // modulus-switched input
    BrJob job[WARPS];
    unsigned long long full[kRing], empty[kRing];
    uint32_t tmem_base;                   // Tensor Memory holding each warp's product mod p0
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait on the mbarrier phase `parity` for at most kWaitNs; on timeout record
// it in the error word and return false.  Once any wait has given up, later
// waits return at once, so a failed launch ends quickly instead of spinning.
__device__ __forceinline__ bool mbar_try(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// A phase that has already completed returns at once, without touching the
// error word or the timer (the common case: the chunk landed during the
// transform).  Otherwise the wait is bounded as above.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int *err)
{
    if (mbar_try(bar, parity)) return true;
    if (*reinterpret_cast<volatile int *>(err) != kDevOk) return false;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) {
            atomicExch(err, kDevTimeout);
            return false;
        }
    }
}

// Bounded wait that ignores the error word: lets copies still in flight land
// before the CTA exits.
__device__ __forceinline__ void mbar_drain(unsigned long long *bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try(bar, parity) && global_ns() - t0 <= kWaitNs) {
    }
}

__device__ __forceinline__ void load_chunk(uint32_t *dst, const uint32_t *src, unsigned long long *bar)
{
    constexpr uint32_t bytes = kChunkWords * 4;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Tensor Memory as per-lane scratch: a warp reaches only the 32 lanes of
// quarter (warp id mod 4); each thread reads and writes its own lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Issue a load of 8 columns without waiting: the registers are valid only
// after tmem_wait_ld(), and nothing may read them before.
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x * w mod p in [0, 2p) for any x < 2^32 (Shoup, ws = floor(w 2^32 / p)).
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t ws, uint32_t p)
{
    const uint32_t q = __umulhi(x, ws);
    return x * w - q * p;
}

__device__ __forceinline__ uint32_t red2(uint32_t x, uint32_t m) { return min(x, x - m); }  // [0,2m) -> [0,m)

// x mod p into [0, 2p) for any x < 2^32: Shoup's reduction with w = 1, pinv = floor(2^32 / p).
__device__ __forceinline__ uint32_t red_shoup(uint32_t x, uint32_t pinv, uint32_t p) { return x - __umulhi(x, pinv) * p; }

// Bits [s, s + 7) of y placed at bits [b, b + 7), everything else zero (s and b
// are constants after unrolling: one shift and one masked OR).
__device__ __forceinline__ uint32_t field7(uint32_t y, int s, int b)
{
    return (s >= b ? (y >> (s - b)) : (y << (b - s))) & (127u << b);
}

// Cooley-Tukey butterfly without reduction: t = w Y mod p is below 2p, so
// outputs exceed the inputs' bound by less than 2p.
__device__ __forceinline__ void bf_fwd(uint32_t &X, uint32_t &Y, uint32_t w, uint32_t ws, uint32_t p)
{
    const uint32_t x = X;
    const uint32_t t = mul_shoup(Y, w, ws, p);
    X = x + t;
    Y = x - t + 2 * p;
}

// Gentleman-Sande butterfly of inverse stage k, inputs below B = 2p << (k mod 3):
// Y = w (x - y) mod p below 2p; X = x + y below 2B, brought back below 2p on
// every third stage (k mod 3 == 2, where 2B = 16p).
template <int k>
__device__ __forceinline__ void bf_inv(uint32_t &X, uint32_t &Y, uint32_t w, uint32_t ws, uint32_t p, uint32_t pinv)
{
    const uint32_t x = X, y = Y;
    X = (k % 3 == 2) ? red_shoup(x + y, pinv, p) : x + y;
    Y = mul_shoup(x - y + ((2 * p) << (k % 3)), w, ws, p);
}

// 32x32 transpose of a warp's registers through shared memory: lane L's x[t]
// becomes lane t's x[L].  It maps the column layout (lane L holds points
// L + 32t) to the row layout (lane L holds points 32L + t) and back.  Each
// lane stores its 32 values as one row with 16-byte stores whose chunk
// order is XOR-swizzled by the row, so both the stores (8 lanes per 128-byte
// wavefront) and the column reads hit 32 distinct banks.
__device__ __forceinline__ void transpose32(uint32_t (&x)[32], uint32_t *m, int lane)
{
    uint4 *row = reinterpret_cast<uint4 *>(m + 32 * lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) row[j ^ (lane & 7)] = make_uint4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 32; ++t) x[t] = m[32 * t + 4 * ((lane >> 2) ^ (t & 7)) + (lane & 3)];
    __syncwarp();
}

// Forward negacyclic NTT mod kP[pi] of one polynomial: column layout in
// (values below 2p), row layout out (transform order), values below 22p.  Every loop has a
// compile-time trip count and every array index is a compile-time constant,
// so the 32 points stay in registers.
// S0 = 2: stages 0 and 1 were already applied (the digit path's lookups).
template <int S0>
__device__ __forceinline__ void ntt_fwd(uint32_t (&x)[32], int pi, uint32_t *xch, int lane, const uint2 *twl)
{
    const uint32_t p = kP[0] + (uint32_t)pi * (kP[1] - kP[0]);
    const uint2 *cw = &cWp[pi][0][0];
#pragma unroll
    for (int s = S0; s < 5; ++s) {           // distance 512 >> s: within a lane
        const int dt = 16 >> s;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const int t = (b / dt) * 2 * dt + (b % dt);
            const int k = (1 << s) + (t >> (5 - s));
            const uint2 w = cw[k];
            bf_fwd(x[t], x[t + dt], w.x, w.y, p);
        }
    }
    transpose32(x, xch, lane);
#pragma unroll
    for (int s = 5; s < 10; ++s) {           // distance 512 >> s < 32: within a lane after the transpose
        const int dt = 1 << (9 - s);
        const int base = 32 * ((1 << (s - 5)) - 1);              // groups of the earlier stages
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const int g = b / dt;                                  // group of this lane's points
            const int t = g * 2 * dt + (b % dt);
            const uint2 w = twl[base + g * 32 + lane];
            bf_fwd(x[t], x[t + dt], w.x, w.y, p);
        }
    }
}

// Inverse negacyclic NTT mod kP[pi] of two polynomials at once: row layout
// (transform order) in, values below 2p; column layout out (natural order),
// values below 4p.  The N^-1 scaling is folded into the key.
template <int k>
__device__ __forceinline__ void inv_stage_in_lane(uint32_t (&a)[32], uint32_t (&c)[32], const uint2 *twl, int lane,
                                                  uint32_t p, uint32_t pinv)
{
    constexpr int dt = 1 << k;
    constexpr int base = 32 * (32 - (32 >> k));                    // groups of the earlier stages: 16, 8, 4, 2
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const int g = b / dt;
        const int t = g * 2 * dt + (b % dt);
        const uint2 w = twl[base + g * 32 + lane];
        bf_inv<k>(a[t], a[t + dt], w.x, w.y, p, pinv);
        bf_inv<k>(c[t], c[t + dt], w.x, w.y, p, pinv);
    }
}

template <int k>
__device__ __forceinline__ void inv_stage_uniform(uint32_t (&a)[32], uint32_t (&c)[32], const uint2 *cw, uint32_t p,
                                                  uint32_t pinv)
{
    constexpr int dt = 1 << (k - 5);
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const int t = (b / dt) * 2 * dt + (b % dt);
        const int idx = (512 >> k) + (t >> (k - 4));
        const uint2 w = cw[idx];
        bf_inv<k>(a[t], a[t + dt], w.x, w.y, p, pinv);
        bf_inv<k>(c[t], c[t + dt], w.x, w.y, p, pinv);
    }
}

__device__ __forceinline__ void ntt_inv2(uint32_t (&a)[32], uint32_t (&c)[32], int pi, uint32_t *xch, int lane,
                                         const uint2 *twl)
{
    const uint32_t p = kP[0] + (uint32_t)pi * (kP[1] - kP[0]);
    const uint32_t pinv = pi ? 22u : 25u;                       // floor(2^32 / p)
    // distance 1 << k: within a lane
    inv_stage_in_lane<0>(a, c, twl, lane, p, pinv);
    inv_stage_in_lane<1>(a, c, twl, lane, p, pinv);
    inv_stage_in_lane<2>(a, c, twl, lane, p, pinv);
    inv_stage_in_lane<3>(a, c, twl, lane, p, pinv);
    inv_stage_in_lane<4>(a, c, twl, lane, p, pinv);
    transpose32(a, xch, lane);
    transpose32(c, xch, lane);
    // distance 32 << (k - 5): within a lane after the transpose
    const uint2 *cw = &cWp[pi][1][0];
    inv_stage_uniform<5>(a, c, cw, p, pinv);
    inv_stage_uniform<6>(a, c, cw, p, pinv);
    inv_stage_uniform<7>(a, c, cw, p, pinv);
    inv_stage_uniform<8>(a, c, cw, p, pinv);
    inv_stage_uniform<9>(a, c, cw, p, pinv);
}

// CTA c takes jobs [c * per, c * per + per) (per <= WARPS); its other warps idle.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1)
br_ntt_kernel(const BrJob *__restrict__ jobs, int njobs, int per, const uint32_t *__restrict__ bkhat,
              uint32_t *__restrict__ big, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    Smem<WARPS> &S = *reinterpret_cast<Smem<WARPS> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int job0 = blockIdx.x * per;
    const int nact = min(per, njobs - job0);

    if (tid < WARPS) {
        BrJob j{};
        if (tid < nact) j = jobs[job0 + tid];
        S.job[tid] = j;
    }
    {
        const uint2 *src = &gWL[0][0][0];
        uint2 *dst = &S.twl[0][0][0];
        for (int k = tid; k < 4 * kTwLane; k += WARPS * 32) dst[k] = src[k];
        for (int k = tid; k < 2 * 3 * 128; k += WARPS * 32) (&S.tab[0][0][0])[k] = (&gTab[0][0][0])[k];
    }
    if (tid == 0) {
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&S.full[r], 1);
            mbar_init(&S.empty[r], (uint32_t)nact);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // warp 0 allocates the CTA's Tensor Memory and frees it at the end
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // Warp 0 keeps the key stream kRing chunks ahead: it issues the first
    // chunks now and chunk c + kRing once every warp has released chunk c.
    if (warp == 0 && lane == 0)
        for (int c = 0; c < kRing && c < kChunks; ++c)
            load_chunk(S.ring[c], bkhat + (size_t)c * kChunkWords, &S.full[c]);
    if (warp >= nact) return;

    const BrJob J = S.job[warp];
    uint32_t *acc = S.acc[warp];
    // this warp's columns in its lane quarter: [0, 32) and [32, 64) the product mod p0
    // (components a, b); [64, 112) the digit polynomials, 8 packed words per row
    const uint32_t tres = S.tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + kTmemWarpCols * (uint32_t)(warp >> 2);
    const uint32_t tdig = tres + 64;
    uint32_t *xch = S.xch[warp];
    uint16_t *abar = S.abar[warp];

    // Gate pre-combination and modulus switch.
    for (int i = lane; i < kLweWords; i += 32) {
        uint32_t c = (i == kn) ? J.cst : 0u;
        if (J.in0) c += (uint32_t)J.s0 * J.in0[i];
        if (J.in1) c += (uint32_t)J.s1 * J.in1[i];
        abar[i] = (uint16_t)((c + (1u << 20)) >> 21);
    }
    __syncwarp();
    // ACC = (0, X^{-bbar} v), v = mu * sum_j X^j
    {
        const uint32_t bbar = abar[kn];
        for (int k = lane; k < kN; k += 32) {
            const uint32_t u = ((uint32_t)k + bbar) & (kTwoN - 1);
            acc[k] = 0u;
            acc[kN + k] = (u < (uint32_t)kN) ? kMu : (0u - kMu);
        }
    }
    __syncwarp();

    constexpr uint32_t kOff = (1u << 31) + (1u << 24) + (1u << 17) + (1u << 10);
    const uint32_t p0 = kP[0], p1 = kP[1];

#pragma unroll 1
    for (int i = 0; i < kn; ++i) {
        const uint32_t ab = abar[i];
        // Rotate, subtract, decompose into 6 digit polynomials (row r = 2(p-1)+q),
        // digit + 64 packed four per word; lane L owns coefficients L + 32m,
        // which are exactly the points it feeds into the forward transforms,
        // so the digits stay in its Tensor Memory lane.
        {
            uint32_t packed[kRows * 8];
#pragma unroll
            for (int w = 0; w < kRows * 8; ++w) packed[w] = 0u;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const int k = lane + 32 * m;
                const uint32_t src = ((uint32_t)k - ab) & (kTwoN - 1);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t *a = acc + q * kN;
                    uint32_t v = a[src & (kN - 1)];
                    if (src >= (uint32_t)kN) v = 0u - v;
                    const uint32_t y = v - a[k] + kOff;
                    const int sh = 8 * (m & 3), w = m >> 2;
                    packed[(0 * 2 + q) * 8 + w] |= field7(y, 25, sh);
                    packed[(1 * 2 + q) * 8 + w] |= field7(y, 18, sh);
                    packed[(2 * 2 + q) * 8 + w] |= field7(y, 11, sh);
                }
            }
            tmem_st16(tdig, packed);
            tmem_st16(tdig + 16, packed + 16);
            tmem_st16(tdig + 32, packed + 32);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        __syncwarp();

#pragma unroll 1
        for (int pi = 0; pi < 2; ++pi) {
            const uint32_t p = pi ? p1 : p0;
            const uint32_t pinv = pi ? 22u : 25u;                     // floor(2^32 / p)
            uint32_t a0[32], a1[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) { a0[t] = 0u; a1[t] = 0u; }
            uint32_t dw[8];
            tmem_ld8(tdig, dw);
#pragma unroll 1
            for (int r = 0; r < kRows; ++r) {
                uint32_t x[32];
                // stages 0 and 1 by lookups.  For u < 8, with bytes b_j of
                // digits j = u, u+8, u+16, u+24: stage 0 gives s = x_u +
                // psi^512 d_{u+16} and s' = x_u - psi^512 d_{u+16}; stage 1
                // pairs (u, u+8) with psi^256 and (u+16, u+24) with psi^768,
                // whose products are psi^256 d_{u+8} + psi^768 d_{u+24} and
                // psi^768 d_{u+8} + psi^256 d_{u+24}.  Outputs below 6p, as
                // two multiplying stages give.
                const uint32_t *T0 = S.tab[pi][0], *Ua = S.tab[pi][1], *Ub = S.tab[pi][2];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t b0 = __byte_perm(dw[u >> 2], 0u, 0x4440u | (u & 3));
                    const uint32_t b8 = __byte_perm(dw[(u + 8) >> 2], 0u, 0x4440u | (u & 3));
                    const uint32_t b16 = __byte_perm(dw[(u + 16) >> 2], 0u, 0x4440u | (u & 3));
                    const uint32_t b24 = __byte_perm(dw[(u + 24) >> 2], 0u, 0x4440u | (u & 3));
                    const uint32_t xv = b0 + (p - 64u), t0 = T0[b16];
                    const uint32_t s0 = xv + t0, s1 = xv - t0 + 2 * p;
                    const uint32_t m0 = Ua[b8] + Ub[b24], m1 = Ub[b8] + Ua[b24];
                    x[u] = s0 + m0;
                    x[u + 8] = s0 - m0 + 2 * p;
                    x[u + 16] = s1 + m1;
                    x[u + 24] = s1 - m1 + 2 * p;
                }
                // the next row's digits arrive while this row is transformed
                if (r + 1 < kRows) tmem_ld8_async(tdig + 8 * (r + 1), dw);
                ntt_fwd<2>(x, pi, xch, lane, S.twl[pi][0]);
                const int c = (i * 2 + pi) * kRows + r;               // chunk of the key stream
                const int slot = c % kRing;
                mbar_wait(&S.full[slot], (uint32_t)((c / kRing) & 1), err);
                const uint4 *kv = reinterpret_cast<const uint4 *>(S.ring[slot]) + lane;   // (w0, w0', w1, w1')
                // Lazy accumulation: each product is below 2p, the six-row sums
                // below 12p < 2^32.
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const uint4 v = kv[32 * t];
                    a0[t] += mul_shoup(x[t], v.x, v.y, p);
                    a1[t] += mul_shoup(x[t], v.z, v.w, p);
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&S.empty[slot]);
                    if (warp == 0 && c + kRing < kChunks &&
                        mbar_wait(&S.empty[slot], (uint32_t)((c / kRing) & 1), err))
                        load_chunk(S.ring[slot], bkhat + (size_t)(c + kRing) * kChunkWords, &S.full[slot]);
                }
                __syncwarp();
                tmem_wait_ld();
            }
#pragma unroll
            for (int t = 0; t < 32; ++t) { a0[t] = red_shoup(a0[t], pinv, p); a1[t] = red_shoup(a1[t], pinv, p); }
            ntt_inv2(a0, a1, pi, xch, lane, S.twl[pi][1]);
            if (pi == 0) {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    a0[t] = red2(red_shoup(a0[t], pinv, p), p);
                    a1[t] = red2(red_shoup(a1[t], pinv, p), p);
                }
                tmem_st32(tres, a0);
                tmem_st32(tres + 32, a1);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            } else {
                // CRT: v = x0 + p0 * t, t = (x1 - x0) p0^-1 mod p1, is the product
                // coefficient in [0, P).  Its exact value has magnitude below
                // 6 * N * 64 * 2^32 < 2^50.6, so t < 2^50.6 / p0 < 2^23.3 when it
                // is non-negative and t > p1 - 2^23.3 when it is negative: it is
                // negative exactly when t > p1 / 2 (2^26.5), and then v - P is
                // taken.  Only v mod 2^32 is needed.
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint32_t x0v[32];
                    tmem_ld32(tres + 32 * j, x0v);
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const int k = lane + 32 * t;
                        const uint32_t x0 = x0v[t];                       // < p0
                        const uint32_t x1 = j ? a1[t] : a0[t];            // < 4 p1: x1 - x0 + p1 < 2^32
                        const uint32_t tq = red2(mul_shoup(x1 - x0 + p1, cP.crt_inv, cP.crt_inv_s, p1), p1);
                        const uint32_t lo = x0 + p0 * tq - (tq > (p1 >> 1) ? kPmod32 : 0u);
                        acc[j * kN + k] += lo;
                    }
                }
            }
        }
        __syncwarp();
    }

    // Sample extract: a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0.
    uint32_t *row = big + (size_t)J.big * kBigWords;
    for (int k = lane; k < kN; k += 32) row[k == 0 ? 0 : kN - k] = k == 0 ? acc[0] : 0u - acc[k];
    if (lane == 0) row[kN] = acc[kN];

    // Copies still in flight after a timed-out wait must land before the
    // shared memory is released.
    if (warp == 0 && lane == 0 && *reinterpret_cast<volatile int *>(err) != kDevOk)
        for (int r = 0; r < kRing; ++r) mbar_drain(&S.full[r], 0u), mbar_drain(&S.full[r], 1u);

    // All active compute warps are done with Tensor Memory: warp 0 frees it.
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, %0;" ::"r"(nact * 32) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// One warp per (step, prime, row, component): reduce the BK polynomial mod p,
// transform it with the same forward NTT, fold N^-1, and store the values and
// their Shoup companions in the order the pointwise stage reads (index
// t*32 + lane for transform point 32*lane + t) inside the chunk of its
// (step, prime, row).
__global__ void __launch_bounds__(128) bk_ntt_kernel(const uint32_t *__restrict__ bk, uint32_t *__restrict__ out)
{
    __shared__ __align__(16) uint32_t xch[4][kXch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t id = (size_t)blockIdx.x * 4 + warp;       // ((i * 2 + pi) * 6 + r) * 2 + j
    if (id >= (size_t)kChunks * 2) return;
    const int j = (int)(id % 2);
    const int r = (int)((id / 2) % kRows);
    const int pi = (int)((id / (2 * kRows)) % 2);
    const size_t i = id / (2 * kRows * 2);
    const uint32_t p = kP[0] + (uint32_t)pi * (kP[1] - kP[0]);
    const uint32_t *src = bk + ((i * kRows + r) * 2 + j) * kN;
    uint32_t x[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) x[t] = src[lane + 32 * t] % p;
    ntt_fwd<0>(x, pi, xch[warp], lane, gWL[pi][0]);
    // chunk layout: [t][lane][w0, w0', w1, w1'] for transform point 32*lane + t
    uint32_t *dst = out + (id / 2) * kChunkWords + (size_t)j * 2;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint32_t v = (uint32_t)(((unsigned long long)(x[t] % p) * cP.scale[pi]) % p);
        dst[(t * 32 + lane) * 4] = v;
        dst[(t * 32 + lane) * 4 + 1] = (uint32_t)(((unsigned long long)v << 32) / p);
    }
}

uint32_t powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return (uint32_t)r;
}

int brv10(int k)
{
    int r = 0;
    for (int b = 0; b < 10; ++b) r |= ((k >> b) & 1) << (9 - b);
    return r;
}

bool g_tables_ready[64] = {false};

int upload_tables()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_tables_ready[dev]) return 0;
    static uint32_t W[2][2][kN], Ws[2][2][kN];
    PrimeConsts pc{};
    for (int pi = 0; pi < 2; ++pi) {
        const uint64_t p = kP[pi];
        const uint32_t psi = powmod(3, (p - 1) / kTwoN, p);      // 3 generates Z_p^* for both primes
        if (powmod(psi, kN, p) != p - 1) return -1;              // psi must be a primitive 2N-th root
        const uint32_t ipsi = powmod(psi, p - 2, p);
        for (int k = 0; k < kN; ++k) {
            W[pi][0][k] = powmod(psi, brv10(k), p);
            W[pi][1][k] = powmod(ipsi, brv10(k), p);
            for (int d = 0; d < 2; ++d) Ws[pi][d][k] = (uint32_t)(((uint64_t)W[pi][d][k] << 32) / p);
        }
        pc.p[pi] = (uint32_t)p;
        pc.scale[pi] = powmod(kN, p - 2, p);
    }
    pc.crt_inv = powmod(kP[0], kP[1] - 2, kP[1]);
    pc.crt_inv_s = (uint32_t)(((uint64_t)pc.crt_inv << 32) / kP[1]);
    static uint2 Wp[2][2][kN];
    for (int pi = 0; pi < 2; ++pi)
        for (int d = 0; d < 2; ++d)
            for (int k = 0; k < kN; ++k) Wp[pi][d][k] = make_uint2(W[pi][d][k], Ws[pi][d][k]);
    if (cudaMemcpyToSymbol(cWp, Wp, sizeof Wp) != cudaSuccess) return -1;
    static uint2 WL[2][2][kTwLane];
    for (int pi = 0; pi < 2; ++pi)
        for (int L = 0; L < 32; ++L) {
            for (int s = 5, base = 0; s < 10; base += 32 << (s - 5), ++s)          // forward, after the transpose
                for (int g = 0; g < (1 << (s - 5)); ++g) {
                    const int k = (1 << s) + (L << (s - 5)) + g;
                    WL[pi][0][base + g * 32 + L] = make_uint2(W[pi][0][k], Ws[pi][0][k]);
                }
            for (int k5 = 0, base = 0; k5 < 5; base += 32 * (16 >> k5), ++k5)       // inverse, before the transpose
                for (int g = 0; g < (16 >> k5); ++g) {
                    const int k = (512 >> k5) + (L << (4 - k5)) + g;
                    WL[pi][1][base + g * 32 + L] = make_uint2(W[pi][1][k], Ws[pi][1][k]);
                }
        }
    if (cudaMemcpyToSymbol(gWL, WL, sizeof WL) != cudaSuccess) return -1;
    // psi^512, psi^256, psi^768 are the forward twiddles of stage 0 (k = 1)
    // and stage 1 (k = 2, 3): psi^brv10(k)
    static uint32_t Tab[2][3][128];
    for (int pi = 0; pi < 2; ++pi)
        for (int w = 0; w < 3; ++w)
            for (int b = 0; b < 128; ++b)
                Tab[pi][w][b] = (uint32_t)(((uint64_t)W[pi][0][w + 1] * (uint64_t)((b - 64 + (int64_t)kP[pi]) % kP[pi])) %
                                           kP[pi]);
    if (cudaMemcpyToSymbol(gTab, Tab, sizeof Tab) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(cP, &pc, sizeof pc) != cudaSuccess) return -1;
    if (dev >= 0 && dev < 64) g_tables_ready[dev] = true;
    return 0;
}

template <int W> int configure_w()
{
    return cudaFuncSetAttribute(br_ntt_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Smem<W>)) == cudaSuccess ? 0 : -1;
}

template <int W> void launch_w(const BrJob *jobs, int njobs, int per, const uint32_t *bk_ntt, uint32_t *big,
                               int *err, cudaStream_t st)
{
    br_ntt_kernel<W><<<(njobs + per - 1) / per, W * 32, sizeof(Smem<W>), st>>>(jobs, njobs, per, bk_ntt, big, err);
}

// Tuned per-wave time of each variant (ms for one full wave of 152 CTAs);
// zero until velopir's autotuner has measured it.
float g_wave_ms[kMaxWarps + 1] = {0};
static_assert(sizeof(Smem<kMaxWarps>) <= 232448, "shared memory per CTA");
static_assert(3 * kTmemWarpCols <= kTmemCols, "Tensor Memory per CTA");
int g_sms = 0;

}  // namespace

size_t bk_ntt_words() { return kBkNttWords; }

int prepare_bk_ntt(const uint32_t *bk, uint32_t *bk_ntt, cudaStream_t st)
{
    if (upload_tables() != 0) return 0;
    const size_t warps = (size_t)kChunks * 2;
    bk_ntt_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(bk, bk_ntt);
    return 1;
}

// Raise the dynamic shared-memory limit once per process (outside any stream capture).
int configure_br_ntt()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    return (configure_w<6>() | configure_w<8>() | configure_w<9>() | configure_w<10>() | configure_w<12>()) ? -1 : 0;
}

int ntt_shape_count() { return 5; }

// Blind rotations in one full wave of the most efficient tuned shape (the
// least wave time per bootstrap), or 0 before the autotuner has run.
int ntt_full_wave()
{
    const int sms = g_sms > 0 ? g_sms : 152;
    int best = 0;
    for (int i = 0; i < (int)(sizeof(kShapes) / sizeof(kShapes[0])); ++i) {
        const int w = kShapes[i];
        if (g_wave_ms[w] <= 0) return 0;
        if (best == 0 || g_wave_ms[w] / w < g_wave_ms[best] / best) best = w;
    }
    return sms * best;
}
int ntt_shape(int i) { return kShapes[i]; }
void ntt_set_wave_ms(int warps, float ms) { if (warps >= 1 && warps <= kMaxWarps) g_wave_ms[warps] = ms; }

// Bootstraps per CTA for a launch of njobs: the shape with the smallest
// (waves x tuned wave time); without tuning, the largest CTA.
int ntt_pick_warps(int njobs)
{
    int best = kMaxWarps;
    double best_t = 0;
    const int sms = g_sms > 0 ? g_sms : 152;
    for (int i = 0; i < 5; ++i) {
        const int w = kShapes[i];
        if (g_wave_ms[w] <= 0) return kMaxWarps;
        const int ctas = (njobs + w - 1) / w;
        const double t = (double)((ctas + sms - 1) / sms) * g_wave_ms[w];
        if (i == 0 || t < best_t) { best = w; best_t = t; }
    }
    return best;
}

namespace {

// The tuned shape with the shortest wave time among those holding b
// bootstraps per CTA (a partly filled CTA runs about as long as a full one).
int shape_for(int b)
{
    int best = -1;
    for (int i = 0; i < 5; ++i) {
        const int w = kShapes[i];
        if (w >= b && (best < 0 || g_wave_ms[w] < g_wave_ms[best])) best = w;
    }
    return best < 0 ? kMaxWarps : best;
}

// Wave plan of a launch: the per-SM load L = ceil(njobs / SMs) is split into
// waves of b_i bootstraps per CTA (sum b_i = L), minimising the sum of the
// tuned wave times of the shapes that hold them.  A wave of b per CTA costs
// about the wave time of its shape whether or not the shape is full, because
// each warp runs at a latency-bound speed; the plan therefore prefers full
// 12-wide waves and covers the remainder with waves that keep at most two
// warps per SM sub-partition.
struct Wave { int shape, per; };

const std::vector<Wave> &plan_waves(int njobs)
{
    static std::vector<std::pair<int, std::vector<Wave>>> cache;
    for (auto &e : cache)
        if (e.first == njobs) return e.second;
    const int sms = g_sms > 0 ? g_sms : 152;
    const int L = (njobs + sms - 1) / sms;
    std::vector<double> cost(L + 1, 0.0);
    std::vector<int> choice(L + 1, 0);
    for (int l = 1; l <= L; ++l) {
        cost[l] = -1;
        for (int b = 1; b <= kMaxWarps && b <= l; ++b) {
            const double c = cost[l - b] + g_wave_ms[shape_for(b)];
            if (cost[l] < 0 || c < cost[l] - 1e-9) { cost[l] = c; choice[l] = b; }
        }
    }
    std::vector<Wave> plan;
    for (int l = L; l > 0; l -= choice[l]) plan.push_back({shape_for(choice[l]), choice[l]});
    std::sort(plan.begin(), plan.end(), [](const Wave &a, const Wave &b) { return a.per > b.per; });
    if (cache.size() > 256) cache.clear();
    cache.emplace_back(njobs, plan);
    return cache.back().second;
}

}  // namespace

int launch_br_ntt_w(const BrJob *jobs, int njobs, const uint32_t *bk_ntt, uint32_t *big, int *err, cudaStream_t st,
                    int warps, int per)
{
    if (njobs <= 0) return 0;
    if (per <= 0 || per > warps) per = warps;
    switch (warps) {
    case 6: launch_w<6>(jobs, njobs, per, bk_ntt, big, err, st); break;
    case 8: launch_w<8>(jobs, njobs, per, bk_ntt, big, err, st); break;
    case 9: launch_w<9>(jobs, njobs, per, bk_ntt, big, err, st); break;
    case 10: launch_w<10>(jobs, njobs, per, bk_ntt, big, err, st); break;
    default: launch_w<12>(jobs, njobs, per, bk_ntt, big, err, st); break;
    }
    return 1;
}

int launch_br_ntt(const BrJob *jobs, int njobs, const uint32_t *bk_ntt, uint32_t *big, int *err, cudaStream_t st)
{
    if (njobs <= 0) return 0;
    for (int i = 0; i < 5; ++i)
        if (g_wave_ms[kShapes[i]] <= 0)   // not tuned: one launch of the widest shape
            return launch_br_ntt_w(jobs, njobs, bk_ntt, big, err, st, kMaxWarps, kMaxWarps);
    const int sms = g_sms > 0 ? g_sms : 152;
    int launches = 0, off = 0;
    for (const Wave &w : plan_waves(njobs)) {
        if (off >= njobs) break;
        const int n = std::min(njobs - off, sms * w.per);
        launches += launch_br_ntt_w(jobs + off, n, bk_ntt, big, err, st, w.shape, w.per);
        off += n;
    }
    return launches;
}

}  // namespace vp
