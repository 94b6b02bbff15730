// Blind rotation with the external product on the 5th-generation tensor cores
// (tcgen05.mma .kind::f16), exact by construction.
//
// Per step i the product out_j[m] = sum_{r,k} T_{r,j}[m][k] d_r[k] (paper
// Section 2.2's gate bootstrap; the CMux step of tfhe-2) is a dense
// contraction of the negacyclic Toeplitz matrices of the key rows
// (T[m][k] = BK[m-k], or -BK[m-k+N] when m < k) with the digit polynomials.
// It is evaluated exactly in floating point:
//   * every key word is split into four balanced 8-bit limbs b_l in
//     [-128, 127] with sum_l b_l 2^(8l) = BK (mod 2^32); limbs and digits
//     (|d| <= 64) are integers that fp16 holds exactly;
//   * one digit row contributes 1024 products of magnitude <= 2^13 to an
//     output, so each fp32 accumulator holds an integer of magnitude
//     <= 2^23, exactly;
//   * per row the four limb accumulators are read from Tensor Memory,
//     converted to integers and combined as sum_l S_l << 8l mod 2^32.
// The result equals the integer contraction mod 2^32, bit for bit.
//
// Operand layout.  Reversing the digit order (k' = N-1-k) turns the Toeplitz
// matrix into a Hankel matrix, A[m][k'] = u[m + k'] with
// u[e] = T-entry for m - k = e - (N-1).  Stored as "8-way shifted" rows --
// group g holds the 8 rows u[8g + rr .. 8g + rr + 7], rr < 8, 128 bytes --
// the core matrix of rows 8a.. and columns 8b.. is group a + b, so one
// K-major descriptor without swizzling whose leading and stride byte offsets
// are both 128 walks the whole Hankel matrix: no Toeplitz tile is ever
// materialised.  The expanded key is built once per key on the device.
//
// Structure per blind-rotation step (one launch pair per step):
//   tc_digits_kernel: ACC of each bootstrap (global, L2-resident) ->
//     X^abar ACC - ACC -> six digit rows, reversed, as fp16 in the K-major
//     core-matrix layout of the MMA's B operand;
//   tc_mma_kernel: CTA = (128 output coefficients, 128 bootstraps).  Warp 0
//     streams key windows and digit blocks into a five-stage ring with bulk
//     asynchronous copies; warp 1 issues the MMAs (M = 128 coefficients,
//     N = 128 bootstraps, K = 16) into four limb accumulators (512 Tensor
//     Memory columns); warps 2-5 read each row's accumulators, combine the
//     limbs and keep the integer sums in shared memory; at the end they add
//     them into ACC.
// Every mbarrier wait is bounded (kWaitNs) and records a timeout in the
// error word instead of spinning.
#include "vp_internal.h"

#include <cuda_fp16.h>

namespace vp {
namespace {

constexpr int kLimbs = 4;
constexpr int kGroups = 256;                       // Hankel groups of one (step, row, limb, comp) (2N entries / 8)
constexpr int kGroupHalves = 64;                   // 8 rows x 8 fp16
constexpr size_t kTcPolyHalves = (size_t)kGroups * kGroupHalves;   // 32 KB
// expanded key: [step][row][limb][comp][group][8][8] fp16
constexpr size_t kBkTcHalves = (size_t)kn * kRows * kLimbs * 2 * kTcPolyHalves;

constexpr int TM = 128;                            // output coefficients per CTA (MMA M)
constexpr int TN = 128;                            // bootstraps per CTA (MMA N)
constexpr int KB = 64;                             // K per pipeline stage (4 MMAs of K = 16)
constexpr int KBLOCKS = kN / KB;                   // 16 stages per digit row
constexpr int AWIN = (TM + KB) / 8;                // 24 Hankel groups per (limb, stage)
constexpr int ABYTES = AWIN * 128;                 // 3 KB
constexpr int BBYTES = TN * KB * 2;                // 16 KB: 128 bootstraps x 64 digits
constexpr int kStages = 5;                         // ring depth: hides the L2 latency of a 28 KB stage behind 4 stages of MMAs
constexpr uint32_t kTmemCols = 512;                // 4 limbs x 128 bootstraps

// Digits in global memory: [tile of 128 bootstraps][row][k' group (128)][n group (16)][8 n][8 k'] fp16, so
// that the 64-digit block kb of a row is one contiguous 16 KB range laid out
// exactly as the B operand wants it in shared memory.
constexpr size_t kDigTileHalves = (size_t)kRows * kN * TN;

struct __align__(1024) MmaSmem;
static_assert(kStages * (BBYTES + kLimbs * ABYTES) + TN * TM * 4 + 1024 <= 232448, "shared memory per CTA");

struct __align__(1024) MmaSmem {
    __half b[kStages][TN * KB];                    // 80 KB; placed first so that any descriptor read of it stays inside the block
    __half a[kStages][kLimbs][AWIN * 64];          // 60 KB
    uint32_t part[TN * TM];                        // 64 KB: integer sums, [bootstrap][coefficient]
    unsigned long long full[kStages], empty[kStages], acc_full, acc_empty;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

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

// Bounded wait: false (and the error word set) after kWaitNs, or at once if
// an earlier wait of this launch already gave up.
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

__device__ __forceinline__ void mbar_drain(unsigned long long *bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try(bar, parity) && global_ns() - t0 <= kWaitNs) {
    }
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzling: start address,
// leading (K-direction) and stride (M/N-direction) byte offsets between 8x16-byte
// core matrices, all in units of 16 bytes; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D fp32, A and B fp16, both K-major, N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
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

// Balanced base-256 limb l of a 32-bit word (limb 3 absorbs the carry mod 2^32).
__device__ __forceinline__ int limb_of(uint32_t v, int l)
{
    int64_t x = (int64_t)v;
    int d = 0;
    for (int i = 0; i <= l; ++i) {
        d = (int)(((x + 128) & 255) - 128);
        x = (x - d) >> 8;
    }
    return d;
}

// One thread per (step, row, limb, comp, group, rr): 8 fp16 of the expanded
// Hankel key, u[8g + rr + c] for c < 8, with u[e] the Toeplitz entry of
// m - k = e - (N-1) (negated when it wraps) and u[2N-1] = 0.
__global__ void bk_tc_kernel(const uint32_t *__restrict__ bk, __half *__restrict__ out)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // ((((i*6+r)*4+l)*2+j)*256+g)*8+rr
    if (id >= kBkTcHalves / 8) return;
    const int rr = (int)(id % 8);
    const int g = (int)((id / 8) % kGroups);
    const int j = (int)((id / (8 * kGroups)) % 2);
    const int l = (int)((id / (16 * kGroups)) % kLimbs);
    const size_t ir = id / (16 * kGroups * kLimbs);                   // i * 6 + r
    const uint32_t *row = bk + (ir * 2 + (size_t)j) * kN;
    __align__(16) __half h[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int e = 8 * g + rr + c - (kN - 1);   // m - k
        uint32_t v = 0u;
        if (e >= 0 && e < kN) v = row[e];
        else if (e < 0 && e > -kN) v = 0u - row[e + kN];
        h[c] = __int2half_rn(limb_of(v, l));
    }
    *reinterpret_cast<uint4 *>(out + id * 8) = *reinterpret_cast<const uint4 *>(h);
}

// Gate pre-combination, modulus switch and ACC = (0, X^{-bbar} v) for each
// bootstrap; one warp per bootstrap.
__global__ void tc_prologue_kernel(const BrJob *__restrict__ jobs, int njobs, uint16_t *__restrict__ abar,
                                   uint32_t *__restrict__ acc)
{
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (b >= njobs) return;
    const BrJob J = jobs[b];
    uint16_t *ab = abar + (size_t)b * kSlotWords;
    for (int i = lane; i < kLweWords; i += 32) {
        uint32_t c = (i == kn) ? J.cst : 0u;
        if (J.in0) c += (uint32_t)J.s0 * J.in0[i];
        if (J.in1) c += (uint32_t)J.s1 * J.in1[i];
        ab[i] = (uint16_t)((c + (1u << 20)) >> 21);
    }
    __syncwarp();
    const uint32_t bbar = ab[kn] & (kTwoN - 1);
    uint32_t *a = acc + (size_t)b * kTwoN;
    for (int k = lane; k < kN; k += 32) {
        const uint32_t u = ((uint32_t)k + bbar) & (kTwoN - 1);
        a[k] = 0u;
        a[kN + k] = (u < (uint32_t)kN) ? kMu : (0u - kMu);
    }
}

// Step i: the six reversed digit rows of each bootstrap, fp16, in the B
// operand layout.  One CTA of 128 threads per bootstrap; thread t owns the 8
// reversed positions k' = 8t .. 8t + 7 (coefficients k = N-1-k').
__global__ void __launch_bounds__(128) tc_digits_kernel(int step, int njobs, const uint16_t *__restrict__ abar,
                                                        const uint32_t *__restrict__ acc, __half *__restrict__ dig)
{
    __shared__ uint32_t a[kTwoN];
    const int b = blockIdx.x, t = threadIdx.x;
    if (b >= njobs) return;
    const uint32_t *src = acc + (size_t)b * kTwoN;
    for (int k = t; k < kTwoN / 4; k += 128) reinterpret_cast<uint4 *>(a)[k] = reinterpret_cast<const uint4 *>(src)[k];
    __syncthreads();
    const uint32_t ab = abar[(size_t)b * kSlotWords + step] & (kTwoN - 1);
    constexpr uint32_t kOff = (1u << 31) + (1u << 24) + (1u << 17) + (1u << 10);
    __align__(16) __half h[kRows][8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int k = kN - 1 - (8 * t + c);
        const uint32_t s = ((uint32_t)k - ab) & (kTwoN - 1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            uint32_t v = a[q * kN + (s & (kN - 1))];
            if (s >= (uint32_t)kN) v = 0u - v;
            const uint32_t y = v - a[q * kN + k] + kOff;
#pragma unroll
            for (int p = 1; p <= kL; ++p)
                h[2 * (p - 1) + q][c] = __int2half_rn((int)((y >> (32 - kBgBits * p)) & 127u) - 64);
        }
    }
    // [tile][row][k' group][n group][8 n][8 k']
    const size_t tile = (size_t)(b / TN);
    const int n = b % TN;
    __half *base = dig + tile * kDigTileHalves + (size_t)(n / 8) * 64 + (size_t)(n % 8) * 8;
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        *reinterpret_cast<uint4 *>(base + ((size_t)r * (kN / 8) + t) * (TN / 8) * 64) =
            *reinterpret_cast<const uint4 *>(h[r]);
}

// Step i of the external product for one (coefficient tile, bootstrap tile).
// blockIdx.x = mtile (0..15: component j = mtile / 8, coefficients 128 (mtile % 8) ..),
// blockIdx.y = bootstrap tile.  ACC += sum_r T(BK_i[r][j]) d_r, exactly.
__global__ void __launch_bounds__(192, 1) tc_mma_kernel(int step, int njobs, const __half *__restrict__ bktc,
                                                         const __half *__restrict__ dig, uint32_t *__restrict__ acc,
                                                         int *err)
{
    extern __shared__ unsigned char smem_raw[];
    MmaSmem &S = *reinterpret_cast<MmaSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x, j = mtile / 8, m0 = (mtile % 8) * TM;
    const int tile = blockIdx.y;
    const int nact = min(TN, njobs - tile * TN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.acc_full, 1);
        mbar_init(&S.acc_empty, 128);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int x = threadIdx.x; x < TN * TM; x += blockDim.x) S.part[x] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    constexpr int kIters = kRows * KBLOCKS;   // 96 pipeline stages per step
    const __half *dtile = dig + (size_t)tile * kDigTileHalves;
    if (warp == 0) {
        if (lane == 0) {
            for (int it = 0; it < kIters; ++it) {
                const int s = it % kStages, r = it / KBLOCKS, kb = it % KBLOCKS;
                if (it >= kStages && !mbar_wait(&S.empty[s], (uint32_t)(((it / kStages) - 1) & 1), err)) break;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.full[s])),
                             "r"((uint32_t)(kLimbs * ABYTES + BBYTES))
                             : "memory");
                bulk_load(S.b[s], dtile + ((size_t)r * kN + (size_t)kb * KB) * TN, BBYTES, &S.full[s]);
                for (int l = 0; l < kLimbs; ++l) {
                    const __half *poly = bktc + ((((size_t)step * kRows + r) * kLimbs + l) * 2 + j) * kTcPolyHalves;
                    bulk_load(S.a[s][l], poly + (size_t)(m0 / 8 + kb * (KB / 8)) * kGroupHalves, ABYTES, &S.full[s]);
                }
            }
            // the last MMAs' arrivals on the ring must land before the CTA exits
            for (int it = kIters - kStages; it < kIters; ++it)
                mbar_drain(&S.empty[it % kStages], (uint32_t)((it / kStages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t tmem = S.tmem_base;
            for (int it = 0; it < kIters; ++it) {
                const int s = it % kStages, r = it / KBLOCKS, kb = it % KBLOCKS;
                if (kb == 0 && r > 0) {   // the epilogue has read the previous row's accumulators
                    if (!mbar_wait(&S.acc_empty, (uint32_t)((r - 1) & 1), err)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                if (!mbar_wait(&S.full[s], (uint32_t)((it / kStages) & 1), err)) break;
                const uint32_t bb = smem_u32(S.b[s]);
#pragma unroll
                for (int l = 0; l < kLimbs; ++l) {
                    const uint32_t ab = smem_u32(S.a[s][l]);
#pragma unroll
                    for (int ks = 0; ks < KB / 16; ++ks) {
                        // A: Hankel window, core matrix (a, b) at group a + b (LBO = SBO = 128 B);
                        // B: [k' group][n group][8][8], K-adjacent core matrices TN/8 x 128 B apart.
                        const uint64_t ad = smem_desc(ab + (uint32_t)(2 * ks) * 128u, 128u, 128u);
                        const uint64_t bd = smem_desc(bb + (uint32_t)(2 * ks) * (TN / 8) * 128u, (TN / 8) * 128u, 128u);
                        mma_f16(tmem + (uint32_t)(l * TN), ad, bd, (kb > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&S.empty[s]);
                if (kb == KBLOCKS - 1) mma_commit(&S.acc_full);
            }
        }
    } else {
        // epilogue: warp w reads lane quarter w % 4, i.e. coefficients 32 (w % 4) .. + 31
        const int q = warp & 3, m = 32 * q + lane;
        const uint32_t trow = S.tmem_base + ((uint32_t)(32 * q) << 16);
        for (int r = 0; r < kRows; ++r) {
            if (!mbar_wait(&S.acc_full, (uint32_t)(r & 1), err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int cb = 0; cb < TN / 32; ++cb) {
                uint32_t sum[32];
#pragma unroll
                for (int x = 0; x < 32; ++x) sum[x] = 0u;
#pragma unroll
                for (int l = 0; l < kLimbs; ++l) {
                    uint32_t v[32];
                    tmem_ld32(trow + (uint32_t)(l * TN + 32 * cb), v);
#pragma unroll
                    for (int x = 0; x < 32; ++x)
                        sum[x] += (uint32_t)__float2int_rn(__uint_as_float(v[x])) << (8 * l);
                }
#pragma unroll
                for (int x = 0; x < 32; ++x) S.part[(32 * cb + x) * TM + m] += sum[x];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&S.acc_empty);
        }
        // ACC_j[m0 + m] += the step's product, for each bootstrap of the tile:
        // 16 loads in flight at a time instead of one read-modify-write per
        // L2 round trip
        uint32_t *col = acc + ((size_t)tile * TN) * kTwoN + (size_t)j * kN + m0 + m;
        for (int n0 = 0; n0 < nact; n0 += 16) {
            uint32_t v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (n0 + k < nact) v[k] = __ldcg(col + (size_t)(n0 + k) * kTwoN);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (n0 + k < nact) __stcg(col + (size_t)(n0 + k) * kTwoN, v[k] + S.part[(n0 + k) * TM + m]);
        }
    }

    // Copies in flight after a timed-out wait must land before the shared
    // memory is released.
    if (threadIdx.x == 0 && *reinterpret_cast<volatile int *>(err) != kDevOk)
        for (int s = 0; s < kStages; ++s) mbar_drain(&S.full[s], 0u), mbar_drain(&S.full[s], 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// Sample extract: a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0.
__global__ void tc_extract_kernel(const BrJob *__restrict__ jobs, int njobs, const uint32_t *__restrict__ acc,
                                  uint32_t *__restrict__ big)
{
    const int b = blockIdx.x;
    if (b >= njobs) return;
    const uint32_t *a = acc + (size_t)b * kTwoN;
    uint32_t *row = big + (size_t)jobs[b].big * kBigWords;
    for (int k = threadIdx.x; k < kN; k += blockDim.x) row[k == 0 ? 0 : kN - k] = k == 0 ? a[0] : 0u - a[k];
    if (threadIdx.x == 0) row[kN] = a[kN];
}

}  // namespace

size_t bk_tc_bytes() { return kBkTcHalves * sizeof(__half); }

int prepare_bk_tc(const uint32_t *bk, void *bk_tc, cudaStream_t st)
{
    const size_t threads = kBkTcHalves / 8;
    bk_tc_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(bk, reinterpret_cast<__half *>(bk_tc));
    return 1;
}

// Scratch of a launch of njobs bootstraps: ACC (8 KB each), the modulus-switched
// inputs and the digit rows of the padded tiles.
size_t tc_scratch_bytes(int njobs)
{
    const size_t tiles = ((size_t)njobs + TN - 1) / TN;
    return (size_t)njobs * kTwoN * 4 + (size_t)njobs * kSlotWords * 2 + tiles * kDigTileHalves * 2 + 1024;
}

int configure_br_tc()
{
    return cudaFuncSetAttribute(tc_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MmaSmem)) ==
                   cudaSuccess
               ? 0
               : -1;
}

int launch_br_tc(const BrJob *jobs, int njobs, const void *bk_tc, void *scratch, uint32_t *big, int *err,
                 cudaStream_t st)
{
    if (njobs <= 0) return 0;
    const size_t tiles = ((size_t)njobs + TN - 1) / TN;
    unsigned char *p = reinterpret_cast<unsigned char *>(scratch);
    uint32_t *acc = reinterpret_cast<uint32_t *>(p);
    p += (size_t)njobs * kTwoN * 4;
    __half *dig = reinterpret_cast<__half *>(p);
    p += tiles * kDigTileHalves * 2;
    uint16_t *abar = reinterpret_cast<uint16_t *>(p);
    int launches = 0;
    tc_prologue_kernel<<<(njobs + 3) / 4, 128, 0, st>>>(jobs, njobs, abar, acc);
    ++launches;
    // the padding bootstraps of the last tile read zero digits
    if (tiles * TN > (size_t)njobs) cudaMemsetAsync(dig, 0, tiles * kDigTileHalves * 2, st);
    const __half *key = reinterpret_cast<const __half *>(bk_tc);
    const dim3 grid(16, (unsigned)tiles);
    for (int i = 0; i < kn; ++i) {
        tc_digits_kernel<<<njobs, 128, 0, st>>>(i, njobs, abar, acc, dig);
        tc_mma_kernel<<<grid, 192, sizeof(MmaSmem), st>>>(i, njobs, key, dig, acc, err);
        launches += 2;
    }
    tc_extract_kernel<<<njobs, 128, 0, st>>>(jobs, njobs, acc, big);
    return launches + 1;
}

}  // namespace vp
