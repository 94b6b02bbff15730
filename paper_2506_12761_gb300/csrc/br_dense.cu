// Blind rotation with the external product computed as a dense negacyclic
// contraction on the integer pipe (exact uint32 arithmetic).
//
// Bootstrap = BlindRotate -> SampleExtract -> KeySwitch (paper Section 2.2;
// internals from tfhe-2).  Per blind-rotation step i (n = 630 steps):
//   Delta = X^abar_i * ACC - ACC                       (negacyclic rotation)
//   d_{p,q} = balanced base-2^7 digits of Delta_q    (l = 3 levels, q = a, b)
//   ACC_j += sum_{p,q} d_{p,q}(X) * BK_i[2(p-1)+q][j](X)  mod (X^N+1, 2^32)
// One CTA owns 8 bootstraps for all 630 steps: they share each step's 48 KB
// BK_i, staged into shared memory by a bulk asynchronous copy completing on
// an mbarrier.  Each thread keeps 8 coefficients x 4 bootstraps x 2
// polynomials of ACC in registers and accumulates its slice of the product
// out_j[k] = sum_m BK[r][j][m] * D'_r[k - m], where D' is the digit polynomial
// extended negacyclically (D'[x] = -D[x+N] for x < 0), stored once per step
// as int8 so that the Toeplitz window slides through shared memory.
#include "vp_internal.h"

namespace vp {
namespace {

constexpr int BT = 8;         // bootstraps per CTA
constexpr int THREADS = 256;  // 128 coefficient groups x 2 bootstrap groups
constexpr int RK = 8;         // coefficients per thread
constexpr int RB = 4;         // bootstraps per thread

struct __align__(128) Smem {
    uint32_t bk[kRows * 2 * kN];          // 49152 B: BK_i
    uint32_t acc[BT * 2 * kN];            // 65536 B: ACC staging for the rotation
    int8_t dig[BT * kRows * kTwoN];       // 98304 B: extended digit polynomials
    uint16_t abar[BT * kSlotWords];       // 10112 B: modulus-switched input
    BrJob job[BT];
    unsigned long long mbar;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issue the 48 KB copy of BK_i into shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void load_bk_step(uint32_t *dst, const uint32_t *src, unsigned long long *bar)
{
    constexpr uint32_t bytes = kBkStepWords * 4;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
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
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int *err)
{
    if (*reinterpret_cast<volatile int *>(err) != kDevOk) return false;
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitNs) {
            atomicExch(err, kDevTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ int32_t sbyte(uint32_t w, int b) { return (int32_t)(int8_t)(w >> (8 * b)); }

__global__ void __launch_bounds__(THREADS, 1)
br_dense_kernel(const BrJob *__restrict__ jobs, int njobs, const uint32_t *__restrict__ bk,
                uint32_t *__restrict__ big, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int job0 = blockIdx.x * BT;

    if (tid < BT) {
        BrJob j{};
        if (job0 + tid < njobs) j = jobs[job0 + tid];
        S.job[tid] = j;
    }
    if (tid == 0) mbar_init(&S.mbar, 1);
    __syncthreads();
    if (tid == 0) load_bk_step(S.bk, bk, &S.mbar);

    // Gate pre-combination and modulus switch: abar = round(c * 2N / 2^32) mod 2N.
    for (int idx = tid; idx < BT * kLweWords; idx += THREADS) {
        const int b = idx / kLweWords, i = idx - b * kLweWords;
        const BrJob &j = S.job[b];
        uint32_t c = (i == kn) ? j.cst : 0u;
        if (j.in0) c += (uint32_t)j.s0 * j.in0[i];
        if (j.in1) c += (uint32_t)j.s1 * j.in1[i];
        S.abar[b * kSlotWords + i] = (uint16_t)((c + (1u << 20)) >> 21);
    }
    __syncthreads();

    const int kg = tid & 127, bg = tid >> 7;
    const int k0 = kg * RK;
    uint32_t acc[2][RB][RK];
    // ACC = (0, X^{-bbar} v) with v = mu * sum_j X^j.
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        const uint32_t bbar = S.abar[(bg * RB + b) * kSlotWords + kn];
#pragma unroll
        for (int kk = 0; kk < RK; ++kk) {
            const uint32_t u = (uint32_t)(k0 + kk + bbar) & (kTwoN - 1);
            acc[0][b][kk] = 0u;
            acc[1][b][kk] = (u < (uint32_t)kN) ? kMu : (0u - kMu);
        }
    }

    constexpr uint32_t kOff = (1u << 31) + (1u << 24) + (1u << 17) + (1u << 10);

#pragma unroll 1
    for (int i = 0; i < kn; ++i) {
        // ACC -> shared memory for the rotation.
#pragma unroll
        for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint4 *dst = reinterpret_cast<uint4 *>(S.acc + ((bg * RB + b) * 2 + j) * kN + k0);
                dst[0] = make_uint4(acc[j][b][0], acc[j][b][1], acc[j][b][2], acc[j][b][3]);
                dst[1] = make_uint4(acc[j][b][4], acc[j][b][5], acc[j][b][6], acc[j][b][7]);
            }
        __syncthreads();
        if (tid == 0 && i > 0) load_bk_step(S.bk, bk + (size_t)i * kBkStepWords, &S.mbar);

        // Rotate, subtract, decompose: items = (bootstrap, component, 4 coefficients).
        for (int it = tid; it < BT * 2 * (kN / 4); it += THREADS) {
            const int k4 = it & (kN / 4 - 1), q = (it >> 8) & 1, b = it >> 9;
            const uint32_t abar = S.abar[b * kSlotWords + i];
            const uint32_t *a = S.acc + (b * 2 + q) * kN;
            uint32_t dp[kL] = {0u, 0u, 0u}, dn[kL] = {0u, 0u, 0u};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k4 * 4 + e;
                const uint32_t u = ((uint32_t)k - abar) & (kTwoN - 1);
                uint32_t v = a[u & (kN - 1)];
                if (u >= (uint32_t)kN) v = 0u - v;
                const uint32_t y = v - a[k] + kOff;
#pragma unroll
                for (int p = 0; p < kL; ++p) {
                    const int32_t d = (int32_t)((y >> (32 - kBgBits * (p + 1))) & 127u) - 64;
                    dp[p] |= ((uint32_t)d & 0xFFu) << (8 * e);
                    dn[p] |= ((uint32_t)(-d) & 0xFFu) << (8 * e);
                }
            }
#pragma unroll
            for (int p = 0; p < kL; ++p) {
                int8_t *row = S.dig + (b * kRows + 2 * p + q) * kTwoN;
                *reinterpret_cast<uint32_t *>(row + kN + k4 * 4) = dp[p];
                *reinterpret_cast<uint32_t *>(row + k4 * 4) = dn[p];
            }
        }
        __syncthreads();
        mbar_wait(&S.mbar, (uint32_t)(i & 1), err);

        // ACC_j[k] += sum_r sum_m BK[r][j][m] * D'_r[k - m]
#pragma unroll 1
        for (int r = 0; r < kRows; ++r) {
            const uint32_t *bk0 = S.bk + (r * 2 + 0) * kN;
            const uint32_t *bk1 = S.bk + (r * 2 + 1) * kN;
            const int8_t *drow = S.dig + ((bg * RB) * kRows + r) * kTwoN + k0 + kN - 8;
#pragma unroll 1
            for (int m0 = 0; m0 < kN; m0 += 8) {
                const uint4 x0 = *reinterpret_cast<const uint4 *>(bk0 + m0);
                const uint4 x1 = *reinterpret_cast<const uint4 *>(bk0 + m0 + 4);
                const uint4 y0 = *reinterpret_cast<const uint4 *>(bk1 + m0);
                const uint4 y1 = *reinterpret_cast<const uint4 *>(bk1 + m0 + 4);
                const uint32_t B0[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const uint32_t B1[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const int8_t *src = drow + b * kRows * kTwoN - m0;
                    const uint2 lo = *reinterpret_cast<const uint2 *>(src);
                    const uint2 hi = *reinterpret_cast<const uint2 *>(src + 8);
                    const uint32_t wv[4] = {lo.x, lo.y, hi.x, hi.y};
                    int32_t W[16];
#pragma unroll
                    for (int x = 1; x < 16; ++x) W[x] = sbyte(wv[x >> 2], x & 3);
#pragma unroll
                    for (int kk = 0; kk < RK; ++kk)
#pragma unroll
                        for (int mm = 0; mm < 8; ++mm) {
                            const uint32_t d = (uint32_t)W[kk - mm + 8];
                            acc[0][b][kk] += B0[mm] * d;
                            acc[1][b][kk] += B1[mm] * d;
                        }
                }
            }
        }
    }

    // Sample extract: a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0.
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        const int jb = bg * RB + b;
        if (job0 + jb >= njobs) continue;
        uint32_t *row = big + (size_t)S.job[jb].big * kBigWords;
#pragma unroll
        for (int kk = 0; kk < RK; ++kk) {
            const int k = k0 + kk;
            if (k == 0) {
                row[0] = acc[0][b][0];
                row[kN] = acc[1][b][0];
            } else {
                row[kN - k] = 0u - acc[0][b][kk];
            }
        }
    }
}

// Diagnostic: the bounded wait of the blind-rotation kernels on a barrier
// nothing ever arrives at.  It gives up after kWaitNs, records kDevTimeout in
// the error word and the kernel returns normally.
__global__ void wait_selftest_kernel(int *err)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    mbar_wait(&bar, 0u, err);
}

}  // namespace

int launch_wait_selftest(int *err, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(err);
    return 1;
}

int br_dense_jobs_per_cta() { return BT; }

// Raise the dynamic shared-memory limit once per process (outside any stream capture).
int configure_br_dense()
{
    return cudaFuncSetAttribute(br_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) == cudaSuccess ? 0 : -1;
}

int launch_br_dense(const BrJob *jobs, int njobs, const uint32_t *bk, uint32_t *big, int *err,
                    cudaStream_t st)
{
    if (njobs <= 0) return 0;
    static bool configured = false;
    const int smem = (int)sizeof(Smem);
    if (!configured) {
        if (cudaFuncSetAttribute(br_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return 0;  // the launch error surfaces through cudaGetLastError()
        configured = true;
    }
    const int grid = (njobs + BT - 1) / BT;
    br_dense_kernel<<<grid, THREADS, smem, st>>>(jobs, njobs, bk, big, err);
    return 1;
}

}  // namespace vp
