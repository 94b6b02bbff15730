// LWE key switching (dimension N = 1024 under K -> n = 630 under s), plus the
// bootstrap-free gates and the key-layout kernel.
//
// Key switch (tfhe-2; parameters from the paper's Appendix table, base 2^2,
// t = 8 levels): each extracted mask word a'_i is rounded to 16 bits,
// abar_i = a'_i + 2^15, split into 8 base-4 digits d_ij (j = 0 most
// significant), and out = (0, b') - sum_{i,j: d_ij != 0} KSK[i][j][d_ij].
//
// It is a gather-sum.  A CTA owns G gates, one warp each.  For every i the
// 24 candidate rows KSK[i][j][1..3] (60.7 KB, three contiguous rows per level)
// are staged into shared memory by bulk asynchronous copies, double-buffered
// on mbarriers, so each row crosses L2 once per CTA however many of its gates
// select it.  Each warp then subtracts, per level, the staged row its gate's
// digit selects: the digit is uniform across the warp, so a digit of 0 skips
// the level without divergence, and lane L owns the 16-byte columns
// L + 32m of the 632-word padded row, so the shared-memory reads are
// conflict-free.  The bound is shared-memory bandwidth: every gate reads
// about 6,144 selected rows of 2,528 bytes.
#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kKsRows = kKsT * (kKsBase - 1);                  // 24 staged rows per i
constexpr uint32_t kKsRowBytes = kKskQuads * 16;               // 2,528
constexpr uint32_t kKsLevelBytes = (kKsBase - 1) * kKsRowBytes; // rows d = 1..3 of one level, contiguous
constexpr uint32_t kKsStageBytes = kKsRows * kKsRowBytes;      // 60,672
constexpr int kKsQuadsPerLane = (kKskQuads + 31) / 32;         // 5

template <int G> struct __align__(128) KsSmem {
    uint4 stage[2][kKsRows][kKskQuads];
    uint16_t top[G][kN];          // 16-bit rounded a'_i: its 8 base-4 digits
    uint32_t bprime[G];
    KsJob job[G];
    unsigned long long full[2];
};

__device__ __forceinline__ uint32_t ks_smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t ks_global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool ks_try(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(ks_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (kWaitNs); a timeout is recorded in the error word, and once
// the error word is set a wait that is not already satisfied returns at once.
__device__ __forceinline__ void ks_wait(unsigned long long *bar, uint32_t parity, int *err)
{
    if (ks_try(bar, parity)) return;
    if (*reinterpret_cast<volatile int *>(err) != kDevOk) return;
    const uint64_t t0 = ks_global_ns();
    while (!ks_try(bar, parity)) {
        if (ks_global_ns() - t0 > kWaitNs) {
            atomicExch(err, kDevTimeout);
            return;
        }
    }
}

// Stage the 24 candidate rows of mask word i into buffer `dst` (one thread).
__device__ __forceinline__ void ks_stage(uint4 (*dst)[kKskQuads], const uint4 *ksk, int i, unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ks_smem_u32(bar)), "r"(kKsStageBytes)
                 : "memory");
#pragma unroll 1
    for (int j = 0; j < kKsT; ++j) {
        const uint4 *src = ksk + ((size_t)(i * kKsT + j) * kKsBase + 1) * kKskQuads;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                ks_smem_u32(dst[j * (kKsBase - 1)])),
            "l"(src), "r"(kKsLevelBytes), "r"(ks_smem_u32(bar))
            : "memory");
    }
}

template <int G>
__global__ void __launch_bounds__(G * 32, 1)
key_switch_kernel(const KsJob *__restrict__ jobs, int njobs, const uint32_t *__restrict__ big,
                  const uint4 *__restrict__ ksk, int *err)
{
    extern __shared__ unsigned char ks_smem_raw[];
    KsSmem<G> &S = *reinterpret_cast<KsSmem<G> *>(ks_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int job0 = blockIdx.x * G;
    const int nj = min(G, njobs - job0);

    if (tid < G) {
        KsJob j{};
        j.e0 = -1;
        j.e1 = -1;
        if (tid < nj) j = jobs[job0 + tid];
        S.job[tid] = j;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ks_smem_u32(&S.full[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ks_smem_u32(&S.full[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        ks_stage(S.stage[0], ksk, 0, &S.full[0]);
        ks_stage(S.stage[1], ksk, 1, &S.full[1]);
    }
    for (int idx = tid; idx < G * (kN + 1); idx += G * 32) {
        const int b = idx / (kN + 1), i = idx - b * (kN + 1);
        const KsJob &j = S.job[b];
        uint32_t a = 0u;
        if (j.e0 >= 0) a = big[(size_t)j.e0 * kBigWords + i];
        if (j.e1 >= 0) a += big[(size_t)j.e1 * kBigWords + i];
        if (i < kN) S.top[b][i] = (uint16_t)((a + (1u << 15)) >> 16);
        else S.bprime[b] = a + j.cst;
    }
    __syncthreads();

    uint4 acc[kKsQuadsPerLane];
#pragma unroll
    for (int m = 0; m < kKsQuadsPerLane; ++m) acc[m] = make_uint4(0u, 0u, 0u, 0u);
    const bool active = warp < nj;

#pragma unroll 1
    for (int i = 0; i < kN; ++i) {
        const int buf = i & 1;
        ks_wait(&S.full[buf], (uint32_t)((i >> 1) & 1), err);
        if (active) {
            const uint32_t t = S.top[warp][i];
#pragma unroll
            for (int j = 0; j < kKsT; ++j) {
                const uint32_t d = (t >> (14 - 2 * j)) & 3u;
                if (d) {
                    const uint4 *row = S.stage[buf][j * (kKsBase - 1) + (int)d - 1];
#pragma unroll
                    for (int m = 0; m < kKsQuadsPerLane; ++m) {
                        const int q = lane + 32 * m;
                        if (q < kKskQuads) {
                            const uint4 v = row[q];
                            acc[m].x -= v.x;
                            acc[m].y -= v.y;
                            acc[m].z -= v.z;
                            acc[m].w -= v.w;
                        }
                    }
                }
            }
        }
        __syncthreads();   // every warp is done with this buffer: refill it
        if (tid == 0 && i + 2 < kN) ks_stage(S.stage[buf], ksk, i + 2, &S.full[buf]);
    }

    // Copies still in flight after a timed-out wait must land before the
    // shared memory is released.
    if (tid == 0 && *reinterpret_cast<volatile int *>(err) != kDevOk) {
        for (int b = 0; b < 2; ++b)
            for (uint32_t ph = 0; ph < 2; ++ph) {
                const uint64_t t0 = ks_global_ns();
                while (!ks_try(&S.full[b], ph) && ks_global_ns() - t0 <= kWaitNs) {
                }
            }
    }
    if (!active) return;
    uint32_t *out = S.job[warp].out;
#pragma unroll
    for (int m = 0; m < kKsQuadsPerLane; ++m) {
        const int q = lane + 32 * m;
        const uint32_t v[4] = {acc[m].x, acc[m].y, acc[m].z, acc[m].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int w = 4 * q + e;
            if (w < kn) out[w] = v[e];
            else if (w == kn) out[kn] = S.bprime[warp] + v[e];
        }
    }
}

__global__ void free_gate_kernel(const FreeJob *__restrict__ jobs, int njobs)
{
    const int j = blockIdx.x;
    if (j >= njobs) return;
    const FreeJob fj = jobs[j];
    for (int w = threadIdx.x; w < kLweWords; w += blockDim.x) {
        uint32_t v = fj.in ? (uint32_t)fj.s * fj.in[w] : 0u;
        if (w == kn) v += fj.cst;
        fj.out[w] = v;
    }
}

// out = sum_k s[k] in[k]: the multi-input pre-combinations of a layer.
__global__ void sum_kernel(const SumJob *__restrict__ jobs, int njobs)
{
    const int j = blockIdx.x;
    if (j >= njobs) return;
    const SumJob sj = jobs[j];
    for (int w = threadIdx.x; w < kLweWords; w += blockDim.x) {
        uint32_t v = 0u;
        for (int k = 0; k < sj.n; ++k) v += (uint32_t)sj.s[k] * sj.in[k][w];
        sj.out[w] = v;
    }
}

// Gate trace: one record of kTraceWords words per sampled gate (the layout of
// velopir_trace_rec): header, then the inputs (zero beyond nin), then the output.

__global__ void trace_kernel(const TraceJob *__restrict__ jobs, int njobs, uint32_t *__restrict__ records)
{
    const int j = blockIdx.x;
    if (j >= njobs) return;
    const TraceJob &t = jobs[j];
    uint32_t *r = records + (size_t)t.rec * kTraceWords;
    if (threadIdx.x == 0) {
        r[0] = (uint32_t)t.nrot;
        r[1] = (uint32_t)t.nin;
        r[2] = t.ks_cst;
        r[3] = t.cst[0];
        r[4] = t.cst[1];
    }
    if (threadIdx.x < 2 * kSumMax) r[5 + threadIdx.x] = (uint32_t)t.coef[threadIdx.x / kSumMax][threadIdx.x % kSumMax];
    for (int k = 0; k <= kSumMax; ++k) {
        const uint32_t *src = k < kSumMax ? (k < t.nin ? t.in[k] : nullptr) : t.out;
        uint32_t *dst = r + kTraceHead + (size_t)k * kLweWords;
        for (int w = threadIdx.x; w < kLweWords; w += blockDim.x) dst[w] = src ? src[w] : 0u;
    }
}

__global__ void pad_ksk_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, size_t rows)
{
    const size_t r = blockIdx.x;
    if (r >= rows) return;
    for (int w = threadIdx.x; w < kSlotWords; w += blockDim.x)
        dst[r * kSlotWords + w] = (w < kLweWords) ? src[r * kLweWords + w] : 0u;
}

}  // namespace

int configure_key_switch()
{
    if (cudaFuncSetAttribute(key_switch_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(KsSmem<8>)) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(key_switch_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(KsSmem<16>)) != cudaSuccess)
        return -1;
    return 0;
}

// 16 gates per CTA stage each row for more gates; 8 when that would leave SMs idle.
int launch_key_switch(const KsJob *jobs, int njobs, const uint32_t *big, const uint32_t *ksk_dev, int *err,
                      cudaStream_t st)
{
    if (njobs <= 0) return 0;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    const uint4 *k4 = reinterpret_cast<const uint4 *>(ksk_dev);
    if (njobs < 16 * sms)
        key_switch_kernel<8><<<(njobs + 7) / 8, 8 * 32, sizeof(KsSmem<8>), st>>>(jobs, njobs, big, k4, err);
    else
        key_switch_kernel<16><<<(njobs + 15) / 16, 16 * 32, sizeof(KsSmem<16>), st>>>(jobs, njobs, big, k4, err);
    return 1;
}

int launch_free(const FreeJob *jobs, int njobs, cudaStream_t st)
{
    if (njobs <= 0) return 0;
    free_gate_kernel<<<njobs, 128, 0, st>>>(jobs, njobs);
    return 1;
}

int launch_sum(const SumJob *jobs, int njobs, cudaStream_t st)
{
    if (njobs <= 0) return 0;
    sum_kernel<<<njobs, 128, 0, st>>>(jobs, njobs);
    return 1;
}

int launch_trace(const TraceJob *jobs, int njobs, uint32_t *records, cudaStream_t st)
{
    if (njobs <= 0) return 0;
    trace_kernel<<<njobs, 128, 0, st>>>(jobs, njobs, records);
    return 1;
}

int launch_pad_ksk(const uint32_t *ksk_abi, uint32_t *ksk_dev, cudaStream_t st)
{
    const size_t rows = (size_t)kN * kKsT * kKsBase;
    pad_ksk_kernel<<<(unsigned)rows, 256, 0, st>>>(ksk_abi, ksk_dev, rows);
    return 1;
}

}  // namespace vp
