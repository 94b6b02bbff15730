// LWE key switching (dimension N = 1024 under K -> n = 630 under s), plus the
// bootstrap-free gates and the key-layout kernel.
//
// Key switch (tfhe-2; parameters from the paper's Appendix table, base 2^2,
// t = 8 levels): each extracted mask word a'_i is rounded to 16 bits,
// abar_i = a'_i + 2^15, split into 8 base-4 digits d_ij (j = 0 most
// significant), and out = (0, b') - sum_{i,j: d_ij != 0} KSK[i][j][d_ij].
// It is a gather-sum bound by memory bandwidth: a CTA owns 8 or 16 gates and
// streams the 2,528-byte KSK rows of digits 1..3 once for all of them (digit 0
// selects nothing), every thread owning one 16-byte column of the padded
// 632-word row.
#include "vp_internal.h"

namespace vp {
namespace {

constexpr int KS_THREADS = 160;  // 158 active 16-byte columns

// KS_JOBS gates per CTA: 16 reuses each gathered row more; 8 gives small
// layers enough CTAs to fill the GPU.
template <int KS_JOBS>
__global__ void __launch_bounds__(KS_THREADS)
key_switch_kernel(const KsJob *__restrict__ jobs, int njobs, const uint32_t *__restrict__ big,
                  const uint4 *__restrict__ ksk)
{
    __shared__ uint16_t top[KS_JOBS][kN];   // 16-bit rounded a'_i: its 8 base-4 digits
    __shared__ uint32_t bprime[KS_JOBS];
    __shared__ KsJob sj[KS_JOBS];
    const int tid = threadIdx.x;
    const int job0 = blockIdx.x * KS_JOBS;
    const int nj = min(KS_JOBS, njobs - job0);

    if (tid < KS_JOBS) {
        KsJob j{};
        j.e0 = -1;
        j.e1 = -1;
        if (tid < nj) j = jobs[job0 + tid];
        sj[tid] = j;
    }
    __syncthreads();
    for (int idx = tid; idx < KS_JOBS * (kN + 1); idx += KS_THREADS) {
        const int b = idx / (kN + 1), i = idx - b * (kN + 1);
        const KsJob &j = sj[b];
        uint32_t a = 0u;
        if (j.e0 >= 0) a = big[(size_t)j.e0 * kBigWords + i];
        if (j.e1 >= 0) a += big[(size_t)j.e1 * kBigWords + i];
        if (i < kN) top[b][i] = (uint16_t)((a + (1u << 15)) >> 16);
        else bprime[b] = a + j.cst;
    }
    __syncthreads();
    const int c = tid;
    if (c >= kKskQuads) return;

    uint4 acc[KS_JOBS];
#pragma unroll
    for (int b = 0; b < KS_JOBS; ++b) acc[b] = make_uint4(0u, 0u, 0u, 0u);

    // Per (i, j) the three candidate rows d = 1, 2, 3 are loaded once,
    // unconditionally and for all eight levels before any is used, so each
    // thread keeps 24 independent 16-byte loads in flight; every gate then
    // subtracts the row its digit selects (a CTA-uniform branch: the digits
    // come from shared memory).
#pragma unroll 1
    for (int i = 0; i < kN; ++i) {
        uint32_t t[KS_JOBS];
#pragma unroll
        for (int b = 0; b < KS_JOBS; ++b) t[b] = top[b][i];
        const uint4 *rows = ksk + (size_t)i * kKsT * kKsBase * kKskQuads + c;
        uint4 r[kKsT][kKsBase - 1];
#pragma unroll
        for (int j = 0; j < kKsT; ++j)
#pragma unroll
            for (int d = 1; d < kKsBase; ++d) r[j][d - 1] = __ldg(rows + (size_t)(j * kKsBase + d) * kKskQuads);
#pragma unroll
        for (int j = 0; j < kKsT; ++j) {
#pragma unroll
            for (int b = 0; b < KS_JOBS; ++b) {
                const uint32_t d = (t[b] >> (14 - 2 * j)) & 3u;
                if (d) {
                    const uint4 v = d == 1u ? r[j][0] : (d == 2u ? r[j][1] : r[j][2]);
                    acc[b].x -= v.x;
                    acc[b].y -= v.y;
                    acc[b].z -= v.z;
                    acc[b].w -= v.w;
                }
            }
        }
    }
#pragma unroll
    for (int b = 0; b < KS_JOBS; ++b) {
        if (b >= nj) break;
        uint32_t *out = sj[b].out;
        const uint32_t v[4] = {acc[b].x, acc[b].y, acc[b].z, acc[b].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int w = 4 * c + e;
            if (w < kn) out[w] = v[e];
            else if (w == kn) out[kn] = bprime[b] + v[e];
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

__global__ void pad_ksk_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, size_t rows)
{
    const size_t r = blockIdx.x;
    if (r >= rows) return;
    for (int w = threadIdx.x; w < kSlotWords; w += blockDim.x)
        dst[r * kSlotWords + w] = (w < kLweWords) ? src[r * kLweWords + w] : 0u;
}

}  // namespace

int launch_key_switch(const KsJob *jobs, int njobs, const uint32_t *big, const uint32_t *ksk_dev,
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
    if ((njobs + 15) / 16 < 2 * sms)
        key_switch_kernel<8><<<(njobs + 7) / 8, KS_THREADS, 0, st>>>(jobs, njobs, big, k4);
    else
        key_switch_kernel<16><<<(njobs + 15) / 16, KS_THREADS, 0, st>>>(jobs, njobs, big, k4);
    return 1;
}

int launch_free(const FreeJob *jobs, int njobs, cudaStream_t st)
{
    if (njobs <= 0) return 0;
    free_gate_kernel<<<njobs, 128, 0, st>>>(jobs, njobs);
    return 1;
}

int launch_pad_ksk(const uint32_t *ksk_abi, uint32_t *ksk_dev, cudaStream_t st)
{
    const size_t rows = (size_t)kN * kKsT * kKsBase;
    pad_ksk_kernel<<<(unsigned)rows, 256, 0, st>>>(ksk_abi, ksk_dev, rows);
    return 1;
}

}  // namespace vp
