// Integer multiply-pipe throughput of this GPU, per SM clock: the peak that
// the blind-rotation roofline counts against.  Three instruction streams,
// each as 8 independent dependency chains per thread, 4 CTAs of 512 threads
// per SM (64 resident warps):
//   lo     x = x * a + b           (32-bit low multiply-add)
//   hi     x = umulhi(x, a) ^ b    (32-bit high multiply)
//   shoup  x = x * w - umulhi(x, w') * p   (one Shoup modular product, the
//          NTT kernel's multiply: one high and two low multiplies)
// Each CTA times itself with clock64(); the three streams run back to back,
// so their throughput ratios (how many low multiplies a high multiply or a
// Shoup product costs) do not depend on the clock.  The absolute rates are
// per clock64 tick, which on this GPU need not equal an SM clock cycle
// under boost.  A standalone program (not part of libvelopir.so);
// paper_2506_12761_gb300/int_peak.py builds and runs it.
#include <cstdint>
#include <cstdio>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>

template <int MODE>
__global__ void __launch_bounds__(512) chains(uint32_t *out, unsigned long long *cycles, uint32_t a, uint32_t as,
                                              uint32_t p, int iters)
{
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 8u + k + blockIdx.x * 977u;
    __syncthreads();
    const unsigned long long t0 = clock64();
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (MODE == 0) x[k] = x[k] * a + p;
            else if (MODE == 1) x[k] = __umulhi(x[k], as) ^ a;
            else x[k] = x[k] * a - __umulhi(x[k], as) * p;
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

int main()
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) return 1;
    const int per_sm = 4, threads = 512, iters = 20000, blocks = sms * per_sm;
    uint32_t *out = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * 4) != cudaSuccess) return 1;
    if (cudaMalloc(&cyc, (size_t)blocks * 8) != cudaSuccess) return 1;
    const uint32_t p = 167772161u, a = 123456789u, as = (uint32_t)(((uint64_t)a << 32) / p);
    const char *names[3] = {"lo", "hi", "shoup"};
    std::vector<unsigned long long> h(blocks);
    for (int mode = 0; mode < 3; ++mode) {
        double best = 0;
        for (int rep = 0; rep < 3; ++rep) {
            if (mode == 0) chains<0><<<blocks, threads>>>(out, cyc, a, as, p, iters);
            else if (mode == 1) chains<1><<<blocks, threads>>>(out, cyc, a, as, p, iters);
            else chains<2><<<blocks, threads>>>(out, cyc, a, as, p, iters);
            if (cudaMemcpy(h.data(), cyc, (size_t)blocks * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
            std::sort(h.begin(), h.end());
            const double per_sm_ops = (double)per_sm * threads * iters * 8;
            best = std::max(best, per_sm_ops / (double)h[blocks / 2]);   // median CTA: all 4 CTAs of an SM run together
        }
        printf("{\"op\": \"%s\", \"lane_ops_per_tick_per_sm\": %.2f}\n", names[mode], best);
    }
    const cudaError_t err = cudaGetLastError();
    cudaFree(out);
    cudaFree(cyc);
    if (err != cudaSuccess) {
        printf("{\"error\": \"%s\"}\n", cudaGetErrorString(err));
        return 1;
    }
    return 0;
}
