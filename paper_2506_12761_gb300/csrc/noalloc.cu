// velopir_bootstrap_batch_noalloc: the batched gate bootstrap for callers
// that cannot allocate device memory at call time.
//
// Some callers fix their device-memory footprint before they start working:
// a serving process that reserves its HBM at start-up, code that runs under a
// hard memory cap or behind a caching allocator that must not see foreign
// allocations, or a latency-critical loop in which a cudaMalloc or cudaFree
// (cudaFree synchronises the whole device) would stall every other stream.
// velopir_bootstrap_batch allocates its scratch (job lists, extracted rows)
// on demand, which such callers cannot accept.  This entry point takes its
// scratch from one file-scope device array instead, so a call allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// The array holds at most VELOPIR_NOALLOC_MAX_GATES gates (two blind
// rotations per MUX) and stays resident on every device that loads this
// library until the process exits.  All calls share it: calls whose work
// overlaps on the GPU race and must be serialised by the caller (one stream,
// or events between streams).  Every word a call reads from the array is
// written earlier in the same call, so nothing in it needs clearing between
// calls.
#include <mutex>

#include "../../include/velopir.h"
#include "sched.h"
#include "vp_internal.h"

namespace {

using namespace vp;

constexpr size_t kMaxGates = VELOPIR_NOALLOC_MAX_GATES;
constexpr size_t kMaxRotations = 2 * kMaxGates;

struct NoAllocScratch {
    uint32_t big[kMaxRotations * kBigWords];   // extracted rows between blind rotation and key switch
    BrJob br[kMaxRotations];
    KsJob ks[kMaxGates];
};

// 2.1 MB per device.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mu;
NoAllocScratch *g_scratch_addr[256] = {nullptr};   // per device, filled once

// One thread per gate: the blind-rotation and key-switch job records.
__global__ void noalloc_jobs_kernel(int mux, const uint32_t *in, uint32_t *out, int count, int32_t s1, int32_t s2,
                                    uint32_t cst, NoAllocScratch *S)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    KsJob k{};
    k.out = out + (size_t)g * kLweWords;
    if (!mux) {
        const uint32_t *c = in + (size_t)g * 2 * kLweWords;
        S->br[g] = BrJob{c, c + kLweWords, s1, s2, cst, g};
        k.e0 = g;
        k.e1 = -1;
    } else {
        const uint32_t *c = in + (size_t)g * 3 * kLweWords;
        S->br[2 * g] = BrJob{c, c + kLweWords, 1, 1, 0u - kMu, 2 * g};                  // AND(c, a)
        S->br[2 * g + 1] = BrJob{c, c + 2 * kLweWords, -1, 1, 0u - kMu, 2 * g + 1};     // AND(NOT c, b)
        k.e0 = 2 * g;
        k.e1 = 2 * g + 1;
        k.cst = kMu;
    }
    S->ks[g] = k;
}

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int velopir_bootstrap_batch_noalloc(velopir_ctx *ctx, velopir_gate gate, const uint32_t *lwe_in,
                                               uint32_t *lwe_out, size_t count)
{
    if (!ctx) return VELOPIR_ERR_ARG;
    if ((int)gate < VP_AND || (int)gate > VP_MUX) return ctx_fail(ctx, VELOPIR_ERR_ARG, "unknown gate");
    if (count == 0) return VELOPIR_OK;
    if (count > kMaxGates)
        return ctx_fail(ctx, VELOPIR_ERR_ARG,
                        "count exceeds VELOPIR_NOALLOC_MAX_GATES (256): split the batch or use velopir_bootstrap_batch");
    if (!lwe_in || !lwe_out) return ctx_fail(ctx, VELOPIR_ERR_ARG, "null ciphertext buffer");
    CtxResources R{};
    if (int rc = ctx_resources(ctx, &R)) return rc;
    if (!R.key_loaded) return ctx_fail(ctx, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    if (R.device < 0 || R.device >= 256) return ctx_fail(ctx, VELOPIR_ERR_ARG, "device index out of range");
    if (cudaSetDevice(R.device) != cudaSuccess) return ctx_fail(ctx, VELOPIR_ERR_CUDA, "cudaSetDevice failed");
    if (!on_device(lwe_in) || !on_device(lwe_out))
        return ctx_fail(ctx, VELOPIR_ERR_ARG, "lwe_in and lwe_out must be device memory for the no-allocation call");

    NoAllocScratch *S;
    {
        // Set-up, once per device, with that device current: the device
        // address of the scratch array (a host reference to the symbol is
        // not a device address).
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_addr[R.device]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return ctx_fail(ctx, VELOPIR_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
            }
            g_scratch_addr[R.device] = reinterpret_cast<NoAllocScratch *>(p);
        }
        S = g_scratch_addr[R.device];
    }

    const bool mux = gate == VP_MUX;
    uint32_t cst = 0;
    int32_t s1 = 0, s2 = 0;
    gate_combination((int)gate, &cst, &s1, &s2);
    const int n = (int)count;
    noalloc_jobs_kernel<<<(n + 127) / 128, 128, 0, R.stream>>>(mux ? 1 : 0, lwe_in, lwe_out, n, s1, s2, cst, S);
    const int nrot = mux ? 2 * n : n;
    uint64_t launches = 1;
    if (R.bk_ntt) launches += launch_br_ntt(S->br, nrot, R.bk_ntt, S->big, R.err, R.stream);
    else launches += launch_br_dense(S->br, nrot, R.bk, S->big, R.err, R.stream);
    launches += launch_key_switch(S->ks, n, S->big, R.ksk, R.err, R.stream);
    return ctx_finish(ctx, launches);
}
