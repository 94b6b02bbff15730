// Internal declarations of libvelopir.so (not part of the public ABI).
//
// Parameters are fixed at compile time to the TFHE 128-bit set the paper uses
// (Appendix parameter table): n = 630, N = 1024, k = 1, l = 3, Bg = 2^7,
// key-switch base 2^2 with t = 8 levels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace vp {

constexpr int kN = 1024;            // ring degree
constexpr int kTwoN = 2 * kN;
constexpr int kn = 630;             // LWE dimension
constexpr int kLweWords = kn + 1;   // ABI ciphertext length
constexpr int kSlotWords = 632;     // device-internal ciphertext stride (16-byte rows)
constexpr int kL = 3;               // gadget levels
constexpr int kBgBits = 7;
constexpr int kRows = 2 * kL;       // TRGSW rows
constexpr int kKsT = 8;             // key-switch levels
constexpr int kKsBaseBits = 2;
constexpr int kKsBase = 1 << kKsBaseBits;
constexpr int kBigWords = 1028;     // extracted LWE (N + 1 words) row stride
constexpr uint32_t kMu = 1u << 29;  // 1/8
constexpr size_t kBkStepWords = (size_t)kRows * 2 * kN;          // 12288 words = 48 KB
constexpr size_t kBkWords = (size_t)kn * kBkStepWords;
constexpr size_t kKskAbiWords = (size_t)kN * kKsT * kKsBase * kLweWords;
constexpr int kKskQuads = kSlotWords / 4;                         // 158 uint4 per padded row
constexpr size_t kKskDevWords = (size_t)kN * kKsT * kKsBase * kSlotWords;

// Gate pre-combination of one blind rotation: c = s0*in0 + s1*in1 + T(cst).
// A null input contributes nothing.  The extracted result goes to scratch
// row `big`.
struct BrJob {
    const uint32_t *in0;
    const uint32_t *in1;
    int32_t s0, s1;
    uint32_t cst;
    int32_t big;
};
static_assert(sizeof(BrJob) == 32, "BrJob layout");

// Key switch of e0 (+ e1) + T(cst) (extracted rows of this chunk) into `out`
// (631 words).  e1 < 0 means a single input.
struct KsJob {
    int32_t e0, e1;
    uint32_t cst;
    int32_t pad;
    uint32_t *out;
    uint64_t pad2;
};
static_assert(sizeof(KsJob) == 32, "KsJob layout");

// A gate that needs no bootstrap: out = s*in + T(cst) (NOT, copy, XNOR or
// AND against a plaintext bit, trivial constants).
struct FreeJob {
    const uint32_t *in;
    uint32_t *out;
    int32_t s;
    uint32_t cst;
    uint64_t pad;
};
static_assert(sizeof(FreeJob) == 32, "FreeJob layout");

// A multi-input linear pre-combination materialised before a layer's blind
// rotations (the g-input XOR of the fan-in HomSum): out = sum_k s[k] in[k]
// over the first n terms.  The blind rotation that reads `out` adds the
// gate's constant.
constexpr int kSumMax = 8;
struct SumJob {
    const uint32_t *in[kSumMax];
    int32_t s[kSumMax];
    uint32_t *out;
    int32_t n;
    uint32_t pad;
};
static_assert(sizeof(SumJob) == 112, "SumJob layout");

// One sampled gate of the gate trace: copy its inputs and output into record
// `rec` of the trace buffer, with its pre-combination (the layout of
// velopir_trace_rec).
struct TraceJob {
    const uint32_t *in[kSumMax];
    const uint32_t *out;
    int32_t coef[2][kSumMax];
    uint32_t cst[2];
    uint32_t ks_cst;
    int32_t nrot, nin;
    int32_t rec;
};
static_assert(sizeof(TraceJob) == 160, "TraceJob layout");
// Words of one trace record: nrot, nin, ks_cst, cst[2], coef[2][kSumMax],
// in[kSumMax][kLweWords], out[kLweWords].
constexpr int kTraceHead = 5 + 2 * kSumMax;
constexpr int kTraceWords = kTraceHead + (kSumMax + 1) * kLweWords;

// Device-side error codes written to the context's error word.
enum : int { kDevOk = 0, kDevTimeout = 1 };
constexpr unsigned long long kWaitNs = 2000000000ull;   // bound of every device-side wait (2 s)

// ---- kernel launchers (each returns the number of kernel launches issued) ----
int launch_br_dense(const BrJob *jobs, int njobs, const uint32_t *bk, uint32_t *big, int *err,
                    cudaStream_t st);
int br_dense_jobs_per_cta();

int configure_br_dense();
int configure_br_ntt();
int launch_br_ntt(const BrJob *jobs, int njobs, const uint32_t *bk_ntt, uint32_t *big, int *err,
                  cudaStream_t st);
int prepare_bk_ntt(const uint32_t *bk, uint32_t *bk_ntt, cudaStream_t st);
int launch_br_ntt_w(const BrJob *jobs, int njobs, const uint32_t *bk_ntt, uint32_t *big, int *err, cudaStream_t st,
                    int warps, int per = 0);    // a fixed shape of `warps` warps, `per` (<= warps) bootstraps per CTA
int ntt_shape_count();                         // tile shapes of the NTT kernel (bootstraps per CTA)
int ntt_shape(int i);                          // the i-th shape, ascending
int ntt_pick_warps(int njobs);                 // the tuned choice for a launch of njobs
void ntt_set_wave_ms(int warps, float ms);     // record a measured full-wave time
int ntt_full_wave();                           // bootstraps in one full wave of the best tuned shape (0: untuned)
size_t bk_ntt_words();

// Tensor-core path (exact fp16 limbs on tcgen05.mma kind::f16).
size_t bk_tc_bytes();                                     // expanded Hankel key, fp16 limbs
int prepare_bk_tc(const uint32_t *bk, void *bk_tc, cudaStream_t st);
size_t tc_scratch_bytes(int njobs);                       // ACC, digits and inputs of a launch of njobs
int configure_br_tc();
int launch_br_tc(const BrJob *jobs, int njobs, const void *bk_tc, void *scratch, uint32_t *big, int *err,
                 cudaStream_t st);

int configure_key_switch();
int launch_key_switch(const KsJob *jobs, int njobs, const uint32_t *big, const uint32_t *ksk_dev, int *err,
                      cudaStream_t st);
int launch_free(const FreeJob *jobs, int njobs, cudaStream_t st);
int launch_sum(const SumJob *jobs, int njobs, cudaStream_t st);
int launch_trace(const TraceJob *jobs, int njobs, uint32_t *records, cudaStream_t st);
int launch_pad_ksk(const uint32_t *ksk_abi, uint32_t *ksk_dev, cudaStream_t st);
int launch_wait_selftest(int *err, cudaStream_t st);   // a bounded wait that is never satisfied

// What an entry point outside api.cu needs from a context.
struct CtxResources {
    int device;
    cudaStream_t stream;
    bool key_loaded;
    const uint32_t *bk;       // dense-path key
    const uint32_t *ksk;      // padded key-switching key
    const uint32_t *bk_ntt;   // transformed key, or null if the NTT path is not selected and ready
    int *err;                 // device error word
};

}  // namespace vp

struct velopir_ctx;
namespace vp {
int ctx_resources(velopir_ctx *c, CtxResources *r);
int ctx_fail(velopir_ctx *c, int code, const char *msg);
int ctx_finish(velopir_ctx *c, uint64_t launches);   // count launches, sync, map the device error word
}  // namespace vp
