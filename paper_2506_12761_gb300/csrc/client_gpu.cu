// Client-side preprocessing on the GPU: key generation (Section 2.2 KeyGen:
// the bootstrapping key BK = TRGSW encryptions of the LWE key bits and the
// key-switching key KSK), encryption of bits (Enc with Ecd), Alg. PubKeyGen
// (one encryption of zero per database bit) and Alg. ServerEnc (adding
// (0, Ecd(bit)) to a public-key ciphertext).
//
// These are the same computations as the host-only client library
// (libvelopir_client.so), from the same caller-supplied random numbers, so
// the ciphertexts are bit-identical; on the GPU a cloud key is generated in
// well under a second and can be loaded into a context without leaving the
// device, and a server can run Alg. ServerEnc over a large database where it
// already holds it.  All arithmetic is mod 2^32.
//
// Kernels (all integer, HBM- or issue-bound, run once per key or database):
//   bk_keygen_kernel     one CTA per TRGSW row (630 x 6): b = a K + e (+ the
//                        gadget term s_i 2^(32-7p) on component q), the
//                        negacyclic product with the binary TRLWE key K as a
//                        signed sum of rotations of a over the set bits of K;
//   lwe_encrypt_kernel   one warp per LWE sample: (a, <a, s> + m + e), which
//                        serves the KSK rows (m = v K_i 2^(32-2(j+1))), Enc
//                        (m = Ecd(bit)) and Alg. PubKeyGen (m = 0);
//   server_encrypt_kernel elementwise: ct = pk + (0, Ecd(bit)).
#include <vector>

#include "../../include/velopir.h"
#include "vp_internal.h"

namespace {

using namespace vp;

constexpr int kKeygenThreads = 256;

// One TRGSW row of BK per CTA.  Row ir = i * 6 + r, r = 2(p-1) + q.
// Output row: [a (N words)][b (N words)].
__global__ void __launch_bounds__(kKeygenThreads) bk_keygen_kernel(const uint32_t *__restrict__ s,
                                                                   const uint32_t *__restrict__ K,
                                                                   const uint32_t *__restrict__ bk_a,
                                                                   const uint32_t *__restrict__ bk_e,
                                                                   uint32_t *__restrict__ bk_out)
{
    __shared__ uint32_t a[kN];
    __shared__ uint32_t kb[kN];
    const size_t ir = blockIdx.x;
    const int tid = threadIdx.x;
    const uint32_t *src = bk_a + ir * kN;
    for (int k = tid; k < kN; k += kKeygenThreads) {
        a[k] = src[k];
        kb[k] = K[k] & 1u;
    }
    __syncthreads();
    constexpr int kPer = kN / kKeygenThreads;   // outputs per thread: k = tid + 256 m
    uint32_t acc[kPer];
#pragma unroll
    for (int m = 0; m < kPer; ++m) acc[m] = bk_e[ir * kN + tid + kKeygenThreads * m];
    // b = e + sum over i with K_i = 1 of X^i a: coefficient k gains a[k - i],
    // negated when k - i wraps below 0 (X^N = -1).  K_i is the same for every
    // thread, so the branch is uniform.
#pragma unroll 4
    for (int i = 0; i < kN; ++i) {
        if (!kb[i]) continue;
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int k = tid + kKeygenThreads * m;
            const uint32_t v = a[(k - i) & (kN - 1)];
            acc[m] += (k >= i) ? v : 0u - v;
        }
    }
    const int r = (int)(ir % kRows), p = r / 2 + 1, q = r % 2;
    const uint32_t g = (s[ir / kRows] & 1u) ? (1u << (32 - kBgBits * p)) : 0u;
    uint32_t *ra = bk_out + ir * 2 * kN, *rb = ra + kN;
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
        const int k = tid + kKeygenThreads * m;
        ra[k] = a[k] + ((k == 0 && q == 0) ? g : 0u);
        rb[k] = acc[m] + ((k == 0 && q == 1) ? g : 0u);
    }
}

enum : int { kMsgZero = 0, kMsgBits = 1, kMsgKsk = 2 };

// One warp per LWE sample c: out_c = (a_c, <a_c, s> + m_c + e_c), where m_c
// is 0 (Alg. PubKeyGen), Ecd(bits[c]) (Enc), or, for the key-switching key
// sample c = (i t + j) base + v, v K_i 2^(32 - 2(j+1)).
__global__ void __launch_bounds__(256) lwe_encrypt_kernel(const uint32_t *__restrict__ s,
                                                          const uint32_t *__restrict__ a,
                                                          const uint32_t *__restrict__ e,
                                                          const uint32_t *__restrict__ msg, int mode,
                                                          size_t count, uint32_t *__restrict__ out)
{
    const size_t c = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= count) return;
    const uint32_t *ac = a + c * kn;
    uint32_t *o = out + c * kLweWords;
    uint32_t dot = 0;
    for (int k = lane; k < kn; k += 32) {
        const uint32_t v = ac[k];
        o[k] = v;
        dot += (__ldg(s + k) & 1u) ? v : 0u;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, d);
    if (lane == 0) {
        uint32_t m = 0;
        if (mode == kMsgBits) {
            m = msg[c] ? kMu : 0u - kMu;
        } else if (mode == kMsgKsk) {
            const size_t i = c / (kKsT * kKsBase);
            const int j = (int)((c / kKsBase) % kKsT), v = (int)(c % kKsBase);
            m = (uint32_t)v * (msg[i] & 1u) * (1u << (32 - kKsBaseBits * (j + 1)));
        }
        o[kn] = dot + m + e[c];
    }
}

// ct = pk + (0, Ecd(bit)), one thread per word.
__global__ void server_encrypt_kernel(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ bits,
                                      size_t words, uint32_t *__restrict__ out)
{
    const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= words) return;
    const size_t c = w / kLweWords;
    uint32_t v = pk[w];
    if (w % kLweWords == (size_t)kn) v += bits[c] ? kMu : 0u - kMu;
    out[w] = v;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device views of caller buffers for one call: device pointers pass through;
// host buffers get a stream-ordered temporary (inputs copied in, outputs
// copied back by finish()), released when the call ends.
struct Staging {
    velopir_ctx *ctx;
    cudaStream_t st;
    std::vector<void *> temps;
    struct Back { void *host; const void *dev; size_t bytes; };
    std::vector<Back> back;
    int rc = VELOPIR_OK;

    Staging(velopir_ctx *c, cudaStream_t s) : ctx(c), st(s) {}
    ~Staging()
    {
        for (void *p : temps) cudaFreeAsync(p, st);
        if (!temps.empty()) cudaStreamSynchronize(st);
    }
    void *temp(size_t bytes)
    {
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes ? bytes : 4, st) != cudaSuccess) {
            cudaGetLastError();
            rc = ctx_fail(ctx, VELOPIR_ERR_OOM, "cannot allocate device staging for a host buffer");
            return nullptr;
        }
        temps.push_back(p);
        return p;
    }
    const uint32_t *in(const uint32_t *src, size_t words)
    {
        if (rc) return nullptr;
        if (on_device(src)) return src;
        void *d = temp(words * 4);
        if (d && cudaMemcpyAsync(d, src, words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            rc = ctx_fail(ctx, VELOPIR_ERR_CUDA, "host-to-device copy failed");
            return nullptr;
        }
        return static_cast<const uint32_t *>(d);
    }
    uint32_t *out(uint32_t *dst, size_t words)
    {
        if (rc) return nullptr;
        if (on_device(dst)) return dst;
        void *d = temp(words * 4);
        if (d) back.push_back({dst, d, words * 4});
        return static_cast<uint32_t *>(d);
    }
    // Copy host outputs back and wait for the stream.
    int finish(uint64_t launches)
    {
        if (rc) return rc;
        for (const Back &b : back)
            if (cudaMemcpyAsync(b.host, b.dev, b.bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
                cudaGetLastError();
                return ctx_fail(ctx, VELOPIR_ERR_CUDA, "device-to-host copy failed");
            }
        return ctx_finish(ctx, launches);
    }
};

int begin(velopir_ctx *ctx, CtxResources *R)
{
    if (!ctx) return VELOPIR_ERR_ARG;
    if (int rc = ctx_resources(ctx, R)) return rc;
    if (cudaSetDevice(R->device) != cudaSuccess) return ctx_fail(ctx, VELOPIR_ERR_CUDA, "cudaSetDevice failed");
    return VELOPIR_OK;
}

bool paper_params(const velopir_params *p)
{
    return p && p->n == kn && p->N == kN && p->k == 1 && p->l == kL && p->bg_bits == kBgBits && p->ks_t == kKsT &&
           p->ks_base_bits == kKsBaseBits;
}

unsigned blocks_for_warps(size_t warps) { return (unsigned)((warps + 7) / 8); }   // 8 warps per 256-thread CTA

constexpr size_t kMaxSamples = (size_t)1 << 24;   // per call: 16 Mi LWE samples (42 GB of masks)

int encrypt_common(velopir_ctx *ctx, const uint32_t *s, const uint32_t *bits, const uint32_t *a, const uint32_t *e,
                   size_t count, uint32_t *out, int mode)
{
    CtxResources R{};
    if (int rc = begin(ctx, &R)) return rc;
    if (count == 0) return VELOPIR_OK;
    if (!s || !a || !e || !out || (mode == kMsgBits && !bits))
        return ctx_fail(ctx, VELOPIR_ERR_ARG, "null buffer");
    if (count > kMaxSamples) return ctx_fail(ctx, VELOPIR_ERR_ARG, "count above 2^24 samples per call");
    Staging S(ctx, R.stream);
    const uint32_t *ds = S.in(s, kn);
    const uint32_t *da = S.in(a, count * kn);
    const uint32_t *de = S.in(e, count);
    const uint32_t *db = mode == kMsgBits ? S.in(bits, count) : nullptr;
    uint32_t *dout = S.out(out, count * kLweWords);
    if (S.rc) return S.rc;
    lwe_encrypt_kernel<<<blocks_for_warps(count), 256, 0, R.stream>>>(ds, da, de, db, mode, count, dout);
    return S.finish(1);
}

}  // namespace

extern "C" {

int velopir_gpu_keygen(velopir_ctx *ctx, const velopir_params *params, const uint32_t *s, const uint32_t *K,
                       const uint32_t *bk_a, const uint32_t *bk_e, const uint32_t *ksk_a, const uint32_t *ksk_e,
                       uint32_t *bk_out, uint32_t *ksk_out)
{
    CtxResources R{};
    if (int rc = begin(ctx, &R)) return rc;
    if (!paper_params(params))
        return ctx_fail(ctx, VELOPIR_ERR_ARG, "parameters must be n=630 N=1024 k=1 l=3 Bg=2^7 t=8 base=2^2");
    if (!s || !K || !bk_a || !bk_e || !ksk_a || !ksk_e || !bk_out || !ksk_out)
        return ctx_fail(ctx, VELOPIR_ERR_ARG, "null buffer");
    constexpr size_t bk_rows = (size_t)kn * kRows;
    constexpr size_t ksk_samples = (size_t)kN * kKsT * kKsBase;
    Staging S(ctx, R.stream);
    const uint32_t *ds = S.in(s, kn);
    const uint32_t *dK = S.in(K, kN);
    const uint32_t *dbka = S.in(bk_a, bk_rows * kN);
    const uint32_t *dbke = S.in(bk_e, bk_rows * kN);
    const uint32_t *dkska = S.in(ksk_a, ksk_samples * kn);
    const uint32_t *dkske = S.in(ksk_e, ksk_samples);
    uint32_t *dbk = S.out(bk_out, bk_rows * 2 * kN);
    uint32_t *dksk = S.out(ksk_out, ksk_samples * kLweWords);
    if (S.rc) return S.rc;
    bk_keygen_kernel<<<(unsigned)bk_rows, kKeygenThreads, 0, R.stream>>>(ds, dK, dbka, dbke, dbk);
    lwe_encrypt_kernel<<<blocks_for_warps(ksk_samples), 256, 0, R.stream>>>(ds, dkska, dkske, dK, kMsgKsk,
                                                                            ksk_samples, dksk);
    return S.finish(2);
}

int velopir_gpu_encrypt_bits(velopir_ctx *ctx, const uint32_t *s, const uint32_t *bits, const uint32_t *a,
                             const uint32_t *e, size_t count, uint32_t *out)
{
    return encrypt_common(ctx, s, bits, a, e, count, out, kMsgBits);
}

int velopir_gpu_pubkeygen(velopir_ctx *ctx, const uint32_t *s, const uint32_t *a, const uint32_t *e, size_t count,
                          uint32_t *pk_out)
{
    return encrypt_common(ctx, s, nullptr, a, e, count, pk_out, kMsgZero);
}

int velopir_gpu_server_encrypt(velopir_ctx *ctx, const uint32_t *pk, const uint32_t *bits, size_t count,
                               uint32_t *ct_out)
{
    CtxResources R{};
    if (int rc = begin(ctx, &R)) return rc;
    if (count == 0) return VELOPIR_OK;
    if (!pk || !bits || !ct_out) return ctx_fail(ctx, VELOPIR_ERR_ARG, "null buffer");
    if (count > kMaxSamples) return ctx_fail(ctx, VELOPIR_ERR_ARG, "count above 2^24 samples per call");
    Staging S(ctx, R.stream);
    const uint32_t *dpk = S.in(pk, count * kLweWords);
    const uint32_t *db = S.in(bits, count);
    uint32_t *dout = S.out(ct_out, count * kLweWords);
    if (S.rc) return S.rc;
    const size_t words = count * kLweWords;
    server_encrypt_kernel<<<(unsigned)((words + 255) / 256), 256, 0, R.stream>>>(dpk, db, words, dout);
    return S.finish(1);
}

}  // extern "C"
