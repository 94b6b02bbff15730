// libvelopir_client.so, the host-only side of VeLoPIR (velopir_client.h): key
// generation, encryption and decryption from caller-supplied random numbers
// (paper Section 2.2: KeyGen, Enc with Ecd: m -> m/4 - 1/8, Dec by the sign of
// the phase), Alg. PubKeyGen and Alg. ServerEnc.  Plain C++: built with the
// host compiler, linked against no CUDA library.
//
// The TRLWE mask products a(X) * K(X) use the binary key directly: the
// product is the signed sum of the negacyclic shifts X^i a(X) over the set
// bits K_i = 1.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/velopir_client.h"

namespace {

constexpr int n = 630, N = 1024, L = 3, BG = 7, T = 8, B = 2, BASE = 4;
constexpr uint32_t MU = 1u << 29;

// out += X^i * a  (mod X^N + 1)
void add_shifted(uint32_t *out, const uint32_t *a, int i)
{
    for (int k = 0; k < N - i; ++k) out[k + i] += a[k];
    for (int k = N - i; k < N; ++k) out[k + i - N] -= a[k];
}

template <class F> void parallel_for(size_t count, F f)
{
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([=] {
            for (size_t i = t; i < count; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

bool paper_params(const velopir_params *p)
{
    return p && p->n == n && p->N == N && p->k == 1 && p->l == L && p->bg_bits == BG && p->ks_t == T &&
           p->ks_base_bits == B;
}

}  // namespace

extern "C" {

int velopir_client_keygen(const velopir_params *params, const uint32_t *s, const uint32_t *K, const uint32_t *bk_a,
                          const uint32_t *bk_e, const uint32_t *ksk_a, const uint32_t *ksk_e, uint32_t *bk_out,
                          uint32_t *ksk_out)
{
    if (!paper_params(params) || !s || !K || !bk_a || !bk_e || !ksk_a || !ksk_e || !bk_out || !ksk_out)
        return VELOPIR_ERR_ARG;
    std::vector<int> ones;
    for (int i = 0; i < N; ++i)
        if (K[i] & 1u) ones.push_back(i);
    // BK_i row r = 2(p-1)+q: (a, a*K + e) plus s_i * 2^(32-7p) on component q.
    parallel_for((size_t)n * 2 * L, [&](size_t ir) {
        const size_t i = ir / (2 * L);
        const int r = (int)(ir % (2 * L));
        const uint32_t *a = bk_a + ir * N;
        const uint32_t *e = bk_e + ir * N;
        uint32_t *ra = bk_out + ir * 2 * N;
        uint32_t *rb = ra + N;
        std::memcpy(ra, a, N * 4);
        std::memcpy(rb, e, N * 4);
        for (int k : ones) add_shifted(rb, a, k);
        const int p = r / 2 + 1, q = r % 2;
        const uint32_t g = (s[i] & 1u) ? (1u << (32 - BG * p)) : 0u;
        (q == 0 ? ra : rb)[0] += g;
    });
    // KSK[i][j][v] = (a, <a, s> + v * K_i * 2^(32 - 2(j+1)) + e)
    parallel_for((size_t)N, [&](size_t i) {
        for (int j = 0; j < T; ++j)
            for (int v = 0; v < BASE; ++v) {
                const size_t idx = (i * T + j) * BASE + v;
                const uint32_t *a = ksk_a + idx * n;
                uint32_t *row = ksk_out + idx * (n + 1);
                uint32_t dot = 0;
                for (int k = 0; k < n; ++k) {
                    row[k] = a[k];
                    dot += (s[k] & 1u) ? a[k] : 0u;
                }
                row[n] = dot + (uint32_t)v * (K[i] & 1u) * (1u << (32 - B * (j + 1))) + ksk_e[idx];
            }
    });
    return VELOPIR_OK;
}

int velopir_client_encrypt_bits(const uint32_t *s, const uint32_t *bits, const uint32_t *a, const uint32_t *e,
                                size_t count, uint32_t *out)
{
    if (!s || !bits || !a || !e || (!out && count)) return VELOPIR_ERR_ARG;
    for (size_t c = 0; c < count; ++c) {
        uint32_t dot = 0;
        const uint32_t *ac = a + c * n;
        uint32_t *o = out + c * (n + 1);
        for (int k = 0; k < n; ++k) {
            o[k] = ac[k];
            dot += (s[k] & 1u) ? ac[k] : 0u;
        }
        o[n] = dot + (bits[c] ? MU : 0u - MU) + e[c];
    }
    return VELOPIR_OK;
}

int velopir_client_pubkeygen(const uint32_t *s, const uint32_t *a, const uint32_t *e, size_t count, uint32_t *pk_out)
{
    // Alg. PubKeyGen: one fresh encryption of zero per database bit, (a, <a, s> + e).
    if (!s || !a || !e || (!pk_out && count)) return VELOPIR_ERR_ARG;
    for (size_t c = 0; c < count; ++c) {
        uint32_t dot = 0;
        const uint32_t *ac = a + c * n;
        uint32_t *o = pk_out + c * (n + 1);
        for (int k = 0; k < n; ++k) {
            o[k] = ac[k];
            dot += (s[k] & 1u) ? ac[k] : 0u;
        }
        o[n] = dot + e[c];
    }
    return VELOPIR_OK;
}

int velopir_server_encrypt(const uint32_t *pk, const uint32_t *bits, size_t count, uint32_t *ct_out)
{
    // Alg. ServerEnc: ct = (0, Ecd(bit)) + pk, with Ecd(1) = 1/8 and Ecd(0) = -1/8.
    if (!pk || !bits || (!ct_out && count)) return VELOPIR_ERR_ARG;
    for (size_t c = 0; c < count; ++c) {
        const uint32_t *p = pk + c * (n + 1);
        uint32_t *o = ct_out + c * (n + 1);
        for (int k = 0; k < n; ++k) o[k] = p[k];
        o[n] = p[n] + (bits[c] ? MU : 0u - MU);
    }
    return VELOPIR_OK;
}

int velopir_client_decrypt_bits(const uint32_t *s, const uint32_t *ct, size_t count, uint32_t *bits_out)
{
    if (!s || !ct || (!bits_out && count)) return VELOPIR_ERR_ARG;
    for (size_t c = 0; c < count; ++c) {
        const uint32_t *x = ct + c * (n + 1);
        uint32_t dot = 0;
        for (int k = 0; k < n; ++k) dot += (s[k] & 1u) ? x[k] : 0u;
        bits_out[c] = (int32_t)(x[n] - dot) >= 0 ? 1u : 0u;
    }
    return VELOPIR_OK;
}

}  // extern "C"
