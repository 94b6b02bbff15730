/*
 * TFHE oracle for VeLoPIR's server-side hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU implementation of gate bootstrapping
 * over the 32-bit discretised torus and of the plaintext-database circuits of
 * VeLoPIR's three modes.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The CUDA library shares
 * no code, header, table or helper with it.
 *
 * Paper: "Versatile and Fast Location-Based PIR with FHE over the Torus"
 * (VeLoPIR).  The paper defers bootstrapping internals to the TFHE journal
 * paper (Chillotti et al., J. Cryptol. 2020, cited as tfhe-2); the promised
 * explanation in its appendix is absent, so the blind-rotation, extraction and
 * key-switching steps follow tfhe-2's definitions.  Readings that the paper
 * leaves open are marked "reading:" below.
 *
 * Conventions (uint32 torus, 1.0 == 2^32, all arithmetic mod 2^32):
 *   LWE ciphertext   : u32[n+1] = a[0..n-1], b.  phase = b - <a,s>.
 *   TRLWE ciphertext : u32[2][N] = a(X), b(X).   phase = b - a*K mod X^N+1.
 *   Bootstrapping key: u32[n][2l][2][N]; row r = 2(p-1)+q (level p=1..l,
 *                      component q: 0 = a, 1 = b) is a TRLWE_K encryption of 0
 *                      plus s_i * 2^(32-bg_bits*p) added to component q.
 *   Key-switch key   : u32[N][t][base][n+1]; entry [i][j][v] = LWE_s(v*K_i*2^(32-B(j+1))).
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, brute force or truth tables (see each
 * function's comment for which pin).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;            /* LWE dimension                        (630)  */
    int32_t N;            /* ring degree, power of two            (1024) */
    int32_t l;            /* gadget levels                        (3)    */
    int32_t bg_bits;      /* log2 of the gadget base Bg           (7)    */
    int32_t ks_t;         /* key-switch levels                    (8)    */
    int32_t ks_base_bits; /* log2 of the key-switch base          (2)    */
} orc_params;

enum { ORC_AND = 0, ORC_NAND, ORC_OR, ORC_NOR, ORC_XOR, ORC_XNOR,
       ORC_ANDNY, ORC_ANDYN, ORC_ORNY, ORC_ORYN, ORC_MUX };

#define MU_1_8 0x20000000u   /* 1/8 on the torus */
#define MU_1_4 0x40000000u   /* 1/4 on the torus */

static int ilog2(int x) { int r = 0; while ((1 << r) < x) r++; return r; }

/* ------------------------------------------------------------------------- */
/* Negacyclic polynomial arithmetic in Z_{2^32}[X]/(X^N+1).                  */
/* ------------------------------------------------------------------------- */

/* Definition of the ring product: X^(i+j) = -X^(i+j-N) when i+j >= N.
 * Pin: X^a identities and the Karatsuba product below. */
void orc_poly_mul_schoolbook(uint32_t *out, const uint32_t *a, const uint32_t *b, int N)
{
    memset(out, 0, sizeof(uint32_t) * (size_t)N);
    for (int i = 0; i < N; i++) {
        for (int j = 0; j < N; j++) {
            uint32_t prod = a[i] * b[j];
            int k = i + j;
            if (k < N) out[k] += prod;
            else out[k - N] -= prod;
        }
    }
}

/* Linear (non-reduced) product r[0..2n) of two length-n arrays, Karatsuba
 * recursion a*b = a0b0 + ((a0+a1)(b0+b1) - a0b0 - a1b1) X^h + a1b1 X^n, which is
 * an identity over any commutative ring, so it is exact mod 2^32. */
static void kara_linear(uint32_t *r, const uint32_t *a, const uint32_t *b, int n, uint32_t *tmp)
{
    if (n <= 32) {
        memset(r, 0, sizeof(uint32_t) * 2 * (size_t)n);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                r[i + j] += a[i] * b[j];
        return;
    }
    int h = n / 2;
    kara_linear(r, a, b, h, tmp);            /* a0*b0 -> r[0..n)  */
    kara_linear(r + n, a + h, b + h, h, tmp); /* a1*b1 -> r[n..2n) */
    uint32_t *sa = tmp, *sb = tmp + h, *t = tmp + 2 * h, *rest = tmp + 2 * h + n;
    for (int i = 0; i < h; i++) { sa[i] = a[i] + a[h + i]; sb[i] = b[i] + b[h + i]; }
    kara_linear(t, sa, sb, h, rest);
    for (int i = 0; i < n; i++) t[i] -= r[i] + r[n + i];
    for (int i = 0; i < n; i++) r[h + i] += t[i];
}

/* Same ring product via Karatsuba, then the negacyclic fold c_k - c_{k+N}.
 * Pin: equals orc_poly_mul_schoolbook on random and edge inputs. */
void orc_poly_mul_karatsuba(uint32_t *out, const uint32_t *a, const uint32_t *b, int N)
{
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)N);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * 4 * (size_t)N);
    kara_linear(r, a, b, N, tmp);
    for (int k = 0; k < N; k++) out[k] = r[k] - r[k + N];
    free(r);
    free(tmp);
}

/* out = X^e * p for any integer e (taken mod 2N).  Coefficient k of the
 * result is +p[u] if u = (k - e) mod 2N < N, else -p[u - N].
 * Pin: X^a X^b = X^(a+b), X^N = -1, exhaustively at toy N. */
void orc_poly_mul_xe(uint32_t *out, const uint32_t *p, int e, int N)
{
    int twoN = 2 * N;
    e %= twoN;
    if (e < 0) e += twoN;
    for (int k = 0; k < N; k++) {
        int u = ((k - e) % twoN + twoN) % twoN;
        out[k] = (u < N) ? p[u] : (uint32_t)(0u - p[u - N]);
    }
}

/* ------------------------------------------------------------------------- */
/* LWE encryption / decryption (Section 2.2: Enc, Dec, Ecd).                 */
/* ------------------------------------------------------------------------- */

uint32_t orc_lwe_phase(int n, const uint32_t *s, const uint32_t *ct)
{
    uint32_t acc = 0;
    for (int i = 0; i < n; i++) acc += ct[i] * s[i];
    return ct[n] - acc;
}

/* ct = (a, <a,s> + mu + e) with mask a and noise e drawn by the caller. */
void orc_lwe_encrypt(int n, const uint32_t *s, const uint32_t *a, uint32_t e, uint32_t mu, uint32_t *ct)
{
    uint32_t acc = 0;
    for (int i = 0; i < n; i++) { ct[i] = a[i]; acc += a[i] * s[i]; }
    ct[n] = acc + mu + e;
}

/* Ecd: m -> m/4 - 1/8, i.e. true = +1/8, false = -1/8. */
uint32_t orc_encode_bit(int m) { return m ? MU_1_8 : (uint32_t)(0u - MU_1_8); }

/* Dec: round the phase to the nearer of +-1/8.  reading: a phase of exactly 0
 * decodes as true (the sign convention of the blind rotation below). */
int orc_lwe_decrypt_bit(int n, const uint32_t *s, const uint32_t *ct)
{
    return (int32_t)orc_lwe_phase(n, s, ct) >= 0;
}

void orc_lwe_trivial(int n, uint32_t mu, uint32_t *ct)
{
    memset(ct, 0, sizeof(uint32_t) * (size_t)n);
    ct[n] = mu;
}

/* NOT c = -c (the phase changes sign, so +-1/8 swap). Free: no bootstrap. */
void orc_lwe_not(int n, const uint32_t *c, uint32_t *out)
{
    for (int i = 0; i <= n; i++) out[i] = 0u - c[i];
}

/* ------------------------------------------------------------------------- */
/* Key generation from caller-supplied randomness (Section 2.2 KeyGen).      */
/* ------------------------------------------------------------------------- */

/* BK_i = TRGSW_K(s_i): row r = 2(p-1)+q holds (a, a*K + e) + s_i*2^(32-bg_bits*p) on component q. */
void orc_keygen_bk(const orc_params *P, const uint32_t *s, const uint32_t *K,
                   const uint32_t *bk_a, const uint32_t *bk_e, uint32_t *bk)
{
    const int n = P->n, N = P->N, l = P->l;
    uint32_t *prod = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    for (int i = 0; i < n; i++) {
        for (int r = 0; r < 2 * l; r++) {
            const uint32_t *a = bk_a + ((size_t)i * 2 * l + r) * N;
            const uint32_t *e = bk_e + ((size_t)i * 2 * l + r) * N;
            uint32_t *ra = bk + (((size_t)i * 2 * l + r) * 2 + 0) * N;
            uint32_t *rb = bk + (((size_t)i * 2 * l + r) * 2 + 1) * N;
            orc_poly_mul_schoolbook(prod, a, K, N);
            for (int k = 0; k < N; k++) { ra[k] = a[k]; rb[k] = prod[k] + e[k]; }
            int p = r / 2 + 1, q = r % 2;
            uint32_t h = s[i] ? (1u << (32 - P->bg_bits * p)) : 0u;
            /* the gadget term is the constant polynomial s_i * h_p */
            if (q == 0) ra[0] += h; else rb[0] += h;
        }
    }
    free(prod);
}

/* KSK[i][j][v] = LWE_s(v * K_i * 2^(32 - B(j+1))), B = ks_base_bits. */
void orc_keygen_ksk(const orc_params *P, const uint32_t *s, const uint32_t *K,
                    const uint32_t *ksk_a, const uint32_t *ksk_e, uint32_t *ksk)
{
    const int n = P->n, N = P->N, t = P->ks_t, B = P->ks_base_bits, base = 1 << B;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < t; j++)
            for (int v = 0; v < base; v++) {
                size_t idx = ((size_t)i * t + j) * base + v;
                uint32_t mu = (uint32_t)v * K[i] * (1u << (32 - B * (j + 1)));
                orc_lwe_encrypt(n, s, ksk_a + idx * n, ksk_e[idx], mu, ksk + idx * (n + 1));
            }
}

/* ------------------------------------------------------------------------- */
/* Bootstrapping: BlindRotate, SampleExtract, KeySwitch (Section 2.2; tfhe-2) */
/* ------------------------------------------------------------------------- */

/* Modulus switch to Z_{2N}: round(x * 2N / 2^32) mod 2N, ties rounded up. */
uint32_t orc_modswitch(uint32_t x, int N)
{
    int s = 32 - ilog2(2 * N);
    return ((x + (1u << (s - 1))) >> s) & (uint32_t)(2 * N - 1);
}

/* Balanced gadget decomposition: digits d_1..d_l in [-Bg/2, Bg/2) with
 * sum_p d_p 2^(32 - bg_bits*p) equal to x rounded to the nearest multiple of
 * 2^(32 - l*bg_bits) (ties up).  d_1 is the most significant digit.
 * Pin: |sum - x| <= 2^(31 - l*bg_bits), digit range. */
void orc_decompose(const orc_params *P, uint32_t x, int32_t *d)
{
    const int l = P->l, bb = P->bg_bits;
    const uint32_t half = 1u << (bb - 1), mask = (1u << bb) - 1;
    uint32_t off = 1u << (32 - l * bb - 1);               /* rounding offset */
    for (int p = 1; p <= l; p++) off += half << (32 - bb * p); /* balancing */
    uint32_t y = x + off;
    for (int p = 1; p <= l; p++)
        d[p - 1] = (int32_t)((y >> (32 - bb * p)) & mask) - (int32_t)half;
}

/* Blind rotation of the LWE sample `lwe` (dimension n) with test vector
 * v = mu * sum_j X^j.  ACC starts as the trivial TRLWE (0, X^(-bbar) v); for
 * i = 0..n-1 in order, ACC <- ACC + ExtProd(BK_i, X^(abar_i) ACC - ACC), where
 * ExtProd decomposes both components of its TRLWE argument and sums the digit
 * polynomials times the matching BK_i rows.  acc = u32[2][N] (a then b).
 * Pin: closed form with a noiseless key encrypting s = 0 (ACC = X^(-bbar) v). */
void orc_blind_rotate(const orc_params *P, const uint32_t *bk, const uint32_t *lwe, uint32_t mu,
                      uint32_t *acc, int use_karatsuba)
{
    const int n = P->n, N = P->N, l = P->l;
    uint32_t *testv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *rot = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *diff = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)N);
    uint32_t *dig = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)l * N);
    uint32_t *prod = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    int32_t dd[16];

    for (int k = 0; k < N; k++) testv[k] = mu;
    uint32_t bbar = orc_modswitch(lwe[n], N);
    memset(acc, 0, sizeof(uint32_t) * (size_t)N);                    /* a(X) = 0 */
    orc_poly_mul_xe(acc + N, testv, -(int)bbar, N);                  /* b(X) = X^-bbar v */

    for (int i = 0; i < n; i++) {
        uint32_t abar = orc_modswitch(lwe[i], N);
        /* X^abar * ACC - ACC, both components */
        for (int q = 0; q < 2; q++) {
            orc_poly_mul_xe(rot, acc + (size_t)q * N, (int)abar, N);
            for (int k = 0; k < N; k++) diff[(size_t)q * N + k] = rot[k] - acc[(size_t)q * N + k];
        }
        /* digit polynomials: row r = 2(p-1)+q */
        for (int q = 0; q < 2; q++)
            for (int k = 0; k < N; k++) {
                orc_decompose(P, diff[(size_t)q * N + k], dd);
                for (int p = 1; p <= l; p++)
                    dig[((size_t)2 * (p - 1) + q) * N + k] = (uint32_t)dd[p - 1];
            }
        /* ACC_j += sum_r dig_r * BK_i[r][j] */
        for (int j = 0; j < 2; j++)
            for (int r = 0; r < 2 * l; r++) {
                const uint32_t *row = bk + (((size_t)i * 2 * l + r) * 2 + j) * N;
                if (use_karatsuba) orc_poly_mul_karatsuba(prod, dig + (size_t)r * N, row, N);
                else orc_poly_mul_schoolbook(prod, dig + (size_t)r * N, row, N);
                for (int k = 0; k < N; k++) acc[(size_t)j * N + k] += prod[k];
            }
    }
    free(testv); free(rot); free(diff); free(dig); free(prod);
}

/* LWE of dimension N under the flattened key (K_0..K_{N-1}) whose phase is
 * coefficient 0 of the TRLWE phase: a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0.
 * Pin: phase invariant on random TRLWE samples. */
void orc_sample_extract(int N, const uint32_t *acc, uint32_t *big)
{
    big[0] = acc[0];
    for (int j = 1; j < N; j++) big[j] = 0u - acc[N - j];
    big[N] = acc[N];
}

/* Key switch from dimension N (key K) to dimension n (key s): round each a'_i
 * to t*B bits, take its base-2^B digits d_ij (j = 0 most significant), and
 * return (0, b') - sum over d_ij != 0 of KSK[i][j][d_ij].
 * Pin: closed form with a noiseless KSK. */
void orc_key_switch(const orc_params *P, const uint32_t *ksk, const uint32_t *big, uint32_t *out)
{
    const int n = P->n, N = P->N, t = P->ks_t, B = P->ks_base_bits, base = 1 << B;
    const uint32_t round_off = 1u << (32 - t * B - 1);
    memset(out, 0, sizeof(uint32_t) * (size_t)n);
    out[n] = big[N];
    for (int i = 0; i < N; i++) {
        uint32_t abar = big[i] + round_off;
        for (int j = 0; j < t; j++) {
            uint32_t d = (abar >> (32 - B * (j + 1))) & (uint32_t)(base - 1);
            if (d == 0) continue;
            const uint32_t *row = ksk + ((((size_t)i * t + j) * base + d) * (size_t)(n + 1));
            for (int k = 0; k <= n; k++) out[k] -= row[k];
        }
    }
}

/* Bootstrap(c) = KeySwitch(SampleExtract(BlindRotate(c, mu = 1/8))). */
void orc_bootstrap(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                   const uint32_t *in, uint32_t *out)
{
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)P->N);
    uint32_t *big = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)P->N + 1));
    orc_blind_rotate(P, bk, in, MU_1_8, acc, 1);
    orc_sample_extract(P->N, acc, big);
    orc_key_switch(P, ksk, big, out);
    free(acc); free(big);
}

/* ------------------------------------------------------------------------- */
/* Gates (Section 2.2: HomAND = Bootstrap((0,-1/8)+ct1+ct2); the other       */
/* binary gates are tfhe-2's linear pre-combinations under the same Ecd).    */
/* ------------------------------------------------------------------------- */

/* c = T(const) + s1*c1 + s2*c2 for the ten binary gates. */
static void gate_combination(int gate, uint32_t *cst, int32_t *s1, int32_t *s2)
{
    switch (gate) {
    case ORC_AND:   *cst = 0u - MU_1_8; *s1 = 1;  *s2 = 1;  break;
    case ORC_NAND:  *cst = MU_1_8;      *s1 = -1; *s2 = -1; break;
    case ORC_OR:    *cst = MU_1_8;      *s1 = 1;  *s2 = 1;  break;
    case ORC_NOR:   *cst = 0u - MU_1_8; *s1 = -1; *s2 = -1; break;
    case ORC_XOR:   *cst = MU_1_4;      *s1 = 2;  *s2 = 2;  break;
    case ORC_XNOR:  *cst = 0u - MU_1_4; *s1 = -2; *s2 = -2; break;
    case ORC_ANDNY: *cst = 0u - MU_1_8; *s1 = -1; *s2 = 1;  break;
    case ORC_ANDYN: *cst = 0u - MU_1_8; *s1 = 1;  *s2 = -1; break;
    case ORC_ORNY:  *cst = MU_1_8;      *s1 = -1; *s2 = 1;  break;
    case ORC_ORYN:  *cst = MU_1_8;      *s1 = 1;  *s2 = -1; break;
    default:        *cst = 0; *s1 = 0; *s2 = 0; break;
    }
}

void orc_gate_combine(int n, int gate, const uint32_t *c1, const uint32_t *c2, uint32_t *out)
{
    uint32_t cst; int32_t s1, s2;
    gate_combination(gate, &cst, &s1, &s2);
    for (int i = 0; i <= n; i++) out[i] = (uint32_t)s1 * c1[i] + (uint32_t)s2 * c2[i];
    out[n] += cst;
}

/* MUX(c, a, b) = c ? a : b: two blind rotations (AND(c,a) and AND(NOT c, b)),
 * both extracted, summed with T(1/8), one key switch (tfhe-2's construction;
 * the argument order follows the proof of HomCompLE in the paper's appendix). */
void orc_gate(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int gate,
              const uint32_t *c1, const uint32_t *c2, const uint32_t *c3, uint32_t *out)
{
    const int n = P->n, N = P->N;
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (gate != ORC_MUX) {
        orc_gate_combine(n, gate, c1, c2, tmp);
        orc_bootstrap(P, bk, ksk, tmp, out);
    } else {
        uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)N);
        uint32_t *big1 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)N + 1));
        uint32_t *big2 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)N + 1));
        for (int i = 0; i < n; i++) tmp[i] = c1[i] + c2[i];
        tmp[n] = c1[n] + c2[n] - MU_1_8;
        orc_blind_rotate(P, bk, tmp, MU_1_8, acc, 1);
        orc_sample_extract(N, acc, big1);
        for (int i = 0; i < n; i++) tmp[i] = (0u - c1[i]) + c3[i];
        tmp[n] = (0u - c1[n]) + c3[n] - MU_1_8;
        orc_blind_rotate(P, bk, tmp, MU_1_8, acc, 1);
        orc_sample_extract(N, acc, big2);
        for (int i = 0; i <= N; i++) big1[i] += big2[i];
        big1[N] += MU_1_8;
        orc_key_switch(P, ksk, big1, out);
        free(acc); free(big1); free(big2);
    }
    free(tmp);
}

/* Independent gates of one layer, OpenMP over gates.  in = [count][arity][n+1]. */
void orc_gate_batch(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int gate,
                    const uint32_t *in, uint32_t *out, int64_t count, int nthreads)
{
    const int n1 = P->n + 1, ar = (gate == ORC_MUX) ? 3 : 2;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t g = 0; g < count; g++) {
        const uint32_t *c = in + (size_t)g * ar * n1;
        orc_gate(P, bk, ksk, gate, c, c + n1, ar == 3 ? c + 2 * n1 : NULL, out + (size_t)g * n1);
    }
}

/* ------------------------------------------------------------------------- */
/* Circuits of the three modes with a plaintext database.                    */
/* Bits are LSB first: ct[i] encrypts bit i, ct[l-1] is the top (sign) bit.  */
/* ------------------------------------------------------------------------- */

/* XNOR against a plaintext bit c is free: c ? x : NOT x. */
static void xnor_plain(int n, const uint32_t *x, int c, uint32_t *out)
{
    if (c) memcpy(out, x, sizeof(uint32_t) * (size_t)(n + 1));
    else orc_lwe_not(n, x, out);
}

static void gate2(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int gate,
                  const uint32_t *c1, const uint32_t *c2, uint32_t *out)
{
    orc_gate(P, bk, ksk, gate, c1, c2, NULL, out);
}

/* HomEqOPT (Section 5, Alg. HomEqOPT) with the second operand a plaintext
 * value: t[i] = XNOR(x_i, v_i) (free), then the pairwise AND reduction
 * t[i] = AND(t[i], t[i+k]) for k = 1, 2, 4, ... and i = 0, 2k, 4k, ... with
 * i + k < l; the result is t[0].  l - 1 bootstraps. */
void orc_eq_plain(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                  const uint32_t *x, int l, uint64_t v, uint32_t *out)
{
    const int n1 = P->n + 1;
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)l * n1);
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    for (int i = 0; i < l; i++) xnor_plain(P->n, x + (size_t)i * n1, (int)((v >> i) & 1), t + (size_t)i * n1);
    for (int k = 1; k < l; k *= 2)
        for (int i = 0; i + k < l; i += 2 * k) {
            gate2(P, bk, ksk, ORC_AND, t + (size_t)i * n1, t + (size_t)(i + k) * n1, r);
            memcpy(t + (size_t)i * n1, r, sizeof(uint32_t) * (size_t)n1);
        }
    memcpy(out, t, sizeof(uint32_t) * (size_t)n1);
    free(t); free(r);
}

/* HomEqOPT with both operands encrypted (bootstrapped XNORs): the paper's
 * encrypted-database form. */
void orc_eq_enc(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                const uint32_t *x, const uint32_t *y, int l, uint32_t *out)
{
    const int n1 = P->n + 1;
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)l * n1);
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    for (int i = 0; i < l; i++) gate2(P, bk, ksk, ORC_XNOR, x + (size_t)i * n1, y + (size_t)i * n1, t + (size_t)i * n1);
    for (int k = 1; k < l; k *= 2)
        for (int i = 0; i + k < l; i += 2 * k) {
            gate2(P, bk, ksk, ORC_AND, t + (size_t)i * n1, t + (size_t)(i + k) * n1, r);
            memcpy(t + (size_t)i * n1, r, sizeof(uint32_t) * (size_t)n1);
        }
    memcpy(out, t, sizeof(uint32_t) * (size_t)n1);
    free(t); free(r);
}

/* HomCompLeOPT / HomCompL (Section 4 Alg. HomCompLE, HomCompL; Section 5 Alg.
 * HomCompLeOPT) with all operands encrypted: t0 = XOR(ct1_top, ct2_top);
 * t1 = T(+1/8) for <= or T(-1/8) for <; t_xnor[i] = XNOR(ct1[i], ct2[i]);
 * t1 = MUX(t_xnor[i], t1, ct2[i]) for i = 0..l-2; r = MUX(t0, ct1_top, t1).
 * The comparison is signed two's complement (proof of Theorem comple). */
void orc_comp_enc(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                  const uint32_t *c1, const uint32_t *c2, int l, int strict, uint32_t *out)
{
    const int n = P->n, n1 = n + 1;
    uint32_t *t0 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    uint32_t *t1 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    uint32_t *tx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)l * n1);
    gate2(P, bk, ksk, ORC_XOR, c1 + (size_t)(l - 1) * n1, c2 + (size_t)(l - 1) * n1, t0);
    orc_lwe_trivial(n, strict ? 0u - MU_1_8 : MU_1_8, t1);
    for (int i = 0; i <= l - 2; i++)
        gate2(P, bk, ksk, ORC_XNOR, c1 + (size_t)i * n1, c2 + (size_t)i * n1, tx + (size_t)i * n1);
    for (int i = 0; i <= l - 2; i++) {
        orc_gate(P, bk, ksk, ORC_MUX, tx + (size_t)i * n1, t1, c2 + (size_t)i * n1, r);
        memcpy(t1, r, sizeof(uint32_t) * (size_t)n1);
    }
    orc_gate(P, bk, ksk, ORC_MUX, t0, c1 + (size_t)(l - 1) * n1, t1, out);
    free(t0); free(t1); free(r); free(tx);
}

/* The same comparators with one plaintext operand, every XNOR and every MUX
 * reduced to a single gate by case analysis of c ? a : b (reading: an exact
 * rewrite of Alg. HomCompLeOPT for a plaintext database; see the brute-force
 * pins).  t1 starts as a trivial ciphertext and the first ripple gate is a
 * real bootstrap.
 *   plain_first = 1: compute  a <= x  (a plaintext, x encrypted)  [HomCompLE(a, x)]
 *                    ripple: a_i = 0 -> t = OR(x_i, t);  a_i = 1 -> t = AND(x_i, t)
 *                    final : a_top = 0 -> ANDNY(x_top, t); a_top = 1 -> ORNY(x_top, t)
 *   plain_first = 0: compute  x < b  (x encrypted, b plaintext)   [HomCompL(x, b)]
 *                    ripple: b_i = 0 -> t = ANDNY(x_i, t); b_i = 1 -> t = ORNY(x_i, t)
 *                    final : b_top = 0 -> OR(x_top, t);   b_top = 1 -> AND(x_top, t)
 * strict selects < (t starts at T(-1/8)) or <= (T(+1/8)).
 * is_unsigned: compare as unsigned integers by flipping the top bit on both
 * sides (reading: the paper's comparator is signed; the workloads are unsigned). */
void orc_comp_plain(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                    const uint32_t *x, uint64_t plain, int l, int plain_first, int strict,
                    int is_unsigned, uint32_t *out)
{
    const int n = P->n, n1 = n + 1;
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    uint32_t *top = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
    if (is_unsigned) {
        plain ^= (uint64_t)1 << (l - 1);
        orc_lwe_not(n, x + (size_t)(l - 1) * n1, top);
    } else {
        memcpy(top, x + (size_t)(l - 1) * n1, sizeof(uint32_t) * (size_t)n1);
    }
    orc_lwe_trivial(n, strict ? 0u - MU_1_8 : MU_1_8, t);
    for (int i = 0; i <= l - 2; i++) {
        int bit = (int)((plain >> i) & 1);
        int g = plain_first ? (bit ? ORC_AND : ORC_OR) : (bit ? ORC_ORNY : ORC_ANDNY);
        gate2(P, bk, ksk, g, x + (size_t)i * n1, t, r);
        memcpy(t, r, sizeof(uint32_t) * (size_t)n1);
    }
    int tb = (int)((plain >> (l - 1)) & 1);
    int g = plain_first ? (tb ? ORC_ORNY : ORC_ANDNY) : (tb ? ORC_AND : ORC_OR);
    gate2(P, bk, ksk, g, top, t, out);
    free(t); free(r); free(top);
}

/* IntV (Alg. InterValid): v = AND(AND(LE(x_lo, x), L(x, x_hi)), AND(LE(y_lo, y), L(y, y_hi))),
 * half-open intervals x_lo <= x < x_hi; rect = {x_lo, x_hi, y_lo, y_hi}. */
void orc_intv_entry(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                    const uint32_t *cx, const uint32_t *cy, int l, const uint64_t *rect,
                    int is_unsigned, uint32_t *out)
{
    const int n1 = P->n + 1;
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * 6 * (size_t)n1);
    orc_comp_plain(P, bk, ksk, cx, rect[0], l, 1, 0, is_unsigned, v + 0 * n1); /* x_lo <= x */
    orc_comp_plain(P, bk, ksk, cx, rect[1], l, 0, 1, is_unsigned, v + 1 * (size_t)n1); /* x < x_hi */
    orc_comp_plain(P, bk, ksk, cy, rect[2], l, 1, 0, is_unsigned, v + 2 * (size_t)n1); /* y_lo <= y */
    orc_comp_plain(P, bk, ksk, cy, rect[3], l, 0, 1, is_unsigned, v + 3 * (size_t)n1); /* y < y_hi */
    gate2(P, bk, ksk, ORC_AND, v + 0, v + (size_t)n1, v + 4 * (size_t)n1);                  /* v_x */
    gate2(P, bk, ksk, ORC_AND, v + 2 * (size_t)n1, v + 3 * (size_t)n1, v + 5 * (size_t)n1); /* v_y */
    gate2(P, bk, ksk, ORC_AND, v + 4 * (size_t)n1, v + 5 * (size_t)n1, out);               /* v   */
    free(v);
}

/* CoV (Alg. CoV) on an encrypted cell (bits 0..w-1 = x, bits w..2w-1 = y)
 * against plaintext (x, y): AND(EQ_w(x, loc_x), EQ_w(y, loc_y)). */
void orc_cov_entry(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                   const uint32_t *cell, int w, uint64_t loc_x, uint64_t loc_y, uint32_t *out)
{
    const int n1 = P->n + 1;
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)n1);
    orc_eq_plain(P, bk, ksk, cell, w, loc_x, v);
    orc_eq_plain(P, bk, ksk, cell + (size_t)w * n1, w, loc_y, v + n1);
    gate2(P, bk, ksk, ORC_AND, v, v + n1, out);
    free(v);
}

/* Batched entries, OpenMP over independent database entries. */
void orc_idm_batch(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                   const uint32_t *x, int l, const uint64_t *ids, int64_t D, uint32_t *out, int nthreads)
{
    const int n1 = P->n + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t d = 0; d < D; d++) orc_eq_plain(P, bk, ksk, x, l, ids[d], out + (size_t)d * n1);
}

void orc_intv_batch(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                    const uint32_t *cx, const uint32_t *cy, int l, const uint64_t *rects, int64_t D,
                    int is_unsigned, uint32_t *out, int nthreads)
{
    const int n1 = P->n + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t d = 0; d < D; d++)
        orc_intv_entry(P, bk, ksk, cx, cy, l, rects + 4 * (size_t)d, is_unsigned, out + (size_t)d * n1);
}

void orc_cov_batch(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                   const uint32_t *cell, int w, const uint64_t *locs /* [D][2] */, int64_t D,
                   uint32_t *out, int nthreads)
{
    const int n1 = P->n + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t d = 0; d < D; d++)
        orc_cov_entry(P, bk, ksk, cell, w, locs[2 * d], locs[2 * d + 1], out + (size_t)d * n1);
}

/* Zero-out with a plaintext payload bit (Alg. HomBitwiseAND with a trivial
 * second operand): AND(v, Enc(1)) = v, AND(v, Enc(0)) = Enc(0); reading: no
 * bootstrap is spent, the result is v itself or the trivial T(-1/8). */
void orc_zero_out_plain(int n, const uint32_t *v, int bit, uint32_t *out)
{
    if (bit) memcpy(out, v, sizeof(uint32_t) * (size_t)(n + 1));
    else orc_lwe_trivial(n, 0u - MU_1_8, out);
}

/* HomSum by the pairwise XOR reduction of Section 5 (Outermost optimisation,
 * aggregation via HomSum): for k = 1, 2, 4, ... and i = 0, 2k, ... with
 * i + k < M: S_i[j] = XOR(S_i[j], S_{i+k}[j]) for every bit j.  S = [M][lS][n+1],
 * reduced in place; the result is S_0.  Within one k, independent gates run
 * under OpenMP. */
void orc_homsum_tree(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                     uint32_t *S, int64_t M, int lS, int nthreads)
{
    const int n1 = P->n + 1;
    for (int64_t k = 1; k < M; k *= 2) {
        int64_t pairs = (M - k + 2 * k - 1) / (2 * k);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t w = 0; w < pairs * lS; w++) {
            int64_t i = (w / lS) * 2 * k;
            int j = (int)(w % lS);
            if (i + k >= M) continue;
            uint32_t *a = S + ((size_t)i * lS + j) * n1;
            const uint32_t *b = S + ((size_t)(i + k) * lS + j) * n1;
            uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n1);
            gate2(P, bk, ksk, ORC_XOR, a, b, r);
            memcpy(a, r, sizeof(uint32_t) * (size_t)n1);
            free(r);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* A gate given by its linear pre-combinations.                              */
/* ------------------------------------------------------------------------- */

/* Section 2.2 writes a bootstrapped gate as Bootstrap(T(c) + a linear
 * combination of its input ciphertexts); tfhe-2's MUX blind-rotates two such
 * combinations and sums their extractions before one key switch.  This is
 * that definition with the combination spelled out: rotation r < nrot
 * blind-rotates c_r = sum_{k < nin} coef[r][k] * in_k + T(cst[r]) (test
 * vector 1/8) and extracts it; the extractions are summed, T(ks_cst) is
 * added to b, and the sum is key-switched.  coef = [2][8], in = [nin][n+1].
 * Pin: decryption against the sign of the noiseless combined phase, and
 * equality with orc_gate for the ten gates and MUX. */
void orc_gate_linear(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int nrot, int nin,
                     const int32_t *coef, const uint32_t *cst, const uint32_t *in, uint32_t ks_cst,
                     uint32_t *out)
{
    const int n = P->n, N = P->N;
    uint32_t *c = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)N);
    uint32_t *big = (uint32_t *)calloc((size_t)N + 1, sizeof(uint32_t));
    uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)N + 1));
    for (int r = 0; r < nrot; r++) {
        memset(c, 0, sizeof(uint32_t) * ((size_t)n + 1));
        for (int k = 0; k < nin; k++)
            for (int i = 0; i <= n; i++) c[i] += (uint32_t)coef[r * 8 + k] * in[(size_t)k * (n + 1) + i];
        c[n] += cst[r];
        orc_blind_rotate(P, bk, c, MU_1_8, acc, 1);
        orc_sample_extract(N, acc, ext);
        for (int i = 0; i <= N; i++) big[i] += ext[i];
    }
    big[N] += ks_cst;
    orc_key_switch(P, ksk, big, out);
    free(c); free(acc); free(big); free(ext);
}

/* Independent linear gates, OpenMP over gates.  nrot, nin, ks_cst = [count];
 * coef = [count][2][8]; cst = [count][2]; in = [count][8][n+1]. */
void orc_gate_linear_batch(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int64_t count,
                           const int32_t *nrot, const int32_t *nin, const int32_t *coef, const uint32_t *cst,
                           const uint32_t *ks_cst, const uint32_t *in, uint32_t *out, int nthreads)
{
    const int n1 = P->n + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t g = 0; g < count; g++)
        orc_gate_linear(P, bk, ksk, nrot[g], nin[g], coef + g * 16, cst + g * 2, in + (size_t)g * 8 * n1, ks_cst[g],
                        out + (size_t)g * n1);
}

/* ------------------------------------------------------------------------- */
/* Fan-in-g HomSum (a cheaper variant of the Section 5 aggregation).         */
/* ------------------------------------------------------------------------- */

/* XOR of g bits with one bootstrap.  Reading: with Ecd's +-1/8, the sum of g
 * encodings of which t are true is (2t - g)/8; doubled, each true input moves
 * it by 1/2, so 2 * sum_k c_k + T((g-1)/4) has phase +1/4 for odd t and -1/4
 * for even t (mod 1), and the blind rotation's sign test returns Enc(t mod 2).
 * g = 2 is tfhe-2's XOR gate T(1/4) + 2(c1 + c2).  The input noise is doubled
 * against a margin of 1/4 (the same ratio as a two-input gate's 1/8), and
 * grows as sqrt(g).  in = [g][n+1].
 * Pin: decryption of every input pattern, equality with the XOR gate at
 * g = 2, and the measured pre-bootstrap noise against the variance bound. */
void orc_xor_many(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, const uint32_t *in, int g,
                  uint32_t *out)
{
    const int n = P->n;
    uint32_t *c = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    for (int k = 0; k < g; k++)
        for (int i = 0; i <= n; i++) c[i] += 2u * in[(size_t)k * (n + 1) + i];
    c[n] += (uint32_t)(g - 1) * MU_1_4;
    orc_bootstrap(P, bk, ksk, c, out);
    free(c);
}

/* HomSum with fan-in g: for k = 1, g, g^2, ... and i = 0, gk, 2gk, ...:
 * S_i[j] = XOR of S_{i + m k}[j] over the m < g with i + m k < M (when there
 * are at least two), every bit j.  S = [M][lS][n+1], reduced in place; the
 * result is S_0.  g = 2 is orc_homsum_tree's pairing exactly.  Within one k,
 * independent gates run under OpenMP. */
void orc_homsum_tree_fanin(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, uint32_t *S, int64_t M,
                           int lS, int g, int nthreads)
{
    const int n1 = P->n + 1;
    for (int64_t k = 1; k < M; k *= g) {
        const int64_t groups = (M + g * k - 1) / (g * k);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t w = 0; w < groups * lS; w++) {
            const int64_t i = (w / lS) * g * k;
            const int j = (int)(w % lS);
            int m = 0;
            while (m < g && i + m * k < M) m++;
            if (m < 2) continue;
            uint32_t *in = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * n1);
            for (int q = 0; q < m; q++)
                memcpy(in + (size_t)q * n1, S + ((size_t)(i + q * k) * lS + j) * n1, sizeof(uint32_t) * (size_t)n1);
            orc_xor_many(P, bk, ksk, in, m, S + ((size_t)i * lS + j) * n1);
            free(in);
        }
    }
}
