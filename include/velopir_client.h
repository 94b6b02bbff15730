/*
 * velopir_client.h -- C ABI of libvelopir_client.so, the host-only side of
 * VeLoPIR: key generation, encryption and decryption (Section 2.2: KeyGen,
 * Enc with Ecd: 1 -> 1/8, 0 -> -1/8, Dec by the sign of the phase), and the
 * encrypted-database preprocessing (Alg. PubKeyGen on the client, Alg.
 * ServerEnc on the server).  Plain C++ on the CPU: the library links no CUDA
 * runtime and needs no GPU, so a client that only encrypts queries and
 * decrypts answers never loads the GPU library.
 *
 * Randomness is supplied by the caller (masks, noise integers, key bits), so
 * any seeded generator can drive these functions.  Layouts and status codes
 * as in velopir_common.h; every function returns 0 or VELOPIR_ERR_ARG.
 */
#ifndef VELOPIR_CLIENT_H
#define VELOPIR_CLIENT_H

#include <stddef.h>
#include <stdint.h>

#include "velopir_common.h"

#ifdef __cplusplus
extern "C" {
#endif

/* BK and KSK from: s[630] and K[1024] key bits (0/1), bk_a/bk_e
 * uint32_t[630][6][1024] masks and noise, ksk_a uint32_t[1024][8][4][630],
 * ksk_e uint32_t[1024][8][4].  Outputs in the layouts velopir_load_cloud_key
 * takes.  Errors: ERR_ARG. */
int velopir_client_keygen(const velopir_params *params, const uint32_t *s, const uint32_t *K,
                          const uint32_t *bk_a, const uint32_t *bk_e,
                          const uint32_t *ksk_a, const uint32_t *ksk_e,
                          uint32_t *bk_out, uint32_t *ksk_out);

/* Encrypt `count` bits (Section 2.2 Enc with Ecd): ct_i = (a_i, <a_i,s> + Ecd(bit_i) + e_i).
 * a: uint32_t[count][630], e: uint32_t[count], out: uint32_t[count][631]. */
int velopir_client_encrypt_bits(const uint32_t *s, const uint32_t *bits, const uint32_t *a,
                                const uint32_t *e, size_t count, uint32_t *out);

/* Decrypt `count` ciphertexts (Section 2.2 Dec): bit = phase in [0, 1/2). */
int velopir_client_decrypt_bits(const uint32_t *s, const uint32_t *ct, size_t count, uint32_t *bits_out);

/* Alg. PubKeyGen: count encryptions of zero, pk_i = (a_i, <a_i, s> + e_i).
 * s: uint32_t[630] (0/1), a: uint32_t[count][630] uniform, e: uint32_t[count]
 * noise (torus words), pk_out: uint32_t[count][631].  Host only.  Errors: ERR_ARG. */
int velopir_client_pubkeygen(const uint32_t *s, const uint32_t *a, const uint32_t *e, size_t count,
                             uint32_t *pk_out);

/* Alg. ServerEnc: ct_i = (0, Ecd(bit_i)) + pk_i (Ecd(1) = 1/8, Ecd(0) = -1/8).
 * pk: uint32_t[count][631], bits: uint32_t[count] (0/1), ct_out:
 * uint32_t[count][631].  Host only; uses no secret.  Errors: ERR_ARG. */
int velopir_server_encrypt(const uint32_t *pk, const uint32_t *bits, size_t count, uint32_t *ct_out);

#ifdef __cplusplus
}
#endif
#endif /* VELOPIR_CLIENT_H */
