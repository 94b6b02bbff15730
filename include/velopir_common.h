/*
 * velopir_common.h -- definitions shared by libvelopir.so (velopir.h, the GPU
 * library) and libvelopir_client.so (velopir_client.h, the host-only client
 * library): sizes of the TFHE parameter set, status codes and the parameter
 * record.
 *
 * Paper: "Versatile and Fast Location-Based PIR with FHE over the Torus"
 * (VeLoPIR); parameters from its Appendix table (n = 630, N = 1024, k = 1,
 * l = 3, Bg = 2^7, key-switch base 2^2 with t = 8 levels), uint32 torus
 * (1.0 == 2^32, arithmetic mod 2^32).
 */
#ifndef VELOPIR_COMMON_H
#define VELOPIR_COMMON_H

#include <stdint.h>

#define VELOPIR_LWE_N 630     /* LWE dimension n (Appendix parameter table) */
#define VELOPIR_RING_N 1024   /* polynomial size N (Appendix parameter table) */
#define VELOPIR_LWE_WORDS 631 /* n mask words + b */

enum {
    VELOPIR_OK = 0,
    VELOPIR_ERR_ARG = -1,     /* null pointer, bad size, unknown gate, bad params */
    VELOPIR_ERR_NOKEY = -2,   /* no cloud key loaded on this context */
    VELOPIR_ERR_OOM = -3,     /* request exceeds the HBM budget or cudaMalloc failed */
    VELOPIR_ERR_CUDA = -4,    /* a CUDA runtime call or kernel launch failed */
    VELOPIR_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up */
    VELOPIR_ERR_BUSY = -6,    /* serving queue full / ticket not finished */
    VELOPIR_ERR_NOCUDA = -7,  /* no CUDA device is visible */
    VELOPIR_ERR_PLAN = -8,    /* a dry run found a gate reading a value that was
                                 not yet written or already overwritten */
    VELOPIR_ERR_CANCELLED = -9 /* velopir_poll: the ticket was cancelled */
};

typedef struct {
    int32_t n, N, k, l, bg_bits, ks_t, ks_base_bits; /* must be 630,1024,1,3,7,8,2 */
} velopir_params;

#endif /* VELOPIR_COMMON_H */
