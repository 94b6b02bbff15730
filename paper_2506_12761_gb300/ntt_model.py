"""Executed int32 multiply-pipe operation count of the exact-NTT blind rotation.

Per blind-rotation step (N = 1024, two primes, l = 3 levels x 2 components):
  * 12 forward NTTs (6 digit polynomials x 2 primes) and 4 inverse NTTs
    (2 output polynomials x 2 primes), N/2 * log2(N) = 5,120 butterflies each,
    3 multiplies per butterfly (Shoup: high product, two low products);
  * 2 primes x 6 rows x 2 outputs x N pointwise Shoup products against the
    stored key and its companions, 3 multiplies each;
  * 2 x N Chinese-remainder lifts, 5 multiplies each (Shoup 3, 64-bit p0 * t 2).
Digit decomposition and rotation use no multiplies.
"""
N = 1024
LOG2N = 10
STEPS = 630
BUTTERFLIES_PER_NTT = N // 2 * LOG2N
NTTS_PER_STEP = 12 + 4
MUL_PER_BUTTERFLY = 3
POINTWISE_PER_STEP = 2 * 6 * 2 * N
MUL_PER_POINTWISE = 3
CRT_PER_STEP = 2 * N
MUL_PER_CRT = 5

IMAD_OPS_PER_STEP = (NTTS_PER_STEP * BUTTERFLIES_PER_NTT * MUL_PER_BUTTERFLY
                     + POINTWISE_PER_STEP * MUL_PER_POINTWISE + CRT_PER_STEP * MUL_PER_CRT)
IMAD_OPS_PER_BOOTSTRAP = IMAD_OPS_PER_STEP * STEPS
DENSE_MACS_PER_BOOTSTRAP = 12 * N * N * STEPS                # 7,927,234,560
