"""Algorithmic int32 multiply work of the exact-NTT blind rotation, and its
cost on the integer multiply pipe.

Per blind-rotation step (N = 1024, two primes, l = 3 levels x 2 components):
  * 12 forward NTTs (6 digit polynomials x 2 primes) and 4 inverse NTTs
    (2 output polynomials x 2 primes), N/2 * log2(N) = 5,120 butterflies each,
    one Shoup multiplication per butterfly: a high-half product
    floor(x w' / 2^32) and two low-half products (x w, q p) -- except the
    first two stages of each forward NTT, whose multiplicands are 7-bit digits
    (stage 0) or d + psi^512 d' (stage 1): their products are table lookups
    (psi^512 d, psi^256 d, psi^768 d), no multiplication, so a forward NTT
    executes 8 multiplying stages of 512 butterflies;
  * 2 primes x 6 rows x 2 outputs x N pointwise Shoup products against the
    stored key and its companions;
  * 2 x N Chinese-remainder lifts: one Shoup product and one low product
    (p0 t).
Digit decomposition, rotation, additions and the lazy reductions are not
counted: they are not multiplications of the algorithm.

Pipe cost.  32-bit IMAD runs on the FMA pipe's heavy half, 16 lanes per SM
sub-partition per clock (64 per SM).  A high-half multiply (IMAD.HI) holds
that pipe twice as long as a low one: on the NTT kernel, ncu measures the
heavy half busy 83.1% of cycles while FMA-pipe instructions issue at 0.322
per cycle per sub-partition (64.4% if each took two cycles), and the 18.7%
excess equals the high-half share of the kernel's multiplies (29%) at two
extra cycles each.  IMAD_SLOTS counts a low product as one lane-slot of the
64 per SM per clock and a high product as two: the roofline of the kernel is
IMAD_SLOTS_PER_BOOTSTRAP / (152 SMs x 64 x clock).
"""
N = 1024
LOG2N = 10
STEPS = 630
BUTTERFLIES_PER_NTT = N // 2 * LOG2N
LOOKUP_STAGES = 2                                  # forward stages done by table lookups
FWD_NTTS_PER_STEP, INV_NTTS_PER_STEP = 12, 4
POINTWISE_PER_STEP = 2 * 6 * 2 * N
CRT_PER_STEP = 2 * N

SHOUP_PER_STEP = (FWD_NTTS_PER_STEP * (BUTTERFLIES_PER_NTT - LOOKUP_STAGES * N // 2)
                  + INV_NTTS_PER_STEP * BUTTERFLIES_PER_NTT + POINTWISE_PER_STEP + CRT_PER_STEP)
HI_PER_STEP = SHOUP_PER_STEP                       # one high-half product per Shoup multiplication
LO_PER_STEP = 2 * SHOUP_PER_STEP + CRT_PER_STEP    # two low products per Shoup, plus p0 t in the lift

IMAD_OPS_PER_STEP = HI_PER_STEP + LO_PER_STEP
IMAD_OPS_PER_BOOTSTRAP = IMAD_OPS_PER_STEP * STEPS             # 183,214,080 multiplies
HI_SLOTS = 2                                                   # pipe slots of one high-half multiply
IMAD_SLOTS_PER_STEP = HI_SLOTS * HI_PER_STEP + LO_PER_STEP
IMAD_SLOTS_PER_BOOTSTRAP = IMAD_SLOTS_PER_STEP * STEPS         # 243,855,360 lane-slots
DENSE_MACS_PER_BOOTSTRAP = 12 * N * N * STEPS                  # 7,927,234,560
