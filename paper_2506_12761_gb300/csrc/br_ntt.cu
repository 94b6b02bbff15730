// Blind rotation with an exact two-prime number-theoretic transform (placeholder
// until the transform kernels land; the path reports itself unavailable).
#include "vp_internal.h"

namespace vp {
size_t bk_ntt_words() { return 0; }
int prepare_bk_ntt(const uint32_t *, uint32_t *, cudaStream_t) { return 0; }
int launch_br_ntt(const BrJob *, int, const uint32_t *, uint32_t *, int *, cudaStream_t) { return 0; }
}  // namespace vp
