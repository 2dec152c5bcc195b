// hancock32_2d.cu - the 2D FP32-bulk MUSCL-Hancock kernels.  Variants: the
// tile shapes 16 x 15 (256 threads), 32 x 15 (512), 32 x 7 (256); a van Leer
// context and a context with general closures run the 32 x 7 tile.  A tile
// holds its primitives, face slots and evolved edge states in shared memory
// (about 104 KB for 32 x 7 reactive cells): two CTAs of 256 threads per SM.
#include "hancock32_launch.cuh"

using namespace dis;

namespace {
template <bool RX>
void step2(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int v) {
  if (general_closures(c)) {
    hancock32_launch<2, RX, 32, 7, 256, 2, -1, true>(c, st, a, 2);
  } else if (c->phys.limiter) {
    hancock32_launch<2, RX, 32, 7, 256, 2, 1, false>(c, st, a, 2);
  } else if (v == 0) {
    hancock32_launch<2, RX, 16, 15, 256, 2, 0, false>(c, st, a, 0);
  } else if (v == 1) {
    hancock32_launch<2, RX, 32, 15, 512, 1, 0, false>(c, st, a, 1);
  } else {
    hancock32_launch<2, RX, 32, 7, 256, 2, 0, false>(c, st, a, 2);
  }
}
}  // namespace

void hancock32_step_2d(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int v) {
  if (c->y >= 0) step2<true>(c, st, a, v);
  else step2<false>(c, st, a, v);
}
