// hancock32_1d.cu - the 1D FP32-bulk MUSCL-Hancock kernels: per-step launches
// over the tiles of all problems and the persistent batch form (one CTA per
// problem, all steps of a call).  Variants: tiles of 122, 250, 506 cells
// (128, 256, 512 threads); a van Leer context and a context with general
// closures run the 250-cell tile.
#include "hancock32_launch.cuh"

using namespace dis;

namespace {
template <bool RX>
void step1(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int v) {
  if (general_closures(c)) {
    hancock32_launch<1, RX, 250, 1, 256, 1, -1, true>(c, st, a, 1);
  } else if (c->phys.limiter) {
    hancock32_launch<1, RX, 250, 1, 256, 1, 1, false>(c, st, a, 1);
  } else if (v == 0) {
    hancock32_launch<1, RX, 122, 1, 128, 1, 0, false>(c, st, a, 0);
  } else if (v == 1) {
    hancock32_launch<1, RX, 250, 1, 256, 1, 0, false>(c, st, a, 1);
  } else {
    hancock32_launch<1, RX, 506, 1, 512, 1, 0, false>(c, st, a, 2);
  }
}

template <bool RX>
void batch1(dis_ctx* c, cudaStream_t st, const StepArgs32& a, float* q0, float* q1, int n, int scratch, int v) {
  if (general_closures(c)) {
    hancock32_batch_launch<RX, 250, 256, 1, -1, true>(c, st, a, q0, q1, n, scratch, 1);
  } else if (c->phys.limiter) {
    hancock32_batch_launch<RX, 250, 256, 1, 1, false>(c, st, a, q0, q1, n, scratch, 1);
  } else if (v == 0) {
    hancock32_batch_launch<RX, 122, 128, 1, 0, false>(c, st, a, q0, q1, n, scratch, 0);
  } else if (v == 1) {
    hancock32_batch_launch<RX, 250, 256, 1, 0, false>(c, st, a, q0, q1, n, scratch, 1);
  } else {
    hancock32_batch_launch<RX, 506, 512, 1, 0, false>(c, st, a, q0, q1, n, scratch, 2);
  }
}
}  // namespace

void hancock32_step_1d(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int v) {
  if (c->y >= 0) step1<true>(c, st, a, v);
  else step1<false>(c, st, a, v);
}

void hancock32_batch_1d(dis_ctx* c, cudaStream_t st, const StepArgs32& a, float* q0, float* q1, int n,
                        int scratch, int v) {
  if (c->y >= 0) batch1<true>(c, st, a, q0, q1, n, scratch, v);
  else batch1<false>(c, st, a, q0, q1, n, scratch, v);
}
