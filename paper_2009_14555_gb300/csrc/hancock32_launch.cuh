// hancock32_launch.cuh - launchers of the FP32-bulk MUSCL-Hancock kernels
// (instantiated per dimension in hancock32_1d.cu and hancock32_2d.cu, so the
// two compile in parallel).
#pragma once
#include "ctx.cuh"
#include "hancock32.cuh"

namespace dis {

template <int DIM, bool RX, int TX, int TY, int NT, int MINB, int LIM, bool GEN>
void hancock32_launch(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int shape) {
  constexpr size_t smem = hancock32_smem<DIM, RX, TX, TY>();
  static_assert(smem <= 227 * 1024, "shared memory of one CTA");
  static bool attr_set = false;  // per instantiation, per process
  if (!attr_set) {
    cudaFuncSetAttribute(k_hancock32<DIM, RX, TX, TY, NT, MINB, LIM, GEN>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_hancock32<DIM, RX, TX, TY, NT, MINB, LIM, GEN>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_set = true;
  }
  k_hancock32<DIM, RX, TX, TY, NT, MINB, LIM, GEN><<<(unsigned)c->tiles[shape].size(), NT, smem, st>>>(
      c->phys, c->physf, a, c->d_tiles[shape]);
}

template <bool RX, int TX, int NT, int MINB, int LIM, bool GEN>
void hancock32_batch_launch(dis_ctx* c, cudaStream_t st, const StepArgs32& a, float* q0, float* q1, int n,
                            int scratch, int shape) {
  constexpr size_t smem = hancock32_smem<1, RX, TX, 1>();
  static bool attr_set = false;  // per instantiation, per process
  if (!attr_set) {
    cudaFuncSetAttribute(k_hbatch32<RX, TX, NT, MINB, LIM, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_hbatch32<RX, TX, NT, MINB, LIM, GEN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         100);
    attr_set = true;
  }
  Bufs32 b;
  b.q[0] = q0;
  b.q[1] = q1;
  b.q[2] = nullptr;
  k_hbatch32<RX, TX, NT, MINB, LIM, GEN><<<(unsigned)c->np, NT, smem, st>>>(
      c->phys, c->physf, a, b, c->rate, c->d_order, c->d_tile0[shape], c->d_tiles[shape], n, scratch,
      c->rate_valid ? 1 : 0);
}

}  // namespace dis
