// query.cuh - device reductions behind dis_query: conserved totals and the
// volume-fraction range of the current state.
//
// Totals of Section 3's conserved quantities (phi_l rho_l, rho u, rho v,
// rho E, phi_y rho_y lam) times the cell volume, and min / max of phi1 over
// every interior cell of every patch.  Deterministic: one CTA per segment
// writes its partial sums (fixed-order tree in shared memory), and one CTA
// then adds the partials in segment order.
#pragma once
#include "step32.cuh"

namespace dis {

constexpr int NQ = 8;  // mass 1, mass 2, x momentum, y momentum, energy, reactant, phi min, phi max

// Cell volume: dx dy (dy = 1 in 1D); cylindrical geometry 2 pi r dx dy.
__device__ __forceinline__ double cell_volume(const PatchDev& pd, int i, int cyl) {
  const double v = pd.dx * pd.dy;
  return cyl ? v * 6.283185307179586 * (pd.x0 + (i + 0.5) * pd.dx) : v;
}

// One CTA of SEG threads per segment; q64 (float64 padded layout) or, if
// null, q32 (FP32-bulk layout, converted through the closures' kappa).
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_query_partial(Phys P, const PatchDev* __restrict__ pds,
                                                       const int4* __restrict__ segs, const double* q64,
                                                       const float* q32, long long T, double* part) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  __shared__ double red[NQ][SEG];
  const int4 g = segs[blockIdx.x];
  const int t = threadIdx.x;
  double v[NQ] = {0, 0, 0, 0, 0, 0, 1e300, -1e300};
  if (t < g.w) {
    const PatchDev pd = pds[g.x];
    const int i = g.z + t, j = g.y;
    const long long k = cidx(pd, i, j);
    double s[NF];
    if (q64) {
#pragma unroll
      for (int c = 0; c < NF; ++c) s[c] = q64[c * T + k];
    } else {
      state32_to_64<DIM, RX>(P, q32, T, k, s);
    }
    const double vol = cell_volume(pd, i, P.cyl);
    v[0] = vol * s[L::A1];
    v[1] = vol * s[L::A2];
    v[2] = vol * s[L::MX];
    if constexpr (DIM == 2) v[3] = vol * s[L::MY];
    v[4] = vol * s[L::E];
    if constexpr (RX) v[5] = vol * s[L::AL];
    v[6] = v[7] = s[L::PHI];
  }
#pragma unroll
  for (int c = 0; c < NQ; ++c) red[c][t] = v[c];
  __syncthreads();
  for (int h = SEG / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int c = 0; c < 6; ++c) red[c][t] += red[c][t + h];
      red[6][t] = fmin(red[6][t], red[6][t + h]);
      red[7][t] = fmax(red[7][t], red[7][t + h]);
    }
    __syncthreads();
  }
  if (t < NQ) part[(long long)blockIdx.x * NQ + t] = red[t][0];
}

// One CTA: the partials of n segments, summed in segment order per thread
// slice, then a fixed-order tree; out[NQ].
__global__ void __launch_bounds__(SEG) k_query_final(const double* part, long long n, double* out) {
  __shared__ double red[NQ][SEG];
  const int t = threadIdx.x;
  double v[NQ] = {0, 0, 0, 0, 0, 0, 1e300, -1e300};
  for (long long b = t; b < n; b += SEG) {
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] += part[b * NQ + c];
    v[6] = fmin(v[6], part[b * NQ + 6]);
    v[7] = fmax(v[7], part[b * NQ + 7]);
  }
#pragma unroll
  for (int c = 0; c < NQ; ++c) red[c][t] = v[c];
  __syncthreads();
  for (int h = SEG / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int c = 0; c < 6; ++c) red[c][t] += red[c][t + h];
      red[6][t] = fmin(red[6][t], red[6][t + h]);
      red[7][t] = fmax(red[7][t], red[7][t + h]);
    }
    __syncthreads();
  }
  if (t < NQ) out[t] = red[t][0];
}

}  // namespace dis
