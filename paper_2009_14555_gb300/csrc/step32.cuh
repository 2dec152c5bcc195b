// step32.cuh - kernels of the FP32-bulk step (sm_103a).
//
// State: the volume fraction phi1 and the total energy rho E are float64
// planes (q64: plane 0 = phi1, plane 1 = rho E); every other conservative
// field is a float32 plane (q32, indexed by the same field slots as the
// float64 layout; the phi1 and rho E slots are unused).  Primitives and face
// data are float32.  Float64 is used where cancellation needs it:
//   * recovery: p = [rho E - KE - kappa(phi) - soft reference] / xi with the
//     bracket in float64 (kappa(phi) = kappa_1 phi1 + kappa_2 (1 - phi1) reaches
//     1e11 J/m^3 against a thermal part of 1e5);
//   * update: phi1 and rho E accumulate in float64; the energy flux is
//     F_soft + kappa_2 X + (kappa_1 - kappa_2) phi_K X, the kappa part formed in
//     float64 from the same float face values phi_K, X that the phi1 flux uses;
//   * the plastic update runs in float64 in mixed cells (1e-3 < phi1 < 1 - 1e-3).
#pragma once
#include "physics32.cuh"
#include "step_kernels.cuh"

namespace dis {

struct StepArgs32 {
  const PatchDev* pd;
  long long T, NFX, NFY;
  const double* q64src;
  const float* q32src;
  const double* q64n;
  const float* q32n;
  double* q64dst;
  float* q32dst;
  float* W;  // float32 primitives of every padded cell (precomputed-primitive variants, primitive output)
  unsigned long long* rate;
  const double* dtfix;
  double* dtlast;
  int* status;
  double a, b;
  int last;
  double kap2, dkap;  // kappa_2 and kappa_1 - kappa_2 (float64): energy flux kappa part
};

// Primitives of one cell from its FP32-bulk conservative state: phi1 and
// rho E in float64, the other fields in v (float32, conservative slots; the
// phi1 and rho E slots are not read).
template <int DIM, bool RX>
__device__ __forceinline__ PrimF prim32_of(const Phys& P, const PhysF& F, double phi_d, double E,
                                           const float* v) {
  using L = Lay<DIM, RX>;
  PrimF w;
  const float phi = (float)phi_d;
  const float a1 = v[L::A1], a2 = v[L::A2];
  const float rho = a1 + a2;
  const float mx = v[L::MX];
  float my = 0.f;
  if constexpr (DIM == 2) my = v[L::MY];
  w.phi = phi;
  w.r1 = a1 / phi;
  w.r2 = a2 / (float)(1.0 - phi_d);
  const float irho = 1.f / rho;
  w.u = mx * irho;
  w.v = my * irho;
  w.V11 = v[L::V11];
  w.V12 = 0.f;
  w.V21 = 0.f;
  if constexpr (DIM == 2) {
    w.V12 = v[L::V12];
    w.V21 = v[L::V21];
  }
  w.V22 = v[L::V22];
  w.V33 = v[L::V33];
  float arl = 0.f;
  w.lam = 0.f;
  if constexpr (RX) {
    arl = v[L::AL];
    w.lam = arl / (P.y == 0 ? a1 : a2);
  }
  const StrainF s = strain_f(w.V11, w.V12, w.V21, w.V22, w.V33);
  const float KE = 0.5f * (mx * w.u + my * w.v);
  // float64 bracket: (rho E - kappa(phi)) - (KE + soft reference); the small
  // terms are summed in float32
  const double kap = fma(phi_d, P.m[0].kap - P.m[1].kap, P.m[1].kap);
  const double num = (E - kap) - (double)(KE + soft_ref_f(F, phi, a1, a2, arl, s.J2));
  w.p = (float)num / xi_f(F, phi);
  return w;
}

template <int DIM, bool RX>
__device__ __forceinline__ PrimF cons_to_prim32(const Phys& P, const PhysF& F, const double* q64,
                                                const float* q32, long long T, long long k) {
  constexpr int NF = Lay<DIM, RX>::NF;
  float v[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) v[c] = (c == Lay<DIM, RX>::PHI || c == Lay<DIM, RX>::E) ? 0.f : q32[c * T + k];
  return prim32_of<DIM, RX>(P, F, q64[k], q64[T + k], v);
}

template <int DIM, bool RX>
__device__ __forceinline__ void store_prim32(float* W, long long T, long long k, const PrimF& w) {
  using L = Lay<DIM, RX>;
  W[L::PHI * T + k] = w.phi;
  W[L::A1 * T + k] = w.r1;
  W[L::A2 * T + k] = w.r2;
  W[L::MX * T + k] = w.u;
  if constexpr (DIM == 2) W[L::MY * T + k] = w.v;
  W[L::E * T + k] = w.p;
  W[L::V11 * T + k] = w.V11;
  if constexpr (DIM == 2) { W[L::V12 * T + k] = w.V12; W[L::V21 * T + k] = w.V21; }
  W[L::V22 * T + k] = w.V22;
  W[L::V33 * T + k] = w.V33;
  if constexpr (RX) W[L::AL * T + k] = w.lam;
}

// Primitives of every padded cell (ghosts by the index map) into W, and the
// per-patch CFL rate max over interior cells when rate_on.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_prim32(Phys P, PhysF F, StepArgs32 A, const int4* __restrict__ segs,
                                                int rate_on) {
  const int4 g = segs[blockIdx.x];
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x;
  const int j = g.y;
  const bool valid = threadIdx.x < g.w;
  float r = 0.f;
  if (valid) {
    bool fx = false, fy = false;
    const int si = ghost_map(i, pd.nx, pd.bc[0], pd.bc[1], fx);
    const int sj = DIM == 2 ? ghost_map(j, pd.ny, pd.bc[2], pd.bc[3], fy) : 0;
    PrimF w = cons_to_prim32<DIM, RX>(P, F, A.q64src, A.q32src, A.T, cidx(pd, si, sj));
    if (fx) { w.u = -w.u; w.V12 = -w.V12; w.V21 = -w.V21; }
    if (fy) { w.v = -w.v; w.V12 = -w.V12; w.V21 = -w.V21; }
    store_prim32<DIM, RX>(A.W, A.T, cidx(pd, i, j), w);
    if (rate_on && i >= 0 && i < pd.nx && j >= 0 && j < pd.ny) {
      const StrainF s = strain_f(w.V11, w.V12, w.V21, w.V22, w.V33);
      const float rho = w.phi * w.r1 + (1.f - w.phi) * w.r2;
      const float cL2 = cL2_f(F, w.phi, rho, w.p, s.J2);
      if (!(cL2 > 0.f) || !(rho > 0.f)) flag_bad(A.status, g.x, i + pd.nx * j);
      const float cL = sqrtf(fmaxf(cL2, 0.f));
      r = (fabsf(w.u) + cL) / (float)pd.dx;
      if (DIM == 2) r += (fabsf(w.v) + cL) / (float)pd.dy;
    }
  }
  if (rate_on) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0 && r > 0.f)
      atomicMax(A.rate + g.x, (unsigned long long)__double_as_longlong((double)r));
  }
}
// Packed float64 <-> mixed-precision state (interior cells).  Loading from
// primitives goes through the float64 conversion, then rounds the float fields.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_unpack32(Phys P, const PatchDev* __restrict__ pds,
                                                  const int4* __restrict__ segs, const double* src,
                                                  double* q64, float* q32, long long T, int primitive) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
  double v[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) v[c] = src[s0 + c * ncell];
  if (primitive) {
    const double phi = v[L::PHI], r1 = v[L::A1], r2 = v[L::A2];
    const double u = v[L::MX], p = v[L::E];
    double vv = 0.0, v12 = 0.0, v21 = 0.0, arl = 0.0;
    const double a1 = phi * r1, a2 = (1.0 - phi) * r2, rho = a1 + a2;
    if constexpr (DIM == 2) { vv = v[L::MY]; v12 = v[L::V12]; v21 = v[L::V21]; }
    if constexpr (RX) arl = (P.y == 0 ? a1 : a2) * v[L::AL];
    const Strain s = strain_of(v[L::V11], v12, v21, v[L::V22], v[L::V33]);
    v[L::A1] = a1;
    v[L::A2] = a2;
    v[L::MX] = rho * u;
    if constexpr (DIM == 2) v[L::MY] = rho * vv;
    v[L::E] = xi_of(P, phi) * p + ref_energy(P, phi, a1, a2, arl, s.J2) + 0.5 * rho * (u * u + vv * vv);
    if constexpr (RX) v[L::AL] = arl;
  }
#pragma unroll
  for (int c = 0; c < NF; ++c)
    if (c != L::PHI && c != L::E) q32[c * T + k] = (float)v[c];
  q64[k] = v[L::PHI];
  q64[T + k] = v[L::E];
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack32(const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                                                const double* q64, const float* q32, double* dst,
                                                long long T) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
#pragma unroll
  for (int c = 0; c < NF; ++c)
    dst[s0 + c * ncell] = c == L::PHI ? q64[k] : (c == L::E ? q64[T + k] : (double)q32[c * T + k]);
}

// Primitive export (W32 -> packed float64).
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack_w32(const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                                                  const float* W, double* dst, long long T) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
#pragma unroll
  for (int c = 0; c < NF; ++c) dst[s0 + c * ncell] = (double)W[c * T + k];
}

}  // namespace dis
