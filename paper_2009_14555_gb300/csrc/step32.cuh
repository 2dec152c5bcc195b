// step32.cuh - state layout, recovery and conversions of the FP32-bulk step (sm_103a).
//
// State: NF + 1 float32 planes (of T padded cells each), indexed by the field
// slots of the float64 layout, with two changes that keep float64 accuracy
// where the closures cancel:
//   * slot E holds the soft energy e_s = rho E - kappa(phi1), kappa(phi1) =
//     kappa_2 + (kappa_1 - kappa_2) phi1, kappa_l = gamma_l p_inf,l / Gamma_l.
//     kappa reaches 1e11 J/m^3 in a stiff solid against a thermal part of
//     1e5, so rho E itself would need float64; e_s carries only the thermal,
//     kinetic, shear and chemical energy, and the pressure function of
//     Appendix B becomes p = [e_s - KE - soft reference] / xi with no
//     cancellation;
//   * phi1 is a float-float pair (slot PHI the high part, plane NF the low
//     part, about 48 bits): 1 - phi1 of a 1e-8 trace keeps its digits.
// The energy equation is advanced for e_s directly.  With the flux split of
// fused32.cuh (rho E flux = soft flux + kappa(phi_K) X) and the phi1 equation
// (flux phi_K u_face, source phi div u_face), d e_s / dt = d rho E / dt -
// (kappa_1 - kappa_2) d phi1 / dt loses the (kappa_1 - kappa_2) div(phi_K
// u_face) part exactly, in exact arithmetic.  Conversions to and from rho E
// (set/get state) are done once, in float64.
#pragma once
#include "physics32.cuh"
#include "step_kernels.cuh"

namespace dis {

// ---- float-float arithmetic (about 48-bit significands from float32 pairs):
// Knuth's TwoSum, Dekker's Fast2Sum and the fused-multiply-add form of
// Dekker's TwoProduct (exact product error); with float32 denormals flushed
// the error terms of tiny operands are lost, which only matters below 1e-38.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.h, b);
  return fast_two_sum(p.h, fmaf(a.l, b, p.l));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.h, b.h);
  return fast_two_sum(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}
// float-float of a float64 (host or device)
__host__ __device__ __forceinline__ ff ff_of(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}
__host__ __device__ __forceinline__ double ff_val(float h, float l) { return (double)h + (double)l; }

struct StepArgs32 {
  const PatchDev* pd;
  long long T, NFX, NFY;
  const float* src;  // stage source state (NF + 1 planes)
  const float* qn;   // q^n (NF + 1 planes), read when a != 0
  float* dst;        // stage result (NF + 1 planes)
  const unsigned long long* rate;  // per-patch CFL rate of q^n (bits of a positive double)
  unsigned long long* rate_next;   // last stage: per-patch CFL rate of q^{n+1} (atomic max)
  const double* dtfix;
  double* dtlast;
  int* status;
  double a, b;
  int last;
  double dkap;  // kappa_1 - kappa_2 (float64; the e_s source term, the cylindrical energy term)
};

// Primitives of one cell from its FP32-bulk state v (NF + 1 values, slot E =
// e_s, slot PHI and plane NF = phi1 high and low parts).  Also returns
// 1 - phi1 from the float-float pair (the partial density of a trace phase).
template <int DIM, bool RX, bool GEN = true>
__device__ __forceinline__ PrimF prim32_of(const Phys& P, const PhysF& F, const float* v) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  PrimF w;
  const float phi = v[L::PHI];
  const float phi2 = (1.f - phi) - v[NF];  // 1 - phi exact for phi in [1/2, 1]
  const float a1 = v[L::A1], a2 = v[L::A2];
  const float rho = a1 + a2;
  const float mx = v[L::MX];
  float my = 0.f;
  if constexpr (DIM == 2) my = v[L::MY];
  w.phi = phi;
  w.r1 = a1 / phi;
  w.r2 = a2 / phi2;
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
  w.p = (v[L::E] - (KE + soft_ref_f<GEN>(F, phi, a1, a2, arl, s.J2, w.r1, w.r2))) / xi_f(F, phi);
  return w;
}

template <int DIM, bool RX>
__device__ __forceinline__ void load32(const float* q, long long T, long long k, float* v) {
  constexpr int NS = Lay<DIM, RX>::NF + 1;
#pragma unroll
  for (int c = 0; c < NS; ++c) v[c] = q[c * T + k];
}

template <int DIM, bool RX, bool GEN = true>
__device__ __forceinline__ PrimF cons_to_prim32(const Phys& P, const PhysF& F, const float* q, long long T,
                                                long long k) {
  float v[Lay<DIM, RX>::NF + 1];
  load32<DIM, RX>(q, T, k, v);
  return prim32_of<DIM, RX, GEN>(P, F, v);
}

// CFL rate sum_d (|u_d| + c_L) / dx_d of one cell from its primitives; flags
// a cell without a real sound speed or a positive density.
template <int DIM, bool GEN = true>
__device__ __forceinline__ float cfl_rate_of(const PhysF& F, const PrimF& w, float idx, float idy, int* status,
                                             int patch, int cell) {
  const StrainF s = strain_f(w.V11, w.V12, w.V21, w.V22, w.V33);
  const float rho = w.phi * w.r1 + (1.f - w.phi) * w.r2;
  const float cL2 = cL2_f<GEN>(F, w.phi, rho, w.p, s.J2, w.r1, w.r2);
  if (!(cL2 > 0.f) || !(rho > 0.f)) flag_bad(status, patch, cell);
  const float cL = sqrtf(fmaxf(cL2, 0.f));
  float r = (fabsf(w.u) + cL) * idx;
  if (DIM == 2) r += (fabsf(w.v) + cL) * idy;
  return r;
}

// Float64 state (packed layout) <-> FP32-bulk state (interior cells).  From
// primitives the conservative state is formed in float64 first; rho E becomes
// e_s = rho E - kappa(phi1) in float64 before rounding.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_unpack32(Phys P, const PatchDev* __restrict__ pds,
                                                  const int4* __restrict__ segs, const double* src, float* q,
                                                  long long T, int primitive, long long base = 0) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff - base + (long long)j * pd.nx + i;
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
  const double kap = P.m[1].kap + (P.m[0].kap - P.m[1].kap) * v[L::PHI];
  const ff ph = ff_of(v[L::PHI]);
#pragma unroll
  for (int c = 0; c < NF; ++c)
    q[c * T + k] = c == L::PHI ? ph.h : (float)(c == L::E ? v[c] - kap : v[c]);
  q[NF * T + k] = ph.l;
}

// FP32-bulk state -> float64 conservative state; out_packed selects the
// packed (interior-only) layout, else the padded layout of the float64 step.
template <int DIM, bool RX>
__device__ __forceinline__ void state32_to_64(const Phys& P, const float* q, long long T, long long k,
                                              double* v) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
#pragma unroll
  for (int c = 0; c < NF; ++c) v[c] = (double)q[c * T + k];
  v[L::PHI] = ff_val(q[L::PHI * T + k], q[NF * T + k]);
  v[L::E] += P.m[1].kap + (P.m[0].kap - P.m[1].kap) * v[L::PHI];
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack32(Phys P, const PatchDev* __restrict__ pds,
                                                const int4* __restrict__ segs, const float* q, double* dst,
                                                long long T, long long base = 0) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff - base + (long long)j * pd.nx + i;
  double v[NF];
  state32_to_64<DIM, RX>(P, q, T, cidx(pd, i, j), v);
#pragma unroll
  for (int c = 0; c < NF; ++c) dst[s0 + c * ncell] = v[c];
}

// Primitive export: the float32 primitives of every interior cell, packed.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack_prim32(Phys P, PhysF F, const PatchDev* __restrict__ pds,
                                                     const int4* __restrict__ segs, const float* q, double* dst,
                                                     long long T, long long base = 0) {
  using L = Lay<DIM, RX>;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff - base + (long long)j * pd.nx + i;
  const PrimF w = cons_to_prim32<DIM, RX>(P, F, q, T, cidx(pd, i, j));
  double* o = dst + s0;
  o[L::PHI * ncell] = w.phi;
  o[L::A1 * ncell] = w.r1;
  o[L::A2 * ncell] = w.r2;
  o[L::MX * ncell] = w.u;
  if constexpr (DIM == 2) o[L::MY * ncell] = w.v;
  o[L::E * ncell] = w.p;
  o[L::V11 * ncell] = w.V11;
  if constexpr (DIM == 2) { o[L::V12 * ncell] = w.V12; o[L::V21 * ncell] = w.V21; }
  o[L::V22 * ncell] = w.V22;
  o[L::V33 * ncell] = w.V33;
  if constexpr (RX) o[L::AL * ncell] = w.lam;
}

// New closure constants between steps: e_s += (kappa_2,old - kappa_2,new) +
// ((kappa_1 - kappa_2)_old - (kappa_1 - kappa_2)_new) phi1, so rho E is kept.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_rekappa32(const PatchDev* __restrict__ pds,
                                                   const int4* __restrict__ segs, float* q, long long T,
                                                   double dk2, double ddk) {
  using L = Lay<DIM, RX>;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const long long k = cidx(pd, g.z + threadIdx.x, g.y);
  const double phi = ff_val(q[L::PHI * T + k], q[L::NF * T + k]);
  q[L::E * T + k] = (float)((double)q[L::E * T + k] + dk2 + ddk * phi);
}

}  // namespace dis
