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
  float* W;
  float* Fx;
  float* Fy;
  unsigned long long* rate;
  const double* dtfix;
  double* dtlast;
  int* status;
  double a, b;
  int last;
  double kap2, dkap;  // kappa_2 and kappa_1 - kappa_2 (float64): energy flux kappa part
};

// Extra float face slots after the nf flux slots and the u_n / V row extras.
template <int DIM>
struct Face32 {
  static constexpr int EXTRA = DIM == 2 ? 3 : 2;
};

template <int DIM, bool RX>
__device__ __forceinline__ PrimF cons_to_prim32(const Phys& P, const PhysF& F, const double* q64,
                                                const float* q32, long long T, long long k) {
  using L = Lay<DIM, RX>;
  PrimF w;
  const double phi_d = q64[k];
  const double E = q64[T + k];
  const float phi = (float)phi_d;
  const float a1 = q32[L::A1 * T + k], a2 = q32[L::A2 * T + k];
  const float rho = a1 + a2;
  const float mx = q32[L::MX * T + k];
  float my = 0.f;
  if constexpr (DIM == 2) my = q32[L::MY * T + k];
  w.phi = phi;
  w.r1 = a1 / phi;
  w.r2 = a2 / (float)(1.0 - phi_d);
  const float irho = 1.f / rho;
  w.u = mx * irho;
  w.v = my * irho;
  w.V11 = q32[L::V11 * T + k];
  w.V12 = 0.f;
  w.V21 = 0.f;
  if constexpr (DIM == 2) {
    w.V12 = q32[L::V12 * T + k];
    w.V21 = q32[L::V21 * T + k];
  }
  w.V22 = q32[L::V22 * T + k];
  w.V33 = q32[L::V33 * T + k];
  float arl = 0.f;
  w.lam = 0.f;
  if constexpr (RX) {
    arl = q32[L::AL * T + k];
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

template <int DIM, bool RX>
__device__ __forceinline__ PrimF load_prim32(const float* __restrict__ W, long long T, long long k) {
  using L = Lay<DIM, RX>;
  PrimF w;
  w.phi = W[L::PHI * T + k];
  w.r1 = W[L::A1 * T + k];
  w.r2 = W[L::A2 * T + k];
  w.u = W[L::MX * T + k];
  w.v = 0.f;
  w.V12 = 0.f;
  w.V21 = 0.f;
  w.lam = 0.f;
  if constexpr (DIM == 2) {
    w.v = W[L::MY * T + k];
    w.V12 = W[L::V12 * T + k];
    w.V21 = W[L::V21 * T + k];
  }
  w.p = W[L::E * T + k];
  w.V11 = W[L::V11 * T + k];
  w.V22 = W[L::V22 * T + k];
  w.V33 = W[L::V33 * T + k];
  if constexpr (RX) w.lam = W[L::AL * T + k];
  return w;
}

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

template <int DIM, bool RX, int DIR>
__global__ void __launch_bounds__(SEG) k_flux32(PhysF P, StepArgs32 A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const long long T = A.T;
  const float* __restrict__ W = A.W;
  const int f = (DIR == 0 ? g.z : g.y) + (DIR == 0 ? threadIdx.x : 0);
  const int col = DIR == 0 ? g.y : g.z + threadIdx.x;
  const int a = (DIR == 0 ? f : g.y) - 1;
  auto at = [&](int s) -> long long { return DIR == 0 ? cidx(pd, s, col) : cidx(pd, col, s); };

  float ph[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) ph[s] = W[L::PHI * T + at(a - 2 + s)];
  float phiL, phiR;
  {
    CandF c[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float beta = 2.51f;
      if (DIM == 2 && P.thinc) {
        const long long k = at(a - 1 + s);
        const float* Ph = W + L::PHI * T;
        const long long sx = DIR == 0 ? 1 : (long long)pd.pitch;
        const long long sy = DIR == 0 ? (long long)pd.pitch : 1;
        const float dn = (Ph[k + sx + sy] + 2.f * Ph[k + sx] + Ph[k + sx - sy]) -
                         (Ph[k - sx + sy] + 2.f * Ph[k - sx] + Ph[k - sx - sy]);
        const float dt_ = (Ph[k + sy + sx] + 2.f * Ph[k + sy] + Ph[k + sy - sx]) -
                          (Ph[k - sy + sx] + 2.f * Ph[k - sy] + Ph[k - sy - sx]);
        const float gn = dn / (float)(DIR == 0 ? pd.dx : pd.dy), gt = dt_ / (float)(DIR == 0 ? pd.dy : pd.dx);
        const float nrm = sqrtf(gn * gn + gt * gt);
        beta = 2.5f * (nrm == 0.f ? 1.f : fabsf(gn) / nrm) + 0.01f;
      }
      c[s] = phi_cand_f(ph[s], ph[s + 1], ph[s + 2], beta, P.thinc != 0);
    }
    float Lt, Rt;
    bvd_f(c[0], c[1], c[2], Lt, Rt);
    phiL = Rt;
    bvd_f(c[1], c[2], c[3], Lt, Rt);
    phiR = Lt;
  }
  const PrimF w0 = load_prim32<DIM, RX>(W, T, at(a - 1));
  const PrimF w1 = load_prim32<DIM, RX>(W, T, at(a));
  const PrimF w2 = load_prim32<DIM, RX>(W, T, at(a + 1));
  const PrimF w3 = load_prim32<DIM, RX>(W, T, at(a + 2));
  PrimF wl, wr;
#define DIS_REC32(fld)                                            \
  {                                                               \
    const float s1 = minmod_f(w1.fld - w0.fld, w2.fld - w1.fld);  \
    const float s2 = minmod_f(w2.fld - w1.fld, w3.fld - w2.fld);  \
    wl.fld = w1.fld + 0.5f * s1;                                  \
    wr.fld = w2.fld - 0.5f * s2;                                  \
  }
  DIS_REC32(r1) DIS_REC32(r2) DIS_REC32(u) DIS_REC32(p) DIS_REC32(V11) DIS_REC32(V22) DIS_REC32(V33)
  if constexpr (DIM == 2) { DIS_REC32(v) DIS_REC32(V12) DIS_REC32(V21) }
  else { wl.v = wr.v = 0.f; wl.V12 = wr.V12 = wl.V21 = wr.V21 = 0.f; }
  if constexpr (RX) { DIS_REC32(lam) } else { wl.lam = wr.lam = 0.f; }
#undef DIS_REC32
  wl.phi = phiL;
  wr.phi = phiR;
  FStateF sl = face_state_f<DIR>(P, wl);
  if (!(sl.cL > 0.f)) sl = face_state_f<DIR>(P, w1);
  FStateF sr = face_state_f<DIR>(P, wr);
  if (!(sr.cL > 0.f)) sr = face_state_f<DIR>(P, w2);
  sl.cL = sqrtf(sl.cL);
  sr.cL = sqrtf(sr.cL);
  const FaceOutF o = hlld_f<DIR>(sl, sr);

  const float fu = DIR == 0 ? o.un : o.ut;
  const float fv = DIR == 0 ? o.ut : o.un;
  float* Fo = DIR == 0 ? A.Fx : A.Fy;
  const long long NFc = DIR == 0 ? A.NFX : A.NFY;
  const long long fi = DIR == 0 ? pd.fxoff + (long long)col * (pd.nx + 1) + f
                                : pd.fyoff + (long long)g.y * pd.nx + col;
  constexpr int XS = NF + Face32<DIM>::EXTRA;  // slots: X, phi_K
  Fo[L::PHI * NFc + fi] = o.phi * o.un;
  Fo[L::A1 * NFc + fi] = o.Far1;
  Fo[L::A2 * NFc + fi] = o.Far2;
  Fo[L::MX * NFc + fi] = DIR == 0 ? o.Fmn : o.Fmt;
  if constexpr (DIM == 2) Fo[L::MY * NFc + fi] = DIR == 0 ? o.Fmt : o.Fmn;
  Fo[L::E * NFc + fi] = o.FE;
  if constexpr (RX) Fo[L::AL * NFc + fi] = o.Farl;
  Fo[XS * NFc + fi] = o.X;
  Fo[(XS + 1) * NFc + fi] = o.phi;
  if constexpr (DIR == 0) {
    Fo[L::V11 * NFc + fi] = 0.f;
    if constexpr (DIM == 2) {
      Fo[L::V12 * NFc + fi] = 0.f;
      Fo[L::V21 * NFc + fi] = o.V21 * fu - o.V11 * fv;
      Fo[L::V22 * NFc + fi] = o.V22 * fu - o.V12 * fv;
    } else {
      Fo[L::V22 * NFc + fi] = o.V22 * fu;
    }
    Fo[L::V33 * NFc + fi] = o.V33 * fu;
    Fo[(NF + 0) * NFc + fi] = o.un;
    Fo[(NF + 1) * NFc + fi] = o.V11;
    if constexpr (DIM == 2) Fo[(NF + 2) * NFc + fi] = o.V12;
  } else if constexpr (DIM == 2) {
    Fo[L::V11 * NFc + fi] = o.V11 * fv - o.V21 * fu;
    Fo[L::V12 * NFc + fi] = o.V12 * fv - o.V22 * fu;
    Fo[L::V21 * NFc + fi] = 0.f;
    Fo[L::V22 * NFc + fi] = 0.f;
    Fo[L::V33 * NFc + fi] = o.V33 * fv;
    Fo[(NF + 0) * NFc + fi] = o.un;
    Fo[(NF + 1) * NFc + fi] = o.V21;
    Fo[(NF + 2) * NFc + fi] = o.V22;
  }
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_update32(Phys P, PhysF F, StepArgs32 A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  constexpr int XS = NF + Face32<DIM>::EXTRA;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long k = cidx(pd, i, j);
  const long long T = A.T;
  float q[NF], D[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) q[c] = (c == L::PHI || c == L::E) ? 0.f : A.q32src[c * T + k];
  const double phi_d = A.q64src[k];
  const double E_d = A.q64src[T + k];
  const float idx_ = 1.f / (float)pd.dx;
  const double idx_d = 1.0 / pd.dx;
  const long long fl = pd.fxoff + (long long)j * (pd.nx + 1) + i;
  const long long NFX = A.NFX;
  const float* Fx = A.Fx;
#pragma unroll
  for (int c = 0; c < NF; ++c) D[c] = (Fx[c * NFX + fl + 1] - Fx[c * NFX + fl]) * idx_;
  float divu = (Fx[NF * NFX + fl + 1] - Fx[NF * NFX + fl]) * idx_;
  float bx = (Fx[(NF + 1) * NFX + fl + 1] - Fx[(NF + 1) * NFX + fl]) * idx_;
  float by = 0.f;
  // float64 parts: phi flux, soft energy flux and the kappa part of the energy flux
  double Dphi = ((double)Fx[L::PHI * NFX + fl + 1] - (double)Fx[L::PHI * NFX + fl]) * idx_d;
  auto kapflux = [&](const float* Fp, long long NFc, long long f_) {
    const double X = Fp[XS * NFc + f_], ph = Fp[(XS + 1) * NFc + f_];
    return (double)Fp[L::E * NFc + f_] + A.kap2 * X + A.dkap * (ph * X);
  };
  double DE = (kapflux(Fx, NFX, fl + 1) - kapflux(Fx, NFX, fl)) * idx_d;
  double divu_d = ((double)Fx[NF * NFX + fl + 1] - (double)Fx[NF * NFX + fl]) * idx_d;
  if constexpr (DIM == 2) {
    by = (Fx[(NF + 2) * NFX + fl + 1] - Fx[(NF + 2) * NFX + fl]) * idx_;
    const float idy = 1.f / (float)pd.dy;
    const double idy_d = 1.0 / pd.dy;
    const long long NFY = A.NFY;
    const float* Fy = A.Fy;
    const long long fb = pd.fyoff + (long long)j * pd.nx + i;
    const long long ft = fb + pd.nx;
#pragma unroll
    for (int c = 0; c < NF; ++c) D[c] += (Fy[c * NFY + ft] - Fy[c * NFY + fb]) * idy;
    divu += (Fy[NF * NFY + ft] - Fy[NF * NFY + fb]) * idy;
    bx += (Fy[(NF + 1) * NFY + ft] - Fy[(NF + 1) * NFY + fb]) * idy;
    by += (Fy[(NF + 2) * NFY + ft] - Fy[(NF + 2) * NFY + fb]) * idy;
    Dphi += ((double)Fy[L::PHI * NFY + ft] - (double)Fy[L::PHI * NFY + fb]) * idy_d;
    DE += (kapflux(Fy, NFY, ft) - kapflux(Fy, NFY, fb)) * idy_d;
    divu_d += ((double)Fy[NF * NFY + ft] - (double)Fy[NF * NFY + fb]) * idy_d;
  }
  const float rho = q[L::A1] + q[L::A2];
  const float uc = q[L::MX] / rho;
  float vc = 0.f;
  if constexpr (DIM == 2) vc = q[L::MY] / rho;
  const float t23 = 2.f / 3.f;
  Dphi -= phi_d * divu_d;
  D[L::V11] -= t23 * q[L::V11] * divu - uc * bx;
  D[L::V22] -= t23 * q[L::V22] * divu - vc * by;
  D[L::V33] -= t23 * q[L::V33] * divu;
  if constexpr (DIM == 2) {
    D[L::V12] -= t23 * q[L::V12] * divu - uc * by;
    D[L::V21] -= t23 * q[L::V21] * divu - vc * bx;
  }
  const double dt = A.dtfix ? A.dtfix[g.x] : P.cfl / __longlong_as_double((long long)A.rate[g.x]);
  const float dtf = (float)dt;
  float o[NF];
  double ophi, oE;
  if (A.a == 0.0) {
#pragma unroll
    for (int c = 0; c < NF; ++c) o[c] = q[c] - dtf * D[c];
    ophi = phi_d - dt * Dphi;
    oE = E_d - dt * DE;
  } else {
    const float af = (float)A.a, bf = (float)A.b;
#pragma unroll
    for (int c = 0; c < NF; ++c)
      o[c] = (c == L::PHI || c == L::E) ? 0.f : af * A.q32n[c * T + k] + bf * (q[c] - dtf * D[c]);
    ophi = A.a * A.q64n[k] + A.b * (phi_d - dt * Dphi);
    oE = A.a * A.q64n[T + k] + A.b * (E_d - dt * DE);
  }
  if (A.last) {
    float v12 = 0.f, v21 = 0.f;
    if constexpr (DIM == 2) { v12 = o[L::V12]; v21 = o[L::V21]; }
    if (ophi > 1e-3 && ophi < 1.0 - 1e-3) {
      // mixed cell: radial return in float64
      double d11 = o[L::V11], d12 = v12, d21 = v21, d22 = o[L::V22], d33 = o[L::V33];
      plastic(P, ophi, dt, d11, d12, d21, d22, d33);
      o[L::V11] = (float)d11; v12 = (float)d12; v21 = (float)d21; o[L::V22] = (float)d22; o[L::V33] = (float)d33;
    } else {
      plastic_f(F, (float)ophi, dtf, o[L::V11], v12, v21, o[L::V22], o[L::V33]);
    }
    if constexpr (DIM == 2) { o[L::V12] = v12; o[L::V21] = v21; }
    if constexpr (RX) {
      const int y = P.y;
      const MatT<float>& m = F.m[y];
      const float phi1 = (float)ophi;
      const float ary = y == 0 ? o[L::A1] : o[L::A2];
      const float phy = y == 0 ? phi1 : (float)(1.0 - ophi);
      const float rr = o[L::A1] + o[L::A2];
      const float mx = o[L::MX];
      float my = 0.f;
      if constexpr (DIM == 2) my = o[L::MY];
      const float KE = 0.5f * (mx * mx + my * my) / rr;
      const StrainF s = strain_f(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
      const double kap = ophi * P.m[0].kap + (1.0 - ophi) * P.m[1].kap;
      const double num = oE - kap - (double)KE - (double)soft_ref_f(F, phi1, o[L::A1], o[L::A2], 0.f, s.J2);
      const float xi = xi_f(F, phi1);
      const float p0 = (float)num / xi;
      const float Tfac = m.iGm1 / ((ary / phy) * m.cv);
      const float Qx = m.Q / xi;
      auto fr = [&](float Lm) {
        const float Tk = (p0 - Qx * Lm) * Tfac;
        return Tk > 0.f ? -m.A * Lm * expf(-m.Tact / Tk) : 0.f;
      };
      const float L0 = o[L::AL];
      const float k1 = fr(L0);
      const float k2 = fr(L0 + 0.5f * dtf * k1);
      const float k3 = fr(L0 + 0.5f * dtf * k2);
      const float k4 = fr(L0 + dtf * k3);
      o[L::AL] = L0 + dtf / 6.f * (k1 + 2.f * k2 + 2.f * k3 + k4);
    }
    bool bad = !(ophi >= -1e-6 && ophi <= 1.0 + 1e-6) || !isfinite(oE);
#pragma unroll
    for (int c = 0; c < NF; ++c) bad |= (c != L::PHI && c != L::E) && !isfinite(o[c]);
    if (bad) flag_bad(A.status, g.x, i + pd.nx * j);
    if (i == 0 && j == 0) A.dtlast[g.x] = dt;
  }
#pragma unroll
  for (int c = 0; c < NF; ++c)
    if (c != L::PHI && c != L::E) A.q32dst[c * T + k] = o[c];
  A.q64dst[k] = ophi;
  A.q64dst[T + k] = oE;
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
