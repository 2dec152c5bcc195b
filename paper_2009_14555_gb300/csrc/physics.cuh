// physics.cuh - device closures of the diffuse-interface step (sm_103a).
//
// Written for the GPU from the paper's equations (arXiv 2009.14555), in the
// reduced forms that a stiffened-gas Mie-Grueneisen closure with constant
// shear modulus allows:
//   * mixture pressure (Appendix B pressure function, Section 2.2 mixture rules):
//       p = [rhoE - KE - sum_l phi_l (kap_l + gG_l J2) - sum_l ar_l e_inf,l
//            + Q_y (ar_y - arl)] / xi,     xi = sum_l phi_l / Gamma_l,
//     kap_l = gamma_l p_inf,l / Gamma_l, gG_l = gamma_l G_l / Gamma_l (shear
//     energy G J2 / rho enters the reference curves of the MG form);
//   * rho xi c^2 = sum_l phi_l (gamma_l p + gamma_l p_inf,l + gamma_l G_l J2) / Gamma_l
//     (frozen mixture sound speed; no phasic density needed), c_L^2 = c^2 + 4/3 G/rho;
//   * dev(H) = dev(1/4 (B - B^-1)), B = V V^T, in plane-strain block form
//     (Bazant approximation, Section 3.2), J2 = |dev H|^2;
//   * sigma = -p I + 2 G_mix dev(H);
//   * HLLD-type elastic Riemann solver (reading of the HLLD of Section 3.1):
//     longitudinal waves S_L, S_R, shear waves S* -/+ c_s, contact S*; star
//     stretch tensor rows scaled by r^-2/3 (normal) and r^1/3 (others),
//     r = (S_K - u_nK) / (S_K - S*); shear jumps add w x (normal row) to the
//     tangential row, w = (u_t,K - u_t**) / (S*_K - S*);
//   * THINC edge values and BVD choice (Appendix A);
//   * plastic update with the radial-return root of the objective and the
//     first Pade approximant (Section 3.2); RK4 reaction (Section 3.3) with
//     the Arrhenius law or the k sqrt(lam) law of Section 4.1 (switched on
//     above a pressure).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace dis {

constexpr int NG = 3;  // ghost layers: a face's BVD choice reaches 3 cells out

// Equation-of-state families of Section 2.3 (all with a constant Gruneisen
// coefficient Gamma = gamma - 1): stiffened gas (cold pressure -gamma p_inf,
// cold energy e_inf, constant G); Romenskii solid (cold energy
// K0 / (2 rho0 a^2) ((rho/rho0)^a - 1)^2, shear modulus G0 (rho/rho0)^(b+1));
// JWL (cold pressure A e^(-R1 rho0/rho) + B e^(-R2 rho0/rho), G = 0).
enum { EOS_SG = 0, EOS_ROMENSKII = 1, EOS_JWL = 2 };

template <class R>
struct MatT {
  R gamma, pinf, einf, G, sigy, chi0, Q, cv, A, Tact;
  int plastic, reactive;
  int eos;                  // EOS_SG, EOS_ROMENSKII or EOS_JWL
  R rho0, K0, ar, br;       // Romenskii: reference density, K0, exponents alpha-bar, beta-bar
  R jA, jB, jR1, jR2;       // JWL constants (rho0 shared)
  int two;                  // reactive material with a product closure of its own
  R pg, ppi, pcv;           // product gamma, p_inf, C_V (two closures)
  int law;  // reaction rate law: 0 Arrhenius, 1 A sqrt(lam) above the pressure pign
  R pign;
  R iGm1;  // 1 / (gamma - 1)
  R gi;    // gamma / (gamma - 1)
  R kap;   // gamma p_inf / (gamma - 1)
  R gG;    // gamma G / (gamma - 1)
  R GoG;   // G / (gamma - 1)
  R JY;    // yield strain invariant sigma_y / (sqrt(6) G)
  // Johnson-Cook plasticity (plastic == 3; sigy is c1): c2, c3, n, m, T_melt, T0
  R jc2, jc3, jcn, jcm, jcTm, jcT0;
};

template <class R>
struct PhysT {
  MatT<R> m[2];
  int y;      // reactive material (0/1) or -1
  int thinc;  // THINC-BVD steepening on phi1
  R cfl;
  int cyl;    // axisymmetric geometry (x = r, y = z): geometric source s_g
  int limiter;  // MUSCL slope limiter: 0 minmod, 1 van Leer
};

using MatDev = MatT<double>;
using Phys = PhysT<double>;

// Single-precision copy of the closure parameters (for the FP32-bulk kernels).
inline PhysT<float> to_float(const Phys& P) {
  PhysT<float> f{};
  for (int l = 0; l < 2; ++l) {
    const MatDev& d = P.m[l];
    MatT<float>& m = f.m[l];
    m.gamma = (float)d.gamma; m.pinf = (float)d.pinf; m.einf = (float)d.einf; m.G = (float)d.G;
    m.sigy = (float)d.sigy; m.chi0 = (float)d.chi0; m.Q = (float)d.Q; m.cv = (float)d.cv;
    m.A = (float)d.A; m.Tact = (float)d.Tact; m.plastic = d.plastic; m.reactive = d.reactive;
    m.law = d.law; m.pign = (float)d.pign;
    m.iGm1 = (float)d.iGm1; m.gi = (float)d.gi; m.kap = (float)d.kap; m.gG = (float)d.gG;
    m.GoG = (float)d.GoG; m.JY = (float)d.JY;
    m.eos = d.eos; m.rho0 = (float)d.rho0; m.K0 = (float)d.K0; m.ar = (float)d.ar; m.br = (float)d.br;
    m.jA = (float)d.jA; m.jB = (float)d.jB; m.jR1 = (float)d.jR1; m.jR2 = (float)d.jR2;
    m.two = d.two; m.pg = (float)d.pg; m.ppi = (float)d.ppi; m.pcv = (float)d.pcv;
    m.jc2 = (float)d.jc2; m.jc3 = (float)d.jc3; m.jcn = (float)d.jcn; m.jcm = (float)d.jcm;
    m.jcTm = (float)d.jcTm; m.jcT0 = (float)d.jcT0;
  }
  f.y = P.y;
  f.thinc = P.thinc;
  f.cfl = (float)P.cfl;
  f.cyl = P.cyl;
  f.limiter = P.limiter;
  return f;
}

// Field slots of the conservative and primitive states (same positions).
template <int DIM, bool RX>
struct Lay;
template <bool RX>
struct Lay<1, RX> {
  static constexpr int PHI = 0, A1 = 1, A2 = 2, MX = 3, MY = -1, E = 4, V11 = 5, V12 = -1, V21 = -1,
                       V22 = 6, V33 = 7, AL = RX ? 8 : -1, NF = RX ? 9 : 8;
  static constexpr int NX_EXTRA = 2;  // x-face extras: u_n, V11
};
template <bool RX>
struct Lay<2, RX> {
  static constexpr int PHI = 0, A1 = 1, A2 = 2, MX = 3, MY = 4, E = 5, V11 = 6, V12 = 7, V21 = 8,
                       V22 = 9, V33 = 10, AL = RX ? 11 : -1, NF = RX ? 12 : 11;
  static constexpr int NX_EXTRA = 3;  // face extras: u_n, V_n1, V_n2
};

template <class R>
struct PrimT {
  R phi, r1, r2, u, v, p, V11, V12, V21, V22, V33, lam;
};
using Prim = PrimT<double>;

template <class R>
struct StrainT {
  R H11, H12, H22, H33, J2;
};
using Strain = StrainT<double>;

template <class T>
__device__ __forceinline__ StrainT<T> strain_of(T a, T b, T c, T d, T e) {
  const T B11 = a * a + b * b, B12 = a * c + b * d, B22 = c * c + d * d, B33 = e * e;
  const T idet = 1.0 / (B11 * B22 - B12 * B12);
  const T M11 = 0.25 * (B11 - B22 * idet);
  const T M22 = 0.25 * (B22 - B11 * idet);
  const T M12 = 0.25 * (B12 + B12 * idet);
  const T M33 = 0.25 * (B33 - 1.0 / B33);
  const T t3 = (M11 + M22 + M33) * (1.0 / 3.0);
  StrainT<T> s;
  s.H11 = M11 - t3;
  s.H22 = M22 - t3;
  s.H33 = M33 - t3;
  s.H12 = M12;
  s.J2 = s.H11 * s.H11 + s.H22 * s.H22 + s.H33 * s.H33 + 2.0 * s.H12 * s.H12;
  return s;
}

// Reference curves of a Romenskii or JWL material at phasic density r and
// strain J2: E_ref, p_ref = r^2 dE_ref/dr, and their density derivatives.
// The shear energy G(r) J2 / r adds (r G' - G) J2 to the reference pressure.
template <class T>
struct RefT {
  T e, p, dp, de;
};
// a^b for a > 0 (the dual-number form lives with the Dual type)
__device__ __forceinline__ double powr(double a, double b) { return ::pow(a, b); }
__device__ __forceinline__ float powr(float a, float b) { return ::powf(a, b); }
template <class T, class R>
__device__ __forceinline__ RefT<T> ref_curves(const MatT<R>& m, T r, T J2) {
  RefT<T> o;
  if (m.eos == EOS_ROMENSKII) {
    const T x = r / m.rho0;
    const T xa = powr(x, T(m.ar));
    const T G = m.G * powr(x, T(m.br + 1.0));
    const T pc = m.K0 / m.ar * xa * x * (xa - 1.0);
    o.e = m.K0 / (2.0 * m.rho0 * m.ar * m.ar) * (xa - 1.0) * (xa - 1.0) + G * J2 / r;
    o.p = pc + m.br * G * J2;
    o.dp = m.K0 / (m.ar * m.rho0) * xa * ((2.0 * m.ar + 1.0) * xa - (m.ar + 1.0)) + m.br * (m.br + 1.0) * G / r * J2;
    o.de = (pc + m.br * G * J2) / (r * r);
  } else {
    const T e1 = m.jA * exp(-m.jR1 * m.rho0 / r), e2 = m.jB * exp(-m.jR2 * m.rho0 / r);
    o.e = e1 / (m.jR1 * m.rho0) + e2 / (m.jR2 * m.rho0);
    o.p = e1 + e2;
    o.dp = (e1 * m.jR1 + e2 * m.jR2) * m.rho0 / (r * r);
    o.de = o.p / (r * r);
  }
  return o;
}

// Reactive material with distinct reactant and product closures (Section
// 2.3.1, Appendix B), both stiffened gases without shear modulus: the
// reactant takes the material's gamma, p_inf, C_V, the product pg, ppi, pcv.
// With s = lam rho_y / rho_alpha the reactant's share of the mixture volume,
// the pressure function depends on the densities through s only:
// 1 / Gamma_y = s / Gamma_a + (1 - s) / Gamma_b, kappa_y = s kappa_a +
// (1 - s) kappa_b; the temperature equality T_a = T_b gives s in closed form
// at a known pressure, and by bisection over s in [0, 1] from the
// conservative state (mixture_pressure).
template <class T>
__device__ __forceinline__ T mix_share(const MatT<T>& m, T lam, T p) {
  const T wa = lam * (m.gamma - 1.0) * m.cv * (p + m.pg * m.ppi);
  const T wb = (1.0 - lam) * (m.pg - 1.0) * m.pcv * (p + m.gamma * m.pinf);
  return wa / (wa + wb);
}
template <class T>
__device__ __forceinline__ void mix_consts(const MatT<T>& m, T s, T& iG, T& kap) {
  iG = s / (m.gamma - 1.0) + (1.0 - s) / (m.pg - 1.0);
  kap = s * (m.gamma * m.pinf / (m.gamma - 1.0)) + (1.0 - s) * (m.pg * m.ppi / (m.pg - 1.0));
}
// The closures with the reactive material's effective constants at (lam, p)
// (unchanged without two closures), so the reduced stiffened-gas forms hold:
// gi p + kap = rho_y c_y^2 / Gamma_y with gi = 1 + 1 / Gamma_y.
template <class T>
__device__ __forceinline__ PhysT<T> at_state(const PhysT<T>& P, T lam, T p) {
  PhysT<T> Q = P;
  if (P.y >= 0 && P.m[P.y].two) {
    MatT<T>& m = Q.m[P.y];
    T iG, kap;
    mix_consts(m, mix_share(m, lam, p), iG, kap);
    m.iGm1 = iG;
    m.kap = kap;
    m.gi = 1.0 + iG;
  }
  return Q;
}
// Common temperature of a two-closure mixture at phasic density r:
// sum_k share_k (p + gamma_k p_inf,k) / (Gamma_k C_V,k) / r.
template <class T>
__device__ __forceinline__ T mix_temperature(const MatT<T>& m, T lam, T p, T r) {
  const T s = mix_share(m, lam, p);
  return (s * (p + m.gamma * m.pinf) / ((m.gamma - 1.0) * m.cv) + (1.0 - s) * (p + m.pg * m.ppi) / ((m.pg - 1.0) * m.pcv)) / r;
}

// Shear modulus of a material at phasic density r (constant but for Romenskii).
template <class T, class R>
__device__ __forceinline__ T shear_of(const MatT<R>& m, T r) {
  if (m.eos == EOS_ROMENSKII) return m.G * powr(r / m.rho0, T(m.br + 1.0));
  return T(m.G);
}

// The pieces of the pressure function that do not depend on the internal
// energy: sum_l phi_l rho_l (E_ref,l - p_ref,l / (rho_l Gamma_l)) and the heat
// release; the stiffened gas in its reduced form (kappa_l = gamma_l p_inf,l /
// Gamma_l, gG_l = gamma_l G_l / Gamma_l), other families at rho_l = ar_l / phi_l.
template <class T>
__device__ __forceinline__ T ref_energy(const PhysT<T>& P, T phi1, T ar1, T ar2, T arl, T J2) {
  const T phi2 = 1.0 - phi1;
  T s;
  if (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG) {
    s = phi1 * (P.m[0].kap + P.m[0].gG * J2) + phi2 * (P.m[1].kap + P.m[1].gG * J2) + ar1 * P.m[0].einf +
        ar2 * P.m[1].einf;
  } else {
    s = T(0.0);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const MatT<T>& m = P.m[l];
      const T ph = l == 0 ? phi1 : phi2, ar = l == 0 ? ar1 : ar2;
      if (m.eos == EOS_SG) {
        s += ph * (m.kap + m.gG * J2) + ar * m.einf;
      } else {
        const T r = ar / ph;
        const RefT<T> c = ref_curves(m, r, J2);
        s += ar * (c.e - c.p * m.iGm1 / r);
      }
    }
  }
  if (P.y >= 0) {
    const T ary = P.y == 0 ? ar1 : ar2;
    s -= P.m[P.y].Q * (ary - arl);
  }
  return s;
}

template <class T>
__device__ __forceinline__ T xi_of(const PhysT<T>& P, T phi1) {
  return phi1 * P.m[0].iGm1 + (1.0 - phi1) * P.m[1].iGm1;
}

// Pressure of a state whose reactive material has two closures, from its
// conservative variables (Appendix B): bisection of the temperature-equality
// residual (1 - lam)(pg - 1) pcv (p + gamma p_inf) s - lam (gamma - 1) cv
// (p + pg ppi)(1 - s) over s in [0, 1] (64 halvings), the pressure at each s
// from the pressure function; s_out receives the share.
template <class T>
__device__ __forceinline__ T mixture_pressure(const PhysT<T>& P, T phi1, T ar1, T ar2, T arl, T rhoe, T J2,
                                              T& s_out) {
  const int y = P.y, x = 1 - P.y;
  const MatT<T>& m = P.m[y];
  const MatT<T>& mi = P.m[x];
  const T phx = x == 0 ? phi1 : 1.0 - phi1, phy = y == 0 ? phi1 : 1.0 - phi1;
  const T arx = x == 0 ? ar1 : ar2, ary = y == 0 ? ar1 : ar2;
  T Rx;
  if (mi.eos == EOS_SG) {
    Rx = phx * (mi.kap + mi.gG * J2) + arx * mi.einf;
  } else {
    const T r = arx / phx;
    const RefT<T> c = ref_curves(mi, r, J2);
    Rx = arx * (c.e - c.p * mi.iGm1 / r);
  }
  const T xix = phx * mi.iGm1;
  const T num0 = rhoe - Rx + m.Q * (ary - arl);
  const T lam = arl / ary;
  T lo = 0.0, hi = 1.0;
  for (int it = 0; it < 64; ++it) {
    const T s = 0.5 * (lo + hi);
    T iG, kap;
    mix_consts(m, s, iG, kap);
    const T p = (num0 - phy * kap) / (xix + phy * iG);
    const T g = (1.0 - lam) * (m.pg - 1.0) * m.pcv * (p + m.gamma * m.pinf) * s -
                lam * (m.gamma - 1.0) * m.cv * (p + m.pg * m.ppi) * (1.0 - s);
    if (g < 0.0) lo = s;
    else hi = s;
  }
  s_out = 0.5 * (lo + hi);
  T iG, kap;
  mix_consts(m, s_out, iG, kap);
  return (num0 - phy * kap) / (xix + phy * iG);
}

// rho_l c_l^2 / Gamma_l of one material at pressure p (Mie-Grueneisen form,
// c^2 = (dp/drho)_E + p / rho^2 (dp/dE)_rho at fixed strain).
template <class T>
__device__ __forceinline__ T rc2_of(const MatT<T>& m, T r, T p, T J2) {
  if (m.eos == EOS_SG) return m.gi * p + m.kap + m.gG * J2;
  const RefT<T> c = ref_curves(m, r, J2);
  const T Gam = m.gamma - 1.0;
  return m.iGm1 * (r * c.dp + m.gamma * p - c.p - r * r * Gam * c.de);
}

// c_L^2 for a state (frozen mixture sound speed plus 4/3 G_mix / rho); r1,
// r2 are the phasic densities (read only by the Romenskii and JWL forms).
template <class T>
__device__ __forceinline__ T cL2_of(const PhysT<T>& P, T phi1, T rho, T p, T J2, T r1, T r2) {
  const T phi2 = 1.0 - phi1;
  const T xi = xi_of(P, phi1);
  if (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG) {
    const T a = phi1 * (P.m[0].gi * p + P.m[0].kap + P.m[0].gG * J2) +
                phi2 * (P.m[1].gi * p + P.m[1].kap + P.m[1].gG * J2);
    const T Gm = (phi1 * P.m[0].GoG + phi2 * P.m[1].GoG) / xi;
    return (a / xi + (4.0 / 3.0) * Gm) / rho;
  }
  const T a = phi1 * rc2_of(P.m[0], r1, p, J2) + phi2 * rc2_of(P.m[1], r2, p, J2);
  const T Gm = (phi1 * shear_of(P.m[0], r1) * P.m[0].iGm1 + phi2 * shear_of(P.m[1], r2) * P.m[1].iGm1) / xi;
  return (a / xi + (4.0 / 3.0) * Gm) / rho;
}

template <class T>
__device__ __forceinline__ T Gmix_of(const PhysT<T>& P, T phi1, T r1, T r2) {
  if (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG)
    return (phi1 * P.m[0].GoG + (1.0 - phi1) * P.m[1].GoG) / xi_of(P, phi1);
  return (phi1 * shear_of(P.m[0], r1) * P.m[0].iGm1 + (1.0 - phi1) * shear_of(P.m[1], r2) * P.m[1].iGm1) /
         xi_of(P, phi1);
}

template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
  return (a * b > 0.0) ? copysign(fmin(fabs(a), fabs(b)), a) : T(0.0);
}

// van Leer's limited slope, the harmonic mean 2 a b / (a + b) of the two
// one-sided differences when they have the same sign, else 0.
template <class T>
__device__ __forceinline__ T vanleer(T a, T b) {
  const T ab = a * b;
  return (ab > 0.0) ? 2.0 * ab / (a + b) : T(0.0);
}

// Limited slope of the MUSCL reconstruction: lim 0 minmod, 1 van Leer.
template <class T>
__device__ __forceinline__ T limited(T a, T b, int lim) {
  return lim ? vanleer(a, b) : minmod(a, b);
}

// MUSCL and THINC edge candidates of phi in one cell (Appendix A).
template <class T>
struct CandT {
  T mL, mR, tL, tR;
};
using Cand = CandT<double>;

// beta_of() gives the THINC steepness; it is evaluated only in a mixed cell.
template <class T, class BetaFn>
__device__ __forceinline__ CandT<T> phi_cand_lazy(T qm, T qc, T qp, const BetaFn& beta_of, bool thinc,
                                                  int lim = 0) {
  CandT<T> c;
  const T s = limited(qc - qm, qp - qc, lim);
  c.mL = qc - 0.5 * s;
  c.mR = qc + 0.5 * s;
  c.tL = c.mL;
  c.tR = c.mR;
  if (thinc) {
    const T qmin = fmin(qm, qp);
    const T jump = fmax(qm, qp) - qmin;
    const T C = (qc - qmin + 1e-20) / (jump + 1e-20);
    if (C > 1e-5 && C < 1.0 - 1e-5 && (qp - qc) * (qc - qm) > 0.0) {
      const T beta = beta_of();
      const T th = (qp - qm) > 0.0 ? T(1.0) : T(-1.0);
      const T B = exp(th * beta * (2.0 * C - 1.0));
      const T tb = tanh(beta);
      const T A = (B / cosh(beta) - 1.0) / tb;
      c.tL = qmin + 0.5 * jump * (1.0 + th * A);
      c.tR = qmin + 0.5 * jump * (1.0 + th * (tb + A) / (1.0 + A * tb));
    }
  }
  return c;
}

template <class T>
__device__ __forceinline__ CandT<T> phi_cand(T qm, T qc, T qp, T beta, bool thinc) {
  return phi_cand_lazy(qm, qc, qp, [&]() { return beta; }, thinc);
}

// BVD choice for the middle cell: THINC only if its total boundary variation
// is strictly smaller (ties keep MUSCL).
template <class T>
__device__ __forceinline__ void bvd(const CandT<T>& km, const CandT<T>& k, const CandT<T>& kp, T& L, T& R) {
  const T tT = fmin(fabs(km.mR - k.tL), fabs(km.tR - k.tL)) +
                    fmin(fabs(k.tR - kp.mL), fabs(k.tR - kp.tL));
  const T tM = fmin(fabs(km.mR - k.mL), fabs(km.tR - k.mL)) +
                    fmin(fabs(k.mR - kp.mL), fabs(k.mR - kp.tL));
  const bool useT = tT < tM;
  L = useT ? k.tL : k.mL;
  R = useT ? k.tR : k.mR;
}

// Thermodynamic face state for the Riemann solver.  Direction: n = normal
// velocity component, t = tangential; Vn* = row of V along the normal.
template <class T>
struct FStateT {
  T phi, ar1, ar2, arl, rho, un, ut, rhoE, snn, snt, cL, Gm;
  T V11, V12, V21, V22, V33;
};
using FState = FStateT<double>;

template <int DIR, class T>
__device__ __forceinline__ FStateT<T> face_state(const PhysT<T>& P0, const PrimT<T>& w) {
  const PhysT<T> P = at_state(P0, w.lam, w.p);  // two-closure reactive mixture at (lam, p)
  FStateT<T> s;
  const StrainT<T> st = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  s.phi = w.phi;
  s.ar1 = w.phi * w.r1;
  s.ar2 = (1.0 - w.phi) * w.r2;
  s.rho = s.ar1 + s.ar2;
  s.arl = 0.0;
  if (P.y >= 0) s.arl = (P.y == 0 ? s.ar1 : s.ar2) * w.lam;
  const T xi = xi_of(P, w.phi);
  s.rhoE = xi * w.p + ref_energy(P, w.phi, s.ar1, s.ar2, s.arl, st.J2) +
           0.5 * s.rho * (w.u * w.u + w.v * w.v);
  const T Gm = Gmix_of(P, w.phi, w.r1, w.r2);
  s.Gm = Gm;
  if (DIR == 0) {
    s.un = w.u;
    s.ut = w.v;
    s.snn = -w.p + 2.0 * Gm * st.H11;
  } else {
    s.un = w.v;
    s.ut = w.u;
    s.snn = -w.p + 2.0 * Gm * st.H22;
  }
  s.snt = 2.0 * Gm * st.H12;
  s.cL = cL2_of(P, w.phi, s.rho, w.p, st.J2, w.r1, w.r2);  // squared here; k_flux takes the root
  s.V11 = w.V11;
  s.V12 = w.V12;
  s.V21 = w.V21;
  s.V22 = w.V22;
  s.V33 = w.V33;
  return s;
}

// Output of one face: conservative fluxes plus the face state at x/t = 0.
template <class T>
struct FaceOutT {
  T Far1, Far2, Farl, Fmn, Fmt, FE;
  T phi, un, ut, V11, V12, V21, V22, V33;
};
using FaceOut = FaceOutT<double>;

// Star (longitudinal-wave) state of one side.
template <class T>
struct StarT {
  T r, snn, E, V11, V12, V21, V22, V33;
};

template <int DIR, class T>
__device__ __forceinline__ StarT<T> star_of(const FStateT<T>& K, T S, T Ss) {
  StarT<T> t;
  const T inv = 1.0 / (S - Ss);
  t.r = (S - K.un) * inv;
  const T m = K.rho * (S - K.un);
  t.snn = K.snn - m * (Ss - K.un);
  // energy jump: E*(S - S*) = E (S - u_n) + u.sigma_n - u*.sigma*_n (tangential work cancels)
  t.E = (K.rhoE * (S - K.un) + K.un * K.snn - Ss * t.snn) * inv;
  const T c1 = cbrt(t.r);        // r^(1/3): rows off the normal
  const T cn = 1.0 / (c1 * c1);  // r^(-2/3): row along the normal
  if (DIR == 0) {
    t.V11 = cn * K.V11; t.V12 = cn * K.V12;
    t.V21 = c1 * K.V21; t.V22 = c1 * K.V22;
  } else {
    t.V11 = c1 * K.V11; t.V12 = c1 * K.V12;
    t.V21 = cn * K.V21; t.V22 = cn * K.V22;
  }
  t.V33 = c1 * K.V33;
  return t;
}

// A product rounded on its own, never fused into a neighbouring addition.
// The numerator of the contact speed S* must cancel exactly for mirrored
// face states (a reflective wall: u_n,L = -u_n,R, equal sigma_nn), as it does
// in plain float64 arithmetic; with one product fused into the subtraction
// the rounding error of the other decides the sign of S* = 0 and so which
// star state (whose V12 differs in sign) becomes the face state.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <int DIR, class T>
__device__ __forceinline__ FaceOutT<T> hllc(const FStateT<T>& L, const FStateT<T>& R) {
  const T SL = fmin(L.un - L.cL, R.un - R.cL);
  const T SR = fmax(L.un + L.cL, R.un + R.cL);
  const T mL = L.rho * (SL - L.un);
  const T mR = R.rho * (SR - R.un);
  const T Ss = ((L.snn - R.snn) + mul_rn(mL, L.un) - mul_rn(mR, R.un)) / (mL - mR);
  const StarT<T> sL = star_of<DIR>(L, SL, Ss);
  const StarT<T> sR = star_of<DIR>(R, SR, Ss);
  // shear waves of the star regions and the common tangential state
  const T rsL = sL.r * L.rho, rsR = sR.r * R.rho;
  const T csL = sqrt(L.Gm / rsL), csR = sqrt(R.Gm / rsR);
  const T ZL = rsL * csL, ZR = rsR * csR;
  const T SsL = Ss - csL, SsR = Ss + csR;
  T ut2L = L.ut, ut2R = R.ut, st2L = L.snt, st2R = R.snt;
  if (ZL + ZR > 0.0) {
    const T ut2 = (ZL * L.ut + ZR * R.ut + R.snt - L.snt) / (ZL + ZR);
    const T st2 = L.snt + ZL * (ut2 - L.ut);
    ut2L = ut2R = ut2;
    st2L = st2R = st2;
  }
  // region at x/t = 0 and its side
  int level;
  bool left;
  if (SL >= 0.0) { left = true; level = 0; }
  else if (SsL >= 0.0) { left = true; level = 1; }
  else if (Ss >= 0.0) { left = true; level = 2; }
  else if (SsR >= 0.0) { left = false; level = 2; }
  else if (SR >= 0.0) { left = false; level = 1; }
  else { left = false; level = 0; }
  const FStateT<T>& K = left ? L : R;
  const StarT<T>& sK = left ? sL : sR;
  const T S = left ? SL : SR;
  const T Sh = left ? SsL : SsR;
  const T ut2 = left ? ut2L : ut2R;
  const T st2 = left ? st2L : st2R;
  const T un = K.un, ut = K.ut;
  FaceOutT<T> o;
  T Far1 = K.ar1 * un, Far2 = K.ar2 * un, Farl = K.arl * un;
  T Fmn = K.rho * un * un - K.snn;
  T Fmt = K.rho * ut * un - K.snt;
  T FE = K.rhoE * un - (un * K.snn + ut * K.snt);
  o.phi = K.phi;
  if (level == 0) {
    o.un = un;
    o.ut = ut;
    o.V11 = K.V11; o.V12 = K.V12; o.V21 = K.V21; o.V22 = K.V22; o.V33 = K.V33;
  } else {
    const T r1 = sK.r - 1.0;
    Far1 += S * r1 * K.ar1;
    Far2 += S * r1 * K.ar2;
    Farl += S * r1 * K.arl;
    Fmn += S * (sK.r * K.rho * Ss - K.rho * un);
    Fmt += S * r1 * K.rho * ut;
    FE += S * (sK.E - K.rhoE);
    o.un = Ss;
    o.ut = ut;
    o.V11 = sK.V11; o.V12 = sK.V12; o.V21 = sK.V21; o.V22 = sK.V22; o.V33 = sK.V33;
    if (level == 2) {
      const T dS = Sh - Ss;
      const T rs = sK.r * K.rho;
      if (dS != 0.0) {
        const T idS = 1.0 / dS;
        Fmt += Sh * rs * (ut2 - ut);
        FE -= Sh * (ut2 * st2 - ut * K.snt) * idS;
        const T w = (ut - ut2) * idS;
        if (DIR == 0) {
          o.V21 = sK.V21 + w * sK.V11;
          o.V22 = sK.V22 + w * sK.V12;
        } else {
          o.V11 = sK.V11 + w * sK.V21;
          o.V12 = sK.V12 + w * sK.V22;
        }
        o.ut = ut2;
      }
    }
  }
  o.Far1 = Far1; o.Far2 = Far2; o.Farl = Farl; o.Fmn = Fmn; o.Fmt = Fmt; o.FE = FE;
  return o;
}

// Johnson-Cook input of the plastic step: the material's temperature at the
// state entering the step and its plastic strain eps_p.
template <class T>
struct JcIn {
  T temp, eps;
};

// Johnson-Cook relaxed strain norm of one material (Section 2.3.2 rate law
// in the objective of Section 3.2): bisection (64 halvings) of
// R(J) = J - J* + dt chi0 exp((sqrt(3/2) 2 G J / sigma_Y - 1) / c3) on [0, J*]
// with sigma_Y = (c1 + c2 max(eps_p + J* - J, 0)^n)(1 - T*^m), T* the
// homologous temperature clamped to [0, 1]; no strength (sigma_Y <= 0) makes
// the rate unbounded and the root 0.
template <class T, class R>
__device__ __forceinline__ T jc_relax(const MatT<R>& m, T Js, T Gl, T dt, const JcIn<T>& in) {
  T Ts = (in.temp - m.jcT0) / (m.jcTm - m.jcT0);
  Ts = fmin(fmax(Ts, T(0.0)), T(1.0));
  const T soft = 1.0 - powr(Ts, T(m.jcm));
  const T k = sqrt(T(1.5)) * T(2.0);
  T lo = 0.0, hi = Js;
  for (int it = 0; it < 64; ++it) {
    const T mid = 0.5 * (lo + hi);
    const T e = fmax(in.eps + (Js - mid), T(0.0));
    const T sY = (m.sigy + m.jc2 * (m.jcn == 1.0 ? e : powr(e, T(m.jcn)))) * soft;  // e^1 = e exactly
    bool neg = false;
    if (sY > 0.0) {
      const T rate = m.chi0 * exp((k * Gl * mid / sY - 1.0) / m.jc3);
      neg = mid - Js + dt * rate < 0.0;
    }
    if (neg) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Plastic update of Section 3.2 on one cell's stretch tensor (in place).  r1,
// r2: phasic densities (the Romenskii yield strain sigma_y / (sqrt 6 G(r))).
// A Johnson-Cook material reads jc (its temperature and plastic strain) and
// returns the growth J* - J*_l of its plastic strain in *deps.
template <class T>
__device__ __forceinline__ void plastic(const PhysT<T>& P, T phi1, T dt, T& V11,
                                        T& V12, T& V21, T& V22, T& V33, T r1, T r2,
                                        const JcIn<T>* jc = nullptr, T* deps = nullptr) {
  const StrainT<T> s = strain_of(V11, V12, V21, V22, V33);
  const T Js = sqrt(s.J2);
  T num = 0.0, den = 0.0;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const MatT<T>& m = P.m[l];
    const T ph = l == 0 ? phi1 : 1.0 - phi1;
    const T JY = m.eos == EOS_ROMENSKII ? m.sigy / (2.449489742783178 * shear_of(m, l == 0 ? r1 : r2)) : m.JY;
    T Jl;
    if (m.G == 0.0) {
      Jl = T(0.0);  // a fluid keeps no shear strain
    } else if (m.plastic == 1) {
      Jl = fmin(Js, JY);
    } else if (m.plastic == 2) {
      Jl = Js > JY ? fmax(Js - dt * m.chi0, JY) : Js;
    } else if (m.plastic == 3 && jc) {
      Jl = jc_relax(m, Js, shear_of(m, l == 0 ? r1 : r2), dt, *jc);
      if (deps) *deps = Js - Jl;
    } else {
      Jl = Js;
    }
    num += ph * m.iGm1 * Jl;
    den += ph * m.iGm1;
  }
  const T Jn = num / den;
  const T sc = Js > 0.0 ? Jn / Js : T(0.0);
  const T h11 = sc * s.H11, h12 = sc * s.H12, h22 = sc * s.H22, h33 = sc * s.H33;
  // V = (I - H/2)^-1 (I + H/2) on the in-plane block and the zz entry
  const T x11 = 1.0 - 0.5 * h11, x12 = -0.5 * h12, x22 = 1.0 - 0.5 * h22;
  const T y11 = 1.0 + 0.5 * h11, y12 = 0.5 * h12, y22 = 1.0 + 0.5 * h22;
  const T id = 1.0 / (x11 * x22 - x12 * x12);
  const T i11 = x22 * id, i12 = -x12 * id, i22 = x11 * id;
  V11 = i11 * y11 + i12 * y12;
  V12 = i11 * y12 + i12 * y22;
  V21 = i12 * y11 + i22 * y12;
  V22 = i12 * y12 + i22 * y22;
  V33 = (1.0 + 0.5 * h33) / (1.0 - 0.5 * h33);
}

}  // namespace dis
