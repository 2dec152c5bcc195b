// physics32.cuh - single-precision closures for the FP32-bulk step (sm_103a).
//
// Same mathematics as physics.cuh, arranged for float arithmetic:
//   * the strain uses B = I + X with X formed from V - I, and
//     B - B^-1 = X + (I + X)^-1 X, so small elastic strains (1e-3) keep their
//     relative precision instead of cancelling in B - B^-1;
//   * the face energy omits the stiff reference part sum_l phi_l gamma_l p_inf,l / Gamma_l
//     (kappa_l phi_l, up to 1e11 J/m^3 against a thermal part of 1e5): that part
//     of the energy flux is kappa(phi_K) X with X = u_n (outside the star
//     regions) or u_n + S_K (r_K - 1) (inside), and is rebuilt in float64 by
//     the update kernel from the same face values that update phi, so the
//     pressure recovered from rho E - kappa(phi) keeps float64 cancellation.
#pragma once
#include "physics.cuh"

namespace dis {

using PhysF = PhysT<float>;
using PrimF = PrimT<float>;
using StrainF = StrainT<float>;

__device__ __forceinline__ StrainF strain_f(float a, float b, float c, float d, float e) {
  const float ea = a - 1.f, ed = d - 1.f, ee = e - 1.f;
  const float X11 = ea * (2.f + ea) + b * b;
  const float X22 = ed * (2.f + ed) + c * c;
  const float X12 = a * c + b * d;
  const float X33 = ee * (2.f + ee);
  const float B11 = 1.f + X11, B22 = 1.f + X22;
  const float id = 1.f / (B11 * B22 - X12 * X12);
  const float Y11 = (B22 * X11 - X12 * X12) * id;
  const float Y22 = (B11 * X22 - X12 * X12) * id;
  const float Y12 = X12 * id;  // (B22 X12 - X12 X22) / det with B22 - X22 = 1
  const float Y33 = X33 / (1.f + X33);
  const float M11 = 0.25f * (X11 + Y11), M22 = 0.25f * (X22 + Y22);
  const float M12 = 0.25f * (X12 + Y12), M33 = 0.25f * (X33 + Y33);
  const float t3 = (M11 + M22 + M33) * (1.f / 3.f);
  StrainF s;
  s.H11 = M11 - t3;
  s.H22 = M22 - t3;
  s.H33 = M33 - t3;
  s.H12 = M12;
  s.J2 = s.H11 * s.H11 + s.H22 * s.H22 + s.H33 * s.H33 + 2.f * s.H12 * s.H12;
  return s;
}

__device__ __forceinline__ float xi_f(const PhysF& P, float phi1) {
  return phi1 * P.m[0].iGm1 + (1.f - phi1) * P.m[1].iGm1;
}

// Reference energy without the stiff kappa part: shear, e_inf and heat
// release of a stiffened gas; the whole reference part ar_l (E_ref,l -
// p_ref,l / (rho_l Gamma_l)) of a Romenskii or JWL material (their kappa is
// zero) at its phasic density r_l.
// GEN: the kernels of contexts with a Romenskii or JWL material (GEN false:
// stiffened gases only, and none of the general code is compiled in).
template <bool GEN = true>
__device__ __forceinline__ float soft_ref_f(const PhysF& P, float phi1, float ar1, float ar2, float arl,
                                            float J2, float r1, float r2) {
  float s;
  if (!GEN || (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG)) {
    s = (phi1 * P.m[0].gG + (1.f - phi1) * P.m[1].gG) * J2 + ar1 * P.m[0].einf + ar2 * P.m[1].einf;
  } else {
    s = 0.f;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const MatT<float>& m = P.m[l];
      const float ar = l == 0 ? ar1 : ar2, r = l == 0 ? r1 : r2;
      if (m.eos == EOS_SG) {
        s += (l == 0 ? phi1 : 1.f - phi1) * m.gG * J2 + ar * m.einf;
      } else {
        const RefT<float> c = ref_curves(m, r, J2);
        s += ar * (c.e - c.p * m.iGm1 / r);
      }
    }
  }
  if (P.y >= 0) s -= P.m[P.y].Q * ((P.y == 0 ? ar1 : ar2) - arl);
  return s;
}

// Mixture shear modulus (phi / Gamma weights) at the phasic densities.
template <bool GEN = true>
__device__ __forceinline__ float Gmix_f(const PhysF& P, float phi1, float r1, float r2) {
  const float ixi = 1.f / xi_f(P, phi1);
  if (!GEN || (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG))
    return (phi1 * P.m[0].GoG + (1.f - phi1) * P.m[1].GoG) * ixi;
  return (phi1 * shear_of(P.m[0], r1) * P.m[0].iGm1 + (1.f - phi1) * shear_of(P.m[1], r2) * P.m[1].iGm1) * ixi;
}

template <bool GEN = true>
__device__ __forceinline__ float cL2_f(const PhysF& P, float phi1, float rho, float p, float J2, float r1,
                                       float r2) {
  const float phi2 = 1.f - phi1;
  const float ixi = 1.f / xi_f(P, phi1);
  if (!GEN || (P.m[0].eos == EOS_SG && P.m[1].eos == EOS_SG)) {
    const float a = phi1 * (P.m[0].gi * p + P.m[0].kap + P.m[0].gG * J2) +
                    phi2 * (P.m[1].gi * p + P.m[1].kap + P.m[1].gG * J2);
    const float Gm = (phi1 * P.m[0].GoG + phi2 * P.m[1].GoG) * ixi;
    return (a * ixi + (4.f / 3.f) * Gm) / rho;
  }
  const float a = phi1 * rc2_of(P.m[0], r1, p, J2) + phi2 * rc2_of(P.m[1], r2, p, J2);
  return (a * ixi + (4.f / 3.f) * Gmix_f<GEN>(P, phi1, r1, r2)) / rho;
}

// minmod(a, b) as the median of (0, a, b): the smaller magnitude for equal
// signs, 0 otherwise; four min/max operations and no multiply.
__device__ __forceinline__ float minmod_f(float a, float b) {
  return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.f));
}

// Limited slope: LIM 0 minmod, 1 van Leer (2 a b / (a + b) for a b > 0);
// a compile-time choice, so the default minmod kernels carry no branch.
template <int LIM>
__device__ __forceinline__ float limited_f(float a, float b, int lim_rt = 0) {
  if constexpr (LIM == 0) return minmod_f(a, b);
  if constexpr (LIM < 0) {  // chosen at run time (the general-closure kernels)
    if (!lim_rt) return minmod_f(a, b);
  }
  const float ab = a * b;
  return ab > 0.f ? 2.f * ab / (a + b) : 0.f;
}

struct CandF {
  float mL, mR, tL, tR;
  bool mixed;  // THINC applied (tL, tR differ from mL, mR only then)
};

// beta_of() gives the THINC steepness; it is evaluated only in a mixed cell.
template <int LIM = 0, class BetaFn>
__device__ __forceinline__ CandF phi_cand_f(float qm, float qc, float qp, const BetaFn& beta_of, bool thinc,
                                            int lim_rt = 0) {
  CandF c;
  const float s = limited_f<LIM>(qc - qm, qp - qc, lim_rt);
  c.mL = qc - 0.5f * s;
  c.mR = qc + 0.5f * s;
  c.tL = c.mL;
  c.tR = c.mR;
  c.mixed = false;
  if (thinc) {
    const float qmin = fminf(qm, qp);
    const float jump = fmaxf(qm, qp) - qmin;
    const float C = (qc - qmin + 1e-20f) / (jump + 1e-20f);
    if (C > 1e-5f && C < 1.f - 1e-5f && (qp - qc) * (qc - qm) > 0.f) {
      const float beta = beta_of();
      const float th = (qp - qm) > 0.f ? 1.f : -1.f;
      const float B = expf(th * beta * (2.f * C - 1.f));
      const float tb = tanhf(beta);
      const float A = (B / coshf(beta) - 1.f) / tb;
      c.tL = qmin + 0.5f * jump * (1.f + th * A);
      c.tR = qmin + 0.5f * jump * (1.f + th * (tb + A) / (1.f + A * tb));
      c.mixed = true;
    }
  }
  return c;
}

__device__ __forceinline__ void bvd_f(const CandF& km, const CandF& k, const CandF& kp, float& L, float& R) {
  const float tT = fminf(fabsf(km.mR - k.tL), fabsf(km.tR - k.tL)) + fminf(fabsf(k.tR - kp.mL), fabsf(k.tR - kp.tL));
  const float tM = fminf(fabsf(km.mR - k.mL), fabsf(km.tR - k.mL)) + fminf(fabsf(k.mR - kp.mL), fabsf(k.mR - kp.tL));
  const bool useT = tT < tM;
  L = useT ? k.tL : k.mL;
  R = useT ? k.tR : k.mR;
}

struct FStateF {
  float phi, ar1, ar2, arl, rho, un, ut, rhoE, snn, snt, cL, Gm;  // rhoE: soft part only
  float V11, V12, V21, V22, V33;
};

template <int DIR, bool GEN = true>
__device__ __forceinline__ FStateF face_state_f(const PhysF& P, const PrimF& w) {
  FStateF s;
  const StrainF st = strain_f(w.V11, w.V12, w.V21, w.V22, w.V33);
  s.phi = w.phi;
  s.ar1 = w.phi * w.r1;
  s.ar2 = (1.f - w.phi) * w.r2;
  s.rho = s.ar1 + s.ar2;
  s.arl = 0.f;
  if (P.y >= 0) s.arl = (P.y == 0 ? s.ar1 : s.ar2) * w.lam;
  const float ixi = 1.f / xi_f(P, w.phi);
  s.rhoE = w.p / ixi + soft_ref_f<GEN>(P, w.phi, s.ar1, s.ar2, s.arl, st.J2, w.r1, w.r2) +
           0.5f * s.rho * (w.u * w.u + w.v * w.v);
  const float Gm = Gmix_f<GEN>(P, w.phi, w.r1, w.r2);
  s.Gm = Gm;
  if (DIR == 0) {
    s.un = w.u;
    s.ut = w.v;
    s.snn = -w.p + 2.f * Gm * st.H11;
  } else {
    s.un = w.v;
    s.ut = w.u;
    s.snn = -w.p + 2.f * Gm * st.H22;
  }
  s.snt = 2.f * Gm * st.H12;
  s.cL = cL2_f<GEN>(P, w.phi, s.rho, w.p, st.J2, w.r1, w.r2);  // squared; k_flux32 takes the root
  s.V11 = w.V11;
  s.V12 = w.V12;
  s.V21 = w.V21;
  s.V22 = w.V22;
  s.V33 = w.V33;
  return s;
}

struct FaceOutF {
  float Far1, Far2, Farl, Fmn, Fmt, FE, X;  // FE: soft energy flux; X: kappa flux factor
  float D;                                  // X - u_face (small: star compression correction)
  float phi, un, ut, V11, V12, V21, V22, V33;
};

// HLLD-type solver of physics.cuh in float, with the kappa part split off.
template <int DIR>
__device__ __forceinline__ FaceOutF hlld_f(const FStateF& L, const FStateF& R) {
  const float SL = fminf(L.un - L.cL, R.un - R.cL);
  const float SR = fmaxf(L.un + L.cL, R.un + R.cL);
  const float mL = L.rho * (SL - L.un);
  const float mR = R.rho * (SR - R.un);
  const float Ss = ((L.snn - R.snn) + mul_rn(mL, L.un) - mul_rn(mR, R.un)) / (mL - mR);
  const float rL = (SL - L.un) / (SL - Ss), rR = (SR - R.un) / (SR - Ss);
  const float rsL = rL * L.rho, rsR = rR * R.rho;
  const float csL = sqrtf(L.Gm / rsL), csR = sqrtf(R.Gm / rsR);
  const float ZL = rsL * csL, ZR = rsR * csR;
  const float SsL = Ss - csL, SsR = Ss + csR;
  float ut2 = 0.f, st2 = 0.f;
  const bool shear = ZL + ZR > 0.f;
  if (shear) {
    ut2 = (ZL * L.ut + ZR * R.ut + R.snt - L.snt) / (ZL + ZR);
    st2 = L.snt + ZL * (ut2 - L.ut);
  }
  int level;
  bool left;
  if (SL >= 0.f) { left = true; level = 0; }
  else if (SsL >= 0.f) { left = true; level = 1; }
  else if (Ss >= 0.f) { left = true; level = 2; }
  else if (SsR >= 0.f) { left = false; level = 2; }
  else if (SR >= 0.f) { left = false; level = 1; }
  else { left = false; level = 0; }
  const float phi = left ? L.phi : R.phi, ar1 = left ? L.ar1 : R.ar1, ar2 = left ? L.ar2 : R.ar2;
  const float arl = left ? L.arl : R.arl, rho = left ? L.rho : R.rho, un = left ? L.un : R.un;
  const float ut = left ? L.ut : R.ut, rhoE = left ? L.rhoE : R.rhoE, snn = left ? L.snn : R.snn;
  const float snt = left ? L.snt : R.snt;
  const float V11 = left ? L.V11 : R.V11, V12 = left ? L.V12 : R.V12, V21 = left ? L.V21 : R.V21;
  const float V22 = left ? L.V22 : R.V22, V33 = left ? L.V33 : R.V33;
  const float S = left ? SL : SR, r = left ? rL : rR, Sh = left ? SsL : SsR;
  const float ut2K = shear ? ut2 : ut, st2K = shear ? st2 : snt;
  FaceOutF o;
  o.Far1 = ar1 * un;
  o.Far2 = ar2 * un;
  o.Farl = arl * un;
  o.Fmn = rho * un * un - snn;
  o.Fmt = rho * ut * un - snt;
  o.FE = rhoE * un - (un * snn + ut * snt);
  o.X = un;
  o.D = 0.f;
  o.phi = phi;
  o.un = un;
  o.ut = ut;
  o.V11 = V11; o.V12 = V12; o.V21 = V21; o.V22 = V22; o.V33 = V33;
  if (level > 0) {
    const float r1 = r - 1.f;
    const float snn_s = snn - rho * (S - un) * (Ss - un);
    const float E_s = (rhoE * (S - un) + un * snn - Ss * snn_s) / (S - Ss);
    o.Far1 += S * r1 * ar1;
    o.Far2 += S * r1 * ar2;
    o.Farl += S * r1 * arl;
    o.Fmn += S * (r * rho * Ss - rho * un);
    o.Fmt += S * r1 * rho * ut;
    o.FE += S * (E_s - rhoE);
    o.X = un + S * r1;
    o.D = (Ss - un) * Ss / (S - Ss);
    o.un = Ss;
    // r^(1/3) and r^(-2/3) as powers of two of log2(r) / 3 (r > 0)
    const float lr = __log2f(r) * (1.f / 3.f);
    const float c1 = exp2f(lr);
    const float cn = exp2f(-2.f * lr);
    if (DIR == 0) {
      o.V11 = cn * V11; o.V12 = cn * V12; o.V21 = c1 * V21; o.V22 = c1 * V22;
    } else {
      o.V11 = c1 * V11; o.V12 = c1 * V12; o.V21 = cn * V21; o.V22 = cn * V22;
    }
    o.V33 = c1 * V33;
    if (level == 2) {
      const float dS = Sh - Ss;
      if (dS != 0.f) {
        const float idS = 1.f / dS;
        o.Fmt += Sh * r * rho * (ut2K - ut);
        o.FE -= Sh * (ut2K * st2K - ut * snt) * idS;
        const float w = (ut - ut2K) * idS;
        if (DIR == 0) {
          o.V21 += w * o.V11;
          o.V22 += w * o.V12;
        } else {
          o.V11 += w * o.V21;
          o.V12 += w * o.V22;
        }
        o.ut = ut2K;
      }
    }
  }
  return o;
}

// Plastic update of Section 3.2 in float; r1, r2 the phasic densities (the
// Romenskii yield strain sigma_y / (sqrt 6 G(r))).
template <bool GEN = true>
__device__ __forceinline__ void plastic_f(const PhysF& P, float phi1, float dt, float& V11, float& V12,
                                          float& V21, float& V22, float& V33, float r1, float r2) {
  const StrainF s = strain_f(V11, V12, V21, V22, V33);
  const float Js = sqrtf(s.J2);
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const MatT<float>& m = P.m[l];
    const float ph = l == 0 ? phi1 : 1.f - phi1;
    const float JY = GEN && m.eos == EOS_ROMENSKII ? m.sigy / (2.4494897f * shear_of(m, l == 0 ? r1 : r2)) : m.JY;
    float Jl;
    if (m.G == 0.f) Jl = 0.f;
    else if (m.plastic == 1) Jl = fminf(Js, JY);
    else if (m.plastic == 2) Jl = Js > JY ? fmaxf(Js - dt * m.chi0, JY) : Js;
    else Jl = Js;
    num += ph * m.iGm1 * Jl;
    den += ph * m.iGm1;
  }
  const float sc = Js > 0.f ? (num / den) / Js : 0.f;
  const float h11 = sc * s.H11, h12 = sc * s.H12, h22 = sc * s.H22, h33 = sc * s.H33;
  const float x11 = 1.f - 0.5f * h11, x12 = -0.5f * h12, x22 = 1.f - 0.5f * h22;
  const float y11 = 1.f + 0.5f * h11, y12 = 0.5f * h12, y22 = 1.f + 0.5f * h22;
  const float id = 1.f / (x11 * x22 - x12 * x12);
  const float i11 = x22 * id, i12 = -x12 * id, i22 = x11 * id;
  V11 = i11 * y11 + i12 * y12;
  V12 = i11 * y12 + i12 * y22;
  V21 = i12 * y11 + i22 * y12;
  V22 = i12 * y12 + i22 * y22;
  V33 = (1.f + 0.5f * h33) / (1.f - 0.5f * h33);
}

}  // namespace dis
