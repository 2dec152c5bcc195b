// local_vjp.cuh - hand-written reverses (vector-Jacobian products) of the
// local maps of the float64 step: the face Riemann problem (riemann_outputs /
// hllc of face.cuh and physics.cuh), the face-state map (face_state), the
// conservative -> primitive recovery (prim_of), the THINC-BVD edge values of
// phi (face_phi) and the source steps (plastic, sources).
//
// Given the adjoint of the face outputs (NF fluxes + the face-state extras),
// accumulate the adjoints of the two face states (FState fields, c_L still
// squared as face_state returns it).  The forward pass is recomputed here in
// the same order, so every branch (wave-speed min / max, shear coupling,
// region at x/t = 0, zero shear-wave width) is the one the forward step took;
// ties and non-differentiable points follow the conventions of dual.cuh
// (min / max of equal values split the derivative, sqrt has derivative 0 at
// 0).  face_state_vjp, prim_of_vjp and face_phi_vjp reverse the other maps
// the same way.  A
// test compares these reverses with the dual-number evaluation of the same
// forward code.
#pragma once
#include "face.cuh"

namespace dis {

// d minmod(a, b) / da and / db on the branch the forward took; equal
// magnitudes split the derivative (the min convention of dual.cuh).
__device__ __forceinline__ void minmod_grad(double a, double b, double& da, double& db) {
  da = db = 0.0;
  if (a * b > 0.0) {
    if (fabs(b) < fabs(a)) db = 1.0;
    else if (fabs(a) < fabs(b)) da = 1.0;
    else da = db = 0.5;
  }
}

// The same for the limiter lim (0 minmod; 1 van Leer's harmonic limiter
// 2ab / (a + b) where ab > 0: d/da = 2 b^2 / (a + b)^2, d/db = 2 a^2 / (a + b)^2).
__device__ __forceinline__ void limiter_grad(double a, double b, int lim, double& da, double& db) {
  if (lim == 0) {
    minmod_grad(a, b, da, db);
    return;
  }
  da = db = 0.0;
  if (a * b > 0.0) {
    const double s = a + b;
    da = 2.0 * b * b / (s * s);
    db = 2.0 * a * a / (s * s);
  }
}

// Adjoint of one star state (star_of) into its side K, S and S*.
template <int DIR>
__device__ __forceinline__ void star_of_vjp(const FState& K, double S, double Ss, const StarT<double>& t,
                                            const StarT<double>& tb, FState& Kb, double& Sb, double& Ssb) {
  const double inv = 1.0 / (S - Ss);
  const double c1 = cbrt(t.r);
  const double cn = 1.0 / (c1 * c1);
  double c1b = 0.0, cnb = 0.0;
  if (DIR == 0) {
    cnb += tb.V11 * K.V11 + tb.V12 * K.V12;
    Kb.V11 += tb.V11 * cn;
    Kb.V12 += tb.V12 * cn;
    c1b += tb.V21 * K.V21 + tb.V22 * K.V22;
    Kb.V21 += tb.V21 * c1;
    Kb.V22 += tb.V22 * c1;
  } else {
    c1b += tb.V11 * K.V11 + tb.V12 * K.V12;
    Kb.V11 += tb.V11 * c1;
    Kb.V12 += tb.V12 * c1;
    cnb += tb.V21 * K.V21 + tb.V22 * K.V22;
    Kb.V21 += tb.V21 * cn;
    Kb.V22 += tb.V22 * cn;
  }
  c1b += tb.V33 * K.V33;
  Kb.V33 += tb.V33 * c1;
  c1b += cnb * (-2.0 * cn / c1);          // cn = c1^-2
  double rb = tb.r + c1b / (3.0 * c1 * c1);  // c1 = r^(1/3)
  // E* = A inv, A = rhoE (S - un) + un snn - Ss snn*
  const double A = K.rhoE * (S - K.un) + K.un * K.snn - Ss * t.snn;
  const double Ab = tb.E * inv;
  double invb = tb.E * A;
  Kb.rhoE += Ab * (S - K.un);
  Sb += Ab * K.rhoE;
  Kb.un += Ab * (K.snn - K.rhoE);
  Kb.snn += Ab * K.un;
  Ssb -= Ab * t.snn;
  const double snnb = tb.snn - Ab * Ss;
  // snn* = snn - m (Ss - un), m = rho (S - un)
  const double m = K.rho * (S - K.un);
  Kb.snn += snnb;
  const double mb = -snnb * (Ss - K.un);
  Ssb -= snnb * m;
  Kb.un += snnb * m;
  Kb.rho += mb * (S - K.un);
  Sb += mb * K.rho;
  Kb.un -= mb * K.rho;
  // r = (S - un) inv, inv = 1 / (S - Ss)
  Sb += rb * inv;
  Kb.un -= rb * inv;
  invb += rb * (S - K.un);
  const double d = -invb * inv * inv;
  Sb += d;
  Ssb -= d;
}

// min / max with the split-derivative tie convention: adjoint of the result
// into the two arguments.
__device__ __forceinline__ void min_vjp(double a, double b, double rb, double& ab, double& bb) {
  if (b < a) bb += rb;
  else if (a < b) ab += rb;
  else { ab += 0.5 * rb; bb += 0.5 * rb; }
}
__device__ __forceinline__ void max_vjp(double a, double b, double rb, double& ab, double& bb) {
  if (b > a) bb += rb;
  else if (a > b) ab += rb;
  else { ab += 0.5 * rb; bb += 0.5 * rb; }
}

// Reverse of riemann_outputs<DIM, RX, DIR>(L0, R0, F): Fb holds the adjoint of
// F (n_face_out values); Lb, Rb (zero on entry) receive the adjoints of L0, R0.
template <int DIM, bool RX, int DIR>
__device__ void riemann_outputs_vjp(const FState& L0, const FState& R0, const double* Fb, FState& Lb,
                                    FState& Rb) {
  using L_ = Lay<DIM, RX>;
  constexpr int NF = L_::NF;
  // ---- forward, as in riemann_outputs / hllc
  FState L = L0, R = R0;
  L.cL = sqrt(L0.cL);
  R.cL = sqrt(R0.cL);
  const double aL = L.un - L.cL, aR = R.un - R.cL, bL = L.un + L.cL, bR = R.un + R.cL;
  const double SL = fmin(aL, aR), SR = fmax(bL, bR);
  const double mL = L.rho * (SL - L.un), mR = R.rho * (SR - R.un);
  const double num = (L.snn - R.snn) + mul_rn(mL, L.un) - mul_rn(mR, R.un), den = mL - mR;
  const double Ss = num / den;
  const StarT<double> sL = star_of<DIR>(L, SL, Ss), sR = star_of<DIR>(R, SR, Ss);
  const double rsL = sL.r * L.rho, rsR = sR.r * R.rho;
  const double csL = sqrt(L.Gm / rsL), csR = sqrt(R.Gm / rsR);
  const double ZL = rsL * csL, ZR = rsR * csR;
  const double SsL = Ss - csL, SsR = Ss + csR;
  const bool shear = ZL + ZR > 0.0;
  double ut2c = 0.0, st2c = 0.0;
  if (shear) {
    ut2c = (ZL * L.ut + ZR * R.ut + R.snt - L.snt) / (ZL + ZR);
    st2c = L.snt + ZL * (ut2c - L.ut);
  }
  int level;
  bool left;
  if (SL >= 0.0) { left = true; level = 0; }
  else if (SsL >= 0.0) { left = true; level = 1; }
  else if (Ss >= 0.0) { left = true; level = 2; }
  else if (SsR >= 0.0) { left = false; level = 2; }
  else if (SR >= 0.0) { left = false; level = 1; }
  else { left = false; level = 0; }
  const FState& K = left ? L : R;
  const StarT<double>& sK = left ? sL : sR;
  const double S = left ? SL : SR;
  const double Sh = left ? SsL : SsR;
  const double ut2 = shear ? ut2c : K.ut;
  const double st2 = shear ? st2c : K.snt;
  const double un = K.un, ut = K.ut;
  const double dS = Sh - Ss;
  const bool shear_region = level == 2 && dS != 0.0;
  const double idS = shear_region ? 1.0 / dS : 0.0;
  const double w = shear_region ? (ut - ut2) * idS : 0.0;
  // face state (o) values needed by the output map
  double o_un = level == 0 ? un : Ss;
  double o_ut = shear_region ? ut2 : ut;
  double oV11 = level == 0 ? K.V11 : sK.V11, oV12 = level == 0 ? K.V12 : sK.V12;
  double oV21 = level == 0 ? K.V21 : sK.V21, oV22 = level == 0 ? K.V22 : sK.V22;
  const double oV33 = level == 0 ? K.V33 : sK.V33;
  if (shear_region) {
    if (DIR == 0) {
      oV21 = sK.V21 + w * sK.V11;
      oV22 = sK.V22 + w * sK.V12;
    } else {
      oV11 = sK.V11 + w * sK.V21;
      oV12 = sK.V12 + w * sK.V22;
    }
  }
  const double o_phi = K.phi;

  // ---- reverse of the output map (riemann_outputs)
  double phib = 0.0, unb = 0.0, utb = 0.0;
  double V11b = 0.0, V12b = 0.0, V21b = 0.0, V22b = 0.0, V33b = 0.0;
  const double Far1b = Fb[L_::A1], Far2b = Fb[L_::A2];
  const double Farlb = RX ? Fb[L_::AL] : 0.0;
  double Fmnb, Fmtb = 0.0;
  if (DIR == 0) {
    Fmnb = Fb[L_::MX];
    if constexpr (DIM == 2) Fmtb = Fb[L_::MY];
  } else {
    Fmtb = Fb[L_::MX];
    Fmnb = Fb[L_::MY];
  }
  const double FEb = Fb[L_::E];
  phib += Fb[L_::PHI] * o_un;
  unb += Fb[L_::PHI] * o_phi;
  const double fu = DIR == 0 ? o_un : o_ut, fv = DIR == 0 ? o_ut : o_un;
  double fub = 0.0, fvb = 0.0;
  if (DIR == 0) {
    if constexpr (DIM == 2) {
      const double b21 = Fb[L_::V21], b22 = Fb[L_::V22];
      V21b += b21 * fu; fub += b21 * oV21; V11b -= b21 * fv; fvb -= b21 * oV11;
      V22b += b22 * fu; fub += b22 * oV22; V12b -= b22 * fv; fvb -= b22 * oV12;
      V12b += Fb[NF + 2];
    } else {
      const double b22 = Fb[L_::V22];
      V22b += b22 * fu; fub += b22 * oV22;
    }
    const double b33 = Fb[L_::V33];
    V33b += b33 * fu; fub += b33 * oV33;
    unb += Fb[NF + 0];
    V11b += Fb[NF + 1];
    unb += fub;
    utb += fvb;
  } else if constexpr (DIM == 2) {
    const double b11 = Fb[L_::V11], b12 = Fb[L_::V12], b33 = Fb[L_::V33];
    V11b += b11 * fv; fvb += b11 * oV11; V21b -= b11 * fu; fub -= b11 * oV21;
    V12b += b12 * fv; fvb += b12 * oV12; V22b -= b12 * fu; fub -= b12 * oV22;
    V33b += b33 * fv; fvb += b33 * oV33;
    unb += Fb[NF + 0];
    V21b += Fb[NF + 1];
    V22b += Fb[NF + 2];
    utb += fub;
    unb += fvb;
  }

  // ---- reverse of hllc
  FState& Kb = left ? Lb : Rb;
  StarT<double> sLb{}, sRb{};
  StarT<double>& sKb = left ? sLb : sRb;
  double Sb = 0.0, Shb = 0.0, Ssb = 0.0, ut2b = 0.0, st2b = 0.0;
  Kb.phi += phib;
  if (level == 0) {
    Kb.un += unb;
    Kb.ut += utb;
    Kb.V11 += V11b; Kb.V12 += V12b; Kb.V21 += V21b; Kb.V22 += V22b; Kb.V33 += V33b;
  } else {
    Ssb += unb;
    if (shear_region) ut2b += utb;
    else Kb.ut += utb;
    double wb = 0.0;
    if (shear_region) {
      if (DIR == 0) {
        sKb.V21 += V21b; wb += V21b * sK.V11; sKb.V11 += V21b * w;
        sKb.V22 += V22b; wb += V22b * sK.V12; sKb.V12 += V22b * w;
        sKb.V11 += V11b; sKb.V12 += V12b;
      } else {
        sKb.V11 += V11b; wb += V11b * sK.V21; sKb.V21 += V11b * w;
        sKb.V12 += V12b; wb += V12b * sK.V22; sKb.V22 += V12b * w;
        sKb.V21 += V21b; sKb.V22 += V22b;
      }
      sKb.V33 += V33b;
      // Fmt += Sh rs (ut2 - ut), rs = sK.r K.rho
      const double rs = sK.r * K.rho;
      Shb += Fmtb * rs * (ut2 - ut);
      const double rsb = Fmtb * Sh * (ut2 - ut);
      ut2b += Fmtb * Sh * rs;
      Kb.ut -= Fmtb * Sh * rs;
      // FE -= Sh P idS, P = ut2 st2 - ut snt
      const double Pv = ut2 * st2 - ut * K.snt;
      Shb -= FEb * Pv * idS;
      const double Pb = -FEb * Sh * idS;
      double idSb = -FEb * Sh * Pv;
      ut2b += Pb * st2;
      st2b += Pb * ut2;
      Kb.ut -= Pb * K.snt;
      Kb.snt -= Pb * ut;
      // w = (ut - ut2) idS
      Kb.ut += wb * idS;
      ut2b -= wb * idS;
      idSb += wb * (ut - ut2);
      const double dSb = -idSb * idS * idS;
      Shb += dSb;
      Ssb -= dSb;
      sKb.r += rsb * K.rho;
      Kb.rho += rsb * sK.r;
    } else {
      sKb.V11 += V11b; sKb.V12 += V12b; sKb.V21 += V21b; sKb.V22 += V22b; sKb.V33 += V33b;
    }
    // level >= 1 increments
    const double r1 = sK.r - 1.0;
    double r1b = 0.0;
    Sb += Far1b * r1 * K.ar1; r1b += Far1b * S * K.ar1; Kb.ar1 += Far1b * S * r1;
    Sb += Far2b * r1 * K.ar2; r1b += Far2b * S * K.ar2; Kb.ar2 += Far2b * S * r1;
    Sb += Farlb * r1 * K.arl; r1b += Farlb * S * K.arl; Kb.arl += Farlb * S * r1;
    const double X = sK.r * K.rho * Ss - K.rho * un;
    Sb += Fmnb * X;
    const double Xb = Fmnb * S;
    sKb.r += Xb * K.rho * Ss;
    Kb.rho += Xb * (sK.r * Ss - un);
    Ssb += Xb * sK.r * K.rho;
    Kb.un -= Xb * K.rho;
    Sb += Fmtb * r1 * K.rho * ut;
    r1b += Fmtb * S * K.rho * ut;
    Kb.rho += Fmtb * S * r1 * ut;
    Kb.ut += Fmtb * S * r1 * K.rho;
    Sb += FEb * (sK.E - K.rhoE);
    sKb.E += FEb * S;
    Kb.rhoE -= FEb * S;
    sKb.r += r1b;
  }
  // base fluxes of side K
  Kb.ar1 += Far1b * un; Kb.un += Far1b * K.ar1;
  Kb.ar2 += Far2b * un; Kb.un += Far2b * K.ar2;
  Kb.arl += Farlb * un; Kb.un += Farlb * K.arl;
  Kb.rho += Fmnb * un * un; Kb.un += Fmnb * 2.0 * K.rho * un; Kb.snn -= Fmnb;
  Kb.rho += Fmtb * ut * un; Kb.ut += Fmtb * K.rho * un; Kb.un += Fmtb * K.rho * ut; Kb.snt -= Fmtb;
  Kb.rhoE += FEb * un; Kb.un += FEb * (K.rhoE - K.snn); Kb.snn -= FEb * un; Kb.ut -= FEb * K.snt;
  Kb.snt -= FEb * ut;
  // S, Sh and the shear state of the chosen side
  double SLb = 0.0, SRb = 0.0, SsLb = 0.0, SsRb = 0.0;
  if (left) { SLb += Sb; SsLb += Shb; } else { SRb += Sb; SsRb += Shb; }
  double ZLb = 0.0, ZRb = 0.0;
  if (shear) {
    // st2 = L.snt + ZL (ut2 - L.ut)
    Lb.snt += st2b;
    ZLb += st2b * (ut2c - L.ut);
    ut2b += st2b * ZL;
    Lb.ut -= st2b * ZL;
    // ut2 = N / Zs, N = ZL L.ut + ZR R.ut + R.snt - L.snt, Zs = ZL + ZR
    const double Zs = ZL + ZR;
    const double Nb = ut2b / Zs;
    const double Zsb = -ut2b * ut2c / Zs;
    ZLb += Nb * L.ut + Zsb;
    Lb.ut += Nb * ZL;
    ZRb += Nb * R.ut + Zsb;
    Rb.ut += Nb * ZR;
    Rb.snt += Nb;
    Lb.snt -= Nb;
  } else {
    Kb.ut += ut2b;
    Kb.snt += st2b;
  }
  // Z = rs cs, cs = sqrt(Gm / rs); SsL = Ss - csL, SsR = Ss + csR
  {
    const double csb = ZLb * rsL - SsLb;
    double rsb = ZLb * csL;
    Ssb += SsLb;
    if (csL > 0.0) {
      const double xb = csb / (2.0 * csL);
      Lb.Gm += xb / rsL;
      rsb -= xb * L.Gm / (rsL * rsL);
    }
    sLb.r += rsb * L.rho;
    Lb.rho += rsb * sL.r;
  }
  {
    const double csb = ZRb * rsR + SsRb;
    double rsb = ZRb * csR;
    Ssb += SsRb;
    if (csR > 0.0) {
      const double xb = csb / (2.0 * csR);
      Rb.Gm += xb / rsR;
      rsb -= xb * R.Gm / (rsR * rsR);
    }
    sRb.r += rsb * R.rho;
    Rb.rho += rsb * sR.r;
  }
  // star states
  star_of_vjp<DIR>(L, SL, Ss, sL, sLb, Lb, SLb, Ssb);
  star_of_vjp<DIR>(R, SR, Ss, sR, sRb, Rb, SRb, Ssb);
  // Ss = num / den
  const double numb = Ssb / den, denb = -Ssb * Ss / den;
  Lb.snn += numb;
  Rb.snn -= numb;
  const double mLb = numb * L.un + denb, mRb = -numb * R.un - denb;
  Lb.un += numb * mL;
  Rb.un -= numb * mR;
  Lb.rho += mLb * (SL - L.un); SLb += mLb * L.rho; Lb.un -= mLb * L.rho;
  Rb.rho += mRb * (SR - R.un); SRb += mRb * R.rho; Rb.un -= mRb * R.rho;
  // SL = min(L.un - L.cL, R.un - R.cL), SR = max(L.un + L.cL, R.un + R.cL)
  double aLb = 0.0, aRb = 0.0, bLb = 0.0, bRb = 0.0;
  min_vjp(aL, aR, SLb, aLb, aRb);
  max_vjp(bL, bR, SRb, bLb, bRb);
  Lb.un += aLb + bLb;
  Rb.un += aRb + bRb;
  double cLLb = Lb.cL - aLb + bLb;  // Lb.cL may hold nothing yet: the sqrt'ed c_L enters only here
  double cLRb = Rb.cL - aRb + bRb;
  // c_L = sqrt(c_L^2)
  Lb.cL = L.cL > 0.0 ? cLLb / (2.0 * L.cL) : 0.0;
  Rb.cL = R.cL > 0.0 ? cLRb / (2.0 * R.cL) : 0.0;
}

// Adjoint of strain_of (physics.cuh): given the adjoints of H11, H12, H22,
// H33 and J2, add those of V11, V12, V21, V22, V33.  The
// map dev(1/4 (B - B^-1)), B = V V^T in plane-strain block form, is reversed
// through B and the 2 x 2 inverse.
__device__ __forceinline__ void strain_vjp(double a, double b, double c, double d, double e, double H11b,
                                           double H12b, double H22b, double H33b_in, double J2b, double& ab,
                                           double& bb, double& cb, double& db, double& eb) {
  const double B11 = a * a + b * b, B12 = a * c + b * d, B22 = c * c + d * d, B33 = e * e;
  const double idet = 1.0 / (B11 * B22 - B12 * B12);
  const double M11 = 0.25 * (B11 - B22 * idet);
  const double M22 = 0.25 * (B22 - B11 * idet);
  const double M12 = 0.25 * (B12 + B12 * idet);
  const double M33 = 0.25 * (B33 - 1.0 / B33);
  const double t3 = (M11 + M22 + M33) * (1.0 / 3.0);
  const double H11 = M11 - t3, H22 = M22 - t3, H33 = M33 - t3, H12 = M12;
  // J2 = H11^2 + H22^2 + H33^2 + 2 H12^2, H_ii = M_ii - t3
  H11b += 2.0 * H11 * J2b;
  H22b += 2.0 * H22 * J2b;
  const double H33b = H33b_in + 2.0 * H33 * J2b;
  H12b += 4.0 * H12 * J2b;
  const double t3b = -(H11b + H22b + H33b) * (1.0 / 3.0);
  const double M11b = H11b + t3b, M22b = H22b + t3b, M33b = H33b + t3b, M12b = H12b;
  double B11b = 0.25 * M11b - 0.25 * M22b * idet;
  double B22b = 0.25 * M22b - 0.25 * M11b * idet;
  double B12b = 0.25 * M12b * (1.0 + idet);
  const double idetb = -0.25 * M11b * B22 - 0.25 * M22b * B11 + 0.25 * M12b * B12;
  const double B33b = 0.25 * M33b * (1.0 + 1.0 / (B33 * B33));
  const double detb = -idetb * idet * idet;
  B11b += detb * B22;
  B22b += detb * B11;
  B12b -= 2.0 * detb * B12;
  ab += 2.0 * a * B11b + c * B12b;
  bb += 2.0 * b * B11b + d * B12b;
  cb += a * B12b + 2.0 * c * B22b;
  db += b * B12b + 2.0 * d * B22b;
  eb += 2.0 * e * B33b;
}

// Adjoint of the cylindrical geometric source (add_geometric, step_kernels.cuh;
// the s_g of Section 3 with x = r): given Db, the adjoint of the stage operator
// D at a cell of radius r, add the adjoints of the cell's conservative state q
// (qb), of its primitives w (wb: p, u, v, phi and V through the stress) and of
// the shear moduli G_1, G_2 (thb[0], thb[3]; may be null).
template <int DIM, bool RX>
__device__ __forceinline__ void geometric_vjp(const Phys& P, const double* q, const Prim& w, double r,
                                              const double* Db, double* qb, Prim& wb, double* thb) {
  using L = Lay<DIM, RX>;
  const double ir = 1.0 / r;
  const Strain st = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const double xi = xi_of(P, w.phi);
  const double Nm = w.phi * P.m[0].GoG + (1.0 - w.phi) * P.m[1].GoG;
  const double Gm2 = 2.0 * Nm / xi;
  const double srr = -w.p + Gm2 * st.H11, szr = Gm2 * st.H12;
  const double ur = w.u, uz = DIM == 2 ? w.v : 0.0;
  const double rho = q[L::A1] + q[L::A2];
  double urb = 0.0, uzb = 0.0, srrb = 0.0, szrb = 0.0, sttb = 0.0, rhob = 0.0;
  // D_l += q_l u_r / r for the partial densities (and phi_y rho_y lam)
  qb[L::A1] += Db[L::A1] * ur * ir;
  qb[L::A2] += Db[L::A2] * ur * ir;
  urb += (Db[L::A1] * q[L::A1] + Db[L::A2] * q[L::A2]) * ir;
  if constexpr (RX) {
    qb[L::AL] += Db[L::AL] * ur * ir;
    urb += Db[L::AL] * q[L::AL] * ir;
  }
  // D_mr += (rho u_r^2 - s_rr + s_tt) / r
  rhob += Db[L::MX] * ur * ur * ir;
  urb += Db[L::MX] * 2.0 * rho * ur * ir;
  srrb -= Db[L::MX] * ir;
  sttb += Db[L::MX] * ir;
  if constexpr (DIM == 2) {  // D_mz += (rho u_z u_r - s_zr) / r
    rhob += Db[L::MY] * uz * ur * ir;
    uzb += Db[L::MY] * rho * ur * ir;
    urb += Db[L::MY] * rho * uz * ir;
    szrb -= Db[L::MY] * ir;
  }
  // D_E += (rho E u_r - u_r s_rr - u_z s_zr) / r
  qb[L::E] += Db[L::E] * ur * ir;
  urb += Db[L::E] * (q[L::E] - srr) * ir;
  uzb -= Db[L::E] * szr * ir;
  srrb -= Db[L::E] * ur * ir;
  szrb -= Db[L::E] * uz * ir;
  // D_Vij += u_r V_ij / (3 r) (i not theta), D_V33 += (1/3 - 1) u_r V33 / r
  const double t = (1.0 / 3.0) * ur * ir;
  double tb = Db[L::V11] * q[L::V11] + Db[L::V22] * q[L::V22];
  qb[L::V11] += Db[L::V11] * t;
  qb[L::V22] += Db[L::V22] * t;
  if constexpr (DIM == 2) {
    tb += Db[L::V12] * q[L::V12] + Db[L::V21] * q[L::V21];
    qb[L::V12] += Db[L::V12] * t;
    qb[L::V21] += Db[L::V21] * t;
  }
  urb += tb * (1.0 / 3.0) * ir;
  qb[L::V33] += Db[L::V33] * (1.0 / 3.0 - 1.0) * ur * ir;
  urb += Db[L::V33] * (1.0 / 3.0 - 1.0) * q[L::V33] * ir;
  qb[L::A1] += rhob;
  qb[L::A2] += rhob;
  // s_rr = -p + Gm2 H11, s_zr = Gm2 H12, s_tt = -p + Gm2 H33
  wb.p -= srrb + sttb;
  const double Gm2b = srrb * st.H11 + szrb * st.H12 + sttb * st.H33;
  strain_vjp(w.V11, w.V12, w.V21, w.V22, w.V33, srrb * Gm2, szrb * Gm2, 0.0, sttb * Gm2, 0.0, wb.V11, wb.V12,
             wb.V21, wb.V22, wb.V33);
  // Gm2 = 2 N / xi, N = phi GoG_1 + (1 - phi) GoG_2, xi = phi iGm1_1 + (1 - phi) iGm1_2
  const double Nb = 2.0 * Gm2b / xi, xib = -Gm2b * Gm2 / xi;
  wb.phi += Nb * (P.m[0].GoG - P.m[1].GoG) + xib * (P.m[0].iGm1 - P.m[1].iGm1);
  if (thb) {  // GoG_l = G_l / Gamma_l
    thb[0] += Nb * w.phi * P.m[0].iGm1;
    thb[3] += Nb * (1.0 - w.phi) * P.m[1].iGm1;
  }
  wb.u += urb;
  if constexpr (DIM == 2) wb.v += uzb;
}


// Adjoint of face_state (primitives -> face state, physics.cuh) at the
// primitive state w: Sb is the adjoint of the face state (c_L squared, as
// face_state returns it); the primitive adjoints are added to wb and, where
// thb is not null, the adjoints of the parameters (G_l at 3 l, Q_l at 3 l + 2;
// sigma_y does not enter) to thb.
template <int DIR>
__device__ __forceinline__ void face_state_vjp(const Phys& P, const Prim& w, const FState& Sb, Prim& wb,
                                               double* thb) {
  const MatDev& m0 = P.m[0];
  const MatDev& m1 = P.m[1];
  const double phi = w.phi, phi2 = 1.0 - phi;
  // forward
  const StrainT<double> st = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const double H11 = st.H11, H22 = st.H22, H12 = st.H12, J2 = st.J2;
  const double ar1 = phi * w.r1, ar2 = phi2 * w.r2, rho = ar1 + ar2;
  const double xi = phi * m0.iGm1 + phi2 * m1.iGm1;
  const double NG_ = phi * m0.GoG + phi2 * m1.GoG;
  const double Gm = NG_ / xi;
  const double A0 = m0.gi * w.p + m0.kap + m0.gG * J2, A1 = m1.gi * w.p + m1.kap + m1.gG * J2;
  const double Aa = phi * A0 + phi2 * A1;
  const double cL2 = (Aa / xi + (4.0 / 3.0) * Gm) / rho;
  // reverse
  double phib = Sb.phi, ar1b = Sb.ar1, ar2b = Sb.ar2, rhob = Sb.rho, pb = 0.0, ub = 0.0, vb = 0.0;
  double Gmb = Sb.Gm, xib = 0.0, J2b = 0.0, H11b = 0.0, H22b = 0.0, H12b = 0.0;
  double gG0b = 0.0, gG1b = 0.0, GoG0b = 0.0, GoG1b = 0.0;
  // c_L^2 = (Aa / xi + 4/3 Gm) / rho
  const double Aab = Sb.cL / (xi * rho);
  xib -= Sb.cL * Aa / (xi * xi * rho);
  Gmb += Sb.cL * (4.0 / 3.0) / rho;
  rhob -= Sb.cL * cL2 / rho;
  phib += Aab * (A0 - A1);
  pb += Aab * (phi * m0.gi + phi2 * m1.gi);
  J2b += Aab * (phi * m0.gG + phi2 * m1.gG);
  gG0b += Aab * phi * J2;
  gG1b += Aab * phi2 * J2;
  // snt = 2 Gm H12; snn = -p + 2 Gm H_nn; un, ut
  Gmb += Sb.snt * 2.0 * H12;
  H12b += Sb.snt * 2.0 * Gm;
  pb -= Sb.snn;
  if (DIR == 0) {
    Gmb += Sb.snn * 2.0 * H11;
    H11b += Sb.snn * 2.0 * Gm;
    ub += Sb.un;
    vb += Sb.ut;
  } else {
    Gmb += Sb.snn * 2.0 * H22;
    H22b += Sb.snn * 2.0 * Gm;
    vb += Sb.un;
    ub += Sb.ut;
  }
  // Gm = NG / xi
  const double NGb = Gmb / xi;
  xib -= Gmb * Gm / xi;
  phib += NGb * (m0.GoG - m1.GoG);
  GoG0b += NGb * phi;
  GoG1b += NGb * phi2;
  // rhoE = xi p + ref + 1/2 rho (u^2 + v^2)
  const double refb = Sb.rhoE;
  xib += Sb.rhoE * w.p;
  pb += Sb.rhoE * xi;
  rhob += Sb.rhoE * 0.5 * (w.u * w.u + w.v * w.v);
  ub += Sb.rhoE * rho * w.u;
  vb += Sb.rhoE * rho * w.v;
  // ref = sum_l phi_l (kap_l + gG_l J2) + sum_l ar_l einf_l - Q_y (ar_y - arl)
  phib += refb * ((m0.kap + m0.gG * J2) - (m1.kap + m1.gG * J2));
  J2b += refb * (phi * m0.gG + phi2 * m1.gG);
  gG0b += refb * phi * J2;
  gG1b += refb * phi2 * J2;
  ar1b += refb * m0.einf;
  ar2b += refb * m1.einf;
  double arlb = Sb.arl, Qb = 0.0;
  if (P.y >= 0) {
    const double ary = P.y == 0 ? ar1 : ar2;
    const double arl = ary * w.lam;
    const double Q = P.m[P.y].Q;
    arlb += refb * Q;
    Qb -= refb * (ary - arl);
    // arl = ar_y lam
    const double aryb = -refb * Q + arlb * w.lam;
    wb.lam += arlb * ary;
    if (P.y == 0) ar1b += aryb;
    else ar2b += aryb;
  }
  // xi = phi iGm1_0 + (1 - phi) iGm1_1
  phib += xib * (m0.iGm1 - m1.iGm1);
  // rho = ar1 + ar2; ar1 = phi r1; ar2 = (1 - phi) r2
  ar1b += rhob;
  ar2b += rhob;
  phib += ar1b * w.r1 - ar2b * w.r2;
  wb.r1 += ar1b * phi;
  wb.r2 += ar2b * phi2;
  wb.phi += phib;
  wb.p += pb;
  wb.u += ub;
  wb.v += vb;
  wb.V11 += Sb.V11;
  wb.V12 += Sb.V12;
  wb.V21 += Sb.V21;
  wb.V22 += Sb.V22;
  wb.V33 += Sb.V33;
  strain_vjp(w.V11, w.V12, w.V21, w.V22, w.V33, H11b, H12b, H22b, 0.0, J2b, wb.V11, wb.V12, wb.V21, wb.V22,
             wb.V33);
  if (thb) {
    // G_l enters through gG_l = gamma_l G_l / (gamma_l - 1), GoG_l = G_l / (gamma_l - 1)
    thb[0] += gG0b * m0.gi + GoG0b * m0.iGm1;
    thb[3] += gG1b * m1.gi + GoG1b * m1.iGm1;
    if (P.y >= 0) thb[3 * P.y + 2] += Qb;
  }
}

// Adjoint of prim_of (face.cuh: conservative -> primitive recovery through the
// mixture pressure function) at the conservative state q: wb is the adjoint of
// the primitive state; the adjoints of the NF conservative slots are added to
// qb and, where thb is not null, those of the parameters (G_l at 3 l through
// the shear energy, Q_l at 3 l + 2) to thb.
template <int DIM, bool RX>
__device__ __forceinline__ void prim_of_vjp(const Phys& P, const double* q, const Prim& wb, double* qb,
                                            double* thb) {
  using L = Lay<DIM, RX>;
  const MatDev& m0 = P.m[0];
  const MatDev& m1 = P.m[1];
  // forward
  const double phi = q[L::PHI], phi2 = 1.0 - phi, a1 = q[L::A1], a2 = q[L::A2];
  const double rho = a1 + a2;
  const double mx = q[L::MX];
  double my = 0.0, V12 = 0.0, V21 = 0.0, arl = 0.0;
  if constexpr (DIM == 2) {
    my = q[L::MY];
    V12 = q[L::V12];
    V21 = q[L::V21];
  }
  if constexpr (RX) arl = q[L::AL];
  const double V11 = q[L::V11], V22 = q[L::V22], V33 = q[L::V33];
  const double u = mx / rho, v = my / rho;
  const StrainT<double> st = strain_of(V11, V12, V21, V22, V33);
  const double xi = phi * m0.iGm1 + phi2 * m1.iGm1;
  const double p = (q[L::E] - 0.5 * (mx * u + my * v) - ref_energy(P, phi, a1, a2, arl, st.J2)) / xi;
  // reverse: p = (E - KE - ref) / xi, KE = (mx^2 + my^2) / (2 rho)
  double phib = wb.phi, a1b = 0.0, a2b = 0.0, rhob = 0.0, mxb = wb.u / rho, myb = wb.v / rho, arlb = 0.0;
  rhob -= (wb.u * u + wb.v * v) / rho;
  const double numb = wb.p / xi;
  phib -= wb.p * p / xi * (m0.iGm1 - m1.iGm1);
  const double Eb = numb;
  mxb -= numb * u;
  myb -= numb * v;
  rhob += numb * 0.5 * (u * u + v * v);
  const double refb = -numb;
  // ref = sum_l phi_l (kap_l + gG_l J2) + a1 einf_1 + a2 einf_2 - Q_y (a_y - arl)
  phib += refb * ((m0.kap + m0.gG * st.J2) - (m1.kap + m1.gG * st.J2));
  const double J2b = refb * (phi * m0.gG + phi2 * m1.gG);
  a1b += refb * m0.einf;
  a2b += refb * m1.einf;
  double Qb = 0.0, ayb = 0.0;
  const double ay = P.y == 0 ? a1 : a2;
  if (P.y >= 0) {
    const double Q = P.m[P.y].Q;
    arlb += refb * Q;
    ayb -= refb * Q;
    Qb = -refb * (ay - arl);
  }
  // lam = arl / a_y
  if constexpr (RX) {
    arlb += wb.lam / ay;
    ayb -= wb.lam * (arl / ay) / ay;
  }
  if (P.y == 0) a1b += ayb;
  else if (P.y == 1) a2b += ayb;
  // r1 = a1 / phi, r2 = a2 / (1 - phi), rho = a1 + a2
  a1b += wb.r1 / phi + rhob;
  a2b += wb.r2 / phi2 + rhob;
  phib += -wb.r1 * (a1 / phi) / phi + wb.r2 * (a2 / phi2) / phi2;
  double V11b = wb.V11, V12b = wb.V12, V21b = wb.V21, V22b = wb.V22, V33b = wb.V33;
  strain_vjp(V11, V12, V21, V22, V33, 0.0, 0.0, 0.0, 0.0, J2b, V11b, V12b, V21b, V22b, V33b);
  qb[L::PHI] += phib;
  qb[L::A1] += a1b;
  qb[L::A2] += a2b;
  qb[L::MX] += mxb;
  qb[L::E] += Eb;
  qb[L::V11] += V11b;
  qb[L::V22] += V22b;
  qb[L::V33] += V33b;
  if constexpr (DIM == 2) {
    qb[L::MY] += myb;
    qb[L::V12] += V12b;
    qb[L::V21] += V21b;
  }
  if constexpr (RX) qb[L::AL] += arlb;
  if (thb) {
    thb[0] += refb * phi * st.J2 * m0.gi;
    thb[3] += refb * phi2 * st.J2 * m1.gi;
    if (P.y >= 0) thb[3 * P.y + 2] += Qb;
  }
}

// Adjoint of one cell's MUSCL / THINC edge candidates (phi_cand, physics.cuh)
// along the edge the BVD choice kept: side 0 = left edge, 1 = right edge;
// thinc_kept: the THINC value was chosen.  Adds the adjoints of q_{i-1},
// q_i, q_{i+1} to qb[0..2] and returns that of beta.
template <class BetaFn>
__device__ __forceinline__ double phi_cand_vjp(double qm, double qc, double qp, const BetaFn& beta_of, bool thinc,
                                               int side, bool thinc_kept, double gb, double* qb, int lim = 0) {
  const bool mixed = [&] {
    if (!thinc) return false;
    const double qmin = fmin(qm, qp);
    const double jump = fmax(qm, qp) - qmin;
    const double C = (qc - qmin + 1e-20) / (jump + 1e-20);
    return C > 1e-5 && C < 1.0 - 1e-5 && (qp - qc) * (qc - qm) > 0.0;
  }();
  if (!(thinc_kept && mixed)) {
    // MUSCL edge q_i -/+ lim(q_i - q_{i-1}, q_{i+1} - q_i) / 2 (the THINC
    // candidate of a cell that is not mixed is the MUSCL one)
    double da, db;
    limiter_grad(qc - qm, qp - qc, lim, da, db);
    const double h = side == 0 ? -0.5 * gb : 0.5 * gb;
    qb[0] -= h * da;
    qb[1] += gb + h * (da - db);
    qb[2] += h * db;
    return 0.0;
  }
  const double beta = beta_of();
  const bool up = qp > qm;  // ordering of the neighbours (strict in a mixed cell)
  const double qmin = up ? qm : qp, qmax = up ? qp : qm;
  const double jump = qmax - qmin;
  const double C = (qc - qmin + 1e-20) / (jump + 1e-20);
  const double th = up ? 1.0 : -1.0;
  const double Bx = exp(th * beta * (2.0 * C - 1.0));
  const double tb = tanh(beta), ch = cosh(beta);
  const double A = (Bx / ch - 1.0) / tb;
  double qminb = gb, jumpb = 0.0, Ab = 0.0, tbb = 0.0;
  if (side == 0) {  // tL = qmin + jump (1 + th A) / 2
    jumpb += gb * 0.5 * (1.0 + th * A);
    Ab += gb * 0.5 * jump * th;
  } else {  // tR = qmin + jump (1 + th (tb + A) / (1 + A tb)) / 2
    const double D = 1.0 + A * tb;
    const double Rr = (tb + A) / D;
    jumpb += gb * 0.5 * (1.0 + th * Rr);
    const double Rrb = gb * 0.5 * jump * th;
    const double Nb = Rrb / D, Db = -Rrb * Rr / D;
    tbb += Nb + Db * A;
    Ab += Nb + Db * tb;
  }
  // A = (B / cosh(beta) - 1) / tanh(beta), B = exp(th beta (2 C - 1))
  const double Bxb = Ab / (ch * tb);
  const double chb = -Ab * Bx / (ch * ch * tb);
  tbb -= Ab * A / tb;
  const double zb = Bxb * Bx;
  double betab = zb * th * (2.0 * C - 1.0) + tbb * (1.0 - tb * tb) + chb * sinh(beta);
  const double Cb = zb * th * beta * 2.0;
  // C = (q_i - qmin + eps) / (jump + eps), jump = qmax - qmin
  const double ie = 1.0 / (jump + 1e-20);
  qb[1] += Cb * ie;
  qminb -= Cb * ie;
  jumpb -= Cb * C * ie;
  const double qmaxb = jumpb;
  qminb -= jumpb;
  qb[up ? 0 : 2] += qminb;
  qb[up ? 2 : 0] += qmaxb;
  return betab;
}

// Adjoint of face_phi (face.cuh): the two phi edge values of a face from the
// 3 x 6 stencil B (rows: tangential neighbours, used only by the 2D Youngs
// normal).  gpL, gpR: adjoints of the left and right edge values; the
// adjoints of the stencil values are added to Bb.  The BVD choices are
// recomputed from the same candidates as the forward code.
template <int DIM>
__device__ __forceinline__ void face_phi_vjp(const double (&B)[3][6], bool thinc, double hn, double ht,
                                             double gpL, double gpR, double (&Bb)[3][6], int lim = 0) {
  const bool normals = DIM == 2 && thinc;
  // THINC steepness of candidate cell s, evaluated only where a mixed cell needs it
  auto beta_of = [&](int s) -> double {
    if (!normals) return 2.51;
    const double dn = (B[2][s + 2] + 2.0 * B[1][s + 2] + B[0][s + 2]) - (B[2][s] + 2.0 * B[1][s] + B[0][s]);
    const double dt_ = (B[2][s + 2] + 2.0 * B[2][s + 1] + B[2][s]) - (B[0][s + 2] + 2.0 * B[0][s + 1] + B[0][s]);
    const double gn = dn / hn, gt = dt_ / ht;
    const double nrm = sqrt(gn * gn + gt * gt);
    return 2.5 * (nrm == 0.0 ? 1.0 : fabs(gn) / nrm) + 0.01;
  };
  Cand c[4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
    c[s] = phi_cand_lazy(B[1][s], B[1][s + 1], B[1][s + 2], [&]() { return beta_of(s); }, thinc, lim);
  // BVD choices (the test of bvd in physics.cuh): the right edge of cell 1
  // (phiL) and the left edge of cell 2 (phiR)
  auto use_thinc = [](const Cand& km, const Cand& k, const Cand& kp) {
    const double tT = fmin(fabs(km.mR - k.tL), fabs(km.tR - k.tL)) + fmin(fabs(k.tR - kp.mL), fabs(k.tR - kp.tL));
    const double tM = fmin(fabs(km.mR - k.mL), fabs(km.tR - k.mL)) + fmin(fabs(k.mR - kp.mL), fabs(k.mR - kp.tL));
    return tT < tM;
  };
  const bool t1 = use_thinc(c[0], c[1], c[2]);
  const bool t2 = use_thinc(c[1], c[2], c[3]);
  double betab[4] = {0.0, 0.0, 0.0, 0.0};
  if (gpL != 0.0) {
    double qb[3] = {0.0, 0.0, 0.0};
    betab[1] = phi_cand_vjp(B[1][1], B[1][2], B[1][3], [&]() { return beta_of(1); }, thinc, 1, t1, gpL, qb, lim);
    Bb[1][1] += qb[0];
    Bb[1][2] += qb[1];
    Bb[1][3] += qb[2];
  }
  if (gpR != 0.0) {
    double qb[3] = {0.0, 0.0, 0.0};
    betab[2] = phi_cand_vjp(B[1][2], B[1][3], B[1][4], [&]() { return beta_of(2); }, thinc, 0, t2, gpR, qb, lim);
    Bb[1][2] += qb[0];
    Bb[1][3] += qb[1];
    Bb[1][4] += qb[2];
  }
  if constexpr (DIM == 2) {
  if (!thinc) return;
#pragma unroll
  for (int s = 1; s <= 2; ++s) {
    if (betab[s] == 0.0) continue;
    const double dn = (B[2][s + 2] + 2.0 * B[1][s + 2] + B[0][s + 2]) - (B[2][s] + 2.0 * B[1][s] + B[0][s]);
    const double dt_ = (B[2][s + 2] + 2.0 * B[2][s + 1] + B[2][s]) - (B[0][s + 2] + 2.0 * B[0][s + 1] + B[0][s]);
    const double gn = dn / hn, gt = dt_ / ht;
    const double nrm = sqrt(gn * gn + gt * gt);
    if (nrm == 0.0) continue;  // beta = 2.51 there
    // beta = 2.5 |gn| / nrm + 0.01
    const double r = fabs(gn) / nrm;
    const double rb = 2.5 * betab[s];
    const double nrmb = -rb * r / nrm;
    const double gnb = rb / nrm * (gn > 0.0 ? 1.0 : (gn < 0.0 ? -1.0 : 0.0)) + nrmb * gn / nrm;
    const double gtb = nrmb * gt / nrm;
    const double dnb = gnb / hn, dtb = gtb / ht;
    Bb[2][s + 2] += dnb + dtb;
    Bb[1][s + 2] += 2.0 * dnb;
    Bb[0][s + 2] += dnb - dtb;
    Bb[2][s] += -dnb + dtb;
    Bb[1][s] += -2.0 * dnb;
    Bb[0][s] += -dnb - dtb;
    Bb[2][s + 1] += 2.0 * dtb;
    Bb[0][s + 1] += -2.0 * dtb;
  }
  }
}

// Adjoint of plastic (physics.cuh) on one cell: V[5] = (V11, V12, V21, V22,
// V33) before the plastic step, Vb[5] the adjoint of its output, replaced by
// the adjoint of its input; adds the adjoint of phi1 to phib and, where thb
// is not null, those of G_l (3 l) and sigma_y,l (3 l + 1) through the yield
// strain J_Y = sigma_y / (sqrt(6) G).  The output of the 2 x 2 block is
// V = X^-1 Y with X = I - h/2, Y = I + h/2, so dV = X^-1 dh (I + V) / 2.
__device__ __forceinline__ void plastic_vjp(const Phys& P, double phi1, double dt, const double (&V)[5],
                                            double (&Vb)[5], double& phib, double* thb) {
  // forward
  const Strain st = strain_of(V[0], V[1], V[2], V[3], V[4]);
  const double Js = sqrt(st.J2);
  double num = 0.0, den = 0.0, Jl[2];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const MatDev& m = P.m[l];
    const double ph = l == 0 ? phi1 : 1.0 - phi1;
    if (m.G == 0.0) Jl[l] = 0.0;
    else if (m.plastic == 1) Jl[l] = fmin(Js, m.JY);
    else if (m.plastic == 2) Jl[l] = Js > m.JY ? fmax(Js - dt * m.chi0, m.JY) : Js;
    else Jl[l] = Js;
    num += ph * m.iGm1 * Jl[l];
    den += ph * m.iGm1;
  }
  const double Jn = num / den;
  const double sc = Js > 0.0 ? Jn / Js : 0.0;
  const double h11 = sc * st.H11, h12 = sc * st.H12, h22 = sc * st.H22, h33 = sc * st.H33;
  const double x11 = 1.0 - 0.5 * h11, x12 = -0.5 * h12, x22 = 1.0 - 0.5 * h22;
  const double y11 = 1.0 + 0.5 * h11, y12 = 0.5 * h12, y22 = 1.0 + 0.5 * h22;
  const double id = 1.0 / (x11 * x22 - x12 * x12);
  const double i11 = x22 * id, i12 = -x12 * id, i22 = x11 * id;
  const double o11 = i11 * y11 + i12 * y12, o12 = i11 * y12 + i12 * y22;
  const double o21 = i12 * y11 + i22 * y12, o22 = i12 * y12 + i22 * y22;
  // reverse: hb = X^-1 Vb (I + V_out)^T / 2 (X^-1 symmetric)
  const double t00 = i11 * Vb[0] + i12 * Vb[2], t01 = i11 * Vb[1] + i12 * Vb[3];
  const double t10 = i12 * Vb[0] + i22 * Vb[2], t11 = i12 * Vb[1] + i22 * Vb[3];
  const double hb00 = 0.5 * (t00 * (1.0 + o11) + t01 * o12);
  const double hb01 = 0.5 * (t00 * o21 + t01 * (1.0 + o22));
  const double hb10 = 0.5 * (t10 * (1.0 + o11) + t11 * o12);
  const double hb11 = 0.5 * (t10 * o21 + t11 * (1.0 + o22));
  const double h11b = hb00, h22b = hb11, h12b = hb01 + hb10;
  const double d33 = 1.0 - 0.5 * h33;
  const double h33b = Vb[4] / (d33 * d33);  // V33 = (1 + h33/2) / (1 - h33/2)
  double H11b = sc * h11b, H12b = sc * h12b, H22b = sc * h22b, H33b = sc * h33b;
  const double scb = h11b * st.H11 + h12b * st.H12 + h22b * st.H22 + h33b * st.H33;
  double Jsb = 0.0, Jnb = 0.0;
  if (Js > 0.0) {
    Jnb = scb / Js;
    Jsb = -scb * sc / Js;
  }
  const double numb = Jnb / den, denb = -Jnb * Jn / den;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const MatDev& m = P.m[l];
    const double ph = l == 0 ? phi1 : 1.0 - phi1;
    const double sg = l == 0 ? 1.0 : -1.0;
    phib += sg * (numb * m.iGm1 * Jl[l] + denb * m.iGm1);
    const double Jlb = numb * ph * m.iGm1;
    double JYb = 0.0;
    if (m.G == 0.0) {
    } else if (m.plastic == 1) {  // min(Js, J_Y), equal values split
      if (m.JY < Js) JYb += Jlb;
      else if (Js < m.JY) Jsb += Jlb;
      else { Jsb += 0.5 * Jlb; JYb += 0.5 * Jlb; }
    } else if (m.plastic == 2 && Js > m.JY) {  // max(Js - dt chi0, J_Y)
      const double a = Js - dt * m.chi0;
      if (m.JY > a) JYb += Jlb;
      else if (a > m.JY) Jsb += Jlb;
      else { Jsb += 0.5 * Jlb; JYb += 0.5 * Jlb; }
    } else {
      Jsb += Jlb;
    }
    if (thb && JYb != 0.0 && m.plastic && m.G > 0.0) {
      thb[3 * l] += JYb * (-m.JY / m.G);
      thb[3 * l + 1] += JYb / (sqrt(6.0) * m.G);
    }
  }
  const double J2b = Js > 0.0 ? Jsb / (2.0 * Js) : 0.0;
  double Vin_b[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  strain_vjp(V[0], V[1], V[2], V[3], V[4], H11b, H12b, H22b, H33b, J2b, Vin_b[0], Vin_b[1], Vin_b[2], Vin_b[3],
             Vin_b[4]);
#pragma unroll
  for (int c = 0; c < 5; ++c) Vb[c] = Vin_b[c];
}

// Adjoint of sources (face.cuh: the plastic step, then, with RX, the RK4
// reaction step) on one cell: o is the conservative state before the source
// steps, ob the adjoint of the state after them (replaced by the adjoint of
// the state before); parameter adjoints are added to thb where not null
// (G_l at 3 l, sigma_y,l at 3 l + 1, Q_l at 3 l + 2).
template <int DIM, bool RX>
__device__ __forceinline__ void sources_vjp(const Phys& P, double dt, const double* o, double* ob, double* thb) {
  using L = Lay<DIM, RX>;
  double V[5] = {o[L::V11], 0.0, 0.0, o[L::V22], o[L::V33]};
  if constexpr (DIM == 2) {
    V[1] = o[L::V12];
    V[2] = o[L::V21];
  }
  double Vb[5] = {ob[L::V11], 0.0, 0.0, ob[L::V22], ob[L::V33]};
  if constexpr (DIM == 2) {
    Vb[1] = ob[L::V12];
    Vb[2] = ob[L::V21];
  }
  double phib = 0.0;
  if constexpr (RX) {
    // forward: V after the plastic step, then the reaction's frozen quantities
    double Vp[5] = {V[0], V[1], V[2], V[3], V[4]};
    plastic(P, o[L::PHI], dt, Vp[0], Vp[1], Vp[2], Vp[3], Vp[4], o[L::A1] / o[L::PHI],
            o[L::A2] / (1.0 - o[L::PHI]));
    const int y = P.y;
    const MatDev& m = P.m[y];
    const double phi1 = o[L::PHI], a1 = o[L::A1], a2 = o[L::A2];
    const double ary = y == 0 ? a1 : a2;
    const double phy = y == 0 ? phi1 : 1.0 - phi1;
    const double rr = a1 + a2;
    const double mx = o[L::MX];
    double my = 0.0;
    if constexpr (DIM == 2) my = o[L::MY];
    const double KE = 0.5 * (mx * mx + my * my) / rr;
    const Strain st = strain_of(Vp[0], Vp[1], Vp[2], Vp[3], Vp[4]);
    const double xi = xi_of(P, phi1);
    const double ref0 = ref_energy(P, phi1, a1, a2, 0.0, st.J2);
    const double p0 = (o[L::E] - KE - ref0) / xi;
    const double cTy = m.iGm1 / m.cv;
    const double Tfac = m.iGm1 / ((ary / phy) * m.cv);
    const double Qx = m.Q / xi;
    const double L0 = o[L::AL];
    const bool sq = m.law == 1;  // k sqrt(lam) law with the pressure switch
    auto f = [&](double Lm) {
      if (sq) return (p0 - Qx * Lm) > m.pign && Lm > 0.0 ? -m.A * sqrt(ary * Lm) : 0.0;
      const double Tk = (p0 - Qx * Lm) * Tfac;
      return Tk > 0.0 ? -m.A * Lm * exp(-m.Tact / Tk) : 0.0;
    };
    const double k1 = f(L0);
    const double L2 = L0 + 0.5 * dt * k1;
    const double k2 = f(L2);
    const double L3 = L0 + 0.5 * dt * k2;
    const double k3 = f(L3);
    const double L4 = L0 + dt * k3;
    // reverse of the RK4 combination (and of the clamp at lam = 0) and stages
    const bool clamped = sq && !(L0 + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + f(L4)) > 0.0);
    const double outb = clamped ? 0.0 : ob[L::AL];
    double L0b = outb;
    double kb[4] = {dt / 6.0 * outb, dt / 3.0 * outb, dt / 3.0 * outb, dt / 6.0 * outb};
    double p0b = 0.0, Qxb = 0.0, Tfacb = 0.0, aryb_r = 0.0;
    auto stage_b = [&](double Lm, double kbar) -> double {  // returns the adjoint of Lm
      if (sq) {  // the switch is a step: no derivative through the pressure
        if (!((p0 - Qx * Lm) > m.pign && Lm > 0.0) || kbar == 0.0) return 0.0;
        const double r = sqrt(ary * Lm);
        aryb_r += kbar * (-m.A * 0.5 * Lm / r);
        return kbar * (-m.A * 0.5 * ary / r);
      }
      const double Tk = (p0 - Qx * Lm) * Tfac;
      if (!(Tk > 0.0) || kbar == 0.0) return 0.0;
      const double e = exp(-m.Tact / Tk);
      const double fTk = -m.A * Lm * e * m.Tact / (Tk * Tk);
      const double Tkb = kbar * fTk;
      p0b += Tkb * Tfac;
      Qxb -= Tkb * Lm * Tfac;
      Tfacb += Tkb * (p0 - Qx * Lm);
      return kbar * (-m.A * e) + Tkb * (-Qx * Tfac);
    };
    const double L4b = stage_b(L4, kb[3]);
    L0b += L4b;
    kb[2] += dt * L4b;
    const double L3b = stage_b(L3, kb[2]);
    L0b += L3b;
    kb[1] += 0.5 * dt * L3b;
    const double L2b = stage_b(L2, kb[1]);
    L0b += L2b;
    kb[0] += 0.5 * dt * L2b;
    L0b += stage_b(L0, kb[0]);
    ob[L::AL] = L0b;
    // p0 = (E - KE - ref0) / xi, Qx = Q / xi, Tfac = cTy phy / ary
    double xib = -p0b * p0 / xi - Qxb * Qx / xi;
    ob[L::E] += p0b / xi;
    const double KEb = -p0b / xi, ref0b = -p0b / xi;
    double Qb = Qxb / xi;
    const double phyb = Tfacb * cTy / ary;
    double aryb = -Tfacb * Tfac / ary + aryb_r;
    double a1b = 0.0, a2b = 0.0;
    phib += y == 0 ? phyb : -phyb;
    // KE = (mx^2 + my^2) / (2 rr), rr = a1 + a2
    ob[L::MX] += KEb * mx / rr;
    if constexpr (DIM == 2) ob[L::MY] += KEb * my / rr;
    const double rrb = -KEb * KE / rr;
    a1b += rrb;
    a2b += rrb;
    // ref0 = sum_l phi_l (kap_l + gG_l J2) + a1 einf_1 + a2 einf_2 - Q_y a_y
    const MatDev& m0 = P.m[0];
    const MatDev& m1 = P.m[1];
    phib += ref0b * ((m0.kap + m0.gG * st.J2) - (m1.kap + m1.gG * st.J2));
    const double J2b = ref0b * (phi1 * m0.gG + (1.0 - phi1) * m1.gG);
    a1b += ref0b * m0.einf;
    a2b += ref0b * m1.einf;
    aryb -= ref0b * m.Q;
    Qb -= ref0b * ary;
    phib += xib * (m0.iGm1 - m1.iGm1);
    if (y == 0) a1b += aryb;
    else a2b += aryb;
    ob[L::A1] += a1b;
    ob[L::A2] += a2b;
    if (thb) {
      thb[3 * y + 2] += Qb;
      thb[0] += ref0b * phi1 * st.J2 * m0.gi;
      thb[3] += ref0b * (1.0 - phi1) * st.J2 * m1.gi;
    }
    // the reaction reads the stretch after the plastic step through J2
    double Vpb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    strain_vjp(Vp[0], Vp[1], Vp[2], Vp[3], Vp[4], 0.0, 0.0, 0.0, 0.0, J2b, Vpb[0], Vpb[1], Vpb[2], Vpb[3],
               Vpb[4]);
#pragma unroll
    for (int c = 0; c < 5; ++c) Vb[c] += Vpb[c];
  }
  plastic_vjp(P, o[L::PHI], dt, V, Vb, phib, thb);
  ob[L::PHI] += phib;
  ob[L::V11] = Vb[0];
  ob[L::V22] = Vb[3];
  ob[L::V33] = Vb[4];
  if constexpr (DIM == 2) {
    ob[L::V12] = Vb[1];
    ob[L::V21] = Vb[2];
  }
}

}  // namespace dis
