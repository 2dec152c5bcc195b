// riemann_vjp.cuh - hand-written reverse of the face Riemann problem
// (riemann_outputs / hllc of face.cuh and physics.cuh), float64.
//
// Given the adjoint of the face outputs (NF fluxes + the face-state extras),
// accumulate the adjoints of the two face states (FState fields, c_L still
// squared as face_state returns it).  The forward pass is recomputed here in
// the same order, so every branch (wave-speed min / max, shear coupling,
// region at x/t = 0, zero shear-wave width) is the one the forward step took;
// ties and non-differentiable points follow the conventions of dual.cuh
// (min / max of equal values split the derivative, sqrt has derivative 0 at
// 0).  A test compares this reverse with the dual-number evaluation of the
// same forward code.
#pragma once
#include "face.cuh"

namespace dis {

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
  const double num = L.snn - R.snn + mL * L.un - mR * R.un, den = mL - mR;
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

}  // namespace dis
