// face.cuh - the per-cell and per-face functions of the float64 step, written
// once and templated on the scalar type T: with T = double they are the
// forward step; with T = Dual (dual.cuh) the same code returns one
// directional derivative, which the adjoint kernels contract with the
// incoming adjoint to form vector-Jacobian products.  Branches (limiter,
// BVD choice, Riemann region, fallback, radial return) compare values only,
// so a Dual evaluation differentiates the branch the forward step took.
#pragma once
#include "dual.cuh"
#include "physics.cuh"

namespace dis {

// Conservative -> primitive state of one cell (Section 2.2 mixture rules and
// the pressure function of Appendix B, solved for p).
template <int DIM, bool RX, class T>
__device__ __forceinline__ PrimT<T> prim_of(const PhysT<T>& P, const T* q) {
  using L = Lay<DIM, RX>;
  PrimT<T> w;
  const T phi = q[L::PHI], a1 = q[L::A1], a2 = q[L::A2];
  const T rho = a1 + a2;
  const T mx = q[L::MX];
  T my = 0.0;
  if constexpr (DIM == 2) my = q[L::MY];
  const T E = q[L::E];
  w.phi = phi;
  w.r1 = a1 / phi;
  w.r2 = a2 / (1.0 - phi);
  w.u = mx / rho;
  w.v = my / rho;
  w.V11 = q[L::V11];
  w.V12 = 0.0;
  w.V21 = 0.0;
  if constexpr (DIM == 2) {
    w.V12 = q[L::V12];
    w.V21 = q[L::V21];
  }
  w.V22 = q[L::V22];
  w.V33 = q[L::V33];
  T arl = 0.0;
  w.lam = 0.0;
  if constexpr (RX) {
    arl = q[L::AL];
    w.lam = arl / (P.y == 0 ? a1 : a2);
  }
  const StrainT<T> s = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const T KE = 0.5 * (mx * w.u + my * w.v);
  if (RX && P.m[P.y].two) {
    T sh;
    w.p = mixture_pressure(P, phi, a1, a2, arl, E - KE, s.J2, sh);
  } else {
    w.p = (E - KE - ref_energy(P, phi, a1, a2, arl, s.J2)) / xi_of(P, phi);
  }
  return w;
}

// Primitive -> conservative state of one cell (mixture rules; the energy from
// the Mie-Grueneisen form), in place on the NF slots.
template <int DIM, bool RX, class T>
__device__ __forceinline__ void cons_of(const PhysT<T>& P0, T* v) {
  using L = Lay<DIM, RX>;
  const PhysT<T> P = at_state(P0, RX ? v[Lay<DIM, RX>::AL > 0 ? Lay<DIM, RX>::AL : 0] : T(0.0), v[L::E]);
  const T phi = v[L::PHI], r1 = v[L::A1], r2 = v[L::A2];
  const T u = v[L::MX], p = v[L::E];
  T vv = 0.0, v12 = 0.0, v21 = 0.0, arl = 0.0;
  const T a1 = phi * r1, a2 = (1.0 - phi) * r2, rho = a1 + a2;
  if constexpr (DIM == 2) {
    vv = v[L::MY];
    v12 = v[L::V12];
    v21 = v[L::V21];
  }
  if constexpr (RX) arl = (P.y == 0 ? a1 : a2) * v[L::AL];
  const StrainT<T> s = strain_of(v[L::V11], v12, v21, v[L::V22], v[L::V33]);
  v[L::A1] = a1;
  v[L::A2] = a2;
  v[L::MX] = rho * u;
  if constexpr (DIM == 2) v[L::MY] = rho * vv;
  v[L::E] = xi_of(P, phi) * p + ref_energy(P, phi, a1, a2, arl, s.J2) + 0.5 * rho * (u * u + vv * vv);
  if constexpr (RX) v[L::AL] = arl;
}

// Primitive components in the slot order of Lay (phi, rho1, rho2, u, [v], p,
// V11, [V12, V21], V22, V33, [lam]).
template <int DIM, bool RX, class T>
__device__ __forceinline__ T& prim_slot(PrimT<T>& w, int k) {
  using L = Lay<DIM, RX>;
  if (k == L::PHI) return w.phi;
  if (k == L::A1) return w.r1;
  if (k == L::A2) return w.r2;
  if (k == L::MX) return w.u;
  if (DIM == 2 && k == L::MY) return w.v;
  if (k == L::E) return w.p;
  if (k == L::V11) return w.V11;
  if (DIM == 2 && k == L::V12) return w.V12;
  if (DIM == 2 && k == L::V21) return w.V21;
  if (k == L::V22) return w.V22;
  if (k == L::V33) return w.V33;
  return w.lam;
}

// phi edge values at one face (Appendix A): MUSCL and THINC candidates of the
// four cells a-1 .. a+2 and the BVD choice for cells a and a+1.  B[1][c] is
// phi at sweep position a-2+c; rows B[0], B[2] are the neighbouring lines
// (used only by the 2D Youngs normal, (1,2,1)-weighted central differences).
template <int DIM, class T>
__device__ __forceinline__ void face_phi(const T (&B)[3][6], bool thinc, double hn, double ht,
                                         T& phiL, T& phiR, int lim = 0) {
  CandT<T> c[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    auto beta_of = [&]() -> T {
      T beta = 2.51;  // beta0 |n_d| + 0.01 with |n_d| = 1 in 1D
      if (DIM == 2 && thinc) {
        const T dn = (B[2][s + 2] + 2.0 * B[1][s + 2] + B[0][s + 2]) - (B[2][s] + 2.0 * B[1][s] + B[0][s]);
        const T dt_ = (B[2][s + 2] + 2.0 * B[2][s + 1] + B[2][s]) - (B[0][s + 2] + 2.0 * B[0][s + 1] + B[0][s]);
        const T gn = dn / hn, gt = dt_ / ht;
        const T nrm = sqrt(gn * gn + gt * gt);
        beta = 2.5 * (nrm == 0.0 ? T(1.0) : fabs(gn) / nrm) + 0.01;
      }
      return beta;
    };
    c[s] = phi_cand_lazy(B[1][s], B[1][s + 1], B[1][s + 2], beta_of, thinc, lim);
  }
  T Lt, Rt;
  bvd(c[0], c[1], c[2], Lt, Rt);
  phiL = Rt;  // right edge of cell a
  bvd(c[1], c[2], c[3], Lt, Rt);
  phiR = Lt;  // left edge of cell a+1
}

// Left and right edge values of phi in the middle cell of a 3 x 5 stencil
// (columns: cells i-2 .. i+2 along the axis; rows: tangential neighbours, used
// only by the 2D Youngs normal): MUSCL and THINC candidates of cells i-1, i,
// i+1 and the BVD choice for cell i (Appendix A), as in face_phi.
template <int DIM, class T>
__device__ __forceinline__ void cell_phi_edges(const T (&B)[3][5], bool thinc, double hn, double ht,
                                               T& eL, T& eR, int lim = 0) {
  CandT<T> c[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    auto beta_of = [&]() -> T {
      T beta = 2.51;
      if (DIM == 2 && thinc) {
        const T dn = (B[2][s + 2] + 2.0 * B[1][s + 2] + B[0][s + 2]) - (B[2][s] + 2.0 * B[1][s] + B[0][s]);
        const T dt_ = (B[2][s + 2] + 2.0 * B[2][s + 1] + B[2][s]) - (B[0][s + 2] + 2.0 * B[0][s + 1] + B[0][s]);
        const T gn = dn / hn, gt = dt_ / ht;
        const T nrm = sqrt(gn * gn + gt * gt);
        beta = 2.5 * (nrm == 0.0 ? T(1.0) : fabs(gn) / nrm) + 0.01;
      }
      return beta;
    };
    c[s] = phi_cand_lazy(B[1][s], B[1][s + 1], B[1][s + 2], beta_of, thinc, lim);
  }
  bvd(c[0], c[1], c[2], eL, eR);
}

// MUSCL face values of one primitive from cells a-1 .. a+2 (limited slopes:
// lim 0 minmod, 1 van Leer).
template <class T>
__device__ __forceinline__ void muscl_pair(T w0, T w1, T w2, T w3, T& l, T& r, int lim = 0) {
  const T s1 = limited(w1 - w0, w2 - w1, lim);
  const T s2 = limited(w2 - w1, w3 - w2, lim);
  l = w1 + 0.5 * s1;
  r = w2 - 0.5 * s2;
}

// Number of per-face outputs: NF conservative fluxes plus the face-state
// extras used by the non-conservative terms (u_n and the normal row of V).
template <int DIM, bool RX>
__host__ __device__ constexpr int n_face_out() {
  return Lay<DIM, RX>::NF + Lay<DIM, RX>::NX_EXTRA;
}

// Riemann problem of one face from the two face states (face_state output,
// c_L still squared; the caller has applied the non-hyperbolic fallback) and
// the outputs of the face: fluxes and extras.
template <int DIM, bool RX, int DIR, class T>
__device__ __forceinline__ void face_outputs(const FaceOutT<T>& o, T* F);

template <int DIM, bool RX, int DIR, class T>
__device__ __forceinline__ void riemann_outputs(FStateT<T> sl, FStateT<T> sr, T* F) {
  sl.cL = sqrt(sl.cL);
  sr.cL = sqrt(sr.cL);
  face_outputs<DIM, RX, DIR, T>(hllc<DIR>(sl, sr), F);
}

// Physical flux of one state along DIR as a face output (the flux of a face
// whose two sides are that state; single-stage MUSCL-Hancock predictor).
template <int DIR, class T>
__device__ __forceinline__ FaceOutT<T> physical_faceout(const FStateT<T>& K) {
  FaceOutT<T> o;
  o.Far1 = K.ar1 * K.un;
  o.Far2 = K.ar2 * K.un;
  o.Farl = K.arl * K.un;
  o.Fmn = K.rho * K.un * K.un - K.snn;
  o.Fmt = K.rho * K.ut * K.un - K.snt;
  o.FE = K.rhoE * K.un - (K.un * K.snn + K.ut * K.snt);
  o.phi = K.phi;
  o.un = K.un;
  o.ut = K.ut;
  o.V11 = K.V11; o.V12 = K.V12; o.V21 = K.V21; o.V22 = K.V22; o.V33 = K.V33;
  return o;
}

// Conservative fluxes (NF slots) and face extras (u_n, normal row of V) of a
// face output.
template <int DIM, bool RX, int DIR, class T>
__device__ __forceinline__ void face_outputs(const FaceOutT<T>& o, T* F) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const T fu = DIR == 0 ? o.un : o.ut;
  const T fv = DIR == 0 ? o.ut : o.un;
  F[L::PHI] = o.phi * o.un;
  F[L::A1] = o.Far1;
  F[L::A2] = o.Far2;
  F[L::MX] = DIR == 0 ? o.Fmn : o.Fmt;
  if constexpr (DIM == 2) F[L::MY] = DIR == 0 ? o.Fmt : o.Fmn;
  F[L::E] = o.FE;
  if constexpr (RX) F[L::AL] = o.Farl;
  // stretch fluxes V_ij u_d - V_dj u_i at the face state
  if constexpr (DIR == 0) {
    F[L::V11] = 0.0;
    if constexpr (DIM == 2) {
      F[L::V12] = 0.0;
      F[L::V21] = o.V21 * fu - o.V11 * fv;
      F[L::V22] = o.V22 * fu - o.V12 * fv;
    } else {
      F[L::V22] = o.V22 * fu;
    }
    F[L::V33] = o.V33 * fu;
    F[NF + 0] = o.un;
    F[NF + 1] = o.V11;
    if constexpr (DIM == 2) F[NF + 2] = o.V12;
  } else if constexpr (DIM == 2) {
    F[L::V11] = o.V11 * fv - o.V21 * fu;
    F[L::V12] = o.V12 * fv - o.V22 * fu;
    F[L::V21] = 0.0;
    F[L::V22] = 0.0;
    F[L::V33] = o.V33 * fv;
    F[NF + 0] = o.un;
    F[NF + 1] = o.V21;
    F[NF + 2] = o.V22;
  }
}

// Plastic (Section 3.2) and reactive (Section 3.3) source steps of one cell,
// applied to the conservative state o after the last Runge-Kutta stage.
template <int DIM, bool RX, class T>
__device__ __forceinline__ void sources(const PhysT<T>& P, double dt, T* o) {
  using L = Lay<DIM, RX>;
  T v12 = 0.0, v21 = 0.0;
  if constexpr (DIM == 2) {
    v12 = o[L::V12];
    v21 = o[L::V21];
  }
  // (a two-closure reactive mixture weighs its material by 1 / Gamma_y at the
  // state's own share, from the pressure of the conservative state)
  PhysT<T> Pp = P;
  if constexpr (RX) {
    if (P.m[P.y].two) {
      const T rr = o[L::A1] + o[L::A2];
      T my_ = 0.0;
      if constexpr (DIM == 2) my_ = o[L::MY];
      const T KE0 = 0.5 * (o[L::MX] * o[L::MX] + my_ * my_) / rr;
      const StrainT<T> s0 = strain_of(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
      T sh;
      const T p0 = mixture_pressure(P, o[L::PHI], o[L::A1], o[L::A2], o[L::AL], o[L::E] - KE0, s0.J2, sh);
      Pp = at_state(P, o[L::AL] / (P.y == 0 ? o[L::A1] : o[L::A2]), p0);
    }
  }
  // a Johnson-Cook material: its temperature at the state entering the step
  // (Debye form of the thermal energy, Section 2.2: T0 (r/rho0)^Gamma +
  // (p - p_ref) / (r Gamma C_V) at the mixture pressure) and its plastic strain
  JcIn<T> jc{T(0.0), T(0.0)};
  bool is_jc = false;
  if constexpr (RX) {
    const MatT<T>& m = P.m[P.y];
    if (m.plastic == 3) {
      is_jc = true;
      const T rr = o[L::A1] + o[L::A2];
      T my_ = 0.0;
      if constexpr (DIM == 2) my_ = o[L::MY];
      const T KE0 = 0.5 * (o[L::MX] * o[L::MX] + my_ * my_) / rr;
      const StrainT<T> s0 = strain_of(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
      const T p0 = (o[L::E] - KE0 - ref_energy(P, o[L::PHI], o[L::A1], o[L::A2], o[L::AL], s0.J2)) /
                   xi_of(P, o[L::PHI]);
      const T ary = P.y == 0 ? o[L::A1] : o[L::A2];
      const T ry = P.y == 0 ? o[L::A1] / o[L::PHI] : o[L::A2] / (1.0 - o[L::PHI]);
      const RefT<T> c = ref_curves(m, ry, s0.J2);
      jc.temp = m.jcT0 * powr(ry / m.rho0, T(m.gamma - 1.0)) + (p0 - c.p) / (ry * (m.gamma - 1.0) * m.cv);
      jc.eps = o[L::AL] / ary;
    }
  }
  T deps = 0.0;
  plastic(Pp, o[L::PHI], T(dt), o[L::V11], v12, v21, o[L::V22], o[L::V33], o[L::A1] / o[L::PHI],
          o[L::A2] / (1.0 - o[L::PHI]), is_jc ? &jc : nullptr, &deps);
  if constexpr (DIM == 2) {
    o[L::V12] = v12;
    o[L::V21] = v21;
  }
  if constexpr (RX) {
    if (is_jc) {  // the history row's source over the step: rho_y phi_y (J* - J*_y)
      o[L::AL] += (P.y == 0 ? o[L::A1] : o[L::A2]) * deps;
      return;
    }
    const int y = P.y;
    const MatT<T>& m = P.m[y];
    const T phi1 = o[L::PHI];
    const T ary = y == 0 ? o[L::A1] : o[L::A2];
    const T phy = y == 0 ? phi1 : 1.0 - phi1;
    const T rr = o[L::A1] + o[L::A2];
    const T mx = o[L::MX];
    T my = 0.0;
    if constexpr (DIM == 2) my = o[L::MY];
    const T KE = 0.5 * (mx * mx + my * my) / rr;
    const StrainT<T> s = strain_of(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
    const T xi = xi_of(P, phi1);
    const T p0 = (o[L::E] - KE - ref_energy(P, phi1, o[L::A1], o[L::A2], T(0.0), s.J2)) / xi;
    const T Tfac = m.iGm1 / ((ary / phy) * m.cv);  // T = p / (rho_y Gamma c_V)
    const T Qx = m.Q / xi;
    // the rate of phi_y rho_y lam at Lm = phi_y rho_y lam, other fields frozen;
    // two closures: the pressure of each stage from the root finder
    auto f = [&](T Lm) -> T {
      T pk;
      if (m.two) {
        T sh;
        pk = mixture_pressure(P, phi1, o[L::A1], o[L::A2], Lm, o[L::E] - KE, s.J2, sh);
      } else {
        pk = p0 - Qx * Lm;
      }
      if (m.law == 1)  // -k sqrt(lam) rho_y phi_y where p > p_ign
        return pk > m.pign && Lm > 0.0 ? -m.A * sqrt(ary * Lm) : T(0.0);
      const T Tk = m.two ? mix_temperature(m, Lm / ary, pk, ary / phy) : pk * Tfac;
      return Tk > 0.0 ? -m.A * Lm * exp(-m.Tact / Tk) : T(0.0);
    };
    const T L0 = o[L::AL];
    const T k1 = f(L0);
    const T k2 = f(L0 + 0.5 * dt * k1);
    const T k3 = f(L0 + 0.5 * dt * k2);
    const T k4 = f(L0 + dt * k3);
    const T L1 = L0 + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    o[L::AL] = m.law == 1 && !(L1 > 0.0) ? T(0.0) : L1;
  }
}

}  // namespace dis
