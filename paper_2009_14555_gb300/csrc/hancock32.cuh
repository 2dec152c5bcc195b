// hancock32.cuh - the single-stage MUSCL-Hancock step in the FP32-bulk
// layout: one fused kernel per time step.
//
// The single-stage alternative to SSP-RK3 (van Leer's predictor-corrector
// MUSCL-Hancock form; Toro, "Riemann Solvers and Numerical Methods for Fluid
// Dynamics", Sec. 14.4) with the reconstruction, Riemann solver and
// non-conservative terms of Section 3.1.  A CTA owns a tile of TX x TY cells:
//   1. primitives of the tile and a 3-cell halo into shared memory
//      (fill_tile of the stage kernel);
//   2. predictor, for every cell of the tile and of the one-cell ring beside
//      its sides whose edge state a face of the tile takes: the left and
//      right edge states of each axis (MUSCL on the primitives,
//      MUSCL-BVD-THINC on phi1; the cell-centre state where an edge state is
//      not hyperbolic), D_c of the cell from their physical fluxes (the
//      non-conservative terms with the cell-centre coefficients), and the
//      edge states the faces take, as conservative states moved by
//      -dt/2 D_c, into shared memory;
//   3. corrector: the Riemann problem of every face between its two evolved
//      edge states (the cell-centre state at t^n where an evolved state is
//      not hyperbolic), into the face slots of the stage kernel;
//   4. the update of the stage kernel with a = 0, b = 1: q^{n+1} = q^n - dt D,
//      then the plastic and reactive steps and the CFL rate of the new state.
// Energy: the predictor advances e_s = rho E - kappa(phi1) with the e_s form
// of the operator (fused32.cuh); a cell's own edge states have no star
// region, so their kappa-flux correction D vanishes.
// The step reads q^n (with its halo) and writes the other buffer of a pair;
// the two buffers exchange roles from step to step.  Planar geometry.
#pragma once
#include "fused32.cuh"

namespace dis {

// Shared memory: the stage kernel's primitives and face records, then the
// evolved edge states of both sides of every face (2 NF values per face).
template <int DIM, bool RX, int TX, int TY>
constexpr size_t hancock32_smem() {
  using TL = TileLay<DIM, RX, TX, TY>;
  return sizeof(float) * ((size_t)TL::END + (size_t)2 * Lay<DIM, RX>::NF * TL::NFA);
}

// Physical flux of one state as a face output (no star region: D = 0).
__device__ __forceinline__ FaceOutF phys_out_f(const FStateF& K) {
  FaceOutF o;
  o.Far1 = K.ar1 * K.un;
  o.Far2 = K.ar2 * K.un;
  o.Farl = K.arl * K.un;
  o.Fmn = K.rho * K.un * K.un - K.snn;
  o.Fmt = K.rho * K.ut * K.un - K.snt;
  o.FE = K.rhoE * K.un - (K.un * K.snn + K.ut * K.snt);
  o.X = K.un;
  o.D = 0.f;
  o.phi = K.phi;
  o.un = K.un;
  o.ut = K.ut;
  o.V11 = K.V11; o.V12 = K.V12; o.V21 = K.V21; o.V22 = K.V22; o.V33 = K.V33;
  return o;
}

// Face state along DIR of a conservative state v (NF values; phi1 as one
// float, slot E = e_s): primitive recovery and face state share one strain
// evaluation, and the soft energy is v's own.
template <int DIM, bool RX, int DIR, bool GEN>
__device__ __forceinline__ FStateF face_state_cons_f(const PhysF& F, const float* v) {
  using L = Lay<DIM, RX>;
  FStateF s;
  const float phi = v[L::PHI];
  const float a1 = v[L::A1], a2 = v[L::A2];
  const float rho = a1 + a2;
  const float r1 = a1 / phi, r2 = a2 / (1.f - phi);
  const float irho = 1.f / rho;
  const float mx = v[L::MX];
  float my = 0.f, V12 = 0.f, V21 = 0.f;
  if constexpr (DIM == 2) {
    my = v[L::MY];
    V12 = v[L::V12];
    V21 = v[L::V21];
  }
  const float u = mx * irho, w = my * irho;
  const float V11 = v[L::V11], V22 = v[L::V22], V33 = v[L::V33];
  float arl = 0.f;
  if constexpr (RX) arl = v[L::AL];
  const StrainF st = strain_f(V11, V12, V21, V22, V33);
  const float KE = 0.5f * (mx * u + my * w);
  const float p = (v[L::E] - (KE + soft_ref_f<GEN>(F, phi, a1, a2, arl, st.J2, r1, r2))) / xi_f(F, phi);
  const float Gm = Gmix_f<GEN>(F, phi, r1, r2);
  s.phi = phi;
  s.ar1 = a1;
  s.ar2 = a2;
  s.rho = rho;
  s.arl = arl;
  s.rhoE = v[L::E];
  s.Gm = Gm;
  if (DIR == 0) {
    s.un = u;
    s.ut = w;
    s.snn = -p + 2.f * Gm * st.H11;
  } else {
    s.un = w;
    s.ut = u;
    s.snn = -p + 2.f * Gm * st.H22;
  }
  s.snt = 2.f * Gm * st.H12;
  s.cL = cL2_f<GEN>(F, phi, rho, p, st.J2, r1, r2);
  s.V11 = V11; s.V12 = V12; s.V21 = V21; s.V22 = V22; s.V33 = V33;
  return s;
}

// Left (lo) and right (hi) edge states along DIR of the SMEM cell kc with
// primitives wc: MUSCL on the primitives, MUSCL-BVD-THINC on phi1 (the
// values the stage kernel's faces take on either side of the cell).
template <int DIM, bool RX, int DIR, int LIM>
__device__ __forceinline__ void cell_edges_f(const PhysF& P, const float* __restrict__ Wsm, int HX, int plane,
                                             int kc, float dxn, float dxt, const PrimF& wc, PrimF& lo,
                                             PrimF& hi) {
  using L = Lay<DIM, RX>;
  const int sx = DIR == 0 ? 1 : HX, sy = DIR == 0 ? HX : 1;
  const float* Wphi = Wsm + PR * plane;
  float ph[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) ph[s] = Wphi[kc + (s - 2) * sx];
  auto cand = [&](int s) {
    auto beta_of = [&]() -> float { return thinc_beta_f<DIM>(P, Wphi, kc + (s - 1) * sx, sx, sy, dxn, dxt); };
    return phi_cand_f<LIM>(ph[s], ph[s + 1], ph[s + 2], beta_of, P.thinc != 0, P.limiter);
  };
  // a cell that is not mixed keeps its MUSCL values (its THINC candidate is
  // the same), so the BVD choice is made only in a mixed cell
  const CandF c1 = cand(1);
  lo.phi = c1.mL;
  hi.phi = c1.mR;
  if (c1.mixed) bvd_f(cand(0), c1, cand(2), lo.phi, hi.phi);
  PrimF wm, wp;
  load_prim_sm<DIM, RX>(Wsm, kc - sx, wm);
  load_prim_sm<DIM, RX>(Wsm, kc + sx, wp);
#define DIS_EDGE(fld)                                                                \
  {                                                                                  \
    const float s_ = limited_f<LIM>(wc.fld - wm.fld, wp.fld - wc.fld, P.limiter);    \
    lo.fld = wc.fld - 0.5f * s_;                                                     \
    hi.fld = wc.fld + 0.5f * s_;                                                     \
  }
  DIS_EDGE(r1) DIS_EDGE(r2) DIS_EDGE(u) DIS_EDGE(p) DIS_EDGE(V11) DIS_EDGE(V22) DIS_EDGE(V33)
  if constexpr (DIM == 2) { DIS_EDGE(v) DIS_EDGE(V12) DIS_EDGE(V21) }
  else { lo.v = hi.v = 0.f; lo.V12 = hi.V12 = lo.V21 = hi.V21 = 0.f; }
  if constexpr (RX) { DIS_EDGE(lam) } else { lo.lam = hi.lam = 0.f; }
#undef DIS_EDGE
}

// D_c contributions of the edge pair (lo, hi) of one axis: flux differences
// of their physical fluxes (phi slot: phi u_n; E slot: the soft energy flux),
// div u, the stretch-row differences b, and the soft part of the e_s
// divergence.
template <int DIM, bool RX, int DIR>
__device__ __forceinline__ void own_flux_diff(const FStateF& lo, const FStateF& hi, float ih, float k2f,
                                              float* D, float& divu, float& bx, float& by, float& small) {
  using L = Lay<DIM, RX>;
  using R = Rec<DIM, RX, DIR>;
  float a[FA + 4], b[FA + 4];
  face_slots_f<DIM, RX, DIR>(phys_out_f(lo), [&](int s, float v) { a[s] = v; });
  face_slots_f<DIM, RX, DIR>(phys_out_f(hi), [&](int s, float v) { b[s] = v; });
#pragma unroll
  for (int c = 0; c < L::NF; ++c)
    if (!R::zero(c)) D[c] += (b[R::pos(c)] - a[R::pos(c)]) * ih;
  const float du = b[R::UF] - a[R::UF];
  divu += du * ih;
  bx += (b[R::VA] - a[R::VA]) * ih;
  if constexpr (DIM == 2) by += (b[R::VB] - a[R::VB]) * ih;
  small += ((b[R::pos(L::E)] - a[R::pos(L::E)]) + k2f * du) * ih;
}

// The conservative state (phi1, partial densities, momentum, e_s, V, the
// reactant slot) of a face state along DIR into slots base + c * stride.
template <int DIM, bool RX, int DIR>
__device__ __forceinline__ void put_cons(const FStateF& s, float* base, int stride) {
  using L = Lay<DIM, RX>;
  base[L::PHI * stride] = s.phi;
  base[L::A1 * stride] = s.ar1;
  base[L::A2 * stride] = s.ar2;
  base[L::MX * stride] = s.rho * (DIR == 0 ? s.un : s.ut);
  if constexpr (DIM == 2) base[L::MY * stride] = s.rho * (DIR == 0 ? s.ut : s.un);
  base[L::E * stride] = s.rhoE;
  base[L::V11 * stride] = s.V11;
  if constexpr (DIM == 2) {
    base[L::V12 * stride] = s.V12;
    base[L::V21 * stride] = s.V21;
  }
  base[L::V22 * stride] = s.V22;
  base[L::V33 * stride] = s.V33;
  if constexpr (RX) base[L::AL * stride] = s.arl;
}

// Edge states of one axis of the SMEM cell kc, with the cell-centre state
// where an edge state is not hyperbolic.
template <int DIM, bool RX, int DIR, int LIM, bool GEN>
__device__ __forceinline__ void edge_states(const PhysF& F, const float* __restrict__ Wsm, int HX, int plane,
                                            int kc, float dxn, float dxt, const PrimF& wc, FStateF& sl,
                                            FStateF& sh) {
  PrimF lo, hi;
  cell_edges_f<DIM, RX, DIR, LIM>(F, Wsm, HX, plane, kc, dxn, dxt, wc, lo, hi);
  sl = face_state_f<DIR, GEN>(F, lo);
  sh = face_state_f<DIR, GEN>(F, hi);
  if (!(sl.cL > 0.f) || !(sh.cL > 0.f)) {
    const FStateF sc = face_state_f<DIR, GEN>(F, wc);
    if (!(sl.cL > 0.f)) sl = sc;
    if (!(sh.cL > 0.f)) sh = sc;
  }
}

// Phase 2: the predictor.  Work items: the TX x TY tile cells, then the
// x ring (columns -1 and TX of the tile's rows), then the y ring (rows -1
// and TY of its columns); a cell's edge states go to the faces of the tile
// that take them (side 1 of the face to its left / below, side 0 of the face
// to its right / above), evolved by -h D_c, h = dt / 2.
template <int DIM, bool RX, int TX, int TY, int NT, int LIM, bool GEN>
__device__ __forceinline__ void predict_tile(const PhysF& F, const StepArgs32& A, const int4 t,
                                             float* __restrict__ sm, const TileConst& K) {
  using L = Lay<DIM, RX>;
  using TL = TileLay<DIM, RX, TX, TY>;
  constexpr int NF = L::NF;
  constexpr int HX = TL::HX, plane = TL::PLANE;
  constexpr int NFX = TL::NFX, NFA = TL::NFA;
  constexpr int NI = TX * TY, NRX = DIM == 2 ? 2 * TY : 2, NRY = DIM == 2 ? 2 * TX : 0;
  const float* Wsm = sm;
  float* E = sm + TL::END;
  const PatchDev pd = A.pd[t.x];
  const int i0 = t.y, j0 = t.z;
  const float dxf = (float)pd.dx, dyf = (float)pd.dy;
  const float k2f = F.m[1].kap, dkf = F.m[0].kap - F.m[1].kap;
  const float h = 0.5f * K.dth;
  for (int c = threadIdx.x; c < NI + NRX + NRY; c += NT) {
    int lx, ly;
    if (c < NI) {
      lx = c % TX;
      ly = c / TX;
    } else if (c < NI + NRX) {
      const int r = c - NI;
      lx = (r & 1) ? TX : -1;
      ly = r >> 1;
    } else {
      const int r = c - NI - NRX;
      ly = (r & 1) ? TY : -1;
      lx = r >> 1;
    }
    const int i = i0 + lx, j = j0 + ly;
    // the faces of the tile that take this cell's edge states
    const bool row = DIM == 1 || (ly >= 0 && ly < TY && j < pd.ny);
    const bool xlo = row && lx >= 0 && i <= pd.nx;     // side 1 of x face lx
    const bool xhi = row && lx < TX && i < pd.nx;      // side 0 of x face lx + 1
    bool ylo = false, yhi = false;
    if constexpr (DIM == 2) {
      const bool col = lx >= 0 && lx < TX && i < pd.nx;
      ylo = col && ly >= 0 && j <= pd.ny;              // side 1 of y face ly
      yhi = col && ly < TY && j < pd.ny;               // side 0 of y face ly + 1
    }
    if (!(xlo || xhi || ylo || yhi)) continue;
    const int kc = (ly + (DIM == 2 ? NG : 0)) * HX + lx + NG;
    PrimF wc;
    load_prim_sm<DIM, RX>(Wsm, kc, wc);
    float D[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) D[q] = 0.f;
    float divu = 0.f, bx = 0.f, by = 0.f, small = 0.f;
    const int fxl = DIM == 2 ? ly * (TX + 1) + lx : lx;  // x face to the cell's left
    float* Exl = E + (NF * NFA + fxl);                     // side 1 of face fxl
    float* Exh = E + (fxl + 1);                            // side 0 of face fxl + 1
    {
      FStateF sl, sh;
      edge_states<DIM, RX, 0, LIM, GEN>(F, Wsm, HX, plane, kc, dxf, dyf, wc, sl, sh);
      own_flux_diff<DIM, RX, 0>(sl, sh, K.ihx, k2f, D, divu, bx, by, small);
      if (xlo) put_cons<DIM, RX, 0>(sl, Exl, NFA);
      if (xhi) put_cons<DIM, RX, 0>(sh, Exh, NFA);
    }
    float* Eyl = E;
    float* Eyh = E;
    if constexpr (DIM == 2) {
      const int fyl = NFX + ly * TX + lx;  // y face below the cell
      Eyl = E + (NF * NFA + fyl);
      Eyh = E + (fyl + TX);
      FStateF sl, sh;
      edge_states<DIM, RX, 1, LIM, GEN>(F, Wsm, HX, plane, kc, dyf, dxf, wc, sl, sh);
      own_flux_diff<DIM, RX, 1>(sl, sh, K.ihy, k2f, D, divu, bx, by, small);
      if (ylo) put_cons<DIM, RX, 1>(sl, Eyl, NFA);
      if (yhi) put_cons<DIM, RX, 1>(sh, Eyh, NFA);
    }
    // non-conservative terms with the cell-centre coefficients; the e_s row
    const float t23 = 2.f / 3.f;
    D[L::PHI] -= wc.phi * divu;
    D[L::E] = small + dkf * wc.phi * divu;
    D[L::V11] -= t23 * wc.V11 * divu - wc.u * bx;
    D[L::V22] -= t23 * wc.V22 * divu - wc.v * by;
    D[L::V33] -= t23 * wc.V33 * divu;
    if constexpr (DIM == 2) {
      D[L::V12] -= t23 * wc.V12 * divu - wc.u * by;
      D[L::V21] -= t23 * wc.V21 * divu - wc.v * bx;
    }
    auto evolve = [&](float* e) {
#pragma unroll
      for (int q = 0; q < NF; ++q) e[q * NFA] -= h * D[q];
    };
    if (xlo) evolve(Exl);
    if (xhi) evolve(Exh);
    if constexpr (DIM == 2) {
      if (ylo) evolve(Eyl);
      if (yhi) evolve(Eyh);
    }
  }
}

// One face of the corrector: the Riemann problem between the evolved states
// of sides 0 and 1 of face f (SMEM cells ka, kb for the fallback), into the
// face slots fidx of Fsm.
template <int DIM, bool RX, int DIR, bool GEN>
__device__ __forceinline__ void corr_face(const PhysF& F, const float* __restrict__ Wsm,
                                          const float* __restrict__ E, int NFA, int f, int ka, int kb,
                                          float* __restrict__ Fa, float* __restrict__ Fb) {
  constexpr int NF = Lay<DIM, RX>::NF;
  float v[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) v[q] = E[q * NFA + f];
  FStateF sl = face_state_cons_f<DIM, RX, DIR, GEN>(F, v);
  if (!(sl.cL > 0.f)) {
    PrimF w;
    load_prim_sm<DIM, RX>(Wsm, ka, w);
    sl = face_state_f<DIR, GEN>(F, w);
  }
#pragma unroll
  for (int q = 0; q < NF; ++q) v[q] = E[(NF + q) * NFA + f];
  FStateF sr = face_state_cons_f<DIM, RX, DIR, GEN>(F, v);
  if (!(sr.cL > 0.f)) {
    PrimF w;
    load_prim_sm<DIM, RX>(Wsm, kb, w);
    sr = face_state_f<DIR, GEN>(F, w);
  }
  sl.cL = sqrtf(sl.cL);
  sr.cL = sqrtf(sr.cL);
  const FaceOutF o = hlld_f<DIR>(sl, sr);
  put_face<DIM, RX, DIR>(o, Fa, Fb, f);
}

// Phase 3: the corrector over all x and y faces of the tile.
template <int DIM, bool RX, int TX, int TY, int NT, bool GEN>
__device__ __forceinline__ void correct_tile(const PhysF& F, const StepArgs32& A, const int4 t,
                                             float* __restrict__ sm) {
  using TL = TileLay<DIM, RX, TX, TY>;
  constexpr int HX = TL::HX, NFX = TL::NFX, NFA = TL::NFA;
  const float* Wsm = sm;
  float* Fa = sm + TL::FAO;
  float* Fb = sm + TL::FBO;
  const float* E = sm + TL::END;
  const PatchDev pd = A.pd[t.x];
  const int i0 = t.y, j0 = t.z;
  for (int f = threadIdx.x; f < NFA; f += NT) {
    if (f < NFX) {
      const int fx = f % (TX + 1), fy = f / (TX + 1);
      if (i0 + fx > pd.nx || (DIM == 2 && j0 + fy >= pd.ny)) continue;
      const int kb = (DIM == 2 ? fy + NG : 0) * HX + fx + NG;  // the cell right of the face
      corr_face<DIM, RX, 0, GEN>(F, Wsm, E, NFA, f, kb - 1, kb, Fa, Fb);
    } else if constexpr (DIM == 2) {
      const int g = f - NFX;
      const int fx = g % TX, fy = g / TX;
      if (i0 + fx >= pd.nx || j0 + fy > pd.ny) continue;
      const int kb = (fy + NG) * HX + fx + NG;  // the cell above the face
      corr_face<DIM, RX, 1, GEN>(F, Wsm, E, NFA, f, kb - HX, kb, Fa, Fb);
    }
  }
}

// One MUSCL-Hancock step on the tile t (A: a = 0, b = 1, last stage; src =
// q^n, dst = the other buffer).
template <int DIM, bool RX, int TX, int TY, int NT, int LIM, bool GEN>
__device__ __forceinline__ void hancock32_tile(const Phys& P, const PhysF& F, const StepArgs32& A, const int4 t,
                                               float* __restrict__ sm, unsigned* rate_cta) {
  __shared__ TileConst K;
  if (threadIdx.x == 0) tile_consts(P, A, t, K);
  fill_tile<DIM, RX, TX, TY, NT, GEN>(P, F, A, t, sm);
  __syncthreads();
  predict_tile<DIM, RX, TX, TY, NT, LIM, GEN>(F, A, t, sm, K);
  __syncthreads();
  correct_tile<DIM, RX, TX, TY, NT, GEN>(F, A, t, sm);
  __syncthreads();
  update_tile<DIM, RX, TX, TY, NT, false, GEN>(P, F, A, t, sm, K, rate_cta);
}

template <int DIM, bool RX, int TX, int TY, int NT, int MINB, int LIM, bool GEN>
__global__ void __launch_bounds__(NT, MINB) k_hancock32(Phys P, PhysF F, StepArgs32 A,
                                                        const int4* __restrict__ tiles) {
  extern __shared__ __align__(16) float sm[];
  hancock32_tile<DIM, RX, TX, TY, NT, LIM, GEN>(P, F, A, tiles[blockIdx.x], sm, nullptr);
}

// Persistent 1D batch form: one CTA per problem runs n_steps steps over its
// tiles in turn; step s reads B.q[s & 1] and writes B.q[(s + 1) & 1].
// rate_ready = 0: the CFL rate of the state in B.q[0] is taken first.
// scratch (tuning, n_steps = 1): the rate of the new state is not kept.
template <bool RX, int TX, int NT, int MINB, int LIM, bool GEN>
__global__ void __launch_bounds__(NT, MINB) k_hbatch32(Phys P, PhysF F, StepArgs32 A, Bufs32 B,
                                                       unsigned long long* rate, const int* __restrict__ order,
                                                       const int* __restrict__ tile0,
                                                       const int4* __restrict__ tiles, int n_steps, int scratch,
                                                       int rate_ready) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float wmax[NT / 32];
  __shared__ unsigned rnext;
  const int p = order[blockIdx.x];
  const int ta = tile0[p], tb = tile0[p + 1];
  const PatchDev pd = A.pd[p];
  if (!rate_ready) {
    float r = 0.f;
    for (int i = threadIdx.x; i < pd.nx; i += NT)
      r = fmaxf(r, cfl_rate_of<1, GEN>(F, cons_to_prim32<1, RX, GEN>(P, F, B.q[0], A.T, cidx(pd, i, 0)),
                                       1.f / (float)pd.dx, 1.f, A.status, p, i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) m = fmaxf(m, wmax[w]);
      rate[p] = (unsigned long long)__double_as_longlong((double)m);
    }
    __syncthreads();
  }
  for (int n = 0; n < n_steps; ++n) {
    if (threadIdx.x == 0) rnext = 0u;  // ordered before the update's atomics by the tile barriers
    StepArgs32 a = A;
    a.src = B.q[n & 1];
    a.qn = a.src;
    a.dst = B.q[(n + 1) & 1];
    a.rate = rate;
    a.a = 0.0;
    a.b = 1.0;
    a.last = true;
    for (int t = ta; t < tb; ++t) {
      hancock32_tile<1, RX, TX, 1, NT, LIM, GEN>(P, F, a, tiles[t], sm, &rnext);
      __syncthreads();
    }
    // the next step's rate (thread 0 reads it, for dt, in the next tile)
    if (threadIdx.x == 0 && !scratch)
      rate[p] = (unsigned long long)__double_as_longlong((double)__uint_as_float(rnext));
  }
}

}  // namespace dis
