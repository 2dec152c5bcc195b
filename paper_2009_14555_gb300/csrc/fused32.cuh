// fused32.cuh - one fused kernel per SSP-RK3 stage for the FP32-bulk step.
//
// A CTA owns a tile of TX x TY interior cells (TX cells of one row in 1D).
// It recovers the primitives of the tile plus a 3-cell halo into shared
// memory (ghosts by index map), computes every x face and y face of the tile
// (MUSCL/THINC-BVD + HLLD) into shared memory, and updates its cells
// (divergence, non-conservative terms, RK3 combination; last stage: plastic
// and reactive steps, and the CFL rate of the new state for the next step's
// time step).  Primitives and face data never go to HBM: per stage the tile
// reads q_src (with halo, mostly from L2) and q^n and writes q_dst.  No
// float64 arithmetic runs outside the rare mixed-cell plastic branch.
//
// Energy (state slot E = e_s = rho E - kappa(phi1), step32.cuh): the rho E
// flux is the float soft flux plus kappa(phi_K) X, X = u_face + D (D a small
// star compression term), kappa(phi) = kappa_2 + (kappa_1 - kappa_2) phi.
// Subtracting (kappa_1 - kappa_2) times the phi1 equation (flux phi_K u_face,
// source phi div u_face) leaves
//   d e_s/dt = -[div F_soft + kappa_2 div X + (kappa_1 - kappa_2) div(phi_K D)
//                + (kappa_1 - kappa_2) phi div u_face],
// whose terms are differences of face values that are formed before any
// large factor multiplies them.  phi1 itself is advanced in float-float from
// the exact (TwoSum) differences of its float face fluxes.
#pragma once
#include "step32.cuh"

namespace dis {

// Shared-memory records.  A tile keeps its primitives and its face data as
// records of consecutive floats, read and written as float4 (and float2 or
// float4 tails), so a cell or a face costs a few 128-bit shared-memory
// accesses instead of one access per field:
//   * a cell: PR = 12 floats, the primitives in the slots of the conservative
//     layout (PHI phi1, A1 rho1, A2 rho2, MX u, MY v, E p, V, AL lam), plus a
//     separate plane of phi1 for the THINC stencils;
//   * a face normal to DIR: Rec<DIM, RX, DIR> below, FA = 12 floats plus (2D)
//     FB = 4 floats held apart.
// A stride of 12 floats (48 B) maps the 8 lanes of a quarter warp onto
// distinct banks, so the float4 accesses of consecutive cells or faces are
// free of bank conflicts.
constexpr int PR = 12;
constexpr int FA = 12;

template <int DIM>
constexpr int face_fb() {
  return DIM == 2 ? 4 : 0;
}

// Face record along DIR: the fluxes of the fields that have one (the V row
// fluxes V_ij u_d - V_dj u_i vanish for i = d: V11 and V12 on x faces, V21
// and V22 on y faces), then u_face, the V row of the face (VA, and VB in 2D),
// phi_K and D.  The phi slot holds F_phi = phi_K u_face, the E slot the soft
// energy flux.
template <int DIM, bool RX, int DIR>
struct Rec {
  using L = Lay<DIM, RX>;
  static constexpr bool zero(int c) {
    return DIR == 0 ? (c == L::V11 || (DIM == 2 && c == L::V12)) : (c == L::V21 || c == L::V22);
  }
  static constexpr int pos(int c) {
    int p = 0;
    for (int k = 0; k < c; ++k) p += zero(k) ? 0 : 1;
    return p;
  }
  static constexpr int NFL = L::NF - (DIM == 2 ? 2 : 1);
  static constexpr int UF = NFL, VA = NFL + 1, VB = DIM == 2 ? NFL + 2 : -1;
  static constexpr int PK = DIM == 2 ? NFL + 3 : NFL + 2, DD = PK + 1, N = DD + 1;
  static_assert(N <= FA + face_fb<DIM>(), "face record size");
};

// Offsets (in floats) of a tile's shared-memory regions: cell records, the
// phi1 plane (padded to a multiple of 4), face records A, face records B.
template <int DIM, bool RX, int TX, int TY>
struct TileLay {
  static constexpr int HX = TX + 2 * NG, HY = DIM == 2 ? TY + 2 * NG : 1, PLANE = HX * HY;
  static constexpr int NFX = (TX + 1) * TY, NFY = DIM == 2 ? TX * (TY + 1) : 0, NFA = NFX + NFY;
  static constexpr int PHI = PR * PLANE;
  static constexpr int FAO = PHI + ((PLANE + 3) / 4) * 4;
  static constexpr int FBO = FAO + FA * NFA;
  static constexpr int END = FBO + face_fb<DIM>() * NFA;
};

// Face record r (N values of Rec) of face f into / out of shared memory.
template <int DIM>
__device__ __forceinline__ void store_face(float* __restrict__ Fa, float* __restrict__ Fb, int f, const float* r) {
  float4* a = reinterpret_cast<float4*>(Fa + FA * f);
  a[0] = make_float4(r[0], r[1], r[2], r[3]);
  a[1] = make_float4(r[4], r[5], r[6], r[7]);
  a[2] = make_float4(r[8], r[9], r[10], r[11]);
  if constexpr (DIM == 2)
    reinterpret_cast<float4*>(Fb)[f] = make_float4(r[12], r[13], r[14], r[15]);
}
template <int DIM>
__device__ __forceinline__ void load_face(const float* __restrict__ Fa, const float* __restrict__ Fb, int f,
                                          float* r) {
  const float4* a = reinterpret_cast<const float4*>(Fa + FA * f);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const float4 x = a[v];
    r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
  }
  if constexpr (DIM == 2) {
    const float4 x = reinterpret_cast<const float4*>(Fb)[f];
    r[12] = x.x; r[13] = x.y; r[14] = x.z; r[15] = x.w;
  }
}

// THINC steepness of the cell at SMEM index k (phi plane Wphi; sx along the
// sweep, sy across it): Youngs normal from the 3 x 3 neighbourhood in 2D
// (Appendix A), the 1D value otherwise.
template <int DIM>
__device__ __forceinline__ float thinc_beta_f(const PhysF& P, const float* __restrict__ Wphi, int k, int sx,
                                              int sy, float dxn, float dxt) {
  float beta = 2.51f;
  if (DIM == 2 && P.thinc) {
    const float dn = (Wphi[k + sx + sy] + 2.f * Wphi[k + sx] + Wphi[k + sx - sy]) -
                     (Wphi[k - sx + sy] + 2.f * Wphi[k - sx] + Wphi[k - sx - sy]);
    const float dt_ = (Wphi[k + sy + sx] + 2.f * Wphi[k + sy] + Wphi[k + sy - sx]) -
                      (Wphi[k - sy + sx] + 2.f * Wphi[k - sy] + Wphi[k - sy - sx]);
    const float gn = dn / dxn, gt = dt_ / dxt;
    const float nrm = sqrtf(gn * gn + gt * gt);
    beta = 2.5f * (nrm == 0.f ? 1.f : fabsf(gn) / nrm) + 0.01f;
  }
  return beta;
}

// The face record (Rec) of a face output o on a face normal to DIR, through
// put(position, value).
template <int DIM, bool RX, int DIR, class Put>
__device__ __forceinline__ void face_slots_f(const FaceOutF& o, const Put& put) {
  using L = Lay<DIM, RX>;
  using R = Rec<DIM, RX, DIR>;
  const float fu = DIR == 0 ? o.un : o.ut;
  const float fv = DIR == 0 ? o.ut : o.un;
  put(R::pos(L::PHI), o.phi * o.un);
  put(R::pos(L::A1), o.Far1);
  put(R::pos(L::A2), o.Far2);
  put(R::pos(L::MX), DIR == 0 ? o.Fmn : o.Fmt);
  if constexpr (DIM == 2) put(R::pos(L::MY), DIR == 0 ? o.Fmt : o.Fmn);
  put(R::pos(L::E), o.FE);
  if constexpr (RX) put(R::pos(L::AL), o.Farl);
  put(R::UF, o.un);
  put(R::PK, o.phi);
  put(R::DD, o.D);
  if constexpr (DIR == 0) {
    if constexpr (DIM == 2) {
      put(R::pos(L::V21), o.V21 * fu - o.V11 * fv);
      put(R::pos(L::V22), o.V22 * fu - o.V12 * fv);
      put(R::VA, o.V11);
      put(R::VB, o.V12);
    } else {
      put(R::pos(L::V22), o.V22 * fu);
      put(R::VA, o.V11);
    }
    put(R::pos(L::V33), o.V33 * fu);
  } else if constexpr (DIM == 2) {
    put(R::pos(L::V11), o.V11 * fv - o.V21 * fu);
    put(R::pos(L::V12), o.V12 * fv - o.V22 * fu);
    put(R::pos(L::V33), o.V33 * fv);
    put(R::VA, o.V21);
    put(R::VB, o.V22);
  }
}

// Face record of o into face f of (Fa, Fb).
template <int DIM, bool RX, int DIR>
__device__ __forceinline__ void put_face(const FaceOutF& o, float* __restrict__ Fa, float* __restrict__ Fb,
                                         int f) {
  float r[FA + 4];
#pragma unroll
  for (int k = 0; k < FA + 4; ++k) r[k] = 0.f;
  face_slots_f<DIM, RX, DIR>(o, [&](int k, float v) { r[k] = v; });
  store_face<DIM>(Fa, Fb, f, r);
}

// Primitives of the SMEM cell k (its record of PR floats, slots as the
// conservative layout: PHI phi1, A1 rho1, A2 rho2, MX u, MY v, E p, V, AL lam).
template <int DIM, bool RX>
__device__ __forceinline__ void load_prim_sm(const float* __restrict__ Wsm, int k, PrimF& w) {
  using L = Lay<DIM, RX>;
  constexpr int NV = (L::NF + 3) / 4;
  float r[PR];
  const float4* a = reinterpret_cast<const float4*>(Wsm + PR * k);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 x = a[v];
    r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
  }
  w.phi = r[L::PHI]; w.r1 = r[L::A1]; w.r2 = r[L::A2]; w.u = r[L::MX];
  w.p = r[L::E]; w.V11 = r[L::V11]; w.V22 = r[L::V22]; w.V33 = r[L::V33];
  w.v = 0.f; w.V12 = 0.f; w.V21 = 0.f; w.lam = 0.f;
  if constexpr (DIM == 2) { w.v = r[L::MY]; w.V12 = r[L::V12]; w.V21 = r[L::V21]; }
  if constexpr (RX) w.lam = r[L::AL];
}

// The record of SMEM cell c and its entry in the phi1 plane (plane cells).
template <int DIM, bool RX>
__device__ __forceinline__ void store_prim_sm(float* __restrict__ Wsm, int plane, int c, const PrimF& w) {
  using L = Lay<DIM, RX>;
  constexpr int NV = (L::NF + 3) / 4;
  float r[PR];
#pragma unroll
  for (int k = 0; k < PR; ++k) r[k] = 0.f;
  r[L::PHI] = w.phi; r[L::A1] = w.r1; r[L::A2] = w.r2; r[L::MX] = w.u;
  r[L::E] = w.p; r[L::V11] = w.V11; r[L::V22] = w.V22; r[L::V33] = w.V33;
  if constexpr (DIM == 2) { r[L::MY] = w.v; r[L::V12] = w.V12; r[L::V21] = w.V21; }
  if constexpr (RX) r[L::AL] = w.lam;
  float4* a = reinterpret_cast<float4*>(Wsm + PR * c);
#pragma unroll
  for (int v = 0; v < NV; ++v) a[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
  Wsm[PR * plane + c] = w.phi;
}

template <int DIM, bool RX, int DIR, int LIM, bool GEN>
__device__ __forceinline__ void face32(const PhysF& P, const float* __restrict__ Wsm, int HX, int HY, int hx,
                                       int hy, float dxn, float dxt, float* __restrict__ Fa,
                                       float* __restrict__ Fb, int fidx) {
  // hx, hy: SMEM coordinates of the face's left (DIR 0) or lower (DIR 1) cell
  const int plane = HX * HY;
  const int sx = DIR == 0 ? 1 : HX;  // along the sweep
  const int sy = DIR == 0 ? HX : 1;  // across it
  const int k0 = hy * HX + hx;       // cell a
  const float* Wphi = Wsm + PR * plane;
  float ph[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) ph[s] = Wphi[k0 + (s - 2) * sx];
  // MUSCL-BVD-THINC edge values of cells a and a + 1.  A cell that is not
  // mixed has identical MUSCL and THINC candidates, so the BVD choice (and
  // the candidate of its outer neighbour, which only that choice reads) is
  // needed only for a mixed cell.
  auto cand = [&](int s) {
    auto beta_of = [&]() -> float { return thinc_beta_f<DIM>(P, Wphi, k0 + (s - 1) * sx, sx, sy, dxn, dxt); };
    return phi_cand_f<LIM>(ph[s], ph[s + 1], ph[s + 2], beta_of, P.thinc != 0, P.limiter);
  };
  const CandF c1 = cand(1), c2 = cand(2);
  float phiL = c1.mR, phiR = c2.mL;
  if (c1.mixed) {
    float Lt;
    bvd_f(cand(0), c1, c2, Lt, phiL);
  }
  if (c2.mixed) {
    float Rt;
    bvd_f(c1, c2, cand(3), phiR, Rt);
  }
  // the two edge states one after the other (fewer values live at once):
  // cell a's right edge from cells a - 1, a, a + 1, cell a + 1's left edge
  // from cells a, a + 1, a + 2
  auto edge = [&](int kc, float sgn, float phi_e, PrimF& we, PrimF& wc) {
    PrimF wm, wp;
    load_prim_sm<DIM, RX>(Wsm, kc - sx, wm);
    load_prim_sm<DIM, RX>(Wsm, kc, wc);
    load_prim_sm<DIM, RX>(Wsm, kc + sx, wp);
#define DIS_RECF(fld) we.fld = wc.fld + sgn * (0.5f * limited_f<LIM>(wc.fld - wm.fld, wp.fld - wc.fld, P.limiter));
    DIS_RECF(r1) DIS_RECF(r2) DIS_RECF(u) DIS_RECF(p) DIS_RECF(V11) DIS_RECF(V22) DIS_RECF(V33)
    if constexpr (DIM == 2) { DIS_RECF(v) DIS_RECF(V12) DIS_RECF(V21) }
    else { we.v = 0.f; we.V12 = we.V21 = 0.f; }
    if constexpr (RX) { DIS_RECF(lam) } else { we.lam = 0.f; }
#undef DIS_RECF
    we.phi = phi_e;
  };
  FStateF sl, sr;
  {
    PrimF we, wc;
    edge(k0, 1.f, phiL, we, wc);
    sl = face_state_f<DIR, GEN>(P, we);
    if (!(sl.cL > 0.f)) sl = face_state_f<DIR, GEN>(P, wc);
  }
  {
    PrimF we, wc;
    edge(k0 + sx, -1.f, phiR, we, wc);
    sr = face_state_f<DIR, GEN>(P, we);
    if (!(sr.cL > 0.f)) sr = face_state_f<DIR, GEN>(P, wc);
  }
  sl.cL = sqrtf(sl.cL);
  sr.cL = sqrtf(sr.cL);
  const FaceOutF o = hlld_f<DIR>(sl, sr);
  put_face<DIM, RX, DIR>(o, Fa, Fb, fidx);
}

// Shared memory bytes of a tile.
template <int DIM, bool RX, int TX, int TY>
constexpr size_t fused32_smem() {
  return sizeof(float) * (size_t)TileLay<DIM, RX, TX, TY>::END;
}

// Positive float -> bits that order like the value (for integer atomic max).
__device__ __forceinline__ unsigned rate_bits(float r) { return __float_as_uint(fmaxf(r, 0.f)); }

// Per-tile constants of the update, formed by one thread: dt as float-float
// and float, the RK weights (b as float-float), the inverse cell sizes.
struct TileConst {
  float dth, dtl, af, bh, bl, ihx, ihy;
};

__device__ __forceinline__ void tile_consts(const Phys& P, const StepArgs32& A, const int4 t, TileConst& K) {
  const PatchDev& pd = A.pd[t.x];
  const double dt = A.dtfix ? A.dtfix[t.x] : P.cfl / __longlong_as_double((long long)A.rate[t.x]);
  const ff d = ff_of(dt), b = ff_of(A.b);
  K.dth = d.h;
  K.dtl = d.l;
  K.af = (float)A.a;
  K.bh = b.h;
  K.bl = b.l;
  K.ihx = 1.f / (float)pd.dx;
  K.ihy = 1.f / (float)pd.dy;
  if (A.last && t.y == 0 && t.z == 0) A.dtlast[t.x] = dt;
}

// Phase 1: primitives of the tile t and its halo (ghosts by the index map)
// into the shared-memory planes of sm, by the NT threads of the CTA.
template <int DIM, bool RX, int TX, int TY, int NT, bool GEN>
__device__ __forceinline__ void fill_tile(const Phys& P, const PhysF& F, const StepArgs32& A, const int4 t,
                                          float* __restrict__ sm) {
  using L = Lay<DIM, RX>;
  constexpr int HX = TX + 2 * NG, HY = DIM == 2 ? TY + 2 * NG : 1;
  float* Wsm = sm;
  const PatchDev pd = A.pd[t.x];
  const int i0 = t.y, j0 = t.z;
  const long long T = A.T;
  constexpr int NC = HX * HY, NS = Lay<DIM, RX>::NF + 1;
  // two cells per thread and pass: both cells' loads are in flight before
  // either recovery starts
  for (int c0 = threadIdx.x; c0 < NC; c0 += 2 * NT) {
    float v[2][NS];
    bool ok[2], fx[2], fy[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int c = c0 + m * NT;
      const int hx = c % HX, hy = c / HX;
      const int i = i0 - NG + hx;
      const int j = DIM == 2 ? j0 - NG + hy : 0;
      ok[m] = c < NC && !(i < -NG || i >= pd.nx + NG || (DIM == 2 && (j < -NG || j >= pd.ny + NG)));
      fx[m] = fy[m] = false;
      if (ok[m]) {
        const int si = ghost_map(i, pd.nx, pd.bc[0], pd.bc[1], fx[m]);
        const int sj = DIM == 2 ? ghost_map(j, pd.ny, pd.bc[2], pd.bc[3], fy[m]) : 0;
        load32<DIM, RX>(A.src, T, cidx(pd, si, sj), v[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (!ok[m]) continue;
      PrimF w = prim32_of<DIM, RX, GEN>(P, F, v[m]);
      if (fx[m]) { w.u = -w.u; w.V12 = -w.V12; w.V21 = -w.V21; }
      if (fy[m]) { w.v = -w.v; w.V12 = -w.V12; w.V21 = -w.V21; }
      store_prim_sm<DIM, RX>(Wsm, NC, c0 + m * NT, w);
    }
  }
}

// Phase 2: all x faces ((TX + 1) per interior row) and y faces (TX per face
// row, TY + 1 face rows) of the tile, in one loop so the threads stay busy.
template <int DIM, bool RX, int TX, int TY, int NT, int LIM, bool GEN>
__device__ __forceinline__ void faces_tile(const PhysF& F, const StepArgs32& A, const int4 t,
                                           float* __restrict__ sm) {
  using TL = TileLay<DIM, RX, TX, TY>;
  constexpr int HX = TL::HX, HY = TL::HY, NFX = TL::NFX, NFY = TL::NFY;
  const float* Wsm = sm;
  float* Fa = sm + TL::FAO;
  float* Fb = sm + TL::FBO;
  const PatchDev pd = A.pd[t.x];
  const int i0 = t.y, j0 = t.z;
  const float dxf = (float)pd.dx, dyf = (float)pd.dy;
  for (int f = threadIdx.x; f < NFX + NFY; f += NT) {
    if (f < NFX) {
      const int fx = f % (TX + 1), fy = f / (TX + 1);
      const int i = i0 + fx, j = j0 + fy;  // face between cells i-1 and i
      if (i > pd.nx || (DIM == 2 && j >= pd.ny)) continue;
      face32<DIM, RX, 0, LIM, GEN>(F, Wsm, HX, HY, fx + NG - 1, DIM == 2 ? fy + NG : 0, dxf, dyf, Fa, Fb, f);
    } else if constexpr (DIM == 2) {
      const int g = f - NFX;
      const int fx = g % TX, fy = g / TX;
      const int i = i0 + fx, j = j0 + fy;  // face between rows j-1 and j
      if (i >= pd.nx || j > pd.ny) continue;
      face32<DIM, RX, 1, LIM, GEN>(F, Wsm, HX, HY, fx + NG, fy + NG - 1, dyf, dxf, Fa, Fb, f);
    }
  }
}

// Phase 3: update of the tile's cells from the faces in sm (divergence,
// non-conservative terms, RK combination; last stage: plastic and reactive
// steps and the CFL rate of the new state, by warp max into rate_cta (shared,
// if not null) or A.rate_next[patch] (global)).  Every lane of a warp with a
// tile cell reaches the warp max.
template <int DIM, bool RX, int TX, int TY, int NT, bool CYL, bool GEN>
__device__ __forceinline__ void update_tile(const Phys& P, const PhysF& F, const StepArgs32& A, const int4 t,
                                            const float* __restrict__ sm, const TileConst& K,
                                            unsigned* rate_cta) {
  static_assert(TX * TY <= NT, "one thread per tile cell in the update phase");
  using L = Lay<DIM, RX>;
  using TL = TileLay<DIM, RX, TX, TY>;
  constexpr int NF = L::NF;
  constexpr int HX = TL::HX, NFX = TL::NFX;
  const float* Wsm = sm;
  const float* Fa = sm + TL::FAO;
  const float* Fb = sm + TL::FBO;
  const PatchDev pd = A.pd[t.x];
  const int i0 = t.y, j0 = t.z;
  const int tid = threadIdx.x;
  const float dxf = (float)pd.dx;
  const long long T = A.T;
  const float dth_sh = K.dth, dtl_sh = K.dtl, af_sh = K.af, bh_sh = K.bh, bl_sh = K.bl, ihx_sh = K.ihx,
              ihy_sh = K.ihy;

  // 3. update of the tile's cells (every lane of a warp with a tile cell
  //    reaches the warp max of the last stage)
  if (tid >= ((TX * TY + 31) / 32) * 32) return;
  const int lx = tid % TX, ly = tid / TX;
  const int i = i0 + lx, j = j0 + ly;
  const bool valid = tid < TX * TY && i < pd.nx && (DIM == 1 || j < pd.ny);
  float rate = 0.f;
  if (valid) {
    const long long k = cidx(pd, i, j);
    float q[NF + 1], D[NF];
    load32<DIM, RX>(A.src, T, k, q);
    const float idx_ = ihx_sh;
    const int fl = ly * (TX + 1) + lx, fr = fl + 1;
    using RXf = Rec<DIM, RX, 0>;
    float xl[FA + 4], xr[FA + 4];
    load_face<DIM>(Fa, Fb, fl, xl);
    load_face<DIM>(Fa, Fb, fr, xr);
    auto FX = [&](int s, bool right) { return right ? xr[s] : xl[s]; };
#pragma unroll
    for (int c = 0; c < NF; ++c)
      D[c] = RXf::zero(c) ? 0.f : (FX(RXf::pos(c), true) - FX(RXf::pos(c), false)) * idx_;
    float divu = (FX(RXf::UF, true) - FX(RXf::UF, false)) * idx_;
    float bx = (FX(RXf::VA, true) - FX(RXf::VA, false)) * idx_;
    float by = 0.f;
    if constexpr (DIM == 2) by = (xr[RXf::VB] - xl[RXf::VB]) * idx_;
    const float k2f = F.m[1].kap, dkf = F.m[0].kap - F.m[1].kap;
    // phi1 flux divergence from the exact differences of the float fluxes
    ff Dc = ff_mul_f(two_sum(xr[RXf::pos(L::PHI)], -xl[RXf::pos(L::PHI)]), idx_);
    // soft part of the e_s divergence: differences first, then the large factors
    float small = ((xr[RXf::pos(L::E)] - xl[RXf::pos(L::E)]) +
                   k2f * ((xr[RXf::UF] - xl[RXf::UF]) + (xr[RXf::DD] - xl[RXf::DD])) +
                   dkf * (xr[RXf::PK] * xr[RXf::DD] - xl[RXf::PK] * xl[RXf::DD])) * idx_;
    if constexpr (DIM == 2) {
      using RYf = Rec<DIM, RX, 1>;
      const float idy = ihy_sh;
      const int fb = NFX + ly * TX + lx, ft = fb + TX;
      float yb[FA + 4], yt[FA + 4];
      load_face<DIM>(Fa, Fb, fb, yb);
      load_face<DIM>(Fa, Fb, ft, yt);
#pragma unroll
      for (int c = 0; c < NF; ++c)
        if (!RYf::zero(c)) D[c] += (yt[RYf::pos(c)] - yb[RYf::pos(c)]) * idy;
      divu += (yt[RYf::UF] - yb[RYf::UF]) * idy;
      bx += (yt[RYf::VA] - yb[RYf::VA]) * idy;
      by += (yt[RYf::VB] - yb[RYf::VB]) * idy;
      Dc = ff_add(Dc, ff_mul_f(two_sum(yt[RYf::pos(L::PHI)], -yb[RYf::pos(L::PHI)]), idy));
      small += ((yt[RYf::pos(L::E)] - yb[RYf::pos(L::E)]) +
                k2f * ((yt[RYf::UF] - yb[RYf::UF]) + (yt[RYf::DD] - yb[RYf::DD])) +
                dkf * (yt[RYf::PK] * yt[RYf::DD] - yb[RYf::PK] * yb[RYf::DD])) * idy;
    }
    const ff phi_c = {q[L::PHI], q[NF]};
    const ff Dphi = ff_add(Dc, ff_neg(ff_mul_f(phi_c, divu)));
    float Des = small + dkf * phi_c.h * divu;
    const float rho = q[L::A1] + q[L::A2];
    const float uc = q[L::MX] / rho;
    float vc = 0.f;
    if constexpr (DIM == 2) vc = q[L::MY] / rho;
    if constexpr (CYL) {
      // cylindrical geometric source (x = r, y = z) from the cell's primitives
      // in shared memory; energy: rho E u_r with rho E = e_s + kappa(phi1)
      const int kc = (ly + (DIM == 2 ? NG : 0)) * HX + lx + NG;
      PrimF wc;
      load_prim_sm<DIM, RX>(Wsm, kc, wc);
      const float wp = wc.p, wphi = wc.phi, wu = wc.u, wv = wc.v;
      const StrainF st = strain_f(wc.V11, wc.V12, wc.V21, wc.V22, wc.V33);
      const float Gm2 = 2.f * Gmix_f<GEN>(F, wphi, wc.r1, wc.r2);
      const float srr = -wp + Gm2 * st.H11, szr = Gm2 * st.H12, stt = -wp + Gm2 * st.H33;
      const float r = (float)pd.x0 + ((float)i + 0.5f) * dxf;
      const float ir = 1.f / r;
      D[L::A1] += q[L::A1] * wu * ir;
      D[L::A2] += q[L::A2] * wu * ir;
      if constexpr (RX) D[L::AL] += q[L::AL] * wu * ir;
      D[L::MX] += (rho * wu * wu - srr + stt) * ir;
      if constexpr (DIM == 2) D[L::MY] += (rho * wv * wu - szr) * ir;
      Des += (q[L::E] * wu + (k2f + dkf * phi_c.h) * wu - (wu * srr + wv * szr)) * ir;
      const float tt = wu * ir * (1.f / 3.f);
      D[L::V11] += tt * q[L::V11];
      D[L::V22] += tt * q[L::V22];
      D[L::V33] -= 2.f * tt * q[L::V33];
      if constexpr (DIM == 2) {
        D[L::V12] += tt * q[L::V12];
        D[L::V21] += tt * q[L::V21];
      }
    }
    const float t23 = 2.f / 3.f;
    D[L::V11] -= t23 * q[L::V11] * divu - uc * bx;
    D[L::V22] -= t23 * q[L::V22] * divu - vc * by;
    D[L::V33] -= t23 * q[L::V33] * divu;
    if constexpr (DIM == 2) {
      D[L::V12] -= t23 * q[L::V12] * divu - uc * by;
      D[L::V21] -= t23 * q[L::V21] * divu - vc * bx;
    }
    const float dtf = dth_sh;
    const ff dt_ff = {dth_sh, dtl_sh};
    float o[NF + 1];
    const ff yphi = ff_add(phi_c, ff_neg(ff_mul(dt_ff, Dphi)));
    const float yE = q[L::E] - dtf * Des;
    ff ophi;
    if (af_sh == 0.f) {
#pragma unroll
      for (int c = 0; c < NF; ++c) o[c] = q[c] - dtf * D[c];
      ophi = yphi;
      o[L::E] = yE;
    } else {
      const float af = af_sh, bf = bh_sh;
      float qn[NF + 1];
      load32<DIM, RX>(A.qn, T, k, qn);
#pragma unroll
      for (int c = 0; c < NF; ++c) o[c] = af * qn[c] + bf * (q[c] - dtf * D[c]);
      o[L::E] = af * qn[L::E] + bf * yE;
      const ff phin = {qn[L::PHI], qn[NF]};
      ophi = ff_add(phin, ff_mul({bh_sh, bl_sh}, ff_add(yphi, ff_neg(phin))));
    }
    o[L::PHI] = ophi.h;
    o[NF] = ophi.l;
    if (A.last) {
      const float ophf = ophi.h;
      float v12 = 0.f, v21 = 0.f;
      if constexpr (DIM == 2) { v12 = o[L::V12]; v21 = o[L::V21]; }
      const float oph2 = (1.f - ophf) - ophi.l;
      const float or1 = o[L::A1] / ophf, or2 = o[L::A2] / oph2;
      if (ophf > 1e-3f && ophf < 1.f - 1e-3f) {
        const double dt = ff_val(dth_sh, dtl_sh);
        double d11 = o[L::V11], d12 = v12, d21 = v21, d22 = o[L::V22], d33 = o[L::V33];
        const double ph = ff_val(ophi.h, ophi.l);
        plastic(P, ph, dt, d11, d12, d21, d22, d33, (double)o[L::A1] / ph, (double)o[L::A2] / (1.0 - ph));
        o[L::V11] = (float)d11; v12 = (float)d12; v21 = (float)d21; o[L::V22] = (float)d22; o[L::V33] = (float)d33;
      } else {
        plastic_f<GEN>(F, ophf, dtf, o[L::V11], v12, v21, o[L::V22], o[L::V33], or1, or2);
      }
      if constexpr (DIM == 2) { o[L::V12] = v12; o[L::V21] = v21; }
      if constexpr (RX) {
        const int y = P.y;
        const MatT<float>& m = F.m[y];
        const float ary = y == 0 ? o[L::A1] : o[L::A2];
        const float phy = y == 0 ? ophf : oph2;
        const float rr = o[L::A1] + o[L::A2];
        const float mx = o[L::MX];
        float my = 0.f;
        if constexpr (DIM == 2) my = o[L::MY];
        const float KE = 0.5f * (mx * mx + my * my) / rr;
        const StrainF s = strain_f(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
        const float xi = xi_f(F, ophf);
        const float p0 = (o[L::E] - KE - soft_ref_f<GEN>(F, ophf, o[L::A1], o[L::A2], 0.f, s.J2, or1, or2)) / xi;
        const float Tfac = m.iGm1 / ((ary / phy) * m.cv);
        const float Qx = m.Q / xi;
        auto fr_ = [&](float Lm) {
          if (m.law == 1) {
            const float pk = p0 - Qx * Lm;
            return pk > m.pign && Lm > 0.f ? -m.A * sqrtf(ary * Lm) : 0.f;
          }
          const float Tk = (p0 - Qx * Lm) * Tfac;
          return Tk > 0.f ? -m.A * Lm * expf(-m.Tact / Tk) : 0.f;
        };
        const float L0 = o[L::AL];
        const float k1 = fr_(L0);
        const float k2 = fr_(L0 + 0.5f * dtf * k1);
        const float k3 = fr_(L0 + 0.5f * dtf * k2);
        const float k4 = fr_(L0 + dtf * k3);
        const float L1 = L0 + dtf / 6.f * (k1 + 2.f * k2 + 2.f * k3 + k4);
        o[L::AL] = m.law == 1 && !(L1 > 0.f) ? 0.f : L1;
      }
      bool bad = !(ophf >= -1e-6f && ophf <= 1.f + 1e-6f);
#pragma unroll
      for (int c = 0; c <= NF; ++c) bad |= !isfinite(o[c]);
      if (bad) flag_bad(A.status, t.x, i + pd.nx * j);
      // CFL rate of the new state: the next step's time step
      rate = cfl_rate_of<DIM, GEN>(F, prim32_of<DIM, RX, GEN>(P, F, o), ihx_sh, ihy_sh, A.status, t.x,
                                   i + pd.nx * j);
    }
#pragma unroll
    for (int c = 0; c <= NF; ++c) A.dst[c * T + k] = o[c];
  }
  if (A.last) {
#pragma unroll
    for (int s_ = 16; s_ > 0; s_ >>= 1) rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, s_));
    if ((tid & 31) == 0 && rate > 0.f) {
      if (rate_cta) atomicMax(rate_cta, rate_bits(rate));
      else atomicMax(A.rate_next + t.x, (unsigned long long)__double_as_longlong((double)rate));
    }
  }
}


// One stage on one tile t = (patch, i0, j0) by the NT threads of a CTA, with
// the tile's primitives and faces in the shared memory sm.  The stage kernel
// runs it once per CTA; the persistent 1D batch kernel runs it for every tile
// of its problem in turn (the caller synchronises the CTA between tiles).
template <int DIM, bool RX, int TX, int TY, int NT, bool CYL = false, int LIM = 0, bool GEN = false>
__device__ __forceinline__ void stage32_tile(const Phys& P, const PhysF& F, const StepArgs32& A, const int4 t,
                                             float* __restrict__ sm, unsigned* rate_cta) {
  __shared__ TileConst K;
  if (threadIdx.x == 0) tile_consts(P, A, t, K);
  fill_tile<DIM, RX, TX, TY, NT, GEN>(P, F, A, t, sm);
  __syncthreads();
  faces_tile<DIM, RX, TX, TY, NT, LIM, GEN>(F, A, t, sm);
  __syncthreads();
  update_tile<DIM, RX, TX, TY, NT, CYL, GEN>(P, F, A, t, sm, K, rate_cta);
}

template <int DIM, bool RX, int TX, int TY, int NT, int MINB, bool CYL = false, int LIM = 0, bool GEN = false>
__global__ void __launch_bounds__(NT, MINB) k_stage32(Phys P, PhysF F, StepArgs32 A, const int4* __restrict__ tiles) {
  extern __shared__ __align__(16) float sm[];
  stage32_tile<DIM, RX, TX, TY, NT, CYL, LIM, GEN>(P, F, A, tiles[blockIdx.x], sm, nullptr);
}

// CFL rate of the state at the start of a step (FP32-bulk), for the first
// step after the state was set (later steps take it from the last stage of
// the step before): per-patch max of sum_d (|u_d| + c_L) / dx_d.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_cfl32(Phys P, PhysF F, StepArgs32 A, unsigned long long* rate,
                                               const int4* __restrict__ segs) {
  const int4 g = segs[blockIdx.x];
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  float r = 0.f;
  if (threadIdx.x < g.w)
    r = cfl_rate_of<DIM>(F, cons_to_prim32<DIM, RX>(P, F, A.src, A.T, cidx(pd, i, j)), 1.f / (float)pd.dx,
                         1.f / (float)pd.dy, A.status, g.x, i + pd.nx * j);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0 && r > 0.f)
    atomicMax(rate + g.x, (unsigned long long)__double_as_longlong((double)r));
}

// Persistent 1D batch kernel: CTA b owns problem order[b] (the problems sorted
// by length, longest first, so the block scheduler balances them) and runs
// n_steps whole time steps of it in one launch: the three stages, each over
// the problem's tiles tiles[tile0[p] .. tile0[p + 1]) in turn, with the
// buffer rotation of the per-step path (0 -> 1 -> 2 -> 0).  The CFL rate of
// q^n is rate[p] (computed here first when rate_ready is 0); the last stage
// of every step leaves the rate of the new state in shared memory for the
// next one, and the final rate goes back to rate[p].  A problem's three state
// buffers stay in L2 between stages and steps.  The tile arithmetic is
// stage32_tile's; compiled as another kernel, its multiply-add contractions
// may differ, so the result matches the per-step launches to rounding.
// scratch_last (tuning, n_steps = 1): the last stage writes buffer 1.
struct Bufs32 {
  float* q[3];
};

template <bool RX, int TX, int NT, int MINB, bool CYL = false, int LIM = 0, bool GEN = false>
__global__ void __launch_bounds__(NT, MINB) k_batch32(Phys P, PhysF F, StepArgs32 A, Bufs32 B,
                                                      unsigned long long* rate, const int* __restrict__ order,
                                                      const int* __restrict__ tile0,
                                                      const int4* __restrict__ tiles, int n_steps,
                                                      int scratch_last, int rate_ready) {
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
    if (threadIdx.x == 0) rnext = 0u;  // ordered before the last stage's atomics by the tile barriers
    for (int stg = 0; stg < 3; ++stg) {
      StepArgs32 a = A;
      const bool s0 = stg == 0, s1 = stg == 1, to1 = s0 || (!s1 && scratch_last);
      a.src = B.q[stg];
      a.qn = B.q[0];
      a.dst = to1 ? B.q[1] : (s1 ? B.q[2] : B.q[0]);
      a.rate = rate;
      a.a = s0 ? 0.0 : (s1 ? 0.75 : 1.0 / 3.0);
      a.b = s0 ? 1.0 : (s1 ? 0.25 : 2.0 / 3.0);
      a.last = stg == 2;
      for (int t = ta; t < tb; ++t) {
        stage32_tile<1, RX, TX, 1, NT, CYL, LIM, GEN>(P, F, a, tiles[t], sm, &rnext);
        __syncthreads();
      }
    }
    // the next step's rate (thread 0 also reads it, for dt, in the next tile)
    if (threadIdx.x == 0 && !scratch_last)
      rate[p] = (unsigned long long)__double_as_longlong((double)__uint_as_float(rnext));
  }
}

}  // namespace dis
