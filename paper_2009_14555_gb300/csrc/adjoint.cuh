// adjoint.cuh - reverse-mode kernels of the float64 step (sm_103a).
//
// The step is q^{n+1} = S(o3), o_k = a_k q^n + b_k (x_k - dt D(x_k)) with the
// SSP-RK3 coefficients (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3) and S the
// plastic + reactive source steps; dt is frozen (recorded by the forward run).
// D(x) = sum_d (F_{i+1/2} - F_{i-1/2}) / h_d - N(x, face extras), where the
// face outputs F come from primitives W(x) of a 6-cell stencil.
//
// Reverse of one stage, given the adjoint obar of its output:
//   k_adj_cell  (per cell)   source-step adjoint (last stage), qn_acc += a obar,
//                            xbar = b obar + (dN/dx)^T, and the per-cell
//                            coefficients G = (Dbar, Nbar) that the two faces
//                            of each direction share;
//   k_adj_face  (per face)   Fbar = (G_left - G_right) / h, then the
//                            vector-Jacobian product through the Riemann solver
//                            and the reconstruction into Wbar (atomics: a cell
//                            is in the stencil of up to 6 faces per direction);
//   k_adj_prim  (per padded cell, ghosts included) Wbar -> xbar of the source
//                            cell of the ghost map (sign flips of reflective
//                            walls applied), again by atomics.
// Local Jacobians are never formed.  Every local map - the Riemann problem of
// a face, the map from face primitives to face states, the THINC-BVD edge
// values of phi, the recovery of primitives and the source steps - is
// reversed by hand (local_vjp.cuh).  REF = true instantiates the reference
// form instead: each map reversed one input direction at a time by a
// Dual-number evaluation of the forward code (face.cuh), contracted with the
// adjoint (the reference the hand-written reverses are tested against).
#pragma once
#include "local_vjp.cuh"
#include "step_kernels.cuh"
#include "step32.cuh"

namespace dis {

constexpr int NPARAM = 6;  // per material l: G_l, sigma_y_l, Q_l at 3 l + {0, 1, 2}

// Closure parameters as Dual numbers with the derivative along parameter k
// (-1: none).  Derived constants follow their definitions:
//   gG = gamma G / (gamma - 1), GoG = G / (gamma - 1), JY = sigma_y / (sqrt(6) G).
__device__ __forceinline__ PhysT<Dual> lift_phys(const Phys& P, int k) {
  PhysT<Dual> D;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const MatDev& m = P.m[l];
    MatT<Dual>& d = D.m[l];
    d.gamma = m.gamma; d.pinf = m.pinf; d.einf = m.einf; d.G = m.G; d.sigy = m.sigy;
    d.chi0 = m.chi0; d.Q = m.Q; d.cv = m.cv; d.A = m.A; d.Tact = m.Tact;
    d.plastic = m.plastic; d.reactive = m.reactive; d.law = m.law; d.pign = m.pign;
    d.iGm1 = m.iGm1; d.gi = m.gi; d.kap = m.kap; d.gG = m.gG; d.GoG = m.GoG; d.JY = m.JY;
    d.eos = m.eos; d.rho0 = m.rho0; d.K0 = m.K0; d.ar = m.ar; d.br = m.br;
    d.jA = m.jA; d.jB = m.jB; d.jR1 = m.jR1; d.jR2 = m.jR2;
    d.two = m.two; d.pg = m.pg; d.ppi = m.ppi; d.pcv = m.pcv;
  }
  D.y = P.y;
  D.thinc = P.thinc;
  D.cfl = P.cfl;
  D.cyl = P.cyl;
  D.limiter = P.limiter;
  if (k >= 0) {
    const int l = k / 3, kind = k % 3;
    const MatDev& m = P.m[l];
    MatT<Dual>& d = D.m[l];
    const bool finite_JY = m.plastic && m.G > 0.0;
    if (kind == 0) {
      d.G.d = 1.0;
      d.gG.d = m.gi;
      d.GoG.d = m.iGm1;
      if (finite_JY) d.JY.d = -m.JY / m.G;
    } else if (kind == 1) {
      d.sigy.d = 1.0;
      if (finite_JY) d.JY.d = 1.0 / (sqrt(6.0) * m.G);
    } else {
      d.Q.d = 1.0;
    }
  }
  return D;
}

__device__ __forceinline__ PrimT<Dual> lift_prim(const Prim& w) {
  PrimT<Dual> d;
  d.phi = w.phi; d.r1 = w.r1; d.r2 = w.r2; d.u = w.u; d.v = w.v; d.p = w.p;
  d.V11 = w.V11; d.V12 = w.V12; d.V21 = w.V21; d.V22 = w.V22; d.V33 = w.V33; d.lam = w.lam;
  return d;
}

// Sum the per-thread parameter adjoints of a warp and add them to theta.
__device__ __forceinline__ void flush_theta(double (&th)[NPARAM], double* theta, unsigned pmask) {
#pragma unroll
  for (int k = 0; k < NPARAM; ++k) {
    if (!((pmask >> k) & 1u)) continue;
    double v = th[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(theta + k, v);
  }
}

__device__ __forceinline__ void add_nz(double* p, double v) {
  if (v != 0.0) atomicAdd(p, v);
}

struct AdjArgs {
  const PatchDev* pd;
  long long T, NFX, NFY;
  const double* x;     // stage input (padded)
  const double* W;     // primitives of x (padded, ghost cells filled)
  const double* Fx;    // face outputs of x
  const double* Fy;
  const double* obar;  // adjoint of the stage output
  const double* opre;  // last stage: stage output before the source steps
  double* xbar;        // adjoint of x (written by k_adj_cell, accumulated by k_adj_prim)
  double* qnacc;       // accumulated adjoint of q^n
  double* G;           // per-cell face coefficients, NF + NX_EXTRA planes
  double* Wbar;        // adjoint of W, NF planes (zeroed before k_adj_cell)
  double* theta;       // parameter adjoints [NPARAM]
  const double* dt;    // per-patch dt of the step
  double a, b;
  int last;
  int first;           // qnacc = a obar (else +=)
  unsigned pmask;      // parameters to differentiate
};

// <a, b.d> over the fields of two face states.
__device__ __forceinline__ double fstate_dot(const FState& a, const FStateT<Dual>& b) {
  return a.phi * b.phi.d + a.ar1 * b.ar1.d + a.ar2 * b.ar2.d + a.arl * b.arl.d + a.rho * b.rho.d +
         a.un * b.un.d + a.ut * b.ut.d + a.rhoE * b.rhoE.d + a.snn * b.snn.d + a.snt * b.snt.d +
         a.cL * b.cL.d + a.Gm * b.Gm.d + a.V11 * b.V11.d + a.V12 * b.V12.d + a.V21 * b.V21.d +
         a.V22 * b.V22.d + a.V33 * b.V33.d;
}

// ---------------------------------------------------------------------------
// Per interior cell: source-step adjoint, RK combination, non-conservative
// terms; writes xbar (direct part), qnacc and the face coefficients G.
// ---------------------------------------------------------------------------
template <int DIM, bool RX, bool REF>
__global__ void __launch_bounds__(SEG) k_adj_cell(Phys P, AdjArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  constexpr int NE = L::NX_EXTRA;
  const int4 g = segs[blockIdx.x];
  double th[NPARAM];
#pragma unroll
  for (int k = 0; k < NPARAM; ++k) th[k] = 0.0;
  if (threadIdx.x < g.w) {
    const PatchDev pd = A.pd[g.x];
    const int i = g.z + threadIdx.x, j = g.y;
    const long long k = cidx(pd, i, j);
    const long long T = A.T;
    const double dt = A.dt[g.x];
    double ob[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) ob[c] = A.obar[c * T + k];
    if constexpr (!REF) {
      if (A.last) {
        // adjoint of the source steps about the pre-source state (by hand)
        double op[NF], thp[NPARAM] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int c = 0; c < NF; ++c) op[c] = A.opre[c * T + k];
        sources_vjp<DIM, RX>(P, dt, op, ob, thp);
#pragma unroll
        for (int kk = 0; kk < NPARAM; ++kk)
          if ((A.pmask >> kk) & 1u) th[kk] += thp[kk];
      }
    } else if (A.last) {
      // the same with dual numbers (reference form)
      double op[NF], nb[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) op[c] = A.opre[c * T + k];
      const PhysT<Dual> PD = lift_phys(P, -1);
#pragma unroll 1
      for (int s = 0; s < NF; ++s) {
        Dual o[NF];
#pragma unroll
        for (int c = 0; c < NF; ++c) o[c] = Dual(op[c], c == s ? 1.0 : 0.0);
        sources<DIM, RX, Dual>(PD, dt, o);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < NF; ++c) acc += ob[c] * o[c].d;
        nb[s] = acc;
      }
#pragma unroll 1
      for (int kk = 0; kk < NPARAM; ++kk) {
        if (!((A.pmask >> kk) & 1u)) continue;
        const PhysT<Dual> PK = lift_phys(P, kk);
        Dual o[NF];
#pragma unroll
        for (int c = 0; c < NF; ++c) o[c] = Dual(op[c]);
        sources<DIM, RX, Dual>(PK, dt, o);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < NF; ++c) acc += ob[c] * o[c].d;
        th[kk] += acc;
      }
#pragma unroll
      for (int c = 0; c < NF; ++c) ob[c] = nb[c];
    }
    if (A.a != 0.0) {
#pragma unroll
      for (int c = 0; c < NF; ++c) {
        const double v = A.a * ob[c];
        A.qnacc[c * T + k] = A.first ? v : A.qnacc[c * T + k] + v;
      }
    }
    // forward quantities of the non-conservative terms at this cell
    double q[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) q[c] = A.x[c * T + k];
    const double idx_ = 1.0 / pd.dx;
    const long long fl = pd.fxoff + (long long)j * (pd.nx + 1) + i;
    const long long NFX = A.NFX;
    double divu = (A.Fx[NF * NFX + fl + 1] - A.Fx[NF * NFX + fl]) * idx_;
    double bx = (A.Fx[(NF + 1) * NFX + fl + 1] - A.Fx[(NF + 1) * NFX + fl]) * idx_;
    double by = 0.0;
    if constexpr (DIM == 2) {
      by = (A.Fx[(NF + 2) * NFX + fl + 1] - A.Fx[(NF + 2) * NFX + fl]) * idx_;
      const double idy = 1.0 / pd.dy;
      const long long NFY = A.NFY;
      const long long fb = pd.fyoff + (long long)j * pd.nx + i;
      const long long ft = fb + pd.nx;
      divu += (A.Fy[NF * NFY + ft] - A.Fy[NF * NFY + fb]) * idy;
      bx += (A.Fy[(NF + 1) * NFY + ft] - A.Fy[(NF + 1) * NFY + fb]) * idy;
      by += (A.Fy[(NF + 2) * NFY + ft] - A.Fy[(NF + 2) * NFY + fb]) * idy;
    }
    const double rho = q[L::A1] + q[L::A2];
    const double uc = q[L::MX] / rho;
    double vc = 0.0;
    if constexpr (DIM == 2) vc = q[L::MY] / rho;
    const double t23 = 2.0 / 3.0;
    // o = a qn + b (x - dt D(x)):  xbar = b obar - dt b (dD/dx)^T obar
    double xb[NF], Db[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      xb[c] = A.b * ob[c];
      Db[c] = -dt * xb[c];
    }
    // D_phi -= phi divu;  D_Vij -= 2/3 V_ij divu - (u_c or v_c)(bx or by)
    double gdiv = -Db[L::PHI] * q[L::PHI];
    gdiv -= t23 * (Db[L::V11] * q[L::V11] + Db[L::V22] * q[L::V22] + Db[L::V33] * q[L::V33]);
    double gbx = Db[L::V11] * uc;
    double gby = 0.0;
    double ub = Db[L::V11] * bx;
    double vb = 0.0;
    xb[L::PHI] -= Db[L::PHI] * divu;
    xb[L::V11] -= t23 * Db[L::V11] * divu;
    xb[L::V22] -= t23 * Db[L::V22] * divu;
    xb[L::V33] -= t23 * Db[L::V33] * divu;
    if constexpr (DIM == 2) {
      gdiv -= t23 * (Db[L::V12] * q[L::V12] + Db[L::V21] * q[L::V21]);
      gbx += Db[L::V21] * vc;
      gby = Db[L::V22] * vc + Db[L::V12] * uc;
      ub += Db[L::V12] * by;
      vb = Db[L::V22] * by + Db[L::V21] * bx;
      xb[L::V12] -= t23 * Db[L::V12] * divu;
      xb[L::V21] -= t23 * Db[L::V21] * divu;
    }
    // u_c = mx / rho, v_c = my / rho, rho = ar1 + ar2
    xb[L::MX] += ub / rho;
    double rb = -ub * uc / rho;
    if constexpr (DIM == 2) {
      xb[L::MY] += vb / rho;
      rb -= vb * vc / rho;
    }
    xb[L::A1] += rb;
    xb[L::A2] += rb;
    if (P.cyl) {
      // geometric source: into xbar and into Wbar of this cell (zeroed
      // before this kernel; the face kernels add to it afterwards)
      Prim wb{};
      double thg[NPARAM] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      geometric_vjp<DIM, RX>(P, q, load_prim<DIM, RX>(A.W, T, k), pd.x0 + (i + 0.5) * pd.dx, Db, xb, wb, thg);
#pragma unroll
      for (int c = 0; c < NF; ++c) A.Wbar[c * T + k] = prim_slot<DIM, RX>(wb, c);
#pragma unroll
      for (int kk = 0; kk < NPARAM; ++kk)
        if ((A.pmask >> kk) & 1u) th[kk] += thg[kk];
    }
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      A.xbar[c * T + k] = xb[c];
      A.G[c * T + k] = Db[c];
    }
    A.G[NF * T + k] = gdiv;
    A.G[(NF + 1) * T + k] = gbx;
    if constexpr (NE > 2) A.G[(NF + 2) * T + k] = gby;
  }
  flush_theta(th, A.theta, A.pmask);
}

// ---------------------------------------------------------------------------
// Per face: adjoint of the face outputs, then back through the Riemann solver,
// the non-hyperbolic fallback and the reconstruction into Wbar.
// ---------------------------------------------------------------------------
template <int DIM, bool RX, int DIR, bool REF>
__global__ void __launch_bounds__(SEG) k_adj_face(Phys P, AdjArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  constexpr int NO = n_face_out<DIM, RX>();
  const int4 g = segs[blockIdx.x];
  double th[NPARAM];
#pragma unroll
  for (int k = 0; k < NPARAM; ++k) th[k] = 0.0;
  bool active = threadIdx.x < g.w;
  const PatchDev pd = A.pd[g.x];
  const long long T = A.T;
  const int f = (DIR == 0 ? g.z : g.y) + (DIR == 0 ? (int)threadIdx.x : 0);
  const int col = DIR == 0 ? g.y : g.z + (int)threadIdx.x;
  const int a = (DIR == 0 ? f : g.y) - 1;
  const int n = DIR == 0 ? pd.nx : pd.ny;
  auto at = [&](int s) -> long long { return DIR == 0 ? cidx(pd, s, col) : cidx(pd, col, s); };
  const double h = DIR == 0 ? pd.dx : pd.dy;
  double Fb[NO];
  if (active) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < NO; ++c) {
      const double gl = a >= 0 ? A.G[c * T + at(a)] : 0.0;
      const double gr = a + 1 < n ? A.G[c * T + at(a + 1)] : 0.0;
      Fb[c] = (gl - gr) / h;
      any |= Fb[c] != 0.0;
    }
    active = any;
  }
  if (active) {
    const double* __restrict__ W = A.W;
    const long long stride_t = DIR == 0 ? (long long)pd.pitch : 1;
    const bool normals = DIM == 2 && P.thinc;
    const double hn = DIR == 0 ? pd.dx : pd.dy, ht = DIR == 0 ? pd.dy : pd.dx;
    // phi stencil of the face (line a-2 .. a+3 and, for the Youngs normal, the
    // neighbouring lines); loaded again where the reverse needs it
    auto load_B = [&](double (&B)[3][6]) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        B[1][c] = W[L::PHI * T + at(a - 2 + c)];
        B[0][c] = normals ? W[L::PHI * T + at(a - 2 + c) - stride_t] : 0.0;
        B[2][c] = normals ? W[L::PHI * T + at(a - 2 + c) + stride_t] : 0.0;
      }
    };
    // forward reconstruction: the two face states the Riemann solver saw
    Prim pl, pr;
    FState fsl, fsr;  // their face states, as the forward Riemann solver saw them
    bool okL, okR;
    {
      double B[3][6];
      load_B(B);
      double phiL, phiR;
      face_phi<DIM, double>(B, P.thinc != 0, hn, ht, phiL, phiR, P.limiter);
      Prim w[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) w[s] = load_prim<DIM, RX>(W, T, at(a - 1 + s));
      Prim wl, wr;
#pragma unroll
      for (int c = 0; c < NF; ++c) {
        if (c == L::PHI) continue;
        muscl_pair(prim_slot<DIM, RX>(w[0], c), prim_slot<DIM, RX>(w[1], c), prim_slot<DIM, RX>(w[2], c),
                   prim_slot<DIM, RX>(w[3], c), prim_slot<DIM, RX>(wl, c), prim_slot<DIM, RX>(wr, c), P.limiter);
      }
      if constexpr (DIM == 1) {
        wl.v = wr.v = 0.0;
        wl.V12 = wr.V12 = wl.V21 = wr.V21 = 0.0;
      }
      if constexpr (!RX) wl.lam = wr.lam = 0.0;
      wl.phi = phiL;
      wr.phi = phiR;
      fsl = face_state<DIR>(P, wl);
      fsr = face_state<DIR>(P, wr);
      okL = fsl.cL > 0.0;
      okR = fsr.cL > 0.0;
      pl = okL ? wl : w[1];
      pr = okR ? wr : w[2];
      if (!okL) fsl = face_state<DIR>(P, pl);
      if (!okR) fsr = face_state<DIR>(P, pr);
    }

    // Riemann solver: gradient with respect to the two chosen face states
    double gL[NF], gR[NF];
    if constexpr (!REF) {
      // hand-written reverse of the Riemann problem into the face states, then
      // of the face-state map (primitives -> face state)
      FState Lb{}, Rb{};
      riemann_outputs_vjp<DIM, RX, DIR>(fsl, fsr, Fb, Lb, Rb);
      Prim pbL{}, pbR{};
      double thf[NPARAM] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      face_state_vjp<DIR>(P, pl, Lb, pbL, thf);
      face_state_vjp<DIR>(P, pr, Rb, pbR, thf);
#pragma unroll
      for (int c = 0; c < NF; ++c) {
        gL[c] = prim_slot<DIM, RX>(pbL, c);
        gR[c] = prim_slot<DIM, RX>(pbR, c);
      }
#pragma unroll
      for (int kk = 0; kk < NPARAM; ++kk)
        if ((A.pmask >> kk) & 1u) th[kk] += thf[kk];
    } else {
      const PhysT<Dual> PD = lift_phys(P, -1);
#pragma unroll 1
      for (int s = 0; s < 2 * NF; ++s) {
        PrimT<Dual> dl = lift_prim(pl), dr = lift_prim(pr);
        if (s < NF) prim_slot<DIM, RX>(dl, s).d = 1.0;
        else prim_slot<DIM, RX>(dr, s - NF).d = 1.0;
        Dual out[NO];
        riemann_outputs<DIM, RX, DIR>(face_state<DIR>(PD, dl), face_state<DIR>(PD, dr), out);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < NO; ++c) acc += Fb[c] * out[c].d;
        if (s < NF) gL[s] = acc;
        else gR[s - NF] = acc;
      }
#pragma unroll 1
      for (int kk = 0; kk < NPARAM; ++kk) {
        if (!((A.pmask >> kk) & 1u)) continue;
        const PhysT<Dual> PK = lift_phys(P, kk);
        Dual out[NO];
        riemann_outputs<DIM, RX, DIR>(face_state<DIR>(PK, lift_prim(pl)), face_state<DIR>(PK, lift_prim(pr)), out);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < NO; ++c) acc += Fb[c] * out[c].d;
        th[kk] += acc;
      }
    }

    // reconstruction of the fields other than phi (or the fallback)
    double wb[4][NF];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < NF; ++c) wb[s][c] = 0.0;
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      if (c == L::PHI) continue;
      const double v0 = W[c * T + at(a - 1)], v1 = W[c * T + at(a)];
      const double v2 = W[c * T + at(a + 1)], v3 = W[c * T + at(a + 2)];
      if (okL) {  // wl = w1 + lim(w1 - w0, w2 - w1) / 2
        double da, db;
        limiter_grad(v1 - v0, v2 - v1, P.limiter, da, db);
        wb[0][c] += gL[c] * (-0.5 * da);
        wb[1][c] += gL[c] * (1.0 + 0.5 * (da - db));
        wb[2][c] += gL[c] * (0.5 * db);
      } else {
        wb[1][c] += gL[c];
      }
      if (okR) {  // wr = w2 - lim(w2 - w1, w3 - w2) / 2
        double da, db;
        limiter_grad(v2 - v1, v3 - v2, P.limiter, da, db);
        wb[1][c] += gR[c] * (0.5 * da);
        wb[2][c] += gR[c] * (1.0 - 0.5 * (da - db));
        wb[3][c] += gR[c] * (-0.5 * db);
      } else {
        wb[2][c] += gR[c];
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < NF; ++c)
        if (c != L::PHI) add_nz(A.Wbar + c * T + at(a - 1 + s), wb[s][c]);

    // phi: fallback sides take the cell value; reconstructed sides go back
    // through the THINC-BVD edge values (and the Youngs normals in 2D)
    const double gpL = okL ? gL[L::PHI] : 0.0, gpR = okR ? gR[L::PHI] : 0.0;
    if (!okL) add_nz(A.Wbar + L::PHI * T + at(a), gL[L::PHI]);
    if (!okR) add_nz(A.Wbar + L::PHI * T + at(a + 1), gR[L::PHI]);
    if ((gpL != 0.0 || gpR != 0.0) && !REF) {
      double B[3][6], Bb[3][6];
      load_B(B);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) Bb[r][c] = 0.0;
      face_phi_vjp<DIM>(B, P.thinc != 0, hn, ht, gpL, gpR, Bb, P.limiter);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!normals && r != 1) continue;
#pragma unroll
        for (int c = 0; c < 6; ++c)
          add_nz(A.Wbar + L::PHI * T + at(a - 2 + c) + (long long)(r - 1) * stride_t, Bb[r][c]);
      }
    } else if (REF && (gpL != 0.0 || gpR != 0.0)) {
      double B[3][6];
      load_B(B);
      const int r0 = normals ? 0 : 1, r1 = normals ? 2 : 1;
#pragma unroll 1
      for (int r = r0; r <= r1; ++r) {
#pragma unroll 1
        for (int c = 0; c < 6; ++c) {
          Dual Bd[3][6];
#pragma unroll
          for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) Bd[rr][cc] = Dual(B[rr][cc], (rr == r && cc == c) ? 1.0 : 0.0);
          Dual pL, pR;
          face_phi<DIM, Dual>(Bd, P.thinc != 0, hn, ht, pL, pR, P.limiter);
          const double v = gpL * pL.d + gpR * pR.d;
          add_nz(A.Wbar + L::PHI * T + at(a - 2 + c) + (long long)(r - 1) * stride_t, v);
        }
      }
    }
  }
  flush_theta(th, A.theta, A.pmask);
}

// ---------------------------------------------------------------------------
// Per padded cell (ghosts by the index map): Wbar -> xbar of the source cell.
// ---------------------------------------------------------------------------
template <int DIM, bool RX, bool REF>
__global__ void __launch_bounds__(SEG) k_adj_prim(Phys P, AdjArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  double th[NPARAM];
#pragma unroll
  for (int k = 0; k < NPARAM; ++k) th[k] = 0.0;
  if (threadIdx.x < g.w) {
    const PatchDev pd = A.pd[g.x];
    const int i = g.z + threadIdx.x;
    const int j = g.y;
    const long long T = A.T;
    const long long kc = cidx(pd, i, j);
    double wb[NF];
    bool any = false;
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      wb[c] = A.Wbar[c * T + kc];
      any |= wb[c] != 0.0;
    }
    if (any) {
      bool fx = false, fy = false;
      const int si = ghost_map(i, pd.nx, pd.bc[0], pd.bc[1], fx);
      const int sj = DIM == 2 ? ghost_map(j, pd.ny, pd.bc[2], pd.bc[3], fy) : 0;
      const long long ks = cidx(pd, si, sj);
      // the reflective copy negates u, V12, V21 (x walls) or v, V12, V21 (y walls)
      if (fx) {
        wb[L::MX] = -wb[L::MX];
        if constexpr (DIM == 2) { wb[L::V12] = -wb[L::V12]; wb[L::V21] = -wb[L::V21]; }
      }
      if constexpr (DIM == 2) {
        if (fy) { wb[L::MY] = -wb[L::MY]; wb[L::V12] = -wb[L::V12]; wb[L::V21] = -wb[L::V21]; }
      }
      double q[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) q[c] = A.x[c * T + ks];
      if constexpr (!REF) {
        Prim w{};
#pragma unroll
        for (int c = 0; c < NF; ++c) prim_slot<DIM, RX>(w, c) = wb[c];
        double qb[NF], thp[NPARAM] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int c = 0; c < NF; ++c) qb[c] = 0.0;
        prim_of_vjp<DIM, RX>(P, q, w, qb, thp);
#pragma unroll
        for (int c = 0; c < NF; ++c) add_nz(A.xbar + c * T + ks, qb[c]);
#pragma unroll
        for (int kk = 0; kk < NPARAM; ++kk)
          if ((A.pmask >> kk) & 1u) th[kk] += thp[kk];
      } else {
        const PhysT<Dual> PD = lift_phys(P, -1);
#pragma unroll 1
        for (int s = 0; s < NF; ++s) {
          Dual qd[NF];
#pragma unroll
          for (int c = 0; c < NF; ++c) qd[c] = Dual(q[c], c == s ? 1.0 : 0.0);
          PrimT<Dual> w = prim_of<DIM, RX, Dual>(PD, qd);
          double acc = 0.0;
#pragma unroll
          for (int c = 0; c < NF; ++c) acc += wb[c] * prim_slot<DIM, RX>(w, c).d;
          add_nz(A.xbar + s * T + ks, acc);
        }
#pragma unroll 1
        for (int kk = 0; kk < NPARAM; ++kk) {
          if (!((A.pmask >> kk) & 1u)) continue;
          const PhysT<Dual> PK = lift_phys(P, kk);
          Dual qd[NF];
#pragma unroll
          for (int c = 0; c < NF; ++c) qd[c] = Dual(q[c]);
          PrimT<Dual> w = prim_of<DIM, RX, Dual>(PK, qd);
          double acc = 0.0;
#pragma unroll
          for (int c = 0; c < NF; ++c) acc += wb[c] * prim_slot<DIM, RX>(w, c).d;
          th[kk] += acc;
        }
      }
    }
  }
  flush_theta(th, A.theta, A.pmask);
}

// ---------------------------------------------------------------------------
// Running objective J = sum_steps dt sum_cells phi_l (rho u) dA (material l):
// value (forward) and its injection into the adjoint of q^{n+1}.
// ---------------------------------------------------------------------------
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_obj(const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                                            const double* q, long long T, const double* dt, int mat,
                                            double* J) {
  using L = Lay<DIM, RX>;
  const int4 g = segs[blockIdx.x];
  double v = 0.0;
  if (threadIdx.x < g.w) {
    const PatchDev pd = pds[g.x];
    const long long k = cidx(pd, g.z + threadIdx.x, g.y);
    const double phi = q[L::PHI * T + k];
    const double ph = mat == 0 ? phi : 1.0 - phi;
    v = dt[g.x] * pd.dx * pd.dy * ph * q[L::MX * T + k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(J, v);
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_obj_adj(const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                                                const double* q, double* qbar, long long T, const double* dt,
                                                int mat, double jbar) {
  using L = Lay<DIM, RX>;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const long long k = cidx(pd, g.z + threadIdx.x, g.y);
  const double s = jbar * dt[g.x] * pd.dx * pd.dy;
  const double phi = q[L::PHI * T + k];
  const double ph = mat == 0 ? phi : 1.0 - phi;
  qbar[L::PHI * T + k] += s * (mat == 0 ? 1.0 : -1.0) * q[L::MX * T + k];
  qbar[L::MX * T + k] += s * ph;
}

// FP32-bulk state (float32 planes with the soft energy and the float-float
// phi1 of step32.cuh) to the float64 layout of the same padded cells
// (interior cells).
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_state32_to_64(Phys P, const PatchDev* __restrict__ pds,
                                                      const int4* __restrict__ segs, const float* q32, double* out,
                                                      long long T) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const long long k = cidx(pd, g.z + threadIdx.x, g.y);
  double v[NF];
  state32_to_64<DIM, RX>(P, q32, T, k, v);
#pragma unroll
  for (int c = 0; c < NF; ++c) out[c * T + k] = v[c];
}

// qbar = xbar + qnacc on interior cells.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_adj_sum(const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                                                const double* xb, const double* acc, double* out, long long T) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const long long k = cidx(pd, g.z + threadIdx.x, g.y);
#pragma unroll
  for (int c = 0; c < NF; ++c) out[c * T + k] = xb[c * T + k] + acc[c * T + k];
}

// Adjoint of the primitive -> conservative conversion of the initial state:
// wbar = (dq/dw)^T qbar at the primitives W (interior cells, packed output),
// plus the parameter adjoints of the conversion.
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_adj_p2c(Phys P, const PatchDev* __restrict__ pds,
                                                const int4* __restrict__ segs, const double* W,
                                                const double* qbar, double* wbar_packed, long long T,
                                                double* theta, unsigned pmask) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  double th[NPARAM];
#pragma unroll
  for (int k = 0; k < NPARAM; ++k) th[k] = 0.0;
  if (threadIdx.x < g.w) {
    const PatchDev pd = pds[g.x];
    const int i = g.z + threadIdx.x, j = g.y;
    const long long k = cidx(pd, i, j);
    const long long ncell = (long long)pd.nx * pd.ny;
    const long long s0 = pd.poff + (long long)j * pd.nx + i;
    double w[NF], qb[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      w[c] = W[c * T + k];
      qb[c] = qbar[c * T + k];
    }
    const PhysT<Dual> PD = lift_phys(P, -1);
#pragma unroll 1
    for (int s = 0; s < NF; ++s) {
      Dual v[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) v[c] = Dual(w[c], c == s ? 1.0 : 0.0);
      cons_of<DIM, RX, Dual>(PD, v);
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < NF; ++c) acc += qb[c] * v[c].d;
      wbar_packed[s0 + s * ncell] = acc;
    }
#pragma unroll 1
    for (int kk = 0; kk < NPARAM; ++kk) {
      if (!((pmask >> kk) & 1u)) continue;
      const PhysT<Dual> PK = lift_phys(P, kk);
      Dual v[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) v[c] = Dual(w[c]);
      cons_of<DIM, RX, Dual>(PK, v);
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < NF; ++c) acc += qb[c] * v[c].d;
      th[kk] += acc;
    }
  }
  flush_theta(th, theta, pmask);
}

}  // namespace dis
