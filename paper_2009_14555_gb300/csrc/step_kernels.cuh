// step_kernels.cuh - kernels of one SSP-RK3 stage and the source steps (sm_103a).
//
// Data layout in HBM: every conservative or primitive field is one plane of
// T float64 values holding all patches back to back; a patch occupies
// (ny + 2 NG) rows (1 row in 1D) of pitch nx + 2 NG cells, ghost cells
// included, starting at a 32-element aligned offset.  Face data are planes of
// per-face values (x faces: ny rows of nx + 1; y faces: ny + 1 rows of nx).
//
// Work is described by host-built segment tables: one CTA of 128 threads per
// segment = (patch, row, first index, count), so every launch covers any
// batch of uneven patches and accesses are unit-stride along x.
#pragma once
#include "physics.cuh"

namespace dis {

constexpr int SEG = 128;

struct PatchDev {
  int nx, ny, pitch, rows;
  int bc[4];
  long long off;    // first padded cell of the patch in a field plane
  long long fxoff;  // first x face
  long long fyoff;  // first y face
  long long poff;   // first cell in the packed (interior-only) layout
  double dx, dy;
};

struct StepArgs {
  const PatchDev* pd;
  long long T, NFX, NFY;
  const double* qsrc;
  const double* qn;
  double* qdst;
  double* W;
  double* Fx;
  double* Fy;
  unsigned long long* rate;  // per-patch max CFL rate (bit pattern of a positive double)
  const double* dtfix;       // per-patch prescribed dt, or null
  double* dtlast;
  int* status;               // [flag, patch, cell]
  double a, b;               // q_dst = a q_n + b (q_src - dt D(q_src)), a = 0 -> no q_n
  int last;                  // apply plastic and reactive steps, record dt
};

__device__ __forceinline__ long long cidx(const PatchDev& p, int i, int j) {
  return p.off + (long long)(j + (p.rows > 1 ? NG : 0)) * p.pitch + (i + NG);
}

// Ghost index map of one axis: returns the source index and whether the
// reflective boundary flips this axis' normal velocity.
__device__ __forceinline__ int ghost_map(int i, int n, int bclo, int bchi, bool& flip) {
  if (i < 0) {
    if (bclo == 1) return i + n;
    if (bclo == 2) { flip = !flip; return -1 - i; }
    return 0;
  }
  if (i >= n) {
    if (bchi == 1) return i - n;
    if (bchi == 2) { flip = !flip; return 2 * n - 1 - i; }
    return n - 1;
  }
  return i;
}

template <int DIM, bool RX>
__device__ __forceinline__ Prim cons_to_prim(const Phys& P, const double* q, long long T, long long k) {
  using L = Lay<DIM, RX>;
  Prim w;
  const double phi = q[L::PHI * T + k], a1 = q[L::A1 * T + k], a2 = q[L::A2 * T + k];
  const double rho = a1 + a2;
  const double mx = q[L::MX * T + k];
  double my = 0.0;
  if constexpr (DIM == 2) my = q[L::MY * T + k];
  const double E = q[L::E * T + k];
  w.phi = phi;
  w.r1 = a1 / phi;
  w.r2 = a2 / (1.0 - phi);
  w.u = mx / rho;
  w.v = my / rho;
  w.V11 = q[L::V11 * T + k];
  w.V12 = 0.0;
  w.V21 = 0.0;
  if constexpr (DIM == 2) {
    w.V12 = q[L::V12 * T + k];
    w.V21 = q[L::V21 * T + k];
  }
  w.V22 = q[L::V22 * T + k];
  w.V33 = q[L::V33 * T + k];
  double arl = 0.0;
  w.lam = 0.0;
  if constexpr (RX) {
    arl = q[L::AL * T + k];
    w.lam = arl / (P.y == 0 ? a1 : a2);
  }
  const Strain s = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const double KE = 0.5 * (mx * w.u + my * w.v);
  w.p = (E - KE - ref_energy(P, phi, a1, a2, arl, s.J2)) / xi_of(P, phi);
  return w;
}

template <int DIM, bool RX>
__device__ __forceinline__ void store_prim(double* W, long long T, long long k, const Prim& w) {
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
__device__ __forceinline__ Prim load_prim(const double* __restrict__ W, long long T, long long k) {
  using L = Lay<DIM, RX>;
  Prim w;
  w.phi = W[L::PHI * T + k];
  w.r1 = W[L::A1 * T + k];
  w.r2 = W[L::A2 * T + k];
  w.u = W[L::MX * T + k];
  w.v = 0.0;
  w.V12 = 0.0;
  w.V21 = 0.0;
  w.lam = 0.0;
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

__device__ __forceinline__ void flag_bad(int* status, int patch, int cell) {
  if (atomicCAS(status, 0, 1) == 0) {
    status[1] = patch;
    status[2] = cell;
  }
}

// ---------------------------------------------------------------------------
// Primitive recovery on every padded cell (ghosts by index map), and the
// per-patch CFL rate max over interior cells when `rate_on`.
// ---------------------------------------------------------------------------
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_prim(Phys P, StepArgs A, const int4* __restrict__ segs,
                                              int rate_on) {
  const int4 g = segs[blockIdx.x];
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x;
  const int j = g.y;
  const bool valid = threadIdx.x < g.w;
  double r = 0.0;
  if (valid) {
    bool fx = false, fy = false;
    const int si = ghost_map(i, pd.nx, pd.bc[0], pd.bc[1], fx);
    const int sj = DIM == 2 ? ghost_map(j, pd.ny, pd.bc[2], pd.bc[3], fy) : 0;
    Prim w = cons_to_prim<DIM, RX>(P, A.qsrc, A.T, cidx(pd, si, sj));
    if (fx) { w.u = -w.u; w.V12 = -w.V12; w.V21 = -w.V21; }
    if (fy) { w.v = -w.v; w.V12 = -w.V12; w.V21 = -w.V21; }
    store_prim<DIM, RX>(A.W, A.T, cidx(pd, i, j), w);
    if (rate_on && i >= 0 && i < pd.nx && j >= 0 && j < pd.ny) {
      const Strain s = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
      const double rho = w.phi * w.r1 + (1.0 - w.phi) * w.r2;
      const double cL2 = cL2_of(P, w.phi, rho, w.p, s.J2);
      // a state that has lost hyperbolicity (or a density) is reported, not stepped silently
      if (!(cL2 > 0.0) || !(rho > 0.0)) flag_bad(A.status, g.x, i + pd.nx * j);
      const double cL = sqrt(fmax(cL2, 0.0));
      r = (fabs(w.u) + cL) / pd.dx;
      if (DIM == 2) r += (fabs(w.v) + cL) / pd.dy;
    }
  }
  if (rate_on) {
    // warp-shuffle max, then one atomic per warp (all threads share the patch)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0 && r > 0.0)
      atomicMax(A.rate + g.x, (unsigned long long)__double_as_longlong(r));
  }
}

// ---------------------------------------------------------------------------
// Face fluxes.  DIR 0: x faces, segment = (patch, row j, first face f0, n);
// face f lies between cells f-1 and f.  DIR 1: y faces, segment = (patch,
// face row j, first column i0, n); face row j lies between cell rows j-1, j.
// ---------------------------------------------------------------------------
template <int DIM, bool RX, int DIR>
__global__ void __launch_bounds__(SEG) k_flux(Phys P, StepArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const long long T = A.T;
  const double* __restrict__ W = A.W;
  // cell index along the sweep of the face's left cell, and the fixed coordinate
  const int f = (DIR == 0 ? g.z : g.y) + (DIR == 0 ? threadIdx.x : 0);
  const int col = DIR == 0 ? g.y : g.z + threadIdx.x;  // row (x sweep) or column (y sweep)
  const int a = (DIR == 0 ? f : g.y) - 1;
  auto at = [&](int s) -> long long {  // cell at sweep position s on this line
    return DIR == 0 ? cidx(pd, s, col) : cidx(pd, col, s);
  };
  const long long stride_t = DIR == 0 ? (long long)pd.pitch : 1;  // transverse neighbour step

  // volume fraction on the line, cells a-2 .. a+3
  double ph[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) ph[s] = W[L::PHI * T + at(a - 2 + s)];

  // phi edge values of cells a (right edge) and a+1 (left edge)
  double phiL, phiR;
  {
    Cand c[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      double beta = 2.51;  // beta0 |n_d| + 0.01 with |n_d| = 1 in 1D
      if (DIM == 2 && P.thinc) {
        // Youngs normal from the (1,2,1)-weighted central differences of phi
        const long long k = at(a - 1 + s);
        const double* Ph = W + L::PHI * T;
        const long long sx = DIR == 0 ? 1 : (long long)pd.pitch;  // along the sweep
        const long long sy = DIR == 0 ? (long long)pd.pitch : 1;  // across it
        const double dn = (Ph[k + sx + sy] + 2.0 * Ph[k + sx] + Ph[k + sx - sy]) -
                          (Ph[k - sx + sy] + 2.0 * Ph[k - sx] + Ph[k - sx - sy]);
        const double dt_ = (Ph[k + sy + sx] + 2.0 * Ph[k + sy] + Ph[k + sy - sx]) -
                           (Ph[k - sy + sx] + 2.0 * Ph[k - sy] + Ph[k - sy - sx]);
        const double hn = DIR == 0 ? pd.dx : pd.dy, ht = DIR == 0 ? pd.dy : pd.dx;
        const double gn = dn / hn, gt = dt_ / ht;
        const double nrm = sqrt(gn * gn + gt * gt);
        beta = 2.5 * (nrm == 0.0 ? 1.0 : fabs(gn) / nrm) + 0.01;
      }
      c[s] = phi_cand(ph[s], ph[s + 1], ph[s + 2], beta, P.thinc != 0);
    }
    double Lt, Rt;
    bvd(c[0], c[1], c[2], Lt, Rt);
    phiL = Rt;  // right edge of cell a
    bvd(c[1], c[2], c[3], Lt, Rt);
    phiR = Lt;  // left edge of cell a+1
  }
  (void)stride_t;

  // MUSCL on the other primitives: cells a-1, a, a+1, a+2
  const Prim w0 = load_prim<DIM, RX>(W, T, at(a - 1));
  const Prim w1 = load_prim<DIM, RX>(W, T, at(a));
  const Prim w2 = load_prim<DIM, RX>(W, T, at(a + 1));
  const Prim w3 = load_prim<DIM, RX>(W, T, at(a + 2));
  Prim wl, wr;
#define DIS_REC(fld)                                            \
  {                                                             \
    const double s1 = minmod(w1.fld - w0.fld, w2.fld - w1.fld); \
    const double s2 = minmod(w2.fld - w1.fld, w3.fld - w2.fld); \
    wl.fld = w1.fld + 0.5 * s1;                                 \
    wr.fld = w2.fld - 0.5 * s2;                                 \
  }
  DIS_REC(r1) DIS_REC(r2) DIS_REC(u) DIS_REC(p) DIS_REC(V11) DIS_REC(V22) DIS_REC(V33)
  if constexpr (DIM == 2) { DIS_REC(v) DIS_REC(V12) DIS_REC(V21) }
  else { wl.v = wr.v = 0.0; wl.V12 = wr.V12 = wl.V21 = wr.V21 = 0.0; }
  if constexpr (RX) { DIS_REC(lam) } else { wl.lam = wr.lam = 0.0; }
#undef DIS_REC
  wl.phi = phiL;
  wr.phi = phiR;

  // A reconstructed face state that is not hyperbolic (c_L^2 <= 0) falls back
  // to its cell-centre state on that side of the face.
  FState sl = face_state<DIR>(P, wl);
  if (!(sl.cL > 0.0)) sl = face_state<DIR>(P, w1);
  FState sr = face_state<DIR>(P, wr);
  if (!(sr.cL > 0.0)) sr = face_state<DIR>(P, w2);
  sl.cL = sqrt(sl.cL);
  sr.cL = sqrt(sr.cL);
  const FaceOut o = hllc<DIR>(sl, sr);

  // velocity of the face state in x/y components
  const double fu = DIR == 0 ? o.un : o.ut;
  const double fv = DIR == 0 ? o.ut : o.un;
  double* F = DIR == 0 ? A.Fx : A.Fy;
  const long long NFc = DIR == 0 ? A.NFX : A.NFY;
  const long long fi = DIR == 0 ? pd.fxoff + (long long)col * (pd.nx + 1) + f
                                : pd.fyoff + (long long)g.y * pd.nx + col;
  F[L::PHI * NFc + fi] = o.phi * o.un;
  F[L::A1 * NFc + fi] = o.Far1;
  F[L::A2 * NFc + fi] = o.Far2;
  F[L::MX * NFc + fi] = DIR == 0 ? o.Fmn : o.Fmt;
  if constexpr (DIM == 2) F[L::MY * NFc + fi] = DIR == 0 ? o.Fmt : o.Fmn;
  F[L::E * NFc + fi] = o.FE;
  if constexpr (RX) F[L::AL * NFc + fi] = o.Farl;
  // stretch fluxes V_ij u_d - V_dj u_i at the face state
  if constexpr (DIR == 0) {
    F[L::V11 * NFc + fi] = 0.0;
    if constexpr (DIM == 2) {
      F[L::V12 * NFc + fi] = 0.0;
      F[L::V21 * NFc + fi] = o.V21 * fu - o.V11 * fv;
      F[L::V22 * NFc + fi] = o.V22 * fu - o.V12 * fv;
    } else {
      F[L::V22 * NFc + fi] = o.V22 * fu;
    }
    F[L::V33 * NFc + fi] = o.V33 * fu;
    F[(L::NF + 0) * NFc + fi] = o.un;
    F[(L::NF + 1) * NFc + fi] = o.V11;
    if constexpr (DIM == 2) F[(L::NF + 2) * NFc + fi] = o.V12;
  } else if constexpr (DIM == 2) {
    F[L::V11 * NFc + fi] = o.V11 * fv - o.V21 * fu;
    F[L::V12 * NFc + fi] = o.V12 * fv - o.V22 * fu;
    F[L::V21 * NFc + fi] = 0.0;
    F[L::V22 * NFc + fi] = 0.0;
    F[L::V33 * NFc + fi] = o.V33 * fv;
    F[(L::NF + 0) * NFc + fi] = o.un;
    F[(L::NF + 1) * NFc + fi] = o.V21;
    F[(L::NF + 2) * NFc + fi] = o.V22;
  }
}

// ---------------------------------------------------------------------------
// Divergence, non-conservative terms, RK combination; on the last stage the
// plastic and reactive source steps (pointwise) and the status check.
// ---------------------------------------------------------------------------
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_update(Phys P, StepArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long k = cidx(pd, i, j);
  const long long T = A.T;
  double q[NF], D[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) q[c] = A.qsrc[c * T + k];
  const double idx_ = 1.0 / pd.dx;
  const long long fl = pd.fxoff + (long long)j * (pd.nx + 1) + i;
  const long long NFX = A.NFX;
#pragma unroll
  for (int c = 0; c < NF; ++c) D[c] = (A.Fx[c * NFX + fl + 1] - A.Fx[c * NFX + fl]) * idx_;
  double divu = (A.Fx[NF * NFX + fl + 1] - A.Fx[NF * NFX + fl]) * idx_;
  double bx = (A.Fx[(NF + 1) * NFX + fl + 1] - A.Fx[(NF + 1) * NFX + fl]) * idx_;
  double by = 0.0;
  if constexpr (DIM == 2) {
    by = (A.Fx[(NF + 2) * NFX + fl + 1] - A.Fx[(NF + 2) * NFX + fl]) * idx_;
    const double idy = 1.0 / pd.dy;
    const long long NFY = A.NFY;
    const long long fb = pd.fyoff + (long long)j * pd.nx + i;
    const long long ft = fb + pd.nx;
#pragma unroll
    for (int c = 0; c < NF; ++c) D[c] += (A.Fy[c * NFY + ft] - A.Fy[c * NFY + fb]) * idy;
    divu += (A.Fy[NF * NFY + ft] - A.Fy[NF * NFY + fb]) * idy;
    bx += (A.Fy[(NF + 1) * NFY + ft] - A.Fy[(NF + 1) * NFY + fb]) * idy;
    by += (A.Fy[(NF + 2) * NFY + ft] - A.Fy[(NF + 2) * NFY + fb]) * idy;
  }
  const double rho = q[L::A1] + q[L::A2];
  const double uc = q[L::MX] / rho;
  double vc = 0.0;
  if constexpr (DIM == 2) vc = q[L::MY] / rho;
  const double t23 = 2.0 / 3.0;
  D[L::PHI] -= q[L::PHI] * divu;
  D[L::V11] -= t23 * q[L::V11] * divu - uc * bx;
  D[L::V22] -= t23 * q[L::V22] * divu - vc * by;
  D[L::V33] -= t23 * q[L::V33] * divu;
  if constexpr (DIM == 2) {
    D[L::V12] -= t23 * q[L::V12] * divu - uc * by;
    D[L::V21] -= t23 * q[L::V21] * divu - vc * bx;
  }
  const double dt = A.dtfix ? A.dtfix[g.x] : P.cfl / __longlong_as_double((long long)A.rate[g.x]);
  double o[NF];
  if (A.a == 0.0) {
#pragma unroll
    for (int c = 0; c < NF; ++c) o[c] = q[c] - dt * D[c];
  } else {
#pragma unroll
    for (int c = 0; c < NF; ++c) o[c] = A.a * A.qn[c * T + k] + A.b * (q[c] - dt * D[c]);
  }
  if (A.last) {
    double v12 = 0.0, v21 = 0.0;
    if constexpr (DIM == 2) { v12 = o[L::V12]; v21 = o[L::V21]; }
    plastic(P, o[L::PHI], dt, o[L::V11], v12, v21, o[L::V22], o[L::V33]);
    if constexpr (DIM == 2) { o[L::V12] = v12; o[L::V21] = v21; }
    if constexpr (RX) {
      const int y = P.y;
      const MatDev& m = P.m[y];
      const double phi1 = o[L::PHI];
      const double ary = y == 0 ? o[L::A1] : o[L::A2];
      const double phy = y == 0 ? phi1 : 1.0 - phi1;
      const double rr = o[L::A1] + o[L::A2];
      const double mx = o[L::MX];
      double my = 0.0;
      if constexpr (DIM == 2) my = o[L::MY];
      const double KE = 0.5 * (mx * mx + my * my) / rr;
      const Strain s = strain_of(o[L::V11], v12, v21, o[L::V22], o[L::V33]);
      const double xi = xi_of(P, phi1);
      const double p0 = (o[L::E] - KE - ref_energy(P, phi1, o[L::A1], o[L::A2], 0.0, s.J2)) / xi;
      const double Tfac = m.iGm1 / ((ary / phy) * m.cv);  // T = p / (rho_y Gamma c_V)
      const double Qx = m.Q / xi;
      auto f = [&](double Lm) {
        const double Tk = (p0 - Qx * Lm) * Tfac;
        return Tk > 0.0 ? -m.A * Lm * exp(-m.Tact / Tk) : 0.0;
      };
      const double L0 = o[L::AL];
      const double k1 = f(L0);
      const double k2 = f(L0 + 0.5 * dt * k1);
      const double k3 = f(L0 + 0.5 * dt * k2);
      const double k4 = f(L0 + dt * k3);
      o[L::AL] = L0 + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }
    bool bad = !(o[L::PHI] >= -1e-6 && o[L::PHI] <= 1.0 + 1e-6);
#pragma unroll
    for (int c = 0; c < NF; ++c) bad |= !isfinite(o[c]);
    if (bad) flag_bad(A.status, g.x, i + pd.nx * j);
    if (i == 0 && j == 0) A.dtlast[g.x] = dt;
  }
#pragma unroll
  for (int c = 0; c < NF; ++c) A.qdst[c * T + k] = o[c];
}

// ---------------------------------------------------------------------------
// Packed <-> padded transfers (interior cells), with primitive -> conservative
// conversion on load (MG form solved for the energy, mixture rules).
// ---------------------------------------------------------------------------
template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_unpack(Phys P, const PatchDev* __restrict__ pds,
                                                const int4* __restrict__ segs, const double* src,
                                                double* q, long long T, int primitive) {
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
  for (int c = 0; c < NF; ++c) q[c * T + k] = v[c];
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack(const PatchDev* __restrict__ pds,
                                              const int4* __restrict__ segs, const double* q,
                                              double* dst, long long T) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
#pragma unroll
  for (int c = 0; c < NF; ++c) dst[s0 + c * ncell] = q[c * T + k];
}

}  // namespace dis
