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
#include "face.cuh"

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
  double x0;        // x of the low face (radius in cylindrical geometry)
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
  double* E;                 // MUSCL-Hancock: evolved edge states, plane (2 d + side) NF + field
};

__device__ __forceinline__ long long cidx(const PatchDev& p, int i, int j) {
  return p.off + (long long)(j + (p.rows > 1 ? NG : 0)) * p.pitch + (i + NG);
}

// Ghost index map of one axis: returns the source index and whether the
// reflective boundary flips this axis' normal velocity.
__device__ __forceinline__ int ghost_map(int i, int n, int bclo, int bchi, bool& flip) {
  if (i < 0) {
    if (bclo == 3) return i;  // external: the stored ghost layer
    if (bclo == 1) return i + n;
    if (bclo == 2) { flip = !flip; return -1 - i; }
    return 0;
  }
  if (i >= n) {
    if (bchi == 3) return i;
    if (bchi == 1) return i - n;
    if (bchi == 2) { flip = !flip; return 2 * n - 1 - i; }
    return n - 1;
  }
  return i;
}

template <int DIM, bool RX>
__device__ __forceinline__ Prim cons_to_prim(const Phys& P, const double* q, long long T, long long k) {
  constexpr int NF = Lay<DIM, RX>::NF;
  double v[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) v[c] = q[c * T + k];
  return prim_of<DIM, RX, double>(P, v);
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
      const double cL2 = cL2_of(at_state(P, w.lam, w.p), w.phi, rho, w.p, s.J2, w.r1, w.r2);
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

  // volume fraction on the line (cells a-2 .. a+3) and, for the 2D Youngs
  // normal, on the two neighbouring lines
  double B[3][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) B[1][c] = W[L::PHI * T + at(a - 2 + c)];
  const bool normals = DIM == 2 && P.thinc;
  if (normals) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      B[0][c] = W[L::PHI * T + at(a - 2 + c) - stride_t];
      B[2][c] = W[L::PHI * T + at(a - 2 + c) + stride_t];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) B[0][c] = B[2][c] = 0.0;
  }
  double phiL, phiR;
  face_phi<DIM, double>(B, P.thinc != 0, DIR == 0 ? pd.dx : pd.dy, DIR == 0 ? pd.dy : pd.dx, phiL, phiR,
                        P.limiter);

  // MUSCL on the other primitives: cells a-1, a, a+1, a+2
  const Prim w0 = load_prim<DIM, RX>(W, T, at(a - 1));
  const Prim w1 = load_prim<DIM, RX>(W, T, at(a));
  const Prim w2 = load_prim<DIM, RX>(W, T, at(a + 1));
  const Prim w3 = load_prim<DIM, RX>(W, T, at(a + 2));
  Prim wl, wr;
  muscl_pair(w0.r1, w1.r1, w2.r1, w3.r1, wl.r1, wr.r1, P.limiter);
  muscl_pair(w0.r2, w1.r2, w2.r2, w3.r2, wl.r2, wr.r2, P.limiter);
  muscl_pair(w0.u, w1.u, w2.u, w3.u, wl.u, wr.u, P.limiter);
  muscl_pair(w0.p, w1.p, w2.p, w3.p, wl.p, wr.p, P.limiter);
  muscl_pair(w0.V11, w1.V11, w2.V11, w3.V11, wl.V11, wr.V11, P.limiter);
  muscl_pair(w0.V22, w1.V22, w2.V22, w3.V22, wl.V22, wr.V22, P.limiter);
  muscl_pair(w0.V33, w1.V33, w2.V33, w3.V33, wl.V33, wr.V33, P.limiter);
  if constexpr (DIM == 2) {
    muscl_pair(w0.v, w1.v, w2.v, w3.v, wl.v, wr.v, P.limiter);
    muscl_pair(w0.V12, w1.V12, w2.V12, w3.V12, wl.V12, wr.V12, P.limiter);
    muscl_pair(w0.V21, w1.V21, w2.V21, w3.V21, wl.V21, wr.V21, P.limiter);
  } else {
    wl.v = wr.v = 0.0;
    wl.V12 = wr.V12 = wl.V21 = wr.V21 = 0.0;
  }
  if constexpr (RX) muscl_pair(w0.lam, w1.lam, w2.lam, w3.lam, wl.lam, wr.lam, P.limiter);
  else wl.lam = wr.lam = 0.0;
  wl.phi = phiL;
  wr.phi = phiR;

  // A reconstructed face state that is not hyperbolic (c_L^2 <= 0) falls back
  // to its cell-centre state on that side of the face.
  FState sl = face_state<DIR>(P, wl);
  if (!(sl.cL > 0.0)) sl = face_state<DIR>(P, w1);
  FState sr = face_state<DIR>(P, wr);
  if (!(sr.cL > 0.0)) sr = face_state<DIR>(P, w2);
  constexpr int NO = n_face_out<DIM, RX>();
  double out[NO];
  riemann_outputs<DIM, RX, DIR>(sl, sr, out);

  double* F = DIR == 0 ? A.Fx : A.Fy;
  const long long NFc = DIR == 0 ? A.NFX : A.NFY;
  const long long fi = DIR == 0 ? pd.fxoff + (long long)col * (pd.nx + 1) + f
                                : pd.fyoff + (long long)g.y * pd.nx + col;
#pragma unroll
  for (int c = 0; c < NO; ++c) F[c * NFc + fi] = out[c];
}

// Cylindrical geometry (x = r, y = z): add to the operator D of a cell at
// radius r the bracket of s_g = -(1/r) (...) of Section 3, from the cell's
// conservative state q and primitives w (stress sigma = -p I + 2 G dev H).
template <int DIM, bool RX>
__device__ __forceinline__ void add_geometric(const Phys& P, const double* q, const Prim& w, double r, double* D) {
  using L = Lay<DIM, RX>;
  const double ir = 1.0 / r;
  const Strain st = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const double Gm2 = 2.0 * Gmix_of(at_state(P, w.lam, w.p), w.phi, w.r1, w.r2);
  const double srr = -w.p + Gm2 * st.H11, szr = Gm2 * st.H12, stt = -w.p + Gm2 * st.H33;
  const double ur = w.u, uz = w.v;
  const double rho = q[L::A1] + q[L::A2];
  D[L::A1] += q[L::A1] * ur * ir;
  D[L::A2] += q[L::A2] * ur * ir;
  if constexpr (RX) D[L::AL] += q[L::AL] * ur * ir;
  D[L::MX] += (rho * ur * ur - srr + stt) * ir;
  if constexpr (DIM == 2) D[L::MY] += (rho * uz * ur - szr) * ir;
  D[L::E] += (q[L::E] * ur - (ur * srr + uz * szr)) * ir;
  const double t = (1.0 / 3.0) * ur * ir;
  D[L::V11] += t * q[L::V11];
  D[L::V22] += t * q[L::V22];
  D[L::V33] += (1.0 / 3.0 - 1.0) * ur * ir * q[L::V33];
  if constexpr (DIM == 2) {
    D[L::V12] += t * q[L::V12];
    D[L::V21] += t * q[L::V21];
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
  if (P.cyl) add_geometric<DIM, RX>(P, q, load_prim<DIM, RX>(A.W, T, k), pd.x0 + (i + 0.5) * pd.dx, D);
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
    sources<DIM, RX, double>(P, dt, o);
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
                                                double* q, long long T, int primitive, long long base = 0) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff - base + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
  double v[NF];
#pragma unroll
  for (int c = 0; c < NF; ++c) v[c] = src[s0 + c * ncell];
  if (primitive) cons_of<DIM, RX, double>(P, v);
#pragma unroll
  for (int c = 0; c < NF; ++c) q[c * T + k] = v[c];
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_pack(const PatchDev* __restrict__ pds,
                                              const int4* __restrict__ segs, const double* q,
                                              double* dst, long long T, long long base = 0) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const long long ncell = (long long)pd.nx * pd.ny;
  const long long s0 = pd.poff - base + (long long)j * pd.nx + i;
  const long long k = cidx(pd, i, j);
#pragma unroll
  for (int c = 0; c < NF; ++c) dst[s0 + c * ncell] = q[c * T + k];
}

// ---------------------------------------------------------------------------
// Single-stage MUSCL-Hancock update (the Runge-Kutta alternative with one
// Riemann solve per face and step).  k_hancock, per padded cell within one
// cell of the interior: the left and right edge states along each axis (MUSCL
// on the primitives, MUSCL-BVD-THINC on phi, cell-centre state where not
// hyperbolic), moved by -dt/2 D_c with D_c the operator of the cell evaluated
// on its own edge states (physical fluxes, non-conservative terms with the
// cell-centre coefficients), back to primitives (cell-centre state where not
// hyperbolic), stored in E.  k_flux_h: the Riemann problem of each face
// between the evolved edge states of its two cells; k_update (a = 0, b = 1,
// last) completes the step.
// ---------------------------------------------------------------------------
// c_L^2 > 0 for a primitive state (the value face_state returns as cL).
__device__ __forceinline__ bool hyperbolic(const Phys& P, const Prim& w) {
  const Strain st = strain_of(w.V11, w.V12, w.V21, w.V22, w.V33);
  const double rho = w.phi * w.r1 + (1.0 - w.phi) * w.r2;
  return cL2_of(at_state(P, w.lam, w.p), w.phi, rho, w.p, st.J2, w.r1, w.r2) > 0.0;
}

// Edge states of cell k along axis D (MUSCL, MUSCL-BVD-THINC on phi, the
// cell-centre state wc where not hyperbolic) and their physical outputs.
template <int DIM, bool RX, int D>
__device__ __forceinline__ void hancock_edges(const Phys& P, const double* __restrict__ W, long long T,
                                              long long k, const PatchDev& pd, const Prim& wc, Prim& lo,
                                              Prim& hi, double* Fm, double* Fp) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const long long st = D == 0 ? 1 : (long long)pd.pitch;  // along the axis
  const long long sx = D == 0 ? (long long)pd.pitch : 1;  // across it
  double B[3][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) B[1][c] = W[L::PHI * T + k + (c - 2) * st];
  const bool normals = DIM == 2 && P.thinc;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    B[0][c] = normals ? W[L::PHI * T + k + (c - 2) * st - sx] : 0.0;
    B[2][c] = normals ? W[L::PHI * T + k + (c - 2) * st + sx] : 0.0;
  }
  double eL, eR;
  cell_phi_edges<DIM, double>(B, P.thinc != 0, D == 0 ? pd.dx : pd.dy, D == 0 ? pd.dy : pd.dx, eL, eR,
                              P.limiter);
  Prim wm = load_prim<DIM, RX>(W, T, k - st);
  Prim wp = load_prim<DIM, RX>(W, T, k + st);
  Prim m = wc;
  lo = wc;
  hi = wc;
#pragma unroll
  for (int c = 0; c < NF; ++c) {
    if (c == L::PHI) continue;
    const double sl = limited(prim_slot<DIM, RX>(m, c) - prim_slot<DIM, RX>(wm, c),
                              prim_slot<DIM, RX>(wp, c) - prim_slot<DIM, RX>(m, c), P.limiter);
    prim_slot<DIM, RX>(lo, c) = prim_slot<DIM, RX>(m, c) - 0.5 * sl;
    prim_slot<DIM, RX>(hi, c) = prim_slot<DIM, RX>(m, c) + 0.5 * sl;
  }
  lo.phi = eL;
  hi.phi = eR;
  FState fl = face_state<D>(P, lo), fh = face_state<D>(P, hi);
  const bool okl = fl.cL > 0.0, okh = fh.cL > 0.0;
  if (!okl || !okh) {
    const FState fc = face_state<D>(P, wc);
    if (!okl) { lo = wc; fl = fc; }
    if (!okh) { hi = wc; fh = fc; }
  }
  face_outputs<DIM, RX, D, double>(physical_faceout<D>(fl), Fm);
  face_outputs<DIM, RX, D, double>(physical_faceout<D>(fh), Fp);
}

template <int DIM, bool RX>
__global__ void __launch_bounds__(SEG) k_hancock(Phys P, StepArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  constexpr int NO = n_face_out<DIM, RX>();
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  if (i < -1 || i > pd.nx || (DIM == 2 && (j < -1 || j > pd.ny))) return;
  const long long T = A.T;
  const double* __restrict__ W = A.W;
  const long long k = cidx(pd, i, j);
  const Prim wc = load_prim<DIM, RX>(W, T, k);
  // edge states e[2 d] (left / lower), e[2 d + 1] (right / upper) and D_c of
  // the cell from their physical outputs
  Prim e[2 * DIM];
  double D[NF];
  double divu, bx, by = 0.0;
  {
    double Fm[NO], Fp[NO];
    hancock_edges<DIM, RX, 0>(P, W, T, k, pd, wc, e[0], e[1], Fm, Fp);
    const double ih = 1.0 / pd.dx;
#pragma unroll
    for (int c = 0; c < NF; ++c) D[c] = (Fp[c] - Fm[c]) * ih;
    divu = (Fp[NF] - Fm[NF]) * ih;
    bx = (Fp[NF + 1] - Fm[NF + 1]) * ih;
    if constexpr (DIM == 2) by = (Fp[NF + 2] - Fm[NF + 2]) * ih;
  }
  if constexpr (DIM == 2) {
    double Fm[NO], Fp[NO];
    hancock_edges<DIM, RX, 1>(P, W, T, k, pd, wc, e[2], e[3], Fm, Fp);
    const double ih = 1.0 / pd.dy;
#pragma unroll
    for (int c = 0; c < NF; ++c) D[c] += (Fp[c] - Fm[c]) * ih;
    divu += (Fp[NF] - Fm[NF]) * ih;
    bx += (Fp[NF + 1] - Fm[NF + 1]) * ih;
    by += (Fp[NF + 2] - Fm[NF + 2]) * ih;
  }
  // cell-centre conservative coefficients (ghosts by the index map, reflective flips)
  double q[NF];
  {
    bool fx = false, fy = false;
    const int si = ghost_map(i, pd.nx, pd.bc[0], pd.bc[1], fx);
    const int sj = DIM == 2 ? ghost_map(j, pd.ny, pd.bc[2], pd.bc[3], fy) : 0;
    const long long ks = cidx(pd, si, sj);
#pragma unroll
    for (int c = 0; c < NF; ++c) q[c] = A.qsrc[c * T + ks];
    if (fx) {
      q[L::MX] = -q[L::MX];
      if constexpr (DIM == 2) { q[L::V12] = -q[L::V12]; q[L::V21] = -q[L::V21]; }
    }
    if constexpr (DIM == 2) {
      if (fy) { q[L::MY] = -q[L::MY]; q[L::V12] = -q[L::V12]; q[L::V21] = -q[L::V21]; }
    }
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
  const double h = 0.5 * dt;
#pragma unroll
  for (int s = 0; s < 2 * DIM; ++s) {
    double v[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) v[c] = prim_slot<DIM, RX>(e[s], c);
    cons_of<DIM, RX, double>(P, v);
#pragma unroll
    for (int c = 0; c < NF; ++c) v[c] -= h * D[c];
    Prim w = prim_of<DIM, RX, double>(P, v);
    if (!hyperbolic(P, w)) w = wc;
#pragma unroll
    for (int c = 0; c < NF; ++c) A.E[((long long)s * NF + c) * T + k] = prim_slot<DIM, RX>(w, c);
  }
}

template <int DIM, bool RX, int DIR>
__global__ void __launch_bounds__(SEG) k_flux_h(Phys P, StepArgs A, const int4* __restrict__ segs) {
  using L = Lay<DIM, RX>;
  constexpr int NF = L::NF;
  const int4 g = segs[blockIdx.x];
  if (threadIdx.x >= g.w) return;
  const PatchDev pd = A.pd[g.x];
  const long long T = A.T;
  const int f = (DIR == 0 ? g.z : g.y) + (DIR == 0 ? threadIdx.x : 0);
  const int col = DIR == 0 ? g.y : g.z + threadIdx.x;
  const int a = (DIR == 0 ? f : g.y) - 1;
  const long long ka = DIR == 0 ? cidx(pd, a, col) : cidx(pd, col, a);
  const long long kb = DIR == 0 ? cidx(pd, a + 1, col) : cidx(pd, col, a + 1);
  Prim wl{}, wr{};
#pragma unroll
  for (int c = 0; c < NF; ++c) {
    prim_slot<DIM, RX>(wl, c) = A.E[((long long)(2 * DIR + 1) * NF + c) * T + ka];
    prim_slot<DIM, RX>(wr, c) = A.E[((long long)(2 * DIR) * NF + c) * T + kb];
  }
  constexpr int NO = n_face_out<DIM, RX>();
  double out[NO];
  riemann_outputs<DIM, RX, DIR>(face_state<DIR>(P, wl), face_state<DIR>(P, wr), out);
  double* F = DIR == 0 ? A.Fx : A.Fy;
  const long long NFc = DIR == 0 ? A.NFX : A.NFY;
  const long long fi = DIR == 0 ? pd.fxoff + (long long)col * (pd.nx + 1) + f
                                : pd.fyoff + (long long)g.y * pd.nx + col;
#pragma unroll
  for (int c = 0; c < NO; ++c) F[c * NFc + fi] = out[c];
}

}  // namespace dis
