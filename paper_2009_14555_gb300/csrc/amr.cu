// amr.cu - structured adaptive mesh refinement of the float64 step.
//
// Section 3 (the AMR platform paragraph): a hierarchy of levels refined
// recursively by a flagging criterion; on level l the mesh widths and the
// time step are 2^l times finer than on level 0; the single-grid update runs
// on every patch of a level.  Section 4.2: difference-based flagging.  The
// structured-AMR parts the paper leaves to its platform (subcycling, ghost
// cells from the coarser level, average-down, refluxing, blocks and proper
// nesting) follow the readings written out in include/dis.h.
//
// Layout: level 0 is one patch (the domain, its boundary conditions); level
// l >= 1 is one context whose patches are the refined blocks (2B x 2B cells,
// 2B in 1D), stepped as one batch by the float64 step.  A block side inside
// the domain (or on a periodic domain side) reads its ghost layers as stored
// (DIS_BC_EXTERNAL); before every Runge-Kutta stage a table-driven kernel
// fills them from the same level's blocks (copies) or from the coarser level
// (conservative linear interpolation in space, linear in time).  Flux
// registers collect the Runge-Kutta-weighted fluxes of the coarse-fine faces
// after each stage's flux kernels; after the two steps of level l + 1 a kernel
// averages it down into level l and another refluxes level l.  All tables
// are built on the host at each regrid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dis.h"
#include "ctx.cuh"

using namespace dis;

#define AFAIL(code, ...) dis_internal_error(code, __VA_ARGS__)
#define ACU(x)                                                                                     \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) return dis_internal_error(DIS_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

namespace {

// one cell of the fill table: dst <- copy of src (same level), or the
// interpolation of the coarse centre src with neighbours nb (x-, x+, y-, y+)
struct FillE {
  long long dst, src, nb[4];
  int kind;  // 0 copy, 1 interpolation
  int flip;  // bit 2k: neighbour k mirrored across an x wall, bit 2k + 1: across a y wall
  int ox, oy;
};
struct RegE {
  long long face;  // index in the Fx (dir 0) or Fy (dir 1) planes of the register's level
  int dir;
};
struct RefluxE {
  long long cell;  // coarse cell (index in the coarse level's planes)
  int c[4];        // coarse register of its x-lo, x-hi, y-lo, y-hi face (-1: not coarse-fine)
  int fa[4], fb[4];  // fine registers of those faces (fb: the second fine face in 2D, else -1)
};
struct AvgE {
  long long cell, ch[4];
};

struct Fields {
  int nf, ncons, cons[6];
  int flipx[3], nflipx, flipy[3], nflipy;
};

Fields fields_of(int dim, bool rx) {
  Fields f{};
  f.nf = (dim == 2 ? 11 : 8) + (rx ? 1 : 0);
  if (dim == 1) {
    int c[] = {1, 2, 3, 4};
    f.ncons = 4;
    for (int k = 0; k < 4; ++k) f.cons[k] = c[k];
    if (rx) f.cons[f.ncons++] = 8;
    f.flipx[0] = 3;
    f.nflipx = 1;
    f.nflipy = 0;
  } else {
    int c[] = {1, 2, 3, 4, 5};
    f.ncons = 5;
    for (int k = 0; k < 5; ++k) f.cons[k] = c[k];
    if (rx) f.cons[f.ncons++] = 11;
    f.flipx[0] = 3; f.flipx[1] = 7; f.flipx[2] = 8;
    f.nflipx = 3;
    f.flipy[0] = 4; f.flipy[1] = 7; f.flipy[2] = 8;
    f.nflipy = 3;
  }
  return f;
}

__device__ __forceinline__ double mm(double a, double b) {
  // minmod with the sign of a (a * b > 0 selects)
  return a * b > 0.0 ? (a > 0.0 ? fmin(a, b) : fmax(a, b)) : 0.0;
}

__device__ __forceinline__ double lerp_rn(double w0, double a, double w1, double b) {
  return __dadd_rn(__dmul_rn(w0, a), __dmul_rn(w1, b));
}

__global__ void k_amr_fill(const FillE* __restrict__ E, int n, Fields F, int dim, double* q, long long T,
                           const double* __restrict__ qco, const double* __restrict__ qcn, long long Tc,
                           double theta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const FillE f = E[e];
  const double w0 = 1.0 - theta, w1 = theta;
  for (int c = 0; c < F.nf; ++c) {
    if (f.kind == 0) {
      q[c * T + f.dst] = q[c * T + f.src];
      continue;
    }
    bool fx = false, fy = false;
    for (int k = 0; k < F.nflipx; ++k) fx |= F.flipx[k] == c;
    for (int k = 0; k < F.nflipy; ++k) fy |= F.flipy[k] == c;
    auto nbv = [&](int k) {
      const double v = lerp_rn(w0, qco[c * Tc + f.nb[k]], w1, qcn[c * Tc + f.nb[k]]);
      const bool m = ((f.flip >> (2 * k)) & 1) ? fx : false;
      const bool my = ((f.flip >> (2 * k + 1)) & 1) ? fy : false;
      return (m != my) ? -v : v;
    };
    const double ctr = lerp_rn(w0, qco[c * Tc + f.src], w1, qcn[c * Tc + f.src]);
    const double sx = mm(nbv(1) - ctr, ctr - nbv(0));
    double v = ctr + sx * (0.25 * f.ox);
    if (dim == 2) {
      const double sy = mm(nbv(3) - ctr, ctr - nbv(2));
      v = v + sy * (0.25 * f.oy);
    }
    q[c * T + f.dst] = v;
  }
}

__global__ void k_amr_copy(const long long* __restrict__ pairs, int n, int nf, const double* __restrict__ src,
                           long long Ts, double* dst, long long Td) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const long long s = pairs[2 * e], d = pairs[2 * e + 1];
  for (int c = 0; c < nf; ++c) dst[c * Td + d] = src[c * Ts + s];
}

// acc[e * ncons + k] += wdt * F[cons_k][face_e]
__global__ void k_amr_reg(const RegE* __restrict__ R, int n, Fields F, const double* __restrict__ Fx,
                          long long NFX, const double* __restrict__ Fy, long long NFY, double wdt, double* acc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const RegE r = R[e];
  const double* P = r.dir == 0 ? Fx : Fy;
  const long long NFc = r.dir == 0 ? NFX : NFY;
  for (int k = 0; k < F.ncons; ++k) acc[(long long)e * F.ncons + k] += wdt * P[F.cons[k] * NFc + r.face];
}

__global__ void k_amr_setdt(double* dtfix, int n, double dt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dtfix[e] = dt;
}

// substep totals of the fine registers: R = T (first substep) or R + T; T = 0
__global__ void k_amr_close(int n, double* T, double* R, int first) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  R[e] = first ? T[e] : R[e] + T[e];
  T[e] = 0.0;
}

__global__ void k_amr_avg(const AvgE* __restrict__ A, int n, int nf, int dim, double* qc, long long Tc,
                          const double* __restrict__ qf, long long Tf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const AvgE a = A[e];
  for (int c = 0; c < nf; ++c) {
    const double* f = qf + c * Tf;
    if (dim == 1) {
      qc[c * Tc + a.cell] = (f[a.ch[0]] + f[a.ch[1]]) / 2.0;
    } else {
      const double s0 = f[a.ch[0]] + f[a.ch[1]], s1 = f[a.ch[2]] + f[a.ch[3]];
      qc[c * Tc + a.cell] = (s0 + s1) / 4.0;
    }
  }
}

__global__ void k_amr_reflux(const RefluxE* __restrict__ X, int n, Fields F, int dim, double* q, long long T,
                             const double* __restrict__ C, const double* __restrict__ R, double hx, double hy) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const RefluxE x = X[e];
  for (int k = 0; k < F.ncons; ++k) {
    double* qk = q + F.cons[k] * T + x.cell;
    for (int d = 0; d < dim; ++d) {
      const double h = d == 0 ? hx : hy;
      double del[2] = {0.0, 0.0};
      for (int s = 0; s < 2; ++s) {
        const int side = 2 * d + s;
        if (x.c[side] < 0) continue;
        const double fc = C[(long long)x.c[side] * F.ncons + k];
        const double fa = x.fb[side] < 0 ? R[(long long)x.fa[side] * F.ncons + k]
                                         : 0.5 * (R[(long long)x.fa[side] * F.ncons + k] +
                                                  R[(long long)x.fb[side] * F.ncons + k]);
        del[s] = (fa - fc) / h;
      }
      *qk = *qk + (-del[1] + del[0]);
    }
  }
}

// Tags of the interior cells of every patch of a level (Section 4.2): the
// fractional change of phi1, phi_l rho_l, p and the velocity components to
// each face neighbour inside the domain.  Patch p has its origin (I0, J0) in
// level cells; tags go to the level's dense mask (NX x NY).
template <int DIM, bool RX>
__global__ void k_amr_tag(Phys P, const PatchDev* __restrict__ pds, const int4* __restrict__ segs,
                          const int2* __restrict__ org, const double* __restrict__ q, long long T, int NX, int NY,
                          double eps, double u_floor, unsigned char* tag) {
  constexpr int NF = Lay<DIM, RX>::NF;
  const int4 g = segs[blockIdx.x];
  if ((int)threadIdx.x >= g.w) return;
  const PatchDev pd = pds[g.x];
  const int i = g.z + threadIdx.x, j = g.y;
  const int I = org[g.x].x + i, J = org[g.x].y + j;
  auto val = [&](int ii, int jj, double* out) {
    double v[NF];
    const long long k = cidx(pd, ii, jj);
#pragma unroll
    for (int c = 0; c < NF; ++c) v[c] = q[c * T + k];
    const Prim w = prim_of<DIM, RX, double>(P, v);
    out[0] = v[Lay<DIM, RX>::PHI];
    out[1] = v[Lay<DIM, RX>::A1];
    out[2] = v[Lay<DIM, RX>::A2];
    out[3] = w.p;
    out[4] = w.u;
    out[5] = w.v;
  };
  double a[6];
  val(i, j, a);
  const double floors[6] = {1.0, 0.0, 0.0, 0.0, u_floor, u_floor};
  const int nv = DIM == 2 ? 6 : 5;
  bool t = false;
  for (int d = 0; d < DIM && !t; ++d) {
    for (int s = -1; s <= 1 && !t; s += 2) {
      const int In = I + (d == 0 ? s : 0), Jn = J + (d == 1 ? s : 0);
      if (In < 0 || In >= NX || Jn < 0 || Jn >= NY) continue;
      double b[6];
      val(i + (d == 0 ? s : 0), j + (d == 1 ? s : 0), b);
      for (int f = 0; f < nv; ++f) {
        const double x0 = s < 0 ? b[f] : a[f], x1 = s < 0 ? a[f] : b[f];
        const double den = fmax(fmax(fabs(x0), fabs(x1)), floors[f]);
        if (fabs(x1 - x0) > eps * den && den > 0.0) t = true;
      }
    }
  }
  if (t) tag[(long long)J * NX + I] = 1;
}

constexpr int TPB = 128;
unsigned nblk(long long n) { return (unsigned)((n + TPB - 1) / TPB); }

}  // namespace

// ---------------------------------------------------------------------------
struct dis_amr_level {
  dis_ctx* c = nullptr;
  int NX = 0, NY = 0;
  std::vector<int2> org;        // block origins in level cells (level 0: (0, 0))
  std::vector<int> owner;       // NX * NY: owning patch, -1 none
  int2* d_org = nullptr;
  double* q_old = nullptr;      // the state at the start of the level's step
  FillE* d_fill = nullptr;
  int n_fill = 0;
  // fine side (registers of this level's faces on the interface with level l - 1)
  RegE* d_freg = nullptr;
  int n_freg = 0;
  double* d_T = nullptr;
  double* d_R = nullptr;
  // coarse side (interface with level l + 1)
  RegE* d_creg = nullptr;
  int n_creg = 0;
  double* d_C = nullptr;
  RefluxE* d_reflux = nullptr;
  int n_reflux = 0;
  AvgE* d_avg = nullptr;
  int n_avg = 0;
  unsigned char* d_tag = nullptr;
};

struct dis_amr {
  int dim = 1, y = -1, L = 1, B = 8, buffer = 2, regrid_every = 0;
  double eps = 0.1, u_floor = 1.0;
  dis_patch dom{};
  dis_options opt{};
  dis_material mats[2]{};
  bool have_mats = false, have_state = false;
  cudaStream_t st = nullptr;
  Fields F{};
  std::vector<dis_amr_level> lev;
  long long steps = 0;
  // current step bookkeeping for the hooks
  int hl = 0;
  double hdt = 0.0, ht0 = 0.0, hlen = 1.0;
};

namespace {

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_tables(dis_amr_level& L) {
  dfree(L.d_org);
  dfree(L.d_fill);
  dfree(L.d_freg);
  dfree(L.d_T);
  dfree(L.d_R);
  dfree(L.d_creg);
  dfree(L.d_C);
  dfree(L.d_reflux);
  dfree(L.d_avg);
  dfree(L.d_tag);
  L.n_fill = L.n_freg = L.n_creg = L.n_reflux = L.n_avg = 0;
}

void free_level(dis_amr_level& L) {
  free_tables(L);
  dfree(L.q_old);
  if (L.c) dis_destroy(L.c);
  L.c = nullptr;
}

template <class T>
int upload(const std::vector<T>& v, T*& d, cudaStream_t st) {
  dfree(d);
  if (v.empty()) return DIS_OK;
  ACU(cudaMalloc(&d, sizeof(T) * v.size()));
  ACU(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return DIS_OK;
}

int dalloc_zero(double*& d, size_t n, cudaStream_t st) {
  dfree(d);
  if (n == 0) return DIS_OK;
  ACU(cudaMalloc(&d, sizeof(double) * n));
  ACU(cudaMemsetAsync(d, 0, sizeof(double) * n, st));
  return DIS_OK;
}

// index of local cell (i, j) of patch p in the context's planes
long long hidx(const dis_ctx* c, int p, int i, int j) {
  const PatchDev& d = c->pd[p];
  return d.off + (long long)(j + (d.rows > 1 ? NG : 0)) * d.pitch + (i + NG);
}
long long hfx(const dis_ctx* c, int p, int f, int j) { return c->pd[p].fxoff + (long long)j * (c->pd[p].nx + 1) + f; }
long long hfy(const dis_ctx* c, int p, int i, int jf) { return c->pd[p].fyoff + (long long)jf * c->pd[p].nx + i; }

// Build (or rebuild) the context of level l >= 1 from block origins.
int make_level(dis_amr* h, int l, const std::vector<int2>& org, dis_amr_level& L) {
  const int S = 2 * h->B;
  L.NX = h->dom.nx << l;
  L.NY = h->dim == 2 ? (h->dom.ny << l) : 1;
  L.org = org;
  std::vector<dis_patch> ps(org.size());
  for (size_t b = 0; b < org.size(); ++b) {
    dis_patch& p = ps[b];
    p.nx = S;
    p.ny = h->dim == 2 ? S : 1;
    p.dx = h->dom.dx / (1 << l);
    p.dy = h->dim == 2 ? h->dom.dy / (1 << l) : h->dom.dy;
    const int I0 = org[b].x, J0 = org[b].y;
    // x of the block's low face: the radius of its axis-side face in
    // cylindrical geometry (the geometric source takes r at cell centres)
    p.x0 = h->dom.x0 + I0 * p.dx;
    const bool edge[4] = {I0 == 0, I0 + S == L.NX, J0 == 0, J0 + S == L.NY};
    for (int k = 0; k < 4; ++k) {
      const int dbc = h->dom.bc[k];
      p.bc[k] = (edge[k] && dbc != DIS_BC_PERIODIC) ? dbc : DIS_BC_EXTERNAL;
      if (h->dim == 1 && k >= 2) p.bc[k] = 0;
    }
  }
  int rc = dis_internal_create_external(h->dim, (int)ps.size(), ps.data(), h->y, &h->opt, h->st, &L.c);
  if (rc) return rc;
  if ((rc = dis_set_materials(L.c, h->mats, 2))) return rc;
  if ((rc = dis_internal_ensure_ws(L.c))) return rc;
  L.c->have_state = true;
  for (auto& s : L.c->patch_set) s = 1;
  L.owner.assign((size_t)L.NX * L.NY, -1);
  for (size_t b = 0; b < org.size(); ++b)
    for (int j = 0; j < (h->dim == 2 ? S : 1); ++j)
      for (int i = 0; i < S; ++i) L.owner[(size_t)(org[b].y + j) * L.NX + org[b].x + i] = (int)b;
  return DIS_OK;
}

// Coarse cell (I, J) of level l - 1, mapped into the domain by its boundary
// conditions; flip receives the mirror bits (1 x, 2 y); false if outside a
// non-periodic side with no mapping (cannot happen for transmissive/reflective).
void map_coarse(const dis_amr* h, int NX, int NY, int& I, int& J, int& flip) {
  flip = 0;
  auto ax = [&](int& v, int n, int lo, int hi, int bit) {
    if (v < 0) {
      if (lo == DIS_BC_PERIODIC) v += n;
      else if (lo == DIS_BC_REFLECTIVE) { v = -1 - v; flip |= bit; }
      else v = 0;
    } else if (v >= n) {
      if (hi == DIS_BC_PERIODIC) v -= n;
      else if (hi == DIS_BC_REFLECTIVE) { v = 2 * n - 1 - v; flip |= bit; }
      else v = n - 1;
    }
  };
  ax(I, NX, h->dom.bc[0], h->dom.bc[1], 1);
  if (h->dim == 2) ax(J, NY, h->dom.bc[2], h->dom.bc[3], 2);
}

// index of level-l cell (I, J) (inside the domain) in level l's planes, or -1
long long cell_index(const dis_amr_level& L, int I, int J) {
  const int p = L.owner[(size_t)J * L.NX + I];
  if (p < 0) return -1;
  return hidx(L.c, p, I - L.org[p].x, J - L.org[p].y);
}

// Interpolation entry for the level-l cell (I, J) (inside the domain) from level l - 1.
bool interp_entry(const dis_amr* h, int l, int I, int J, long long dst, FillE& e) {
  const dis_amr_level& C = h->lev[l - 1];
  e = FillE{};
  e.dst = dst;
  e.kind = 1;
  const int Ic = I >> 1, Jc = J >> 1;
  e.ox = (I & 1) ? 1 : -1;
  e.oy = (J & 1) ? 1 : -1;
  e.src = cell_index(C, Ic, Jc);
  if (e.src < 0) return false;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  for (int k = 0; k < 4; ++k) {
    if (h->dim == 1 && k >= 2) {
      e.nb[k] = e.src;
      continue;
    }
    int In = Ic + di[k], Jn = Jc + dj[k], fl = 0;
    map_coarse(h, C.NX, C.NY, In, Jn, fl);
    e.nb[k] = cell_index(C, In, Jn);
    if (e.nb[k] < 0) return false;
    if (fl & 1) e.flip |= 1 << (2 * k);
    if (fl & 2) e.flip |= 1 << (2 * k + 1);
  }
  return true;
}

// Fill table of level l >= 1: every stored ghost cell inside the domain
// (periodic sides wrapped).
int build_fill(dis_amr* h, int l) {
  dis_amr_level& L = h->lev[l];
  const int S = 2 * h->B, Sy = h->dim == 2 ? S : 1, G = h->dim == 2 ? NG : 0;
  std::vector<FillE> E;
  for (size_t b = 0; b < L.org.size(); ++b) {
    for (int j = -G; j < Sy + G; ++j)
      for (int i = -NG; i < S + NG; ++i) {
        if (i >= 0 && i < S && j >= 0 && j < Sy) continue;
        int I = L.org[b].x + i, J = L.org[b].y + j;
        auto wrap = [&](int& v, int n, int lo, int hi) {
          if (v < 0) { if (lo != DIS_BC_PERIODIC) return false; v += n; }
          if (v >= n) { if (hi != DIS_BC_PERIODIC) return false; v -= n; }
          return true;
        };
        if (!wrap(I, L.NX, h->dom.bc[0], h->dom.bc[1])) continue;
        if (h->dim == 2 && !wrap(J, L.NY, h->dom.bc[2], h->dom.bc[3])) continue;
        const long long dst = hidx(L.c, (int)b, i, j);
        const long long src = cell_index(L, I, J);
        FillE e{};
        if (src >= 0) {
          e.kind = 0;
          e.dst = dst;
          e.src = src;
        } else if (!interp_entry(h, l, I, J, dst, e)) {
          return AFAIL(DIS_ECUDA, "dis_amr: level %d ghost cell (%d, %d) outside the coarser level (nesting)", l, I, J);
        }
        E.push_back(e);
      }
  }
  L.n_fill = (int)E.size();
  return upload(E, L.d_fill, h->st);
}

// Registers and the reflux / average tables between level l and l + 1.
int build_interface(dis_amr* h, int l) {
  dis_amr_level& C = h->lev[l];
  dis_amr_level& Fn = h->lev[l + 1];
  const int dim = h->dim;
  auto covered = [&](int Ic, int Jc) {  // coarse cell covered by level l + 1
    return Fn.owner[(size_t)(2 * Jc * (dim == 2 ? 1 : 0)) * Fn.NX + 2 * Ic] >= 0;
  };
  std::vector<RegE> creg, freg;
  std::vector<RefluxE> rfx;
  std::vector<AvgE> avg;
  for (int Jc = 0; Jc < C.NY; ++Jc)
    for (int Ic = 0; Ic < C.NX; ++Ic) {
      if (C.owner[(size_t)Jc * C.NX + Ic] < 0) continue;
      const long long ci = cell_index(C, Ic, Jc);
      if (covered(Ic, Jc)) {
        AvgE a{};
        a.cell = ci;
        if (dim == 1) {
          a.ch[0] = cell_index(Fn, 2 * Ic, 0);
          a.ch[1] = cell_index(Fn, 2 * Ic + 1, 0);
          a.ch[2] = a.ch[3] = a.ch[0];
        } else {
          a.ch[0] = cell_index(Fn, 2 * Ic, 2 * Jc);
          a.ch[1] = cell_index(Fn, 2 * Ic + 1, 2 * Jc);
          a.ch[2] = cell_index(Fn, 2 * Ic, 2 * Jc + 1);
          a.ch[3] = cell_index(Fn, 2 * Ic + 1, 2 * Jc + 1);
        }
        for (int k = 0; k < 4; ++k)
          if (a.ch[k] < 0) return AFAIL(DIS_ECUDA, "dis_amr: covered cell without children");
        avg.push_back(a);
        continue;
      }
      RefluxE x{};
      x.cell = ci;
      bool any = false;
      const int p = C.owner[(size_t)Jc * C.NX + Ic];
      const int li = Ic - C.org[p].x, lj = Jc - C.org[p].y;
      for (int side = 0; side < 2 * dim; ++side) {
        x.c[side] = x.fa[side] = x.fb[side] = -1;
        const int d = side / 2, s = side % 2;  // s = 0: low face, 1: high face
        int In = Ic + (d == 0 ? (s ? 1 : -1) : 0), Jn = Jc + (d == 1 ? (s ? 1 : -1) : 0);
        const int n = d == 0 ? C.NX : C.NY;
        int& v = d == 0 ? In : Jn;
        const int bclo = h->dom.bc[2 * d], bchi = h->dom.bc[2 * d + 1];
        if (v < 0) { if (bclo != DIS_BC_PERIODIC) continue; v += n; }
        if (v >= n) { if (bchi != DIS_BC_PERIODIC) continue; v -= n; }
        if (!covered(In, Jn)) continue;
        any = true;
        // coarse face: the cell's own face in its patch
        RegE rc{};
        rc.dir = d;
        rc.face = d == 0 ? hfx(C.c, p, li + s, lj) : hfy(C.c, p, li, lj + s);
        x.c[side] = (int)creg.size();
        creg.push_back(rc);
        // fine faces: on the covered side, the fine block's boundary faces
        for (int t = 0; t < (dim == 2 ? 2 : 1); ++t) {
          int If, Jf;  // the fine cell on the covered side next to the face
          if (d == 0) {
            If = s ? 2 * In : 2 * In + 1;
            Jf = dim == 2 ? 2 * Jc + t : 0;
          } else {
            Jf = s ? 2 * Jn : 2 * Jn + 1;
            If = 2 * Ic + t;
          }
          const int fp = Fn.owner[(size_t)Jf * Fn.NX + If];
          if (fp < 0) return AFAIL(DIS_ECUDA, "dis_amr: covered cell without a fine block");
          const int fi = If - Fn.org[fp].x, fj = Jf - Fn.org[fp].y;
          RegE rf{};
          rf.dir = d;
          // face between the covered fine cell and the uncovered side
          rf.face = d == 0 ? hfx(Fn.c, fp, s ? fi : fi + 1, fj) : hfy(Fn.c, fp, fi, s ? fj : fj + 1);
          if (t == 0) x.fa[side] = (int)freg.size();
          else x.fb[side] = (int)freg.size();
          freg.push_back(rf);
        }
      }
      if (any) rfx.push_back(x);
    }
  int rc;
  C.n_creg = (int)creg.size();
  Fn.n_freg = (int)freg.size();
  C.n_reflux = (int)rfx.size();
  C.n_avg = (int)avg.size();
  if ((rc = upload(creg, C.d_creg, h->st)) || (rc = upload(freg, Fn.d_freg, h->st)) ||
      (rc = upload(rfx, C.d_reflux, h->st)) || (rc = upload(avg, C.d_avg, h->st)))
    return rc;
  const int nc = h->F.ncons;
  if ((rc = dalloc_zero(C.d_C, (size_t)C.n_creg * nc, h->st)) ||
      (rc = dalloc_zero(Fn.d_T, (size_t)Fn.n_freg * nc, h->st)) ||
      (rc = dalloc_zero(Fn.d_R, (size_t)Fn.n_freg * nc, h->st)))
    return rc;
  return DIS_OK;
}

// Tables of level l alone: block origins, tag mask, old-state buffer and
// (l >= 1) the fill table against level l - 1.
int prep_level(dis_amr* h, int l) {
  int rc;
  dis_amr_level& L = h->lev[l];
  free_tables(L);
  if ((rc = upload(L.org, L.d_org, h->st))) return rc;
  ACU(cudaMalloc(&L.d_tag, (size_t)L.NX * L.NY));
  dfree(L.q_old);
  ACU(cudaMalloc(&L.q_old, sizeof(double) * (size_t)h->F.nf * L.c->T));
  if (l >= 1 && (rc = build_fill(h, l))) return rc;
  return DIS_OK;
}

int build_tables(dis_amr* h) {
  int rc;
  for (size_t l = 0; l < h->lev.size(); ++l)
    if ((rc = prep_level(h, (int)l))) return rc;
  for (size_t l = 0; l + 1 < h->lev.size(); ++l)
    if ((rc = build_interface(h, (int)l))) return rc;
  return DIS_OK;
}

// ghost cells of level l >= 1 at fraction theta of level l - 1's step (the
// coarse old state: q_old, or the current state when `current`)
void fill(dis_amr* h, int l, double* q, double theta, bool current) {
  dis_amr_level& L = h->lev[l];
  const dis_amr_level& C = h->lev[l - 1];
  if (!L.n_fill) return;
  const double* qo = current ? C.c->q[0] : C.q_old;
  k_amr_fill<<<nblk(L.n_fill), TPB, 0, h->st>>>(L.d_fill, L.n_fill, h->F, h->dim, q, L.c->T, qo, C.c->q[0], C.c->T,
                                               current ? 1.0 : theta);
}

// Runge-Kutta stage data: the time of each stage input (fraction of dt) and
// the weight of its fluxes in the step.  The MUSCL-Hancock update has one
// stage: input at the start of the step, flux weight 1.
const double kStageT[3] = {0.0, 1.0, 0.5};
const double kStageW[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};

void hook_before(void* u, int stage, double* qsrc) {
  dis_amr* h = (dis_amr*)u;
  const double ts = h->opt.scheme == DIS_HANCOCK ? 0.0 : kStageT[stage];
  if (h->hl >= 1) fill(h, h->hl, qsrc, h->ht0 + ts * h->hlen, false);
}

void hook_after_flux(void* u, int stage) {
  dis_amr* h = (dis_amr*)u;
  dis_amr_level& L = h->lev[h->hl];
  const double wdt = (h->opt.scheme == DIS_HANCOCK ? 1.0 : kStageW[stage]) * h->hdt;
  if (h->hl >= 1 && L.n_freg)
    k_amr_reg<<<nblk(L.n_freg), TPB, 0, h->st>>>(L.d_freg, L.n_freg, h->F, L.c->Fx, L.c->NFX, L.c->Fy, L.c->NFY,
                                                  wdt, L.d_T);
  if (h->hl + 1 < (int)h->lev.size() && L.n_creg)
    k_amr_reg<<<nblk(L.n_creg), TPB, 0, h->st>>>(L.d_creg, L.n_creg, h->F, L.c->Fx, L.c->NFX, L.c->Fy, L.c->NFY,
                                                  wdt, L.d_C);
}

int advance(dis_amr* h, int l, double dt, double t0, double len) {
  dis_amr_level& L = h->lev[l];
  const bool parent = l + 1 < (int)h->lev.size();
  const size_t bytes = sizeof(double) * (size_t)h->F.nf * L.c->T;
  if (parent) {
    ACU(cudaMemcpyAsync(L.q_old, L.c->q[0], bytes, cudaMemcpyDeviceToDevice, h->st));
    if (L.n_creg) ACU(cudaMemsetAsync(L.d_C, 0, sizeof(double) * (size_t)L.n_creg * h->F.ncons, h->st));
  }
  k_amr_setdt<<<nblk(L.c->np), TPB, 0, h->st>>>(L.c->dtfix, L.c->np, dt);
  h->hl = l;
  h->hdt = dt;
  h->ht0 = t0;
  h->hlen = len;
  StepHooks hk;
  hk.before = hook_before;
  hk.after_flux = hook_after_flux;
  hk.user = h;
  int rc = dis_internal_step64_hooked(L.c, hk);
  if (rc) return rc;
  if (l >= 1 && L.n_freg)
    k_amr_close<<<nblk((long long)L.n_freg * h->F.ncons), TPB, 0, h->st>>>(L.n_freg * h->F.ncons, L.d_T, L.d_R,
                                                                           t0 == 0.0 ? 1 : 0);
  if (parent) {
    for (int k = 0; k < 2; ++k)
      if ((rc = advance(h, l + 1, dt / 2, 0.5 * k, 0.5))) return rc;
    dis_amr_level& Fn = h->lev[l + 1];
    if (L.n_avg)
      k_amr_avg<<<nblk(L.n_avg), TPB, 0, h->st>>>(L.d_avg, L.n_avg, h->F.nf, h->dim, L.c->q[0], L.c->T,
                                                  Fn.c->q[0], Fn.c->T);
    if (L.n_reflux)
      k_amr_reflux<<<nblk(L.n_reflux), TPB, 0, h->st>>>(L.d_reflux, L.n_reflux, h->F, h->dim, L.c->q[0], L.c->T,
                                                        L.d_C, Fn.d_R, L.c->pd[0].dx, L.c->pd[0].dy);
  }
  ACU(cudaGetLastError());
  return DIS_OK;
}

// dense host tag mask of level l
int tags_of(dis_amr* h, int l, std::vector<unsigned char>& out) {
  dis_amr_level& L = h->lev[l];
  ACU(cudaMemsetAsync(L.d_tag, 0, (size_t)L.NX * L.NY, h->st));
  dis_ctx* c = L.c;
  const unsigned n = (unsigned)c->seg_cell.size();
  if (h->dim == 1) {
    if (h->y >= 0) k_amr_tag<1, true><<<n, SEG, 0, h->st>>>(c->phys, c->d_pd, c->d_seg_cell, L.d_org, c->q[0], c->T, L.NX, L.NY, h->eps, h->u_floor, L.d_tag);
    else k_amr_tag<1, false><<<n, SEG, 0, h->st>>>(c->phys, c->d_pd, c->d_seg_cell, L.d_org, c->q[0], c->T, L.NX, L.NY, h->eps, h->u_floor, L.d_tag);
  } else {
    if (h->y >= 0) k_amr_tag<2, true><<<n, SEG, 0, h->st>>>(c->phys, c->d_pd, c->d_seg_cell, L.d_org, c->q[0], c->T, L.NX, L.NY, h->eps, h->u_floor, L.d_tag);
    else k_amr_tag<2, false><<<n, SEG, 0, h->st>>>(c->phys, c->d_pd, c->d_seg_cell, L.d_org, c->q[0], c->T, L.NX, L.NY, h->eps, h->u_floor, L.d_tag);
  }
  ACU(cudaGetLastError());
  out.resize((size_t)L.NX * L.NY);
  ACU(cudaMemcpyAsync(out.data(), L.d_tag, out.size(), cudaMemcpyDeviceToHost, h->st));
  ACU(cudaStreamSynchronize(h->st));
  return DIS_OK;
}

// Rebuild levels 1 .. L - 1 (the oracle's regrid).
int regrid(dis_amr* h) {
  int rc;
  const int dim = h->dim, B = h->B;
  for (int l = 0; l + 1 < h->L; ++l) {
    if ((rc = prep_level(h, l))) return rc;  // level l is final (nested in the new level l - 1)
    dis_amr_level& C = h->lev[l];
    if (l >= 1) fill(h, l, C.c->q[0], 1.0, true);
    std::vector<unsigned char> t;
    if ((rc = tags_of(h, l, t))) return rc;
    const int NX = C.NX, NY = C.NY;
    // tags of owned cells, dilated (4-neighbour steps) within the owned cells
    std::vector<unsigned char> own((size_t)NX * NY);
    for (size_t k = 0; k < own.size(); ++k) own[k] = C.owner[k] >= 0;
    for (size_t k = 0; k < t.size(); ++k) t[k] = t[k] && own[k];
    for (int it = 0; it < h->buffer; ++it) {
      std::vector<unsigned char> o = t;
      for (int J = 0; J < NY; ++J)
        for (int I = 0; I < NX; ++I) {
          if (!t[(size_t)J * NX + I]) continue;
          if (I > 0) o[(size_t)J * NX + I - 1] = 1;
          if (I + 1 < NX) o[(size_t)J * NX + I + 1] = 1;
          if (dim == 2 && J > 0) o[(size_t)(J - 1) * NX + I] = 1;
          if (dim == 2 && J + 1 < NY) o[(size_t)(J + 1) * NX + I] = 1;
        }
      t = o;
    }
    for (size_t k = 0; k < t.size(); ++k) t[k] = t[k] && own[k];
    const int nbx = NX / B, nby = dim == 2 ? NY / B : 1, By = dim == 2 ? B : 1;
    std::vector<unsigned char> want((size_t)nbx * nby, 0), full((size_t)nbx * nby, 1);
    for (int J = 0; J < NY; ++J)
      for (int I = 0; I < NX; ++I) {
        const size_t b = (size_t)(J / By) * nbx + I / B;
        if (t[(size_t)J * NX + I]) want[b] = 1;
        if (!own[(size_t)J * NX + I]) full[b] = 0;
      }
    if (l >= 1)
      for (int bj = 0; bj < nby; ++bj)
        for (int bi = 0; bi < nbx; ++bi) {
          bool ok = true;
          for (int dj = (dim == 2 ? -1 : 0); dj <= (dim == 2 ? 1 : 0); ++dj)
            for (int di = -1; di <= 1; ++di) {
              const int x = bi + di, yb = bj + dj;
              if (x < 0 || x >= nbx || yb < 0 || yb >= nby) continue;
              ok = ok && full[(size_t)yb * nbx + x];
            }
          if (!ok) want[(size_t)bj * nbx + bi] = 0;
        }
    std::vector<int2> org;
    for (int bj = 0; bj < nby; ++bj)
      for (int bi = 0; bi < nbx; ++bi)
        if (want[(size_t)bj * nbx + bi]) org.push_back(make_int2(2 * B * bi, dim == 2 ? 2 * B * bj : 0));
    if (org.empty()) {
      for (size_t k = l + 1; k < h->lev.size(); ++k) free_level(h->lev[k]);
      h->lev.resize(l + 1);
      break;
    }
    if ((int)h->lev.size() > l + 1) {  // the same blocks: level l + 1 keeps its context and data
      const std::vector<int2>& oo = h->lev[l + 1].org;
      bool same = oo.size() == org.size();
      for (size_t b = 0; same && b < org.size(); ++b) same = oo[b].x == org[b].x && oo[b].y == org[b].y;
      if (same) continue;
    }
    dis_amr_level N;
    if ((rc = make_level(h, l + 1, org, N))) {
      free_level(N);
      return rc;
    }
    // data: blocks kept from the old level l + 1, else interpolated from level l
    std::vector<long long> pairs;
    std::vector<FillE> init;
    const bool had = (int)h->lev.size() > l + 1;
    const int S = 2 * B, Sy = dim == 2 ? S : 1;
    // the interpolation table needs level l + 1's owner map in h->lev: stage N there
    dis_amr_level old;
    if (had) old = h->lev[l + 1];
    else h->lev.emplace_back();
    h->lev[l + 1] = N;
    for (size_t b = 0; b < org.size(); ++b) {
      const int ob = had ? old.owner[(size_t)org[b].y * old.NX + org[b].x] : -1;
      for (int j = 0; j < Sy; ++j)
        for (int i = 0; i < S; ++i) {
          const long long dst = hidx(N.c, (int)b, i, j);
          if (ob >= 0) {
            pairs.push_back(hidx(old.c, ob, i, j));
            pairs.push_back(dst);
          } else {
            FillE e;
            if (!interp_entry(h, l + 1, org[b].x + i, org[b].y + j, dst, e))
              return AFAIL(DIS_ECUDA, "dis_amr: new block outside the coarser level");
            init.push_back(e);
          }
        }
    }
    if (!pairs.empty()) {
      long long* d = nullptr;
      if ((rc = upload(pairs, d, h->st))) return rc;
      const int n = (int)pairs.size() / 2;
      k_amr_copy<<<nblk(n), TPB, 0, h->st>>>(d, n, h->F.nf, old.c->q[0], old.c->T, N.c->q[0], N.c->T);
      ACU(cudaStreamSynchronize(h->st));
      cudaFree(d);
    }
    if (!init.empty()) {
      FillE* d = nullptr;
      if ((rc = upload(init, d, h->st))) return rc;
      k_amr_fill<<<nblk(init.size()), TPB, 0, h->st>>>(d, (int)init.size(), h->F, dim, N.c->q[0], N.c->T,
                                                         C.c->q[0], C.c->q[0], C.c->T, 1.0);
      ACU(cudaStreamSynchronize(h->st));
      cudaFree(d);
    }
    ACU(cudaGetLastError());
    if (had) free_level(old);
  }
  int rc2 = build_tables(h);
  if (rc2) return rc2;
  // defined ghost cells on every level (the CFL pass recovers them too)
  for (size_t l = 1; l < h->lev.size(); ++l) fill(h, (int)l, h->lev[l].c->q[0], 1.0, true);
  ACU(cudaStreamSynchronize(h->st));
  return DIS_OK;
}

int check_all(dis_amr* h, int* level, int* patch, int* cell) {
  for (size_t l = 0; l < h->lev.size(); ++l) {
    int p = -1, c = -1;
    const int rc = dis_check(h->lev[l].c, &p, &c);
    if (rc) {
      if (level) *level = (int)l;
      if (patch) *patch = p;
      if (cell) *cell = c;
      return rc;
    }
  }
  if (level) *level = -1;
  if (patch) *patch = -1;
  if (cell) *cell = -1;
  return DIS_OK;
}

}  // namespace

int dis_amr_create(int dim, const dis_patch* domain, int reactive_material, const dis_options* opt,
                   const dis_amr_options* a, void* stream, dis_amr** out) {
  if (!out || !domain || !opt || !a) return AFAIL(DIS_EINVAL, "dis_amr_create: NULL argument");
  *out = nullptr;
  if (opt->precision != DIS_FP64 || (opt->scheme != DIS_RK3 && opt->scheme != DIS_HANCOCK) ||
      (opt->geometry != DIS_PLANAR && opt->geometry != DIS_CYLINDRICAL) ||
      (opt->scheme == DIS_HANCOCK && opt->geometry != DIS_PLANAR))
    return AFAIL(DIS_EINVAL,
                 "dis_amr_create: the hierarchy is built for float64 SSP-RK3 (planar or cylindrical) and float64 "
                 "MUSCL-Hancock (planar)");
  if (opt->geometry == DIS_CYLINDRICAL && !(domain->x0 >= 0.0))
    return AFAIL(DIS_EINVAL, "dis_amr_create: cylindrical domain with x0 %g < 0 (a radius)", domain->x0);
  if (a->max_levels < 1 || a->max_levels > 4) return AFAIL(DIS_EINVAL, "dis_amr_create: max_levels in 1..4");
  if (a->block < 4) return AFAIL(DIS_EINVAL, "dis_amr_create: block must be >= 4");
  if (domain->nx % a->block || (dim == 2 && domain->ny % a->block))
    return AFAIL(DIS_EINVAL, "dis_amr_create: block %d does not divide the domain", a->block);
  if (a->buffer < 0 || a->regrid_every < 0 || !(a->u_floor >= 0.0) || !std::isfinite(a->eps))
    return AFAIL(DIS_EINVAL, "dis_amr_create: bad flagging options");
  for (int k = 0; k < (dim == 2 ? 4 : 2); ++k)
    if (domain->bc[k] < 0 || domain->bc[k] > 2) return AFAIL(DIS_EINVAL, "dis_amr_create: bad domain bc");
  dis_amr* h = new dis_amr();
  h->dim = dim;
  h->y = reactive_material;
  h->L = a->max_levels;
  h->B = a->block;
  h->eps = a->eps;
  h->buffer = a->buffer;
  h->u_floor = a->u_floor;
  h->regrid_every = a->regrid_every;
  h->dom = *domain;
  if (dim == 1) h->dom.ny = 1;
  h->opt = *opt;
  h->st = (cudaStream_t)stream;
  h->F = fields_of(dim, reactive_material >= 0);
  h->lev.reserve(4);  // no reallocation while references to levels are held
  h->lev.emplace_back();
  dis_amr_level& L0 = h->lev[0];
  int rc = dis_create(dim, 1, &h->dom, reactive_material, opt, stream, &L0.c);
  if (rc) {
    delete h;
    return rc;
  }
  L0.NX = h->dom.nx;
  L0.NY = dim == 2 ? h->dom.ny : 1;
  L0.org.assign(1, make_int2(0, 0));
  L0.owner.assign((size_t)L0.NX * L0.NY, 0);
  *out = h;
  return DIS_OK;
}

int dis_amr_set_materials(dis_amr* h, const dis_material* m, int n) {
  if (!h || !m) return AFAIL(DIS_EINVAL, "dis_amr_set_materials: NULL argument");
  for (auto& L : h->lev) {
    const int rc = dis_set_materials(L.c, m, n);
    if (rc) return rc;
  }
  for (int k = 0; k < 2; ++k) h->mats[k] = m[k];
  h->have_mats = true;
  return DIS_OK;
}

int dis_amr_set_state(dis_amr* h, const double* src, int kind) {
  if (!h || !src) return AFAIL(DIS_EINVAL, "dis_amr_set_state: NULL argument");
  if (!h->have_mats) return AFAIL(DIS_ESTATE, "dis_amr_set_state: materials first");
  for (size_t k = 1; k < h->lev.size(); ++k) free_level(h->lev[k]);
  h->lev.resize(1);
  cudaPointerAttributes at{};
  const bool dev = cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  int rc = dis_set_state(h->lev[0].c, kind, src, dev ? 1 : 0);
  if (rc) return rc;
  if ((rc = regrid(h))) return rc;
  h->have_state = true;
  h->steps = 0;
  return DIS_OK;
}

int dis_amr_step(dis_amr* h, int n_steps, double* dt_out) {
  if (!h) return AFAIL(DIS_EINVAL, "dis_amr_step: NULL argument");
  if (!h->have_state) return AFAIL(DIS_ESTATE, "dis_amr_step: no state");
  int rc;
  for (int s = 0; s < n_steps; ++s) {
    // the CFL rates of every level, one wait for all of them
    std::vector<std::vector<unsigned long long>> r(h->lev.size());
    for (size_t l = 0; l < h->lev.size(); ++l)
      if ((rc = dis_internal_rates_enqueue(h->lev[l].c))) return rc;
    for (size_t l = 0; l < h->lev.size(); ++l) {
      r[l].resize(h->lev[l].c->np);
      ACU(cudaMemcpyAsync(r[l].data(), h->lev[l].c->rate, sizeof(unsigned long long) * r[l].size(),
                          cudaMemcpyDeviceToHost, h->st));
    }
    ACU(cudaStreamSynchronize(h->st));
    double dt = 0.0;
    for (size_t l = 0; l < h->lev.size(); ++l) {
      double m = 0.0;
      for (unsigned long long bits : r[l]) {
        double v;
        std::memcpy(&v, &bits, sizeof v);
        m = std::max(m, v);
      }
      const double d = h->opt.cfl / m * (double)(1 << l);
      dt = l == 0 ? d : std::min(dt, d);
    }
    if ((rc = advance(h, 0, dt, 0.0, 1.0))) return rc;
    if (dt_out) dt_out[s] = dt;
    ++h->steps;
    if (h->regrid_every && h->steps % h->regrid_every == 0) {
      if ((rc = check_all(h, nullptr, nullptr, nullptr))) return rc;
      if ((rc = regrid(h))) return rc;
    }
  }
  ACU(cudaStreamSynchronize(h->st));
  if ((rc = check_all(h, nullptr, nullptr, nullptr))) return rc;
  return DIS_OK;
}

int dis_amr_levels(const dis_amr* h, int* n_levels, int* counts) {
  if (!h) return AFAIL(DIS_EINVAL, "dis_amr_levels: NULL argument");
  if (n_levels) *n_levels = (int)h->lev.size();
  if (counts)
    for (int l = 0; l < h->L; ++l) counts[l] = l < (int)h->lev.size() ? h->lev[l].c->np : 0;
  return DIS_OK;
}

int dis_amr_get_level(dis_amr* h, int level, int kind, double* dst, unsigned char* active) {
  if (!h || !dst) return AFAIL(DIS_EINVAL, "dis_amr_get_level: NULL argument");
  if (level < 0 || level >= (int)h->lev.size()) return AFAIL(DIS_EINVAL, "dis_amr_get_level: no level %d", level);
  dis_amr_level& L = h->lev[level];
  const int nf = h->F.nf;
  std::vector<double> buf((size_t)nf * L.c->ncells);
  int rc = dis_get_state(L.c, kind, buf.data(), 0);
  if (rc) return rc;
  const size_t plane = (size_t)L.NX * L.NY;
  for (size_t k = 0; k < (size_t)nf * plane; ++k) dst[k] = NAN;
  if (active) std::memset(active, 0, plane);
  size_t off = 0;
  for (int p = 0; p < L.c->np; ++p) {
    const int nx = L.c->pd[p].nx, ny = L.c->pd[p].ny;
    for (int c = 0; c < nf; ++c)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const size_t I = (size_t)L.org[p].x + i, J = (size_t)L.org[p].y + j;
          dst[c * plane + J * L.NX + I] = buf[off + ((size_t)c * ny + j) * nx + i];
          if (active && c == 0) active[J * L.NX + I] = 1;
        }
    off += (size_t)nf * nx * ny;
  }
  return DIS_OK;
}

int dis_amr_totals(dis_amr* h, double* out) {
  if (!h || !out) return AFAIL(DIS_EINVAL, "dis_amr_totals: NULL argument");
  const int nf = h->F.nf;
  for (int c = 0; c < nf; ++c) out[c] = 0.0;
  for (size_t l = 0; l < h->lev.size(); ++l) {
    dis_amr_level& L = h->lev[l];
    const size_t plane = (size_t)L.NX * L.NY;
    std::vector<double> d((size_t)nf * plane);
    std::vector<unsigned char> a(plane);
    int rc = dis_amr_get_level(h, (int)l, DIS_CONSERVATIVE, d.data(), a.data());
    if (rc) return rc;
    const double vol = L.c->pd[0].dx * (h->dim == 2 ? L.c->pd[0].dy : 1.0);
    const bool finer = l + 1 < h->lev.size();
    for (int J = 0; J < L.NY; ++J)
      for (int I = 0; I < L.NX; ++I) {
        if (!a[(size_t)J * L.NX + I]) continue;
        if (finer && h->lev[l + 1].owner[(size_t)(h->dim == 2 ? 2 * J : 0) * h->lev[l + 1].NX + 2 * I] >= 0) continue;
        for (int c = 0; c < nf; ++c) out[c] += d[c * plane + (size_t)J * L.NX + I] * vol;
      }
  }
  return DIS_OK;
}

int dis_amr_check(dis_amr* h, int* level, int* patch, int* cell) {
  if (!h) return AFAIL(DIS_EINVAL, "dis_amr_check: NULL argument");
  return check_all(h, level, patch, cell);
}

void dis_amr_destroy(dis_amr* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& L : h->lev) free_level(L);
  delete h;
}
