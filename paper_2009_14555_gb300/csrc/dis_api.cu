// dis_api.cu - host side of the C ABI declared in include/dis.h.
//
// A context owns the patch description, the host-built segment tables (the
// patch-batch schedule: every launch covers all patches of the batch), the
// workspace carve-up and the launch sequence of one time step:
//
//   per step:  memset(rate)                      (CFL mode only)
//   per stage: k_prim   (ghost map + primitive recovery [+ CFL rate max])
//              k_flux x (+ k_flux y in 2D)       (MUSCL/THINC-BVD + HLLC)
//              k_update (divergence, non-conservative terms, RK3 combination;
//                        last stage: plastic + reactive steps, status)
//
// The time step is computed on the device (dt = CFL / max rate) and read by
// the update kernels; dis_step therefore never synchronises with the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dis.h"
#include "ctx.cuh"
#include "query.cuh"

using namespace dis;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(DIS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Error text for the other translation units of the library.
int dis_internal_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}


// A Romenskii or JWL material in the context: the kernels carry the general
// closures (stiffened-gas contexts run kernels without that code).
bool general_closures(const dis_ctx* c) { return c->phys.m[0].eos != EOS_SG || c->phys.m[1].eos != EOS_SG; }

namespace {

int n_extra(int dim) { return dim == 2 ? 3 : 2; }

// Split rows of [lo, hi) into segments of at most SEG.
void add_row(std::vector<int4>& v, int patch, int row, int lo, int hi) {
  for (int s = lo; s < hi; s += SEG) v.push_back(make_int4(patch, row, s, std::min(SEG, hi - s)));
}

// Tile shapes of the fused FP32-bulk stage kernel (TX x TY cells; 256, 512
// and 256 threads in 2D): the face counts (TX+1) TY + TX (TY+1) fill two
// passes of the threads (511, 1007, 487 faces); the 32 x 15 tile recovers
// 1.66 halo cells per cell against 1.93 and 2.2 for the others.  1D tiles of
// NT - 6 cells make the halo (NT cells) and the faces (NT - 5) one pass each.
constexpr int kTiles2D[3][2] = {{16, 15}, {32, 15}, {32, 7}};
constexpr int kTiles1D[3] = {122, 250, 506};

void tile_tables(dis_ctx* c) {
  for (int v = 0; v < 3; ++v) {
    c->tiles[v].clear();
    c->tile0[v].assign(1, 0);
    const int TX = c->dim == 2 ? kTiles2D[v][0] : kTiles1D[v];
    const int TY = c->dim == 2 ? kTiles2D[v][1] : 1;
    for (int p = 0; p < c->np; ++p) {
      const PatchDev& d = c->pd[p];
      for (int j = 0; j < d.ny; j += TY)
        for (int i = 0; i < d.nx; i += TX) c->tiles[v].push_back(make_int4(p, i, j, 0));
      c->tile0[v].push_back((int)c->tiles[v].size());
    }
  }
  // launch order of the persistent batch kernel: longest problems first
  c->order.resize(c->np);
  for (int p = 0; p < c->np; ++p) c->order[p] = p;
  std::stable_sort(c->order.begin(), c->order.end(),
                   [&](int a, int b) { return c->pd[a].nx * c->pd[a].ny > c->pd[b].nx * c->pd[b].ny; });
}

void layout(dis_ctx* c) {
  const int g2 = c->dim == 2 ? NG : 0;
  long long off = 0, fx = 0, fy = 0, po = 0;
  c->pd.clear();
  c->seg_prim.clear();
  c->seg_fx.clear();
  c->seg_fy.clear();
  c->seg_cell.clear();
  c->seg_cell0.clear();
  for (int p = 0; p < c->np; ++p) {
    const dis_patch& P = c->patches[p];
    PatchDev d{};
    d.nx = P.nx;
    d.ny = c->dim == 2 ? P.ny : 1;
    d.pitch = P.nx + 2 * NG;
    d.rows = d.ny + 2 * g2;
    for (int k = 0; k < 4; ++k) d.bc[k] = P.bc[k];
    d.off = off;
    d.fxoff = fx;
    d.fyoff = fy;
    d.poff = po;
    d.dx = P.dx;
    d.x0 = c->phys.cyl ? P.x0 : 0.0;
    d.dy = c->dim == 2 ? P.dy : 1.0;
    off += ((long long)d.pitch * d.rows + 31) / 32 * 32;
    fx += (long long)d.ny * (d.nx + 1);
    if (c->dim == 2) fy += (long long)(d.ny + 1) * d.nx;
    po += (long long)c->nf * d.nx * d.ny;
    c->pd.push_back(d);
    for (int j = -g2; j < d.ny + g2; ++j) add_row(c->seg_prim, p, j, -NG, d.nx + NG);
    for (int j = 0; j < d.ny; ++j) add_row(c->seg_fx, p, j, 0, d.nx + 1);
    if (c->dim == 2)
      for (int j = 0; j <= d.ny; ++j) add_row(c->seg_fy, p, j, 0, d.nx);
    c->seg_cell0.push_back((int)c->seg_cell.size());
    for (int j = 0; j < d.ny; ++j) add_row(c->seg_cell, p, j, 0, d.nx);
  }
  c->seg_cell0.push_back((int)c->seg_cell.size());
  c->T = off;
  c->NFX = fx;
  c->NFY = fy;
  c->ncells = po / c->nf;
  tile_tables(c);
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  }
};

size_t carve(dis_ctx* c, char* base) {
  Carve k;
  const size_t T = (size_t)c->T;
  const size_t nfx = (size_t)(c->nf + n_extra(c->dim));
  size_t oq0 = 0, oq1 = 0, ow = 0, ofx = 0, ofy = 0, oe = 0;
  size_t o32[3] = {0, 0, 0};
  if (!c->fp32) {
    const size_t dpl = sizeof(double) * T;
    oq0 = k.take(c->nf * dpl);
    oq1 = k.take(c->nf * dpl);
    ow = k.take(c->nf * dpl);
    ofx = k.take(sizeof(double) * nfx * c->NFX);
    ofy = k.take(sizeof(double) * nfx * c->NFY);
    if (c->hancock) oe = k.take((size_t)2 * c->dim * c->nf * dpl);
  } else {
    // Runge-Kutta: q^n and two stage buffers; MUSCL-Hancock: a pair that
    // alternates from step to step
    for (int b = 0; b < (c->hancock ? 2 : 3); ++b) o32[b] = k.take((c->nf + 1) * sizeof(float) * T);
  }
  size_t oio = k.take(sizeof(double) * (size_t)c->nf * c->ncells);
  size_t ort = k.take(2 * sizeof(unsigned long long) * c->np);  // rate of q^n, of q^{n+1}
  size_t odf = k.take(sizeof(double) * c->np);
  size_t odl = k.take(sizeof(double) * c->np);
  size_t ost = k.take(sizeof(int) * 4);
  size_t opd = k.take(sizeof(PatchDev) * c->np);
  size_t oqp = k.take(sizeof(double) * NQ * c->seg_cell.size());  // dis_query partials
  size_t oqo = k.take(sizeof(double) * NQ);
  size_t os1 = k.take(sizeof(int4) * c->seg_prim.size());
  size_t os2 = k.take(sizeof(int4) * c->seg_fx.size());
  size_t os3 = k.take(sizeof(int4) * std::max<size_t>(1, c->seg_fy.size()));
  size_t os4 = k.take(sizeof(int4) * c->seg_cell.size());
  size_t ot[3], ot0[3];
  for (int v = 0; v < 3; ++v) ot[v] = k.take(sizeof(int4) * std::max<size_t>(1, c->tiles[v].size()));
  for (int v = 0; v < 3; ++v) ot0[v] = k.take(sizeof(int) * (size_t)(c->np + 1));
  const size_t oord = k.take(sizeof(int) * (size_t)c->np);
  if (base) {
    for (int v = 0; v < 3; ++v) {
      c->d_tiles[v] = (int4*)(base + ot[v]);
      c->d_tile0[v] = (int*)(base + ot0[v]);
    }
    c->d_order = (int*)(base + oord);
    if (!c->fp32) {
      c->q[0] = (double*)(base + oq0);
      c->q[1] = (double*)(base + oq1);
      c->W = (double*)(base + ow);
      c->Fx = (double*)(base + ofx);
      c->Fy = (double*)(base + ofy);
      c->E = c->hancock ? (double*)(base + oe) : nullptr;
    } else {
      for (int b = 0; b < 3; ++b) c->q32[b] = (c->hancock && b == 2) ? nullptr : (float*)(base + o32[b]);
      c->q32_home = c->q32[0];
    }
    c->io = (double*)(base + oio);
    c->rate = (unsigned long long*)(base + ort);
    c->dtfix = (double*)(base + odf);
    c->dtlast = (double*)(base + odl);
    c->status = (int*)(base + ost);
    c->d_pd = (PatchDev*)(base + opd);
    c->qpart = (double*)(base + oqp);
    c->qout = (double*)(base + oqo);
    c->d_seg_prim = (int4*)(base + os1);
    c->d_seg_fx = (int4*)(base + os2);
    c->d_seg_fy = (int4*)(base + os3);
    c->d_seg_cell = (int4*)(base + os4);
  }
  return k.off;
}

int ensure_ws(dis_ctx* c) {
  if (c->ws_ready) return DIS_OK;
  if (!c->ws) {
    const size_t need = carve(c, nullptr);
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      const cudaError_t e = cudaGetLastError();
      return fail(DIS_ENOMEM, "workspace: cannot allocate %zu bytes (%s)", need, cudaGetErrorString(e));
    }
    c->ws = (char*)p;
    c->ws_bytes = need;
    c->ws_owned = true;
  }
  carve(c, c->ws);
  CU(cudaMemcpyAsync(c->d_pd, c->pd.data(), sizeof(PatchDev) * c->np, cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_seg_prim, c->seg_prim.data(), sizeof(int4) * c->seg_prim.size(),
                     cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_seg_fx, c->seg_fx.data(), sizeof(int4) * c->seg_fx.size(),
                     cudaMemcpyHostToDevice, c->stream));
  if (!c->seg_fy.empty())
    CU(cudaMemcpyAsync(c->d_seg_fy, c->seg_fy.data(), sizeof(int4) * c->seg_fy.size(),
                       cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_seg_cell, c->seg_cell.data(), sizeof(int4) * c->seg_cell.size(),
                     cudaMemcpyHostToDevice, c->stream));

  for (int v = 0; v < 3; ++v) {
    CU(cudaMemcpyAsync(c->d_tiles[v], c->tiles[v].data(), sizeof(int4) * c->tiles[v].size(),
                       cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_tile0[v], c->tile0[v].data(), sizeof(int) * c->tile0[v].size(),
                       cudaMemcpyHostToDevice, c->stream));
  }
  CU(cudaMemcpyAsync(c->d_order, c->order.data(), sizeof(int) * c->order.size(), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, c->stream));
  // The tables above come from host vectors that outlive this call; make sure
  // the copies have finished before the caller may touch them.
  CU(cudaStreamSynchronize(c->stream));
  c->ws_ready = true;
  return DIS_OK;
}

StepArgs base_args(dis_ctx* c) {
  StepArgs a{};
  a.pd = c->d_pd;
  a.T = c->T;
  a.NFX = c->NFX;
  a.NFY = c->NFY;
  a.W = c->W;
  a.Fx = c->Fx;
  a.Fy = c->Fy;
  a.E = c->E;
  a.rate = c->rate;
  a.dtlast = c->dtlast;
  a.status = c->status;
  return a;
}

StepArgs32 base_args32(dis_ctx* c) {
  StepArgs32 a{};
  a.pd = c->d_pd;
  a.T = c->T;
  a.NFX = c->NFX;
  a.NFY = c->NFY;
  a.rate = c->rate;
  a.rate_next = c->rate + c->np;
  a.dtlast = c->dtlast;
  a.status = c->status;
  a.dkap = c->phys.m[0].kap - c->phys.m[1].kap;
  return a;
}

template <int DIM, bool RX, int TX, int TY, int NT, int MINB, bool CYL, int LIM = 0, bool GEN = false>
void stage_fused_c(dis_ctx* c, cudaStream_t st, StepArgs32& a, int shape) {
  constexpr size_t smem = fused32_smem<DIM, RX, TX, TY>();
  static bool attr_set = false;  // per instantiation, per process
  if (!attr_set) {
    cudaFuncSetAttribute(k_stage32<DIM, RX, TX, TY, NT, MINB, CYL, LIM, GEN>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_stage32<DIM, RX, TX, TY, NT, MINB, CYL, LIM, GEN>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_set = true;
  }
  k_stage32<DIM, RX, TX, TY, NT, MINB, CYL, LIM, GEN><<<(unsigned)c->tiles[shape].size(), NT, smem, st>>>(
      c->phys, c->physf, a, c->d_tiles[shape]);
}

// Planar and cylindrical contexts run separate instantiations, so the
// geometric source costs the planar kernels nothing.
template <int DIM, bool RX, int TX, int TY, int NT, int MINB, int LIM = 0, bool GEN = false>
void stage_fused(dis_ctx* c, cudaStream_t st, StepArgs32& a, int shape) {
  if (c->phys.cyl) stage_fused_c<DIM, RX, TX, TY, NT, MINB, true, LIM, GEN>(c, st, a, shape);
  else stage_fused_c<DIM, RX, TX, TY, NT, MINB, false, LIM, GEN>(c, st, a, shape);
}

// FP32-bulk stage variants v = shape + 3 budget: the 3 tile shapes x two
// register budgets (2D: 768 or 1024 resident threads per SM requested from
// the register allocator; 1D: no limit, or 64 registers per thread).  The
// limiter and the closure family are compile-time choices of the kernels:
// stiffened-gas minmod contexts have every variant; van Leer contexts and
// contexts with general closures one (1D: the 250-cell tile; 2D: the 32 x 7
// tile at 1024 threads per SM for van Leer, at 768 for the general closures,
// whose code would spill at 64 registers; the general-closure kernel takes
// the limiter at run time).
//
// MUSCL-Hancock contexts: variant = tile shape (0 .. 2); van Leer and general
// closures the 32 x 7 tile (2D) or the 250-cell tile (1D).
int single_variant(const dis_ctx* c) {
  if (c->hancock) return c->dim == 2 ? 2 : 1;
  return c->dim == 2 ? (general_closures(c) ? 2 : 5) : 1;
}
bool variant_valid(const dis_ctx* c, int v) {
  if (c->phys.limiter || general_closures(c)) return v == single_variant(c);
  return v >= 0 && v < (c->hancock ? 3 : DIS_NVARIANTS);
}

// One FP32-bulk MUSCL-Hancock step of variant v: q32[0] -> q32[1] (the
// caller exchanges the two after enqueueing it; the tuner times it as is).
void hancock32_step(dis_ctx* c, cudaStream_t st, StepArgs32& a, int v) {
  a.src = c->q32[0];
  a.qn = c->q32[0];
  a.dst = c->q32[1];
  a.a = 0.0;
  a.b = 1.0;
  a.last = 1;
  if (c->dim == 2) hancock32_step_2d(c, st, a, v);
  else hancock32_step_1d(c, st, a, v);
}

// The state-buffer parity of an FP32-bulk MUSCL-Hancock context (1: the
// state is in the buffer carved second) and the exchange after each step.
bool any_graph(const dis_ctx* c) {
  for (cudaGraphExec_t g : c->graph)
    if (g) return true;
  return false;
}

// Destroy the captured step graphs (after the replays in flight).
void drop_graphs(dis_ctx* c) {
  if (any_graph(c)) cudaStreamSynchronize(c->stream);
  for (cudaGraphExec_t& g : c->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int h_parity(const dis_ctx* c) { return c->fp32 && c->hancock && c->q32[0] != c->q32_home ? 1 : 0; }
void h_swap(dis_ctx* c) { std::swap(c->q32[0], c->q32[1]); }

// MINB: resident CTAs of 256 threads per SM requested (3 or 4); the
// 512-thread tile asks for half as many.
template <int DIM, bool RX, int MINB>
void stage_kernel_2d(dis_ctx* c, cudaStream_t st, StepArgs32& a, int shape) {
  if (shape == 0) stage_fused<DIM, RX, 16, 15, 256, MINB>(c, st, a, shape);
  else if (shape == 1) stage_fused<DIM, RX, 32, 15, 512, MINB / 2>(c, st, a, shape);
  else stage_fused<DIM, RX, 32, 7, 256, MINB>(c, st, a, shape);
}

// The stage kernel of variant v.
template <int DIM, bool RX>
void stage_kernel_v(dis_ctx* c, cudaStream_t st, StepArgs32& a, int v) {
  const int shape = v % 3;
  if (general_closures(c)) {  // the one general-closure instantiation
    if constexpr (DIM == 2) stage_fused<DIM, RX, 32, 7, 256, 3, -1, true>(c, st, a, 2);
    else stage_fused<DIM, RX, 250, 1, 256, 1, -1, true>(c, st, a, 1);
    return;
  }
  if (c->phys.limiter) {  // van Leer: the one instantiation
    if constexpr (DIM == 2) stage_fused<DIM, RX, 32, 7, 256, 4, 1>(c, st, a, 2);
    else stage_fused<DIM, RX, 250, 1, 256, 1, 1>(c, st, a, 1);
    return;
  }
  if constexpr (DIM == 2) {
    if (v >= 3) stage_kernel_2d<DIM, RX, 4>(c, st, a, shape);
    else stage_kernel_2d<DIM, RX, 3>(c, st, a, shape);
  } else if (v < 3) {
    if (shape == 0) stage_fused<DIM, RX, 122, 1, 128, 1>(c, st, a, shape);
    else if (shape == 1) stage_fused<DIM, RX, 250, 1, 256, 1>(c, st, a, shape);
    else stage_fused<DIM, RX, 506, 1, 512, 1>(c, st, a, shape);
  } else {  // 1024 threads per SM requested: at most 64 registers per thread
    if (shape == 0) stage_fused<DIM, RX, 122, 1, 128, 8>(c, st, a, shape);
    else if (shape == 1) stage_fused<DIM, RX, 250, 1, 256, 4>(c, st, a, shape);
    else stage_fused<DIM, RX, 506, 1, 512, 2>(c, st, a, shape);
  }
}

// CFL rate of q^n (buffer 0) into rate (zeroed first): the first step after
// the state was set; later steps take it from the last stage of the step
// before.
template <int DIM, bool RX>
void cfl_pass32(dis_ctx* c, cudaStream_t st, unsigned long long* rate) {
  StepArgs32 a = base_args32(c);
  a.src = c->q32[0];
  cudaMemsetAsync(rate, 0, sizeof(unsigned long long) * c->np, st);
  k_cfl32<DIM, RX><<<(unsigned)c->seg_cell.size(), SEG, 0, st>>>(c->phys, c->physf, a, rate, c->d_seg_cell);
}

// Persistent 1D batch kernel (FP32-bulk), variant v: tile length v % 3,
// 64 registers per thread for v >= 3; n steps in one launch, one CTA per
// problem.  scratch_last (tuning, n = 1): the step ends in buffer 1.
template <bool RX, int TX, int NT, int MINB, bool CYL, int LIM = 0, bool GEN = false>
void batch_fused_c(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int n, int scratch_last, int shape) {
  constexpr size_t smem = fused32_smem<1, RX, TX, 1>();
  static bool attr_set = false;  // per instantiation, per process
  if (!attr_set) {
    cudaFuncSetAttribute(k_batch32<RX, TX, NT, MINB, CYL, LIM, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_batch32<RX, TX, NT, MINB, CYL, LIM, GEN>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr_set = true;
  }
  Bufs32 b;
  for (int k = 0; k < 3; ++k) b.q[k] = c->q32[k];
  k_batch32<RX, TX, NT, MINB, CYL, LIM, GEN><<<(unsigned)c->np, NT, smem, st>>>(
      c->phys, c->physf, a, b, c->rate, c->d_order, c->d_tile0[shape], c->d_tiles[shape], n, scratch_last,
      c->rate_valid ? 1 : 0);
}

template <bool RX, int TX, int NT, int MINB, int LIM = 0, bool GEN = false>
void batch_fused(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int n, int scratch_last, int shape) {
  if (c->phys.cyl) batch_fused_c<RX, TX, NT, MINB, true, LIM, GEN>(c, st, a, n, scratch_last, shape);
  else batch_fused_c<RX, TX, NT, MINB, false, LIM, GEN>(c, st, a, n, scratch_last, shape);
}

template <bool RX>
void batch_kernel_v(dis_ctx* c, cudaStream_t st, const StepArgs32& a, int n, int scratch_last, int v) {
  const int shape = v % 3;
  if (general_closures(c)) {  // the one general-closure instantiation (250-cell tiles)
    batch_fused<RX, 250, 256, 1, -1, true>(c, st, a, n, scratch_last, 1);
    return;
  }
  if (c->phys.limiter) {  // van Leer: the one instantiation (250-cell tiles)
    batch_fused<RX, 250, 256, 1, 1>(c, st, a, n, scratch_last, 1);
    return;
  }
  if (v < 3) {
    if (shape == 0) batch_fused<RX, 122, 128, 1>(c, st, a, n, scratch_last, shape);
    else if (shape == 1) batch_fused<RX, 250, 256, 1>(c, st, a, n, scratch_last, shape);
    else batch_fused<RX, 506, 512, 1>(c, st, a, n, scratch_last, shape);
  } else {
    if (shape == 0) batch_fused<RX, 122, 128, 8>(c, st, a, n, scratch_last, shape);
    else if (shape == 1) batch_fused<RX, 250, 256, 4>(c, st, a, n, scratch_last, shape);
    else batch_fused<RX, 506, 512, 2>(c, st, a, n, scratch_last, shape);
  }
}

// Buffers of the FP32-bulk stages: q^n (0) -> q1 (1) -> q2 (2) -> q^{n+1} (0).
// A stage kernel reads the halo of its source from neighbouring tiles, so it
// must not write that source.  The last stage overwrites q^n cell by cell,
// read only at the same cell.  scratch_last: the tuner's full step ends in
// buffer 1 instead of q^n.
template <int DIM, bool RX>
void set_stage_args32(dis_ctx* c, StepArgs32& a, int stg, bool scratch_last = false) {
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
  const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
  const int src = stg, dst = stg == 2 ? (scratch_last ? 1 : 0) : stg + 1;
  a.src = c->q32[src];
  a.qn = c->q32[0];
  a.dst = c->q32[dst];
  a.a = ca[stg];
  a.b = cb[stg];
  a.last = stg == 2;
}

// Autotuner: time one full step of every variant with the last stage
// writing a scratch buffer (the state is untouched) and keep the fastest.
// The CFL rate of q^n is taken first (if it is not known); dt is then the
// step's dt.  The trial steps' last stages accumulate into the next-step
// rate buffer, which every real step clears first.
template <int DIM, bool RX>
int autotune32(dis_ctx* c) {
  StepArgs32 a = base_args32(c);
  a.dtfix = nullptr;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  if (!c->rate_valid) {
    cfl_pass32<DIM, RX>(c, c->stream, c->rate);
    c->rate_valid = true;
  }
  double best = 1e30;
  int bv = 0;
  for (int v = 0; v < DIS_NVARIANTS; ++v) {
    if (!variant_valid(c, v)) continue;
    for (int rep = 0; rep < 3; ++rep) {  // rep 0 warms up
      CU(cudaEventRecord(e0, c->stream));
      if (c->hancock) {
        hancock32_step(c, c->stream, a, v);
      } else {
        for (int stg = 0; stg < 3; ++stg) {
          set_stage_args32<DIM, RX>(c, a, stg, true);
          stage_kernel_v<DIM, RX>(c, c->stream, a, v);
        }
      }
      CU(cudaEventRecord(e1, c->stream));
      CU(cudaEventSynchronize(e1));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1) c->tune_ms[v] = ms;
      if (rep == 2) c->tune_ms[v] = 0.5 * (c->tune_ms[v] + ms);
    }
    if (c->tune_ms[v] < best) { best = c->tune_ms[v]; bv = v; }
  }
  // 1D: the persistent batch kernel, one step per variant (the last stage
  // writes buffer 1), against the best per-step schedule
  double best_b = 1e30;
  int bb = -1;
  if constexpr (DIM == 1) {
    if (c->schedule_req != 0) {
      StepArgs32 ab = base_args32(c);
      ab.dtfix = nullptr;
      for (int v = 0; v < DIS_NVARIANTS; ++v) {
        c->tune_batch_ms[v] = 0.0;
        if (!variant_valid(c, v)) continue;
        for (int rep = 0; rep < 3; ++rep) {
          CU(cudaEventRecord(e0, c->stream));
          if (c->hancock) hancock32_batch_1d(c, c->stream, ab, c->q32[0], c->q32[1], 1, 1, v);
          else batch_kernel_v<RX>(c, c->stream, ab, 1, 1, v);
          CU(cudaEventRecord(e1, c->stream));
          CU(cudaEventSynchronize(e1));
          float ms = 0.f;
          CU(cudaEventElapsedTime(&ms, e0, e1));
          if (rep == 1) c->tune_batch_ms[v] = ms;
          if (rep == 2) c->tune_batch_ms[v] = 0.5 * (c->tune_batch_ms[v] + ms);
        }
        if (c->tune_batch_ms[v] < best_b) { best_b = c->tune_batch_ms[v]; bb = v; }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(cudaGetLastError());
  if (c->schedule_req == 1 || (c->schedule_req < 0 && bb >= 0 && best_b < best)) {
    c->variant = bb;
    c->schedule = 1;
  } else {
    c->variant = bv;
    c->schedule = 0;
  }
  return DIS_OK;
}

// Enqueue the kernels of one time step on stream `st`; returns the number of
// kernel launches.
template <int DIM, bool RX>
long long launch_step(dis_ctx* c, cudaStream_t st, bool fixed) {
  if (c->fp32) {
    // the three stages read the rate of q^n (rate) and the last one
    // accumulates the rate of q^{n+1} (rate + np), copied over at the end
    // (MUSCL-Hancock: one kernel, q32[0] -> q32[1]; the caller exchanges them)
    StepArgs32 a = base_args32(c);
    a.dtfix = fixed ? c->dtfix : nullptr;
    const int v = c->variant < 0 ? 0 : c->variant;
    cudaMemsetAsync(c->rate + c->np, 0, sizeof(unsigned long long) * c->np, st);
    if (c->hancock) {
      hancock32_step(c, st, a, v);
    } else {
      for (int stg = 0; stg < 3; ++stg) {
        set_stage_args32<DIM, RX>(c, a, stg);
        stage_kernel_v<DIM, RX>(c, st, a, v);
      }
    }
    cudaMemcpyAsync(c->rate, c->rate + c->np, sizeof(unsigned long long) * c->np, cudaMemcpyDeviceToDevice, st);
    return c->hancock ? 1 : 3;
  }
  StepArgs a = base_args(c);
  a.dtfix = fixed ? c->dtfix : nullptr;
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
  const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
  const unsigned np = (unsigned)c->seg_prim.size(), nfx = (unsigned)c->seg_fx.size(),
                 nfy = (unsigned)c->seg_fy.size(), nc = (unsigned)c->seg_cell.size();
  long long launches = 0;
  if (!fixed) cudaMemsetAsync(c->rate, 0, sizeof(unsigned long long) * c->np, st);
  if (c->hancock) {  // single stage: q^{n+1} = S(q^n - dt D_H(q^n)), in place
    a.qsrc = c->q[0];
    a.qn = c->q[0];
    a.qdst = c->q[0];
    a.a = 0.0;
    a.b = 1.0;
    a.last = 1;
    k_prim<DIM, RX><<<np, SEG, 0, st>>>(c->phys, a, c->d_seg_prim, fixed ? 0 : 1);
    k_hancock<DIM, RX><<<np, SEG, 0, st>>>(c->phys, a, c->d_seg_prim);
    k_flux_h<DIM, RX, 0><<<nfx, SEG, 0, st>>>(c->phys, a, c->d_seg_fx);
    launches += 3;
    if constexpr (DIM == 2) {
      k_flux_h<DIM, RX, 1><<<nfy, SEG, 0, st>>>(c->phys, a, c->d_seg_fy);
      ++launches;
    }
    k_update<DIM, RX><<<nc, SEG, 0, st>>>(c->phys, a, c->d_seg_cell);
    return launches + 1;
  }
  for (int stg = 0; stg < 3; ++stg) {
    a.qsrc = stg == 0 ? c->q[0] : c->q[1];
    a.qn = c->q[0];
    a.qdst = stg == 2 ? c->q[0] : c->q[1];
    a.a = ca[stg];
    a.b = cb[stg];
    a.last = stg == 2;
    k_prim<DIM, RX><<<np, SEG, 0, st>>>(c->phys, a, c->d_seg_prim, (!fixed && stg == 0) ? 1 : 0);
    k_flux<DIM, RX, 0><<<nfx, SEG, 0, st>>>(c->phys, a, c->d_seg_fx);
    launches += 2;
    if constexpr (DIM == 2) {
      k_flux<DIM, RX, 1><<<nfy, SEG, 0, st>>>(c->phys, a, c->d_seg_fy);
      ++launches;
    }
    k_update<DIM, RX><<<nc, SEG, 0, st>>>(c->phys, a, c->d_seg_cell);
    ++launches;
  }
  return launches;
}

// One step with CUDA events around every kernel (no graph), accumulating the
// device time of each kernel class: 0 prim, 1 flux x, 2 flux y, 3 update.
template <int DIM, bool RX>
int timed_steps(dis_ctx* c, int n_steps, double* ms) {
  StepArgs a = base_args(c);
  a.dtfix = nullptr;
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
  const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
  const unsigned np = (unsigned)c->seg_prim.size(), nfx = (unsigned)c->seg_fx.size(),
                 nfy = (unsigned)c->seg_fy.size(), nc = (unsigned)c->seg_cell.size();
  cudaEvent_t ev[5];
  for (int k = 0; k < 5; ++k) CU(cudaEventCreate(&ev[k]));
  double acc[4] = {0, 0, 0, 0};
  if (c->fp32) {
    // slot 0: the CFL pass of a first step (timed on the next-step rate
    // buffer, which every step clears first); slot 1: the stage kernel
    if (c->variant < 0) {
      const int rc = autotune32<DIM, RX>(c);
      if (rc) return rc;
    }
    const int v = c->variant;
    StepArgs32 a32 = base_args32(c);
    if (!c->rate_valid) {
      cfl_pass32<DIM, RX>(c, c->stream, c->rate);
      c->rate_valid = true;
    }
    for (int s = 0; s < n_steps; ++s) {
      float t = 0.f;
      CU(cudaEventRecord(ev[0], c->stream));
      cfl_pass32<DIM, RX>(c, c->stream, c->rate + c->np);
      CU(cudaEventRecord(ev[1], c->stream));
      CU(cudaEventSynchronize(ev[1]));
      CU(cudaEventElapsedTime(&t, ev[0], ev[1]));
      acc[0] += 3.0 * t;
      CU(cudaMemsetAsync(c->rate + c->np, 0, sizeof(unsigned long long) * c->np, c->stream));
      for (int stg = 0; stg < 3; ++stg) {
        set_stage_args32<DIM, RX>(c, a32, stg);
        CU(cudaEventRecord(ev[1], c->stream));
        stage_kernel_v<DIM, RX>(c, c->stream, a32, v);
        CU(cudaEventRecord(ev[2], c->stream));
        CU(cudaEventSynchronize(ev[2]));
        CU(cudaEventElapsedTime(&t, ev[1], ev[2]));
        acc[1] += t;
      }
      CU(cudaMemcpyAsync(c->rate, c->rate + c->np, sizeof(unsigned long long) * c->np, cudaMemcpyDeviceToDevice,
                         c->stream));
    }
    n_steps = -n_steps;  // skip the float64 loop below
  }
  for (int s = 0; s < n_steps; ++s) {
    CU(cudaMemsetAsync(c->rate, 0, sizeof(unsigned long long) * c->np, c->stream));
    for (int stg = 0; stg < 3; ++stg) {
      a.qsrc = stg == 0 ? c->q[0] : c->q[1];
      a.qn = c->q[0];
      a.qdst = stg == 2 ? c->q[0] : c->q[1];
      a.a = ca[stg];
      a.b = cb[stg];
      a.last = stg == 2;
      CU(cudaEventRecord(ev[0], c->stream));
      k_prim<DIM, RX><<<np, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, stg == 0 ? 1 : 0);
      CU(cudaEventRecord(ev[1], c->stream));
      k_flux<DIM, RX, 0><<<nfx, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fx);
      CU(cudaEventRecord(ev[2], c->stream));
      if constexpr (DIM == 2) k_flux<DIM, RX, 1><<<nfy, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fy);
      CU(cudaEventRecord(ev[3], c->stream));
      k_update<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_cell);
      CU(cudaEventRecord(ev[4], c->stream));
      CU(cudaEventSynchronize(ev[4]));
      for (int k = 0; k < 4; ++k) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
        acc[k] += t;
      }
    }
  }
  CU(cudaGetLastError());
  for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
  const double nl = 3.0 * (n_steps < 0 ? -n_steps : n_steps);
  for (int k = 0; k < 4; ++k) ms[k] = acc[k] / nl;
  return DIS_OK;
}

template <int DIM, bool RX>
int run_steps(dis_ctx* c, int n_steps, bool fixed) {
  const int mode = fixed ? 1 : 0;
  if (c->fp32 && c->variant < 0) {
    const int rc = autotune32<DIM, RX>(c);
    if (rc) return rc;
  }
  if constexpr (DIM == 1) {
    const int sched = c->schedule_req >= 0 ? c->schedule_req : std::max(c->schedule, 0);
    if (c->fp32 && sched == 1) {  // all n steps in one persistent launch
      StepArgs32 a = base_args32(c);
      a.dtfix = fixed ? c->dtfix : nullptr;
      if (c->hancock) {
        hancock32_batch_1d(c, c->stream, a, c->q32[0], c->q32[1], n_steps, 0, c->variant);
        if (n_steps & 1) h_swap(c);
      } else {
        batch_kernel_v<RX>(c, c->stream, a, n_steps, 0, c->variant);
      }
      CU(cudaGetLastError());
      c->rate_valid = true;
      c->launches = 1;
      return DIS_OK;
    }
  }
  long long first = 0;
  if (c->fp32 && !c->rate_valid) {  // the rate of q^n for the first step
    cfl_pass32<DIM, RX>(c, c->stream, c->rate);
    c->rate_valid = true;
    first = 1;
  }
  const bool alternate = c->fp32 && c->hancock;  // the state moves to the other buffer each step
  if (!c->use_graphs) {
    long long l = first;
    for (int s = 0; s < n_steps; ++s) {
      l += launch_step<DIM, RX>(c, c->stream, fixed);
      if (alternate) h_swap(c);
    }
    CU(cudaGetLastError());
    c->launches = l;
    return DIS_OK;
  }
  if (!c->cap) {
    CU(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  }
  // captured on the private stream (one graph per mode and buffer parity),
  // replayed on the caller's stream (no cross-stream waits between steps)
  long long l = first;
  for (int s = 0; s < n_steps; ++s) {
    const int gi = mode + 2 * h_parity(c);
    if (!c->graph[gi]) {
      cudaGraph_t g = nullptr;
      CU(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
      const long long lc = launch_step<DIM, RX>(c, c->cap, fixed);
      const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
      if (e != cudaSuccess) return fail(DIS_ECUDA, "step capture failed: %s", cudaGetErrorString(e));
      const cudaError_t e2 = cudaGraphInstantiate(&c->graph[gi], g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) return fail(DIS_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e2));
      c->graph_launches[gi] = lc;
    }
    CU(cudaGraphLaunch(c->graph[gi], c->stream));
    l += c->graph_launches[gi];
    if (alternate) h_swap(c);
  }
  c->launches = l;
  return DIS_OK;
}

int dispatch_steps(dis_ctx* c, int n, bool fixed) {
  const bool rx = c->y >= 0;
  if (c->dim == 1) return rx ? run_steps<1, true>(c, n, fixed) : run_steps<1, false>(c, n, fixed);
  return rx ? run_steps<2, true>(c, n, fixed) : run_steps<2, false>(c, n, fixed);
}

// Segments of the transfer: all patches (patch < 0) or one patch, whose
// packed array then starts at src / dst (base = its packed offset).
struct SegRange {
  const int4* segs;
  unsigned n;
  long long base;
};
SegRange seg_range(const dis_ctx* c, int patch) {
  if (patch < 0) return {c->d_seg_cell, (unsigned)c->seg_cell.size(), 0};
  const int b = c->seg_cell0[patch], e = c->seg_cell0[patch + 1];
  return {c->d_seg_cell + b, (unsigned)(e - b), c->pd[patch].poff};
}

template <int DIM, bool RX>
int do_unpack(dis_ctx* c, const double* src, int prim, int patch = -1) {
  const SegRange r = seg_range(c, patch);
  if (c->fp32) {
    k_unpack32<DIM, RX><<<r.n, SEG, 0, c->stream>>>(c->phys, c->d_pd, r.segs, src, c->q32[0], c->T, prim, r.base);
    CU(cudaGetLastError());
    c->rate_valid = false;
    return DIS_OK;
  }
  k_unpack<DIM, RX><<<r.n, SEG, 0, c->stream>>>(c->phys, c->d_pd, r.segs, src, c->q[0], c->T, prim, r.base);
  CU(cudaGetLastError());
  return DIS_OK;
}

template <int DIM, bool RX>
int do_pack(dis_ctx* c, double* dst, int prim, int patch = -1) {
  const SegRange r = seg_range(c, patch);
  if (c->fp32) {
    if (prim)
      k_pack_prim32<DIM, RX><<<r.n, SEG, 0, c->stream>>>(c->phys, c->physf, c->d_pd, r.segs, c->q32[0], dst, c->T,
                                                         r.base);
    else
      k_pack32<DIM, RX><<<r.n, SEG, 0, c->stream>>>(c->phys, c->d_pd, r.segs, c->q32[0], dst, c->T, r.base);
    CU(cudaGetLastError());
    return DIS_OK;
  }
  const double* from = c->q[0];
  if (prim) {
    StepArgs a = base_args(c);
    a.qsrc = c->q[0];
    k_prim<DIM, RX><<<(unsigned)c->seg_prim.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, 0);
    from = c->W;
  }
  k_pack<DIM, RX><<<r.n, SEG, 0, c->stream>>>(c->d_pd, r.segs, from, dst, c->T, r.base);
  CU(cudaGetLastError());
  return DIS_OK;
}

// Totals, phi range (query.cuh) of the current state into c->qout (device).
template <int DIM, bool RX>
int do_query(dis_ctx* c) {
  const unsigned n = (unsigned)c->seg_cell.size();
  k_query_partial<DIM, RX><<<n, SEG, 0, c->stream>>>(c->phys, c->d_pd, c->d_seg_cell, c->fp32 ? nullptr : c->q[0],
                                                     c->fp32 ? c->q32[0] : nullptr, c->T, c->qpart);
  k_query_final<<<1, SEG, 0, c->stream>>>(c->qpart, n, c->qout);
  CU(cudaGetLastError());
  return DIS_OK;
}

MatDev to_dev(const dis_material& m) {
  MatDev d{};
  d.gamma = m.gamma;
  d.pinf = m.p_inf;
  d.einf = m.e_inf;
  d.G = m.G;
  d.sigy = m.sigma_y;
  d.chi0 = m.chi0;
  d.Q = m.reactive ? m.Q : 0.0;  // the history row of a Johnson-Cook material releases no heat
  d.cv = m.cv;
  d.A = m.A;
  d.Tact = m.T_act;
  d.plastic = m.plastic;
  d.reactive = m.reactive;
  d.law = m.reactive ? m.rate_law : 0;
  d.eos = m.eos;
  d.rho0 = m.rho0;
  d.K0 = m.K0;
  d.ar = m.alpha;
  d.br = m.beta;
  d.jA = m.jwl_A;
  d.jB = m.jwl_B;
  d.jR1 = m.jwl_R1;
  d.jR2 = m.jwl_R2;
  d.two = m.reactive && m.prod_gamma > 0.0 ? 1 : 0;
  d.pg = d.two ? m.prod_gamma : m.gamma;
  d.ppi = d.two ? m.prod_p_inf : m.p_inf;
  d.pcv = d.two ? m.prod_cv : m.cv;
  d.pign = m.reactive ? m.p_ign : 0.0;
  d.iGm1 = 1.0 / (m.gamma - 1.0);
  d.gi = m.gamma * d.iGm1;
  d.kap = m.gamma * m.p_inf * d.iGm1;
  d.gG = m.gamma * m.G * d.iGm1;
  d.GoG = m.G * d.iGm1;
  d.JY = (m.plastic && m.G > 0) ? m.sigma_y / (std::sqrt(6.0) * m.G) : INFINITY;
  d.jc2 = m.jc_c2;
  d.jc3 = m.jc_c3;
  d.jcn = m.jc_n;
  d.jcm = m.jc_m;
  d.jcTm = m.jc_Tmelt;
  d.jcT0 = m.jc_T0;
  return d;
}

}  // namespace

int dis_internal_ensure_ws(dis_ctx* c) { return ensure_ws(c); }

int dis_internal_steps(dis_ctx* c, int n, bool fixed) { return dispatch_steps(c, n, fixed); }

// One float64 step with the per-patch dt of c->dtfix, calling
// h.before(stage, source state) before each stage's recovery and
// h.after_flux(stage) after its flux kernels (all on c->stream): three
// Runge-Kutta stages, or the one stage (stage 0) of the MUSCL-Hancock
// update, in place.
namespace {
template <int DIM, bool RX>
void step64_hooked(dis_ctx* c, const StepHooks& h) {
  StepArgs a = base_args(c);
  a.dtfix = c->dtfix;
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
  const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
  const unsigned np = (unsigned)c->seg_prim.size(), nfx = (unsigned)c->seg_fx.size(),
                 nfy = (unsigned)c->seg_fy.size(), nc = (unsigned)c->seg_cell.size();
  if (c->hancock) {
    a.qsrc = c->q[0];
    a.qn = c->q[0];
    a.qdst = c->q[0];
    a.a = 0.0;
    a.b = 1.0;
    a.last = 1;
    if (h.before) h.before(h.user, 0, c->q[0]);
    k_prim<DIM, RX><<<np, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, 0);
    k_hancock<DIM, RX><<<np, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim);
    k_flux_h<DIM, RX, 0><<<nfx, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fx);
    if constexpr (DIM == 2) k_flux_h<DIM, RX, 1><<<nfy, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fy);
    if (h.after_flux) h.after_flux(h.user, 0);
    k_update<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_cell);
    return;
  }
  for (int stg = 0; stg < 3; ++stg) {
    a.qsrc = stg == 0 ? c->q[0] : c->q[1];
    a.qn = c->q[0];
    a.qdst = stg == 2 ? c->q[0] : c->q[1];
    a.a = ca[stg];
    a.b = cb[stg];
    a.last = stg == 2;
    if (h.before) h.before(h.user, stg, stg == 0 ? c->q[0] : c->q[1]);
    k_prim<DIM, RX><<<np, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, 0);
    k_flux<DIM, RX, 0><<<nfx, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fx);
    if constexpr (DIM == 2) k_flux<DIM, RX, 1><<<nfy, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fy);
    if (h.after_flux) h.after_flux(h.user, stg);
    k_update<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_cell);
  }
}

// Per-patch CFL rate max of the state q[0] (interior cells) into c->rate.
template <int DIM, bool RX>
void rates64(dis_ctx* c) {
  StepArgs a = base_args(c);
  a.qsrc = c->q[0];
  cudaMemsetAsync(c->rate, 0, sizeof(unsigned long long) * c->np, c->stream);
  k_prim<DIM, RX><<<(unsigned)c->seg_prim.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, 1);
}
}  // namespace

int dis_internal_step64_hooked(dis_ctx* c, const StepHooks& h) {
  const bool rx = c->y >= 0;
  if (c->dim == 1) rx ? step64_hooked<1, true>(c, h) : step64_hooked<1, false>(c, h);
  else rx ? step64_hooked<2, true>(c, h) : step64_hooked<2, false>(c, h);
  CU(cudaGetLastError());
  return DIS_OK;
}

int dis_internal_rates_enqueue(dis_ctx* c) {
  const bool rx = c->y >= 0;
  if (c->dim == 1) rx ? rates64<1, true>(c) : rates64<1, false>(c);
  else rx ? rates64<2, true>(c) : rates64<2, false>(c);
  CU(cudaGetLastError());
  return DIS_OK;
}

int dis_internal_rates(dis_ctx* c, double* host) {
  const bool rx = c->y >= 0;
  if (c->dim == 1) rx ? rates64<1, true>(c) : rates64<1, false>(c);
  else rx ? rates64<2, true>(c) : rates64<2, false>(c);
  CU(cudaGetLastError());
  std::vector<unsigned long long> r(c->np);
  CU(cudaMemcpyAsync(r.data(), c->rate, sizeof(unsigned long long) * c->np, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int p = 0; p < c->np; ++p) {
    double v;
    std::memcpy(&v, &r[p], sizeof v);
    host[p] = v;
  }
  return DIS_OK;
}

thread_local bool g_allow_external = false;
int dis_internal_create_external(int dim, int n_patches, const dis_patch* patches, int reactive_material,
                                 const dis_options* opt, void* stream, dis_ctx** out) {
  g_allow_external = true;
  const int rc = dis_create(dim, n_patches, patches, reactive_material, opt, stream, out);
  g_allow_external = false;
  return rc;
}

extern "C" {

const char* dis_last_error(void) { return g_err.c_str(); }

int dis_create(int dim, int n_patches, const dis_patch* patches, int reactive_material,
               const dis_options* opt, void* stream, dis_ctx** out) {
  if (!out) return fail(DIS_EINVAL, "dis_create: out is NULL");
  *out = nullptr;
  if (dim != 1 && dim != 2) return fail(DIS_EINVAL, "dis_create: dim must be 1 or 2 (got %d)", dim);
  if (n_patches <= 0 || !patches) return fail(DIS_EINVAL, "dis_create: need at least one patch");
  if (!opt) return fail(DIS_EINVAL, "dis_create: opt is NULL");
  if (reactive_material < -1 || reactive_material > 1)
    return fail(DIS_EINVAL, "dis_create: reactive_material must be -1, 0 or 1");
  if (!(opt->cfl > 0.0 && opt->cfl <= 1.0)) return fail(DIS_EINVAL, "dis_create: cfl must be in (0, 1]");
  if (opt->precision != DIS_FP64 && opt->precision != DIS_FP32_BULK)
    return fail(DIS_EINVAL, "dis_create: unknown precision %d", opt->precision);
  if (opt->scheme != DIS_RK3 && opt->scheme != DIS_HANCOCK)
    return fail(DIS_EINVAL, "dis_create: unknown scheme %d", opt->scheme);
  if (opt->geometry != DIS_PLANAR && opt->geometry != DIS_CYLINDRICAL)
    return fail(DIS_EINVAL, "dis_create: unknown geometry %d", opt->geometry);
  if (opt->limiter != DIS_MINMOD && opt->limiter != DIS_VANLEER)
    return fail(DIS_EINVAL, "dis_create: unknown limiter %d", opt->limiter);
  if (opt->geometry == DIS_CYLINDRICAL && opt->scheme != DIS_RK3)
    return fail(DIS_EINVAL, "dis_create: cylindrical geometry is built for the Runge-Kutta scheme only");
  for (int p = 0; p < n_patches; ++p) {
    const dis_patch& P = patches[p];
    const int ny = dim == 2 ? P.ny : 1;
    if (P.nx < 4 || ny < (dim == 2 ? 4 : 1) || !(P.dx > 0) || (dim == 2 && !(P.dy > 0)))
      return fail(DIS_EINVAL, "dis_create: patch %d has bad size (nx %d ny %d dx %g dy %g)", p, P.nx,
                  P.ny, P.dx, P.dy);
    if ((long long)P.nx * ny > (1LL << 31))
      return fail(DIS_EINVAL, "dis_create: patch %d is too large", p);
    for (int k = 0; k < (dim == 2 ? 4 : 2); ++k)
      if (P.bc[k] < 0 || P.bc[k] > (g_allow_external ? 3 : 2))
        return fail(DIS_EINVAL, "dis_create: patch %d bad bc", p);
    if (opt->geometry == DIS_CYLINDRICAL && !(P.x0 >= 0.0))
      return fail(DIS_EINVAL, "dis_create: patch %d has x0 %g < 0 (a radius)", p, P.x0);
  }
  dis_ctx* c = new (std::nothrow) dis_ctx();
  if (!c) return fail(DIS_ENOMEM, "dis_create: out of host memory");
  c->dim = dim;
  c->np = n_patches;
  c->y = reactive_material;
  c->nf = (dim == 2 ? 11 : 8) + (reactive_material >= 0 ? 1 : 0);
  c->opt = *opt;
  c->fp32 = opt->precision == DIS_FP32_BULK;
  c->hancock = opt->scheme == DIS_HANCOCK;
  c->patches.assign(patches, patches + n_patches);
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  c->phys.y = reactive_material;
  c->phys.thinc = opt->thinc ? 1 : 0;
  c->phys.cfl = opt->cfl;
  c->phys.cyl = opt->geometry == DIS_CYLINDRICAL ? 1 : 0;
  c->phys.limiter = opt->limiter;
  layout(c);
  c->patch_set.assign(n_patches, 0);
  *out = c;
  return DIS_OK;
}

int dis_set_materials(dis_ctx* c, const dis_material* m, int n) {
  if (!c || !m) return fail(DIS_EINVAL, "dis_set_materials: NULL argument");
  if (n != 2) return fail(DIS_EINVAL, "dis_set_materials: exactly 2 materials are supported (got %d)", n);
  const Phys old = c->phys;
  for (int l = 0; l < 2; ++l) {
    if (!(m[l].gamma > 1.0)) return fail(DIS_EINVAL, "dis_set_materials: gamma must be > 1");
    if (m[l].G < 0 || m[l].p_inf < 0) return fail(DIS_EINVAL, "dis_set_materials: negative G or p_inf");
    if (m[l].plastic < DIS_PLASTIC_NONE || m[l].plastic > DIS_PLASTIC_JC)
      return fail(DIS_EINVAL, "dis_set_materials: bad plastic");
    const bool jc = m[l].plastic == DIS_PLASTIC_JC;
    if (jc && m[l].reactive)
      return fail(DIS_EINVAL, "dis_set_materials: a material carries one history row (reactive or Johnson-Cook)");
    if ((l == c->y) != (m[l].reactive != 0 || jc))
      return fail(DIS_EINVAL, "dis_set_materials: the context's history-row material must be the reactive or "
                              "Johnson-Cook one");
    if (jc && !(m[l].eos == DIS_EOS_ROMENSKII && m[l].G > 0 && m[l].cv > 0 && m[l].chi0 > 0 && m[l].jc_c3 > 0 &&
                m[l].sigma_y >= 0 && m[l].jc_c2 >= 0 && m[l].jc_n > 0 && m[l].jc_m > 0 && m[l].jc_T0 >= 0 &&
                m[l].jc_Tmelt > m[l].jc_T0 && std::isfinite(m[l].jc_Tmelt)))
      return fail(DIS_EINVAL, "dis_set_materials: Johnson-Cook needs a Romenskii solid with G, cv, chi0, c3, n, "
                              "m > 0, sigma_y, c2, T0 >= 0 and finite T_melt > T0");
    if (jc && c->fp32)
      return fail(DIS_EINVAL, "dis_set_materials: Johnson-Cook plasticity is built for float64 contexts only");
    if (m[l].eos < DIS_EOS_STIFFENED || m[l].eos > DIS_EOS_JWL)
      return fail(DIS_EINVAL, "dis_set_materials: unknown eos %d", m[l].eos);
    if (m[l].eos == DIS_EOS_ROMENSKII && !(m[l].rho0 > 0 && m[l].K0 > 0 && m[l].alpha > 0 && m[l].beta >= 0))
      return fail(DIS_EINVAL, "dis_set_materials: Romenskii needs rho0, K0, alpha > 0 and beta >= 0");
    if (m[l].eos == DIS_EOS_JWL && !(m[l].rho0 > 0 && m[l].jwl_R1 > 0 && m[l].jwl_R2 > 0 && m[l].G == 0))
      return fail(DIS_EINVAL, "dis_set_materials: JWL needs rho0, R1, R2 > 0 and G = 0");
    if (m[l].reactive && m[l].eos != DIS_EOS_STIFFENED)
      return fail(DIS_EINVAL, "dis_set_materials: the reactive material must be a stiffened (ideal) gas");
    const bool two = m[l].reactive && m[l].prod_gamma > 0.0;
    if (two && (!(m[l].prod_gamma > 1.0) || m[l].prod_p_inf < 0 || !(m[l].prod_cv > 0) || m[l].G != 0 ||
                !(m[l].cv > 0)))
      return fail(DIS_EINVAL, "dis_set_materials: product closure needs prod_gamma > 1, prod_p_inf >= 0, "
                              "prod_cv > 0 (and G = 0, cv > 0)");
    if (two && c->fp32)
      return fail(DIS_EINVAL, "dis_set_materials: two reactive closures are built for float64 contexts only");
    if (m[l].reactive && !two && (m[l].p_inf != 0 || m[l].G != 0 || !(m[l].cv > 0)))
      return fail(DIS_EINVAL, "dis_set_materials: a reactive material must be an ideal gas with cv > 0");
    if (m[l].reactive && (m[l].rate_law < 0 || m[l].rate_law > 1 || !std::isfinite(m[l].p_ign) ||
                          !std::isfinite(m[l].A) || m[l].A < 0))
      return fail(DIS_EINVAL, "dis_set_materials: bad rate law (rate_law 0 or 1, finite A >= 0 and p_ign)");
  }
  for (int l = 0; l < 2; ++l) c->phys.m[l] = to_dev(m[l]);
  c->physf = to_float(c->phys);
  if (c->fp32 && c->variant >= 0 && !variant_valid(c, c->variant)) c->variant = -1;  // tune again
  if (c->fp32 && c->have_mats && c->have_state && c->ws_ready &&
      (old.m[0].kap != c->phys.m[0].kap || old.m[1].kap != c->phys.m[1].kap)) {
    // an FP32-bulk state holds e_s = rho E - kappa(phi1): keep rho E
    const double dk2 = old.m[1].kap - c->phys.m[1].kap;
    const double ddk = (old.m[0].kap - old.m[1].kap) - (c->phys.m[0].kap - c->phys.m[1].kap);
    const unsigned nc = (unsigned)c->seg_cell.size();
    if (c->dim == 1) {
      if (c->y >= 0) k_rekappa32<1, true><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, c->q32[0], c->T, dk2, ddk);
      else k_rekappa32<1, false><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, c->q32[0], c->T, dk2, ddk);
    } else {
      if (c->y >= 0) k_rekappa32<2, true><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, c->q32[0], c->T, dk2, ddk);
      else k_rekappa32<2, false><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, c->q32[0], c->T, dk2, ddk);
    }
    CU(cudaGetLastError());
  }
  c->rate_valid = false;  // the rate depends on the closures
  c->have_mats = true;
  // captured steps hold the closure parameters by value: capture again
  drop_graphs(c);
  return DIS_OK;
}

size_t dis_workspace_bytes(const dis_ctx* c) {
  if (!c) return 0;
  return carve(const_cast<dis_ctx*>(c), nullptr);
}

size_t dis_state_bytes(const dis_ctx* c, int kind) {
  (void)kind;
  return c ? sizeof(double) * (size_t)c->nf * c->ncells : 0;
}

int dis_bind_workspace(dis_ctx* c, void* dev, size_t bytes) {
  if (!c || !dev) return fail(DIS_EINVAL, "dis_bind_workspace: NULL argument");
  if (((uintptr_t)dev) & 255) return fail(DIS_EINVAL, "dis_bind_workspace: pointer not 256-byte aligned");
  const size_t need = carve(c, nullptr);
  if (bytes < need) return fail(DIS_ENOMEM, "dis_bind_workspace: %zu bytes given, %zu needed", bytes, need);
  if (c->ws_owned) cudaStreamSynchronize(c->stream);  // work may be in flight
  drop_graphs(c);
  if (c->ws_owned) cudaFree(c->ws);
  c->ws = (char*)dev;
  c->ws_bytes = bytes;
  c->ws_owned = false;
  c->ws_ready = false;
  c->have_state = false;
  c->patch_set.assign(c->np, 0);
  c->rate_valid = false;
  return ensure_ws(c);
}

int dis_set_state(dis_ctx* c, int kind, const double* src, int src_on_device) {
  if (!c || !src) return fail(DIS_EINVAL, "dis_set_state: NULL argument");
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_set_state: bad kind");
  if (!c->have_mats) return fail(DIS_ESTATE, "dis_set_state: set materials first");
  int rc = ensure_ws(c);
  if (rc) return rc;
  const double* dsrc = src;
  if (!src_on_device) {
    CU(cudaMemcpyAsync(c->io, src, dis_state_bytes(c, kind), cudaMemcpyHostToDevice, c->stream));
    dsrc = c->io;
  }
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  if (c->dim == 1) rc = rx ? do_unpack<1, true>(c, dsrc, prim) : do_unpack<1, false>(c, dsrc, prim);
  else rc = rx ? do_unpack<2, true>(c, dsrc, prim) : do_unpack<2, false>(c, dsrc, prim);
  if (rc) return rc;
  if (!src_on_device) CU(cudaStreamSynchronize(c->stream));  // the host buffer may be reused
  c->have_state = true;
  c->patch_set.assign(c->np, 1);
  c->steps_total = 0;
  return DIS_OK;
}

int dis_set_patch_state(dis_ctx* c, int patch, int kind, const double* src, int src_on_device) {
  if (!c || !src) return fail(DIS_EINVAL, "dis_set_patch_state: NULL argument");
  if (patch < 0 || patch >= c->np) return fail(DIS_EINVAL, "dis_set_patch_state: patch %d outside 0..%d", patch, c->np - 1);
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_set_patch_state: bad kind");
  if (!c->have_mats) return fail(DIS_ESTATE, "dis_set_patch_state: set materials first");
  int rc = ensure_ws(c);
  if (rc) return rc;
  const size_t bytes = sizeof(double) * (size_t)c->nf * c->pd[patch].nx * c->pd[patch].ny;
  const double* dsrc = src;
  if (!src_on_device) {
    CU(cudaMemcpyAsync(c->io, src, bytes, cudaMemcpyHostToDevice, c->stream));
    dsrc = c->io;
  }
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  if (c->dim == 1) rc = rx ? do_unpack<1, true>(c, dsrc, prim, patch) : do_unpack<1, false>(c, dsrc, prim, patch);
  else rc = rx ? do_unpack<2, true>(c, dsrc, prim, patch) : do_unpack<2, false>(c, dsrc, prim, patch);
  if (rc) return rc;
  if (!src_on_device) CU(cudaStreamSynchronize(c->stream));
  c->rate_valid = false;
  c->patch_set[patch] = 1;
  c->have_state = std::all_of(c->patch_set.begin(), c->patch_set.end(), [](char x) { return x != 0; });
  c->steps_total = 0;
  return DIS_OK;
}

int dis_get_patch_state(dis_ctx* c, int patch, int kind, double* dst, int dst_on_device) {
  if (!c || !dst) return fail(DIS_EINVAL, "dis_get_patch_state: NULL argument");
  if (patch < 0 || patch >= c->np) return fail(DIS_EINVAL, "dis_get_patch_state: patch %d outside 0..%d", patch, c->np - 1);
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_get_patch_state: bad kind");
  if (!c->patch_set[patch]) return fail(DIS_ESTATE, "dis_get_patch_state: patch %d holds no state", patch);
  const size_t bytes = sizeof(double) * (size_t)c->nf * c->pd[patch].nx * c->pd[patch].ny;
  double* ddst = dst_on_device ? dst : c->io;
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  int rc;
  if (c->dim == 1) rc = rx ? do_pack<1, true>(c, ddst, prim, patch) : do_pack<1, false>(c, ddst, prim, patch);
  else rc = rx ? do_pack<2, true>(c, ddst, prim, patch) : do_pack<2, false>(c, ddst, prim, patch);
  if (rc) return rc;
  if (!dst_on_device) {
    CU(cudaMemcpyAsync(dst, c->io, bytes, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return DIS_OK;
}

int dis_get_state(dis_ctx* c, int kind, double* dst, int dst_on_device) {
  if (!c || !dst) return fail(DIS_EINVAL, "dis_get_state: NULL argument");
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_get_state: bad kind");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_get_state: no state loaded");
  double* ddst = dst_on_device ? dst : c->io;
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  int rc;
  if (c->dim == 1) rc = rx ? do_pack<1, true>(c, ddst, prim) : do_pack<1, false>(c, ddst, prim);
  else rc = rx ? do_pack<2, true>(c, ddst, prim) : do_pack<2, false>(c, ddst, prim);
  if (rc) return rc;
  if (!dst_on_device) {
    CU(cudaMemcpyAsync(dst, c->io, dis_state_bytes(c, kind), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return DIS_OK;
}

// Staging buffers, copy streams and events of the pipelined transfers
// (created on first use, released by dis_destroy).
static int ensure_async(dis_ctx* c) {
  if (c->s_in) return DIS_OK;
  const size_t bytes = sizeof(double) * (size_t)c->nf * c->ncells;
  for (int b = 0; b < 2; ++b) {
    if (cudaMalloc(&c->xin[b], bytes) != cudaSuccess || cudaMalloc(&c->xout[b], bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(DIS_ENOMEM, "async transfers: cannot allocate %zu-byte staging buffers", bytes);
    }
    CU(cudaEventCreateWithFlags(&c->in_done[b], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->in_free[b], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->out_ready[b], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->out_free[b], cudaEventDisableTiming));
  }
  CU(cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking));
  CU(cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking));
  return DIS_OK;
}

int dis_set_state_async(dis_ctx* c, int kind, const double* src) {
  if (!c || !src) return fail(DIS_EINVAL, "dis_set_state_async: NULL argument");
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_set_state_async: bad kind");
  if (!c->have_mats) return fail(DIS_ESTATE, "dis_set_state_async: set materials first");
  int rc = ensure_ws(c);
  if (!rc) rc = ensure_async(c);
  if (rc) return rc;
  const int b = c->in_idx;
  c->in_idx ^= 1;
  // the copy may start once the conversion that last read this buffer is done
  CU(cudaStreamWaitEvent(c->s_in, c->in_free[b], 0));
  CU(cudaMemcpyAsync(c->xin[b], src, dis_state_bytes(c, kind), cudaMemcpyHostToDevice, c->s_in));
  CU(cudaEventRecord(c->in_done[b], c->s_in));
  CU(cudaStreamWaitEvent(c->stream, c->in_done[b], 0));
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  if (c->dim == 1) rc = rx ? do_unpack<1, true>(c, c->xin[b], prim) : do_unpack<1, false>(c, c->xin[b], prim);
  else rc = rx ? do_unpack<2, true>(c, c->xin[b], prim) : do_unpack<2, false>(c, c->xin[b], prim);
  if (rc) return rc;
  CU(cudaEventRecord(c->in_free[b], c->stream));
  c->have_state = true;
  c->patch_set.assign(c->np, 1);
  c->steps_total = 0;
  return DIS_OK;
}

int dis_get_state_async(dis_ctx* c, int kind, double* dst) {
  if (!c || !dst) return fail(DIS_EINVAL, "dis_get_state_async: NULL argument");
  if (kind != DIS_CONSERVATIVE && kind != DIS_PRIMITIVE) return fail(DIS_EINVAL, "dis_get_state_async: bad kind");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_get_state_async: no state loaded");
  int rc = ensure_async(c);
  if (rc) return rc;
  const int b = c->out_idx;
  c->out_idx ^= 1;
  // the conversion may overwrite this buffer once its last copy has left
  CU(cudaStreamWaitEvent(c->stream, c->out_free[b], 0));
  const bool rx = c->y >= 0;
  const int prim = kind == DIS_PRIMITIVE;
  if (c->dim == 1) rc = rx ? do_pack<1, true>(c, c->xout[b], prim) : do_pack<1, false>(c, c->xout[b], prim);
  else rc = rx ? do_pack<2, true>(c, c->xout[b], prim) : do_pack<2, false>(c, c->xout[b], prim);
  if (rc) return rc;
  CU(cudaEventRecord(c->out_ready[b], c->stream));
  CU(cudaStreamWaitEvent(c->s_out, c->out_ready[b], 0));
  CU(cudaMemcpyAsync(dst, c->xout[b], dis_state_bytes(c, kind), cudaMemcpyDeviceToHost, c->s_out));
  CU(cudaEventRecord(c->out_free[b], c->s_out));
  return DIS_OK;
}

int dis_sync(dis_ctx* c) {
  if (!c) return fail(DIS_EINVAL, "dis_sync: NULL context");
  if (c->s_in) CU(cudaStreamSynchronize(c->s_in));
  CU(cudaStreamSynchronize(c->stream));
  if (c->s_out) CU(cudaStreamSynchronize(c->s_out));
  return DIS_OK;
}

// Events around a step call (dis_query reports the device time between them).
static int timed_dispatch(dis_ctx* c, int n, bool fixed) {
  if (!c->ev_step[0]) {
    CU(cudaEventCreate(&c->ev_step[0]));
    CU(cudaEventCreate(&c->ev_step[1]));
  }
  CU(cudaEventRecord(c->ev_step[0], c->stream));
  const int rc = dispatch_steps(c, n, fixed);
  if (rc) return rc;
  CU(cudaEventRecord(c->ev_step[1], c->stream));
  c->ev_recorded = true;
  c->last_steps = n;
  c->steps_total += n;
  return DIS_OK;
}

int dis_step(dis_ctx* c, int n_steps, double* dt_out) {
  if (!c) return fail(DIS_EINVAL, "dis_step: NULL context");
  if (n_steps < 0) return fail(DIS_EINVAL, "dis_step: negative step count");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_step: no state loaded (every patch needs one)");
  int rc = timed_dispatch(c, n_steps, false);
  if (rc) return rc;
  if (dt_out && n_steps > 0) {
    CU(cudaMemcpyAsync(dt_out, c->dtlast, sizeof(double) * c->np, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return DIS_OK;
}

int dis_step_fixed_dt(dis_ctx* c, int n_steps, const double* dt) {
  if (!c || !dt) return fail(DIS_EINVAL, "dis_step_fixed_dt: NULL argument");
  if (n_steps < 0) return fail(DIS_EINVAL, "dis_step_fixed_dt: negative step count");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_step_fixed_dt: no state loaded");
  for (int p = 0; p < c->np; ++p)
    if (!(dt[p] > 0.0) || !std::isfinite(dt[p])) return fail(DIS_EINVAL, "dis_step_fixed_dt: bad dt[%d]", p);
  CU(cudaMemcpyAsync(c->dtfix, dt, sizeof(double) * c->np, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return timed_dispatch(c, n_steps, true);
}

int dis_query(dis_ctx* c, dis_stats* out) {
  if (!c || !out) return fail(DIS_EINVAL, "dis_query: NULL argument");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_query: no state loaded");
  const bool rx = c->y >= 0;
  int rc;
  if (c->dim == 1) rc = rx ? do_query<1, true>(c) : do_query<1, false>(c);
  else rc = rx ? do_query<2, true>(c) : do_query<2, false>(c);
  if (rc) return rc;
  double q[NQ];
  std::vector<double> dts(c->np);
  int st[4] = {0, 0, 0, 0};
  CU(cudaMemcpyAsync(q, c->qout, sizeof q, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(dts.data(), c->dtlast, sizeof(double) * c->np, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  dis_stats r{};
  r.mass[0] = q[0];
  r.mass[1] = q[1];
  r.momentum[0] = q[2];
  r.momentum[1] = q[3];
  r.energy = q[4];
  r.reactant = q[5];
  r.phi_min = q[6];
  r.phi_max = q[7];
  if (c->steps_total > 0) {
    r.dt_min = *std::min_element(dts.begin(), dts.end());
    r.dt_max = *std::max_element(dts.begin(), dts.end());
  }
  if (c->ev_recorded) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev_step[0], c->ev_step[1]));
    r.kernel_ms = ms;
  }
  const double per_cell = c->fp32 ? 4.0 * (c->nf + 1) : 8.0 * c->nf;
  r.bytes = 2.0 * per_cell * (double)c->ncells * (double)c->last_steps;
  r.steps = c->steps_total;
  r.launches = c->launches;
  r.status = st[0] ? DIS_ENONPHYSICAL : DIS_OK;
  r.bad_patch = st[0] ? st[1] : -1;
  r.bad_cell = st[0] ? st[2] : -1;
  *out = r;
  return DIS_OK;
}

int dis_check(dis_ctx* c, int* bad_patch, int* bad_cell) {
  if (!c) return fail(DIS_EINVAL, "dis_check: NULL context");
  if (!c->ws_ready) return DIS_OK;
  int st[4] = {0, 0, 0, 0};
  CU(cudaMemcpyAsync(st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  CU(cudaMemsetAsync(c->status, 0, sizeof st, c->stream));
  if (bad_patch) *bad_patch = st[0] ? st[1] : -1;
  if (bad_cell) *bad_cell = st[0] ? st[2] : -1;
  if (st[0]) return fail(DIS_ENONPHYSICAL, "non-physical state in patch %d cell %d", st[1], st[2]);
  return DIS_OK;
}

long long dis_last_launches(const dis_ctx* c) { return c ? c->launches : 0; }

int dis_tile_choice(const dis_ctx* c, int* tx, int* ty, int* precomputed, double* step_ms) {
  if (!c) return fail(DIS_EINVAL, "dis_tile_choice: NULL context");
  if (precomputed) *precomputed = 0;
  if (!c->fp32 || c->variant < 0) {
    if (tx) *tx = 0;
    if (ty) *ty = 0;
    return DIS_OK;
  }
  const int shape = c->variant % 3;
  if (tx) *tx = c->dim == 2 ? kTiles2D[shape][0] : kTiles1D[shape];
  if (ty) *ty = c->dim == 2 ? kTiles2D[shape][1] : 1;
  if (precomputed) *precomputed = 0;
  if (step_ms)
    for (int v = 0; v < DIS_NVARIANTS; ++v) step_ms[v] = variant_valid(c, v) ? c->tune_ms[v] : 0.0;
  return DIS_OK;
}

int dis_set_variant(dis_ctx* c, int variant) {
  if (!c) return fail(DIS_EINVAL, "dis_set_variant: NULL context");
  if (!c->fp32) return fail(DIS_EINVAL, "dis_set_variant: only FP32-bulk contexts have variants");
  if (variant != -1 && !variant_valid(c, variant))
    return fail(DIS_EINVAL, "dis_set_variant: variant %d is not a variant of this context", variant);
  drop_graphs(c);
  c->variant = variant;
  return DIS_OK;
}

int dis_set_schedule(dis_ctx* c, int schedule) {
  if (!c) return fail(DIS_EINVAL, "dis_set_schedule: NULL context");
  if (schedule < -1 || schedule > 1) return fail(DIS_EINVAL, "dis_set_schedule: schedule %d outside -1..1", schedule);
  if (schedule == 1 && (!c->fp32 || c->dim != 1))
    return fail(DIS_EINVAL, "dis_set_schedule: the persistent batch schedule needs a 1D FP32-bulk context");
  c->schedule_req = schedule;
  return DIS_OK;
}

int dis_schedule(const dis_ctx* c, int* schedule, double* batch_ms) {
  if (!c) return fail(DIS_EINVAL, "dis_schedule: NULL context");
  if (schedule) {
    if (c->schedule_req >= 0) *schedule = c->schedule_req;
    else if (c->variant >= 0) *schedule = std::max(c->schedule, 0);
    else *schedule = -1;
  }
  if (batch_ms)
    for (int v = 0; v < DIS_NVARIANTS; ++v) batch_ms[v] = c->tune_batch_ms[v];
  return DIS_OK;
}

int dis_step_timed(dis_ctx* c, int n_steps, double* kernel_ms) {
  if (!c || !kernel_ms) return fail(DIS_EINVAL, "dis_step_timed: NULL argument");
  if (n_steps <= 0) return fail(DIS_EINVAL, "dis_step_timed: n_steps must be positive");
  if (!c->have_state) return fail(DIS_ESTATE, "dis_step_timed: no state loaded");
  if (c->hancock) return fail(DIS_EINVAL, "dis_step_timed: Runge-Kutta contexts only");
  const bool rx = c->y >= 0;
  if (c->dim == 1) return rx ? timed_steps<1, true>(c, n_steps, kernel_ms) : timed_steps<1, false>(c, n_steps, kernel_ms);
  return rx ? timed_steps<2, true>(c, n_steps, kernel_ms) : timed_steps<2, false>(c, n_steps, kernel_ms);
}

void dis_destroy(dis_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);  // replays of the step graphs run on the caller's stream
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->s_in) cudaStreamSynchronize(c->s_in);
  if (c->s_out) cudaStreamSynchronize(c->s_out);
  for (int b = 0; b < 2; ++b) {
    if (c->xin[b]) cudaFree(c->xin[b]);
    if (c->xout[b]) cudaFree(c->xout[b]);
    for (cudaEvent_t e : {c->in_done[b], c->in_free[b], c->out_ready[b], c->out_free[b]})
      if (e) cudaEventDestroy(e);
  }
  if (c->s_in) cudaStreamDestroy(c->s_in);
  if (c->s_out) cudaStreamDestroy(c->s_out);
  if (c->ws_owned && c->ws) cudaFree(c->ws);
  for (cudaEvent_t e : c->ev_step)
    if (e) cudaEventDestroy(e);
  dis_internal_adj_free(c);
  delete c;
}

}  // extern "C"
