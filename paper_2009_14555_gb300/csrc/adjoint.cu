// adjoint.cu - checkpointed reverse sweep of the float64 step (C ABI part of
// include/dis.h: dis_adj_forward, dis_adjoint).
//
// Forward: the state q^n is copied to a checkpoint every K steps and the time
// step of every step and patch is recorded; a running objective
// J = sum_n dt_n sum_cells phi_l (rho u) dA over the states q^{n+1} can be
// accumulated on the device.
// Reverse: segments of K steps are taken last to first.  A segment is
// recomputed from its checkpoint with the recorded dt (bit-identical to the
// forward run), keeping each step's stage inputs, pre-source state and the
// primitives and face outputs of each stage input; then, step by step
// backwards, the stages are reversed (adjoint.cuh).
// Memory: (number of checkpoints + 4 K + 8) states, 3 K sets of primitives
// and face outputs, and the face coefficients, all library-owned and released
// by dis_destroy.
// FP32-bulk contexts: the forward run is the FP32-bulk step; its states are
// checkpointed in float64 and the reverse sweep recomputes each segment with
// the float64 step from those checkpoints (its own float64 primitive and face
// buffers), so the gradient is the float64 adjoint along a trajectory that
// restarts from the FP32-bulk states every K steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <utility>

#include "adjoint.cuh"
#include "ctx.cuh"

using namespace dis;

struct dis_adj {
  int n_steps = 0, every = 0, n_ck = 0, mat = -1;
  bool ready = false;
  int dual_riemann = 0;  // dual-number reference form of the hand-reversed local maps
  char* mem = nullptr;
  size_t mem_bytes = 0;
  double* ck = nullptr;   // n_ck checkpoints
  double* seg = nullptr;  // every + 1 states of one segment
  double* st[3] = {nullptr, nullptr, nullptr};  // scratch stage states of one step
  double* stg = nullptr;  // per step of a segment: q1, q3 and the pre-source state
  char* wf = nullptr;     // per stage input of a segment: primitives and face outputs
  size_t wf_bytes = 0;    // bytes of one such set
  double* ob = nullptr;
  double* xb = nullptr;
  double* acc = nullptr;
  double* G = nullptr;
  double* Wb = nullptr;
  double* dts = nullptr;  // n_steps x n_patches
  double* J = nullptr;
  double* theta = nullptr;
  // float64 primitives and face outputs: the context's own (float64
  // contexts) or allocated here (FP32-bulk contexts); tmp: float64 copy of an
  // FP32-bulk state for the objective
  double* W = nullptr;
  double* Fx = nullptr;
  double* Fy = nullptr;
  double* tmp = nullptr;
};

#define ACU(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return dis_internal_error(DIS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

void dis_internal_adj_free(dis_ctx* c) {
  if (!c || !c->adj) return;
  if (c->adj->mem) cudaFree(c->adj->mem);
  delete c->adj;
  c->adj = nullptr;
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int n_extra(int dim) { return dim == 2 ? 3 : 2; }

int adj_alloc(dis_ctx* c, int n_steps, int every) {
  if (!c->adj) c->adj = new (std::nothrow) dis_adj();
  if (!c->adj) return dis_internal_error(DIS_ENOMEM, "dis_adj_forward: out of host memory");
  dis_adj* d = c->adj;
  const size_t S = sizeof(double) * (size_t)c->nf * c->T;
  const int n_ck = (n_steps + every - 1) / every;
  // states: checkpoints, the segment, its stage states (3 per step), scratch
  // q1 / q3 / pre-source, obar / xbar / qn_acc, Wbar
  const size_t nfo = (size_t)(c->nf + n_extra(c->dim));
  const size_t own = c->fp32 ? 2 * a256(S) + a256(sizeof(double) * nfo * c->NFX) +
                                   a256(sizeof(double) * nfo * std::max<long long>(1, c->NFY))
                             : 0;
  // per stage input of a segment: primitives (nf planes) and x / y face outputs
  const size_t wfb = a256(S) + a256(sizeof(double) * nfo * c->NFX) +
                     a256(sizeof(double) * nfo * std::max<long long>(1, c->NFY));
  const size_t need = a256(S) * (size_t)(n_ck + (every + 1) + 3 * every + 7) + a256(sizeof(double) * nfo * c->T) +
                      a256(sizeof(double) * (size_t)n_steps * c->np) + a256(sizeof(double)) +
                      a256(sizeof(double) * NPARAM) + own + wfb * 3 * (size_t)every;
  if (need > d->mem_bytes) {
    if (d->mem) cudaFree(d->mem);
    d->mem = nullptr;
    d->mem_bytes = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return dis_internal_error(DIS_ENOMEM, "dis_adj_forward: cannot allocate %zu bytes", need);
    }
    d->mem = (char*)p;
    d->mem_bytes = need;
  }
  char* b = d->mem;
  auto take = [&](size_t bytes) {
    char* p = b;
    b += a256(bytes);
    return (double*)p;
  };
  d->ck = take(S * n_ck);
  d->seg = take(S * (every + 1));
  d->stg = take(S * 3 * (size_t)every);
  d->wf_bytes = wfb;
  d->wf = (char*)take(wfb * 3 * (size_t)every);
  for (int k = 0; k < 3; ++k) d->st[k] = take(S);
  d->ob = take(S);
  d->xb = take(S);
  d->acc = take(S);
  d->G = take(sizeof(double) * (size_t)(c->nf + n_extra(c->dim)) * c->T);
  d->Wb = take(S);
  d->dts = take(sizeof(double) * (size_t)n_steps * c->np);
  d->J = take(sizeof(double));
  d->theta = take(sizeof(double) * NPARAM);
  if (c->fp32) {
    d->W = take(S);
    d->tmp = take(S);
    d->Fx = take(sizeof(double) * nfo * c->NFX);
    d->Fy = take(sizeof(double) * nfo * std::max<long long>(1, c->NFY));
  } else {
    d->W = c->W;
    d->Fx = c->Fx;
    d->Fy = c->Fy;
    d->tmp = nullptr;
  }
  if ((size_t)(b - d->mem) > d->mem_bytes)
    return dis_internal_error(DIS_EINVAL, "dis_adj_forward: internal layout exceeds its allocation");
  d->n_steps = n_steps;
  d->every = every;
  d->n_ck = n_ck;
  d->ready = false;
  return DIS_OK;
}

// Primitive and face-output buffers of one stage input.
struct WF {
  double* W;
  double* Fx;
  double* Fy;
};

// The adjoint's scratch buffers (idx < 0), or the stored set idx of the segment.
WF wf_at(dis_ctx* c, int idx) {
  dis_adj* d = c->adj;
  if (idx < 0) return WF{d->W, d->Fx, d->Fy};
  const size_t S = sizeof(double) * (size_t)c->nf * c->T;
  const size_t nfo = (size_t)(c->nf + n_extra(c->dim));
  char* b = d->wf + d->wf_bytes * (size_t)idx;
  WF w;
  w.W = (double*)b;
  w.Fx = (double*)(b + a256(S));
  w.Fy = (double*)(b + a256(S) + a256(sizeof(double) * nfo * c->NFX));
  return w;
}

StepArgs fwd_args(dis_ctx* c, int wf = -1) {
  StepArgs a{};
  a.pd = c->d_pd;
  a.T = c->T;
  a.NFX = c->NFX;
  a.NFY = c->NFY;
  const WF w = wf_at(c, wf);
  a.W = w.W;
  a.Fx = w.Fx;
  a.Fy = w.Fy;
  a.rate = c->rate;
  a.dtlast = c->dtlast;
  a.status = c->status;
  return a;
}

// Primitives and face outputs of state `src` into the context's W, Fx, Fy.
template <int DIM, bool RX>
void fwd_faces(dis_ctx* c, const double* src, bool rate_on, int wf = -1) {
  StepArgs a = fwd_args(c, wf);
  a.qsrc = src;
  k_prim<DIM, RX><<<(unsigned)c->seg_prim.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_prim, rate_on ? 1 : 0);
  k_flux<DIM, RX, 0><<<(unsigned)c->seg_fx.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fx);
  if constexpr (DIM == 2)
    k_flux<DIM, RX, 1><<<(unsigned)c->seg_fy.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_fy);
}

// One Runge-Kutta stage dst = a qn + b (src - dt D(src)) [+ sources if last];
// dt per patch from `dt`, or from the CFL rate when dt is null.
template <int DIM, bool RX>
void fwd_stage(dis_ctx* c, const double* src, const double* qn, double* dst, double a_, double b_, int last,
               const double* dt, bool rate_on, int wf = -1) {
  fwd_faces<DIM, RX>(c, src, rate_on, wf);
  StepArgs a = fwd_args(c, wf);
  a.qsrc = src;
  a.qn = qn;
  a.qdst = dst;
  a.a = a_;
  a.b = b_;
  a.last = last;
  a.dtfix = dt;
  k_update<DIM, RX><<<(unsigned)c->seg_cell.size(), SEG, 0, c->stream>>>(c->phys, a, c->d_seg_cell);
}

// One full step src -> dst with the recorded dt (scratch: st[0]).
template <int DIM, bool RX>
void fwd_step_fixed(dis_ctx* c, const double* src, double* dst, const double* dt) {
  double* q1 = c->adj->st[0];
  fwd_stage<DIM, RX>(c, src, src, q1, 0.0, 1.0, 0, dt, false);
  fwd_stage<DIM, RX>(c, q1, src, q1, 0.75, 0.25, 0, dt, false);
  fwd_stage<DIM, RX>(c, q1, src, dst, 1.0 / 3.0, 2.0 / 3.0, 1, dt, false);
}

template <int DIM, bool RX>
int adj_forward(dis_ctx* c, int n_steps, int mat, bool prescribed) {
  dis_adj* d = c->adj;
  const size_t SD = (size_t)c->nf * c->T;  // doubles per state
  const unsigned nc = (unsigned)c->seg_cell.size();
  ACU(cudaMemsetAsync(d->J, 0, sizeof(double), c->stream));
  for (int n = 0; n < n_steps; ++n) {
    double* ck = d->ck + (size_t)(n / d->every) * SD;
    double* dtn = d->dts + (size_t)n * c->np;
    if (c->fp32) {
      // FP32-bulk step; float64 checkpoints of its states
      if (n % d->every == 0)
        k_state32_to_64<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, c->d_pd, c->d_seg_cell, c->q32[0], ck, c->T);
      if (prescribed)
        ACU(cudaMemcpyAsync(c->dtfix, dtn, sizeof(double) * c->np, cudaMemcpyDeviceToDevice, c->stream));
      const int rc = dis_internal_steps(c, 1, prescribed);
      if (rc) return rc;
      if (!prescribed)
        ACU(cudaMemcpyAsync(dtn, c->dtlast, sizeof(double) * c->np, cudaMemcpyDeviceToDevice, c->stream));
      if (mat >= 0) {
        k_state32_to_64<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, c->d_pd, c->d_seg_cell, c->q32[0], d->tmp,
                                                            c->T);
        k_obj<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, d->tmp, c->T, dtn, mat, d->J);
      }
      continue;
    }
    if (n % d->every == 0)
      ACU(cudaMemcpyAsync(ck, c->q[0], sizeof(double) * SD, cudaMemcpyDeviceToDevice, c->stream));
    if (prescribed) {
      fwd_step_fixed<DIM, RX>(c, c->q[0], c->q[0], dtn);
    } else {
      ACU(cudaMemsetAsync(c->rate, 0, sizeof(unsigned long long) * c->np, c->stream));
      fwd_stage<DIM, RX>(c, c->q[0], c->q[0], c->q[1], 0.0, 1.0, 0, nullptr, true);
      fwd_stage<DIM, RX>(c, c->q[1], c->q[0], c->q[1], 0.75, 0.25, 0, nullptr, false);
      fwd_stage<DIM, RX>(c, c->q[1], c->q[0], c->q[0], 1.0 / 3.0, 2.0 / 3.0, 1, nullptr, false);
      ACU(cudaMemcpyAsync(dtn, c->dtlast, sizeof(double) * c->np, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (mat >= 0)
      k_obj<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, c->q[0], c->T, dtn, mat, d->J);
  }
  ACU(cudaGetLastError());
  return DIS_OK;
}

// Reverse kernels of one stage (REF: dual-number reference form of the
// hand-reversed local maps).
template <int DIM, bool RX, bool REF>
void reverse_kernels(dis_ctx* c, const AdjArgs& A) {
  cudaMemsetAsync(c->adj->Wb, 0, sizeof(double) * (size_t)c->nf * c->T, c->stream);
  k_adj_cell<DIM, RX, REF><<<(unsigned)c->seg_cell.size(), SEG, 0, c->stream>>>(c->phys, A, c->d_seg_cell);
  k_adj_face<DIM, RX, 0, REF><<<(unsigned)c->seg_fx.size(), SEG, 0, c->stream>>>(c->phys, A, c->d_seg_fx);
  if constexpr (DIM == 2)
    k_adj_face<DIM, RX, 1, REF><<<(unsigned)c->seg_fy.size(), SEG, 0, c->stream>>>(c->phys, A, c->d_seg_fy);
  k_adj_prim<DIM, RX, REF><<<(unsigned)c->seg_prim.size(), SEG, 0, c->stream>>>(c->phys, A, c->d_seg_prim);
}

template <int DIM, bool RX>
void reverse_stage(dis_ctx* c, const double* x, const double* opre, double a_, double b_, int last, int first,
                   const double* dt, unsigned pmask, int wf) {
  dis_adj* d = c->adj;
  const WF w = wf_at(c, wf);
  AdjArgs A{};
  A.pd = c->d_pd;
  A.T = c->T;
  A.NFX = c->NFX;
  A.NFY = c->NFY;
  A.x = x;
  A.W = w.W;
  A.Fx = w.Fx;
  A.Fy = w.Fy;
  A.obar = d->ob;
  A.opre = opre;
  A.xbar = d->xb;
  A.qnacc = d->acc;
  A.G = d->G;
  A.Wbar = d->Wb;
  A.theta = d->theta;
  A.dt = dt;
  A.a = a_;
  A.b = b_;
  A.last = last;
  A.first = first;
  A.pmask = pmask;
  // A material that is not a stiffened gas (the adjoint admits the
  // Romenskii solid): the hand-written reverses of the local maps cover the
  // stiffened gas only, so such contexts reverse every local map (recovery,
  // face states and Riemann problem, THINC-BVD edge values, source steps) by
  // its dual-number form, which evaluates the family's forward closure code.
  if (d->dual_riemann || general_closures(c)) reverse_kernels<DIM, RX, true>(c, A);
  else reverse_kernels<DIM, RX, false>(c, A);
}

template <int DIM, bool RX>
int adj_backward(dis_ctx* c, const double* qbar_packed, double jbar, int out_kind, double* out_packed,
                 unsigned pmask) {
  dis_adj* d = c->adj;
  const size_t SD = (size_t)c->nf * c->T;  // doubles per state
  const unsigned nc = (unsigned)c->seg_cell.size();
  ACU(cudaMemsetAsync(d->ob, 0, sizeof(double) * SD, c->stream));
  ACU(cudaMemsetAsync(d->theta, 0, sizeof(double) * NPARAM, c->stream));
  k_unpack<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, c->d_pd, c->d_seg_cell, qbar_packed, d->ob, c->T, 0);
  for (int s = d->n_ck - 1; s >= 0; --s) {
    const int n0 = s * d->every, n1 = std::min(d->n_steps, n0 + d->every);
    ACU(cudaMemcpyAsync(d->seg, d->ck + (size_t)s * SD, sizeof(double) * SD, cudaMemcpyDeviceToDevice, c->stream));
    // recompute the segment from its checkpoint with the recorded dt (the
    // forward run's kernels, so bit-identical), keeping every step's stage
    // states: q1, q3 and the state before the source steps
    for (int m = 0; m < n1 - n0; ++m) {
      const double* qn = d->seg + (size_t)m * SD;
      double* s3 = d->stg + (size_t)3 * m * SD;
      const double* dt = d->dts + (size_t)(n0 + m) * c->np;
      fwd_stage<DIM, RX>(c, qn, qn, s3, 0.0, 1.0, 0, dt, false, 3 * m);
      fwd_stage<DIM, RX>(c, s3, qn, s3 + SD, 0.75, 0.25, 0, dt, false, 3 * m + 1);
      fwd_stage<DIM, RX>(c, s3 + SD, qn, s3 + 2 * SD, 1.0 / 3.0, 2.0 / 3.0, 0, dt, false, 3 * m + 2);
      StepArgs a = fwd_args(c, 3 * m + 2);  // the same stage with the source steps: q^{n+1}
      a.qsrc = s3 + SD;
      a.qn = qn;
      a.qdst = d->seg + (size_t)(m + 1) * SD;
      a.a = 1.0 / 3.0;
      a.b = 2.0 / 3.0;
      a.last = 1;
      a.dtfix = dt;
      k_update<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, a, c->d_seg_cell);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const double* qn = d->seg + (size_t)(n - n0) * SD;
      const double* qnext = d->seg + (size_t)(n - n0 + 1) * SD;
      const double* s3 = d->stg + (size_t)3 * (n - n0) * SD;
      const double* dt = d->dts + (size_t)n * c->np;
      if (d->mat >= 0)
        k_obj_adj<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, qnext, d->ob, c->T, dt, d->mat, jbar);
      // stage inputs q1 (s3), q3 (s3 + SD) and the pre-source state (s3 + 2 SD),
      // with the primitives and face outputs the recomputation stored
      const int m = n - n0;
      reverse_stage<DIM, RX>(c, s3 + SD, s3 + 2 * SD, 1.0 / 3.0, 2.0 / 3.0, 1, 1, dt, pmask, 3 * m + 2);
      std::swap(d->ob, d->xb);
      reverse_stage<DIM, RX>(c, s3, nullptr, 0.75, 0.25, 0, 0, dt, pmask, 3 * m + 1);
      std::swap(d->ob, d->xb);
      reverse_stage<DIM, RX>(c, qn, nullptr, 0.0, 1.0, 0, 0, dt, pmask, 3 * m);
      k_adj_sum<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, d->xb, d->acc, d->ob, c->T);
    }
  }
  if (out_kind == DIS_CONSERVATIVE) {
    k_pack<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->d_pd, c->d_seg_cell, d->ob, out_packed, c->T);
  } else {
    fwd_faces<DIM, RX>(c, d->ck, false);  // primitives of the initial state
    k_adj_p2c<DIM, RX><<<nc, SEG, 0, c->stream>>>(c->phys, c->d_pd, c->d_seg_cell, d->W, d->ob, out_packed,
                                                  c->T, d->theta, pmask);
  }
  ACU(cudaGetLastError());
  return DIS_OK;
}

}  // namespace

extern "C" {

int dis_adj_forward(dis_ctx* c, int n_steps, int checkpoint_every, int objective_material, const double* dt_in,
                    double* dt_out, double* J_out) {
  if (!c) return dis_internal_error(DIS_EINVAL, "dis_adj_forward: NULL context");
  if (!c->have_state) return dis_internal_error(DIS_ESTATE, "dis_adj_forward: no state loaded");
  if (c->hancock)
    return dis_internal_error(DIS_EINVAL, "dis_adj_forward: the adjoint covers the Runge-Kutta scheme only");
  if (c->phys.m[0].two || c->phys.m[1].two)
    return dis_internal_error(DIS_EINVAL,
                              "dis_adj_forward: the adjoint does not cover two-closure reactive materials");
  if (c->phys.m[0].plastic == 3 || c->phys.m[1].plastic == 3)
    return dis_internal_error(DIS_EINVAL, "dis_adj_forward: the adjoint does not cover Johnson-Cook plasticity");
  for (int l = 0; l < 2; ++l)
    if (c->phys.m[l].eos != EOS_SG && c->phys.m[l].eos != EOS_ROMENSKII)
      return dis_internal_error(DIS_EINVAL, "dis_adj_forward: the adjoint does not cover JWL materials");
  if (general_closures(c) && c->phys.cyl)
    return dis_internal_error(DIS_EINVAL,
                              "dis_adj_forward: the adjoint of Romenskii materials is built for planar geometry "
                              "only");
  if (n_steps <= 0 || checkpoint_every <= 0)
    return dis_internal_error(DIS_EINVAL, "dis_adj_forward: n_steps and checkpoint_every must be positive");
  if (objective_material < -1 || objective_material > 1)
    return dis_internal_error(DIS_EINVAL, "dis_adj_forward: objective_material must be -1, 0 or 1");
  if (dt_in)
    for (long long k = 0; k < (long long)n_steps * c->np; ++k)
      if (!(dt_in[k] > 0.0) || !(dt_in[k] < INFINITY))
        return dis_internal_error(DIS_EINVAL, "dis_adj_forward: bad dt_in[%lld]", k);
  int rc = dis_internal_ensure_ws(c);
  if (rc) return rc;
  rc = adj_alloc(c, n_steps, std::min(checkpoint_every, n_steps));
  if (rc) return rc;
  dis_adj* d = c->adj;
  d->mat = objective_material;
  if (dt_in)
    ACU(cudaMemcpyAsync(d->dts, dt_in, sizeof(double) * (size_t)n_steps * c->np, cudaMemcpyHostToDevice,
                        c->stream));
  const bool rx = c->y >= 0;
  if (c->dim == 1) rc = rx ? adj_forward<1, true>(c, n_steps, d->mat, dt_in) : adj_forward<1, false>(c, n_steps, d->mat, dt_in);
  else rc = rx ? adj_forward<2, true>(c, n_steps, d->mat, dt_in) : adj_forward<2, false>(c, n_steps, d->mat, dt_in);
  if (rc) return rc;
  double J = 0.0;
  ACU(cudaMemcpyAsync(&J, d->J, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (dt_out)
    ACU(cudaMemcpyAsync(dt_out, d->dts, sizeof(double) * (size_t)n_steps * c->np, cudaMemcpyDeviceToHost,
                        c->stream));
  ACU(cudaStreamSynchronize(c->stream));
  if (J_out) *J_out = J;
  d->ready = true;
  return DIS_OK;
}

int dis_adjoint(dis_ctx* c, const double* qbar_final, int qbar_on_device, double jbar, int out_kind,
                double* grad_init, int grad_on_device, double* grad_params, unsigned param_mask) {
  if (!c || !grad_init) return dis_internal_error(DIS_EINVAL, "dis_adjoint: NULL argument");
  if (!c->adj || !c->adj->ready)
    return dis_internal_error(DIS_ESTATE, "dis_adjoint: no recorded forward run (call dis_adj_forward)");
  if (out_kind != DIS_CONSERVATIVE && out_kind != DIS_PRIMITIVE)
    return dis_internal_error(DIS_EINVAL, "dis_adjoint: bad out_kind");
  const size_t bytes = sizeof(double) * (size_t)c->nf * c->ncells;
  const double* qb = qbar_final;
  if (!qbar_final) {
    ACU(cudaMemsetAsync(c->io, 0, bytes, c->stream));
    qb = c->io;
  } else if (!qbar_on_device) {
    ACU(cudaMemcpyAsync(c->io, qbar_final, bytes, cudaMemcpyHostToDevice, c->stream));
    qb = c->io;
  }
  double* out = grad_on_device ? grad_init : c->io;
  const unsigned pmask = grad_params ? (param_mask & ((1u << NPARAM) - 1u)) : 0u;
  const bool rx = c->y >= 0;
  int rc;
  if (c->dim == 1)
    rc = rx ? adj_backward<1, true>(c, qb, jbar, out_kind, out, pmask) : adj_backward<1, false>(c, qb, jbar, out_kind, out, pmask);
  else
    rc = rx ? adj_backward<2, true>(c, qb, jbar, out_kind, out, pmask) : adj_backward<2, false>(c, qb, jbar, out_kind, out, pmask);
  if (rc) return rc;
  double th[NPARAM];
  ACU(cudaMemcpyAsync(th, c->adj->theta, sizeof th, cudaMemcpyDeviceToHost, c->stream));
  if (!grad_on_device) ACU(cudaMemcpyAsync(grad_init, c->io, bytes, cudaMemcpyDeviceToHost, c->stream));
  ACU(cudaStreamSynchronize(c->stream));
  if (grad_params)
    for (int k = 0; k < NPARAM; ++k) grad_params[k] = ((pmask >> k) & 1u) ? th[k] : 0.0;
  return DIS_OK;
}

int dis_adj_reference(dis_ctx* c, int on) {
  if (!c) return dis_internal_error(DIS_EINVAL, "dis_adj_reference: NULL context");
  if (!c->adj) c->adj = new (std::nothrow) dis_adj();
  if (!c->adj) return dis_internal_error(DIS_ENOMEM, "dis_adj_reference: out of host memory");
  c->adj->dual_riemann = on ? 1 : 0;
  return DIS_OK;
}

}  // extern "C"
