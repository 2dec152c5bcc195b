// ctx.cuh - the library context shared by the translation units of libdis
// (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/dis.h"
#include "fused32.cuh"

using dis::PatchDev;
using dis::Phys;
using dis::PhysF;

struct dis_adj;  // adjoint buffers and the recorded forward run (adjoint.cu)

struct dis_ctx {
  int dim = 1, np = 0, y = -1, nf = 0;
  dis_options opt{};
  Phys phys{};
  PhysF physf{};
  bool fp32 = false;
  bool have_mats = false, have_state = false;
  std::vector<dis_patch> patches;
  std::vector<PatchDev> pd;
  long long T = 0, NFX = 0, NFY = 0, ncells = 0;
  std::vector<int4> seg_prim, seg_fx, seg_fy, seg_cell;
  std::vector<int> seg_cell0;  // first seg_cell segment of each patch (np + 1)
  cudaStream_t stream = nullptr;
  int device = 0;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false, ws_ready = false;
  double* q[2] = {nullptr, nullptr};  // q^n, stage buffer
  double* W = nullptr;
  double* E = nullptr;  // MUSCL-Hancock evolved edge states (2 dim nf planes)
  bool hancock = false;
  double* Fx = nullptr;
  double* Fy = nullptr;
  double* io = nullptr;
  unsigned long long* rate = nullptr;
  double* dtfix = nullptr;
  double* dtlast = nullptr;
  int* status = nullptr;
  // FP32-bulk stage kernel: tile tables per tile shape; variant v = tile
  // shape v % 3 with the register budget v / 3 (2D: 3 or 4 resident CTAs per
  // SM; 1D: none or 64 registers per thread); chosen variant and tuned
  // per-step times
  std::vector<int4> tiles[3];
  int4* d_tiles[3] = {nullptr, nullptr, nullptr};
  int variant = -1;
  double tune_ms[DIS_NVARIANTS] = {};
  // 1D FP32-bulk batches: schedule 0 = one launch per kernel and stage
  // (captured per step), 1 = the persistent batch kernel (one launch for all
  // steps of a dis_step call, one CTA per problem), -1 = chosen by the tuner;
  // problems in launch order (longest first) and the first tile of each
  // problem per tile shape; tuned one-step times of the persistent kernel
  int schedule = -1, schedule_req = -1;
  std::vector<int> order;
  std::vector<int> tile0[3];
  int* d_order = nullptr;
  int* d_tile0[3] = {nullptr, nullptr, nullptr};
  double tune_batch_ms[DIS_NVARIANTS] = {};
  // FP32-bulk buffers: q^n and two stage buffers of NF + 1 float32 planes
  // (step32.cuh): a stage kernel reads the halo of its source from
  // neighbouring tiles, so no stage may write the buffer it reads.  rate
  // holds 2 np values: the CFL rate of q^n, and that of q^{n+1} accumulated
  // by the last stage; rate_valid: the first holds the rate of the state
  float* q32[3] = {nullptr, nullptr, nullptr};
  bool rate_valid = false;
  PatchDev* d_pd = nullptr;
  // dis_query: per-segment partials and the final totals (workspace); which
  // patches hold a state; events around the last step call; step counts
  double* qpart = nullptr;
  double* qout = nullptr;
  std::vector<char> patch_set;
  cudaEvent_t ev_step[2] = {nullptr, nullptr};
  bool ev_recorded = false;
  long long steps_total = 0, last_steps = 0;
  int4 *d_seg_prim = nullptr, *d_seg_fx = nullptr, *d_seg_fy = nullptr, *d_seg_cell = nullptr;
  long long launches = 0;
  // one captured time step per dt mode (0: CFL, 1: prescribed), replayed per step
  cudaStream_t cap = nullptr;
  // captured steps: index mode (0 CFL dt, 1 fixed dt) + 2 parity (the
  // FP32-bulk MUSCL-Hancock step alternates its two state buffers; parity 1:
  // the state is in the buffer carved second)
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  long long graph_launches[4] = {0, 0, 0, 0};
  float* q32_home = nullptr;  // the buffer carved first
  bool use_graphs = true;
  dis_adj* adj = nullptr;  // created by the first dis_adj_forward
  // pipelined host transfers (dis_set_state_async / dis_get_state_async): two
  // staging buffers per direction, a copy stream per direction, and events
  // that order the copies against the conversions on the context's stream
  double* xin[2] = {nullptr, nullptr};
  double* xout[2] = {nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t in_done[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
  cudaEvent_t out_ready[2] = {nullptr, nullptr}, out_free[2] = {nullptr, nullptr};
  int in_idx = 0, out_idx = 0;
};

// Error text for the thread's dis_last_error (returns code).
int dis_internal_error(int code, const char* fmt, ...);
// Allocate (if the caller bound none) and fill the workspace tables.
int dis_internal_ensure_ws(dis_ctx* c);
// Enqueue n time steps (CFL dt, or the per-patch dt in c->dtfix when fixed).
int dis_internal_steps(dis_ctx* c, int n, bool fixed);
// Release the adjoint buffers of a context.
void dis_internal_adj_free(dis_ctx* c);
// Hooks of dis_internal_step64_hooked: before(user, stage, stage source
// state), after_flux(user, stage), enqueued on the context's stream.
struct StepHooks {
  void (*before)(void* user, int stage, double* qsrc) = nullptr;
  void (*after_flux)(void* user, int stage) = nullptr;
  void* user = nullptr;
};
int dis_internal_step64_hooked(dis_ctx* c, const StepHooks& h);
// Per-patch CFL rate sum_d (|u_d| + c_L) / dx_d, max over the interior
// cells of q^n (host, np values; synchronises).
int dis_internal_rates(dis_ctx* c, double* host);
// The same into c->rate (np values, the bits of doubles), without waiting.
int dis_internal_rates_enqueue(dis_ctx* c);
// dis_create that accepts DIS_BC_EXTERNAL sides (the AMR levels).
int dis_internal_create_external(int dim, int n_patches, const dis_patch* patches, int reactive_material,
                                 const dis_options* opt, void* stream, dis_ctx** out);
// A Romenskii or JWL material in the context (the kernels with the general
// closures run).
bool general_closures(const dis_ctx* c);
// FP32-bulk MUSCL-Hancock (hancock32_1d.cu, hancock32_2d.cu): one step of
// variant v (the tile shape) from a.src to a.dst; the persistent 1D batch
// form, n steps alternating between q0 (the state) and q1.
void hancock32_step_1d(dis_ctx* c, cudaStream_t st, const dis::StepArgs32& a, int v);
void hancock32_step_2d(dis_ctx* c, cudaStream_t st, const dis::StepArgs32& a, int v);
void hancock32_batch_1d(dis_ctx* c, cudaStream_t st, const dis::StepArgs32& a, float* q0, float* q1, int n,
                        int scratch, int v);
