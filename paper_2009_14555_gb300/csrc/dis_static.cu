// dis_static.cu - CFL time step of a packed state with no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a time
// step: code running where an allocation could synchronise the device or be
// refused (a host callback, a region that a framework's caching allocator has
// locked, a process whose device memory was reserved up front).  This entry
// point computes the per-patch CFL time step of a conservative state that the
// caller already holds in device memory, using only a fixed scratch area in
// this library's image (DIS_STATIC_MAX_PATCHES entries, about 0.7 MB per
// device, held by every GPU that loads the library until the process exits).
//
// It is a variant of the CFL reduction done by the stepping kernels: the same
// rate per cell, sum_d (|u_d| + c_L) / dx_d, its maximum per patch by warp
// shuffles and one atomic per warp, then dt = CFL / max.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/dis.h"
#include "physics.cuh"

using namespace dis;

namespace {

constexpr int kMaxPatches = DIS_STATIC_MAX_PATCHES;
constexpr int kMaxDevices = 64;

struct StaticPatch {
  long long poff;  // first value of the patch in the packed state
  int nx, ny;
  double dx, dy;
};

struct StaticScratch {
  unsigned long long rate[kMaxPatches];  // per-patch max rate (bits of a positive double)
  int bad[kMaxPatches];                  // per patch: a cell without a real sound speed or density
  StaticPatch patch[kMaxPatches];
};

// One copy per device that loads the library.  In host code this name is
// only a stand-in: its device address is looked up once per device below.
static __device__ __align__(256) StaticScratch g_scratch;

std::mutex g_mu;
StaticScratch* g_addr[kMaxDevices] = {nullptr};

template <int DIM, bool RX>
__global__ void __launch_bounds__(256) k_cfl_static(Phys P, const double* __restrict__ q,
                                                    StaticScratch* S) {
  const int p = blockIdx.y;
  const StaticPatch sp = S->patch[p];
  const long long n = (long long)sp.nx * sp.ny;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (c < n) {
    using L = Lay<DIM, RX>;
    const double* b = q + sp.poff + c;
    const double phi = b[L::PHI * n], a1 = b[L::A1 * n], a2 = b[L::A2 * n];
    const double rho = a1 + a2;
    const double mx = b[L::MX * n];
    double my = 0.0, V12 = 0.0, V21 = 0.0, arl = 0.0;
    if constexpr (DIM == 2) {
      my = b[L::MY * n];
      V12 = b[L::V12 * n];
      V21 = b[L::V21 * n];
    }
    if constexpr (RX) arl = b[L::AL * n];
    const double u = mx / rho, v = my / rho;
    const Strain s = strain_of(b[L::V11 * n], V12, V21, b[L::V22 * n], b[L::V33 * n]);
    const double KE = 0.5 * (mx * u + my * v);
    const double pr = (b[L::E * n] - KE - ref_energy(P, phi, a1, a2, arl, s.J2)) / xi_of(P, phi);
    const double cL2 = cL2_of(P, phi, rho, pr, s.J2, a1 / phi, a2 / (1.0 - phi));
    const double cL = sqrt(fmax(cL2, 0.0));
    r = (fabs(u) + cL) / sp.dx;
    if (DIM == 2) r += (fabs(v) + cL) / sp.dy;
    // a state that has lost hyperbolicity (or its density, or is not finite)
    // gets no time step: the patch's dt becomes NaN
    if (!(cL2 > 0.0) || !(rho > 0.0) || !(r < INFINITY)) S->bad[p] = 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0 && r > 0.0)
    atomicMax(&S->rate[p], (unsigned long long)__double_as_longlong(r));
}

__global__ void k_dt_static(const StaticScratch* S, int np, double cfl, double* dt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) dt[p] = S->bad[p] ? __longlong_as_double(0x7ff8000000000000LL)
                                : cfl / __longlong_as_double((long long)S->rate[p]);
}

MatDev dev_material(const dis_material& m) {
  MatDev d{};
  d.gamma = m.gamma;
  d.pinf = m.p_inf;
  d.einf = m.e_inf;
  d.G = m.G;
  d.Q = m.Q;
  d.iGm1 = 1.0 / (m.gamma - 1.0);
  d.gi = m.gamma * d.iGm1;
  d.kap = m.gamma * m.p_inf * d.iGm1;
  d.gG = m.gamma * m.G * d.iGm1;
  d.GoG = m.G * d.iGm1;
  d.reactive = m.reactive;
  d.eos = m.eos;
  d.rho0 = m.rho0;
  d.K0 = m.K0;
  d.ar = m.alpha;
  d.br = m.beta;
  d.jA = m.jwl_A;
  d.jB = m.jwl_B;
  d.jR1 = m.jwl_R1;
  d.jR2 = m.jwl_R2;
  d.two = 0;
  return d;
}

}  // namespace

// Error text shared with the rest of the C ABI (dis_last_error).
int dis_internal_error(int code, const char* fmt, ...);

extern "C" int dis_cfl_dt_static(int dim, int n_patches, const dis_patch* patches,
                                 const dis_material* materials, int reactive_material, double cfl,
                                 const double* d_state, double* d_dt, void* stream) {
  // Argument checks on the host, before any device work.
  if (dim != 1 && dim != 2) return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: dim must be 1 or 2");
  if (!patches || !materials || !d_state || !d_dt)
    return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: NULL argument");
  if (n_patches <= 0 || n_patches > kMaxPatches)
    return dis_internal_error(DIS_EINVAL,
                              "dis_cfl_dt_static: %d patches requested, the static scratch holds 1..%d",
                              n_patches, kMaxPatches);
  if (!(cfl > 0.0 && cfl <= 1.0)) return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: cfl not in (0, 1]");
  if (reactive_material < -1 || reactive_material > 1)
    return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: reactive_material must be -1, 0 or 1");
  for (int l = 0; l < 2; ++l) {
    if (!(materials[l].gamma > 1.0)) return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: gamma <= 1");
    if (materials[l].reactive && materials[l].prod_gamma > 0.0)
      return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: a reactive material with two closures is not covered");
  }
  const int nf = (dim == 2 ? 11 : 8) + (reactive_material >= 0 ? 1 : 0);
  long long maxcells = 0;
  for (int p = 0; p < n_patches; ++p) {
    const int ny = dim == 2 ? patches[p].ny : 1;
    if (patches[p].nx < 1 || ny < 1 || !(patches[p].dx > 0) || (dim == 2 && !(patches[p].dy > 0)))
      return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: patch %d has a bad size", p);
    const long long n = (long long)patches[p].nx * ny;
    if (n > maxcells) maxcells = n;
  }
  if (maxcells > (1LL << 31)) return dis_internal_error(DIS_EINVAL, "dis_cfl_dt_static: patch too large");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return dis_internal_error(DIS_ECUDA, "dis_cfl_dt_static: no usable current device");
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    // Set-up, once per device, with that device current: the device address
    // of the static scratch.
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr)
      return dis_internal_error(DIS_ECUDA, "dis_cfl_dt_static: cudaGetSymbolAddress failed: %s",
                                cudaGetErrorString(e));
    g_addr[dev] = (StaticScratch*)ptr;
  }
  StaticScratch* S = g_addr[dev];
  // Patch descriptors go into the static area by a copy from pageable host
  // memory, which the runtime stages before returning, so the host array may
  // be reused afterwards (the lock above serialises its use).  Such a copy
  // cannot be part of a captured graph: the call must not be made while its
  // stream is being captured.
  static StaticPatch staging[kMaxPatches];
  long long poff = 0;
  for (int p = 0; p < n_patches; ++p) {
    const int ny = dim == 2 ? patches[p].ny : 1;
    staging[p].poff = poff;
    staging[p].nx = patches[p].nx;
    staging[p].ny = ny;
    staging[p].dx = patches[p].dx;
    staging[p].dy = dim == 2 ? patches[p].dy : 1.0;
    poff += (long long)nf * patches[p].nx * ny;
  }
  if (cudaMemcpyAsync(S->patch, staging, sizeof(StaticPatch) * n_patches, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return dis_internal_error(DIS_ECUDA, "dis_cfl_dt_static: descriptor copy failed");
  // the per-patch maxima and flags start at zero on every call (the area
  // keeps the last call's values)
  if (cudaMemsetAsync(S->rate, 0, sizeof(unsigned long long) * n_patches, st) != cudaSuccess ||
      cudaMemsetAsync(S->bad, 0, sizeof(int) * n_patches, st) != cudaSuccess)
    return dis_internal_error(DIS_ECUDA, "dis_cfl_dt_static: clearing the scratch failed");
  Phys P{};
  P.m[0] = dev_material(materials[0]);
  P.m[1] = dev_material(materials[1]);
  P.y = reactive_material;
  P.cfl = cfl;
  const dim3 grid((unsigned)((maxcells + 255) / 256), (unsigned)n_patches);
  const bool rx = reactive_material >= 0;
  if (dim == 1) {
    if (rx) k_cfl_static<1, true><<<grid, 256, 0, st>>>(P, d_state, S);
    else k_cfl_static<1, false><<<grid, 256, 0, st>>>(P, d_state, S);
  } else {
    if (rx) k_cfl_static<2, true><<<grid, 256, 0, st>>>(P, d_state, S);
    else k_cfl_static<2, false><<<grid, 256, 0, st>>>(P, d_state, S);
  }
  k_dt_static<<<(n_patches + 255) / 256, 256, 0, st>>>(S, n_patches, cfl, d_dt);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dis_internal_error(DIS_ECUDA, "dis_cfl_dt_static: launch failed: %s", cudaGetErrorString(e));
  return DIS_OK;
}
