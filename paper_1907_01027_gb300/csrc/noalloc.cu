// Operator application that allocates no device memory: the sweep's scratch lives in a fixed file-scope
// device array instead of the buffers lmdg_setup allocates.
//
// Who needs this: code that runs where cudaMalloc is not an option -- a host framework that owns every byte
// of device memory through its own pool and forbids other allocations, a latency-critical loop that cannot
// afford cudaMalloc's implicit device synchronisation, or a library embedded in another runtime that hands
// it only input and output buffers.  Such callers pass all inputs and outputs as device pointers and get
// the scratch from here.
//
// The scratch array below is reserved on every GPU that loads this library, for the lifetime of the
// process.  All calls share it and it keeps the last call's contents; the control words that must start at
// zero are cleared by every call.  Calls whose kernels overlap on the GPU (different streams, or different
// host threads on the same device) race on this scratch and must be serialised by the caller.
#include <mutex>

#include "lmdg_internal.h"
#include "krylov.h"

namespace lmdg {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxDirections = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char *base = nullptr;   // device address of g_scratch on this device
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

__global__ void identity_kernel(int *perm, int count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) perm[k] = k;
}

// bad[0] = number of directions whose signs do not match their quadrant slot (slots of n_omega / 4 directions
// in the order (+,+), (-,+), (-,-), (+,-)) or that lie on an axis
__global__ void quadrant_check_kernel(int nang, const double *__restrict__ ox, const double *__restrict__ oy,
                                      unsigned *__restrict__ bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nang) return;
  const int quad = k / (nang / 4);
  const double a = ox[k], b = oy[k];
  const bool ok = (quad == 0 && a > 0 && b > 0) || (quad == 1 && a < 0 && b > 0) ||
                  (quad == 2 && a < 0 && b < 0) || (quad == 3 && a > 0 && b < 0);
  if (!ok) atomicAdd(bad, 1u);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Groups of at most 8 warps x kMaxA directions, every group non-empty (a fixed shape: no occupancy query).
SweepGeom geom_for(int n, int nq) {
  SweepGeom g;
  g.strips = (n + 31) / 32;
  g.groups = (nq + 8 * kMaxA - 1) / (8 * kMaxA);
  while (g.groups > 1 && (g.groups - 1) * ((nq + g.groups - 1) / g.groups) >= nq) --g.groups;
  const int gsize = (nq + g.groups - 1) / g.groups;
  g.apw = (gsize + 7) / 8;
  g.warps = (gsize + g.apw - 1) / g.apw;
  return g;
}

// Device address of the scratch for the current device; first use on a device (with that device current)
// looks the symbol up and writes the identity direction permutation into the scratch.
int scratch_for_current_device(unsigned char **base, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LMDG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceScratch &d = g_dev[dev];
  if (!d.ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return LMDG_ERR_CUDA;
    d.base = static_cast<unsigned char *>(p);
    int *perm = reinterpret_cast<int *>(d.base);
    identity_kernel<<<(kMaxDirections + 255) / 256, 256, 0, s>>>(perm, kMaxDirections);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return LMDG_ERR_CUDA;
    d.ready = true;
  }
  *base = d.base;
  return 0;
}

}  // namespace
}  // namespace lmdg

using namespace lmdg;

extern "C" int lmdg_sweep_noalloc(int variant, int n, double h, int n_omega, const double *ox, const double *oy,
                                  const double *w, const double *sigma_t, const double *sigma_s_over_eps,
                                  const double *x, double *y, long long spin_limit, void *stream) {
  if (variant < LMDG_STD || variant > LMDG_RLM || n < 1 || !(h > 0) || n_omega < 4 || n_omega % 4 ||
      n_omega > kMaxDirections || !ox || !oy || !w || !sigma_t || !sigma_s_over_eps || !x || !y ||
      spin_limit < 1)
    return LMDG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nq = n_omega / 4;
  const SweepGeom g = geom_for(n, nq);
  const size_t nx = (size_t)n * n;
  const int NR = variant == LMDG_RLM ? 6 : 4;
  // scratch layout: [perm (kMaxDirections ints)] [quadrature moments] [direction check word] [control words]
  // [cell inputs] [partials] [strip traces]
  const size_t off_qm = align256(sizeof(int) * kMaxDirections);
  const size_t off_chk = off_qm + align256(sizeof(double) * 5);
  const size_t off_ctrl = off_chk + align256(sizeof(unsigned));
  const size_t off_cell = off_ctrl + align256(sizeof(unsigned) * (2 + (size_t)g.units()));
  const size_t off_cellh = off_cell + align256(sizeof(double) * 4 * nx);
  const size_t off_part = off_cellh + align256(sizeof(double) * nx);
  const size_t off_ytr = off_part + align256(sizeof(double) * 4 * g.groups * nx * NR);
  const size_t need = off_ytr + sizeof(double) * (size_t)n_omega * g.strips * n * kTraceStride;
  if (need > kScratchBytes) return LMDG_ERR_ARG;   // problem too large for the fixed scratch
  unsigned char *base = nullptr;
  if (int e = scratch_for_current_device(&base, s)) return e;
  // the directions must come grouped by quadrant: checked on the device before the sweep (they stay there)
  {
    unsigned *chk = reinterpret_cast<unsigned *>(base + off_chk);
    unsigned bad = 0;
    if (cudaMemsetAsync(chk, 0, sizeof(unsigned), s) != cudaSuccess) return LMDG_ERR_CUDA;
    add_launches(1);
    quadrant_check_kernel<<<(n_omega + 255) / 256, 256, 0, s>>>(n_omega, ox, oy, chk);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&bad, chk, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LMDG_ERR_CUDA;
    if (bad) return LMDG_ERR_QUAD;
  }

  SweepArgs<double> a{};
  a.ni = n; a.nj = n; a.nq = nq; a.nang = n_omega; a.nx = (int)nx;
  a.h = h; a.eps = 1.0;
  a.g = g;
  a.pd.ox = const_cast<double *>(ox);
  a.pd.oy = const_cast<double *>(oy);
  a.pd.w = const_cast<double *>(w);
  a.pd.sigt = const_cast<double *>(sigma_t);
  a.pd.sse = const_cast<double *>(sigma_s_over_eps);
  a.q_per_angle = 0;
  a.X = x;
  a.p1ra = nullptr;
  a.source = 0;
  a.part = reinterpret_cast<double *>(base + off_part);
  a.pq0 = 0;
  a.npq = 4 * g.groups;
  a.psi = nullptr;
  a.psi_bf16 = 0;
  a.perm = reinterpret_cast<const int *>(base);
  a.ytr = reinterpret_cast<double *>(base + off_ytr);
  a.ctrl = reinterpret_cast<unsigned *>(base + off_ctrl);   // cleared by launch_sweep before the kernel
  a.cellsrc = reinterpret_cast<const double *>(base + off_cell);
  a.cellsh = reinterpret_cast<const double *>(base + off_cellh);
  a.spin_limit = spin_limit;
  // strip traces start empty (the buffer is shared with earlier calls of any size)
  if (fill_u32(reinterpret_cast<unsigned *>(base + off_ytr), kTraceEmpty,
               2 * (size_t)n_omega * g.strips * n * kTraceStride, s) != cudaSuccess)
    return LMDG_ERR_CUDA;
  double *qm = reinterpret_cast<double *>(base + off_qm);
  if (quad_moments(n_omega, ox, oy, w, qm, s) != cudaSuccess) return LMDG_ERR_CUDA;
  if (launch_sweep<double>(variant, a, s) != cudaSuccess) return LMDG_ERR_CUDA;
  if (launch_epilogue<double>(variant, (int)nx, 4 * g.groups, h, a.part, x, sigma_s_over_eps, sigma_t, qm, nullptr,
                              nullptr, 0, y, s) != cudaSuccess)
    return LMDG_ERR_CUDA;
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, a.ctrl + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LMDG_ERR_CUDA;
  return err ? LMDG_ERR_TIMEOUT : 0;
}
