// Total BA cost without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a cost:
// code running under a fixed memory pool that is already fully handed out, a host
// callback or a real-time thread that must not enter the CUDA allocator (whose calls
// can synchronise the device and take unbounded time), or a process whose device
// memory is owned by another framework.  gpo_ba_cost_noalloc serves them: the caller
// passes its own device buffers for the problem and for the result, and the
// reduction's scratch (one partial sum per CTA and a completion counter) lives in a
// file-scope static device array of fixed size instead of allocated memory.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gpo.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;                                    // partials held
constexpr long long kMaxEdges = (long long)kThreads * kMaxBlocks;   // 2,097,152 edges
constexpr int kMaxDevices = 64;

struct Scratch {
  double part[kMaxBlocks];
  unsigned int ticket;
};

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
Scratch* g_addr[kMaxDevices] = {};   // device address of g_scratch, per device

__device__ void residual_cost(const double* c, const double* X, const double* z, double delta, double* out) {
  // R = I + a [w]x + b [w]x^2 (Rodrigues), a = sin t / t, b = (1 - cos t) / t^2
  const double t2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
  double a, b;
  if (t2 < 1e-8) {
    a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
  } else {
    const double t = sqrt(t2);
    double s, co;
    sincos(t, &s, &co);
    a = s / t;
    b = (1.0 - co) / t2;
  }
  const double wx = c[1] * X[2] - c[2] * X[1], wy = c[2] * X[0] - c[0] * X[2], wz = c[0] * X[1] - c[1] * X[0];
  const double wdx = c[0] * X[0] + c[1] * X[1] + c[2] * X[2];
  // [w]x^2 X = w (w.X) - t^2 X
  const double P0 = X[0] + a * wx + b * (c[0] * wdx - t2 * X[0]) + c[3];
  const double P1 = X[1] + a * wy + b * (c[1] * wdx - t2 * X[1]) + c[4];
  const double P2 = X[2] + a * wz + b * (c[2] * wdx - t2 * X[2]) + c[5];
  const double p0 = -P0 / P2, p1 = -P1 / P2;
  const double r2 = p0 * p0 + p1 * p1;
  const double fd = c[6] * (1.0 + c[7] * r2 + c[8] * r2 * r2);
  const double e0 = fd * p0 - z[0], e1 = fd * p1 - z[1];
  const double s = e0 * e0 + e1 * e1;
  *out = 0.5 * ((delta > 0.0 && s > delta * delta) ? 2.0 * delta * sqrt(s) - delta * delta : s);
}

__global__ void __launch_bounds__(kThreads) k_cost_noalloc(const double* cams, const double* pts, const int* ci,
                                                          const int* pi, const double* obs, long long n, double delta,
                                                          double* out, Scratch* scr) {
  __shared__ double red[kThreads];
  __shared__ bool last;
  const long long e = (long long)blockIdx.x * kThreads + threadIdx.x;
  double v = 0.0;
  if (e < n) residual_cost(cams + 9 * (size_t)ci[e], pts + 3 * (size_t)pi[e], obs + 2 * e, delta, &v);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scr->part[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(&scr->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) acc += scr->part[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

extern "C" gpo_status gpo_ba_cost_noalloc(int32_t device, void* cuda_stream, const double* cams,
                                          const double* points, const int32_t* cam_idx, const int32_t* pt_idx,
                                          const double* obs, int64_t n_edges, double huber_delta,
                                          double* cost_out) {
  if (n_edges < 0 || n_edges > kMaxEdges || !cost_out || device < 0 || device >= kMaxDevices)
    return GPO_ERR_ARG;   // n_edges beyond 2,097,152 exceeds the static scratch
  if (n_edges > 0 && (!cams || !points || !cam_idx || !pt_idx || !obs)) return GPO_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return GPO_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return GPO_ERR_CUDA;
  gpo_status st = GPO_OK;
  Scratch* scr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) st = GPO_ERR_CUDA;
      else g_addr[device] = static_cast<Scratch*>(p);
    }
    scr = g_addr[device];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (st == GPO_OK) {
    const int blocks = n_edges > 0 ? (int)((n_edges + kThreads - 1) / kThreads) : 1;
    // the completion counter must start at zero; the partials are overwritten
    if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) st = GPO_ERR_CUDA;
    if (st == GPO_OK) {
      k_cost_noalloc<<<blocks, kThreads, 0, s>>>(cams, points, cam_idx, pt_idx, obs, n_edges, huber_delta, cost_out,
                                                scr);
      if (cudaGetLastError() != cudaSuccess) st = GPO_ERR_CUDA;
    }
  }
  cudaSetDevice(prev);
  return st;
}
