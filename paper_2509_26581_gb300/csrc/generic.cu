// Generic edge kinds compiled into the library and differentiated in forward mode: the
// paper's descriptor workflow (Sec. III: a user declares the residual of a constraint
// over its vertices and the library derives the Jacobian, Listings 1-5 with the circle
// example) on a general graph of equal-size vertices.  Each kind is a struct with its
// arity A, vertex dimension D, residual size M and a residual template evaluated on
// dual numbers; the solver is LM with a block-Jacobi PCG on the full damped system
// (D x D vertex blocks), all vector work in FP64 kernels, the LM and PCG scalars on the
// host (this path serves small, general problems; the bundle-adjustment and
// visual-inertial path is the one tuned for throughput).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "autodiff.cuh"
#include "gpo.h"

namespace {

using gpo::Dual;
using gpo::dvar;

// ---------------------------------------------------------------- registered kinds

// r = x^2 + y^2 - R^2 (the circle constraint of the paper's example; meas = R).
struct CircleEdge {
  static constexpr int A = 1, D = 2, M = 1, MEAS = 1;
  template <class T>
  __device__ static void residual(const T (&x)[A * D], const double* meas, T (&r)[M]) {
    r[0] = (x[0] * x[0] + x[1] * x[1]) + (-meas[0] * meas[0]);
  }
};

// r = |x_i - x_j|^2 - d^2 between two vertices (meas = d).
struct DistanceEdge {
  static constexpr int A = 2, D = 2, M = 1, MEAS = 1;
  template <class T>
  __device__ static void residual(const T (&x)[A * D], const double* meas, T (&r)[M]) {
    const T dx = x[0] - x[2], dy = x[1] - x[3];
    r[0] = (dx * dx + dy * dy) + (-meas[0] * meas[0]);
  }
};

constexpr int kGD = 2;   // vertex dimension of the registered kinds

// Device view of one kind's edges.
struct GenSet {
  int n;                 // edges
  const int* vid;        // [n][A] vertex indices
  const double* meas;    // [n][MEAS]
  const double* delta;   // [n] Huber threshold (0: none)
  const unsigned char* active;   // [n]
  double* r;             // [n][M] weighted residual
  double* J;             // [n][M][A D] weighted rows (fixed vertices' columns zero)
};

__device__ __forceinline__ double huber_rho_d(double s, double delta) {
  if (delta > 0.0 && s > delta * delta) return 2.0 * delta * sqrt(s) - delta * delta;
  return s;
}
__device__ __forceinline__ double huber_w_d(double s, double delta) {
  if (!(delta > 0.0 && s > delta * delta)) return 1.0;
  return sqrt(delta / sqrt(s));
}

// Per edge: mode 0 residual and rows at x (cost partials too), mode 1 cost at x.
template <class E>
__global__ void __launch_bounds__(256) k_gen_eval(GenSet s, const double* x, const unsigned char* fixed, int mode,
                                                  double* cost_part) {
  constexpr int A = E::A, D = E::D, M = E::M, N = A * D;
  __shared__ double red[256];
  const int e = blockIdx.x * 256 + threadIdx.x;
  double c = 0.0;
  if (e < s.n && s.active[e]) {
    Dual<N> xv[N];
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) xv[a * D + k] = dvar<N>(x[(size_t)D * s.vid[A * e + a] + k], a * D + k);
    Dual<N> r[M];
    E::template residual<Dual<N>>(xv, s.meas + (size_t)E::MEAS * e, r);
    double q = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) q += r[m].v * r[m].v;
    c = 0.5 * huber_rho_d(q, s.delta[e]);
    if (mode == 0) {
      const double w = huber_w_d(q, s.delta[e]);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        s.r[(size_t)M * e + m] = w * r[m].v;
#pragma unroll
        for (int a = 0; a < A; ++a) {
          const bool fx = fixed[s.vid[A * e + a]] != 0;
#pragma unroll
          for (int k = 0; k < D; ++k) s.J[((size_t)M * e + m) * N + a * D + k] = fx ? 0.0 : w * r[m].g[a * D + k];
        }
      }
    }
  } else if (e < s.n && mode == 0) {
    for (int m = 0; m < M; ++m) {
      s.r[(size_t)M * e + m] = 0.0;
      for (int j = 0; j < N; ++j) s.J[((size_t)M * e + m) * N + j] = 0.0;
    }
  }
  red[threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) cost_part[blockIdx.x] = red[0];
}

// w_e = J_e v (the edge's rows times its vertices' entries of v)
template <class E>
__global__ void __launch_bounds__(256) k_gen_jv(GenSet s, const double* v, double* w) {
  constexpr int A = E::A, D = E::D, M = E::M, N = A * D;
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= s.n) return;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) acc += s.J[((size_t)M * e + m) * N + a * D + k] * v[(size_t)D * s.vid[A * e + a] + k];
    w[(size_t)M * e + m] = acc;
  }
}

// Incidence of a vertex: (kind, edge, slot) triples in a fixed order, CSR by vertex.
struct GenInc {
  const int* off;        // [V + 1]
  const int* kind;       // [nnz] index of the edge set
  const int* edge;       // [nnz]
  const int* slot;       // [nnz]
};
struct GenSets {
  GenSet s[2];
  int A[2], M[2];
  const double* w[2];    // per set: w_e (products) or r_e (gradient)
};

// Per vertex: out_v = sum over its edges of J_slot^T src_e (+ lam D_v v_v when v given)
__global__ void __launch_bounds__(256) k_gen_jt(GenSets S, GenInc inc, int V, const double* v, const double* Dg,
                                                double lam, double* out) {
  const int u = blockIdx.x * 256 + threadIdx.x;
  if (u >= V) return;
  double acc[kGD] = {0.0, 0.0};
  for (int t = inc.off[u]; t < inc.off[u + 1]; ++t) {
    const int q = inc.kind[t], e = inc.edge[t], a = inc.slot[t];
    const int A = S.A[q], M = S.M[q], N = A * kGD;
    for (int m = 0; m < M; ++m) {
      const double we = S.w[q][(size_t)M * e + m];
      for (int k = 0; k < kGD; ++k) acc[k] += S.s[q].J[((size_t)M * e + m) * N + a * kGD + k] * we;
    }
  }
  for (int k = 0; k < kGD; ++k) {
    double y = acc[k];
    if (v) y += lam * Dg[(size_t)kGD * u + k] * v[(size_t)kGD * u + k];
    out[(size_t)kGD * u + k] = y;
  }
}

// Per vertex: the undamped block H_v = sum J_slot^T J_slot (packed 2 x 2: h00 h01 h11),
// the damping diagonal D_v = clamp(diag H_v) and the preconditioner (H_v + lam D_v)^-1
// (zero for a fixed vertex).
__global__ void __launch_bounds__(256) k_gen_blocks(GenSets S, GenInc inc, int V, const unsigned char* fixed,
                                                    double lam, double dmin, double dmax, int identity_damping,
                                                    double* Dg, double* Minv) {
  const int u = blockIdx.x * 256 + threadIdx.x;
  if (u >= V) return;
  double h00 = 0.0, h01 = 0.0, h11 = 0.0;
  for (int t = inc.off[u]; t < inc.off[u + 1]; ++t) {
    const int q = inc.kind[t], e = inc.edge[t], a = inc.slot[t];
    const int A = S.A[q], M = S.M[q], N = A * kGD;
    for (int m = 0; m < M; ++m) {
      const double* row = S.s[q].J + ((size_t)M * e + m) * N + a * kGD;
      h00 += row[0] * row[0];
      h01 += row[0] * row[1];
      h11 += row[1] * row[1];
    }
  }
  const double d0 = identity_damping ? 1.0 : fmin(fmax(h00, dmin), dmax);
  const double d1 = identity_damping ? 1.0 : fmin(fmax(h11, dmin), dmax);
  Dg[2 * (size_t)u] = d0;
  Dg[2 * (size_t)u + 1] = d1;
  const double a = h00 + lam * d0, b = h01, c = h11 + lam * d1;
  const double det = a * c - b * b;
  double* Mi = Minv + 3 * (size_t)u;
  if (fixed[u] || !(det > 0.0)) {
    Mi[0] = Mi[1] = Mi[2] = 0.0;
  } else {
    Mi[0] = c / det;
    Mi[1] = -b / det;
    Mi[2] = a / det;
  }
}

// z = M r (per vertex 2 x 2)
__global__ void k_gen_precond(int V, const double* Minv, const double* r, double* z) {
  const int u = blockIdx.x * 256 + threadIdx.x;
  if (u >= V) return;
  const double* Mi = Minv + 3 * (size_t)u;
  const double r0 = r[2 * (size_t)u], r1 = r[2 * (size_t)u + 1];
  z[2 * (size_t)u] = Mi[0] * r0 + Mi[1] * r1;
  z[2 * (size_t)u + 1] = Mi[1] * r0 + Mi[2] * r1;
}

// Per-CTA partial sums of a . b over n entries (fixed order; the host adds them)
__global__ void __launch_bounds__(256) k_gen_dot(int n, const double* a, const double* b, double* part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += 256 * gridDim.x) acc += a[i] * b[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// y = a x + b y (axpby on n entries); out may alias y
__global__ void k_gen_axpby(int n, double a, const double* x, double b, const double* y, double* out) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// candidate state x' = x + dx (fixed vertices unchanged)
__global__ void k_gen_step(int V, const unsigned char* fixed, const double* x, const double* dx, double* xc) {
  const int u = blockIdx.x * 256 + threadIdx.x;
  if (u >= V) return;
  for (int k = 0; k < kGD; ++k) xc[kGD * (size_t)u + k] = x[kGD * (size_t)u + k] + (fixed[u] ? 0.0 : dx[kGD * (size_t)u + k]);
}

}  // namespace

// ---------------------------------------------------------------- host side

struct gpo_generic {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int64_t V = 0;
  std::vector<double> x;
  std::vector<unsigned char> fixed;
  struct Set {
    int A = 0, M = 0, MEAS = 0;
    std::vector<int> vid;
    std::vector<double> meas, delta;
    std::vector<unsigned char> active;
  } sets[2];
  std::vector<std::pair<int, int>> eid;   // edge id -> (kind, index in its set)
};

namespace {

template <class E>
void set_shape(gpo_generic::Set& s) {
  s.A = E::A;
  s.M = E::M;
  s.MEAS = E::MEAS;
}

// Device buffers of one optimisation.
struct GenDev {
  std::vector<void*> owned;
  cudaStream_t st;
  bool ok = true;
  template <class T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    owned.push_back(p);
    return static_cast<T*>(p);
  }
  template <class T>
  T* up(const std::vector<T>& h) {
    T* d = alloc<T>(h.size());
    if (d && !h.empty() && cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
      ok = false;
    return d;
  }
  ~GenDev() {
    for (void* p : owned) cudaFreeAsync(p, st);
  }
};

inline int blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + 255) / 256); }

template <class E>
void launch_eval(const GenSet& s, const double* x, const unsigned char* fx, int mode, double* part, cudaStream_t st) {
  if (s.n > 0) k_gen_eval<E><<<blocks(s.n), 256, 0, st>>>(s, x, fx, mode, part);
}
template <class E>
void launch_jv(const GenSet& s, const double* v, double* w, cudaStream_t st) {
  if (s.n > 0) k_gen_jv<E><<<blocks(s.n), 256, 0, st>>>(s, v, w);
}

// Host sum of device partials, in order.
double host_sum(const double* d, int n, cudaStream_t st, bool& ok) {
  std::vector<double> h(std::max(n, 1));
  if (cudaMemcpyAsync(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    ok = false;
    return 0.0;
  }
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += h[i];
  return s;
}

}  // namespace

extern "C" {

gpo_status gpo_generic_create(int32_t vertex_dim, int64_t n_vertices, const double* x0, int32_t device,
                              void* cuda_stream, gpo_generic** out) {
  if (!out || vertex_dim != kGD || n_vertices <= 0 || n_vertices > (int64_t)1 << 30 || !x0) return GPO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GPO_ERR_ARG;
  }
  gpo_generic* g = new (std::nothrow) gpo_generic();
  if (!g) return GPO_ERR_OOM;
  g->device = device;
  g->V = n_vertices;
  g->x.assign(x0, x0 + (size_t)kGD * n_vertices);
  g->fixed.assign((size_t)n_vertices, 0);
  set_shape<CircleEdge>(g->sets[GPO_GE_CIRCLE]);
  set_shape<DistanceEdge>(g->sets[GPO_GE_DISTANCE]);
  if (cuda_stream) {
    g->st = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaSetDevice(device);
    if (cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete g;
      return GPO_ERR_CUDA;
    }
    g->own_stream = true;
  }
  *out = g;
  return GPO_OK;
}

gpo_status gpo_generic_destroy(gpo_generic* g) {
  if (!g) return GPO_OK;
  if (g->own_stream) cudaStreamDestroy(g->st);
  delete g;
  return GPO_OK;
}

gpo_status gpo_generic_add_edges(gpo_generic* g, int32_t kind, int64_t n, const int64_t* vertex_ids,
                                 const double* meas, int32_t loss_kind, double loss_delta, int64_t* first_id) {
  if (!g || kind < GPO_GE_CIRCLE || kind > GPO_GE_DISTANCE || n < 0 || (n > 0 && (!vertex_ids || !meas)))
    return GPO_ERR_ARG;
  if (loss_kind != GPO_LOSS_NONE && loss_kind != GPO_LOSS_HUBER) return GPO_ERR_ARG;
  if (loss_kind == GPO_LOSS_HUBER && !(loss_delta > 0.0 && std::isfinite(loss_delta))) return GPO_ERR_ARG;
  gpo_generic::Set& s = g->sets[kind];
  for (int64_t i = 0; i < n * s.A; ++i)
    if (vertex_ids[i] < 0 || vertex_ids[i] >= g->V) return GPO_ERR_ARG;
  if (first_id) *first_id = (int64_t)g->eid.size();
  for (int64_t i = 0; i < n; ++i) {
    g->eid.emplace_back(kind, (int)(s.delta.size()));
    for (int a = 0; a < s.A; ++a) s.vid.push_back((int)vertex_ids[s.A * i + a]);
    for (int k = 0; k < s.MEAS; ++k) s.meas.push_back(meas[s.MEAS * i + k]);
    s.delta.push_back(loss_kind == GPO_LOSS_HUBER ? loss_delta : 0.0);
    s.active.push_back(1);
  }
  return GPO_OK;
}

gpo_status gpo_generic_set_fixed(gpo_generic* g, int64_t vid, int32_t fixed) {
  if (!g || vid < 0 || vid >= g->V) return GPO_ERR_ARG;
  g->fixed[vid] = fixed ? 1 : 0;
  return GPO_OK;
}

gpo_status gpo_generic_set_edge_active(gpo_generic* g, int64_t eid, int32_t active) {
  if (!g || eid < 0 || eid >= (int64_t)g->eid.size()) return GPO_ERR_ARG;
  g->sets[g->eid[eid].first].active[g->eid[eid].second] = active ? 1 : 0;
  return GPO_OK;
}

gpo_status gpo_generic_get_state(gpo_generic* g, double* out) {
  if (!g || !out) return GPO_ERR_ARG;
  std::memcpy(out, g->x.data(), g->x.size() * sizeof(double));
  return GPO_OK;
}

gpo_status gpo_generic_optimize(gpo_generic* g, int32_t max_iters, const gpo_lm_params* params, gpo_report* rep) {
  if (!g || max_iters < 0) return GPO_ERR_ARG;
  gpo_lm_params prm;
  gpo_lm_params_default(&prm);
  if (params) prm = *params;
  if (!(prm.initial_damping > 0.0)) return GPO_ERR_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return GPO_ERR_CUDA;
  const cudaStream_t st = g->st;
  const int V = (int)g->V, n2 = kGD * V;
  GenDev dv{{}, st};
  // incidence of every vertex, in (kind, edge, slot) order
  std::vector<int> cnt(V + 1, 0);
  for (int q = 0; q < 2; ++q)
    for (int v : g->sets[q].vid) cnt[v + 1]++;
  for (int u = 0; u < V; ++u) cnt[u + 1] += cnt[u];
  const int nnz = cnt[V];
  std::vector<int> ik(std::max(nnz, 1)), ie(std::max(nnz, 1)), is(std::max(nnz, 1)), fill(cnt.begin(), cnt.end() - 1);
  for (int q = 0; q < 2; ++q) {
    const auto& s = g->sets[q];
    const int n = (int)s.delta.size();
    for (int e = 0; e < n; ++e)
      for (int a = 0; a < s.A; ++a) {
        const int t = fill[s.vid[(size_t)s.A * e + a]]++;
        ik[t] = q;
        ie[t] = e;
        is[t] = a;
      }
  }
  GenSets S{};
  GenInc inc{dv.up(cnt), dv.up(ik), dv.up(ie), dv.up(is)};
  double* r_[2];
  double* w_[2];
  int nb = 0;   // cost partial blocks of both sets
  for (int q = 0; q < 2; ++q) {
    const auto& s = g->sets[q];
    const int n = (int)s.delta.size();
    S.A[q] = s.A;
    S.M[q] = s.M;
    S.s[q].n = n;
    S.s[q].vid = dv.up(s.vid);
    S.s[q].meas = dv.up(s.meas);
    S.s[q].delta = dv.up(s.delta);
    S.s[q].active = dv.up(s.active);
    S.s[q].r = r_[q] = dv.alloc<double>((size_t)s.M * n);
    S.s[q].J = dv.alloc<double>((size_t)s.M * s.A * kGD * n);
    w_[q] = dv.alloc<double>((size_t)s.M * n);
    nb += n > 0 ? blocks(n) : 0;
  }
  double* x = dv.up(g->x);
  unsigned char* fx = dv.up(g->fixed);
  double *xc = dv.alloc<double>(n2), *b = dv.alloc<double>(n2), *dx = dv.alloc<double>(n2), *rr = dv.alloc<double>(n2),
         *z = dv.alloc<double>(n2), *p = dv.alloc<double>(n2), *y = dv.alloc<double>(n2), *Dg = dv.alloc<double>(n2),
         *Minv = dv.alloc<double>(3 * (size_t)V);
  double* part = dv.alloc<double>(std::max(nb, 1024));
  if (!dv.ok) return GPO_ERR_OOM;
  bool ok = true;
  auto cost = [&](const double* xs, int mode) {   // mode 0 also linearises
    int off = 0;
    if (S.s[0].n > 0) {
      launch_eval<CircleEdge>(S.s[0], xs, fx, mode, part + off, st);
      off += blocks(S.s[0].n);
    }
    if (S.s[1].n > 0) {
      launch_eval<DistanceEdge>(S.s[1], xs, fx, mode, part + off, st);
      off += blocks(S.s[1].n);
    }
    return off ? host_sum(part, off, st, ok) : 0.0;
  };
  auto dot = [&](int n, const double* a, const double* c) {
    const int nbk = std::min(blocks(n), 1024);
    k_gen_dot<<<nbk, 256, 0, st>>>(n, a, c, part);
    return host_sum(part, nbk, st, ok);
  };
  auto jtw = [&](const double* const* src, const double* v, double lam, double* out) {
    GenSets T = S;
    T.w[0] = src[0];
    T.w[1] = src[1];
    k_gen_jt<<<blocks(V), 256, 0, st>>>(T, inc, V, v, Dg, lam, out);
  };
  auto jv = [&](const double* v) {
    launch_jv<CircleEdge>(S.s[0], v, w_[0], st);
    launch_jv<DistanceEdge>(S.s[1], v, w_[1], st);
  };
  double lam = prm.initial_damping, nu = (prm.initial_nu >= 2.0 && std::isfinite(prm.initial_nu)) ? prm.initial_nu : 2.0;
  double F = cost(x, 1);
  if (!ok) return GPO_ERR_CUDA;
  const double F0 = F;
  int accepted = 0, pcg_total = 0;
  for (int it = 0; it < max_iters; ++it) {
    cost(x, 0);                                       // rows and residuals at x
    const double* rs[2] = {r_[0], r_[1]};
    jtw(rs, nullptr, 0.0, b);                         // b = J^T r
    k_gen_blocks<<<blocks(V), 256, 0, st>>>(S, inc, V, fx, lam, prm.diag_min, prm.diag_max, prm.damping_mode == 1, Dg, Minv);
    // PCG on (J^T J + lam D) dx = -b
    k_gen_axpby<<<blocks(n2), 256, 0, st>>>(n2, -1.0, b, 0.0, b, rr);
    if (cudaMemsetAsync(dx, 0, n2 * sizeof(double), st) != cudaSuccess) return GPO_ERR_CUDA;
    k_gen_precond<<<blocks(V), 256, 0, st>>>(V, Minv, rr, z);
    k_gen_axpby<<<blocks(n2), 256, 0, st>>>(n2, 1.0, z, 0.0, z, p);
    double rz = dot(n2, rr, z);
    const double gn = std::sqrt(dot(n2, rr, rr));
    const double tol = prm.pcg_tol_relative ? prm.pcg_tol * gn : prm.pcg_tol;
    for (int k = 0; k < prm.pcg_max_iters && gn > 0.0 && rz > 0.0; ++k) {
      jv(p);
      const double* ws[2] = {w_[0], w_[1]};
      jtw(ws, p, lam, y);                             // y = (J^T J + lam D) p
      const double pAp = dot(n2, p, y);
      if (!(pAp > 0.0)) break;
      const double alpha = rz / pAp;
      k_gen_axpby<<<blocks(n2), 256, 0, st>>>(n2, alpha, p, 1.0, dx, dx);
      k_gen_axpby<<<blocks(n2), 256, 0, st>>>(n2, -alpha, y, 1.0, rr, rr);
      ++pcg_total;
      if (std::sqrt(dot(n2, rr, rr)) <= tol) break;
      k_gen_precond<<<blocks(V), 256, 0, st>>>(V, Minv, rr, z);
      const double rz2 = dot(n2, rr, z);
      k_gen_axpby<<<blocks(n2), 256, 0, st>>>(n2, 1.0, z, rz2 / rz, p, p);
      rz = rz2;
    }
    // model decrease -b^T dx - 1/2 |J dx|^2, candidate, gain ratio
    jv(dx);
    double jj = 0.0;
    for (int q = 0; q < 2; ++q)
      if (S.s[q].n > 0) jj += dot(S.M[q] * S.s[q].n, w_[q], w_[q]);
    const double L = -dot(n2, b, dx) - 0.5 * jj;
    k_gen_step<<<blocks(V), 256, 0, st>>>(V, fx, x, dx, xc);
    const double Fc = cost(xc, 1);
    if (!ok) return GPO_ERR_CUDA;
    const bool acc = L > 0.0 && std::isfinite(Fc) && Fc < F;
    const double rho = L != 0.0 ? (F - Fc) / L : 0.0;
    if (acc) {
      std::swap(x, xc);
      F = Fc;
      ++accepted;
      lam *= std::max(1.0 / 3.0, 1.0 - std::pow(2.0 * rho - 1.0, 3));
      nu = 2.0;
    } else {
      lam *= nu;
      nu *= 2.0;
    }
    lam = std::min(std::max(lam, prm.lambda_min), prm.lambda_max);
  }
  if (cudaMemcpyAsync(g->x.data(), x, g->x.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return GPO_ERR_CUDA;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->initial_cost = F0;
    rep->final_cost = F;
    rep->iterations = max_iters;
    rep->accepted = accepted;
    rep->final_lambda = lam;
    rep->pcg_iters_total = pcg_total;
    rep->final_nu = nu;
  }
  return GPO_OK;
}

}  // extern "C"
