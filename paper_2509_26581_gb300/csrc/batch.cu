// Batched solves and the serving loop: many independent graphs share every kernel
// launch.  A launch set over the graphs lists their descriptors and which CTA belongs
// to which graph (chunks, camera blocks, point blocks); each graph keeps its own LM
// and PCG state, so a graph's result does not depend on the other graphs it runs with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "graph.h"

using namespace gpo_host;

namespace {

__global__ void k_put_scalars(const DevBA* probs, const Scalars* src, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) *probs[q].sc = src[q];
}

__global__ void k_get_scalars(const DevBA* probs, Scalars* dst, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dst[q] = *probs[q].sc;
}

// Device tables of a launch set over several finalized graphs (stream-ordered memory).
struct BatchSet {
  gpo::LaunchSet ls{};
  char* mem = nullptr;
  Scalars* staging = nullptr;    // device [n]
  int n = 0;

  void release(cudaStream_t st) {
    if (mem) cudaFreeAsync(mem, st);
    mem = nullptr;
    n = 0;
  }
};

gpo_status build_set(gpo_graph* owner, const std::vector<gpo_graph*>& gs, BatchSet& out) {
  const int n = (int)gs.size();
  std::vector<DevBA> probs(n);
  std::vector<int> ch_prob, cb_prob, pb_prob, ch_base(n), cb_base(n), pb_base(n);
  int ch_max = 32, ns_max = 1, np_max = 1;
  for (int q = 0; q < n; ++q) {
    const gpo_graph* g = gs[q];
    probs[q] = g->dev;
    ch_base[q] = (int)ch_prob.size();
    cb_base[q] = (int)cb_prob.size();
    pb_base[q] = (int)pb_prob.size();
    ch_prob.insert(ch_prob.end(), g->ls.n_ch, q);
    cb_prob.insert(cb_prob.end(), g->ls.n_cb, q);
    pb_prob.insert(pb_prob.end(), g->ls.n_pb, q);
    ch_max = std::max(ch_max, g->ls.ch_max);
    ns_max = std::max(ns_max, g->ls.ns_max);
    np_max = std::max(np_max, g->ls.np_max);
  }
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_probs = al(n * sizeof(DevBA)), b_stage = al(n * sizeof(Scalars));
  const size_t b_ch = al(std::max<size_t>(1, ch_prob.size()) * 4), b_cb = al(std::max<size_t>(1, cb_prob.size()) * 4);
  const size_t b_pb = al(std::max<size_t>(1, pb_prob.size()) * 4), b_base = al(n * 4);
  const size_t total = b_probs + b_stage + b_ch + b_cb + b_pb + 3 * b_base + 256;
  cudaStream_t st = owner->stream;
  char* mem = nullptr;
  GPO_CUDA(owner, cudaMallocAsync(reinterpret_cast<void**>(&mem), total, st));
  char* p = mem;
  auto take = [&](size_t b) { char* r = p; p += b; return r; };
  DevBA* probs_d = reinterpret_cast<DevBA*>(take(b_probs));
  Scalars* stage_d = reinterpret_cast<Scalars*>(take(b_stage));
  int* ch_d = reinterpret_cast<int*>(take(b_ch));
  int* cb_d = reinterpret_cast<int*>(take(b_cb));
  int* pb_d = reinterpret_cast<int*>(take(b_pb));
  int* chb_d = reinterpret_cast<int*>(take(b_base));
  int* cbb_d = reinterpret_cast<int*>(take(b_base));
  int* pbb_d = reinterpret_cast<int*>(take(b_base));
  int* running_d = reinterpret_cast<int*>(take(256));
  GPO_CUDA(owner, cudaMemcpyAsync(probs_d, probs.data(), n * sizeof(DevBA), cudaMemcpyHostToDevice, st));
  if (!ch_prob.empty()) GPO_CUDA(owner, cudaMemcpyAsync(ch_d, ch_prob.data(), ch_prob.size() * 4, cudaMemcpyHostToDevice, st));
  if (!cb_prob.empty()) GPO_CUDA(owner, cudaMemcpyAsync(cb_d, cb_prob.data(), cb_prob.size() * 4, cudaMemcpyHostToDevice, st));
  if (!pb_prob.empty()) GPO_CUDA(owner, cudaMemcpyAsync(pb_d, pb_prob.data(), pb_prob.size() * 4, cudaMemcpyHostToDevice, st));
  GPO_CUDA(owner, cudaMemcpyAsync(chb_d, ch_base.data(), n * 4, cudaMemcpyHostToDevice, st));
  GPO_CUDA(owner, cudaMemcpyAsync(cbb_d, cb_base.data(), n * 4, cudaMemcpyHostToDevice, st));
  GPO_CUDA(owner, cudaMemcpyAsync(pbb_d, pb_base.data(), n * 4, cudaMemcpyHostToDevice, st));
  GPO_CUDA(owner, cudaMemsetAsync(running_d, 0, 32, st));
  // the host vectors go out of scope: wait for the copies
  GPO_CUDA(owner, cudaStreamSynchronize(st));
  gpo::LaunchSet ls{};
  ls.probs = probs_d;
  ls.ch_prob = ch_d; ls.ch_base = chb_d;
  ls.cb_prob = cb_d; ls.cb_base = cbb_d;
  ls.pb_prob = pb_d; ls.pb_base = pbb_d;
  ls.running = running_d;
  ls.err = running_d + 1;
  ls.work = running_d + 2;
  ls.spmv_variant = owner->desc.spmv_variant;
  ls.nprob = n;
  ls.n_ch = (int)ch_prob.size();
  ls.n_cb = (int)cb_prob.size();
  ls.n_pb = (int)pb_prob.size();
  ls.ch_max = ch_max;
  ls.ns_max = ns_max;
  ls.np_max = np_max;
  out.ls = ls;
  out.mem = mem;
  out.staging = stage_d;
  out.n = n;
  return GPO_OK;
}

gpo_status put_scalars(gpo_graph* owner, BatchSet& bs, const std::vector<Scalars>& sc) {
  GPO_CUDA(owner, cudaMemcpyAsync(bs.staging, sc.data(), sc.size() * sizeof(Scalars),
                                  cudaMemcpyHostToDevice, owner->stream));
  k_put_scalars<<<(bs.n + 127) / 128, 128, 0, owner->stream>>>(bs.ls.probs, bs.staging, bs.n);
  GPO_CUDA(owner, cudaGetLastError());
  GPO_CUDA(owner, cudaStreamSynchronize(owner->stream));
  return GPO_OK;
}

gpo_status get_scalars(gpo_graph* owner, BatchSet& bs, std::vector<Scalars>& sc) {
  sc.resize(bs.n);
  k_get_scalars<<<(bs.n + 127) / 128, 128, 0, owner->stream>>>(bs.ls.probs, bs.staging, bs.n);
  GPO_CUDA(owner, cudaGetLastError());
  GPO_CUDA(owner, cudaMemcpyAsync(sc.data(), bs.staging, bs.n * sizeof(Scalars), cudaMemcpyDeviceToHost,
                                  owner->stream));
  GPO_CUDA(owner, cudaStreamSynchronize(owner->stream));
  return GPO_OK;
}

void report_from(const Scalars& s, double initial_cost, gpo_report* r) {
  r->initial_cost = initial_cost;
  r->final_cost = s.cost;
  r->final_lambda = s.lambda;
  r->iterations = s.iter;
  r->accepted = s.n_accepted;
  r->pcg_iters_total = s.pcg_total;
  r->reserved0 = 0;
  r->final_nu = s.nu;
}

// Device-memory pool of a server: arenas of retired graphs are kept (keyed by size,
// 1 MiB granularity) and handed to the next admitted graphs, so the serving loop does
// not pay cudaMalloc / cudaFree (which synchronises the device) per request.
struct DevPool {
  std::multimap<size_t, void*> free_blocks;
  std::unordered_map<void*, size_t> block_size;
  size_t held = 0;   // bytes obtained from cudaMalloc and not yet returned

  void trim() {
    for (auto& kv : free_blocks) {
      cudaFree(kv.second);
      held -= kv.first;
      block_size.erase(kv.second);
    }
    free_blocks.clear();
  }
};

void* pool_alloc(size_t bytes, void* ctx) {
  DevPool* pool = static_cast<DevPool*>(ctx);
  const size_t b = (bytes + (size_t(1) << 20) - 1) & ~((size_t(1) << 20) - 1);
  auto it = pool->free_blocks.lower_bound(b);
  if (it != pool->free_blocks.end() && it->first <= 2 * b) {   // reuse a block at most twice as big
    void* p = it->second;
    pool->free_blocks.erase(it);
    return p;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, b) != cudaSuccess) {
    cudaGetLastError();
    pool->trim();
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  pool->block_size[p] = b;
  pool->held += b;
  return p;
}

void pool_free(void* p, void* ctx) {
  DevPool* pool = static_cast<DevPool*>(ctx);
  auto it = pool->block_size.find(p);
  if (it != pool->block_size.end()) pool->free_blocks.emplace(it->second, p);
}

}  // namespace

// ============================================================== serving loop state

struct gpo_server {
  gpo_server_desc desc{};
  gpo_graph* owner = nullptr;     // empty graph carrying the stream, flags and profiler
  struct Req {
    gpo_graph* g;
    int max_iters;
    gpo_lm_params prm;
    int64_t ticket;
    int done_iters;
    size_t bytes;
    double initial_cost;
    gpo_graph_desc saved;   // the graph's own stream and allocator, restored at retirement
    bool adopted_stream;
  };
  DevPool pool;
  std::deque<Req> queue;
  std::vector<Req> resident;
  std::unordered_map<int64_t, gpo_report> finished;
  size_t used = 0;
  int64_t next_ticket = 0;
  BatchSet set;
  bool dirty = true;
  int64_t steps = 0;
};

extern "C" {

gpo_status gpo_optimize_batch(gpo_graph* const* graphs, int32_t n, int32_t max_iters,
                              const gpo_lm_params* params, gpo_report* reports) {
  if (!graphs || n <= 0 || max_iters < 0) return GPO_ERR_ARG;
  gpo_graph* owner = graphs[0];
  if (!owner) return GPO_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!graphs[i]) return fail(owner, GPO_ERR_ARG, "graph %d is null", i);
    if (graphs[i]->prec != owner->prec || graphs[i]->desc.device != owner->desc.device)
      return fail(owner, GPO_ERR_ARG, "graphs of a batch must share precision and device");
    if (graphs[i]->desc.spmv_variant == 4)
      return fail(owner, GPO_ERR_UNSUPPORTED, "graphs with dynamic Jacobians are solved alone");
    for (int j = 0; j < i; ++j)
      if (graphs[j] == graphs[i]) return fail(owner, GPO_ERR_ARG, "graph %d appears twice", i);
  }
  GPO_CUDA(owner, cudaSetDevice(owner->desc.device));
  for (int i = 0; i < n; ++i) {
    gpo_status s = finalize(graphs[i]);
    if (s != GPO_OK) {
      if (graphs[i] != owner) owner->err = graphs[i]->err;
      return s;
    }
    if (graphs[i]->ks != owner->ks)
      return fail(owner, GPO_ERR_ARG, "graphs of a batch must share the camera kind");
  }
  const gpo_lm_params prm = params_or_default(params);
  if (!(prm.initial_damping > 0.0)) return fail(owner, GPO_ERR_ARG, "initial damping must be positive");
  std::vector<gpo_graph*> gs(graphs, graphs + n);
  BatchSet bs;
  gpo_status s = build_set(owner, gs, bs);
  if (s != GPO_OK) return s;
  std::vector<Scalars> sc(n);
  for (int i = 0; i < n; ++i) {
    fill_scalars(graphs[i], prm, prm.initial_damping, sc[i]);
    sc[i].full = 0;   // shared launches run the Schur form
    graphs[i]->pcg_full = 0;
  }
  int max_it = 1;
  for (auto& x : sc) max_it = std::max(max_it, x.max_it);
  if ((s = put_scalars(owner, bs, sc)) == GPO_OK && (s = launch_initial_cost(owner, bs.ls)) == GPO_OK &&
      (s = get_scalars(owner, bs, sc)) == GPO_OK) {
    std::vector<double> F0(n);
    for (int i = 0; i < n; ++i) {
      F0[i] = sc[i].cost;
      if (!std::isfinite(F0[i])) {
        s = fail(owner, GPO_ERR_NUMERIC, "graph %d: initial cost is not finite (%g)", i, F0[i]);
        break;
      }
    }
    for (int it = 0; s == GPO_OK && it < max_iters; ++it) {
      owner->cur_lm_iter = -1;
      if ((s = solve_system(owner, bs.ls, max_it, false)) != GPO_OK) break;
      s = finish_iteration(owner, bs.ls);
    }
    if (s == GPO_OK && (s = get_scalars(owner, bs, sc)) == GPO_OK) {
      for (int i = 0; i < n; ++i) {
        graphs[i]->last_cost = sc[i].cost;
        graphs[i]->cost_valid = true;
        graphs[i]->state_same = false;   // a batched run: the next single run starts afresh
        graphs[i]->hist.clear();
        if (reports) report_from(sc[i], F0[i], &reports[i]);
      }
    }
  }
  if (owner->prof.on) {
    cudaStreamSynchronize(owner->stream);
    prof_resolve(owner);
  }
  bs.release(owner->stream);
  cudaStreamSynchronize(owner->stream);
  return s;
}

gpo_status gpo_server_desc_default(gpo_server_desc* out) {
  if (!out) return GPO_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->precision = GPO_FP32_BF16;
  out->max_resident = 1024;
  return GPO_OK;
}

gpo_status gpo_server_create(const gpo_server_desc* desc, gpo_server** out) {
  if (!desc || !out) return GPO_ERR_ARG;
  if (desc->max_resident <= 0) return GPO_ERR_ARG;
  gpo_graph_desc gd;
  gpo_graph_desc_default(&gd);
  gd.precision = desc->precision;
  gd.device = desc->device;
  gd.cuda_stream = desc->cuda_stream;
  gpo_graph* owner = nullptr;
  gpo_status s = gpo_graph_create(&gd, &owner);
  if (s != GPO_OK) return s;
  if ((s = ensure_runtime(owner)) != GPO_OK) {
    gpo_graph_destroy(owner);
    return s;
  }
  gpo_server* sv = new (std::nothrow) gpo_server();
  if (!sv) {
    gpo_graph_destroy(owner);
    return GPO_ERR_OOM;
  }
  sv->desc = *desc;
  sv->owner = owner;
  *out = sv;
  return GPO_OK;
}

// Gives a graph back its own stream and allocator after the server is done with it.
static void restore_graph(gpo_server::Req& r) {
  r.g->desc.alloc = r.saved.alloc;
  r.g->desc.free = r.saved.free;
  r.g->desc.alloc_ctx = r.saved.alloc_ctx;
  if (r.adopted_stream) r.g->stream = nullptr;
}

gpo_status gpo_server_destroy(gpo_server* sv) {
  if (!sv) return GPO_OK;
  cudaStreamSynchronize(sv->owner->stream);
  for (auto& r : sv->resident) {
    release_device(r.g);
    restore_graph(r);
  }
  for (auto& r : sv->queue) restore_graph(r);
  sv->set.release(sv->owner->stream);
  cudaStreamSynchronize(sv->owner->stream);
  sv->pool.trim();
  gpo_graph_destroy(sv->owner);
  delete sv;
  return GPO_OK;
}

gpo_status gpo_server_submit(gpo_server* sv, gpo_graph* g, int32_t max_iters, const gpo_lm_params* params,
                             int64_t* ticket) {
  if (!sv || !g || max_iters < 0) return GPO_ERR_ARG;
  if (g->prec != sv->owner->prec || g->desc.device != sv->owner->desc.device)
    return fail(sv->owner, GPO_ERR_ARG, "graph precision or device differs from the server's");
  if (g->desc.spmv_variant == 4)
    return fail(sv->owner, GPO_ERR_UNSUPPORTED, "graphs with dynamic Jacobians are solved alone");
  if (g->finalized) return fail(sv->owner, GPO_ERR_STATE, "graph is already resident on the device");
  const gpo::KernelSet* k = &kernels_of(g);
  if (sv->owner->ks && sv->owner->ks != k)
    return fail(sv->owner, GPO_ERR_ARG, "graph camera kind differs from the server's earlier graphs");
  size_t bytes = 0;
  gpo_status s = finalize(g, &bytes);
  if (s != GPO_OK) {
    sv->owner->err = g->err;
    return s;
  }
  if (sv->desc.memory_budget && bytes > sv->desc.memory_budget)
    return fail(sv->owner, GPO_ERR_OOM, "graph needs %zu bytes, more than the server budget %zu", bytes,
                (size_t)sv->desc.memory_budget);
  sv->owner->ks = k;
  gpo_server::Req r{g, max_iters, params_or_default(params), sv->next_ticket++, 0, bytes, 0.0, g->desc, false};
  // a graph without a stream of its own runs on the server's; a graph without an
  // allocator hook takes its arena from the server's pool
  if (!g->stream) {
    g->stream = sv->owner->stream;
    r.adopted_stream = true;
  }
  if (!g->desc.alloc) {
    g->desc.alloc = pool_alloc;
    g->desc.free = pool_free;
    g->desc.alloc_ctx = &sv->pool;
  }
  sv->queue.push_back(r);
  if (ticket) *ticket = r.ticket;
  return GPO_OK;
}

gpo_status gpo_server_step(gpo_server* sv, int32_t* n_resident, int32_t* n_queued, int32_t* n_finished) {
  if (!sv) return GPO_ERR_ARG;
  gpo_graph* owner = sv->owner;
  GPO_CUDA(owner, cudaSetDevice(owner->desc.device));
  int fin = 0;
  // 1. admission: first come, first served, while slots and memory allow; the new
  //    graphs' initial costs are computed together in shared launches
  std::vector<gpo_server::Req> adm;
  while (!sv->queue.empty() && (int)(sv->resident.size() + adm.size()) < sv->desc.max_resident) {
    gpo_server::Req r = sv->queue.front();
    if (sv->desc.memory_budget && sv->used + r.bytes > sv->desc.memory_budget) break;
    gpo_status s = finalize(r.g);
    if (s != GPO_OK) {
      owner->err = r.g->err;
      return s;
    }
    sv->used += r.g->arena_bytes;
    sv->queue.pop_front();
    adm.push_back(r);
  }
  std::vector<gpo_server::Req> retire;   // graphs leaving the device this step
  if (!adm.empty()) {
    std::vector<gpo_graph*> gs;
    for (auto& r : adm) gs.push_back(r.g);
    BatchSet bs;
    gpo_status s = build_set(owner, gs, bs);
    if (s != GPO_OK) return s;
    std::vector<Scalars> sc(adm.size());
    for (size_t i = 0; i < adm.size(); ++i) {
      fill_scalars(adm[i].g, adm[i].prm, adm[i].prm.initial_damping, sc[i]);
      sc[i].full = 0;   // shared launches run the Schur form
      adm[i].g->pcg_full = 0;
    }
    if ((s = put_scalars(owner, bs, sc)) == GPO_OK && (s = launch_initial_cost(owner, bs.ls)) == GPO_OK)
      s = get_scalars(owner, bs, sc);
    bs.release(owner->stream);
    if (s != GPO_OK) return s;
    for (size_t i = 0; i < adm.size(); ++i) {
      adm[i].initial_cost = sc[i].cost;
      if (adm[i].max_iters == 0 || !std::isfinite(adm[i].initial_cost)) {
        gpo_report rep;
        report_from(sc[i], adm[i].initial_cost, &rep);
        sv->finished[adm[i].ticket] = rep;
        retire.push_back(adm[i]);
      } else {
        sv->resident.push_back(adm[i]);
        sv->dirty = true;
      }
    }
  }
  if (!sv->resident.empty()) {
    // 2. one LM iteration for every resident graph, in shared launches
    if (sv->dirty) {
      sv->set.release(owner->stream);
      std::vector<gpo_graph*> gs;
      for (auto& r : sv->resident) gs.push_back(r.g);
      gpo_status s = build_set(owner, gs, sv->set);
      if (s != GPO_OK) return s;
      sv->dirty = false;
    }
    int max_it = 1;
    for (auto& r : sv->resident) max_it = std::max(max_it, r.prm.pcg_max_iters);
    owner->cur_lm_iter = -1;
    gpo_status s = solve_system(owner, sv->set.ls, max_it, false);
    if (s == GPO_OK) s = finish_iteration(owner, sv->set.ls);
    if (s != GPO_OK) return s;
    ++sv->steps;
    // 3. retirement of graphs that ran all their iterations
    bool any = false;
    for (auto& r : sv->resident) any |= (++r.done_iters >= r.max_iters);
    if (any) {
      std::vector<Scalars> sc;
      if ((s = get_scalars(owner, sv->set, sc)) != GPO_OK) return s;
      std::vector<gpo_server::Req> keep;
      for (size_t i = 0; i < sv->resident.size(); ++i) {
        gpo_server::Req& r = sv->resident[i];
        if (r.done_iters < r.max_iters) {
          keep.push_back(r);
          continue;
        }
        gpo_report rep;
        report_from(sc[i], r.initial_cost, &rep);
        sv->finished[r.ticket] = rep;
        r.g->last_cost = sc[i].cost;
        r.g->cost_valid = true;
        r.g->state_same = false;   // a served run: the next single run starts afresh
        retire.push_back(r);
      }
      sv->resident.swap(keep);
      sv->dirty = true;
    }
  }
  if (!retire.empty()) {
    // final states back to the graphs' host arrays: all copies, then one wait
    std::vector<std::vector<double>> pts(retire.size());
    for (size_t i = 0; i < retire.size(); ++i) {
      gpo_status s = download_begin(retire[i].g, pts[i]);
      if (s != GPO_OK) return s;
    }
    GPO_CUDA(owner, cudaStreamSynchronize(owner->stream));
    for (size_t i = 0; i < retire.size(); ++i) {
      gpo_server::Req& r = retire[i];
      if (r.g->stream != owner->stream) GPO_CUDA(owner, cudaStreamSynchronize(r.g->stream));
      download_end(r.g, pts[i]);
      sv->used -= r.g->arena_bytes;
      release_device(r.g);
      restore_graph(r);
      ++fin;
    }
  }
  if (n_resident) *n_resident = (int32_t)sv->resident.size();
  if (n_queued) *n_queued = (int32_t)sv->queue.size();
  if (n_finished) *n_finished = fin;
  return GPO_OK;
}

gpo_status gpo_server_poll(gpo_server* sv, int64_t ticket, int32_t* done, gpo_report* report) {
  if (!sv || !done) return GPO_ERR_ARG;
  auto it = sv->finished.find(ticket);
  if (it == sv->finished.end()) {
    *done = 0;
    return GPO_OK;
  }
  *done = 1;
  if (report) *report = it->second;
  sv->finished.erase(it);
  return GPO_OK;
}

gpo_status gpo_server_memory(gpo_server* sv, size_t* used_bytes) {
  if (!sv || !used_bytes) return GPO_ERR_ARG;
  *used_bytes = sv->used;
  return GPO_OK;
}

const char* gpo_server_last_error(const gpo_server* sv) { return sv ? sv->owner->err.c_str() : ""; }

}  // extern "C"
