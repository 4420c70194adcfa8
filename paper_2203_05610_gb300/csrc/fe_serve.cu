// fe_serve.cu -- continuous-batching request loop (include/fe_serve.h).
//
// A scheduler thread admits queued requests first-fit in arrival order when
// a slot is free and the request's estimated device footprint fits the
// remaining HBM budget; each admitted request runs in its own worker thread
// on its own non-blocking CUDA stream with its own resident mesh, pattern,
// tangent, Krylov and BFGS workspace, so admitted requests overlap on the
// device.  A finished request frees its memory and its slot at once, and the
// scheduler admits the next queued requests that now fit.
//
// Small requests that the batched solver supports (fe_batch.h) are handed
// by their worker, once the mesh is built, to batcher threads: a batcher
// takes every waiting request of one size class (order, precision,
// floor(log2 ndof)) and solves them in one launch, one CTA each; requests
// that arrive meanwhile wait for the next
// launch (continuous batching at launch granularity); there is one batcher
// per slot, so a lone request is not held back.  The launch shape (threads
// per CTA) comes from a small autotuner per size class.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fe_batch.h"
#include "../../include/fe_serve.h"
#include "fe_internal.h"

namespace {

struct Request {
  int64_t id = 0;
  fe_mesh_desc desc{};
  std::vector<double> coords, face_data, fibers, d0;
  std::vector<int32_t> tets, faces, face_kind;
  std::vector<uint8_t> dir_group;
  std::vector<fe_dirichlet_group> groups;
  int method = 0;
  double tol = 1e-8;
  int max_it = 50;
  nl_opts opts{};
  bool has_opts = false;
  double load = 0.0, time = 0.0;
  fe_request_status st{};
  std::vector<double> result;
  std::string error;
  std::string mesh_key;            // the description's bytes (cache identity)
  size_t key_hash = 0;
  struct CachedMesh* cm = nullptr;  // the resident mesh it runs on, if any
  std::vector<struct CachedMesh*> victims;  // idle meshes evicted to admit it
  int64_t charge = 0;              // budget bytes it holds itself while running
};

// A mesh kept on the device between requests with the same description:
// its pattern, colouring, AMG structure and workspace stay resident, and
// the next request skips building them.  One request uses it at a time.
struct CachedMesh {
  std::string key;
  size_t key_hash = 0;
  fe_mesh m = nullptr;
  cudaStream_t stream = nullptr;
  int64_t bytes = 0;  // the admission charge it holds while resident
  bool busy = false;
  uint64_t last_used = 0;
};

// exact identity of a mesh description (geometry, topology, boundary data,
// material, fibres); fe_material has no padding
std::string mesh_key(const Request& r) {
  const fe_mesh_desc& d = r.desc;
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append(reinterpret_cast<const char*>(p), n); };
  const int32_t hdr[6] = {d.order, d.pressure_order, d.nv, d.ne, d.ngroups, d.nf};
  put(hdr, sizeof(hdr));
  put(&d.material, sizeof(d.material));
  put(r.coords.data(), r.coords.size() * sizeof(double));
  put(r.tets.data(), r.tets.size() * sizeof(int32_t));
  put(r.dir_group.data(), r.dir_group.size());
  for (const fe_dirichlet_group& g : r.groups) {  // field by field: the struct has padding
    put(&g.comp_mask, sizeof(g.comp_mask));
    put(g.center, sizeof(g.center));
    put(&g.angle, sizeof(g.angle));
    put(g.translation, sizeof(g.translation));
  }
  put(r.faces.data(), r.faces.size() * sizeof(int32_t));
  put(r.face_kind.data(), r.face_kind.size() * sizeof(int32_t));
  put(r.face_data.data(), r.face_data.size() * sizeof(double));
  put(r.fibers.data(), r.fibers.size() * sizeof(double));
  return k;
}

// device bytes a request will hold, estimated from its description before
// anything is allocated (exact node count; block count from the measured
// blocks per node of tetrahedral meshes, 28 for P2 and 16 for P1, with
// margin)
int64_t estimate_footprint(const Request& r, int64_t* ndof_out) {
  const fe_mesh_desc& d = r.desc;
  int64_t nv = d.nv, ne = d.ne, nn = nv;
  if (d.order == 2) {
    std::vector<uint64_t> keys((size_t)ne * 6);
    static const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int64_t e = 0; e < ne; e++)
      for (int k = 0; k < 6; k++) {
        uint64_t a = (uint64_t)d.tets[4 * e + E[k][0]], b = (uint64_t)d.tets[4 * e + E[k][1]];
        keys[(size_t)e * 6 + k] = (std::min(a, b) << 32) | std::max(a, b);
      }
    std::sort(keys.begin(), keys.end());
    nn += (int64_t)(std::unique(keys.begin(), keys.end()) - keys.begin());
  }
  const int64_t nen = d.order == 1 ? 4 : 10;
  const int64_t ndof = 3 * nn + (d.pressure_order == 1 ? nv : (d.pressure_order == 2 ? ne : 0));
  const int64_t nnzb = (d.order == 1 ? 16 : 28) * nn;
  nl_opts o = r.opts;
  if (!r.has_opts) nl_opts_default((nl_method)r.method, &o);
  const int64_t restart = o.ksp_restart > 0 ? o.ksp_restart : 500;
  const int64_t mpairs = (r.method >= NL_B) ? (o.lbfgs_m > 0 ? o.lbfgs_m : 50) : 0;
  const int64_t sval = o.precision == FE_PREC_FP64 ? 8 : 4;
  int64_t b = 0;
  b += 24 * nn + ne * (4 * nen + 8 + 80 + 4 * nen * nen + 24 * nen + 8 * nen) + 4 * nnzb + 16 * nn;  // mesh
  if (d.fibers) b += 72 * ne;
  if (d.pressure_order) b += ne * (4 * nen * 4 + 32) + 16 * 12 * nn;  // coupling pattern and values
  b += 9 * sval * nnzb + 9 * sval * nn + (o.precision == FE_PREC_MIXED_BF16 ? 18 * nnzb : 0);  // tangent
  b += 8 * ndof * (restart + 1) + 8 * (restart + 1) * (restart + 1);                             // Krylov basis
  b += 8 * ndof * (2 * mpairs + 12);                                                              // BFGS pairs, vectors
  if (o.pc_type >= 1) b += (d.order == 1 ? 2500 : 6000) * nn;  // AMG: P, A P, P^T in FP64 and coarse levels
  *ndof_out = ndof;
  return b + b / 8 + (64 << 20);
}

// a request waiting for (or in) a batched launch
struct BatchItem {
  Request* r = nullptr;
  fe_mesh m = nullptr;
  double* d = nullptr;
  int64_t ndof = 0;
  bool done = false;
  int rc = FE_OK;
  std::string error;
  fe_batch_out out{};
};

struct TuneEntry {
  int batches[2] = {0, 0};
  double cost[2] = {0.0, 0.0};  // best seconds per unit of work, 128 / 256 threads
  int chosen = 0;
};

// size class of the autotuner: (order, precision, floor(log2 ndof))
int64_t tune_key(int order, int prec, int64_t ndof) {
  int cls = 0;
  while ((int64_t(2) << cls) <= ndof) cls++;
  return ((int64_t)order << 40) | ((int64_t)prec << 32) | cls;
}

}  // namespace

struct fe_server_s {
  int device = 0;
  int64_t budget = 0, used = 0;
  int max_active = 8, active = 0;
  bool stop = false;
  int64_t next_id = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::thread scheduler;
  std::map<int64_t, std::thread> workers;  // running requests' threads, by request id
  std::vector<int64_t> finished;           // workers that have returned, to be joined
  // batched path
  bool cache_on = true;
  int64_t batch_max_dofs = 1000;
  std::deque<BatchItem*> bq;               // requests waiting for a batched launch
  std::condition_variable bcv;             // batchers wait here; items are signalled on cv
  std::vector<std::thread> batchers;
  std::map<int64_t, TuneEntry> tune;
  bool stop_batch = false;
  std::vector<std::unique_ptr<CachedMesh>> cache;  // resident meshes
  uint64_t tick = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

static void release_mesh(CachedMesh* c) {
  if (c->m) fe_mesh_destroy(c->m);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

static void run_request(fe_server s, Request* r) {
  int rc = FE_OK;
  double* d = nullptr;
  nl_stats stats{};
  std::vector<double> out;
  cudaSetDevice(s->device);
  // idle resident meshes the scheduler evicted to make room for this one
  for (CachedMesh* v : r->victims) release_mesh(v);
  r->victims.clear();
  // the resident mesh of the same description, or a new one
  const bool reused = r->cm != nullptr;
  CachedMesh* c = reused ? r->cm : new CachedMesh();
  if (!reused) {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = FE_ERR_CUDA;
      fe_set_error("cudaStreamCreate failed");
    }
    fe_mesh_desc desc = r->desc;
    desc.device = s->device;
    desc.stream = c->stream;
    if (rc == FE_OK) rc = fe_mesh_create(&desc, &c->m);
  }
  cudaStream_t stream = c->stream;
  fe_mesh m = c->m;
  if (rc == FE_OK) rc = fe_set_load(m, r->load, r->time);
  int64_t ndof = 0;
  if (rc == FE_OK) {
    fe_mesh_info info;
    fe_mesh_get_info(m, &info);
    ndof = info.ndof;
    if (!r->d0.empty() && (int64_t)r->d0.size() != ndof) {
      rc = FE_ERR_ARG;
      fe_set_error("initial guess has %zu entries, mesh has %lld unknowns", r->d0.size(), (long long)ndof);
    }
  }
  if (rc == FE_OK && cudaMallocAsync((void**)&d, ndof * sizeof(double), stream) != cudaSuccess) {
    rc = FE_ERR_OOM;
    fe_set_error("cudaMalloc of the solution vector failed");
  }
  if (rc == FE_OK) {
    if (r->d0.empty()) cudaMemsetAsync(d, 0, ndof * sizeof(double), stream);
    else cudaMemcpyAsync(d, r->d0.data(), ndof * sizeof(double), cudaMemcpyHostToDevice, stream);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->st.t_start = s->now();
      r->st.ndof = ndof;
    }
    const bool batched = r->has_opts && s->batch_max_dofs > 0 && ndof <= s->batch_max_dofs &&
                         fe_batch_supported(m, r->method, &r->opts);
    if (batched) {
      BatchItem item;
      item.r = r;
      item.m = m;
      item.d = d;
      item.ndof = ndof;
      if (cudaStreamSynchronize(stream) != cudaSuccess) {  // the initial guess is in place
        rc = FE_ERR_CUDA;
        fe_set_error("initial guess copy failed");
      } else {
        std::unique_lock<std::mutex> lk(s->mu);
        s->bq.push_back(&item);
        s->bcv.notify_one();
        s->cv.wait(lk, [&] { return item.done; });
        rc = item.rc;
        if (rc < 0) fe_set_error("%s", item.error.c_str());
      }
      if (rc >= 0) {  // the batched solver's record in nl_solve's form
        const fe_batch_out& o = item.out;
        stats.status = o.status;
        stats.nit = o.nit;
        stats.lit_total = o.lit_total;
        stats.assemblies = o.assemblies;
        stats.r0 = o.r0;
        stats.rfinal = o.rfinal;
        stats.hist_len = std::min(o.hist_len, (int32_t)FE_BATCH_HIST);
        for (int k = 0; k < stats.hist_len; k++) {
          stats.res_hist[k] = o.res_hist[k];
          stats.lit_hist[k] = o.lit_hist[k];
          stats.eta_hist[k] = o.eta_hist[k];
        }
        {
          std::lock_guard<std::mutex> lk(s->mu);
          stats.time_s = s->now() - r->st.t_start;
        }
      }
    } else {
      rc = nl_solve(m, r->method, r->tol, r->max_it, d, r->has_opts ? &r->opts : nullptr, &stats);
    }
    if (rc >= 0) {
      out.resize(ndof);
      if (cudaMemcpyAsync(out.data(), d, ndof * sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess) {
        rc = FE_ERR_CUDA;
        fe_set_error("copying the solution back failed");
      }
    }
  }
  std::string err = rc < 0 ? std::string(fe_last_error()) : std::string();
  if (d) cudaFreeAsync(d, stream);
  // a mesh whose solve ran (converged or not) stays resident for the next
  // request of the same description; one that failed to build or met a
  // CUDA error is freed
  const bool keep = s->cache_on && rc >= 0;
  CachedMesh* drop = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->st.t_end = s->now();
    r->st.state = rc < 0 ? FE_REQ_FAILED : FE_REQ_DONE;
    r->st.result = rc;
    r->st.stats = stats;
    r->result.swap(out);
    r->error = err;
    if (reused) {
      c->busy = false;
      c->last_used = ++s->tick;
      if (!keep) {  // unlink it; its charge goes with it
        for (auto it = s->cache.begin(); it != s->cache.end(); ++it)
          if (it->get() == c) {
            it->release();
            s->cache.erase(it);
            break;
          }
        s->used -= c->bytes;
        drop = c;
      }
    } else if (keep) {  // the request's charge becomes the resident mesh's
      c->key.swap(r->mesh_key);
      c->key_hash = r->key_hash;
      c->bytes = r->charge;
      c->last_used = ++s->tick;
      s->cache.emplace_back(c);
    } else {
      s->used -= r->charge;
      drop = c;
    }
    r->charge = 0;
    r->cm = nullptr;
    s->active--;
    s->finished.push_back(r->id);
  }
  if (drop) release_mesh(drop);
  s->cv.notify_all();
}

// joins the threads of finished requests (called without the lock held)
static void join_finished(fe_server s, std::unique_lock<std::mutex>& lk) {
  std::vector<std::thread> done;
  for (int64_t id : s->finished) {
    auto it = s->workers.find(id);
    if (it != s->workers.end()) {
      done.push_back(std::move(it->second));
      s->workers.erase(it);
    }
  }
  s->finished.clear();
  if (done.empty()) return;
  lk.unlock();
  for (auto& t : done) t.join();
  lk.lock();
}

// Batcher thread: takes every waiting request of the first waiting
// request's size class, solves them in one launch with the autotuner's
// shape, and signals their workers.
static void batcher_loop(fe_server s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->bcv.wait(lk, [s] { return s->stop_batch || !s->bq.empty(); });
    if (s->bq.empty()) break;  // stopping and nothing left
    // one size class per launch (order, precision, floor(log2 ndof)): a
    // launch lasts as long as its slowest request, so small requests do not
    // wait for large ones
    const BatchItem* f = s->bq.front();
    const int64_t key = tune_key(f->m->order, f->r->opts.precision, f->ndof);
    std::vector<BatchItem*> take;
    for (auto it = s->bq.begin(); it != s->bq.end();) {
      if (tune_key((*it)->m->order, (*it)->r->opts.precision, (*it)->ndof) == key) {
        take.push_back(*it);
        it = s->bq.erase(it);
      } else {
        ++it;
      }
    }
    TuneEntry& te = s->tune[key];
    int slot = te.chosen ? (te.chosen == 128 ? 0 : 1) : (te.batches[0] <= te.batches[1] ? 0 : 1);
    const int threads = slot == 0 ? 128 : 256;
    lk.unlock();
    const size_t n = take.size();
    std::vector<fe_mesh> meshes(n);
    std::vector<int> methods(n), max_its(n);
    std::vector<double> tols(n);
    std::vector<nl_opts> opts(n);
    std::vector<double*> ds(n);
    std::vector<fe_batch_out> outs(n);
    for (size_t i = 0; i < n; i++) {
      meshes[i] = take[i]->m;
      methods[i] = take[i]->r->method;
      max_its[i] = take[i]->r->max_it;
      tols[i] = take[i]->r->tol;
      opts[i] = take[i]->r->opts;
      ds[i] = take[i]->d;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = fe_batch_solve((int)n, meshes.data(), methods.data(), tols.data(), max_its.data(), opts.data(),
                                  ds.data(), threads, outs.data());
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const std::string err = rc < 0 ? std::string(fe_last_error()) : std::string();
    lk.lock();
    if (rc == FE_OK) {  // cost per unit of work: ndof x (nonlinear + Krylov iterations)
      double work = 0.0;
      for (size_t i = 0; i < n; i++) work += (double)take[i]->ndof * (double)(outs[i].nit + outs[i].lit_total + 1);
      const double c = dt / std::max(work, 1.0);
      TuneEntry& t2 = s->tune[key];
      t2.batches[slot]++;
      if (t2.cost[slot] == 0.0 || c < t2.cost[slot]) t2.cost[slot] = c;
      if (!t2.chosen && t2.batches[0] > 0 && t2.batches[1] > 0) t2.chosen = t2.cost[0] <= t2.cost[1] ? 128 : 256;
    }
    for (size_t i = 0; i < n; i++) {
      take[i]->rc = rc < 0 ? rc : outs[i].status;
      take[i]->out = outs[i];
      take[i]->error = err;
      take[i]->done = true;
    }
    s->cv.notify_all();
  }
}

static void scheduler_loop(fe_server s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    join_finished(s, lk);  // a long-running server keeps no thread of a finished request
    // first fit in arrival order
    bool admitted = false;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Request* r = s->reqs[*it].get();
      if (r->st.footprint > s->budget) {  // can never fit: reject
        r->st.state = FE_REQ_FAILED;
        r->st.result = FE_ERR_OOM;
        r->error = "request footprint exceeds the server's HBM budget";
        r->st.t_start = r->st.t_end = s->now();
        it = s->queue.erase(it);
        s->cv.notify_all();
        continue;
      }
      if (s->active >= s->max_active) {  // no slot (later oversized requests are still rejected)
        ++it;
        continue;
      }
      // an idle resident mesh of the same description is reused; the
      // request is then charged only what it needs beyond that mesh's charge
      CachedMesh* hit = nullptr;
      if (s->cache_on)
        for (auto& c : s->cache)
          if (!c->busy && c->key_hash == r->key_hash && c->key == r->mesh_key) {
            hit = c.get();
            break;
          }
      const int64_t need = hit ? std::max<int64_t>(0, r->st.footprint - hit->bytes) : r->st.footprint;
      if (s->used + need > s->budget) {
        // room from idle resident meshes, least recently used first
        std::vector<CachedMesh*> idle;
        int64_t idle_bytes = 0;
        for (auto& c : s->cache)
          if (!c->busy && c.get() != hit) {
            idle.push_back(c.get());
            idle_bytes += c->bytes;
          }
        if (s->used - idle_bytes + need > s->budget) {
          ++it;
          continue;
        }
        std::sort(idle.begin(), idle.end(),
                  [](const CachedMesh* a, const CachedMesh* b) { return a->last_used < b->last_used; });
        for (CachedMesh* v : idle) {
          if (s->used + need <= s->budget) break;
          for (auto ci = s->cache.begin(); ci != s->cache.end(); ++ci)
            if (ci->get() == v) {
              ci->release();
              s->cache.erase(ci);
              break;
            }
          s->used -= v->bytes;
          r->victims.push_back(v);  // freed by the request's worker before it builds
        }
      }
      s->used += need;
      s->active++;
      if (hit) {
        hit->busy = true;
        hit->bytes += need;
        r->cm = hit;
        r->charge = 0;
        r->st.mesh_reused = 1;
      } else {
        r->charge = need;
      }
      r->st.state = FE_REQ_RUNNING;
      it = s->queue.erase(it);
      s->workers.emplace(r->id, std::thread(run_request, s, r));
      admitted = true;
    }
    if (s->stop && s->queue.empty() && s->active == 0) break;
    if (!admitted) s->cv.wait(lk);
  }
}

extern "C" int serve_create(const fe_server_opts* opts, fe_server* out) {
  if (!opts || !out) return fe_set_error("NULL argument"), FE_ERR_ARG;
  *out = nullptr;
  FE_CUDA(cudaSetDevice(opts->device));
  size_t free_b = 0, total_b = 0;
  FE_CUDA(cudaMemGetInfo(&free_b, &total_b));
  fe_server s = new fe_server_s();
  s->device = opts->device;
  s->budget = opts->hbm_budget > 0 ? opts->hbm_budget : (int64_t)(0.8 * (double)free_b);
  s->max_active = opts->max_active > 0 ? opts->max_active : 8;
  s->batch_max_dofs = opts->batch_max_dofs == 0 ? 1000 : opts->batch_max_dofs;
  s->cache_on = opts->mesh_cache >= 0;
  s->scheduler = std::thread(scheduler_loop, s);
  // one batcher per slot: a lone small request launches at once, and
  // requests that wait together share a launch
  for (int i = 0; i < s->max_active; i++) s->batchers.emplace_back(batcher_loop, s);
  *out = s;
  return FE_OK;
}

template <class T>
static void copy_in(std::vector<T>& dst, const T* src, size_t n) {
  if (src && n) dst.assign(src, src + n);
  else dst.clear();
}

extern "C" int serve_submit(fe_server s, const fe_request* q, int64_t* id_out) {
  if (!s || !q || !q->mesh || !id_out) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (q->method < NL_NK || q->method > NL_IB || !(q->tol >= 0.0) || q->max_it < 0)
    return fe_set_error("bad method, tol or max_it"), FE_ERR_ARG;
  const fe_mesh_desc& d = *q->mesh;
  if (d.nv < 4 || d.ne < 1 || !d.coords || !d.tets || d.nf < 0 || d.ngroups < 0)
    return fe_set_error("bad mesh description"), FE_ERR_ARG;
  auto r = std::make_unique<Request>();
  copy_in(r->coords, d.coords, 3 * (size_t)d.nv);
  copy_in(r->tets, d.tets, 4 * (size_t)d.ne);
  copy_in(r->dir_group, d.dir_group, (size_t)d.nv);
  copy_in(r->groups, d.groups, (size_t)d.ngroups);
  copy_in(r->faces, d.faces, 3 * (size_t)d.nf);
  copy_in(r->face_kind, d.face_kind, (size_t)d.nf);
  copy_in(r->face_data, d.face_data, 3 * (size_t)d.nf);
  copy_in(r->fibers, d.fibers, d.fibers ? 9 * (size_t)d.ne : 0);
  r->desc = d;
  r->desc.coords = r->coords.data();
  r->desc.tets = r->tets.data();
  r->desc.dir_group = d.dir_group ? r->dir_group.data() : nullptr;
  r->desc.groups = d.ngroups ? r->groups.data() : nullptr;
  r->desc.faces = d.nf ? r->faces.data() : nullptr;
  r->desc.face_kind = d.nf ? r->face_kind.data() : nullptr;
  r->desc.face_data = d.nf ? r->face_data.data() : nullptr;
  r->desc.fibers = d.fibers ? r->fibers.data() : nullptr;
  r->method = q->method;
  r->tol = q->tol;
  r->max_it = q->max_it;
  if (q->opts) {
    r->opts = *q->opts;
    r->has_opts = true;
  }
  r->load = q->load;
  r->time = q->time;
  int64_t ndof = 0;
  r->st.footprint = estimate_footprint(*r, &ndof);
  r->mesh_key = mesh_key(*r);
  r->key_hash = std::hash<std::string>{}(r->mesh_key);
  if (q->d0) r->d0.assign(q->d0, q->d0 + ndof);
  r->st.state = FE_REQ_QUEUED;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->st.t_submit = s->now();
    *id_out = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
  }
  s->cv.notify_all();
  return FE_OK;
}

extern "C" int serve_poll(fe_server s, int64_t id, int wait, fe_request_status* status, double* d_out) {
  if (!s || !status) return fe_set_error("NULL argument"), FE_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fe_set_error("unknown request id %lld", (long long)id), FE_ERR_ARG;
  Request* r = it->second.get();
  if (wait)
    s->cv.wait(lk, [r] { return r->st.state == FE_REQ_DONE || r->st.state == FE_REQ_FAILED; });
  *status = r->st;
  if (r->st.state == FE_REQ_FAILED && !r->error.empty()) fe_set_error("%s", r->error.c_str());
  if (d_out && r->st.state == FE_REQ_DONE) std::memcpy(d_out, r->result.data(), r->result.size() * sizeof(double));
  return FE_OK;
}

extern "C" int serve_tuning(fe_server s, fe_tuning_entry* out, int cap) {
  if (!s) return fe_set_error("NULL server"), FE_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int i = 0;
  for (const auto& kv : s->tune) {
    if (out && i < cap) {
      fe_tuning_entry& e = out[i];
      e.order = (int32_t)(kv.first >> 40);
      e.precision = (int32_t)((kv.first >> 32) & 0xff);
      e.size_class = (int32_t)(kv.first & 0xffffffff);
      e.threads = kv.second.chosen;
      e.batches[0] = kv.second.batches[0];
      e.batches[1] = kv.second.batches[1];
      e.cost[0] = kv.second.cost[0];
      e.cost[1] = kv.second.cost[1];
    }
    i++;
  }
  return i;
}

extern "C" double serve_clock(fe_server s) { return s ? s->now() : 0.0; }

extern "C" int serve_destroy(fe_server s) {
  if (!s) return FE_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->scheduler.join();
  for (auto& t : s->workers) t.second.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_batch = true;
  }
  s->bcv.notify_all();
  for (auto& t : s->batchers) t.join();
  for (auto& c : s->cache) release_mesh(c.release());
  s->cache.clear();
  delete s;
  return FE_OK;
}
