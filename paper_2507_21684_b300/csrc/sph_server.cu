// Serving loop: continuous batching of SPH rollout requests on one GPU.
//
// Requests (forward rollouts, or forward + adjoint for the mean-squared final-position loss of
// the paper's inverse problems, Sec. 4.1) are queued on submission and admitted in arrival order
// while the estimated device bytes of everything admitted stay within the HBM budget.  Admitted
// forward requests keep their particle state resident in one packed batch (segments): every
// iteration advances all of them with the same launches (one per stage); requests that arrive
// while others run join at the next iteration boundary, finished ones leave, and the batch is
// re-packed on the device (no round trip through the host).  Adjoint requests run on a pool of
// workers with a stream each, so they overlap with one another and with the forward batch on the
// device (one adjoint scene of the served sizes fills a fraction of the GPU).
// Every scene's arithmetic is independent of the others in the batch and every step rebuilds the
// cells, so a served result is bitwise the result of running that scene alone (with the cells
// rebuilt every step).
//
// Device memory: the server's scenes allocate from the CUDA stream-ordered pool of the server's
// streams, not through the allocator hook of sph_set_allocator.  The hook may call back into an
// interpreter (the PyTorch binding's caching allocator runs in Python), and the server's threads
// would then contend for that interpreter's lock on every allocation of every re-pack and adjoint
// scene: measured on the 20 requests/s stream, served adjoint requests took twice as long as the
// same requests run alone through the hook's caller.  The HBM budget of the admission covers
// these allocations as before.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "sph.h"
#include "sph_runtime.h"

namespace sph {

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Device bytes one admitted request may hold (state buffers, sort and tile scratch, adjoint tape).
// Upper bound of the device bytes a request's scene uses (admission): per particle, the two
// state buffers, sort keys and values, cell offsets, tiles, staging and the build positions;
// an adjoint adds its checkpoints, the tape slots (state, keys, permutation, offsets, tiles)
// and the adjoint work arrays.
static size_t request_bytes(const sph_params& p, int n, int nw, int steps, int mode, int ckpt) {
  const size_t per = p.dim == 2 ? 256 : 320;
  size_t b = (size_t)n * per + (1 << 20);
  if (nw > 0) b += wall_plan_bytes(p, n - nw, n);  // the fused wall + sweep launch's tile plans
  if (p.diffusion == SPH_DIFFUSION_RENORM && p.density_mode == SPH_DENSITY_CONTINUITY) b += (size_t)n * 16;
  if (mode == SPH_REQ_ADJOINT) {
    const size_t rec = p.dim == 2 ? 72 : 96;  // one copy of the records
    const int k = std::max(ckpt, 1);
    // checkpoints, two tapes of k + 1 slots (records, keys, permutation), the adjoint state and
    // the replay's working copies
    b += (size_t)((steps + k - 1) / k) * n * rec + 2 * (size_t)(k + 1) * n * (rec + 16) + (size_t)n * (3 * rec + 64);
  }
  return b;
}

struct Request {
  uint64_t id = 0;
  sph_params p{};
  int nf = 0, nw = 0, n = 0, d = 2;
  std::vector<float> x, v, rho, mass, xtgt;
  std::vector<float> ghost;  // mDBC ghost nodes of the walls (kept for every re-pack)
  int n_steps = 0, mode = 0, ckpt = 20;
  size_t bytes = 0;
  int phase = 0;  // 0 queued, 1 admitted, 2 done
  int steps_done = 0;
  int seg = -1;   // segment in the current batch
  int status = SPH_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::vector<float> rx, rv, rr, gx, gv, gr;  // results
  double nubar = 0, loss = 0;
};

constexpr int kAdjWorkers = 3;  // adjoint requests in flight at once

struct Server {
  size_t budget = 0;
  int max_active = 0;
  int device = 0;
  cudaStream_t st_fwd = nullptr, st_adj[kAdjWorkers] = {};
  std::thread th_fwd, th_adj[kAdjWorkers];
  std::mutex mu;
  std::condition_variable cv_work, cv_adj, cv_done;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active, joining;
  std::deque<std::shared_ptr<Request>> adj_queue;
  int adj_running = 0;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  size_t used = 0;
  std::unique_ptr<Scene> batch;
  int chunk = 8;
  // statistics
  double particle_steps_fwd = 0, particle_steps_adj = 0;
  int max_batch = 0;
  long long repacks = 0, iterations = 0;

  // Forward requests share one batch only when they share the settings a batch holds in common
  // (the launches' template choices and the rebuild policy).
  static bool same_class(const sph_params& a, const sph_params& b) {
    return a.dim == b.dim && a.kernel == b.kernel && (a.density_mode == 1) == (b.density_mode == 1) &&
           (a.skin > 0.f) == (b.skin > 0.f) && a.rebuild_interval == b.rebuild_interval && a.diffusion == b.diffusion &&
           (a.shift > 0.f) == (b.shift > 0.f) && a.boundary == b.boundary;
  }

  void admit_locked() {
    while (!queue.empty()) {
      auto& r = queue.front();
      const int running = (int)(active.size() + joining.size()) + adj_running + (int)adj_queue.size();
      if (used + r->bytes > budget || running >= max_active) break;
      // a forward request of another class waits (in arrival order) until the batch has drained
      if (r->mode == SPH_REQ_FORWARD) {
        const Request* other = !active.empty() ? active.front().get() : !joining.empty() ? joining.front().get() : nullptr;
        if (other && !same_class(other->p, r->p)) break;
      }
      used += r->bytes;
      r->phase = 1;
      r->t_admit = now_s();
      if (r->mode == SPH_REQ_ADJOINT) {
        adj_queue.push_back(r);
        cv_adj.notify_one();
      } else {
        joining.push_back(r);
      }
      queue.pop_front();
    }
  }

  void finish_locked(const std::shared_ptr<Request>& r, int status, const std::string& err) {
    r->status = status;
    r->err = err;
    r->phase = 2;
    r->t_done = now_s();
    used -= r->bytes;
    cv_done.notify_all();
    cv_work.notify_one();
  }

  // Build the next batch from the running requests followed by the joining ones.  Running
  // scenes are copied device to device from the previous batch; joining ones are uploaded.
  void repack(std::vector<std::shared_ptr<Request>>& next) {
    if (next.empty()) {
      batch.reset();
      return;
    }
    std::vector<sph_params> prm;
    std::vector<int> nfs, nws;
    std::vector<double> mx;
    for (auto& r : next) {
      prm.push_back(r->p);
      nfs.push_back(r->nf);
      nws.push_back(r->nw);
      double m = 1.0;
      for (int q = 0; q < 3; ++q) m = std::max(m, std::max(std::fabs(r->p.box_lo[q]), std::fabs(r->p.box_hi[q])));
      for (float c : r->x) m = std::max(m, (double)std::fabs(c));
      mx.push_back(std::max(m, 16.0));
    }
    auto nb = std::make_unique<Scene>();
    // (no init_mem: the server's scenes allocate from the CUDA stream-ordered pool, see above)
    nb->setup_checked(prm, nfs, nws, mx);
    nb->bind_stream(st_fwd);
    nb->alloc_all();
    nb->use_graphs = false;
    nb->eager_dev = true;  // with a Verlet skin the batch rebuilds when the device decides, not every step
    if (nb->mdbc) {
      std::vector<float> g;
      for (auto& r : next) g.insert(g.end(), r->ghost.begin(), r->ghost.end());
      nb->set_ghosts(g.data(), 0);
    }
    for (size_t k = 0; k < next.size(); ++k) {
      auto& r = next[k];
      if (r->seg >= 0 && batch) {
        const DevSeg& o = batch->segs[r->seg];
        if (nb->D == 2)
          launch_copy_range<2>(batch->buf[batch->cur], o.p0, nb->buf[nb->cur], nb->segs[k].p0, r->n, (int)k, st_fwd);
        else
          launch_copy_range<3>(batch->buf[batch->cur], o.p0, nb->buf[nb->cur], nb->segs[k].p0, r->n, (int)k, st_fwd);
        CKL();
      } else {
        nb->upload((int)k, r->x.data(), r->v.data(), r->rho.data(), r->mass.data(), 0);
      }
      r->seg = (int)k;
    }
    CK(cudaStreamSynchronize(st_fwd));
    for (auto& r : next) {  // inputs are now on the device
      std::vector<float>().swap(r->x);
      std::vector<float>().swap(r->v);
      std::vector<float>().swap(r->rho);
      std::vector<float>().swap(r->mass);
    }
    batch = std::move(nb);
    ++repacks;
  }

  void forward_loop() {
    cudaSetDevice(device);
    while (true) {
      std::vector<std::shared_ptr<Request>> next;
      bool need_repack = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::milliseconds(2),
                         [&] { return stop || !queue.empty() || !joining.empty() || !active.empty(); });
        if (stop) break;
        admit_locked();
        if (!joining.empty()) {
          next = active;
          next.insert(next.end(), joining.begin(), joining.end());
          joining.clear();
          need_repack = true;
        }
      }
      try {
        if (need_repack) {
          repack(next);
          std::lock_guard<std::mutex> lk(mu);
          active = next;
        }
        if (active.empty()) continue;
        int k = chunk;
        for (auto& r : active) k = std::min(k, r->n_steps - r->steps_done);
        if (k > 0) {
          batch->steps(k);
          ++iterations;
        }
        max_batch = std::max(max_batch, (int)active.size());
        std::vector<std::shared_ptr<Request>> done, keep;
        for (auto& r : active) {
          r->steps_done += std::max(k, 0);
          particle_steps_fwd += (double)r->nf * std::max(k, 0);
          (r->steps_done >= r->n_steps ? done : keep).push_back(r);
        }
        if (!done.empty()) {
          // scenes that became unstable fail alone; the others continue
          const std::vector<int> sw = batch->status_words();
          if (sw[0] & ~1) batch->check_status();  // an internal error fails the batch
          if (sw[0] & 1) {
            std::vector<std::shared_ptr<Request>> bad;
            auto unstable = [&](const std::shared_ptr<Request>& r) { return (sw[4 + r->seg] & 1) != 0; };
            for (auto& r : active)
              if (unstable(r)) bad.push_back(r);
            done.erase(std::remove_if(done.begin(), done.end(), unstable), done.end());
            keep.erase(std::remove_if(keep.begin(), keep.end(), unstable), keep.end());
            batch->clear_unstable();
            std::lock_guard<std::mutex> lk(mu);
            for (auto& r : bad)
              finish_locked(r, SPH_EUNSTABLE, "unstable state: non-finite values or density outside [0.5, 2] rho0");
          }
          for (auto& r : done) {
            const DevSeg& g = batch->segs[r->seg];
            float* dev = (float*)batch->mem_tmp(sizeof(float) * (size_t)r->n * (2 * r->d + 1));
            if (batch->D == 2)
              launch_download_range<2>(batch->buf[batch->cur], g.p0, r->n, dev, dev + (size_t)r->n * r->d,
                                       dev + (size_t)2 * r->n * r->d, st_fwd);
            else
              launch_download_range<3>(batch->buf[batch->cur], g.p0, r->n, dev, dev + (size_t)r->n * r->d,
                                       dev + (size_t)2 * r->n * r->d, st_fwd);
            CKL();
            r->rx.resize((size_t)r->n * r->d);
            r->rv.resize((size_t)r->n * r->d);
            r->rr.resize(r->n);
            CK(cudaMemcpyAsync(r->rx.data(), dev, 4 * r->rx.size(), cudaMemcpyDeviceToHost, st_fwd));
            CK(cudaMemcpyAsync(r->rv.data(), dev + r->rx.size(), 4 * r->rv.size(), cudaMemcpyDeviceToHost, st_fwd));
            CK(cudaMemcpyAsync(r->rr.data(), dev + 2 * r->rx.size(), 4 * r->rr.size(), cudaMemcpyDeviceToHost, st_fwd));
            CK(cudaStreamSynchronize(st_fwd));
          }
          // the remaining requests continue in a re-packed batch
          std::vector<std::shared_ptr<Request>> next2 = keep;
          {
            std::lock_guard<std::mutex> lk(mu);
            for (auto& r : done) finish_locked(r, SPH_OK, "");
            admit_locked();
            next2.insert(next2.end(), joining.begin(), joining.end());
            joining.clear();
          }
          repack(next2);
          std::lock_guard<std::mutex> lk(mu);
          active = next2;
        }
      } catch (const Fail& f) {
        // a failed batch fails its requests; the loop keeps serving the queue
        std::string e = last_error();
        std::lock_guard<std::mutex> lk(mu);
        for (auto& r : active) finish_locked(r, f.code, e);
        active.clear();
        batch.reset();
      }
    }
  }

  void adjoint_loop(int w) {
    cudaSetDevice(device);
    while (true) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_adj.wait(lk, [&] { return stop || !adj_queue.empty(); });
        if (stop) break;
        r = adj_queue.front();
        adj_queue.pop_front();
        ++adj_running;
      }
      int status = SPH_OK;
      std::string err;
      try {
        Scene sc;
        double m = 16.0;
        for (float c : r->x) m = std::max(m, (double)std::fabs(c));
        sc.setup_checked({r->p}, {r->nf}, {r->nw}, {m});
        sc.bind_stream(st_adj[w]);
        // a one-off scene: eager steps (capturing graphs costs more than it saves here) that take
        // the device's rebuild decision, so a Verlet skin pays off as in graph-launched steps
        sc.use_graphs = false;
        sc.eager_dev = true;
        sc.alloc_all();
        sc.upload(0, r->x.data(), r->v.data(), r->rho.data(), r->mass.data(), 0);
        sc.rollout(r->n_steps, r->ckpt);
        r->rx.resize((size_t)r->n * r->d);
        r->rv.resize((size_t)r->n * r->d);
        r->rr.resize(r->n);
        sc.get_state(r->rx.data(), r->rv.data(), r->rr.data(), 0);
        // loss L = (1/N) sum_i |x_i^T - x~_i|^2 and its seed 2 (x^T - x~) / N (Sec. 4.1)
        const std::vector<float>& tg = r->xtgt.empty() ? r->x : r->xtgt;
        std::vector<float> seed((size_t)r->n * r->d);
        double L = 0.0;
        for (size_t q = 0; q < seed.size(); ++q) {
          const double e = (double)r->rx[q] - (double)tg[q];
          L += e * e;
          seed[q] = (float)(2.0 * e / r->nf);
        }
        r->loss = L / r->nf;
        r->gx.resize(seed.size());
        r->gv.resize(seed.size());
        r->gr.resize(r->n);
        double nub = 0.0;
        sc.adjoint(seed.data(), nullptr, nullptr, r->gx.data(), r->gv.data(), r->gr.data(), &nub, 0);
        r->nubar = nub;
        std::lock_guard<std::mutex> lk(mu);
        particle_steps_adj += (double)r->nf * r->n_steps;
      } catch (const Fail& f) {
        status = f.code;
        err = last_error();
      }
      std::lock_guard<std::mutex> lk(mu);
      --adj_running;
      finish_locked(r, status, err);
    }
  }
};

}  // namespace sph

using sph::Fail;
using sph::Server;

struct sph_server {
  Server s;
};

extern "C" {

int sph_server_create(size_t hbm_budget_bytes, int max_active, sph_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_active < 1) {
    sph::set_err("sph_server_create: budget > 0 and max_active >= 1 required");
    return SPH_EINVAL;
  }
  try {
    auto* sv = new sph_server();
    Server& s = sv->s;
    s.budget = hbm_budget_bytes;
    s.max_active = max_active;
    CK(cudaGetDevice(&s.device));
    // the adjoint workers' streams take the highest priority: an adjoint request is several times
    // as long as a forward one of its size and sets the tail of the latencies when it shares the
    // GPU with the forward batch
    int prio_lo = 0, prio_hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    CK(cudaStreamCreateWithPriority(&s.st_fwd, cudaStreamNonBlocking, prio_lo));
    for (int w = 0; w < sph::kAdjWorkers; ++w) CK(cudaStreamCreateWithPriority(&s.st_adj[w], cudaStreamNonBlocking, prio_hi));
    s.th_fwd = std::thread([&s] { s.forward_loop(); });
    for (int w = 0; w < sph::kAdjWorkers; ++w) s.th_adj[w] = std::thread([&s, w] { s.adjoint_loop(w); });
    *out = sv;
  } catch (const Fail& f) {
    return f.code;
  }
  return SPH_OK;
}

int sph_submit(sph_server* sv, const sph_request* rq, uint64_t* ticket) {
  if (!sv || !rq || !ticket || !rq->x || !rq->rho || !rq->mass || rq->n_steps < 1 ||
      (rq->mode != SPH_REQ_FORWARD && rq->mode != SPH_REQ_ADJOINT)) {
    sph::set_err("sph_submit: bad request");
    return SPH_EINVAL;
  }
  Server& s = sv->s;
  auto r = std::make_shared<sph::Request>();
  r->p = rq->params;
  r->nf = rq->n_fluid;
  r->nw = rq->n_wall;
  r->n = r->nf + r->nw;
  r->d = rq->params.dim;
  if (r->n < 1 || (r->d != 2 && r->d != 3)) {
    sph::set_err("sph_submit: bad particle counts or dimension");
    return SPH_EINVAL;
  }
  if (rq->mode == SPH_REQ_ADJOINT &&
      (r->nw != 0 || (rq->params.density_mode == SPH_DENSITY_CONTINUITY && rq->params.diffusion != SPH_DIFFUSION_MC) ||
       rq->params.shift > 0.f)) {
    // (no walls, so the wall treatment does not matter)
    sph::set_err("sph_submit: adjoint requests need no wall particles, no shifting and, in continuity mode, the MC diffusion");
    return SPH_EINVAL;
  }
  const size_t nd = (size_t)r->n * r->d;
  r->x.assign(rq->x, rq->x + nd);
  r->v = rq->v ? std::vector<float>(rq->v, rq->v + nd) : std::vector<float>(nd, 0.f);
  r->rho.assign(rq->rho, rq->rho + r->n);
  r->mass.assign(rq->mass, rq->mass + r->n);
  if (rq->x_target) r->xtgt.assign(rq->x_target, rq->x_target + nd);
  if (rq->params.boundary == SPH_BOUNDARY_MDBC && r->nw > 0) {
    if (!rq->ghost) {
      sph::set_err("sph_submit: an mDBC request with walls needs its ghost nodes");
      return SPH_EINVAL;
    }
    r->ghost.assign(rq->ghost, rq->ghost + (size_t)r->nw * r->d);
  }
  r->n_steps = rq->n_steps;
  r->mode = rq->mode;
  r->ckpt = rq->ckpt_every > 0 ? rq->ckpt_every : 20;
  try {  // (validates the parameters: make_seg rejects an invalid scene with SPH_EINVAL)
    r->bytes = sph::request_bytes(rq->params, r->n, r->nw, r->n_steps, r->mode, r->ckpt);
  } catch (const Fail& f) {
    return f.code;
  } catch (...) {
    sph::set_err("sph_submit: unexpected internal exception");
    return SPH_EINTERNAL;
  }
  if (r->bytes > s.budget) {
    sph::set_err("sph_submit: the request alone exceeds the HBM budget");
    return SPH_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s.mu);
  r->id = s.next_id++;
  r->t_submit = sph::now_s();
  s.queue.push_back(r);
  s.all[r->id] = r;
  *ticket = r->id;
  s.cv_work.notify_one();
  return SPH_OK;
}

int sph_poll(sph_server* sv, uint64_t ticket, int* done) {
  if (!sv || !done) return SPH_EINVAL;
  std::lock_guard<std::mutex> lk(sv->s.mu);
  auto it = sv->s.all.find(ticket);
  if (it == sv->s.all.end()) {
    sph::set_err("sph_poll: unknown ticket");
    return SPH_EINVAL;
  }
  *done = it->second->phase == 2;
  return SPH_OK;
}

int sph_wait(sph_server* sv, uint64_t ticket, int timeout_ms, sph_result* res) {
  if (!sv) return SPH_EINVAL;
  Server& s = sv->s;
  std::shared_ptr<sph::Request> r;
  {
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.all.find(ticket);
    if (it == s.all.end()) {
      sph::set_err("sph_wait: unknown ticket");
      return SPH_EINVAL;
    }
    r = it->second;
    const bool ok = s.cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                       [&] { return r->phase == 2; });
    if (!ok) {
      sph::set_err("sph_wait: the request has not finished within the timeout");
      return SPH_ETIMEOUT;
    }
    s.all.erase(it);
  }
  if (r->status != SPH_OK) {
    sph::set_err(r->err);
    return r->status;
  }
  if (res) {
    if (res->x) std::copy(r->rx.begin(), r->rx.end(), res->x);
    if (res->v) std::copy(r->rv.begin(), r->rv.end(), res->v);
    if (res->rho) std::copy(r->rr.begin(), r->rr.end(), res->rho);
    if (r->mode == SPH_REQ_ADJOINT) {
      if (res->xbar0) std::copy(r->gx.begin(), r->gx.end(), res->xbar0);
      if (res->vbar0) std::copy(r->gv.begin(), r->gv.end(), res->vbar0);
      if (res->rhobar0) std::copy(r->gr.begin(), r->gr.end(), res->rhobar0);
    }
    res->nubar = r->nubar;
    res->loss = r->loss;
    res->t_submit = r->t_submit;
    res->t_admit = r->t_admit;
    res->t_done = r->t_done;
  }
  return SPH_OK;
}

int sph_server_stats(sph_server* sv, sph_server_info* st) {
  if (!sv || !st) return SPH_EINVAL;
  Server& s = sv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  st->particle_steps_fwd = s.particle_steps_fwd;
  st->particle_steps_adj = s.particle_steps_adj;
  st->queued = (int)s.queue.size();
  st->active = (int)(s.active.size() + s.joining.size()) + s.adj_running + (int)s.adj_queue.size();
  st->max_batch = s.max_batch;
  st->bytes_in_use = s.used;
  st->repacks = s.repacks;
  st->iterations = s.iterations;
  return SPH_OK;
}

void sph_server_destroy(sph_server* sv) {
  if (!sv) return;
  Server& s = sv->s;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.stop = true;
  }
  s.cv_work.notify_all();
  s.cv_adj.notify_all();
  if (s.th_fwd.joinable()) s.th_fwd.join();
  for (auto& th : s.th_adj)
    if (th.joinable()) th.join();
  s.batch.reset();
  cudaStreamSynchronize(s.st_fwd);
  cudaStreamDestroy(s.st_fwd);
  for (auto& st : s.st_adj) {
    if (!st) continue;
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete sv;
}

}  // extern "C"
