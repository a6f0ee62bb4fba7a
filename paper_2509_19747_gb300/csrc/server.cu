// Host runtime for many systems on one GPU: a first-fit device-memory arena
// (the HBM budget), a request queue with admission by that budget, and a pool
// of worker threads, each with its own CUDA stream, that run
// randrand_build + randrand_solve + randrand_free for one request at a time.
// The kernels of concurrently resident systems overlap on the GPU through
// their separate streams; every system keeps its own captured iteration graph.
//
// randrand_solve_batch is the same machinery for a fixed set of systems:
// submitted largest workspace first (longest-processing-time order), drained,
// results returned in input order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rr_common.cuh"
#include "rr_group.cuh"

namespace {

constexpr size_t kArenaAlign = 256;

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// ------------------------------------------------------------------ arena
// First-fit allocator over [0, bytes) with coalescing of free neighbours.
// Offsets and sizes are multiples of 256 bytes.  Not thread-safe by itself:
// the server holds its lock around every call.
struct rr_arena {
  size_t bytes;
  std::map<size_t, size_t> free_;   // offset -> size
  std::map<size_t, size_t> used_;   // offset -> size

  explicit rr_arena(size_t b) : bytes(b / kArenaAlign * kArenaAlign) {
    if (bytes) free_[0] = bytes;
  }

  bool alloc(size_t want, size_t* off) {
    const size_t sz = round_up(std::max<size_t>(want, 1), kArenaAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < sz) continue;
      const size_t o = it->first, rest = it->second - sz;
      free_.erase(it);
      if (rest) free_[o + sz] = rest;
      used_[o] = sz;
      *off = o;
      return true;
    }
    return false;
  }

  bool release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return false;
    size_t o = off, sz = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(o);
    if (next != free_.end() && next->first == o + sz) {
      sz += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        o = prev->first;
        sz += prev->second;
        free_.erase(prev);
      }
    }
    free_[o] = sz;
    return true;
  }

  size_t largest_free() const {
    size_t m = 0;
    for (const auto& f : free_) m = std::max(m, f.second);
    return m;
  }
  size_t in_use() const {
    size_t s = 0;
    for (const auto& u : used_) s += u.second;
    return s;
  }
};

// ------------------------------------------------------------------ server
struct rr_server {
  unsigned char* base;
  rr_arena arena;
  int device;
  std::chrono::steady_clock::time_point t0;
  std::mutex m;
  std::condition_variable cv_work;   // workers: a request may be admitted
  std::condition_variable cv_done;   // clients: a request finished
  struct Job {
    uint64_t ticket;
    rr_request req;
    size_t ws;
  };
  std::deque<Job> queue;
  std::unordered_map<uint64_t, rr_result> results;
  uint64_t next_ticket = 1;
  int running = 0;
  size_t peak_bytes = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  // shared rounds (rr_server_create_rounds): built systems that qualify are
  // handed to one executor thread, whose group advances all of their Krylov
  // iterations together; the group's workspace sits at the front of the
  // caller's arena, before `base`
  struct Built {
    uint64_t ticket;
    rr_handle* h;
    size_t off;
    rr_request req;
    double t_start, t_build;
    rr_solve_info info[8];
  };
  bool rounds = false;
  rr_rounds_opts ropts;
  unsigned char* group_ws = nullptr;
  size_t group_bytes = 0;
  std::deque<Built*> built;
  bool stop_exec = false;
  std::condition_variable cv_exec;
  std::thread exec;
  int peak_running = 0;
  rr_rounds_stats gstats{};

  rr_server(unsigned char* b, size_t bytes, int dev) : base(b), arena(bytes), device(dev) {
    t0 = std::chrono::steady_clock::now();
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    for (;;) {
      Job job;
      size_t off = 0;
      {
        std::unique_lock<std::mutex> lk(m);
        // strict arrival order: the head of the queue is admitted as soon as
        // its workspace fits in the arena (the allocation is taken here)
        cv_work.wait(lk, [&] {
          if (stop) return true;
          return !queue.empty() && arena.alloc(queue.front().ws, &off);
        });
        if (stop) break;   // rr_server_destroy drains the queue before stopping
        job = queue.front();
        queue.pop_front();
        ++running;
        peak_running = std::max(peak_running, running);
        peak_bytes = std::max(peak_bytes, arena.in_use());
        rr_result& r = results[job.ticket];
        r.start_ms = now_ms(t0);
        r.queue_ms = r.start_ms - r.submit_ms;
      }
      rr_result out;
      memset(&out, 0, sizeof(out));
      double t_build = 0.0, t_end = 0.0;
      const double t_start = now_ms(t0);
      rr_status s = have_stream ? RR_OK : RR_ERR_CUDA;
      rr_handle* h = nullptr;
      if (s == RR_OK) {
        const rr_request& q = job.req;
        s = randrand_build(&q.op, q.mu, q.k, q.sketch, q.seed, &q.opts, base + off, job.ws, st, &h);
        t_build = now_ms(t0);
        if (s == RR_OK && rounds && rr::group_accepts(h, ropts.mp, ropts.kmax)) {
          // the executor thread solves it in the shared rounds and completes the job
          Built* bt = new (std::nothrow) Built();
          if (bt) {
            bt->ticket = job.ticket;
            bt->h = h;
            bt->off = off;
            bt->req = q;
            bt->t_start = t_start;
            bt->t_build = t_build;
            {
              std::lock_guard<std::mutex> lk(m);
              built.push_back(bt);
            }
            cv_exec.notify_all();
            continue;
          }
        }
        if (s == RR_OK) {
          s = randrand_solve(h, q.b, q.nrhs, q.ldb, q.x, q.ldx, 0, q.rtol, q.maxit, out.info);
          randrand_free(h);   // waits for the handle's stream
        }
      }
      t_end = now_ms(t0);
      {
        std::lock_guard<std::mutex> lk(m);
        arena.release(off);
        --running;
        rr_result& r = results[job.ticket];
        memcpy(r.info, out.info, sizeof(r.info));
        r.build_ms = (t_build > 0.0 ? t_build : t_end) - t_start;
        r.solve_ms = t_end - (t_build > 0.0 ? t_build : t_end);
        r.end_ms = t_end;
        r.status = s;
      }
      cv_work.notify_all();
      cv_done.notify_all();
    }
    if (have_stream) cudaStreamDestroy(st);
  }

  // a job of the shared rounds ends: handle freed, arena slice released
  void complete(Built* bt, rr_status s, bool in_rounds) {
    randrand_free(bt->h);
    const double t_end = now_ms(t0);
    {
      std::lock_guard<std::mutex> lk(m);
      arena.release(bt->off);
      --running;
      rr_result& r = results[bt->ticket];
      memcpy(r.info, bt->info, sizeof(r.info));
      r.build_ms = bt->t_build - bt->t_start;
      r.solve_ms = t_end - bt->t_build;
      r.end_ms = t_end;
      r.rounds = in_rounds ? 1 : 0;
      r.status = s;
    }
    delete bt;
    cv_work.notify_all();
    cv_done.notify_all();
  }

  void exec_main() {
    cudaSetDevice(device);
    cudaStream_t gst = nullptr;
    rr_status gs = cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking) == cudaSuccess ? RR_OK : RR_ERR_CUDA;
    rr::Group* g = nullptr;
    if (gs == RR_OK)
      g = rr::group_create(ropts.mp, ropts.kmax, ropts.max_systems, ropts.max_rows,
                           rounds_part_bytes(ropts), group_ws, group_bytes, gst, &gs);
    std::vector<Built*> pending;
    std::vector<rr::GroupDone> done;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m);
        cv_exec.wait(lk, [&] {
          return stop_exec || !built.empty() || !pending.empty() || (g && rr::group_size(g) > 0);
        });
        if (stop_exec && built.empty() && pending.empty() && !(g && rr::group_size(g) > 0)) break;
        while (!built.empty()) {
          pending.push_back(built.front());
          built.pop_front();
        }
      }
      done.clear();
      std::vector<Built*> wait;
      for (Built* bt : pending) {
        rr::GroupReq r;
        r.h = bt->h;
        r.b = bt->req.b;
        r.x = bt->req.x;
        r.ldb = bt->req.ldb;
        r.ldx = bt->req.ldx;
        r.m = bt->req.nrhs;
        r.rtol = bt->req.rtol;
        r.maxit = bt->req.maxit;
        r.info = bt->info;
        r.user = bt;
        rr_status s = g ? rr::group_add(g, r, &done) : gs;
        if (s == RR_ERR_WORKSPACE && g && rr::group_size(g) > 0) {
          wait.push_back(bt);        // joins once systems have left
        } else if (s != RR_OK) {
          // the group cannot take it (too large for its capacity, or no
          // group): solved on its own
          s = randrand_solve(bt->h, bt->req.b, bt->req.nrhs, bt->req.ldb, bt->req.x, bt->req.ldx, 0,
                             bt->req.rtol, bt->req.maxit, bt->info);
          complete(bt, s, false);
        }
      }
      pending = wait;
      if (g && rr::group_size(g) > 0) rr::group_step(g, &done);
      if (g) {
        std::lock_guard<std::mutex> lk(m);
        rr::group_stats(g, &gstats);
      }
      for (const rr::GroupDone& d : done) complete((Built*)d.user, d.status, true);
    }
    rr::group_destroy(g);
    if (gst) cudaStreamDestroy(gst);
  }

  static size_t rounds_part_bytes(const rr_rounds_opts& o) {
    // 16 partial-sum slots per stacked row and column (see group_part_bound)
    return (size_t)o.max_rows * o.mp * 4 * 16;
  }
};

namespace {

rr_status check_request(const rr_request* q) {
  if (!q || !q->b || !q->x) return RR_ERR_INVALID_ARG;
  if (q->nrhs < 1 || q->nrhs > 8 || q->nrhs > q->opts.max_rhs) return RR_ERR_INVALID_ARG;
  if (q->ldb < q->op.n || q->ldx < q->op.n) return RR_ERR_INVALID_ARG;
  if (!(q->rtol > 0.0) || !std::isfinite(q->rtol) || q->maxit < 1) return RR_ERR_INVALID_ARG;
  if (!(q->mu >= 0.0) || !std::isfinite(q->mu)) return RR_ERR_INVALID_ARG;
  return RR_OK;
}

}  // namespace

extern "C" {

rr_status rr_arena_create(size_t bytes, rr_arena** out) {
  if (!out) return RR_ERR_INVALID_ARG;
  *out = new (std::nothrow) rr_arena(bytes);
  return *out ? RR_OK : RR_ERR_INVALID_ARG;
}

rr_status rr_arena_alloc(rr_arena* a, size_t bytes, size_t* offset) {
  if (!a || !offset) return RR_ERR_INVALID_ARG;
  return a->alloc(bytes, offset) ? RR_OK : RR_ERR_WORKSPACE;
}

rr_status rr_arena_free(rr_arena* a, size_t offset) {
  if (!a) return RR_ERR_INVALID_ARG;
  return a->release(offset) ? RR_OK : RR_ERR_INVALID_ARG;
}

rr_status rr_arena_stats(const rr_arena* a, size_t* in_use, size_t* largest_free) {
  if (!a) return RR_ERR_INVALID_ARG;
  if (in_use) *in_use = a->in_use();
  if (largest_free) *largest_free = a->largest_free();
  return RR_OK;
}

void rr_arena_destroy(rr_arena* a) { delete a; }

static rr_status server_create(void* arena, size_t arena_bytes, int32_t workers,
                               const rr_rounds_opts* rounds, unsigned char* group_ws,
                               size_t group_bytes, rr_server** out) {
  if (!out) return RR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!arena || ((uintptr_t)arena & (kArenaAlign - 1)) || arena_bytes < kArenaAlign) return RR_ERR_INVALID_ARG;
  if (workers < 1 || workers > 256) return RR_ERR_INVALID_ARG;
  int dev = 0;
  RR_CUDA_TRY(cudaGetDevice(&dev));
  rr_server* s = new (std::nothrow) rr_server((unsigned char*)arena, arena_bytes, dev);
  if (!s) return RR_ERR_INVALID_ARG;
  // the rounds settings are fixed before any thread starts
  if (rounds) {
    s->rounds = true;
    s->ropts = *rounds;
    s->ropts.max_rows = (rounds->max_rows + 255) / 256 * 256;
    s->group_ws = group_ws;
    s->group_bytes = group_bytes;
  }
  try {
    if (rounds) s->exec = std::thread(&rr_server::exec_main, s);
    for (int i = 0; i < workers; ++i) s->workers.emplace_back(&rr_server::worker_main, s);
  } catch (...) {
    rr_server_destroy(s);
    return RR_ERR_INVALID_ARG;
  }
  *out = s;
  return RR_OK;
}

rr_status rr_server_create(void* arena, size_t arena_bytes, int32_t workers, rr_server** out) {
  return server_create(arena, arena_bytes, workers, nullptr, nullptr, 0, out);
}

rr_status rr_rounds_workspace_bytes(const rr_rounds_opts* o, size_t* bytes) {
  if (!o || !bytes) return RR_ERR_INVALID_ARG;
  if (o->mp < 2 || o->mp > 8 || (o->mp & (o->mp - 1)) || o->kmax < 1 || o->max_systems < 1 ||
      o->max_systems > 152 || o->max_rows < 256)
    return RR_ERR_INVALID_ARG;
  const int64_t rows = (o->max_rows + 255) / 256 * 256;
  rr_rounds_opts p = *o;
  p.max_rows = rows;
  *bytes = round_up(rr::group_bytes(o->mp, o->max_systems, rows, rr_server::rounds_part_bytes(p)),
                    kArenaAlign);
  return RR_OK;
}

rr_status rr_server_create_rounds(void* arena, size_t arena_bytes, int32_t workers,
                                  const rr_rounds_opts* rounds, rr_server** out) {
  if (!rounds) return rr_server_create(arena, arena_bytes, workers, out);
  if (!out) return RR_ERR_INVALID_ARG;
  *out = nullptr;
  size_t gb = 0;
  RR_TRY(rr_rounds_workspace_bytes(rounds, &gb));
  if (!arena || ((uintptr_t)arena & (kArenaAlign - 1)) || arena_bytes < gb + kArenaAlign)
    return RR_ERR_INVALID_ARG;
  return server_create((unsigned char*)arena + gb, arena_bytes - gb, workers, rounds,
                       (unsigned char*)arena, gb, out);
}

rr_status rr_server_submit(rr_server* s, const rr_request* req, uint64_t* ticket) {
  if (!s || !ticket) return RR_ERR_INVALID_ARG;
  RR_TRY(check_request(req));
  size_t ws = 0;
  RR_TRY(randrand_workspace_bytes(&req->op, req->k, &req->opts, &ws));
  if (round_up(ws, kArenaAlign) > s->arena.bytes) return RR_ERR_WORKSPACE;
  {
    std::lock_guard<std::mutex> lk(s->m);
    if (s->stop) return RR_ERR_INVALID_ARG;
    const uint64_t t = s->next_ticket++;
    rr_result r;
    memset(&r, 0, sizeof(r));
    r.status = RR_PENDING;
    r.nrhs = req->nrhs;
    r.ws_bytes = ws;
    r.submit_ms = now_ms(s->t0);
    s->results[t] = r;
    s->queue.push_back(rr_server::Job{t, *req, ws});
    *ticket = t;
  }
  s->cv_work.notify_all();
  return RR_OK;
}

rr_status rr_server_poll(rr_server* s, uint64_t ticket, int32_t wait, rr_result* out) {
  if (!s || !out) return RR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return RR_ERR_INVALID_ARG;
  if (wait)
    s->cv_done.wait(lk, [&] { return s->results[ticket].status != RR_PENDING; });
  *out = s->results[ticket];
  return RR_OK;
}

rr_status rr_server_drain(rr_server* s) {
  if (!s) return RR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->m);
  s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
  return RR_OK;
}

rr_status rr_server_stats(rr_server* s, int32_t* queued, int32_t* running, size_t* bytes_in_use,
                          size_t* peak_bytes) {
  if (!s) return RR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->m);
  if (queued) *queued = (int32_t)s->queue.size();
  if (running) *running = s->running;
  if (bytes_in_use) *bytes_in_use = s->arena.in_use();
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  return RR_OK;
}

rr_status rr_server_rounds_stats(rr_server* s, rr_rounds_stats* out) {
  if (!s || !out) return RR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->m);
  *out = s->gstats;
  return RR_OK;
}

rr_status rr_server_peak_running(rr_server* s, int32_t* peak) {
  if (!s || !peak) return RR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->m);
  *peak = s->peak_running;
  return RR_OK;
}

void rr_server_destroy(rr_server* s) {
  if (!s) return;
  rr_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop_exec = true;
  }
  s->cv_exec.notify_all();
  if (s->exec.joinable()) s->exec.join();
  delete s;
}

rr_status randrand_solve_batch(const rr_request* reqs, int32_t nsys, void* arena,
                               size_t arena_bytes, int32_t workers, rr_result* results) {
  return randrand_solve_batch_rounds(reqs, nsys, arena, arena_bytes, workers, nullptr, results,
                                     nullptr);
}

rr_status randrand_solve_batch_rounds(const rr_request* reqs, int32_t nsys, void* arena,
                                      size_t arena_bytes, int32_t workers,
                                      const rr_rounds_opts* rounds, rr_result* results,
                                      rr_rounds_stats* stats) {
  if (!reqs || !results || nsys < 1) return RR_ERR_INVALID_ARG;
  size_t gb = 0;
  if (rounds) RR_TRY(rr_rounds_workspace_bytes(rounds, &gb));
  std::vector<size_t> ws(nsys);
  for (int i = 0; i < nsys; ++i) {
    RR_TRY(check_request(&reqs[i]));
    RR_TRY(randrand_workspace_bytes(&reqs[i].op, reqs[i].k, &reqs[i].opts, &ws[i]));
    if (round_up(ws[i], kArenaAlign) + gb > arena_bytes) return RR_ERR_WORKSPACE;
  }
  std::vector<int> order(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ws[a] > ws[b]; });
  rr_server* s = nullptr;
  RR_TRY(rr_server_create_rounds(arena, arena_bytes, std::min(workers, nsys), rounds, &s));
  std::vector<uint64_t> tickets(nsys, 0);
  rr_status st = RR_OK;
  for (int i : order) {
    st = rr_server_submit(s, &reqs[i], &tickets[i]);
    if (st != RR_OK) break;
  }
  rr_server_drain(s);
  rr_status worst = st;
  for (int i = 0; i < nsys; ++i) {
    if (!tickets[i]) {
      memset(&results[i], 0, sizeof(rr_result));
      results[i].status = RR_ERR_INVALID_ARG;
      continue;
    }
    rr_server_poll(s, tickets[i], 1, &results[i]);
    if (worst == RR_OK && results[i].status != RR_OK) worst = results[i].status;
  }
  if (stats) rr_server_rounds_stats(s, stats);
  rr_server_destroy(s);
  return worst;
}

}  // extern "C"
