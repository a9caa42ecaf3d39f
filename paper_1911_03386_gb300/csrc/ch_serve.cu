// ch_serve.cu -- continuous-batching server of single-run requests (ch_server_* ABI).
//
// The paper (Sec. 4.1) ran its M = 1024 simulations as separate processes sharing two
// GPUs through the CUDA MPS server.  Here one process serves a stream of single-run
// requests of differing grid size, initial mean and horizon: a worker thread keeps every
// admitted run's field in device memory, steps all of them together with the same kernel
// launches as an uneven batch (ch_create_batch), admits queued requests as soon as a member
// slot and room for their fields in the HBM budget free up, and retires each run the step
// its horizon ends.  Requests that arrive while others run join the next chunk of steps;
// a run's arithmetic depends only on its own size and parameters (per-member tiles, fixed
// reduction order), so its result is the same alone and in any mix.
//
// Memory: the budget is split into two arenas (the fields C and the row-solve scratch W),
// allocated once at creation; a run of nx*ny points takes nx*ny elements at the same
// offset in both (first-fit, 256-byte aligned).  Admission is FIFO: the head of the queue
// waits until it fits, later requests wait behind it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_handle.h"
#include "ch_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kAlignElems = 64;      // 256 B for FP32, 512 B for FP64
constexpr int64_t kMaxChunk = 64;        // steps between retire/admit decisions
constexpr int64_t kMaxQueue = 1 << 20;   // pending requests before CH_EBUSY
constexpr int kDefaultEvery = 100;

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

// First-fit allocator over element offsets of the field arenas.
struct Arena {
  int64_t capacity = 0, used = 0, peak = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length

  void init(int64_t cap) {
    capacity = cap;
    free_.clear();
    if (cap > 0) free_[0] = cap;
  }
  static int64_t round(int64_t n) { return (n + kAlignElems - 1) / kAlignElems * kAlignElems; }
  int64_t alloc(int64_t n) {
    n = round(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        used += n;
        peak = std::max(peak, used);
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    n = round(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Req {
  uint64_t id = 0;
  ch_member_desc d{};
  int64_t nsteps = 0;
  int every = kDefaultEvery;
  double t1 = 0.0;
  double* field_out = nullptr;
  int slot = -1;
  int64_t offset = -1, elems = 0;
  bool comp = false;          // FP32 run at large s: a second arena block holds the lo part
  int64_t lo_offset = -1;
  int status = CH_PENDING;
  Clock::time_point t_submit, t_admit, t_done;
  ch_result res{};
};

}  // namespace

struct ch_server_s {
  ch_ensemble* h = nullptr;
  Arena arena;
  int* dlist = nullptr;  // device list of members to initialise
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<uint64_t> slot_req;  // slot -> request id, 0 = free
  uint64_t next_id = 1;
  bool stop = false;
  int error = CH_OK;
  std::string error_msg;
  std::thread worker;
  // statistics (under mu)
  int64_t submitted = 0, completed = 0, running = 0, max_running = 0;
  int64_t member_steps = 0, point_steps = 0, chunks = 0;
  double busy_s = 0.0;
  Clock::time_point t_created;
};

namespace {

int server_fail_all(ch_server_s* S, int code, const std::string& msg) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->error = code;
  S->error_msg = msg;
  for (auto& kv : S->reqs)
    if (kv.second.status == CH_PENDING) kv.second.status = code;
  S->queue.clear();
  S->cv_done.notify_all();
  return code;
}

// Set up the members admitted into `slots` (parameters, state, initial field), then
// rebuild the tile tables of every present member.
int admit_slots(ch_server_s* S, const std::vector<int>& slots, const std::vector<Req*>& reqs) {
  ch_ensemble* h = S->h;
  std::vector<MemberState> init(slots.size());  // lives until the stream is synchronised below
  for (size_t i = 0; i < slots.size(); ++i) {
    const int k = slots[i];
    const Req& r = *reqs[i];
    if (int rc = chh::fill_params(r.d, h->precision, &h->hp[k])) return rc;
    h->hp[k].offset = r.offset;
    h->hp[k].lo_offset = r.comp ? r.lo_offset : -1;
    h->hp[k].every = r.every;
    h->hp[k].t1 = r.t1;
    h->hp[k].series_cap = 0;
    h->present[k] = 1;
    init[i] = MemberState{};
    init[i].remaining = r.nsteps;
    CH_CHECK_CUDA(cudaMemcpyAsync(h->dms + k, &init[i], sizeof(MemberState), cudaMemcpyHostToDevice, h->stream),
                  "member state");
  }
  if (int rc = chh::build_tiles(h, h->tuning)) return rc;
  if (int rc = chh::upload_tiles(h)) return rc;  // uploads parameters too; synchronises
  CH_CHECK_CUDA(cudaMemcpyAsync(S->dlist, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice, h->stream),
                "member list");
  int64_t maxp = 0;
  for (const Req* r : reqs) maxp = std::max<int64_t>(maxp, (int64_t)r->d.nx * r->d.ny);
  CH_CHECK_CUDA(chk::launch_init_members(h->view(), h->precision, S->dlist, (int)slots.size(), maxp, h->stream),
                "initial fields");
  CH_CHECK_CUDA(cudaStreamSynchronize(h->stream), "admit");
  return CH_OK;
}

void worker_main(ch_server_s* S) {
  ch_ensemble* h = S->h;
  cudaSetDevice(h->device);
  std::vector<MemberState> states;
  std::vector<double> obs(3 * (size_t)h->m), fbuf;
  for (;;) {
    std::vector<int> slots;
    std::vector<Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || S->running > 0; });
      if (S->stop) return;
      while (!S->queue.empty()) {
        Req& r = S->reqs[S->queue.front()];
        auto free_slot = std::find(S->slot_req.begin(), S->slot_req.end(), (uint64_t)0);
        if (free_slot == S->slot_req.end()) break;
        const int64_t off = S->arena.alloc(r.elems);
        if (off < 0) break;
        int64_t lo = -1;
        if (r.comp && (lo = S->arena.alloc(r.elems)) < 0) {
          S->arena.release(off, r.elems);
          break;
        }
        r.slot = (int)(free_slot - S->slot_req.begin());
        r.offset = off;
        r.lo_offset = lo;
        r.t_admit = Clock::now();
        *free_slot = r.id;
        slots.push_back(r.slot);
        admitted.push_back(&r);
        S->queue.pop_front();
        S->running += 1;
        S->max_running = std::max(S->max_running, S->running);
      }
    }
    const auto t0 = Clock::now();
    if (!slots.empty()) {
      if (int rc = admit_slots(S, slots, admitted)) {
        server_fail_all(S, rc, "admission failed");
        return;
      }
    }
    // run until the first present run's horizon ends, at most kMaxChunk steps
    int64_t chunk = kMaxChunk;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (size_t k = 0; k < S->slot_req.size(); ++k)
        if (S->slot_req[k]) {
          const Req& r = S->reqs[S->slot_req[k]];
          chunk = std::min<int64_t>(chunk, r.nsteps - r.res.steps);
        }
    }
    chunk = std::max<int64_t>(chunk, 1);
    chk::stall_if_armed();  // injected stall of this host thread (fault injection)
    if (int rc = chh::launch_steps_direct(h, chunk)) {
      server_fail_all(S, rc, "step launch failed");
      return;
    }
    // states of the occupied slots only (slots are taken lowest-first)
    int hi = 0;
    for (int k = 0; k < h->m; ++k)
      if (h->has(k)) hi = k + 1;
    states.resize(h->m);
    if (hi > 0 && chh::copy_out(h, states.data(), h->dms, sizeof(MemberState) * hi, "read member state") != CH_OK) {
      server_fail_all(S, CH_ECUDA, "state read failed");
      return;
    }
    // finished runs: final observables of their fields, then results out
    std::vector<int> done;
    for (int k = 0; k < hi; ++k)
      if (h->has(k) && states[k].remaining == 0) done.push_back(k);
    if (!done.empty()) {
      cudaError_t e = chk::launch_observe(h->view(), h->precision, h->shape, h->stream);
      if (e != cudaSuccess || chh::copy_out(h, obs.data(), h->dobs, sizeof(double) * obs.size(), "observables")) {
        server_fail_all(S, CH_ECUDA, "final observables failed");
        return;
      }
    }
    std::vector<std::pair<uint64_t, ch_result>> finished;
    for (int k : done) {
      uint64_t id;
      double* fout;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        id = S->slot_req[k];
        fout = S->reqs[id].field_out;
      }
      if (fout) {
        if (int rc = chh::read_member_field(h, k, fout)) {
          server_fail_all(S, rc, "field read failed");
          return;
        }
      }
      ch_result res{};
      res.steps = states[k].step;
      res.F = obs[3 * k];
      res.dFdt = obs[3 * k + 1];
      res.beta = obs[3 * k + 2];
      res.beta_count = states[k].beta_count;
      res.beta_avg = states[k].beta_count ? states[k].beta_sum / (double)states[k].beta_count : NAN;
      res.nonfinite = states[k].nonfinite || !std::isfinite(res.F) || !std::isfinite(res.dFdt);
      finished.emplace_back(id, res);
      h->present[k] = 0;
    }
    if (!done.empty()) {
      if (int rc = chh::build_tiles(h, h->tuning)) {
        server_fail_all(S, rc, "tile rebuild failed");
        return;
      }
      if (int rc = chh::upload_tiles(h)) {
        server_fail_all(S, rc, "tile upload failed");
        return;
      }
    }
    const auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->chunks += 1;
      S->busy_s += seconds(t1 - t0);
      for (size_t k = 0; k < S->slot_req.size(); ++k)
        if (S->slot_req[k]) {
          Req& r = S->reqs[S->slot_req[k]];
          const int64_t adv = std::min<int64_t>(chunk, r.nsteps - r.res.steps);
          r.res.steps += adv;
          S->member_steps += adv;
          S->point_steps += adv * (int64_t)r.d.nx * r.d.ny;
        }
      for (auto& f : finished) {
        Req& r = S->reqs[f.first];
        const int64_t steps_before = r.res.steps;
        r.res = f.second;
        r.res.steps = steps_before;
        r.t_done = t1;
        r.res.t_queued_s = seconds(r.t_admit - r.t_submit);
        r.res.t_run_s = seconds(r.t_done - r.t_admit);
        r.res.t_total_s = seconds(r.t_done - r.t_submit);
        r.status = r.res.nonfinite ? CH_ENONFINITE : CH_OK;
        S->arena.release(r.offset, r.elems);
        if (r.comp) S->arena.release(r.lo_offset, r.elems);
        S->slot_req[r.slot] = 0;
        S->running -= 1;
        S->completed += 1;
      }
      if (!finished.empty()) S->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

int ch_server_create(size_t hbm_budget_bytes, int precision, int max_members, ch_server* out) {
  using chh::fail;
  if (!out) return fail(CH_EINVAL, "out is NULL");
  *out = nullptr;
  if (precision != CH_FP64 && precision != CH_FP32) return fail(CH_EINVAL, "precision must be CH_FP64 or CH_FP32");
  if (max_members < 1 || max_members > (1 << 20)) return fail(CH_EINVAL, "max_members must be in [1, 2^20]");
  const size_t elt = precision == CH_FP64 ? sizeof(double) : sizeof(float);
  const int64_t elems = (int64_t)(hbm_budget_bytes / (2 * elt)) / kAlignElems * kAlignElems;
  if (elems < 25 * 2) return fail(CH_EINVAL, "HBM budget too small for any run");
  ch_server_s* S = new ch_server_s();
  ch_ensemble* h = new ch_ensemble();
  S->h = h;
  h->precision = precision;
  h->m = max_members;
  h->elt = elt;
  cudaGetDevice(&h->device);
  h->hp.assign(max_members, MemberParams{});
  h->hseg.assign(max_members, chk::SegTable{});
  h->hsegy.assign(max_members, chk::SegTable{});
  for (auto& p : h->hp) p.every = 1;
  h->present.assign(max_members, 0);
  // Fused form for both precisions: segment-form rows and columns where a run's size
  // allows (per run, so a result does not depend on the mix), streaming columns (FP64) or
  // panels (FP32) for the others.  The split form's thread-per-line streams need many
  // lines to fill the GPU, which a handful of served runs does not give.
  h->tuning = chh::default_tuning();
  h->tuning.split = 0;
  S->slot_req.assign(max_members, 0);
  S->arena.init(elems);
  cudaError_t e;
  auto cleanup = [&](int code, const std::string& msg) {
    cudaFree(h->C);
    cudaFree(h->W);
    cudaFree(h->dmp);
    cudaFree(h->dms);
    cudaFree(h->dseg);
    cudaFree(h->dsegy);
    cudaFree(h->dobs);
    cudaFree(S->dlist);
    cudaFree(h->drt);  // tile tables, if upload_tiles allocated them before failing
    cudaFree(h->dst);
    cudaFree(h->dct);
    cudaFree(h->dcst);
    cudaFree(h->dres);
    cudaFree(h->dpart);
    if (h->own) cudaStreamDestroy(h->own);
    delete h;
    delete S;
    cudaGetLastError();
    return fail(code, msg);
  };
  if ((e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup(CH_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  h->stream = h->own;
  if ((e = chk::dev_malloc(&h->C, elt * elems)) != cudaSuccess || (e = chk::dev_malloc(&h->W, elt * elems)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&h->dmp, sizeof(MemberParams) * max_members)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&h->dms, sizeof(MemberState) * max_members)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&h->dseg, sizeof(chk::SegTable) * max_members)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&h->dsegy, sizeof(chk::SegTable) * max_members)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&h->dobs, sizeof(double) * 3 * max_members)) != cudaSuccess ||
      (e = chk::dev_malloc((void**)&S->dlist, sizeof(int) * max_members)) != cudaSuccess)
    return cleanup(e == cudaErrorMemoryAllocation ? CH_ENOMEM : CH_ECUDA,
                   std::string("server allocation: ") + cudaGetErrorString(e));
  if ((e = chk::set_kernel_smem_limits(precision)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->dms, 0, sizeof(MemberState) * max_members, h->stream)) != cudaSuccess)
    return cleanup(CH_ECUDA, std::string("server set-up: ") + cudaGetErrorString(e));
  if (int rc = chh::build_tiles(h, h->tuning)) return cleanup(rc, "server tiles");
  if (int rc = chh::upload_tiles(h)) return cleanup(rc, "server tiles");
  S->t_created = Clock::now();
  S->worker = std::thread(worker_main, S);
  *out = S;
  return CH_OK;
}

int ch_submit(ch_server s, const ch_request* r, uint64_t* id) {
  using chh::fail;
  if (!s || !r || !id) return fail(CH_EINVAL, "NULL argument");
  ch_member_desc d;
  d.nx = r->nx;
  d.ny = r->ny;
  d.L = r->L;
  d.gamma = r->gamma;
  d.dt = r->dt;
  d.C0 = r->C0;
  d.seed = r->seed;
  d.counter_base = 0;
  if (int rc = chh::validate_desc(d, 0)) return rc;
  if (r->nsteps < 1) return fail(CH_EINVAL, "nsteps must be >= 1");
  if (r->every < 0) return fail(CH_EINVAL, "every must be >= 0");
  const int64_t elems = (int64_t)r->nx * r->ny;
  MemberParams probe;
  if (int rc = chh::fill_params(d, s->h->precision, &probe)) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error) return fail(s->error, "server failed: " + s->error_msg);
  if (Arena::round(elems) * (probe.comp ? 2 : 1) > s->arena.capacity)
    return fail(CH_ENOMEM, "request larger than the server's HBM budget");
  if ((int64_t)s->queue.size() >= kMaxQueue) return fail(CH_EBUSY, "request queue full");
  Req q;
  q.id = s->next_id++;
  q.d = d;
  q.nsteps = r->nsteps;
  q.every = r->every > 0 ? r->every : kDefaultEvery;
  q.t1 = r->t1 >= 0.0 ? r->t1 : 0.2 * (double)r->nsteps * r->dt;
  q.field_out = r->field_out;
  q.elems = elems;
  q.comp = probe.comp != 0;
  q.t_submit = Clock::now();
  s->reqs.emplace(q.id, q);
  s->queue.push_back(q.id);
  s->submitted += 1;
  *id = q.id;
  s->cv_work.notify_one();
  return CH_OK;
}

int ch_poll(ch_server s, uint64_t id, ch_result* out) {
  using chh::fail;
  if (!s) return fail(CH_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(CH_ENOTFOUND, "unknown request id");
  if (it->second.status == CH_PENDING) return CH_PENDING;
  const int st = it->second.status;
  if (out) *out = it->second.res;
  s->reqs.erase(it);
  if (st != CH_OK) return fail(st, st == CH_ENONFINITE ? "run diverged" : "server failed: " + s->error_msg);
  return CH_OK;
}

int ch_server_wait(ch_server s, uint64_t id, double timeout_s, ch_result* out) {
  using chh::fail;
  if (!s) return fail(CH_EINVAL, "server is NULL");
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
      auto it = s->reqs.find(id);
      return it == s->reqs.end() || it->second.status != CH_PENDING;
    };
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)), ready))
      return fail(CH_ETIMEOUT, "request not finished within the timeout");
  }
  return ch_poll(s, id, out);
}

int ch_server_stats(ch_server s, ch_server_stats_t* out) {
  using chh::fail;
  if (!s || !out) return fail(CH_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->running = s->running;
  out->queued = (int64_t)s->queue.size();
  out->max_running = s->max_running;
  out->member_steps = s->member_steps;
  out->grid_point_steps = s->point_steps;
  out->chunks = s->chunks;
  out->busy_s = s->busy_s;
  out->wall_s = seconds(Clock::now() - s->t_created);
  out->arena_bytes = (size_t)s->arena.capacity * s->h->elt * 2;
  out->arena_peak_bytes = (size_t)s->arena.peak * s->h->elt * 2;
  return CH_OK;
}

void ch_server_destroy(ch_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  ch_ensemble* h = s->h;
  cudaStreamSynchronize(h->stream);
  chh::drop_graph(h);
  cudaFree(h->C);
  cudaFree(h->W);
  cudaFree(h->dmp);
  cudaFree(h->dms);
  cudaFree(h->dseg);
  cudaFree(h->dsegy);
  cudaFree(h->dcst);
  cudaFree(h->drt);
  cudaFree(h->dst);
  cudaFree(h->dct);
  cudaFree(h->dres);
  cudaFree(h->dpart);
  cudaFree(h->dobs);
  cudaFree(s->dlist);
  chh::free_aux(h);
  cudaStreamDestroy(h->own);
  delete h;
  delete s;
}

}  // extern "C"
