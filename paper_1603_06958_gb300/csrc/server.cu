// Serving loop: a request queue in front of the library, with admission by an
// HBM budget and continuous batching.
//
// Requests are guide trees of new families (FAMSA stages I+II on that family)
// and query batches scored against a family kept resident from an earlier
// tree request (the "Pairwise similarities calculation" against the resident
// Peq tables).  Each of `slots` worker threads owns a CUDA stream; a worker
// takes the first queued request that fits the free part of the budget (and
// whose family is resident, for a query), runs it on its stream, and takes
// the next.  Requests that arrive while others run are admitted as soon as a
// slot and enough memory free up, and their kernels overlap on the device
// with the running ones.  A request's result does not depend on what runs
// beside it: each one is exactly the single-request library call.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "famsa_internal.cuh"

namespace famsa {

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int kQueued = -1, kRunning = -2;
constexpr size_t kMaxQueue = 1 << 20;
constexpr int64_t kMaxBypassNs = 1000000000;  // the oldest request waits at most ~1 s behind later ones

struct Request {
  int64_t id = 0;
  int kind = 0;  // 0 tree, 1 query
  std::vector<uint8_t> res;
  std::vector<int64_t> off;
  int32_t n = 0;          // sequences of the family, or queries
  int64_t family = -1;    // query: the tree request holding its family
  bool keep = false;      // tree: keep the packed family resident
  int64_t mem = 0;        // admission estimate while running
  int64_t resident = 0;   // bytes that stay in use while the family is resident
  int status = kQueued;
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  double cells = 0;
  famsa_family *fam = nullptr;
  int users = 0;          // queries running against this family
  bool released = false;
  std::vector<int32_t> pi, merges, sizes, qout;
  std::vector<uint64_t> lnum, hnum;
  std::vector<uint32_t> lden, hden;
};

}  // namespace

struct Server {
  int device = 0;
  int64_t budget = 0, used = 0, peak_used = 0;
  int slots = 1, running = 0, peak_running = 0;
  int64_t next_id = 0, n_done = 0, n_failed = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> workers;
};

static int64_t tree_estimate(const std::vector<int64_t> &off, int32_t k, int64_t *resident) {
  int64_t sum = 0, words = 0;
  for (int32_t i = 0; i < k; ++i) {
    const int64_t l = off[i + 1] - off[i];
    sum += l;
    words += (l + 63) / 64;
  }
  const int64_t groups = (k + 31) / 32;
  // residues, offsets, lengths/permutation, Peq planes, column layout
  *resident = sum + 8 * (int64_t)(k + 1) * 2 + 16 * (int64_t)k + words * 256 + sum + sum / 4 + 1024 * groups;
  // tree build: the row blocks of 16-bit LCS, the row-update state, the finalisation tables
  int64_t B = std::min<int64_t>(std::max<int64_t>((int64_t)(1 << 26) / std::max(k, 1), 64), 2048);
  B = std::min<int64_t>(B, std::max(k - 1, 1));
  const int64_t ld = (k + 1) & ~1ll;
  int64_t lv = 1;
  while ((1ll << lv) <= k) ++lv;
  return *resident + kRowBuffers * B * ld * 2 + (int64_t)k * 160 + (int64_t)k * (96 + 16 * lv) + (16 << 20);
}

static int64_t query_estimate(const std::vector<int64_t> &off, int32_t nq, int32_t k) {
  int64_t sum = 0, words = 0;
  for (int32_t i = 0; i < nq; ++i) {
    const int64_t l = off[i + 1] - off[i];
    sum += l;
    words += (l + 63) / 64;
  }
  return sum + words * 256 + 32 * (int64_t)nq + 4 * (int64_t)nq * k + (4 << 20);
}

// first queued request that may start now (caller holds the lock)
static Request *pick(Server *s) {
  if (s->queue.empty()) return nullptr;
  const int64_t t = now_ns();
  const bool oldest_only = t - s->queue.front()->t_submit > kMaxBypassNs;
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    Request *r = *it;
    if (r->kind == 1) {
      auto f = s->reqs.find(r->family);
      if (f == s->reqs.end() || f->second->kind != 0 ||
          (f->second->status != kQueued && f->second->status != kRunning &&
           (f->second->status != FAMSA_OK || !f->second->fam))) {
        // the family failed, was not kept, or was released: the query cannot run
        r->status = FAMSA_EINVAL;
        r->t_start = r->t_done = t;
        ++s->n_failed;
        s->queue.erase(it);
        s->cv_done.notify_all();
        return pick(s);
      }
      if (f->second->status != FAMSA_OK) {  // family still queued or running
        if (oldest_only) return nullptr;
        continue;
      }
    }
    const bool fits = s->used + r->mem <= s->budget || s->running == 0;
    if (fits) {
      s->queue.erase(it);
      return r;
    }
    if (oldest_only) return nullptr;
  }
  return nullptr;
}

static void run_request(Server *s, Request *r, cudaStream_t st) {
  TraceRange trace(r->kind == 0 ? "served tree request" : "served query request");
  int rc = FAMSA_OK;
  if (r->kind == 0) {
    famsa_family *fam = nullptr;
    rc = famsa_pack_peq(r->res.data(), r->off.data(), r->n, 0, st, &fam);
    if (rc == FAMSA_OK) {
      const size_t k = (size_t)r->n, m = k > 0 ? k - 1 : 0;
      r->pi.resize(k);
      r->lnum.resize(k);
      r->lden.resize(k);
      r->merges.resize(2 * m);
      r->hnum.resize(m);
      r->hden.resize(m);
      r->sizes.resize(m);
      rc = famsa_slink_tree(fam, r->pi.data(), r->lnum.data(), r->lden.data(), r->merges.data(),
                            r->hnum.data(), r->hden.data(), r->sizes.data(), 0, st);
    }
    if (fam) {
      if (rc == FAMSA_OK && r->keep) {
        r->fam = fam;
      } else {
        cudaStreamSynchronize(st);
        AllocStream alloc_on(st);
        free_family(reinterpret_cast<Family *>(fam));
      }
    }
  } else {
    Request *f = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      f = s->reqs[r->family].get();
    }
    r->qout.resize((size_t)r->n * (size_t)f->n);
    rc = famsa_lcs_query(f->fam, r->res.data(), r->off.data(), r->n, 0, r->qout.data(), 0, st);
  }
  r->status = rc;
}

static void release_family(Server *s, Request *f, cudaStream_t st) {
  // caller holds the lock; no query uses f
  if (!f->fam) return;
  cudaStreamSynchronize(st);
  AllocStream alloc_on(st);
  free_family(reinterpret_cast<Family *>(f->fam));
  f->fam = nullptr;
  s->used -= f->resident;
}

static void worker(Server *s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || (r = pick(s)) != nullptr; });
      if (!r) break;
      r->status = kRunning;
      r->t_start = now_ns();
      s->used += r->mem;
      s->peak_used = std::max(s->peak_used, s->used);
      ++s->running;
      s->peak_running = std::max(s->peak_running, s->running);
      if (r->kind == 1) ++s->reqs[r->family]->users;
    }
    run_request(s, r, st);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_done = now_ns();
      s->used -= r->mem;
      if (r->kind == 0 && r->fam) s->used += r->resident;
      --s->running;
      if (r->status == FAMSA_OK) ++s->n_done; else ++s->n_failed;
      if (r->kind == 1) {
        Request *f = s->reqs[r->family].get();
        if (--f->users == 0 && f->released) {
          release_family(s, f, st);
          s->reqs.erase(f->id);
        }
      }
      if (r->released) {
        if (r->kind == 0) release_family(s, r, st);
        if (r->users == 0) s->reqs.erase(r->id);
      }
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &kv : s->reqs)
      if (kv.second->fam && kv.second->users == 0) release_family(s, kv.second.get(), st);
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

static int submit(Server *s, std::unique_ptr<Request> r, int64_t *id) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return FAMSA_EINVAL;
  if (s->queue.size() >= kMaxQueue) return FAMSA_EBUSY;
  r->id = s->next_id++;
  r->t_submit = now_ns();
  *id = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_all();
  return FAMSA_OK;
}

static bool valid_family(const int64_t *off, int32_t n) {
  for (int32_t i = 0; i < n; ++i)
    if (off[i + 1] <= off[i] || off[i + 1] - off[i] > kMaxLen) return false;
  return off[0] >= 0;
}

}  // namespace famsa

using namespace famsa;

extern "C" {

int famsa_server_create(int64_t hbm_budget_bytes, int32_t slots, famsa_server **out) {
  if (!out) return FAMSA_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || slots < 1 || slots > 64) return FAMSA_EINVAL;
  auto *s = new Server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return FAMSA_ECUDA;
  }
  s->budget = hbm_budget_bytes;
  s->slots = slots;
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker, s);
  *out = reinterpret_cast<famsa_server *>(s);
  return FAMSA_OK;
}

int famsa_server_submit_tree(famsa_server *sh, const uint8_t *residues, const int64_t *offsets,
                             int32_t k, int keep_resident, int64_t *request_id) {
  if (!sh || !residues || !offsets || !request_id || k < 1) return FAMSA_EINVAL;
  if (!valid_family(offsets, k)) return FAMSA_EINVAL;
  auto r = std::make_unique<Request>();
  r->kind = 0;
  r->n = k;
  r->keep = keep_resident != 0;
  r->off.assign(offsets, offsets + k + 1);
  for (auto &o : r->off) o -= offsets[0];
  r->res.assign(residues + offsets[0], residues + offsets[k]);
  r->mem = tree_estimate(r->off, k, &r->resident);
  double tot = 0, sq = 0;
  for (int32_t i = 0; i < k; ++i) {
    const double l = (double)(r->off[i + 1] - r->off[i]);
    tot += l;
    sq += l * l;
  }
  r->cells = (tot * tot - sq) / 2;
  return submit(reinterpret_cast<Server *>(sh), std::move(r), request_id);
}

int famsa_server_submit_query(famsa_server *sh, int64_t family_request, const uint8_t *q,
                              const int64_t *q_offsets, int32_t nq, int64_t *request_id) {
  if (!sh || !q || !q_offsets || !request_id || nq < 1) return FAMSA_EINVAL;
  if (!valid_family(q_offsets, nq)) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  int32_t k = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto f = s->reqs.find(family_request);
    if (f == s->reqs.end() || f->second->kind != 0 || !f->second->keep || f->second->released)
      return FAMSA_EINVAL;
    k = f->second->n;
  }
  auto r = std::make_unique<Request>();
  r->kind = 1;
  r->n = nq;
  r->family = family_request;
  r->off.assign(q_offsets, q_offsets + nq + 1);
  for (auto &o : r->off) o -= q_offsets[0];
  r->res.assign(q + q_offsets[0], q + q_offsets[nq]);
  r->mem = query_estimate(r->off, nq, k);
  double tot = 0;
  for (int32_t i = 0; i < nq; ++i) tot += (double)(r->off[i + 1] - r->off[i]);
  r->cells = tot;  // times the family's total length, filled in when it is known
  return submit(s, std::move(r), request_id);
}

int famsa_server_wait(famsa_server *sh, int64_t request_id, int64_t timeout_ms) {
  if (!sh) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return FAMSA_EINVAL;
  Request *r = it->second.get();
  auto done = [&] { return r->status != kQueued && r->status != kRunning; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return FAMSA_ETIMEOUT;
  }
  return r->status;
}

static Request *finished(Server *s, int64_t id, int kind) {
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return nullptr;
  Request *r = it->second.get();
  if (r->kind != kind || r->status != FAMSA_OK) return nullptr;
  return r;
}

int famsa_server_tree_result(famsa_server *sh, int64_t request_id, int32_t *pi, uint64_t *lambda_num,
                             uint32_t *lambda_den, int32_t *merges, uint64_t *h_num, uint32_t *h_den,
                             int32_t *sizes) {
  if (!sh) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  Request *r = finished(s, request_id, 0);
  if (!r) return FAMSA_EINVAL;
  auto put = [](auto *dst, const auto &v) {
    if (dst && !v.empty()) std::copy(v.begin(), v.end(), dst);
  };
  put(pi, r->pi);
  put(lambda_num, r->lnum);
  put(lambda_den, r->lden);
  put(merges, r->merges);
  put(h_num, r->hnum);
  put(h_den, r->hden);
  put(sizes, r->sizes);
  return FAMSA_OK;
}

int famsa_server_query_result(famsa_server *sh, int64_t request_id, int32_t *out) {
  if (!sh || !out) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  Request *r = finished(s, request_id, 1);
  if (!r) return FAMSA_EINVAL;
  std::copy(r->qout.begin(), r->qout.end(), out);
  return FAMSA_OK;
}

int famsa_server_request_info(famsa_server *sh, int64_t request_id, int64_t *info) {
  if (!sh || !info) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return FAMSA_EINVAL;
  const Request *r = it->second.get();
  const bool done = r->status != kQueued && r->status != kRunning;
  info[0] = r->status;
  info[1] = r->kind;
  info[2] = r->n;
  info[3] = (r->status == kQueued) ? -1 : r->t_start - r->t_submit;
  info[4] = done ? r->t_done - r->t_submit : -1;
  double cells = r->cells;
  if (r->kind == 1) {
    auto f = s->reqs.find(r->family);
    double flen = 0;
    if (f != s->reqs.end())
      flen = (double)f->second->res.size();
    cells = r->cells * flen;
  }
  info[5] = (int64_t)cells;
  info[6] = r->mem;
  return FAMSA_OK;
}

int famsa_server_cancel(famsa_server *sh, int64_t request_id) {
  if (!sh) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return FAMSA_EINVAL;
  Request *r = it->second.get();
  if (r->status == kRunning) return FAMSA_EBUSY;
  if (r->status != kQueued) return FAMSA_EINVAL;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == r) {
      s->queue.erase(q);
      break;
    }
  r->status = FAMSA_ECANCELED;
  r->t_start = r->t_done = now_ns();
  s->cv_done.notify_all();
  s->cv_work.notify_all();  // queries waiting on it can now be failed
  return FAMSA_OK;
}

int famsa_server_release(famsa_server *sh, int64_t request_id) {
  if (!sh) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return FAMSA_EINVAL;
  Request *r = it->second.get();
  if (r->status == kQueued || r->status == kRunning || r->users > 0) {
    r->released = true;  // dropped when its work (and its queries') ends
    return FAMSA_OK;
  }
  if (r->fam) {
    // the family holds device memory: free it in stream order of the legacy stream,
    // which no running request uses for this family
    AllocStream alloc_on(nullptr);
    free_family(reinterpret_cast<Family *>(r->fam));
    r->fam = nullptr;
    s->used -= r->resident;
  }
  s->reqs.erase(it);
  s->cv_work.notify_all();
  return FAMSA_OK;
}

int famsa_server_stats(famsa_server *sh, int64_t *stats) {
  if (!sh || !stats) return FAMSA_EINVAL;
  Server *s = reinterpret_cast<Server *>(sh);
  std::lock_guard<std::mutex> lk(s->mu);
  stats[0] = s->next_id;
  stats[1] = s->n_done;
  stats[2] = s->n_failed;
  stats[3] = (int64_t)s->queue.size();
  stats[4] = s->running;
  stats[5] = s->peak_running;
  stats[6] = s->used;
  stats[7] = s->peak_used;
  return FAMSA_OK;
}

void famsa_server_destroy(famsa_server *sh) {
  if (!sh) return;
  Server *s = reinterpret_cast<Server *>(sh);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request *r : s->queue) {
      r->status = FAMSA_EINVAL;
      r->t_done = now_ns();
    }
    s->queue.clear();
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  for (auto &t : s->workers) t.join();
  delete s;
}

}  // extern "C"
