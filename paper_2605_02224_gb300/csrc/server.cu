// Serving loop: continuous batching of k-NN requests over resident clouds.
//
// A scheduler thread owns a device staging arena (the memory budget) and
// a few launch slots, each a stream. Whenever a slot is free it packs the
// pending requests, oldest first, into one launch while they fit in the
// arena's largest free block: per request its queries are copied in,
// locality-sorted, and served by the persistent kernel (one launch for the
// whole pack, each request with its own cloud, k and m); results are copied
// back on the same stream and an event marks completion. Packs run
// concurrently on different slots, so requests arriving while others are
// on the device are admitted as soon as a slot and memory free up. The
// same thread reaps finished slots, stamps each request's completion time
// and returns its memory to the arena.
//
// Host buffers: pinned caller buffers are copied directly; pageable ones go
// through a pinned staging arena of the same size (copied on the host
// before the upload and after completion).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mknn.h"
#include "batch.h"
#include "cloud.h"
#include "knn_kernels.h"

using namespace mknn;

namespace {

using Clock = std::chrono::steady_clock;

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

mknn_status sfail(mknn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

// First-fit allocator over [0, size) with coalescing.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
  }
  size_t largest() const {
    size_t b = 0;
    for (auto& kv : free_) b = std::max(b, kv.second);
    return b;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
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

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

struct ReqRec {
  mknn_request r;
  Clock::time_point t_submit, t_done;
  int32_t state = 0;  // 0 pending, 1 done, <0 failed
  bool q_pinned = false, out_pinned = false;
  // placement inside the pack's region (device and pinned staging)
  size_t q_off = 0, cell_off = 0, perm_off = 0, idx_off = 0, d2_off = 0;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaStream_t aux = nullptr;    // second branch for packs with both kernel families
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t done = nullptr;
  // phase marks of the current launch (timing events): start, after the
  // host-to-device copies, after the kernels; `done` follows the copies back
  cudaEvent_t t0 = nullptr, t_h2d = nullptr, t_kern = nullptr;
  bool busy = false;
  std::vector<uint64_t> tickets;
  size_t off = 0, bytes = 0;
};

bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

size_t request_bytes(int64_t nq, int k) {
  return al((size_t)nq * 12) + 2 * al((size_t)nq * 4) + 2 * al((size_t)nq * k * 4) +
         sizeof(ReqDev);
}

// Room for the work items of a pack: at most one item per query and one
// partial item per request (items may be as small as one query).
size_t items_bytes(int64_t nq_total, size_t nreq) {
  return al(sizeof(Item) * ((size_t)nq_total + 2 * nreq + 64));
}

// Room for a pack's hand-over: the lists' header and a (request, query)
// pair per query (one-lane items on clouds with box trees).
size_t handover_bytes(int64_t nq_total) {
  return al(sizeof(Handover)) + al(sizeof(int2) * (size_t)nq_total);
}

constexpr size_t kPackFixed = kSortHistBytes + 1024;  // histogram, tile totals, counter

}  // namespace

struct mknn_server {
  int device = -1;
  mknn_server_opts o{};
  std::vector<mknn_cloud*> clouds;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<ReqRec> recs;  // index = ticket - 1
  std::deque<uint64_t> pending;
  uint64_t next_ticket = 1;
  std::vector<Slot> slots;
  Arena arena;
  char* d_arena = nullptr;
  char* h_arena = nullptr;  // pinned mirror for pageable caller buffers
  size_t arena_bytes = 0;
  bool stop = false;
  std::thread th;
  int64_t inflight = 0;
  // statistics
  int64_t completed = 0, failed = 0, queries = 0, launches = 0, packed = 0;
  double h2d_ms = 0, kernel_ms = 0, d2h_ms = 0;  // summed over completed launches
  bool have_first = false;
  Clock::time_point t_first, t_last;
  std::vector<std::pair<uint64_t, double>> lat;  // (ticket, ms)

  void run();
  void reap_locked();
  void launch(Slot& sl, std::vector<uint64_t>& tickets, size_t off, size_t bytes);
};

void mknn_server::reap_locked() {
  for (Slot& sl : slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    const Clock::time_point now = Clock::now();
    for (uint64_t t : sl.tickets) {
      ReqRec& R = recs[t - 1];
      if (e == cudaSuccess) {
        if (!R.out_pinned) {
          const size_t nk = (size_t)R.r.nq * R.r.k * 4;
          std::memcpy(R.r.out_idx, h_arena + sl.off + R.idx_off, nk);
          std::memcpy(R.r.out_d2, h_arena + sl.off + R.d2_off, nk);
        }
        R.state = 1;
        ++completed;
        queries += R.r.nq;
      } else {
        R.state = -(int32_t)MKNN_ECUDA;
        ++failed;
      }
      R.t_done = Clock::now();
      t_last = R.t_done;
      lat.emplace_back(t, std::chrono::duration<double, std::milli>(R.t_done - R.t_submit).count());
      (void)now;
    }
    if (e == cudaSuccess) {
      float a = 0, b = 0, c = 0;
      if (cudaEventElapsedTime(&a, sl.t0, sl.t_h2d) == cudaSuccess &&
          cudaEventElapsedTime(&b, sl.t_h2d, sl.t_kern) == cudaSuccess &&
          cudaEventElapsedTime(&c, sl.t_kern, sl.done) == cudaSuccess) {
        h2d_ms += a;
        kernel_ms += b;
        d2h_ms += c;
      } else {
        cudaGetLastError();
      }
    }
    if (e != cudaSuccess) cudaGetLastError();
    arena.release(sl.off, sl.bytes);
    sl.busy = false;
    sl.tickets.clear();
    --inflight;
  }
  cv_done.notify_all();
}

// Issues one pack on a slot (called without the lock held).
void mknn_server::launch(Slot& sl, std::vector<uint64_t>& tickets, size_t off, size_t bytes) {
  cudaStream_t s = sl.s;
  char* dbase = d_arena + off;
  char* hbase = h_arena + off;
  cudaError_t e = cudaEventRecord(sl.t0, s);
  if (o.plain) {
    // baseline: the request alone through the plain entry point
    ReqRec& R = recs[tickets[0] - 1];
    const mknn_request& q = R.r;
    const size_t qb = (size_t)q.nq * 12, nk = (size_t)q.nq * q.k * 4;
    const void* src = q.q;
    if (!R.q_pinned) {
      std::memcpy(hbase + R.q_off, q.q, qb);
      src = hbase + R.q_off;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbase + R.q_off, src, qb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.t_h2d, s);
    mknn_knn_opts ko{};
    ko.lanes = o.lanes;
    ko.workspace = dbase + R.cell_off;
    ko.workspace_bytes = al((size_t)q.nq * 4) * 2 + kSortHistBytes;
    if (e == cudaSuccess &&
        mknn_knn_ex(clouds[q.cloud], (const float*)(dbase + R.q_off), q.nq, 3, q.k, nullptr, q.m,
                    (int32_t*)(dbase + R.idx_off), (float*)(dbase + R.d2_off), &ko,
                    (mknn_stream_t)s) != MKNN_OK)
      e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaEventRecord(sl.t_kern, s);
    void* di = R.out_pinned ? (void*)q.out_idx : (void*)(hbase + R.idx_off);
    void* dd = R.out_pinned ? (void*)q.out_d2 : (void*)(hbase + R.d2_off);
    if (e == cudaSuccess) e = cudaMemcpyAsync(di, dbase + R.idx_off, nk, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dbase + R.d2_off, nk, cudaMemcpyDeviceToHost, s);
  } else {
    // pack layout: [counter][histogram][ReqDev x n][Item x m][hand-over][per request data]
    int* d_next = (int*)dbase;
    void* d_hist = dbase + 256;
    const size_t reqs_off = 256 + kSortHistBytes;
    const int nreq = (int)tickets.size();
    std::vector<ReqDev> rd(nreq);
    std::vector<Item> items;
    std::vector<int> req_k(nreq);
    int64_t pack_nq = 0;  // the pack runs as one launch per variant: its size sets the lanes
    for (int i = 0; i < nreq; ++i) pack_nq += recs[tickets[i] - 1].r.nq;
    std::vector<int> lanes(nreq), placement(nreq);
    for (int i = 0; i < nreq; ++i) {
      const mknn_request& q = recs[tickets[i] - 1].r;
      const mknn_cloud* c = clouds[q.cloud];
      const Mode chosen = choose_mode(q.k, c->n, c->hub_bucket(), pack_nq, c->d_hub_of != nullptr);
      lanes[i] = o.lanes ? o.lanes : chosen.lanes;
      placement[i] = o.lanes ? default_placement(q.k, lanes[i]) : chosen.placement;
    }
    const size_t ho_off = reqs_off + al(sizeof(ReqDev) * nreq) + items_bytes(pack_nq, nreq);
    Handover* d_ho = (Handover*)(dbase + ho_off);
    int2* d_pairs = (int2*)(dbase + ho_off + al(sizeof(Handover)));
    int64_t ho_cap[3] = {0, 0, 0};
    for (int i = 0; i < nreq; ++i) {
      ReqRec& R = recs[tickets[i] - 1];
      const mknn_request& q = R.r;
      const mknn_cloud* c = clouds[q.cloud];
      const CloudDevHost cd = c->dev();
      const size_t qb = (size_t)q.nq * 12;
      const void* src = q.q;
      if (!R.q_pinned) {
        std::memcpy(hbase + R.q_off, q.q, qb);
        src = hbase + R.q_off;
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(dbase + R.q_off, src, qb, cudaMemcpyHostToDevice, s);
      const bool sorted = q.nq >= kSortMinQueries;
      rd[i] = ReqDev{(const float4*)cd.pts, cd.rows, cd.succ, cd.n, 3,
                     (const float*)(dbase + R.q_off), nullptr,
                     sorted ? (const int32_t*)(dbase + R.perm_off) : nullptr,
                     (int32_t*)(dbase + R.idx_off), (float*)(dbase + R.d2_off), c->d_err, q.k,
                     q.m ? q.m : (int32_t)c->n, (const float4*)cd.ent, cd.hub_of,
                     (const int4*)cd.hub_desc, (const float4*)cd.hub_ent,
                     (const float4*)cd.hub_node};
      const int v =
          with_trees(variant_index(lanes[i], q.k, placement[i]), cd.hub_of != nullptr, true);
      if (v == kHandoverVariant || v == kHandoverVariant128) {
        ho_cap[handover_class(q.k)] += q.nq;
        rd[i].ho = d_ho;
      }
      const int per = item_queries(lanes[i], kItemRounds);
      req_k[i] = q.k;
      for (int64_t b0 = 0; b0 < q.nq; b0 += per)
        items.push_back(Item{i, (int32_t)b0, (int32_t)std::min<int64_t>(q.nq, b0 + per), v});
    }
    const std::vector<Segment> segs = make_segments(items, 0, req_k);
    const size_t ni = items.size();
    const size_t items_off = reqs_off + al(sizeof(ReqDev) * nreq);
    // request table and items go through the pinned mirror
    std::memcpy(hbase + reqs_off, rd.data(), sizeof(ReqDev) * nreq);
    std::memcpy(hbase + items_off, items.data(), sizeof(Item) * ni);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dbase + reqs_off, hbase + reqs_off,
                          items_off - reqs_off + sizeof(Item) * ni, cudaMemcpyHostToDevice, s);
    const bool handover = ho_cap[0] + ho_cap[1] + ho_cap[2] > 0;
    if (handover) {  // the lists' header, counters at zero, through the pinned mirror
      Handover h{};
      int64_t at = 0;
      for (int c = 0; c < 3; ++c) {
        h.list[c] = d_pairs + at;
        at += ho_cap[c];
      }
      std::memcpy(hbase + ho_off, &h, sizeof(h));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ho, hbase + ho_off, sizeof(h), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.t_h2d, s);
    // the locality sort of each request, then the pack's kernels
    for (int i = 0; i < nreq && e == cudaSuccess; ++i) {
      const ReqRec& R = recs[tickets[i] - 1];
      if (R.r.nq >= kSortMinQueries)
        e = launch_query_sort_split(clouds[R.r.cloud]->dev(), (const float*)(dbase + R.q_off), 3,
                                    R.r.nq, d_hist, (int32_t*)(dbase + R.cell_off),
                                    (int32_t*)(dbase + R.perm_off), s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, segs.size() * sizeof(int), s);
    // the one-lane kernel on the slot's stream, the group kernels on its
    // second stream, joined before the copies back
    if (e == cudaSuccess)
      e = launch_segments((const ReqDev*)(dbase + reqs_off), (const Item*)(dbase + items_off),
                          d_next, segs, s, sl.aux, sl.fork, sl.join, pack_nq);
    // the handed-over queries, after every segment
    for (int c = 0; c < 3 && handover && e == cudaSuccess; ++c)
      if (ho_cap[c] > 0)
        e = launch_handover((const ReqDev*)(dbase + reqs_off), d_ho, c, handover_grid(c), s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.t_kern, s);
    for (int i = 0; i < nreq && e == cudaSuccess; ++i) {
      ReqRec& R = recs[tickets[i] - 1];
      const size_t nk = (size_t)R.r.nq * R.r.k * 4;
      void* di = R.out_pinned ? (void*)R.r.out_idx : (void*)(hbase + R.idx_off);
      void* dd = R.out_pinned ? (void*)R.r.out_d2 : (void*)(hbase + R.d2_off);
      e = cudaMemcpyAsync(di, dbase + R.idx_off, nk, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dbase + R.d2_off, nk, cudaMemcpyDeviceToHost, s);
    }
  }
  cudaEventRecord(sl.done, s);
  (void)bytes;
}

void mknn_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    if (inflight > 0)
      cv.wait_for(lk, std::chrono::microseconds(50));
    else
      cv.wait(lk, [&] { return stop || !pending.empty(); });
    reap_locked();
    if (stop && pending.empty() && inflight == 0) break;
    if (pending.empty()) continue;
    Slot* free_slot = nullptr;
    for (Slot& sl : slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) continue;
    // pack the oldest pending requests that fit
    const size_t room = arena.largest();
    size_t bytes = o.plain ? 0 : al(kPackFixed);
    int64_t nq_total = 0;
    std::vector<uint64_t> take;
    size_t cursor = o.plain ? 0 : 256 + kSortHistBytes;
    std::vector<size_t> local;
    for (uint64_t t : pending) {
      const ReqRec& R = recs[t - 1];
      const size_t rb = request_bytes(R.r.nq, R.r.k);
      const size_t meta = o.plain ? 0 : al(sizeof(ReqDev) * (take.size() + 1)) +
                                            items_bytes(nq_total + R.r.nq, take.size() + 1) +
                                            handover_bytes(nq_total + R.r.nq);
      if (!take.empty() && (bytes + rb + meta > room || nq_total + R.r.nq > o.max_batch_queries))
        break;
      if (take.empty() && bytes + rb + meta > room) break;  // wait for memory
      take.push_back(t);
      bytes += rb;
      nq_total += R.r.nq;
      if (o.plain) break;
    }
    if (take.empty()) continue;
    const size_t meta = o.plain ? kSortHistBytes + 256
                                : al(sizeof(ReqDev) * take.size()) +
                                      items_bytes(nq_total, take.size()) + handover_bytes(nq_total);
    bytes += meta;
    size_t off = 0;
    if (!arena.alloc(bytes, &off)) continue;
    for (size_t i = 0; i < take.size(); ++i) pending.pop_front();
    // place each request's arrays inside the region
    if (o.plain) {
      ReqRec& R = recs[take[0] - 1];
      const int64_t nq = R.r.nq;
      R.cell_off = 0;  // sort workspace: [hist | cells | perm] at the start
      size_t c = kSortHistBytes + 2 * al((size_t)nq * 4) + 256;
      R.q_off = c;
      c += al((size_t)nq * 12);
      R.idx_off = c;
      c += al((size_t)nq * R.r.k * 4);
      R.d2_off = c;
    } else {
      size_t c = 256 + kSortHistBytes + al(sizeof(ReqDev) * take.size()) +
                 items_bytes(nq_total, take.size()) + handover_bytes(nq_total);
      for (uint64_t t : take) {
        ReqRec& R = recs[t - 1];
        const int64_t nq = R.r.nq;
        R.q_off = c;
        c += al((size_t)nq * 12);
        R.cell_off = c;
        c += al((size_t)nq * 4);
        R.perm_off = c;
        c += al((size_t)nq * 4);
        R.idx_off = c;
        c += al((size_t)nq * R.r.k * 4);
        R.d2_off = c;
        c += al((size_t)nq * R.r.k * 4);
      }
    }
    free_slot->busy = true;
    free_slot->tickets = take;
    free_slot->off = off;
    free_slot->bytes = bytes;
    ++inflight;
    ++launches;
    packed += (int64_t)take.size();
    lk.unlock();
    launch(*free_slot, free_slot->tickets, off, bytes);
    lk.lock();
  }
}

extern "C" {

mknn_status mknn_server_create(const mknn_server_opts* opts, mknn_server** out) {
  if (!out) return sfail(MKNN_EINVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<mknn_server> s(new mknn_server());
  if (opts) s->o = *opts;
  if (s->o.slots <= 0) s->o.slots = 3;
  if (s->o.plain) s->o.slots = 1;
  if (s->o.mem_budget == 0) s->o.mem_budget = (size_t)3 << 30;
  if (s->o.max_batch_queries <= 0) s->o.max_batch_queries = (int64_t)1 << 17;
  if (s->o.lanes && variant_index(s->o.lanes, 1, default_placement(1, s->o.lanes)) < 0)
    return sfail(MKNN_EINVAL, "bad lanes");
  cudaGetDevice(&s->device);
  s->arena_bytes = al(s->o.mem_budget);
  cudaError_t e = cudaMalloc((void**)&s->d_arena, s->arena_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(MKNN_ENOMEM, "device staging arena allocation failed");
  }
  e = cudaMallocHost((void**)&s->h_arena, s->arena_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->d_arena);
    return sfail(MKNN_ENOMEM, "pinned staging arena allocation failed");
  }
  s->arena.init(s->arena_bytes);
  s->slots.resize(s->o.slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sl.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&sl.done) != cudaSuccess || cudaEventCreate(&sl.t0) != cudaSuccess ||
        cudaEventCreate(&sl.t_h2d) != cudaSuccess || cudaEventCreate(&sl.t_kern) != cudaSuccess) {
      cudaGetLastError();
      return sfail(MKNN_ECUDA, "stream/event creation failed");
    }
  }
  mknn_server* raw = s.get();
  s->th = std::thread([raw] { raw->run(); });
  *out = s.release();
  return MKNN_OK;
}

mknn_status mknn_server_add_cloud(mknn_server* s, mknn_cloud* c, int32_t* id) {
  if (!s || !c || !id) return sfail(MKNN_EINVAL, "NULL argument");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != s->device) return sfail(MKNN_EINVAL, "current device differs from the server's");
  mknn_status st = mknn_cloud_upload(c, nullptr);
  if (st != MKNN_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  c->holders++;
  s->clouds.push_back(c);
  *id = (int32_t)s->clouds.size() - 1;
  return MKNN_OK;
}

mknn_status mknn_server_submit(mknn_server* s, const mknn_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return sfail(MKNN_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (r->cloud < 0 || r->cloud >= (int32_t)s->clouds.size())
    return sfail(MKNN_EINVAL, "unknown cloud id");
  const mknn_cloud* c = s->clouds[r->cloud];
  if (r->nq < 1 || r->nq >= kRequestQueryLimit || r->k < 1 || r->k > MKNN_MAX_K ||
      r->m < 0 || r->m > c->n || !r->q || !r->out_idx || !r->out_d2)
    return sfail(MKNN_EINVAL, "bad request (nq, k, m or NULL buffer)");
  const size_t need = request_bytes(r->nq, r->k) + al(kPackFixed) + 4096 + items_bytes(r->nq, 1);
  if (need > s->arena_bytes)
    return sfail(MKNN_ENOMEM, "request alone exceeds the server's memory budget");
  lk.unlock();
  const bool qp = is_pinned(r->q);
  const bool op = is_pinned(r->out_idx) && is_pinned(r->out_d2);
  lk.lock();
  ReqRec R;
  R.r = *r;
  R.q_pinned = qp;
  R.out_pinned = op;
  R.t_submit = Clock::now();
  if (!s->have_first) {
    s->have_first = true;
    s->t_first = R.t_submit;
  }
  const uint64_t t = s->next_ticket++;
  s->recs.push_back(R);
  s->pending.push_back(t);
  *ticket = t;
  lk.unlock();
  s->cv.notify_one();
  return MKNN_OK;
}

mknn_status mknn_server_poll(mknn_server* s, uint64_t ticket, int32_t* state) {
  if (!s || !state) return sfail(MKNN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 1 || ticket >= s->next_ticket) return sfail(MKNN_EINVAL, "unknown ticket");
  *state = s->recs[ticket - 1].state;
  return MKNN_OK;
}

mknn_status mknn_server_drain(mknn_server* s, double timeout_s) {
  if (!s) return sfail(MKNN_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(std::max(0.0, timeout_s)));
  const bool ok = s->cv_done.wait_until(lk, deadline, [&] {
    return s->pending.empty() && s->inflight == 0;
  });
  return ok ? MKNN_OK : sfail(MKNN_ETIMEOUT, "drain timed out with requests outstanding");
}

mknn_status mknn_server_stats(mknn_server* s, mknn_serving_stats* out) {
  if (!s || !out) return sfail(MKNN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  mknn_serving_stats st{};
  st.submitted = (int64_t)s->next_ticket - 1;
  st.completed = s->completed;
  st.failed = s->failed;
  st.queries = s->queries;
  st.launches = s->launches;
  st.mean_requests_per_launch = s->launches ? (double)s->packed / s->launches : 0.0;
  st.h2d_ms = s->h2d_ms;
  st.kernel_ms = s->kernel_ms;
  st.d2h_ms = s->d2h_ms;
  if (s->have_first && s->completed > 0)
    st.elapsed_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
  st.qps = st.elapsed_s > 0 ? (double)s->queries / st.elapsed_s : 0.0;
  std::vector<double> v;
  v.reserve(s->lat.size());
  for (auto& p : s->lat) v.push_back(p.second);
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const double idx = p * (double)(v.size() - 1);
      const size_t lo = (size_t)idx;
      const size_t hi = std::min(v.size() - 1, lo + 1);
      return v[lo] + (v[hi] - v[lo]) * (idx - (double)lo);
    };
    st.p50_ms = pct(0.50);
    st.p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    st.mean_ms = sum / (double)v.size();
    st.max_ms = v.back();
  }
  *out = st;
  return MKNN_OK;
}

mknn_status mknn_server_latencies(mknn_server* s, double* ms, int64_t cap, int64_t* count) {
  if (!s || !count || (cap > 0 && !ms)) return sfail(MKNN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<std::pair<uint64_t, double>> v = s->lat;
  std::sort(v.begin(), v.end());
  const int64_t n = std::min<int64_t>(cap, (int64_t)v.size());
  for (int64_t i = 0; i < n; ++i) ms[i] = v[i].second;
  *count = n;
  return MKNN_OK;
}

mknn_status mknn_server_reset_stats(mknn_server* s) {
  if (!s) return sfail(MKNN_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->completed = s->failed = s->queries = s->launches = s->packed = 0;
  s->h2d_ms = s->kernel_ms = s->d2h_ms = 0;
  s->have_first = false;
  s->lat.clear();
  return MKNN_OK;
}

mknn_status mknn_server_destroy(mknn_server* s, double timeout_s) {
  if (!s) return MKNN_OK;
  mknn_status st = mknn_server_drain(s, timeout_s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending.clear();
  }
  s->cv.notify_all();
  // the thread exits once nothing is in flight; in-flight work always
  // completes (kernels have no unbounded waits)
  s->th.join();
  for (Slot& sl : s->slots) {
    cudaStreamSynchronize(sl.s);
    cudaStreamSynchronize(sl.aux);
    cudaEventDestroy(sl.done);
    cudaEventDestroy(sl.fork);
    cudaEventDestroy(sl.join);
    cudaEventDestroy(sl.t0);
    cudaEventDestroy(sl.t_h2d);
    cudaEventDestroy(sl.t_kern);
    cudaStreamDestroy(sl.s);
    cudaStreamDestroy(sl.aux);
  }
  for (mknn_cloud* c : s->clouds) c->holders--;
  cudaFree(s->d_arena);
  cudaFreeHost(s->h_arena);
  delete s;
  return st;
}

}  // extern "C"
