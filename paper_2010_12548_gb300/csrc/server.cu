// Serving loop for interactive level-of-detail exploration (Sec. 1: visual
// exploration needs interactive responses; users zoom from an overview into
// regions of interest).  Points stay resident on the device; queries arrive at
// any time and are answered with continuous batching:
//
//  * a pool of workers, each with its own CUDA stream; a free worker takes every
//    pending query (up to max_batch) as one batch, so queries that arrive while
//    other batches run on the device join the next free slot and the batches
//    overlap on the device;
//  * per query a covering (viewport-clipped, cover.cu) from the cache, or built
//    for all missing queries of the batch in one pass; the cache keeps coverings
//    in device memory under a byte budget (LRU, entries of running batches are
//    pinned), and a worker takes new work only while the coverings of running
//    batches and the cache fit the budget;
//  * the batch's join is one persistent launch (batch.cu), or one launch per
//    query in the plain form; results are copied to the query's ticket.
//
// Waiting is host-side with timeouts; no device code waits on anything.
#include "sdb_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>

namespace {

using sdb::BatchChunkDev;
using sdb::BatchCore;
using sdb::BatchQueryDev;
using sdb::CoverQuery;
using sdb::CoverSet;

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Ticket {
  uint64_t id = 0;
  sdb_query q{};
  std::vector<uint32_t> subset;
  std::vector<uint64_t> count;
  std::vector<int64_t> sum;
  double t_submit = 0, t_start = 0, t_done = 0;
  uint32_t batch_size = 0, cache_hit = 0;
  uint64_t ranges = 0;
  bool done = false;
  sdb_status status = SDB_OK;
  std::string error;
};

struct Key {
  uint32_t x0, y0, x1, y1;
  uint64_t eps, h;
  uint32_t n;
  bool operator==(const Key& o) const {
    return x0 == o.x0 && y0 == o.y0 && x1 == o.x1 && y1 == o.y1 && eps == o.eps && h == o.h &&
           n == o.n;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t v = k.h ^ (k.eps * 0x9e3779b97f4a7c15ull);
    v ^= ((uint64_t)k.x0 << 32 | k.y0) * 0xff51afd7ed558ccdull;
    v ^= ((uint64_t)k.x1 << 32 | k.y1) * 0xc4ceb9fe1a85ec53ull;
    return (size_t)(v ^ (v >> 29) ^ k.n);
  }
};

Key key_of(const sdb_query& q, const std::vector<uint32_t>& ids) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the subset
  for (uint32_t v : ids) {
    for (int b = 0; b < 4; ++b) {
      h ^= (v >> (8 * b)) & 255u;
      h *= 1099511628211ull;
    }
  }
  return Key{q.x0, q.y0, q.x1, q.y1, q.eps, h, (uint32_t)ids.size()};
}

// device arrays built together, shared by the cache entries of their queries;
// freed when the last entry or running batch lets go of them (uses are
// complete by then: a worker synchronises its stream before releasing)
struct Chunk {
  CoverSet set;
  uint64_t bytes = 0;
  ~Chunk() { set.release(0); }
};

struct Entry {
  std::shared_ptr<Chunk> chunk;
  uint64_t sbase = 0;
  uint32_t R = 0;
  uint64_t bytes = 0;
  std::vector<uint32_t> subset;
  int pins = 0;
  std::list<Key>::iterator lru;
};

uint64_t chunk_bytes(const CoverSet& c) { return c.E * 16 + c.nids * 4; }

}  // namespace

struct sdb_server {
  int device = 0;
  sdb_server_config cfg{};
  const sdb_points* pts = nullptr;
  uint32_t B = 0, P = 0;
  std::vector<uint32_t> ring_off, vx, vy, bb;
  sdb_polygons polys{};
  sdb::PolyEdges pe;  // the polygons as edge sets, converted once
  // queue and tickets
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Ticket>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Ticket>> tickets;
  uint64_t next_id = 1;
  bool stop = false;
  uint64_t inflight_bytes = 0;  // coverings built for running batches, not cached
  std::vector<std::thread> workers;
  // cache
  std::mutex cmu;
  std::unordered_map<Key, Entry, KeyHash> cache;
  std::list<Key> lru;  // front = most recent
  uint64_t cache_bytes = 0;
  sdb_server_stats st{};
};

namespace {

void evict_locked(sdb_server* S) {
  auto it = S->lru.end();
  while (S->cache_bytes > S->cfg.cache_bytes && it != S->lru.begin()) {
    --it;
    auto e = S->cache.find(*it);
    if (e->second.pins > 0) continue;
    S->cache_bytes -= e->second.bytes;
    S->st.evictions++;
    auto victim = it++;
    S->cache.erase(e);
    S->lru.erase(victim);
  }
  S->st.cache_bytes = S->cache_bytes;
  S->st.cache_entries = S->cache.size();
}

sdb_status process(sdb_server* S, std::vector<std::shared_ptr<Ticket>>& batch, cudaStream_t s,
                   uint64_t* built_bytes) {
  const uint32_t Q = (uint32_t)batch.size();
  std::vector<BatchQueryDev> hq(Q);
  std::vector<CoverQuery> cq;
  std::vector<uint32_t> pp, pq, ps, miss;
  std::vector<std::shared_ptr<Chunk>> chunks;  // index = chunk id of the batch
  std::unordered_map<Chunk*, uint32_t> chunk_id;
  std::vector<Key> keys(Q), pinned;
  uint64_t out_off = 0;
  for (uint32_t i = 0; i < Q; ++i) {
    uint32_t F = 0;
    SDB_TRY(sdb::batch_query_dev(S->B, batch[i]->q, out_off, &hq[i], &F));
    out_off += batch[i]->q.poly_cnt;
    keys[i] = key_of(batch[i]->q, batch[i]->subset);
  }
  if (S->cfg.use_cache) {
    std::lock_guard<std::mutex> lk(S->cmu);
    for (uint32_t i = 0; i < Q; ++i) {
      auto e = S->cache.find(keys[i]);
      if (e != S->cache.end() && e->second.subset == batch[i]->subset) {
        Entry& en = e->second;
        en.pins++;
        pinned.push_back(keys[i]);
        S->lru.splice(S->lru.begin(), S->lru, en.lru);
        auto c = chunk_id.find(en.chunk.get());
        uint32_t cid;
        if (c == chunk_id.end()) {
          cid = (uint32_t)chunks.size();
          chunk_id[en.chunk.get()] = cid;
          chunks.push_back(en.chunk);
        } else {
          cid = c->second;
        }
        hq[i].sbase = en.sbase;
        hq[i].R = en.R;
        hq[i].chunk = cid;
        batch[i]->cache_hit = 1;
        S->st.cache_hits++;
      } else {
        miss.push_back(i);
        S->st.cache_misses++;
      }
    }
  } else {
    for (uint32_t i = 0; i < Q; ++i) miss.push_back(i);
  }
  sdb_status rc = SDB_OK;
  if (!miss.empty()) {
    std::vector<BatchQueryDev> mq(miss.size());
    for (uint32_t m = 0; m < miss.size(); ++m) {
      const uint32_t i = miss[m];
      uint32_t F = 0;
      sdb::batch_query_dev(S->B, batch[i]->q, 0, &mq[m], &F);
      cq.push_back(CoverQuery{F, batch[i]->q.x0, batch[i]->q.y0, batch[i]->q.x1, batch[i]->q.y1});
      sdb::viewport_pairs(S->bb, m, batch[i]->q, mq[m].k, batch[i]->subset.data(), pp, pq, ps);
    }
    std::vector<CoverSet> sets;
    uint64_t nr = 0, nc = 0, mr = 0;
    rc = sdb::build_query_coverings(S->pe, S->B, cq, pp, pq, ps, mq, &sets,
                                    (uint32_t)chunks.size(), s, &nr, &nc, &mr);
    for (auto& set : sets) {
      auto c = std::make_shared<Chunk>();
      c->set = set;
      c->bytes = chunk_bytes(set);
      *built_bytes += c->bytes;
      chunks.push_back(c);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->inflight_bytes += *built_bytes;
    }
    if (rc == SDB_OK) {
      for (uint32_t m = 0; m < miss.size(); ++m) {
        const uint32_t i = miss[m];
        hq[i].sbase = mq[m].sbase;
        hq[i].R = mq[m].R;
        hq[i].chunk = mq[m].chunk;
      }
      if (S->cfg.use_cache) {
        std::lock_guard<std::mutex> lk(S->cmu);
        for (uint32_t m = 0; m < miss.size(); ++m) {
          const uint32_t i = miss[m];
          if (S->cache.count(keys[i])) continue;  // another batch cached it meanwhile
          const auto& c = chunks[mq[m].chunk];
          const uint64_t share =
              c->bytes * ((uint64_t)mq[m].R + 1) / std::max<uint64_t>(1, c->set.E);
          Entry en;
          en.chunk = c;
          en.sbase = mq[m].sbase;
          en.R = mq[m].R;
          en.bytes = share;
          en.subset = batch[i]->subset;
          en.pins = 1;
          S->lru.push_front(keys[i]);
          en.lru = S->lru.begin();
          S->cache.emplace(keys[i], std::move(en));
          S->cache_bytes += share;
          pinned.push_back(keys[i]);
        }
        S->st.peak_bytes = std::max(S->st.peak_bytes, S->cache_bytes);
        evict_locked(S);
      }
    }
  }
  for (uint32_t i = 0; i < Q; ++i) batch[i]->ranges = hq[i].R;
  if (rc == SDB_OK) {
    BatchCore core;
    core.pts = S->pts;
    core.Q = Q;
    core.out_len = out_off;
    core.hq = hq;
    for (auto& c : chunks)
      core.hchunks.push_back(BatchChunkDev{c->set.start, c->set.pay, c->set.list_off, c->set.list_ids});
    if (S->cfg.tile) core.tile = S->cfg.tile;
    if (S->cfg.points_per_thread) core.ppt = S->cfg.points_per_thread;
    uint64_t* d_cnt = nullptr;
    int64_t* d_sum = nullptr;
    rc = sdb::batch_core_prepare(&core, s);
    if (rc == SDB_OK && S->cfg.lookup == SDB_LOOKUP_LEARNED)
      rc = sdb::batch_core_index(&core, SDB_BATCH_LEARNED_MIN_RANGES, SDB_BATCH_RANGES_PER_LEAF, s);
    if (rc == SDB_OK) rc = sdb::dalloc_n(&d_cnt, out_off, s);
    if (rc == SDB_OK) rc = sdb::dalloc_n(&d_sum, out_off, s);
    if (rc == SDB_OK)
      rc = sdb::batch_core_run(&core, S->cfg.per_query ? SDB_BATCH_PER_QUERY : SDB_BATCH_PERSISTENT,
                               d_cnt, d_sum, s);
    std::vector<uint64_t> hc(out_off);
    std::vector<int64_t> hs(out_off);
    if (rc == SDB_OK && out_off) {
      cudaMemcpyAsync(hc.data(), d_cnt, out_off * 8, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hs.data(), d_sum, out_off * 8, cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc == SDB_OK && e != cudaSuccess) rc = sdb::cuda_status(e, "batch", __FILE__, __LINE__);
    sdb::dfree(d_cnt, s);
    sdb::dfree(d_sum, s);
    core.release(s);
    cudaStreamSynchronize(s);
    if (rc == SDB_OK) {
      uint64_t o = 0;
      for (auto& t : batch) {
        t->count.assign(hc.begin() + o, hc.begin() + o + t->q.poly_cnt);
        t->sum.assign(hs.begin() + o, hs.begin() + o + t->q.poly_cnt);
        o += t->q.poly_cnt;
      }
    }
  }
  if (!pinned.empty()) {
    std::lock_guard<std::mutex> lk(S->cmu);
    for (const Key& k : pinned) {
      auto e = S->cache.find(k);
      if (e != S->cache.end()) e->second.pins--;
    }
    evict_locked(S);
  }
  return rc;
}

void worker(sdb_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Ticket>> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admission: work while the running batches' coverings fit the budget
      S->cv_work.wait(lk, [&] {
        return S->stop ||
               (!S->pending.empty() && (S->inflight_bytes < S->cfg.cache_bytes ||
                                        S->inflight_bytes == 0));
      });
      if (S->pending.empty() && S->stop) break;
      if (S->pending.empty()) continue;
      while (!S->pending.empty() && batch.size() < S->cfg.max_batch) {
        batch.push_back(S->pending.front());
        S->pending.pop_front();
      }
      S->st.batches++;
    }
    const double t0 = now_ms();
    for (auto& t : batch) {
      t->t_start = t0;
      t->batch_size = (uint32_t)batch.size();
    }
    uint64_t built = 0;
    sdb_status rc = process(S, batch, s, &built);
    std::string err = rc == SDB_OK ? std::string() : std::string(sdb_last_error());
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->inflight_bytes -= built;
      const double t1 = now_ms();
      for (auto& t : batch) {
        t->t_done = t1;
        t->status = rc;
        t->error = err;
        t->done = true;
        S->st.completed++;
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaStreamDestroy(s);
}

}  // namespace

using namespace sdb;

extern "C" {

sdb_status sdb_server_create(const sdb_points* pts, const sdb_polygons* polys,
                             const sdb_server_config* cfg, sdb_server** out) {
  if (!out || !pts || !polys || !cfg || !polys->ring_off || !polys->x || !polys->y) {
    set_error("points, polygons, config and out are required");
    return SDB_EINVAL;
  }
  *out = nullptr;
  if (cfg->workers == 0 || cfg->workers > 64 || cfg->max_batch == 0) {
    set_error("need 1..64 workers and max_batch >= 1");
    return SDB_EINVAL;
  }
  if (cfg->points_per_thread && !(cfg->points_per_thread == 1 || cfg->points_per_thread == 2 ||
                                  cfg->points_per_thread == 4)) {
    set_error("points per thread must be 1, 2 or 4");
    return SDB_EINVAL;
  }
  if (cfg->lookup != SDB_LOOKUP_BINARY && cfg->lookup != SDB_LOOKUP_LEARNED) {
    set_error("server lookup must be binary search or the learned index");
    return SDB_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != pts->device) {
    set_error("points live on another device");
    return SDB_EINVAL;
  }
  sdb_server* S = new (std::nothrow) sdb_server();
  if (!S) {
    set_error("host allocation failed");
    return SDB_ENOMEM;
  }
  S->device = dev;
  S->cfg = *cfg;
  S->pts = pts;
  S->B = pts->B;
  S->P = polys->n_polygons;
  sdb_status st = polygon_bboxes(polys, S->B, &S->bb);
  if (st != SDB_OK) {
    delete S;
    return st;
  }
  const uint32_t V = polys->ring_off[S->P];
  S->ring_off.assign(polys->ring_off, polys->ring_off + S->P + 1);
  S->vx.assign(polys->x, polys->x + V);
  S->vy.assign(polys->y, polys->y + V);
  S->polys = sdb_polygons{S->P, S->ring_off.data(), S->vx.data(), S->vy.data()};
  S->pe = sdb::poly_edges(&S->polys);
  for (uint32_t w = 0; w < cfg->workers; ++w) S->workers.emplace_back(worker, S);
  *out = S;
  return SDB_OK;
}

sdb_status sdb_server_submit(sdb_server* S, const sdb_query* q, const uint32_t* subset_ids,
                             uint64_t* ticket) {
  if (!S || !q || !ticket || (q->poly_cnt && !subset_ids)) {
    set_error("server, query, ticket and subset ids are required");
    return SDB_EINVAL;
  }
  BatchQueryDev d;
  uint32_t F = 0;
  SDB_TRY(batch_query_dev(S->B, *q, 0, &d, &F));
  for (uint32_t t = 0; t < q->poly_cnt; ++t)
    if (subset_ids[t] >= S->P) {
      set_error("polygon id %u out of range", subset_ids[t]);
      return SDB_EINVAL;
    }
  auto t = std::make_shared<Ticket>();
  t->q = *q;
  t->q.poly_off = 0;
  t->subset.assign(subset_ids, subset_ids + q->poly_cnt);
  t->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      set_error("server is shutting down");
      return SDB_EBUSY;
    }
    t->id = S->next_id++;
    S->tickets[t->id] = t;
    S->pending.push_back(t);
    S->st.submitted++;
  }
  S->cv_work.notify_one();
  *ticket = t->id;
  return SDB_OK;
}

sdb_status sdb_server_wait(sdb_server* S, uint64_t ticket, uint32_t timeout_ms,
                           uint64_t* h_count, int64_t* h_sum, sdb_ticket_info* info) {
  if (!S) {
    set_error("server is NULL");
    return SDB_EINVAL;
  }
  std::shared_ptr<Ticket> t;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) {
      set_error("unknown ticket %llu", (unsigned long long)ticket);
      return SDB_EINVAL;
    }
    t = it->second;
    if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return t->done; })) {
      set_error("ticket %llu not done within %u ms", (unsigned long long)ticket, timeout_ms);
      return SDB_ETIMEOUT;
    }
    S->tickets.erase(it);
  }
  if (t->status != SDB_OK) {
    set_error("%s", t->error.c_str());
    return t->status;
  }
  if (h_count && !t->count.empty()) memcpy(h_count, t->count.data(), t->count.size() * 8);
  if (h_sum && !t->sum.empty()) memcpy(h_sum, t->sum.data(), t->sum.size() * 8);
  if (info) {
    info->latency_ms = t->t_done - t->t_submit;
    info->queue_ms = t->t_start - t->t_submit;
    info->batch_size = t->batch_size;
    info->cache_hit = t->cache_hit;
    info->ranges = t->ranges;
  }
  return SDB_OK;
}

sdb_status sdb_server_get_stats(sdb_server* S, sdb_server_stats* out) {
  if (!S || !out) {
    set_error("server or stats is NULL");
    return SDB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::lock_guard<std::mutex> lc(S->cmu);
  *out = S->st;
  out->cache_bytes = S->cache_bytes;
  out->cache_entries = S->cache.size();
  return SDB_OK;
}

void sdb_server_destroy(sdb_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;  // workers drain the queue, then leave
  }
  S->cv_work.notify_all();
  for (auto& w : S->workers) w.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> lc(S->cmu);
    S->cache.clear();  // frees the cached coverings
    S->lru.clear();
  }
  cudaStreamSynchronize(0);
  cudaSetDevice(prev);
  delete S;
}

}  // extern "C"
