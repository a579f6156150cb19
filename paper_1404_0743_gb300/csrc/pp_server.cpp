// pp_server.cpp -- continuous-batching request server for midgame queries.
//
// The paper answers queries with more than 18 stones by a from-scratch
// serial retrograde solve in an asynchronous backend (Section "Open source
// and data").  Here many queries share the GPU: a worker thread keeps the
// fill tables of the admitted queries in a caller-provided device arena and
// advances every admitted query by one level per launch, so queries that
// arrive while others run join at the next level boundary and their levels
// share launches.  Admission is first come, first served, by slot and by
// memory footprint: for a query with k empty cells, its compact fill table
// (F(k) = sum over m of C(k, m) C(m, ceil(m/2)) super values, one per valid
// fill) and 2^k super values of five tables (both colours' masks for every
// subset of the empty cells, 32 bytes each).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pp_internal.h"

using namespace pp;

namespace {

// Arena footprint of a query, in 64-byte units: its compact fill table (one
// entry per fill of every level: 64 bytes, or 32-byte half entries on one
// parity class), then five tables (2^(k+1) masks of 32 bytes).
uint64_t footprint(int k, int parity) {
  return parity >= 0 ? (fills_total(k) + (2ull << k) + 1) / 2 : fills_total(k) + (1ull << k);
}

struct Request {
  uint64_t board, id;
  MidBoard mb;
  double submit_s;
};

struct Active {
  bool used = false;
  bool finishing = false;     // its root level is in flight; slot and arena free once that tick is done
  Request req;
  uint64_t at = 0, size = 0;  // arena range (super values)
  int level = 0;              // next level to compute
  double admit_s = 0;
  const LevelLists* lists = nullptr;
};

// One enqueued launch of the worker: the queries whose roots it computes.
struct Tick {
  bool live = false;
  int rc = 0;
  std::vector<int> finishing;
};

// First-fit allocator over the arena, in super values.
struct Arena {
  std::map<uint64_t, uint64_t> free;  // start -> length
  explicit Arena(uint64_t n) {
    if (n) free[0] = n;
  }
  bool alloc(uint64_t n, uint64_t* at) {
    for (auto it = free.begin(); it != free.end(); ++it)
      if (it->second >= n) {
        *at = it->first;
        uint64_t rest = it->second - n, start = it->first + n;
        free.erase(it);
        if (rest) free[start] = rest;
        return true;
      }
    return false;
  }
  void release(uint64_t at, uint64_t n) {
    auto it = free.emplace(at, n).first;
    auto nx = std::next(it);
    if (nx != free.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free.erase(nx);
    }
    if (it != free.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free.erase(it);
      }
    }
  }
  uint64_t largest() const {
    uint64_t m = 0;
    for (auto& kv : free) m = kv.second > m ? kv.second : m;
    return m;
  }
};

}  // namespace

struct pp_server {
  int device = 0;
  int max_slots = 0, max_empty = 0;
  int parity = -1;  // -1 every rotation; 0 / 1 one parity class (half tables)
  pp_super* arena_base = nullptr;
  void* owned_arena = nullptr;  // the arena when the server allocated it itself
  uint64_t arena_values = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done[2] = {nullptr, nullptr};  // end of the tick in segment buffer 0 / 1
  MidBoard* d_boards = nullptr;   // one descriptor per slot
  MidSeg* d_segs = nullptr;       // one segment per slot per tick, two buffers
  pp_super* d_out = nullptr;      // one result per slot
  MidSeg* h_segs = nullptr;       // pinned staging, two buffers
  pp_super* h_out = nullptr;      // pinned staging
  MidBoard* h_boards = nullptr;   // pinned staging of the descriptors (a slot's stays put while it is used)
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::deque<pp_result> results;  // finished, not yet polled (oldest first)
  bool stop = false;
  int error = 0;
  std::string error_text;
  pp_server_stats stats{};

  std::vector<Active> slots;
  Arena arena{0};
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
};

// The worker keeps one launch in flight while it prepares the next: the
// next tick's segments depend only on the levels, which advance
// deterministically, and the stream orders the launches.  Only what a tick
// finishes waits for it: the results are read and the slots and arena
// ranges freed after its end event, before the tick after it is built in
// the same (double-buffered) segment staging.
void pp_server::run() {
  cudaSetDevice(device);
  Tick tick[2];
  int buf = 0;  // the staging buffer of the next launch; tick[buf ^ 1] may be in flight
  while (true) {
    bool launch = false;
    std::vector<uint16_t> admitted;  // slots admitted now: one descriptor copy and five-table pass for all
    int kmax_admitted = 0;
    {
      std::unique_lock<std::mutex> lock(mu);
      // admit in arrival order while a slot and arena room are free (host
      // work only under the lock: submitters never wait on a CUDA call)
      while (!queue.empty()) {
        int slot = -1;
        for (int i = 0; i < max_slots; i++)
          if (!slots[i].used) {
            slot = i;
            break;
          }
        const Request& r = queue.front();
        const uint64_t need = footprint((int)r.mb.k, parity);
        uint64_t at = 0;
        if (slot < 0 || !arena.alloc(need, &at)) break;
        Active& a = slots[slot];
        a.used = true;
        a.finishing = false;
        a.req = r;
        a.at = at;
        a.size = need;
        a.level = (int)r.mb.k;
        a.admit_s = now();
        {
          std::lock_guard<std::mutex> g(table_mutex());
          std::string err;
          a.lists = level_lists((int)r.mb.k, (int)r.mb.mover, &err);
        }
        MidBoard mb = r.mb;
        mb.out = (uint64_t)slot;
        if (parity >= 0) {  // 32-byte units: half fill table, then the five tables
          mb.table = 2 * at;
          mb.masks = 2 * at + fills_total((int)r.mb.k);
        } else {
          mb.table = at;
          mb.masks = 2 * (at + fills_total((int)r.mb.k));  // 32-byte entries after the fill table
        }
        h_boards[slot] = mb;
        admitted.push_back((uint16_t)slot);
        kmax_admitted = std::max(kmax_admitted, (int)r.mb.k);
        queue.pop_front();
        stats.admitted++;
      }
      int active = 0, ready = 0;
      for (auto& a : slots) active += a.used, ready += a.used && !a.finishing;
      if (!ready && !tick[buf ^ 1].live) {
        if (stop) break;
        cv_work.wait(lock);
        continue;
      }
      launch = ready > 0;
      stats.max_active = active > (int)stats.max_active ? active : stats.max_active;
    }
    if (!admitted.empty()) {
      // the descriptors of the slots from the lowest to the highest admitted
      // one (the others in that range are unused or unchanged), then the
      // admitted queries' five tables in one pass
      const int lo = *std::min_element(admitted.begin(), admitted.end());
      const int hi = *std::max_element(admitted.begin(), admitted.end());
      cudaError_t ae = cudaMemcpyAsync(d_boards + lo, h_boards + lo, (size_t)(hi - lo + 1) * sizeof(MidBoard),
                                       cudaMemcpyHostToDevice, stream);
      int arc = ae ? (int)ae
                   : launch_five_tables_slots(d_boards, admitted.data(), (int)admitted.size(), kmax_admitted,
                                              arena_base, stream);
      if (arc) {
        std::lock_guard<std::mutex> lock(mu);
        if (!error) {
          error = PP_ECUDA;
          error_text = cudaGetErrorString((cudaError_t)arc);
        }
      }
    }
    if (launch) {
      // one launch: every ready query computes its current level
      MidSeg* hs = h_segs + (size_t)buf * max_slots;
      MidSeg* ds = d_segs + (size_t)buf * max_slots;
      Tick& tk = tick[buf];
      tk.finishing.clear();
      uint32_t blocks = 0;
      int nseg = 0;
      for (int i = 0; i < max_slots; i++) {
        Active& a = slots[i];
        if (!a.used || a.finishing) continue;
        MidSeg& sg = hs[nseg++];
        sg = MidSeg{};
        sg.block0 = blocks;
        sg.list = a.lists->d_entries + a.lists->offset[a.level];
        sg.ranks = a.lists->d_ranks + a.lists->ranks_at[a.level];
        sg.loff = (uint32_t)a.lists->offset[a.level];
        sg.coff = a.level < (int)a.req.mb.k ? (uint32_t)a.lists->offset[a.level + 1] : 0u;
        sg.count = a.lists->count[a.level];
        sg.board = (uint32_t)i;
        sg.level = (uint32_t)a.level;
        sg.final = a.level == 0;
        blocks += (sg.count + kBlock - 1) / kBlock;
        if (a.level == 0) {
          tk.finishing.push_back(i);
          a.finishing = true;
        } else {
          a.level--;
        }
      }
      cudaError_t e = cudaMemcpyAsync(ds, hs, nseg * sizeof(MidSeg), cudaMemcpyHostToDevice, stream);
      int rc = e ? (int)e : launch_midgame_level(d_boards, ds, nseg, blocks, arena_base, d_out, 0, stream, arena_base,
                                                 uniform_seg_blocks(hs, nseg, kBlock), parity);
      if (!rc && !tk.finishing.empty()) {
        // the roots finished by this launch, in one copy of the slots from the
        // lowest to the highest of them (the host reads a slot's value only
        // once that slot has finished, and a finished slot's value does not
        // change until it is delivered)
        const int lo = *std::min_element(tk.finishing.begin(), tk.finishing.end());
        const int hi = *std::max_element(tk.finishing.begin(), tk.finishing.end());
        rc = (int)cudaMemcpyAsync(h_out + lo, d_out + lo, (size_t)(hi - lo + 1) * sizeof(pp_super),
                                  cudaMemcpyDeviceToHost, stream);
      }
      if (!rc) rc = (int)cudaEventRecord(done[buf], stream);
      tk.rc = rc;
      tk.live = true;
      std::lock_guard<std::mutex> lock(mu);
      stats.launches++;
      if (rc && !error) {
        error = PP_ECUDA;
        error_text = cudaGetErrorString((cudaError_t)rc);
      }
    }
    // the tick before: wait for its end, deliver its roots, free their room
    Tick& prev = tick[buf ^ 1];
    if (prev.live) {
      int rc = prev.rc;
      if (!rc) rc = (int)cudaEventSynchronize(done[buf ^ 1]);
      std::lock_guard<std::mutex> lock(mu);
      if (rc && !error) {
        error = PP_ECUDA;
        error_text = cudaGetErrorString((cudaError_t)rc);
      }
      const double t = now();
      for (int i : prev.finishing) {
        Active& a = slots[i];
        pp_result res{};
        res.req_id = a.req.id;
        res.status = rc ? PP_ECUDA : PP_OK;
        res.empty = (int32_t)a.req.mb.k;
        res.submit_s = a.req.submit_s;
        res.admit_s = a.admit_s;
        res.done_s = t;
        res.value = h_out[i];
        results.push_back(res);
        arena.release(a.at, a.size);
        a.used = false;
        a.finishing = false;
        stats.completed++;
      }
      prev.live = false;
      prev.finishing.clear();
    }
    if (launch) buf ^= 1;
    cv_done.notify_all();
  }
}

extern "C" {

int pp_server_create(void* d_arena, size_t arena_bytes, int max_slots, int max_empty, pp_server** out) {
  return pp_server_create_parity(d_arena, arena_bytes, max_slots, max_empty, -1, out);
}

int pp_server_create_budget(size_t mem_budget, int max_slots, int max_empty, pp_server** out) {
  if (!out) return report_error(PP_EINVAL, "null server pointer");
  *out = nullptr;
  const size_t bytes = mem_budget & ~(size_t)63;
  if (bytes == 0) return report_error(PP_EINVAL, "memory budget below one super value");
  if (!tables_ready()) return report_error(PP_ENOTINIT, "pp_init has not run");
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, bytes);
  if (e) {
    cudaGetLastError();
    return report_error(e == cudaErrorMemoryAllocation ? PP_ENOMEM : PP_ECUDA, cudaGetErrorString(e));
  }
  int rc = pp_server_create_parity(arena, bytes, max_slots, max_empty, -1, out);
  if (rc) {
    cudaFree(arena);
    return rc;
  }
  (*out)->owned_arena = arena;
  return PP_OK;
}

int pp_server_create_parity(void* d_arena, size_t arena_bytes, int max_slots, int max_empty, int parity,
                            pp_server** out) {
  if (!out) return report_error(PP_EINVAL, "null server pointer");
  *out = nullptr;
  if (parity < -1 || parity > 1) return report_error(PP_EINVAL, "parity must be -1, 0 or 1");
  if (!tables_ready()) return report_error(PP_ENOTINIT, "pp_init has not run");
  if (!d_arena || ((uintptr_t)d_arena & 31)) return report_error(PP_EINVAL, "arena must be 32-byte aligned");
  if (max_slots < 1 || max_slots > 4096) return report_error(PP_EINVAL, "max_slots must be 1..4096");
  if (max_empty < 0 || max_empty > kMaxEmpty) return report_error(PP_EINVAL, "max_empty must be 0..16");
  auto* S = new pp_server;
  S->parity = parity;
  S->max_slots = max_slots;
  S->max_empty = max_empty;
  S->arena_base = (pp_super*)d_arena;
  S->arena_values = arena_bytes / sizeof(pp_super);
  S->arena = Arena(S->arena_values);
  S->slots.resize(max_slots);
  S->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&S->device);
  if (!e) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&S->done[0], cudaEventBlockingSync | cudaEventDisableTiming);
  if (!e) e = cudaEventCreateWithFlags(&S->done[1], cudaEventBlockingSync | cudaEventDisableTiming);
  if (!e) e = cudaMalloc(&S->d_boards, max_slots * sizeof(MidBoard));
  if (!e) e = cudaMalloc(&S->d_segs, 2 * max_slots * sizeof(MidSeg));
  if (!e) e = cudaMalloc(&S->d_out, max_slots * sizeof(pp_super));
  if (!e) e = cudaMallocHost(&S->h_segs, 2 * max_slots * sizeof(MidSeg));
  if (!e) e = cudaMallocHost(&S->h_out, max_slots * sizeof(pp_super));
  if (!e) e = cudaMallocHost(&S->h_boards, max_slots * sizeof(MidBoard));
  if (e) {
    pp_server_destroy(S);
    return report_error(PP_ECUDA, cudaGetErrorString(e));
  }
  // fill lists for every admissible size, both movers (built once)
  for (int k = 0; k <= max_empty; k++)
    for (int mover = 1; mover <= 2; mover++) {
      std::lock_guard<std::mutex> g(table_mutex());
      std::string err;
      if (!level_lists(k, mover, &err)) {
        pp_server_destroy(S);
        return report_error(PP_ECUDA, err.c_str());
      }
    }
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return PP_OK;
}

int pp_server_submit(pp_server* S, uint64_t board, uint64_t req_id) {
  if (!S) return report_error(PP_EINVAL, "null server");
  Request r{};
  r.board = board;
  r.id = req_id;
  int rc = validate_midgame_board(board, S->max_empty, &r.mb, 0);
  if (rc) return rc;
  const uint64_t need = footprint((int)r.mb.k, S->parity);
  if (need > S->arena_values) return report_error(PP_ENOMEM, "query footprint exceeds the whole arena");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->error) return report_error(S->error, S->error_text.c_str());
    r.submit_s = S->now();
    S->queue.push_back(r);
    S->stats.submitted++;
  }
  S->cv_work.notify_one();
  return PP_OK;
}

int pp_server_poll(pp_server* S, pp_result* out, int max) {
  if (!S || (max > 0 && !out)) return -report_error(PP_EINVAL, "bad poll arguments");
  std::lock_guard<std::mutex> lock(S->mu);
  const int n = (int)std::min<size_t>(max > 0 ? (size_t)max : 0, S->results.size());
  std::copy(S->results.begin(), S->results.begin() + n, out);
  S->results.erase(S->results.begin(), S->results.begin() + n);
  return n;
}

int pp_server_wait(pp_server* S, int count, double timeout_s) {
  if (!S) return -report_error(PP_EINVAL, "null server");
  std::unique_lock<std::mutex> lock(S->mu);
  S->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                      [&] { return (int)S->results.size() >= count || S->error; });
  if (S->error) return -report_error(S->error, S->error_text.c_str());
  return (int)S->results.size();
}

int pp_server_get_stats(pp_server* S, pp_server_stats* out) {
  if (!S || !out) return report_error(PP_EINVAL, "bad stats arguments");
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  out->queued = S->queue.size();
  out->arena_free_largest = S->arena.largest() * sizeof(pp_super);
  return PP_OK;
}

void pp_server_destroy(pp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
    S->queue.clear();  // queued but never admitted requests are dropped
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->stream) cudaStreamSynchronize(S->stream);
  cudaFree(S->d_boards);
  cudaFree(S->d_segs);
  cudaFree(S->d_out);
  if (S->h_segs) cudaFreeHost(S->h_segs);
  if (S->h_out) cudaFreeHost(S->h_out);
  if (S->h_boards) cudaFreeHost(S->h_boards);
  if (S->owned_arena) cudaFree(S->owned_arena);
  for (cudaEvent_t ev : S->done)
    if (ev) cudaEventDestroy(ev);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
