// pp_api.cpp -- the C ABI: validation, descriptors and launch sequencing.
//
// Every step of the retrograde path runs in the kernels of pp_kernels.cu;
// this file checks inputs on the host, lays out descriptors and orders the
// launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pp_internal.h"

namespace pp {
namespace {

thread_local std::string g_error;
std::mutex g_mutex;
std::atomic<bool> g_ready{false};  // read without the lock by every entry point
DeviceTables g_dev{};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

int cuda_fail(int e, const char* what) {
  return fail(PP_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// value arrays of the section and line kernels are accessed 256 bits at a time
bool aligned32(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 31) == 0; }

// Colour-subset five tables per board: 2 colours x 2^max_empty masks of 32 bytes.
constexpr size_t kMaskBytes = 32;
size_t mask_entries_per_board(int max_empty) { return (size_t)2 << max_empty; }

uint64_t pow3u(int e);
// Workspace of a plan, per board at most: the compact fill table (one entry
// per fill of every level: 64 bytes, or 32-byte half entries for a plan on
// one parity class), then the five tables.
size_t fill_entry_bytes(int parity) { return parity >= 0 ? sizeof(pp_super) / 2 : sizeof(pp_super); }
size_t plan_bytes_per_board(int max_empty, int parity = -1) {
  return (size_t)fills_total(max_empty) * fill_entry_bytes(parity) + mask_entries_per_board(max_empty) * kMaskBytes;
}

uint64_t pow3u(int e) {
  uint64_t p = 1;
  while (e-- > 0) p *= 3;
  return p;
}

// Host check of a board as given (g = 0): five in a row for a colour.
// The 32 five-cell lines of the board as masks over cells 6R + C.
const std::array<uint64_t, 32>& five_lines() {
  static const std::array<uint64_t, 32> lines = [] {
    std::array<uint64_t, 32> l{};
    const int dir[4][2] = {{0, 1}, {1, 0}, {1, 1}, {1, -1}};
    int n = 0;
    for (int R = 0; R < 6; R++)
      for (int C = 0; C < 6; C++)
        for (auto& d : dir) {
          const int R4 = R + 4 * d[0], C4 = C + 4 * d[1];
          if (R4 < 0 || R4 > 5 || C4 < 0 || C4 > 5) continue;
          uint64_t m = 0;
          for (int i = 0; i < 5; i++) m |= 1ull << (6 * (R + i * d[0]) + C + i * d[1]);
          l[n++] = m;
        }
    return l;
  }();
  return lines;
}

bool shows_five(const int cells[36], int colour) {
  uint64_t own = 0;
  for (int i = 0; i < 36; i++) own |= (uint64_t)(cells[i] == colour) << i;
  for (uint64_t m : five_lines())
    if ((own & m) == m) return true;
  return false;
}

// Decode and validate one midgame root; fills the descriptor (without the
// table/out fields).
int describe_board(uint64_t packed, int max_empty, MidBoard* mb, int i) {
  const HostTables& t = host_tables();
  int cells[36];
  std::memset(mb, 0, sizeof *mb);
  int nb = 0, nw = 0;
  for (int q = 0; q < 4; q++) {
    uint32_t code = (uint32_t)(packed >> (16 * q)) & 0xFFFFu;
    if (code >= (uint32_t)kQStates)
      return fail(PP_EINVAL, "board %d: quadrant %d field %u is not a base-3 code", i, q, code);
    uint32_t dec = t.qdecode[code];
    mb->root_b[q] = dec & 0x1FF;
    mb->root_w[q] = (dec >> 9) & 0x1FF;
    nb += (dec >> 18) & 15;
    nw += (dec >> 22) & 15;
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) {
        int bit = 3 * r + c, R = 3 * (q >> 1) + r, C = 3 * (q & 1) + c;
        cells[6 * R + C] = (mb->root_b[q] >> bit & 1) ? 1 : (mb->root_w[q] >> bit & 1) ? 2 : 0;
      }
  }
  if (nb != nw && nb != nw + 1)
    return fail(PP_EINVAL, "board %d: %d black and %d white is not a position", i, nb, nw);
  int k = 36 - nb - nw;
  if (k > max_empty) return fail(PP_EINVAL, "board %d: %d empty cells > max_empty %d", i, k, max_empty);
  if (shows_five(cells, 1) || shows_five(cells, 2))
    return fail(PP_EINVAL, "board %d already has five in a row", i);
  mb->k = (uint32_t)k;
  mb->mover = nb == nw ? 1u : 2u;
  int slot = 0;
  for (int q = 0; q < 4; q++) {
    mb->qstart[q] = (uint8_t)slot;
    uint32_t empty = ~(mb->root_b[q] | mb->root_w[q]) & 0x1FFu;
    for (int bit = 0; bit < 9; bit++)
      if (empty >> bit & 1) mb->slot_bit[slot++] = (uint8_t)bit;
  }
  mb->qstart[4] = (uint8_t)slot;
  return PP_OK;
}

std::map<std::pair<int, int>, std::unique_ptr<LevelLists>> g_lists;

}  // namespace

int validate_midgame_board(uint64_t packed, int max_empty, MidBoard* mb, int i) {
  return describe_board(packed, max_empty, mb, i);
}

int report_error(int code, const char* message) { return fail(code, "%s", message); }

std::mutex& table_mutex() { return g_mutex; }

bool tables_ready() { return g_ready; }

uint64_t fills_total(int k) {
  // sum over m of C(k, m) C(m, ceil(m/2)), tabulated once (plans ask per board)
  static const std::array<uint64_t, kMaxEmpty + 1> table = [] {
    std::array<uint64_t, kMaxEmpty + 1> f{};
    for (int kk = 0; kk <= kMaxEmpty; kk++)
      for (int m = 0; m <= kk; m++) {
        uint64_t a = 1, b = 1;  // C(kk, m), C(m, ceil(m/2))
        for (int i = 0; i < m; i++) a = a * (kk - i) / (i + 1);
        for (int i = 0; i < (m + 1) / 2; i++) b = b * (m - i) / (i + 1);
        f[kk] += a * b;
      }
    return f;
  }();
  if (k < 0 || k > kMaxEmpty) return 0;
  return table[k];
}

void build_fill_lists(int k, int mover, FillLists* L) {
  std::vector<std::vector<uint64_t>> per(k + 1);
  const uint64_t total = pow3u(k);
  const int other = 3 - mover;
  std::vector<uint32_t> pos(total, 0xFFFFFFFFu);  // fill index -> position in its level
  for (uint64_t idx = 0; idx < total; idx++) {
    uint64_t x = idx;
    uint32_t bm = 0, wm = 0;
    int nm = 0, no = 0;
    for (int i = 0; i < k; i++, x /= 3) {
      int d = (int)(x % 3);
      if (d == 1) bm |= 1u << i;
      if (d == 2) wm |= 1u << i;
      nm += d == mover;
      no += d == other;
    }
    int m = nm + no;
    if (nm != (m + 1) / 2 || no != m / 2) continue;  // stones alternate from the root's mover
    pos[idx] = (uint32_t)per[m].size();
    per[m].push_back(idx | (uint64_t)bm << 32 | (uint64_t)wm << 48);
  }
  L->flat.clear();
  L->offset.clear();
  L->count.clear();
  L->ranks.clear();
  L->ranks_at.clear();
  uint64_t p3[17];
  p3[0] = 1;
  for (int i = 1; i <= 16; i++) p3[i] = p3[i - 1] * 3;
  for (int m = 0; m <= k; m++) {
    L->offset.push_back(L->flat.size());
    L->count.push_back((uint32_t)per[m].size());
    L->flat.insert(L->flat.end(), per[m].begin(), per[m].end());
    L->ranks_at.push_back(L->ranks.size());
    if (m == k) continue;
    const uint64_t c = (m & 1) ? (uint64_t)other : (uint64_t)mover;  // colour placed at level m
    for (uint64_t e : per[m]) {
      const uint64_t idx = e & 0xFFFFFFFFu;
      const uint32_t filled = (uint32_t)(e >> 32 & 0xFFFFu) | (uint32_t)(e >> 48);
      for (int i = 0; i < k; i++)
        if (!(filled >> i & 1)) L->ranks.push_back(pos[idx + c * p3[i]]);
    }
  }
}

const LevelLists* level_lists(int k, int mover, std::string* err) {
  auto key = std::make_pair(k, mover);
  auto it = g_lists.find(key);
  if (it != g_lists.end()) return it->second.get();
  auto L = std::make_unique<LevelLists>();
  L->k = k;
  L->mover = mover;
  FillLists F;
  build_fill_lists(k, mover, &F);
  L->offset = F.offset;
  L->count = F.count;
  L->ranks_at = F.ranks_at;
  L->total = F.flat.size();
  void* d = nullptr;
  void* r = nullptr;
  cudaError_t e = cudaMalloc(&d, F.flat.size() * sizeof(uint64_t));
  if (!e) e = cudaMemcpy(d, F.flat.data(), F.flat.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (!e) e = cudaMalloc(&r, std::max<size_t>(F.ranks.size(), 1) * sizeof(uint32_t));
  if (!e && !F.ranks.empty()) e = cudaMemcpy(r, F.ranks.data(), F.ranks.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e) {
    if (err) *err = std::string("level lists: ") + cudaGetErrorString(e);
    if (d) cudaFree(d);
    if (r) cudaFree(r);
    return nullptr;
  }
  L->d_entries = (uint64_t*)d;
  L->d_ranks = (uint32_t*)r;
  const LevelLists* out = L.get();
  g_lists[key] = std::move(L);
  return out;
}

}  // namespace pp

using namespace pp;

struct pp_midgame_plan {
  int n = 0, max_empty = 0, kmax = 0;
  uint64_t table_entries = 0;  // compact fill-table entries of all boards
  void* d_mem = nullptr;  // one allocation holding the four arrays below
  MidBoard* d_boards = nullptr;
  MidSeg* d_segs = nullptr;
  using Level = MidLevel;
  std::vector<Level> levels;  // levels[j] is stones added m = kmax - j
  MidLevel* d_levels = nullptr;
  uint32_t* d_sync = nullptr;  // barrier count, generation, status (persistent mode)
  int mode = 1;                // 1 persistent, 2 one launch per level, 3 graph of level launches
  int parity = -1;             // -1 every rotation; 0 / 1 only that parity class of g (half tables)
  int ctas_per_sm = 0;
  std::string shape;           // autotuner cache key: max_empty and boards per number of empty cells
  // graph of the level launches, captured for one (workspace, output) pair
  cudaGraphExec_t graph = nullptr;
  void* graph_ws = nullptr;
  void* graph_out = nullptr;
  // one-shot plans (the solve entry points) take d_mem from the stream-ordered
  // pool on this stream and give it back there
  bool pooled = false;
  cudaStream_t pool_stream = nullptr;
};

extern "C" {

}  // extern "C"

namespace pp {
namespace {

// Autotuner cache key of a midgame plan: device, parity class and shape.
std::string midgame_tune_key(const pp_midgame_plan* P) {
  return tune_device_tag() + " midgame parity=" + std::to_string(P->parity) + " " + P->shape;
}

}  // namespace
}  // namespace pp

namespace pp {
namespace {
void clear_ready_cache();
}  // namespace
}  // namespace pp

extern "C" {

int pp_init(void) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_ready) return PP_OK;
  std::string err;
  int e = upload_tables(host_tables(), &g_dev, &err);
  if (e) return fail(PP_ECUDA, "%s", err.c_str());
  // keep stream-ordered temporaries (the transformed children of a slice
  // step, a few GB) cached in the device's default pool between calls
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  g_ready = true;
  return PP_OK;
}

void pp_shutdown(void) {
  clear_ready_cache();
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ready) return;
  cudaFree((void*)g_dev.qdecode);
  cudaFree((void*)g_dev.standard);
  cudaFree((void*)g_dev.qlist);
  cudaFree((void*)g_dev.forms);
  for (auto& kv : g_lists) cudaFree(kv.second->d_entries);
  g_lists.clear();
  g_ready = false;
}

const char* pp_last_error_string(void) { return g_error.c_str(); }

uint64_t pp_launch_count(void) { return launch_total(); }

int pp_quadrant_states(int black, int white, uint16_t* codes, int max) {
  if (black < 0 || white < 0 || black + white > 9) return -fail(PP_EINVAL, "bad counts %d, %d", black, white);
  const HostTables& t = host_tables();
  int n = t.qdim[black][white];
  if (codes)
    for (int i = 0; i < n && i < max; i++) codes[i] = t.qlist[t.qoff[black][white] + i];
  return n;
}

int pp_slice_sections(int n, pp_section_desc* out, int max, uint64_t* total) {
  if (n < 0 || n > 36) return -fail(PP_EINVAL, "slice %d out of range", n);
  auto secs = slice_sections(n, total);
  if (out)
    for (size_t i = 0; i < secs.size() && (int)i < max; i++) out[i] = secs[i];
  return (int)secs.size();
}

int pp_midgame_workspace_bytes(int n, int max_empty, size_t* bytes) {
  if (n < 0 || max_empty < 0 || max_empty > kMaxEmpty || !bytes)
    return fail(PP_EINVAL, "bad workspace query n=%d max_empty=%d", n, max_empty);
  *bytes = (size_t)n * (plan_bytes_per_board(max_empty) + sizeof(pp_super));
  return PP_OK;
}

namespace pp {
namespace {
int midgame_plan_create(const uint64_t* h_boards, int n, int max_empty, pp_midgame_plan** plan,
                        cudaStream_t pool_stream, bool pooled);
}  // namespace
}  // namespace pp

int pp_midgame_plan_create(const uint64_t* h_boards, int n, int max_empty, pp_midgame_plan** plan) {
  return midgame_plan_create(h_boards, n, max_empty, plan, nullptr, false);
}

}  // extern "C"

namespace pp {
namespace {

int midgame_plan_create(const uint64_t* h_boards, int n, int max_empty, pp_midgame_plan** plan,
                        cudaStream_t pool_stream, bool pooled) {
  if (!plan) return fail(PP_EINVAL, "plan pointer is null");
  *plan = nullptr;
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || (n > 0 && !h_boards)) return fail(PP_EINVAL, "bad board array");
  if (max_empty < 0 || max_empty > kMaxEmpty) return fail(PP_EINVAL, "max_empty %d not in 0..16", max_empty);
  auto P = std::make_unique<pp_midgame_plan>();
  P->n = n;
  P->max_empty = max_empty;
  // one persistent launch (measured fastest) where the device can co-schedule it
  P->mode = persistent_midgame_blocks(0) > 0 ? 1 : 2;
  std::vector<MidBoard> boards(n);
  for (int i = 0; i < n; i++) {
    int rc = describe_board(h_boards[i], max_empty, &boards[i], i);
    if (rc) return rc;
    boards[i].table = P->table_entries;  // boards' compact tables back to back
    P->table_entries += fills_total((int)boards[i].k);
    boards[i].out = (uint64_t)i;
    boards[i].masks = (uint64_t)i * mask_entries_per_board(max_empty);
    P->kmax = std::max(P->kmax, (int)boards[i].k);
  }
  {
    int per_k[kMaxEmpty + 1] = {};
    for (const MidBoard& b : boards) per_k[b.k]++;
    P->shape = "max_empty=" + std::to_string(max_empty) + " boards=";
    for (int k = 0; k <= kMaxEmpty; k++)
      if (per_k[k]) P->shape += std::to_string(k) + ":" + std::to_string(per_k[k]) + ",";
  }
  std::vector<MidSeg> segs;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    // each board's level lists, looked up once per (empty cells, mover)
    std::vector<const LevelLists*> lists(n);
    const LevelLists* memo[kMaxEmpty + 1][3] = {};
    for (int i = 0; i < n; i++) {
      const LevelLists*& L = memo[boards[i].k][boards[i].mover];
      if (!L) {
        std::string err;
        if (!(L = level_lists((int)boards[i].k, (int)boards[i].mover, &err))) return fail(PP_ECUDA, "%s", err.c_str());
      }
      lists[i] = L;
    }
    bool same = n > 0;  // every board with the same empty cells and mover
    for (int i = 1; i < n && same; i++) same = boards[i].k == boards[0].k && boards[i].mover == boards[0].mover;
    if (!same) segs.reserve((size_t)n * (P->kmax + 1));
    for (int m = P->kmax; m >= 0 && same; m--) {
      // one shared descriptor per level: segment j is board j
      const LevelLists* L = lists[0];
      MidSeg s{};
      s.list = L->d_entries + L->offset[m];
      s.ranks = L->d_ranks + L->ranks_at[m];
      s.loff = (uint32_t)L->offset[m];
      s.coff = m < P->kmax ? (uint32_t)L->offset[m + 1] : 0u;
      s.count = L->count[m];
      s.level = (uint32_t)m;
      const uint32_t per = (s.count + kBlock - 1) / kBlock;
      if ((uint64_t)per * (uint64_t)n >= (1ull << 31)) return fail(PP_EINVAL, "too many boards for one level launch");
      pp_midgame_plan::Level lv{(int)segs.size(), n, per * (uint32_t)n, per | kSharedSegs};
      segs.push_back(s);
      P->levels.push_back(lv);
    }
    for (int m = P->kmax; m >= 0 && n > 0 && !same; m--) {
      pp_midgame_plan::Level lv{(int)segs.size(), 0, 0, 0};
      for (int i = 0; i < n; i++) {
        if ((int)boards[i].k < m) continue;
        const LevelLists* L = lists[i];
        MidSeg s{};
        s.block0 = lv.blocks;
        s.list = L->d_entries + L->offset[m];
        s.ranks = L->d_ranks + L->ranks_at[m];
        s.loff = (uint32_t)L->offset[m];
        s.coff = m < (int)boards[i].k ? (uint32_t)L->offset[m + 1] : 0u;
        s.count = L->count[m];
        s.board = (uint32_t)i;
        s.level = (uint32_t)m;
        lv.blocks += (s.count + kBlock - 1) / kBlock;
        segs.push_back(s);
        lv.nsegs++;
      }
      lv.seg_blocks = uniform_seg_blocks(segs.data() + lv.seg0, lv.nsegs, kBlock);
      if ((uint64_t)lv.blocks >= (1ull << 31)) return fail(PP_EINVAL, "too many boards for one level launch");
      P->levels.push_back(lv);
    }
  }
  if (n > 0) {
    // boards, segments, levels and the barrier words (zero) packed into one
    // allocation and one copy
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t ob = 0, os = ob + up(boards.size() * sizeof(MidBoard));
    const size_t ol = os + up(segs.size() * sizeof(MidSeg));
    const size_t oy = ol + up(P->levels.size() * sizeof(MidLevel)), total = oy + 4 * sizeof(uint32_t);
    std::vector<char> pack(total, 0);
    std::memcpy(pack.data() + ob, boards.data(), boards.size() * sizeof(MidBoard));
    std::memcpy(pack.data() + os, segs.data(), segs.size() * sizeof(MidSeg));
    std::memcpy(pack.data() + ol, P->levels.data(), P->levels.size() * sizeof(MidLevel));
    cudaError_t e;
    if (pooled) {
      // stream-ordered: no device-wide synchronisation; the pageable source
      // is staged before the copy call returns
      e = cudaMallocAsync(&P->d_mem, total, pool_stream);
      if (!e) e = cudaMemcpyAsync(P->d_mem, pack.data(), total, cudaMemcpyHostToDevice, pool_stream);
      if (e && P->d_mem) cudaFreeAsync(P->d_mem, pool_stream);
    } else {
      e = cudaMalloc(&P->d_mem, total);
      if (!e) e = cudaMemcpy(P->d_mem, pack.data(), total, cudaMemcpyHostToDevice);
      if (e) cudaFree(P->d_mem);
    }
    if (e) {
      P->d_mem = nullptr;
      return cuda_fail(e, "plan upload");
    }
    P->pooled = pooled;
    P->pool_stream = pool_stream;
    char* base = static_cast<char*>(P->d_mem);
    P->d_boards = reinterpret_cast<MidBoard*>(base + ob);
    P->d_segs = reinterpret_cast<MidSeg*>(base + os);
    P->d_levels = reinterpret_cast<MidLevel*>(base + ol);
    P->d_sync = reinterpret_cast<uint32_t*>(base + oy);
  }
  *plan = P.release();
  return PP_OK;
}

}  // namespace
}  // namespace pp

extern "C" {

int pp_midgame_plan_run(pp_midgame_plan* P, void* d_workspace, size_t ws_bytes, pp_super* d_out, pp_stream s) {
  if (!P) return fail(PP_EINVAL, "null plan");
  if (P->n == 0) return PP_OK;
  const size_t need = (size_t)P->table_entries * fill_entry_bytes(P->parity) +
                      (size_t)P->n * mask_entries_per_board(P->max_empty) * kMaskBytes;
  if (ws_bytes < need) return fail(PP_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  if (!d_workspace || !d_out || ((uintptr_t)d_workspace & 31) || !aligned16(d_out))
    return fail(PP_EINVAL, "workspace must be 32-byte and output 16-byte aligned (non-null)");
  // workspace: fill tables of all boards, then their five tables
  void* masks = (char*)d_workspace + (size_t)P->table_entries * fill_entry_bytes(P->parity);
  if (P->mode == 1) {
    int grid = persistent_midgame_blocks(P->ctas_per_sm, P->parity >= 0);
    cudaError_t e = cudaMemsetAsync(P->d_sync, 0, 4 * sizeof(uint32_t), s);
    if (e) return cuda_fail(e, "barrier reset");
    int rc = launch_five_tables(P->d_boards, P->n, P->kmax, masks, s);
    if (!rc)
      rc = launch_midgame_persistent(P->d_boards, P->d_segs, P->d_levels, (int)P->levels.size(),
                                     (pp_super*)d_workspace, d_out, P->d_sync, grid, s, masks, P->parity);
    return rc ? cuda_fail(rc, "persistent midgame launch") : PP_OK;
  }
  if (P->mode == 3) {
    if (!P->graph || P->graph_ws != d_workspace || P->graph_out != d_out) {
      if (P->graph) cudaGraphExecDestroy(P->graph);
      P->graph = nullptr;
      cudaStream_t cs;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e) return cuda_fail(e, "capture stream");
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      int rc = 0;
      set_launch_counting(false);
      if (!e) rc = launch_five_tables(P->d_boards, P->n, P->kmax, masks, (pp_stream)cs);
      for (size_t j = 0; !e && !rc && j < P->levels.size(); j++) {
        const auto& lv = P->levels[j];
        rc = launch_midgame_level(P->d_boards, P->d_segs + lv.seg0, lv.nsegs, lv.blocks, (pp_super*)d_workspace,
                                  d_out, j + 1 == P->levels.size() ? 1 : 0, (pp_stream)cs, masks, lv.seg_blocks,
                                  P->parity);
      }
      set_launch_counting(true);
      cudaError_t e2 = e ? e : cudaStreamEndCapture(cs, &g);
      if (!e2 && !rc) e2 = cudaGraphInstantiate(&P->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (rc) return cuda_fail(rc, "graph capture launch");
      if (e2) return cuda_fail(e2, "graph capture");
      P->graph_ws = d_workspace;
      P->graph_out = d_out;
    }
    cudaError_t e = cudaGraphLaunch(P->graph, s);
    add_launches(P->levels.size() + 1);
    return e ? cuda_fail(e, "graph launch") : PP_OK;
  }
  int e = launch_five_tables(P->d_boards, P->n, P->kmax, masks, s);
  if (e) return cuda_fail(e, "five tables launch");
  for (size_t j = 0; j < P->levels.size(); j++) {
    const auto& lv = P->levels[j];
    const bool final_level = j + 1 == P->levels.size();
    e = launch_midgame_level(P->d_boards, P->d_segs + lv.seg0, lv.nsegs, lv.blocks, (pp_super*)d_workspace,
                             d_out, final_level ? 1 : 0, s, masks, lv.seg_blocks, P->parity);
    if (e) return cuda_fail(e, "midgame level launch");
  }
  return PP_OK;
}

int pp_midgame_plan_configure(pp_midgame_plan* P, const pp_batch_opts* opts) {
  if (!P || !opts) return fail(PP_EINVAL, "null plan or options");
  const int mode = opts->persistent == 0 ? 2 : opts->persistent;
  if (mode < 1 || mode > 3) return fail(PP_EINVAL, "mode %d is not 0..3", opts->persistent);
  if (opts->threads_per_block && opts->threads_per_block != kBlock)
    return fail(PP_EINVAL, "the midgame kernels run %d threads per block", kBlock);
  if (mode == 1 && persistent_midgame_blocks(opts->ctas_per_sm, P->parity >= 0) <= 0)
    return fail(PP_ECUDA, "persistent kernel does not fit on this device");
  P->mode = mode;
  P->ctas_per_sm = opts->ctas_per_sm;
  return PP_OK;
}

int pp_midgame_plan_status(pp_midgame_plan* P, pp_stream s) {
  if (!P) return fail(PP_EINVAL, "null plan");
  if (!P->d_sync) return PP_OK;
  uint32_t st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, P->d_sync + 2, sizeof st, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "plan status");
  if (st == PP_ETIMEOUT) return fail(PP_ETIMEOUT, "a grid barrier of the persistent midgame kernel timed out");
  return PP_OK;
}

int pp_selftest_barrier_timeout(uint32_t* d_sync, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (!d_sync || ((uintptr_t)d_sync & 3)) return fail(PP_EINVAL, "sync words must be a 4-byte aligned device array");
  cudaError_t e = cudaMemsetAsync(d_sync, 0, 4 * sizeof(uint32_t), s);
  if (e) return cuda_fail(e, "probe reset");
  int rc = launch_barrier_probe(d_sync, 1u << 16, s);
  if (rc) return cuda_fail(rc, "probe launch");
  uint32_t st = 0;
  e = cudaMemcpyAsync(&st, d_sync + 2, sizeof st, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "probe status");
  if (st == PP_ETIMEOUT) return fail(PP_ETIMEOUT, "bounded barrier wait expired (expected)");
  return PP_OK;
}

int pp_set_barrier_poll_limit(uint32_t polls) {
  set_barrier_spins(polls);
  return PP_OK;
}

int pp_midgame_plan_autotune(pp_midgame_plan* P, void* d_workspace, size_t ws_bytes, pp_super* d_out, pp_stream s,
                             pp_batch_opts* chosen) {
  if (!P) return fail(PP_EINVAL, "null plan");
  struct Cand {
    int mode, ctas;
  };
  const std::string key = midgame_tune_key(P);
  pp_batch_opts cached;
  if (tune_lookup(key, &cached)) {
    int rc = pp_midgame_plan_configure(P, &cached);
    if (!rc && chosen) *chosen = cached;
    return rc;
  }
  std::vector<Cand> cands = {{2, 0}, {3, 0}, {1, 0}, {1, 1}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(PP_ECUDA, "autotune events");
  float best = 1e30f;
  Cand win = {2, 0};
  for (const Cand& c : cands) {
    pp_batch_opts o{c.mode, 0, c.ctas, 0, 0};
    if (pp_midgame_plan_configure(P, &o)) continue;
    int rc = pp_midgame_plan_run(P, d_workspace, ws_bytes, d_out, s);  // warm-up (and graph capture)
    if (!rc) rc = pp_midgame_plan_status(P, s);
    if (rc) continue;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && !rc; r++) rc = pp_midgame_plan_run(P, d_workspace, ws_bytes, d_out, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) || rc || pp_midgame_plan_status(P, s)) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms, win = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pp_batch_opts o{win.mode, 0, win.ctas, 0, 0};
  int rc = pp_midgame_plan_configure(P, &o);
  if (rc) return rc;
  if (best < 1e30f) tune_record(key, o);  // nothing is recorded when no candidate ran
  if (chosen) *chosen = o;
  return rc;
}

void pp_midgame_plan_destroy(pp_midgame_plan* P) {
  if (!P) return;
  if (P->graph) cudaGraphExecDestroy(P->graph);
  if (P->pooled)
    cudaFreeAsync(P->d_mem, P->pool_stream);
  else
    cudaFree(P->d_mem);
  delete P;
}

int pp_midgame_plan_set_parity(pp_midgame_plan* P, int parity) {
  if (!P) return fail(PP_EINVAL, "null plan");
  if (parity < -1 || parity > 1) return fail(PP_EINVAL, "parity %d is not -1, 0 or 1", parity);
  if (parity != P->parity && P->graph) {  // captured with the other table layout
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  P->parity = parity;
  return PP_OK;
}

int pp_midgame_parity_workspace_bytes(int n, int max_empty, size_t* bytes) {
  if (n < 0 || max_empty < 0 || max_empty > kMaxEmpty || !bytes)
    return fail(PP_EINVAL, "bad workspace query n=%d max_empty=%d", n, max_empty);
  *bytes = (size_t)n * (plan_bytes_per_board(max_empty, 0) + sizeof(pp_super));
  return PP_OK;
}

}  // extern "C"

namespace {

// A one-shot solve runs its plan once.  A shape the autotuner has timed
// takes the recorded mode when it is the persistent launch or the level
// launches.  A recorded graph keeps the plan's default (one persistent
// launch): capturing a graph for a single replay costs more than it saves,
// and the same level launches without a graph measured slower than the
// persistent launch (7.52 against 7.29 ms end to end for 1024 boards x 12
// empty cells).  Untimed shapes keep the default too.
void one_shot_mode(pp_midgame_plan* P) {
  pp_batch_opts o;
  if (!tune_peek(midgame_tune_key(P), &o) || o.persistent == 3) return;
  pp_midgame_plan_configure(P, &o);  // if it fails the plan keeps its default mode
}

int solve_device(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty, int parity, void* d_workspace,
                 size_t ws_bytes, pp_stream s) {
  if (n < 0 || (n > 0 && (!d_boards || !aligned16(d_boards))))
    return fail(PP_EINVAL, "boards must be a non-null 16-byte aligned device array");
  std::vector<uint64_t> h(n);
  if (n > 0) {
    cudaError_t e = cudaMemcpyAsync(h.data(), d_boards, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(e, "reading boards");
  }
  pp_midgame_plan* P = nullptr;
  int rc = midgame_plan_create(h.data(), n, max_empty, &P, s, true);
  if (rc) return rc;
  rc = pp_midgame_plan_set_parity(P, parity);
  if (!rc) one_shot_mode(P);
  if (!rc) rc = pp_midgame_plan_run(P, d_workspace, ws_bytes, d_out, s);
  uint32_t st = 0;
  cudaError_t e = rc ? cudaSuccess : cudaMemcpyAsync(&st, P->d_sync + 2, sizeof st, cudaMemcpyDeviceToHost, s);
  pp_midgame_plan_destroy(P);
  if (!e) e = cudaStreamSynchronize(s);
  if (!rc && e) rc = cuda_fail(e, "midgame solve");
  // a persistent launch whose grid barrier gave up stops early
  if (!rc && st == PP_ETIMEOUT) rc = fail(PP_ETIMEOUT, "a grid barrier of the persistent midgame kernel timed out");
  return rc;
}

}  // namespace

extern "C" {

int pp_midgame_solve(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty, void* d_workspace,
                     size_t ws_bytes, pp_stream s) {
  return solve_device(d_boards, n, d_out, max_empty, -1, d_workspace, ws_bytes, s);
}

int pp_midgame_solve_parity(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty, int parity,
                            void* d_workspace, size_t ws_bytes, pp_stream s) {
  if (parity < 0 || parity > 1) return fail(PP_EINVAL, "parity %d is not 0 or 1", parity);
  return solve_device(d_boards, n, d_out, max_empty, parity, d_workspace, ws_bytes, s);
}

int pp_midgame_solve_host(const uint64_t* h_boards, int n, pp_super* h_out, int max_empty, void* d_workspace,
                          size_t ws_bytes, pp_stream s) {
  if (n < 0 || (n > 0 && (!h_boards || !h_out))) return fail(PP_EINVAL, "bad host arrays");
  if (n == 0) return PP_OK;
  // the caller's workspace holds the plan's tables; results land after them
  const size_t tables = (size_t)n * plan_bytes_per_board(max_empty);
  const size_t need = tables + (size_t)n * sizeof(pp_super);
  if (ws_bytes < need) return fail(PP_ENOMEM, "workspace %zu bytes < %zu needed (tables + results)", ws_bytes, need);
  pp_midgame_plan* P = nullptr;
  int rc = midgame_plan_create(h_boards, n, max_empty, &P, s, true);
  if (rc) return rc;
  pp_super* d_out = (pp_super*)((char*)d_workspace + tables);
  one_shot_mode(P);
  rc = pp_midgame_plan_run(P, d_workspace, tables, d_out, s);
  uint32_t st = 0;
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaMemcpyAsync(h_out, d_out, n * sizeof(pp_super), cudaMemcpyDeviceToHost, s);
  if (!rc && !e) e = cudaMemcpyAsync(&st, P->d_sync + 2, sizeof st, cudaMemcpyDeviceToHost, s);
  pp_midgame_plan_destroy(P);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (!rc && (e || e2)) rc = cuda_fail(e ? e : e2, "midgame solve (host arrays)");
  // a persistent launch whose grid barrier gave up stops early: its values
  // are incomplete, so the call reports PP_ETIMEOUT instead of PP_OK
  if (!rc && st == PP_ETIMEOUT) rc = fail(PP_ETIMEOUT, "a grid barrier of the persistent midgame kernel timed out");
  return rc;
}

}  // extern "C"

namespace pp {
namespace {

// Tasks for the listed sections of slice n; children looked up in slice n+1.
// With d4, secs are D4-minimal sections and in_values holds the D4-minimal
// sections of slice n+1: a child section that is not minimal is read through
// the symmetry that carries it onto its least image.
uint64_t section_boards(const pp_section_desc& d) { return (uint64_t)d.dim[0] * d.dim[1] * d.dim[2] * d.dim[3]; }

int build_tasks(int n, const std::vector<pp_section_desc>& secs, const std::vector<int>& which,
                const pp_super* in_values, const pp_super* const* child_ptrs, bool compact,
                std::vector<SecTask>* tasks, uint32_t* blocks, bool d4 = false,
                const uint64_t* in_offsets = nullptr, uint64_t in_count = 0) {
  const HostTables& t = host_tables();
  std::vector<pp_section_desc> next;
  if (n < 36 && !child_ptrs) next = d4 ? slice_sections_d4(n + 1, nullptr) : slice_sections(n + 1, nullptr);
  const int mover = (n % 2 == 0) ? 1 : 2;
  uint64_t start = 0, nblocks = 0;
  for (int si : which) {
    const pp_section_desc& d = secs[si];
    SecTask tk{};
    tk.block0 = (uint32_t)nblocks;
    tk.size = 1;
    for (int q = 0; q < 4; q++) {
      tk.dim[q] = d.dim[q];
      tk.size *= d.dim[q];
      tk.qoff[q] = (uint16_t)t.qoff[d.bw[q][0]][d.bw[q][1]];
      tk.bw[q][0] = d.bw[q][0];
      tk.bw[q][1] = d.bw[q][1];
    }
    tk.out = compact ? start : d.offset;
    tk.n = (uint8_t)n;
    tk.mover = (uint8_t)mover;
    for (int q = 0; q < 4 && n < 36; q++) {
      if (d.bw[q][0] + d.bw[q][1] >= 9) continue;
      tk.movable |= 1u << q;
      uint8_t cbw[4][2];
      std::memcpy(cbw, d.bw, sizeof cbw);
      cbw[q][mover - 1]++;
      tk.cqoff[q] = (uint16_t)t.qoff[cbw[q][0]][cbw[q][1]];
      if (d4) {  // the stored child section is the least image
        uint8_t least[4][2];
        tk.sym[q] = (uint8_t)least_image(cbw, least);
        std::memcpy(cbw, least, sizeof cbw);
      }
      uint32_t cdim[4];
      for (int r = 0; r < 4; r++) cdim[r] = (uint32_t)t.qdim[cbw[r][0]][cbw[r][1]];
      uint64_t stride = 1;
      for (int r = 0; r < 4; r++) {
        tk.cstride[q][r] = stride;
        stride *= cdim[r];
      }
      if (child_ptrs) {
        if (!child_ptrs[q] || !aligned32(child_ptrs[q]))
          return fail(PP_EINVAL, "child section for quadrant %d must be a non-null 32-byte aligned pointer", q);
        tk.child[q] = child_ptrs[q];
      } else {
        int ci = section_index(next, cbw);
        if (ci < 0) return fail(PP_EINVAL, "child section of quadrant %d not found", q);
        if (in_offsets) {  // sparse input: only some sections of slice n+1 are present
          const uint64_t off = in_offsets[ci], size = section_boards(next[ci]);
          if (off == PP_ABSENT) return fail(PP_EINVAL, "slice %d section %d is read but absent from the input", n + 1, ci);
          if (off > in_count || size > in_count - off)
            return fail(PP_EINVAL, "slice %d section %d lies outside the input's %llu values", n + 1, ci,
                        (unsigned long long)in_count);
          tk.child[q] = in_values + off;
        } else {
          tk.child[q] = in_values + next[ci].offset;
        }
      }
    }
    if (tk.size >= (1ull << 32)) return fail(PP_EINVAL, "sections of 2^32 boards or more are not supported");
    start += tk.size;
    nblocks += (tk.size + kBlock - 1) / kBlock;
    if (nblocks >= (1ull << 31)) return fail(PP_EINVAL, "too many boards for one launch");
    tasks->push_back(tk);
  }
  *blocks = (uint32_t)nblocks;
  return PP_OK;
}

int run_tasks(const std::vector<SecTask>& tasks, uint32_t blocks, pp_super* out, pp_stream s, bool d4 = false) {
  if (tasks.empty() || !blocks) return PP_OK;
  SecTask* d = nullptr;
  size_t bytes = tasks.size() * sizeof(SecTask);
  cudaError_t e = cudaMallocAsync((void**)&d, bytes, s);
  if (!e) e = cudaMemcpyAsync(d, tasks.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e) return cuda_fail(e, "section task upload");
  int rc = launch_sections(d, (int)tasks.size(), blocks, out, s, d4);
  cudaFreeAsync(d, s);
  if (rc) return cuda_fail(rc, "section launch");
  return PP_OK;
}

// Slice 35 by lines: one task per section, grouped by the non-full quadrant.
// The children (slice 36 values) are first turned into X2/X3 in a temporary
// buffer: the whole slice 36 when it is given, else each distinct child
// section passed by pointer.
struct Line35Work {
  struct Kid {
    const pp_super* src;
    uint64_t size, at;  // values, offset in the temporary buffer
  };
  // longest lines first, a new thread block wherever the line axis changes;
  // child = offset into the temporary (values)
  std::vector<LineTask> all;
  uint32_t warps = 0;
  uint64_t tmp_size = 0;
  std::vector<Kid> kids;
  bool on_demand = false;  // no slice-36 input: children evaluated in the kernel
  bool terminal = false;   // slice 36: no children, values from five in a row (line36_kernel)
  // D4-reduced slices: sections whose child section is stored under a
  // non-trivial symmetry are left to the per-board kernel (section index,
  // output position)
  std::vector<std::pair<int, uint64_t>> others;
};

int build_line35(const std::vector<pp_section_desc>& secs, const std::vector<int>& which,
                 const pp_super* in_values, const pp_super* const* child_ptrs, bool compact, Line35Work* W,
                 bool d4 = false) {
  const HostTables& t = host_tables();
  uint64_t total36 = 0;
  std::vector<pp_section_desc> next = d4 ? slice_sections_d4(36, &total36) : slice_sections(36, &total36);
  std::vector<LineTask> tasks;
  uint64_t start = 0;
  W->on_demand = !child_ptrs && !in_values;
  if (!child_ptrs && in_values) {
    W->kids.push_back({in_values, total36, 0});
    W->tmp_size = total36;
  }
  for (int si : which) {
    const pp_section_desc& d = secs[si];
    int Q = -1;
    for (int q = 0; q < 4; q++)
      if (d.bw[q][0] + d.bw[q][1] < 9) Q = q;
    if (Q < 0) return fail(PP_EINVAL, "slice-35 section without an empty cell");
    LineTask tk{};
    uint64_t size = 1, stride = 1;
    for (int q = 0; q < 4; q++) {
      tk.dim[q] = d.dim[q];
      tk.stride[q] = (uint32_t)stride;
      stride *= d.dim[q];
      tk.qoff[q] = (uint16_t)t.qoff[d.bw[q][0]][d.bw[q][1]];
      size *= d.dim[q];
    }
    if (size >= (1ull << 32)) return fail(PP_EINVAL, "section too large");
    tk.lines = (uint32_t)(size / d.dim[Q]);
    tk.mover = 2;  // slice 35: 18 black, 17 white, white moves
    uint8_t cbw[4][2];
    std::memcpy(cbw, d.bw, sizeof cbw);
    cbw[Q][1]++;
    if (d4) {
      uint8_t least[4][2];
      if (least_image(cbw, least) != 0) {
        W->others.push_back({si, compact ? start : d.offset});
        start += size;
        continue;
      }
    }
    uint64_t cs = 1;
    for (int q = 0; q < 4; q++) {
      tk.cstride[q] = (uint32_t)cs;
      cs *= (uint64_t)t.qdim[cbw[q][0]][cbw[q][1]];
    }
    tk.cdim = (uint32_t)t.qdim[cbw[Q][0]][cbw[Q][1]];
    tk.cqoff = (uint32_t)t.qoff[cbw[Q][0]][cbw[Q][1]];
    uint64_t at = 0;
    if (child_ptrs) {
      if (!child_ptrs[Q] || !aligned32(child_ptrs[Q]))
        return fail(PP_EINVAL, "child section for quadrant %d must be a non-null 32-byte aligned pointer", Q);
      int kid = -1;
      for (size_t i = 0; i < W->kids.size(); i++)
        if (W->kids[i].src == child_ptrs[Q]) kid = (int)i;
      if (kid < 0) {
        W->kids.push_back({child_ptrs[Q], cs, W->tmp_size});
        kid = (int)W->kids.size() - 1;
        W->tmp_size += cs;
      }
      at = W->kids[kid].at;
    } else if (!W->on_demand) {
      int ci = section_index(next, cbw);
      if (ci < 0) return fail(PP_EINVAL, "child section not found");
      at = next[ci].offset;
    }
    tk.child = (const pp_super*)(uintptr_t)at;  // an offset until rebased
    tk.out = compact ? start : d.offset;
    tk.q = (uint32_t)Q;
    start += size;
    tasks.push_back(tk);
  }
  // A block's time grows with its line length: the longest lines start
  // first, so the launch ends on short ones.  Blocks never mix line axes
  // (each copies its axis's forms into shared memory).
  std::stable_sort(tasks.begin(), tasks.end(), [](const LineTask& a, const LineTask& b) {
    return a.dim[a.q] != b.dim[b.q] ? a.dim[a.q] > b.dim[b.q] : a.q < b.q;
  });
  uint32_t warp = 0;
  for (size_t i = 0; i < tasks.size(); i++) {
    if (i > 0 && tasks[i].q != tasks[i - 1].q) warp = (warp + kLineWarps - 1) / kLineWarps * kLineWarps;
    tasks[i].warp0 = warp;
    warp += (tasks[i].lines + 31) / 32;
  }
  W->warps = warp;
  W->all = std::move(tasks);
  return PP_OK;
}

// Slice 36 by lines: no children; the line axis of a section is its
// quadrant with the most states (the latest of equals, so that lanes step
// through quadrant 0 and a warp's stores fall on neighbouring values).
int build_line36(const std::vector<pp_section_desc>& secs, const std::vector<int>& which, bool compact,
                 Line35Work* W) {
  const HostTables& t = host_tables();
  std::vector<LineTask> tasks;
  uint64_t start = 0;
  W->terminal = true;
  for (int si : which) {
    const pp_section_desc& d = secs[si];
    LineTask tk{};
    uint64_t size = 1, stride = 1;
    int Q = 3;
    for (int q = 0; q < 4; q++) {
      tk.dim[q] = d.dim[q];
      tk.stride[q] = (uint32_t)stride;
      stride *= d.dim[q];
      tk.qoff[q] = (uint16_t)t.qoff[d.bw[q][0]][d.bw[q][1]];
      size *= d.dim[q];
    }
    for (int q = 2; q >= 0; q--)
      if (d.dim[q] > d.dim[Q]) Q = q;
    if (size >= (1ull << 32)) return fail(PP_EINVAL, "section too large");
    tk.lines = (uint32_t)(size / d.dim[Q]);
    tk.mover = 1;  // slice 36: 18 black, 18 white, black to move
    tk.out = compact ? start : d.offset;
    tk.q = (uint32_t)Q;
    start += size;
    tasks.push_back(tk);
  }
  // longest lines first; blocks never mix line axes
  std::stable_sort(tasks.begin(), tasks.end(), [](const LineTask& a, const LineTask& b) {
    return a.dim[a.q] != b.dim[b.q] ? a.dim[a.q] > b.dim[b.q] : a.q < b.q;
  });
  uint32_t warp = 0;
  for (size_t i = 0; i < tasks.size(); i++) {
    if (i > 0 && tasks[i].q != tasks[i - 1].q) warp = (warp + kLineWarps - 1) / kLineWarps * kLineWarps;
    tasks[i].warp0 = warp;
    warp += (tasks[i].lines + 31) / 32;
  }
  W->warps = warp;
  W->all = std::move(tasks);
  return PP_OK;
}

std::vector<LineTask> rebased(const Line35Work& W, pp_super* tmp) {
  std::vector<LineTask> all = W.all;
  for (auto& tk : all) tk.child = W.on_demand ? nullptr : tmp + (uintptr_t)tk.child;
  return all;
}

int launch_line35_work(const Line35Work& W, const LineTask* d, pp_super* tmp, pp_super* out, pp_stream s) {
  if (W.terminal) return launch_line36(d, (int)W.all.size(), W.warps, out, s);
  int rc = 0;
  for (auto& k : W.kids)
    if (!rc) rc = launch_child_transform(k.src, k.size, tmp + k.at, s);
  if (!rc) rc = launch_line35(d, (int)W.all.size(), W.warps, out, s, W.on_demand);
  return rc;
}

// The per-board tasks of the sections a D4 line build left over, each
// writing at its output position.
int other_tasks(const Line35Work& W, const std::vector<pp_section_desc>& secs, const pp_super* in_values,
                std::vector<SecTask>* tasks, uint32_t* blocks) {
  std::vector<int> which;
  for (auto& o : W.others) which.push_back(o.first);
  int rc = build_tasks(35, secs, which, in_values, nullptr, false, tasks, blocks, true);
  for (size_t i = 0; !rc && i < tasks->size(); i++) (*tasks)[i].out = W.others[i].second;
  return rc;
}

int run_line35(const std::vector<pp_section_desc>& secs, const std::vector<int>& which, const pp_super* in_values,
               const pp_super* const* child_ptrs, bool compact, pp_super* out, pp_stream s, bool d4 = false,
               int n = 35) {
  Line35Work W;
  int rc = n == 36 ? build_line36(secs, which, compact, &W)
                   : build_line35(secs, which, in_values, child_ptrs, compact, &W, d4);
  if (rc) return rc;
  if (!W.others.empty()) {
    std::vector<SecTask> tasks;
    uint32_t blocks = 0;
    if ((rc = other_tasks(W, secs, in_values, &tasks, &blocks))) return rc;
    if ((rc = run_tasks(tasks, blocks, out, s, true))) return rc;
  }
  if (W.all.empty()) return PP_OK;
  pp_super* tmp = nullptr;
  cudaError_t e = W.tmp_size ? cudaMallocAsync((void**)&tmp, W.tmp_size * sizeof(pp_super), s) : cudaSuccess;
  if (e) return cuda_fail(e, "transformed children buffer");
  std::vector<LineTask> all = rebased(W, tmp);
  LineTask* d = nullptr;
  e = cudaMallocAsync((void**)&d, all.size() * sizeof(LineTask), s);
  if (!e) e = cudaMemcpyAsync(d, all.data(), all.size() * sizeof(LineTask), cudaMemcpyHostToDevice, s);
  if (e) {
    cudaFreeAsync(tmp, s);
    return cuda_fail(e, "line task upload");
  }
  rc = launch_line35_work(W, d, tmp, out, s);
  cudaFreeAsync(d, s);
  if (tmp) cudaFreeAsync(tmp, s);
  if (rc) return cuda_fail(rc, "line launch");
  return PP_OK;
}

// Sections reordered largest first, block offsets recomputed (outputs keep
// their places).
void order_largest_first(std::vector<SecTask>* tasks) {
  std::stable_sort(tasks->begin(), tasks->end(), [](const SecTask& a, const SecTask& b) { return a.size > b.size; });
  uint32_t blocks = 0;
  for (auto& tk : *tasks) {
    tk.block0 = blocks;
    blocks += (uint32_t)((tk.size + kBlock - 1) / kBlock);
  }
}

bool valid_section(int n, const pp_section_desc* d) {
  const HostTables& t = host_tables();
  int B = 0, W = 0;
  for (int q = 0; q < 4; q++) {
    if (d->bw[q][0] + d->bw[q][1] > 9) return false;
    if (d->dim[q] != t.qdim[d->bw[q][0]][d->bw[q][1]]) return false;
    B += d->bw[q][0];
    W += d->bw[q][1];
  }
  return B == (n + 1) / 2 && W == n / 2;
}

// Sections of slices below 35 by lines (section_line_kernel), grouped by
// the line axis Q; sections without a non-full quadrant, or whose children
// are read through a symmetry, stay with the per-board kernel.
// Groups g = 6 Q + (RM + 1): line axis Q and the other quadrants with empty
// cells (RM = -1 none, 0..3 exactly that one, 4 several), one launch each.
constexpr int kLineGroups = 24;
struct SecLineWork {
  std::vector<SecLineTask> all;  // grouped by (Q, RM)
  size_t count[kLineGroups] = {};
  uint32_t warps[kLineGroups] = {};
  std::vector<SecTask> rest;     // per-board tasks, block0 renumbered
  uint32_t rest_blocks = 0;
  // D4: child sections that are not minimal, written out in their own
  // layout first (materialise_kernel) so their sections run by lines too.
  // Line tasks name them by offset into that buffer until rebased.
  std::vector<MatTask> mats;
  uint32_t mat_blocks = 0;
  uint64_t mat_values = 0;
  std::vector<std::pair<size_t, int>> mat_refs;  // (index into all, quadrant)
};

void split_line_work(const std::vector<SecTask>& tasks, SecLineWork* W, bool materialise = false) {
  const HostTables& t = host_tables();
  std::vector<SecLineTask> group[kLineGroups];
  std::vector<std::pair<size_t, int>> refs[kLineGroups];
  std::map<uint64_t, uint64_t> made;  // child count key -> offset in the buffer
  for (const SecTask& tk : tasks) {
    int Q = -1;
    uint32_t best = 0;
    bool ok = true;
    for (int q = 0; q < 4; q++) {
      if (!(tk.movable >> q & 1)) continue;
      if (tk.sym[q] != 0 && !materialise) ok = false;
      // the longest lines; on a tie the higher quadrant (its kernels hold fewer registers)
      if (tk.dim[q] >= best) best = tk.dim[q], Q = q;
    }
    if (Q < 0 || !ok) {
      SecTask rest = tk;
      rest.block0 = W->rest_blocks;
      W->rest_blocks += (uint32_t)((tk.size + kBlock - 1) / kBlock);
      W->rest.push_back(rest);
      continue;
    }
    SecLineTask L{};
    L.out = tk.out;
    uint32_t stride = 1;
    for (int q = 0; q < 4; q++) {
      L.child[q] = tk.child[q];
      for (int r = 0; r < 4; r++) L.cstride[q][r] = tk.cstride[q][r];
      L.dim[q] = tk.dim[q];
      L.stride[q] = stride;
      stride *= tk.dim[q];
      L.qoff[q] = tk.qoff[q];
    }
    L.mover = tk.mover;
    L.movable = tk.movable;
    L.prepared = tk.prepared;
    L.lines = (uint32_t)(tk.size / tk.dim[Q]);
    const uint32_t others = tk.movable & ~(1u << Q);
    const int rm = others == 0 ? -1 : (others & (others - 1)) ? 4 : __builtin_ctz(others);
    const int g = 6 * Q + rm + 1;
    for (int q = 0; q < 4; q++) {  // children read through a symmetry: their written-out copies
      if (!(tk.movable >> q & 1) || tk.sym[q] == 0) continue;
      uint8_t cbw[4][2];
      std::memcpy(cbw, tk.bw, sizeof cbw);
      cbw[q][tk.mover - 1]++;
      uint64_t key = 0, size = 1;
      for (int r = 0; r < 4; r++) key = key * 100 + cbw[r][0] * 10 + cbw[r][1];
      MatTask m{};
      for (int r = 0; r < 4; r++) {
        m.dim[r] = (uint32_t)t.qdim[cbw[r][0]][cbw[r][1]];
        m.qoff[r] = (uint16_t)t.qoff[cbw[r][0]][cbw[r][1]];
        size *= m.dim[r];
      }
      auto it = made.find(key);
      if (it == made.end()) {
        m.block0 = W->mat_blocks;
        m.sym = tk.sym[q];
        m.size = size;
        m.dst = W->mat_values;
        m.src = tk.child[q];
        for (int p = 0; p < 4; p++) m.sstride[p] = tk.cstride[q][p];
        W->mat_blocks += (uint32_t)((size + kBlock - 1) / kBlock);
        W->mat_values += size;
        W->mats.push_back(m);
        it = made.emplace(key, m.dst).first;
      }
      L.child[q] = (const pp_super*)(uintptr_t)it->second;  // an offset until rebased
      uint64_t cs = 1;
      for (int r = 0; r < 4; r++) {
        L.cstride[q][r] = cs;
        cs *= m.dim[r];
      }
      refs[g].push_back({group[g].size(), q});
    }
    L.warp0 = W->warps[g];
    W->warps[g] += (L.lines + 31) / 32;
    group[g].push_back(L);
  }
  for (int g = 0; g < kLineGroups; g++) {
    for (auto& rf : refs[g]) W->mat_refs.push_back({W->all.size() + rf.first, rf.second});
    W->count[g] = group[g].size();
    W->all.insert(W->all.end(), group[g].begin(), group[g].end());
  }
}

// Line tasks with their materialised children pointing into mat.
std::vector<SecLineTask> rebased_lines(const SecLineWork& W, pp_super* mat) {
  std::vector<SecLineTask> all = W.all;
  for (auto& rf : W.mat_refs) all[rf.first].child[rf.second] = mat + (uintptr_t)all[rf.first].child[rf.second];
  return all;
}

int launch_line_work(const SecLineWork& W, const SecLineTask* d_lines, const SecTask* d_rest, bool d4, pp_super* out,
                     pp_stream s, const MatTask* d_mats = nullptr, pp_super* mat = nullptr) {
  int rc = W.mats.empty() ? 0 : launch_materialise(d_mats, (int)W.mats.size(), W.mat_blocks, mat, s);
  if (!rc && !W.rest.empty()) rc = launch_sections(d_rest, (int)W.rest.size(), W.rest_blocks, out, s, d4);
  // a step's children are all raw, all prepared or all ready
  const bool ready = !W.all.empty() && W.all[0].prepared == 2;
  size_t off = 0;
  for (int g = 0; g < kLineGroups && !rc; g++) {
    rc = launch_section_lines(g / 6, g % 6 - 1, d_lines + off, (int)W.count[g], W.warps[g], out, s, ready);
    off += W.count[g];
  }
  return rc;
}

int run_section_lines(const std::vector<SecTask>& tasks, bool d4, pp_super* out, pp_stream s) {
  SecLineWork W;
  split_line_work(tasks, &W, d4);
  SecLineTask* dl = nullptr;
  SecTask* dr = nullptr;
  MatTask* dm = nullptr;
  pp_super* mat = nullptr;
  cudaError_t e = cudaSuccess;
  if (!W.mats.empty()) {
    e = cudaMallocAsync((void**)&mat, W.mat_values * sizeof(pp_super), s);
    if (!e) e = cudaMallocAsync((void**)&dm, W.mats.size() * sizeof(MatTask), s);
    if (!e) e = cudaMemcpyAsync(dm, W.mats.data(), W.mats.size() * sizeof(MatTask), cudaMemcpyHostToDevice, s);
  }
  std::vector<SecLineTask> all = rebased_lines(W, mat);
  if (!e && !all.empty()) {
    e = cudaMallocAsync((void**)&dl, all.size() * sizeof(SecLineTask), s);
    if (!e) e = cudaMemcpyAsync(dl, all.data(), all.size() * sizeof(SecLineTask), cudaMemcpyHostToDevice, s);
  }
  if (!e && !W.rest.empty()) {
    e = cudaMallocAsync((void**)&dr, W.rest.size() * sizeof(SecTask), s);
    if (!e) e = cudaMemcpyAsync(dr, W.rest.data(), W.rest.size() * sizeof(SecTask), cudaMemcpyHostToDevice, s);
  }
  int rc = e ? (int)e : launch_line_work(W, dl, dr, d4, out, s, dm, mat);
  if (dl) cudaFreeAsync(dl, s);
  if (dr) cudaFreeAsync(dr, s);
  if (dm) cudaFreeAsync(dm, s);
  if (mat) cudaFreeAsync(mat, s);
  return rc ? cuda_fail(rc, "section line launch") : PP_OK;
}

// Ready child records of slice n+1 for the parents of slice n: one line
// task per section held (at its layout offset, or at in_offsets[i] when
// given; absent sections skipped), the output laid out like the input.
// The public entry point keeps the uploaded task arrays of its recent
// argument sets, so a repeated call is launches only (and can be captured
// in a CUDA graph once it has run outside capture).
struct ReadyTasks {
  LineTask* d = nullptr;
  int ntasks = 0;
  uint32_t warps = 0;
};
std::mutex g_ready_mu;
std::map<std::string, ReadyTasks> g_ready_cache;
std::deque<std::string> g_ready_order;
constexpr size_t kReadyCacheEntries = 64;

void clear_ready_cache() {
  std::lock_guard<std::mutex> lock(g_ready_mu);
  for (auto& kv : g_ready_cache) cudaFree(kv.second.d);
  g_ready_cache.clear();
  g_ready_order.clear();
}

int prepare_ready(int n, bool d4, const pp_super* in, const uint64_t* in_offsets, uint64_t in_count,
                  pp_super* out, pp_stream s, bool cached = false) {
  std::string key;
  if (cached) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the offsets
    const size_t nsec = d4 ? slice_sections_d4(n + 1, nullptr).size() : slice_sections(n + 1, nullptr).size();
    for (size_t i = 0; in_offsets && i < nsec; i++) h = (h ^ in_offsets[i]) * 1099511628211ull;
    char buf[160];
    std::snprintf(buf, sizeof buf, "%d %d %p %p %llu %d %016llx", n, (int)d4, (const void*)in, (void*)out,
                  (unsigned long long)in_count, in_offsets != nullptr, (unsigned long long)h);
    key = buf;
    std::lock_guard<std::mutex> lock(g_ready_mu);
    auto it = g_ready_cache.find(key);
    if (it != g_ready_cache.end()) {
      const int rc = launch_ready(it->second.d, it->second.ntasks, it->second.warps, out, s);
      return rc ? cuda_fail(rc, "ready children") : PP_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
      return fail(PP_EINVAL, "ready children: run these arguments once outside stream capture first");
  }
  const HostTables& t = host_tables();
  uint64_t total = 0;
  auto secs = d4 ? slice_sections_d4(n + 1, &total) : slice_sections(n + 1, &total);
  std::vector<LineTask> tasks;
  std::vector<std::pair<uint64_t, uint64_t>> spans;  // [first, end) of every section held
  for (size_t i = 0; i < secs.size(); i++) {
    const pp_section_desc& d = secs[i];
    const uint64_t at = in_offsets ? in_offsets[i] : d.offset;
    if (at == PP_ABSENT) continue;
    LineTask tk{};
    uint64_t size = 1, stride = 1;
    int Q = 3;
    for (int q = 0; q < 4; q++) {
      tk.dim[q] = d.dim[q];
      tk.stride[q] = (uint32_t)stride;
      stride *= d.dim[q];
      tk.qoff[q] = (uint16_t)t.qoff[d.bw[q][0]][d.bw[q][1]];
      size *= d.dim[q];
    }
    for (int q = 2; q >= 0; q--)
      if (d.dim[q] > d.dim[Q]) Q = q;
    if (at > in_count || size > in_count - at)
      return fail(PP_EINVAL, "section %zu of slice %d lies past the %llu values given", i, n + 1,
                  (unsigned long long)in_count);
    if (size >= (1ull << 32)) return fail(PP_EINVAL, "section too large");
    spans.push_back({at, at + size});
    tk.lines = (uint32_t)(size / d.dim[Q]);
    tk.mover = (n % 2 == 0) ? 1u : 2u;  // the parents' mover
    tk.child = in + at;
    tk.out = at;
    tk.q = (uint32_t)Q;
    tasks.push_back(tk);
  }
  if (tasks.empty()) return PP_OK;
  // sections that share values would race (the pass may run in place)
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); i++)
    if (spans[i].first < spans[i - 1].second) return fail(PP_EINVAL, "two sections of the input overlap");
  std::stable_sort(tasks.begin(), tasks.end(), [](const LineTask& a, const LineTask& b) {
    return a.dim[a.q] != b.dim[b.q] ? a.dim[a.q] > b.dim[b.q] : a.q < b.q;
  });
  uint32_t warp = 0;
  for (size_t i = 0; i < tasks.size(); i++) {
    if (i > 0 && tasks[i].q != tasks[i - 1].q) warp = (warp + kLineWarps - 1) / kLineWarps * kLineWarps;
    tasks[i].warp0 = warp;
    warp += (tasks[i].lines + 31) / 32;
  }
  LineTask* d = nullptr;
  if (cached) {
    cudaError_t e = cudaMalloc((void**)&d, tasks.size() * sizeof(LineTask));
    if (!e) e = cudaMemcpy(d, tasks.data(), tasks.size() * sizeof(LineTask), cudaMemcpyHostToDevice);
    if (e) {
      if (d) cudaFree(d);
      return cuda_fail(e, "ready children tasks");
    }
    std::lock_guard<std::mutex> lock(g_ready_mu);
    if (g_ready_cache.size() >= kReadyCacheEntries) {  // the oldest goes (cudaFree waits for its launches)
      cudaFree(g_ready_cache[g_ready_order.front()].d);
      g_ready_cache.erase(g_ready_order.front());
      g_ready_order.pop_front();
    }
    g_ready_cache[key] = ReadyTasks{d, (int)tasks.size(), warp};
    g_ready_order.push_back(key);
    const int rc = launch_ready(d, (int)tasks.size(), warp, out, s);
    return rc ? cuda_fail(rc, "ready children") : PP_OK;
  }
  cudaError_t e = cudaMallocAsync((void**)&d, tasks.size() * sizeof(LineTask), s);
  if (!e) e = cudaMemcpyAsync(d, tasks.data(), tasks.size() * sizeof(LineTask), cudaMemcpyHostToDevice, s);
  int rc = e ? (int)e : launch_ready(d, (int)tasks.size(), warp, out, s);
  if (d) cudaFreeAsync(d, s);
  return rc ? cuda_fail(rc, "ready children") : PP_OK;
}

int slice_step(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
               const pp_batch_opts* opts, pp_stream s, bool d4, const uint64_t* in_offsets = nullptr,
               uint64_t in_count = 0) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 36) return fail(PP_EINVAL, "slice %d out of range", n);
  if (in_offsets && n > 34) return fail(PP_EINVAL, "sparse input is for slices below 35");
  const int stage = opts ? opts->stage_children : 0;
  // slice 35 without slice 36: children evaluated on demand (full layout, by lines)
  const bool on_demand = n == 35 && !in_values && !d4 && stage != 2;
  if (n < 36 && !on_demand && (!in_values || !aligned32(in_values)))
    return fail(PP_EINVAL, "slice %d needs slice %d values (32-byte aligned)", n, n + 1);
  if (!out_values || !aligned32(out_values)) return fail(PP_EINVAL, "output must be non-null and 32-byte aligned");
  auto secs = d4 ? slice_sections_d4(n, nullptr) : slice_sections(n, nullptr);
  std::vector<int> which;
  for (size_t i = 0; i < secs.size(); i++)
    if (!filter || filter[i]) which.push_back((int)i);
  if (n == 36 && stage != 2) return run_line35(secs, which, nullptr, nullptr, filter != nullptr, out_values, s, d4, 36);
  if (n == 35 && stage != 2)
    return run_line35(secs, which, in_values, nullptr, filter != nullptr, out_values, s, d4);
  std::vector<SecTask> tasks;
  uint32_t blocks = 0;
  int rc = build_tasks(n, secs, which, in_values, nullptr, filter != nullptr, &tasks, &blocks, d4, in_offsets, in_count);
  if (rc) return rc;
  // Below slice 35, when the step writes at least as many boards as its
  // input holds, the input is first turned into ready records in a
  // stream-ordered temporary (one pass over the input) and the boards skip
  // their rmax and their immediate-win lines; otherwise the boards read the
  // input as it is.
  pp_super* prep = nullptr;
  if (n < 35) {
    uint64_t in_n = in_offsets ? in_count : 0, out_n = 0;
    if (!in_offsets) (d4 ? slice_sections_d4(n + 1, &in_n) : slice_sections(n + 1, &in_n));
    for (const SecTask& t : tasks) out_n += t.size;
    if (in_n && out_n >= in_n && cudaMallocAsync((void**)&prep, in_n * sizeof(pp_super), s) == cudaSuccess) {
      if ((rc = prepare_ready(n, d4, in_values, in_offsets, in_n, prep, s))) {
        cudaFreeAsync(prep, s);
        return rc;
      }
      for (SecTask& t : tasks) {
        for (int q = 0; q < 4; q++)
          if (t.child[q]) t.child[q] = prep + (t.child[q] - in_values);
        t.prepared = 2;
      }
    } else {
      cudaGetLastError();  // no room for the temporary: read the input as it is
      prep = nullptr;
    }
  }
  if (n < 35 && stage != 2)
    rc = run_section_lines(tasks, d4, out_values, s);
  else
    rc = run_tasks(tasks, blocks, out_values, s, d4);
  if (prep) cudaFreeAsync(prep, s);
  return rc;
}

}  // namespace
}  // namespace pp

extern "C" {

int pp_section_compute(int n, const pp_section_desc* parent, const pp_super* const d_child[4], pp_super* d_out,
                       pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 36 || !parent || !valid_section(n, parent))
    return fail(PP_EINVAL, "section does not belong to slice %d (counts or dims)", n);
  if (!d_out || !aligned32(d_out)) return fail(PP_EINVAL, "output must be non-null and 32-byte aligned");
  const pp_super* none[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<pp_section_desc> one(1, *parent);
  if (n == 36) return run_line35(one, {0}, nullptr, nullptr, true, d_out, s, false, 36);
  if (n == 35) return run_line35(one, {0}, nullptr, d_child ? d_child : none, true, d_out, s);
  std::vector<SecTask> tasks;
  uint32_t blocks = 0;
  int rc = build_tasks(n, one, {0}, nullptr, d_child ? d_child : none, true, &tasks, &blocks);
  if (rc) return rc;
  if (n < 35) return run_section_lines(tasks, false, d_out, s);
  return run_tasks(tasks, blocks, d_out, s);
}

int pp_section_compute_desc(int n, const pp_section_desc* parent, const pp_super* const d_child[4],
                            const pp_section_desc* const child_desc[4], pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 36 || !parent || !valid_section(n, parent))
    return fail(PP_EINVAL, "section does not belong to slice %d (counts or dims)", n);
  if (n < 36 && d_child) {
    if (!child_desc) return fail(PP_EINVAL, "child descriptors are required with child values");
    const int m = (n % 2 == 0) ? 0 : 1;  // the mover's colour: black on an even number of stones
    for (int q = 0; q < 4; q++) {
      if (parent->bw[q][0] + parent->bw[q][1] >= 9) continue;  // full quadrant: no move there
      const pp_section_desc* c = child_desc[q];
      if (!c || !d_child[q]) return fail(PP_EINVAL, "quadrant %d is not full: its child section is needed", q);
      uint8_t want[4][2];
      std::memcpy(want, parent->bw, sizeof want);
      want[q][m]++;
      if (std::memcmp(c->bw, want, sizeof want))
        return fail(PP_EINVAL, "child descriptor %d: counts differ from the parent's with one more stone in quadrant %d",
                    q, q);
      if (!valid_section(n + 1, c))
        return fail(PP_EINVAL, "child descriptor %d is not a section of slice %d (dims)", q, n + 1);
    }
  }
  return pp_section_compute(n, parent, d_child, d_out, s);
}

int pp_slice_step(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                  const pp_batch_opts* opts, pp_stream s) {
  return slice_step(n, in_values, out_values, filter, opts, s, false);
}

int pp_d4_slice_step(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                     const pp_batch_opts* opts, pp_stream s) {
  return slice_step(n, in_values, out_values, filter, opts, s, true);
}

int pp_slice_step_sparse(int n, int d4, const pp_super* in_values, const uint64_t* in_offsets, uint64_t in_count,
                         pp_super* out_values, const uint8_t* filter, const pp_batch_opts* opts, pp_stream s) {
  if (!in_offsets) return fail(PP_EINVAL, "null input offsets");
  return slice_step(n, in_values, out_values, filter, opts, s, d4 != 0, in_offsets, in_count);
}

int pp_slice_children(int n, int d4, const uint8_t* filter, uint8_t* child_filter) {
  if (n < 0 || n > 35) return fail(PP_EINVAL, "slice %d has no child slice", n);
  if (!child_filter) return fail(PP_EINVAL, "null child filter");
  auto secs = d4 ? slice_sections_d4(n, nullptr) : slice_sections(n, nullptr);
  auto next = d4 ? slice_sections_d4(n + 1, nullptr) : slice_sections(n + 1, nullptr);
  std::memset(child_filter, 0, next.size());
  const int mover = (n % 2 == 0) ? 1 : 2;
  for (size_t i = 0; i < secs.size(); i++) {
    if (filter && !filter[i]) continue;
    for (int q = 0; q < 4; q++) {
      if (secs[i].bw[q][0] + secs[i].bw[q][1] >= 9) continue;
      uint8_t cbw[4][2];
      std::memcpy(cbw, secs[i].bw, sizeof cbw);
      cbw[q][mover - 1]++;
      if (d4) {
        uint8_t least[4][2];
        least_image(cbw, least);
        std::memcpy(cbw, least, sizeof cbw);
      }
      int ci = section_index(next, cbw);
      if (ci < 0) return fail(PP_EINVAL, "child section of slice %d not found", n + 1);
      child_filter[ci] = 1;
    }
  }
  return PP_OK;
}

int pp_d4_slice_sections(int n, pp_section_desc* out, int max, uint64_t* total) {
  if (n < 0 || n > 36) return -fail(PP_EINVAL, "slice %d out of range", n);
  auto secs = slice_sections_d4(n, total);
  for (int i = 0; out && i < max && i < (int)secs.size(); i++) out[i] = secs[i];
  return (int)secs.size();
}

}  // extern "C"

struct pp_slice_plan {
  int n = 0;
  bool d4 = false;               // D4-reduced slices
  bool line = false;             // slice-35 line kernel (else one thread per board)
  int persistent = 2;            // 1 persistent grid with a work counter, 2 one block per 256 boards
  int ctas_per_sm = 0;
  int largest_first = 0;
  pp_super* out = nullptr;
  std::vector<SecTask> natural;  // tasks in section order
  SecTask* d_tasks = nullptr;    // tasks in the configured order
  int ntasks = 0;
  uint32_t blocks = 0;
  uint32_t* d_counter = nullptr;
  Line35Work lw;
  LineTask* d_ltasks = nullptr;
  pp_super* tmp = nullptr;
  // below slice 35: the same sections by lines (stage_children 1) or one
  // thread per board (2)
  bool has_slines = false, slines = false;
  SecLineWork sw;
  SecLineTask* d_sl = nullptr;
  SecTask* d_srest = nullptr;
  MatTask* d_mats = nullptr;  // D4: children written out in their own layout at each run
  pp_super* mat = nullptr;
  int prepared = 0;   // the input holds prepared child values (pp_prepare_children)
  std::string shape;  // autotuner cache key: slice, layout, the sections kept, prepared input

  // device buffers go with the plan, also when its creation fails part-way
  ~pp_slice_plan() {
    cudaFree(d_tasks);
    cudaFree(d_counter);
    cudaFree(d_ltasks);
    cudaFree(tmp);
    cudaFree(d_sl);
    cudaFree(d_srest);
    cudaFree(d_mats);
    cudaFree(mat);
  }
};

namespace {

int upload_order(pp_slice_plan* P) {
  std::vector<SecTask> t = P->natural;
  if (P->largest_first) order_largest_first(&t);
  cudaError_t e = cudaMemcpy(P->d_tasks, t.data(), t.size() * sizeof(SecTask), cudaMemcpyHostToDevice);
  return e ? cuda_fail(e, "slice plan task upload") : PP_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

int slice_plan_create(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                      const pp_batch_opts* opts, pp_slice_plan** plan, bool d4, const uint64_t* in_offsets = nullptr,
                      uint64_t in_count = 0) {
  if (!plan) return fail(PP_EINVAL, "null plan pointer");
  *plan = nullptr;
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 36) return fail(PP_EINVAL, "slice %d out of range", n);
  if (in_offsets && n > 34) return fail(PP_EINVAL, "sparse input is for slices below 35");
  const int stage = opts ? opts->stage_children : 0;
  const bool on_demand = n == 35 && !in_values && !d4 && stage != 2;  // slice 36 evaluated in the kernel
  if (n < 36 && !on_demand && (!in_values || !aligned32(in_values)))
    return fail(PP_EINVAL, "slice %d needs slice %d values (32-byte aligned)", n, n + 1);
  if (!out_values || !aligned32(out_values)) return fail(PP_EINVAL, "output must be non-null and 32-byte aligned");
  auto P = std::make_unique<pp_slice_plan>();
  P->n = n;
  P->d4 = d4;
  P->out = out_values;
  P->line = (n == 35 || n == 36) && stage != 2;
  auto secs = d4 ? slice_sections_d4(n, nullptr) : slice_sections(n, nullptr);
  std::vector<int> which;
  for (size_t i = 0; i < secs.size(); i++)
    if (!filter || filter[i]) which.push_back((int)i);
  int rc;
  if (P->line) {
    rc = n == 36 ? build_line36(secs, which, filter != nullptr, &P->lw)
                 : build_line35(secs, which, in_values, nullptr, filter != nullptr, &P->lw, d4);
    if (rc) return rc;
    if (!P->lw.others.empty()) {  // D4: sections read through a symmetry, one thread per board
      if ((rc = other_tasks(P->lw, secs, in_values, &P->natural, &P->blocks))) return rc;
      P->ntasks = (int)P->natural.size();
      cudaError_t e = cudaMalloc(&P->d_tasks, P->ntasks * sizeof(SecTask));
      if (!e) e = cudaMemcpy(P->d_tasks, P->natural.data(), P->ntasks * sizeof(SecTask), cudaMemcpyHostToDevice);
      if (e) return cuda_fail(e, "slice plan tasks");
    }
    cudaError_t e = cudaMalloc(&P->tmp, std::max<uint64_t>(P->lw.tmp_size, 1) * sizeof(pp_super));
    if (!e) e = cudaMalloc(&P->d_ltasks, std::max<size_t>(P->lw.all.size(), 1) * sizeof(LineTask));
    if (!e) {
      auto all = rebased(P->lw, P->tmp);
      e = cudaMemcpy(P->d_ltasks, all.data(), all.size() * sizeof(LineTask), cudaMemcpyHostToDevice);
    }
    if (e) return cuda_fail(e, "slice plan buffers");
  } else {
    rc = build_tasks(n, secs, which, in_values, nullptr, filter != nullptr, &P->natural, &P->blocks, d4, in_offsets,
                     in_count);
    if (rc) return rc;
    P->ntasks = (int)P->natural.size();
    cudaError_t e = cudaMalloc(&P->d_tasks, std::max(P->ntasks, 1) * sizeof(SecTask));
    if (!e) e = cudaMalloc(&P->d_counter, sizeof(uint32_t));
    if (e) return cuda_fail(e, "slice plan buffers");
    if (opts) {
      P->persistent = opts->persistent == 1 ? 1 : 2;
      P->ctas_per_sm = opts->ctas_per_sm;
      P->largest_first = opts->largest_first;
    }
    if ((rc = upload_order(P.get()))) return rc;
    if (n < 35) {
      split_line_work(P->natural, &P->sw, d4);
      e = cudaSuccess;
      if (!P->sw.mats.empty()) {
        e = cudaMalloc(&P->mat, P->sw.mat_values * sizeof(pp_super));
        if (!e) e = cudaMalloc(&P->d_mats, P->sw.mats.size() * sizeof(MatTask));
        if (!e) e = cudaMemcpy(P->d_mats, P->sw.mats.data(), P->sw.mats.size() * sizeof(MatTask), cudaMemcpyHostToDevice);
      }
      if (!e && !P->sw.all.empty()) {
        auto all = rebased_lines(P->sw, P->mat);
        e = cudaMalloc(&P->d_sl, all.size() * sizeof(SecLineTask));
        if (!e) e = cudaMemcpy(P->d_sl, all.data(), all.size() * sizeof(SecLineTask), cudaMemcpyHostToDevice);
      }
      if (!e && !P->sw.rest.empty()) {
        e = cudaMalloc(&P->d_srest, P->sw.rest.size() * sizeof(SecTask));
        if (!e) e = cudaMemcpy(P->d_srest, P->sw.rest.data(), P->sw.rest.size() * sizeof(SecTask), cudaMemcpyHostToDevice);
      }
      if (e) return cuda_fail(e, "slice plan line buffers");
      P->has_slines = true;
      P->slines = stage != 2;
    }
    uint64_t boards = 0, h = 1469598103934665603ull;  // FNV-1a over the kept sections' counts
    for (const SecTask& t : P->natural) {
      boards += t.size;
      for (int q = 0; q < 4; q++)
        for (int c = 0; c < 2; c++) h = (h ^ t.bw[q][c]) * 1099511628211ull;
    }
    char buf[128];
    std::snprintf(buf, sizeof buf, "slice=%d d4=%d sections=%d boards=%llu h=%016llx", n, (int)d4, P->ntasks,
                  (unsigned long long)boards, (unsigned long long)h);
    P->shape = buf;
    P->shape += " prep=0";
  }
  *plan = P.release();
  return PP_OK;
}

}  // namespace

extern "C" {

int pp_slice_plan_create(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                         const pp_batch_opts* opts, pp_slice_plan** plan) {
  return slice_plan_create(n, in_values, out_values, filter, opts, plan, false);
}

int pp_d4_slice_plan_create(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                            const pp_batch_opts* opts, pp_slice_plan** plan) {
  return slice_plan_create(n, in_values, out_values, filter, opts, plan, true);
}

int pp_slice_plan_create_sparse(int n, int d4, const pp_super* in_values, const uint64_t* in_offsets,
                                uint64_t in_count, pp_super* out_values, const uint8_t* filter,
                                const pp_batch_opts* opts, pp_slice_plan** plan) {
  if (!in_offsets) {
    if (plan) *plan = nullptr;
    return fail(PP_EINVAL, "null input offsets");
  }
  return slice_plan_create(n, in_values, out_values, filter, opts, plan, d4 != 0, in_offsets, in_count);
}

int pp_slice_plan_configure(pp_slice_plan* P, const pp_batch_opts* opts) {
  if (!P || !opts) return fail(PP_EINVAL, "null plan or options");
  if (P->line) return PP_OK;  // the line kernel has one configuration
  if (P->has_slines && opts->stage_children == 1) P->slines = true;
  if (P->has_slines && opts->stage_children == 2) P->slines = false;
  P->persistent = opts->persistent == 1 ? 1 : 2;
  P->ctas_per_sm = opts->ctas_per_sm;
  if (P->persistent == 1 && persistent_section_blocks(P->ctas_per_sm, P->d4) <= 0)
    return fail(PP_ECUDA, "persistent section kernel does not fit");
  if (opts->largest_first != P->largest_first) {
    P->largest_first = opts->largest_first;
    return upload_order(P);
  }
  return PP_OK;
}

int pp_slice_plan_run(pp_slice_plan* P, pp_stream s) {
  if (!P) return fail(PP_EINVAL, "null plan");
  int rc;
  if (P->line) {
    rc = P->ntasks ? launch_sections(P->d_tasks, P->ntasks, P->blocks, P->out, s, true) : 0;
    if (!rc && !P->lw.all.empty()) rc = launch_line35_work(P->lw, P->d_ltasks, P->tmp, P->out, s);
  } else if (P->slines) {
    rc = launch_line_work(P->sw, P->d_sl, P->d_srest, P->d4, P->out, s, P->d_mats, P->mat);
  } else if (P->persistent == 1) {
    rc = launch_sections_persistent(P->d_tasks, P->ntasks, P->blocks, P->out, P->d_counter,
                                    persistent_section_blocks(P->ctas_per_sm, P->d4), s, P->d4);
  } else {
    rc = launch_sections(P->d_tasks, P->ntasks, P->blocks, P->out, s, P->d4);
  }
  return rc ? cuda_fail(rc, "slice plan launch") : PP_OK;
}

int pp_slice_plan_autotune(pp_slice_plan* P, pp_stream s, pp_batch_opts* chosen) {
  if (!P) return fail(PP_EINVAL, "null plan");
  pp_batch_opts win{P->persistent, 0, P->ctas_per_sm, P->line || P->slines ? 1 : 2, P->largest_first};
  if (!P->line) {
    const std::string key = tune_device_tag() + " " + P->shape;
    pp_batch_opts cached;
    if (tune_lookup(key, &cached)) {
      int rc = pp_slice_plan_configure(P, &cached);
      if (!rc && chosen) *chosen = cached;
      return rc;
    }
    std::vector<pp_batch_opts> cands = {{2, 0, 0, 2, 0}, {2, 0, 0, 2, 1}, {1, 0, 0, 2, 1}, {1, 0, 1, 2, 1}, {1, 0, 2, 2, 1}};
    if (P->has_slines) cands.push_back({2, 0, 0, 1, 0});  // by lines
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(PP_ECUDA, "autotune events");
    float best = 1e30f;
    for (const auto& c : cands) {
      if (pp_slice_plan_configure(P, &c) || pp_slice_plan_run(P, s)) continue;
      cudaEventRecord(e0, s);
      int rc = 0;
      for (int r = 0; r < 2 && !rc; r++) rc = pp_slice_plan_run(P, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) || rc) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms, win = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = pp_slice_plan_configure(P, &win);
    if (rc) return rc;
    if (best < 1e30f) tune_record(key, win);
  }
  if (chosen) *chosen = win;
  return PP_OK;
}

void pp_slice_plan_destroy(pp_slice_plan* P) { delete P; }

int pp_slice_plan_set_prepared(pp_slice_plan* P, int prepared) {
  if (!P) return fail(PP_EINVAL, "null plan");
  if (prepared < 0 || prepared > 2) return fail(PP_EINVAL, "prepared must be 0, 1 or 2");
  if (P->n >= 35) return fail(PP_EINVAL, "prepared children are for slices below 35 (this plan: slice %d)", P->n);
  if (prepared == P->prepared) return PP_OK;
  P->prepared = prepared;
  for (SecTask& t : P->natural) t.prepared = (uint8_t)prepared;
  for (SecTask& t : P->sw.rest) t.prepared = (uint8_t)prepared;
  for (SecLineTask& t : P->sw.all) t.prepared = (uint8_t)prepared;
  P->shape = P->shape.substr(0, P->shape.size() - 1) + std::to_string(prepared);
  int rc = upload_order(P);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (P->d_sl && !P->sw.all.empty()) {
    auto all = rebased_lines(P->sw, P->mat);
    e = cudaMemcpy(P->d_sl, all.data(), all.size() * sizeof(SecLineTask), cudaMemcpyHostToDevice);
  }
  if (!e && P->d_srest && !P->sw.rest.empty())
    e = cudaMemcpy(P->d_srest, P->sw.rest.data(), P->sw.rest.size() * sizeof(SecTask), cudaMemcpyHostToDevice);
  return e ? cuda_fail(e, "slice plan task upload") : PP_OK;
}

int pp_prepare_children(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n && (!d_in || !d_out || !aligned16(d_in) || !aligned16(d_out)))
    return fail(PP_EINVAL, "values must be non-null 16-byte aligned device arrays");
  int e = launch_prepare(d_in, n, d_out, s);
  return e ? cuda_fail(e, "prepare children") : PP_OK;
}

int pp_prepare_children_ready(int n, int d4, const pp_super* d_in, const uint64_t* in_offsets, uint64_t in_count,
                              pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 34) return fail(PP_EINVAL, "ready children are for slices 0..34 (got %d)", n);
  if (!d_in || !d_out || !aligned32(d_in) || !aligned32(d_out))
    return fail(PP_EINVAL, "values must be non-null 32-byte aligned device arrays");
  return prepare_ready(n, d4 != 0, d_in, in_offsets, in_count, d_out, s, true);
}

int pp_super_digest(const pp_super* d_values, uint64_t n, uint64_t* d_acc, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if ((n && (!d_values || !aligned16(d_values))) || !d_acc || ((uintptr_t)d_acc & 7))
    return fail(PP_EINVAL, "bad digest arguments");
  int e = launch_digest(d_values, n, d_acc, s);
  return e ? cuda_fail(e, "digest") : PP_OK;
}

// Building blocks, exposed for unit tests of the device functions.
int pp_five_masks(const uint64_t* d_boards, int n, uint64_t* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  int e = launch_five_masks(d_boards, n, d_out, s);
  return e ? cuda_fail(e, "five masks") : PP_OK;
}

int pp_rmax(const pp_super* d_in, int n, pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  int e = launch_rmax(d_in, n, d_out, s);
  return e ? cuda_fail(e, "rmax") : PP_OK;
}

int pp_symmetry_transform(const pp_super* d_in, int n, int sym, const int turns[4], pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (sym < 0 || sym > 7 || !turns) return fail(PP_EINVAL, "symmetry %d out of range or null turns", sym);
  uint32_t packed = 0;
  for (int q = 0; q < 4; q++) {
    if (turns[q] < 0 || turns[q] > 3) return fail(PP_EINVAL, "turns[%d] = %d out of range", q, turns[q]);
    packed |= (uint32_t)turns[q] << (2 * q);
  }
  int e = launch_symmetry(d_in, n, sym, packed, d_out, s);
  return e ? cuda_fail(e, "symmetry transform") : PP_OK;
}

int pp_symmetry_info(int sym, int qmap[4], int* reflects) {
  if (sym < 0 || sym > 7) return fail(PP_EINVAL, "symmetry %d out of range", sym);
  for (int q = 0; q < 4 && qmap; q++) qmap[q] = sym_qmap(sym, q);
  if (reflects) *reflects = sym_reflects(sym) ? 1 : 0;
  return PP_OK;
}

int pp_symmetry_board(uint64_t board, int sym, uint64_t* out) {
  if (sym < 0 || sym > 7 || !out) return fail(PP_EINVAL, "symmetry %d out of range or null output", sym);
  uint64_t r = 0;
  for (int q = 0; q < 4; q++) {
    const int code = (int)((board >> (16 * q)) & 0xFFFFu);
    if (code >= kQStates) return fail(PP_EINVAL, "quadrant %d code %d out of range", q, code);
    r |= (uint64_t)symmetry_pattern(sym, code) << (16 * sym_qmap(sym, q));
  }
  *out = r;
  return PP_OK;
}

int pp_shift(const pp_super* d_in, int n, int q, int u, pp_super* d_out, pp_stream s) {
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (q < 0 || q > 3 || u < 0 || u > 3) return fail(PP_EINVAL, "axis %d / turns %d out of range", q, u);
  int e = launch_shift(d_in, n, q, u, d_out, s);
  return e ? cuda_fail(e, "shift") : PP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Out-of-core slice steps (paper, "Data layout and distribution": slice n
// reads only slice n+1, so a slice larger than the device is made in batches
// while slice n+1 lives partly in host memory).
// ---------------------------------------------------------------------------
struct pp_stager {
  int n = 0;
  bool d4 = false;
  int prepared = 0;
  pp_super* base = nullptr;
  uint64_t base_count = 0;
  std::vector<uint64_t> dev_off;       // per section of slice n+1
  std::vector<const pp_super*> host;   // per section of slice n+1
  std::vector<pp_section_desc> secs, next;
  uint64_t stage_at = 0, half = 0;     // two staging halves of `half` values each
  int turn = 0;
  bool used[2] = {false, false};
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  ~pp_stager() {
    for (int h = 0; h < 2; h++) {
      if (copied[h]) cudaEventDestroy(copied[h]);
      if (freed[h]) cudaEventDestroy(freed[h]);
    }
  }
};

extern "C" {

int pp_stager_create(int n, int d4, pp_super* d_base, uint64_t base_count, const uint64_t* dev_offsets,
                     const pp_super* const* h_src, uint64_t stage_at, uint64_t stage_values, int prepared,
                     pp_stager** out) {
  if (!out) return fail(PP_EINVAL, "null stager pointer");
  *out = nullptr;
  if (!g_ready) return fail(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || n > 34) return fail(PP_EINVAL, "out-of-core steps are for slices below 35 (got %d)", n);
  if (!d_base || !aligned32(d_base) || !dev_offsets || !h_src)
    return fail(PP_EINVAL, "null or misaligned base, offsets or host pointers");
  if (prepared < 0 || prepared > 2) return fail(PP_EINVAL, "prepared must be 0, 1 or 2");
  if (stage_at > base_count || stage_values > base_count - stage_at)
    return fail(PP_EINVAL, "staging room lies outside the base array");
  auto S = std::make_unique<pp_stager>();
  S->n = n;
  S->d4 = d4 != 0;
  S->prepared = prepared;
  S->base = d_base;
  S->base_count = base_count;
  S->secs = S->d4 ? slice_sections_d4(n, nullptr) : slice_sections(n, nullptr);
  S->next = S->d4 ? slice_sections_d4(n + 1, nullptr) : slice_sections(n + 1, nullptr);
  S->dev_off.assign(dev_offsets, dev_offsets + S->next.size());
  S->host.assign(h_src, h_src + S->next.size());
  for (size_t i = 0; i < S->next.size(); i++) {
    const uint64_t off = S->dev_off[i], size = section_boards(S->next[i]);
    if (off == PP_ABSENT) continue;
    if (off > base_count || size > base_count - off)
      return fail(PP_EINVAL, "device section %zu lies outside the base array", i);
    if (off < stage_at + stage_values && off + size > stage_at)
      return fail(PP_EINVAL, "device section %zu overlaps the staging room", i);
  }
  S->stage_at = stage_at;
  S->half = stage_values / 2;
  for (int h = 0; h < 2; h++) {
    cudaError_t e = cudaEventCreateWithFlags(&S->copied[h], cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&S->freed[h], cudaEventDisableTiming);
    if (e) return cuda_fail(e, "stager events");
  }
  *out = S.release();
  return PP_OK;
}

int pp_stager_step(pp_stager* S, pp_super* d_out, const uint8_t* filter, pp_stream s, pp_stream copy_s,
                   uint64_t* staged_values) {
  if (!S) return fail(PP_EINVAL, "null stager");
  if (!d_out || !aligned32(d_out)) return fail(PP_EINVAL, "output must be non-null and 32-byte aligned");
  if (staged_values) *staged_values = 0;
  std::vector<int> which;
  for (size_t i = 0; i < S->secs.size(); i++)
    if (!filter || filter[i]) which.push_back((int)i);
  // the child sections the kept sections read
  std::vector<uint8_t> need(S->next.size(), 0);
  int rc = pp_slice_children(S->n, S->d4 ? 1 : 0, filter, need.data());
  if (rc) return rc;
  std::vector<uint64_t> offs = S->dev_off;
  std::vector<std::pair<int, uint64_t>> copies;  // (section, staged position)
  const int h = S->turn;
  uint64_t at = S->stage_at + (uint64_t)h * S->half, used = 0;
  for (size_t i = 0; i < S->next.size(); i++) {
    if (!need[i] || offs[i] != PP_ABSENT) continue;
    if (!S->host[i]) return fail(PP_EINVAL, "slice %d section %zu is read but held nowhere", S->n + 1, i);
    const uint64_t size = section_boards(S->next[i]);
    if (size > S->half - used)
      return fail(PP_ENOMEM, "the host sections this batch reads need more than half the staging room (%llu values)",
                  (unsigned long long)S->half);
    offs[i] = at + used;
    copies.push_back({(int)i, at + used});
    used += size;
  }
  std::vector<SecTask> tasks;
  uint32_t blocks = 0;
  rc = build_tasks(S->n, S->secs, which, S->base, nullptr, true, &tasks, &blocks, S->d4, offs.data(), S->base_count);
  if (rc) return rc;
  for (SecTask& t : tasks) t.prepared = (uint8_t)S->prepared;
  if (!copies.empty()) {
    // the half is free once the step that last read it is done
    cudaError_t e = S->used[h] ? cudaStreamWaitEvent(copy_s, S->freed[h], 0) : cudaSuccess;
    for (auto& c : copies)
      if (!e)
        e = cudaMemcpyAsync(S->base + c.second, S->host[c.first], section_boards(S->next[c.first]) * sizeof(pp_super),
                            cudaMemcpyHostToDevice, copy_s);
    if (!e) e = cudaEventRecord(S->copied[h], copy_s);
    if (!e) e = cudaStreamWaitEvent(s, S->copied[h], 0);
    if (e) return cuda_fail(e, "staging copies");
  }
  rc = run_section_lines(tasks, S->d4, d_out, s);
  if (rc) return rc;
  cudaError_t e = cudaEventRecord(S->freed[h], s);
  if (e) return cuda_fail(e, "stager event");
  S->used[h] = true;
  S->turn ^= 1;
  if (staged_values) *staged_values = used;
  return PP_OK;
}

void pp_stager_destroy(pp_stager* S) { delete S; }

}  // extern "C"
