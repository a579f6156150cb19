// pp_noalloc.cu -- a midgame entry point that never allocates device memory.
//
// Who needs it: callers that may not call cudaMalloc or any allocator after
// start-up -- a host application whose device memory is wholly owned by
// another framework's pool, a latency-critical service thread that cannot
// afford the device-wide synchronisation a cudaMalloc/cudaFree implies, or a
// plugin host that forbids allocation once it is running.  They pass device
// inputs and outputs only; all scratch space (descriptors, fill lists and the
// fill tables) lives in one fixed array of this file, so the call itself
// allocates nothing.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pp_internal.h"

namespace pp {
namespace {

// The scratch array.  It is a file-scope device variable: every GPU on which
// this file's module is loaded keeps these bytes until the process exits.
constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address, per device ordinal

// Host-side fill lists and child ranks for one (empty cells, root mover):
// the same contents as the device lists of the allocating path, kept on the
// host and copied into the scratch array, so nothing is allocated on the
// device.
std::map<std::pair<int, int>, FillLists> g_host_lists;

const FillLists& host_lists(int k, int mover) {
  auto key = std::make_pair(k, mover);
  auto it = g_host_lists.find(key);
  if (it != g_host_lists.end()) return it->second;
  FillLists L;
  build_fill_lists(k, mover, &L);
  return g_host_lists[key] = std::move(L);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Set-up, once per device, with that device current: the device address of
// the scratch array (in host code its name is only a host-side stand-in).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return report_error(PP_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(PP_EINVAL, "device ordinal out of range");
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e || !p) {
      return report_error(PP_ECUDA, (std::string("scratch address: ") + cudaGetErrorString(e)).c_str());
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" int pp_midgame_solve_noalloc(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty,
                                        pp_stream s) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!tables_ready()) return report_error(PP_ENOTINIT, "pp_init has not run");
  if (n < 0 || max_empty < 0 || max_empty > kMaxEmpty)
    return report_error(PP_EINVAL, "bad board count or max_empty");
  if (n == 0) return PP_OK;
  if (!d_boards || !d_out || ((uintptr_t)d_boards & 15) || ((uintptr_t)d_out & 15))
    return report_error(PP_EINVAL, "boards and output must be non-null, 16-byte aligned device arrays");
  unsigned char* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;

  // the boards, read back once for host-side validation and scheduling
  std::vector<uint64_t> h(n);
  cudaError_t e = cudaMemcpyAsync(h.data(), d_boards, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return report_error(PP_ECUDA, cudaGetErrorString(e));

  std::vector<MidBoard> boards(n);
  int kmax = 0;
  for (int i = 0; i < n; i++) {
    rc = validate_midgame_board(h[i], max_empty, &boards[i], i);
    if (rc) return rc;
    kmax = boards[i].k > (uint32_t)kmax ? (int)boards[i].k : kmax;
  }
  // scratch layout: [level lists + child ranks][board descriptors][segments]
  // [compact fill tables][five tables]
  std::map<std::pair<int, int>, size_t> list_at, ranks_at;  // byte offsets of each list set
  size_t off = 0;
  for (int i = 0; i < n; i++) {
    auto key = std::make_pair((int)boards[i].k, (int)boards[i].mover);
    if (list_at.count(key)) continue;
    const FillLists& L = host_lists(key.first, key.second);
    list_at[key] = off;
    off = align256(off + L.flat.size() * sizeof(uint64_t));
    ranks_at[key] = off;
    off = align256(off + L.ranks.size() * sizeof(uint32_t));
  }
  const size_t boards_at = off;
  off = align256(off + n * sizeof(MidBoard));
  const size_t segs_at = off;
  std::vector<MidSeg> segs;
  struct Level {
    int seg0, nsegs;
    uint32_t blocks;
  };
  std::vector<Level> levels;
  for (int m = kmax; m >= 0; m--) {
    Level lv{(int)segs.size(), 0, 0};
    for (int i = 0; i < n; i++) {
      if ((int)boards[i].k < m) continue;
      auto key = std::make_pair((int)boards[i].k, (int)boards[i].mover);
      const FillLists& L = host_lists(key.first, key.second);
      MidSeg sg{};
      sg.block0 = lv.blocks;
      sg.list = (const uint64_t*)(scratch + list_at[key]) + L.offset[m];
      sg.ranks = (const uint32_t*)(scratch + ranks_at[key]) + L.ranks_at[m];
      sg.loff = (uint32_t)L.offset[m];
      sg.coff = m < (int)boards[i].k ? (uint32_t)L.offset[m + 1] : 0u;
      sg.count = L.count[m];
      sg.board = (uint32_t)i;
      sg.level = (uint32_t)m;
      lv.blocks += (sg.count + kBlock - 1) / kBlock;
      segs.push_back(sg);
      lv.nsegs++;
    }
    levels.push_back(lv);
  }
  off = align256(off + segs.size() * sizeof(MidSeg));
  const size_t tables_at = off;
  uint64_t table_entries = 0;  // compact fill tables of the boards, back to back
  for (int i = 0; i < n; i++) {
    boards[i].table = table_entries;
    table_entries += fills_total((int)boards[i].k);
  }
  // five tables (both colours' masks over every subset of the empty cells,
  // 32 bytes each) after the fill tables
  const size_t masks_at = tables_at + (size_t)table_entries * sizeof(pp_super);
  const uint64_t masks_per_board = 2ull << max_empty;
  const size_t need = masks_at + (size_t)n * masks_per_board * 32;
  if (need > kScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof msg, "batch needs %zu bytes of scratch, more than the fixed %zu bytes (64 MiB)", need,
             kScratchBytes);
    return report_error(PP_ENOMEM, msg);
  }
  for (int i = 0; i < n; i++) {
    boards[i].out = (uint64_t)i;
    boards[i].masks = (uint64_t)i * masks_per_board;
  }
  // copy descriptors into the scratch array (pageable sources are staged
  // before cudaMemcpyAsync returns, so the host vectors may go out of scope)
  for (auto& kv : list_at) {
    const FillLists& L = host_lists(kv.first.first, kv.first.second);
    e = cudaMemcpyAsync(scratch + kv.second, L.flat.data(), L.flat.size() * sizeof(uint64_t),
                        cudaMemcpyHostToDevice, s);
    if (!e && !L.ranks.empty())
      e = cudaMemcpyAsync(scratch + ranks_at[kv.first], L.ranks.data(), L.ranks.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s);
    if (e) return report_error(PP_ECUDA, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(scratch + boards_at, boards.data(), n * sizeof(MidBoard), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(scratch + segs_at, segs.data(), segs.size() * sizeof(MidSeg), cudaMemcpyHostToDevice, s);
  if (e) return report_error(PP_ECUDA, cudaGetErrorString(e));
  // nothing in the scratch needs to start at zero: every fill-table entry
  // read at level m was written at level m + 1 of this same call
  const MidBoard* d_mb = (const MidBoard*)(scratch + boards_at);
  const MidSeg* d_segs = (const MidSeg*)(scratch + segs_at);
  pp_super* tables = (pp_super*)(scratch + tables_at);
  void* masks = scratch + masks_at;
  int ferr = launch_five_tables(d_mb, n, kmax, masks, s);
  if (ferr) return report_error(PP_ECUDA, cudaGetErrorString((cudaError_t)ferr));
  for (size_t j = 0; j < levels.size(); j++) {
    const bool final_level = j + 1 == levels.size();
    int err = launch_midgame_level(d_mb, d_segs + levels[j].seg0, levels[j].nsegs, levels[j].blocks, tables, d_out,
                                   final_level ? 1 : 0, s, masks,
                                   uniform_seg_blocks(segs.data() + levels[j].seg0, levels[j].nsegs, kBlock));
    if (err) return report_error(PP_ECUDA, cudaGetErrorString((cudaError_t)err));
  }
  return PP_OK;
}
