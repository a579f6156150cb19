// pp_internal.h -- shared declarations of the host layer and the kernels.
//
// Nothing here is part of the C ABI; see include/pentago_gb300.h for that.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "pentago_gb300.h"

namespace pp {

constexpr int kQStates = 19683;   // 3^9 patterns of one quadrant
constexpr int kMinStates = 4995;  // rotation classes of one quadrant
constexpr int kFormWords = 12;    // words per (quadrant, pattern) five-table entry
constexpr int kMaxEmpty = 16;     // deepest midgame fill table: 3^16 entries
// sum over c = 0..8 of the 16-bit values with at most c bits set
constexpr int kCappedSubsets = 90683;

// ---------------------------------------------------------------------------
// Rotated five-in-a-row tables (paper, "Abstracting over rotations").
//
// For a line l of five cells and a quadrant q, S_{l,q}(x) is the set of turns
// t in Z4 for which the rotated 9-bit pattern rot^t(x) covers l's cells in q
// (all of Z4 when l misses q).  The colour has five in the board g s iff some
// line has g_q in S_{l,q} for every q, so the 256-bit mask is
//     F = OR_l  (tensor product over q of S_{l,q}).
// Lines touching exactly two quadrants come in six groups ("pairs"); the four
// lines touching three quadrants are "triples".  A 4-bit set S is stored in
// one of two 16-bit forms:
//     rep(S) = S replicated in all four nibbles       (nibble j = S)
//     E(S)   = nibble j all ones iff j in S
// so rep(S_a) & E(S_b) is the outer product with bit i + 4j = [i in S_a][j in
// S_b], and two lines share one 32-bit AND.
//
// Entry layout, forms[q][x][w]:
//   w0..w2  pair slot A (6 lines, line j in word j/2, half j%2)
//   w3..w5  pair slot B (6 lines)
//   w6      pair slot C (2 lines)
//   w7,w8   triple inner forms, triple t in word 7 + t/2, half t%2
//   w9      triple gate nibbles, triple t in bits [4t, 4t+4)
//   w10,11  zero
// Pair groups and slots (rep quadrant first, E quadrant second, compact
// 16-bit mask bit index in brackets):
//   P01 q0.A & q1.A [g0+4g1]     P02 q0.B & q2.B [g0+4g2]
//   P03 q0.C & q3.C [g0+4g3]     P12 q2.C & q1.C [g2+4g1]
//   P13 q3.B & q1.B [g3+4g1]     P23 q2.A & q3.A [g2+4g3]
// Triples (inner pair forms, gate quadrant):
//   T0 {0,1,3}: q0 rep & q1 E [g0+4g1], gate q3
//   T1 {0,2,3}: q0 rep & q2 E [g0+4g2], gate q3
//   T2 {0,1,2}: q0 rep & q1 E [g0+4g1], gate q2
//   T3 {1,2,3}: q2 rep & q1 E [g2+4g1], gate q3
// ---------------------------------------------------------------------------

struct HostTables {
  // per quadrant code: black 9-bit mask | white 9-bit mask << 9 |
  // #black << 18 | #white << 22 (local bit 3r+c)
  uint32_t qdecode[kQStates];
  // per quadrant code y: rank of its rotation-minimal representative m in
  // m's count list | u << 16, where y = rot^u(m) (u anticlockwise turns)
  uint32_t standard[kQStates];
  uint16_t qlist[kMinStates];  // minimal codes, grouped by counts, increasing
  int qoff[10][10];            // first index of (black, white) in qlist
  int qdim[10][10];            // number of minimal states, 0 if b + w > 9
  uint32_t forms[4][512][kFormWords];
  // per mover colour (black, white) and rotation-minimal state i (index into
  // qlist): x = black 9-bit | white 9-bit << 9; for states with exactly one
  // empty cell also y = e | j << 4 | u << 13, where the mover's stone on cell
  // e gives a pattern of rank j (in its count list) turned u times from its
  // minimal representative; y = 0 otherwise
  uint32_t qline[2][kMinStates][2];
  // the same entries with y |= p << 16 (p = position in the count list),
  // each count list reordered by (j, u) of its one move: a line walked in
  // this order reaches every child value in one run; z = the child's
  // rotation-minimal pattern (black 9-bit | white 9-bit << 9), w = 0
  uint32_t qsorted[2][kMinStates][4];
  // per board symmetry s and rotation-minimal state i (index into qlist):
  // the pattern that s's local action makes of state i, standardised: its
  // rank in the (same) count list | t << 12, where that pattern is t
  // anticlockwise turns past its minimal representative
  uint16_t dmin[8][kMinStates];
  // subsets of a midgame board's empty-cell slots: block c (0 <= c <= 8)
  // lists every 16-bit value with at most c bits set, in increasing order,
  // so the subsets of the first k slots with at most c of them are the
  // block's first sum over j <= c of C(k, j) entries
  uint16_t subsets[kCappedSubsets];
};

const HostTables& host_tables();
uint32_t rotate9(uint32_t mask);  // one anticlockwise turn of a 9-bit pattern

// Sections of slice n (count tuples in increasing order), offsets back to back.
std::vector<pp_section_desc> slice_sections(int n, uint64_t* total);
int section_index(const std::vector<pp_section_desc>& secs, const uint8_t bw[4][2]);

// ---------------------------------------------------------------------------
// Global symmetries (paper, "Abstracting over rotations": D4 and the
// semidirect product G = L x| D4).  Symmetry s = k + 4m maps the 6x6 board by
// a left-right mirror (C -> 5 - C) when m = 1, then k anticlockwise quarter
// turns ((R, C) -> (5 - C, R)).  It carries quadrant q to position
// sym_qmap(s, q) and acts on the 3x3 pattern inside by the same map;
// m = 1 reverses the sense of every quadrant turn.  So for g in L,
//     s (g b) = phi_s(g) (s b),   phi_s(g)[sym_qmap(s, q)] = eps * g[q],
// with eps = -1 for reflections, and the super values obey
//     f_{s b}(phi_s(g)) = f_b(g).
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
#define PP_HD __host__ __device__
#else
#define PP_HD
#endif
PP_HD constexpr int sym_qmap(int s, int q) {
  // mirror: q -> q ^ 1; quarter turn: 0 -> 2 -> 3 -> 1 -> 0
  int p = (s >> 2) ? (q ^ 1) : q;
  for (int k = 0; k < (s & 3); k++) p = p == 0 ? 2 : p == 2 ? 3 : p == 3 ? 1 : 0;
  return p;
}
PP_HD constexpr bool sym_reflects(int s) { return (s >> 2) != 0; }

// D4-minimal sections of slice n (paper, "Data layout and distribution": a
// section is computed only when its count tuple is the least of its eight
// images), in increasing order, offsets back to back.
std::vector<pp_section_desc> slice_sections_d4(int n, uint64_t* total);
// Quadrant code under symmetry s's local action (mirror, then s & 3 turns).
int symmetry_pattern(int s, int code);
// The least image of a count tuple and the first symmetry reaching it.
int least_image(const uint8_t bw[4][2], uint8_t out[4][2]);

// Device copies of the tables (set by pp_init).
struct DeviceTables {
  const uint32_t* qdecode;
  const uint32_t* standard;
  const uint16_t* qlist;
  const uint32_t* forms;  // [4][512][kFormWords]
  const uint32_t* qline;    // [2][kMinStates][2]
  const uint32_t* qsorted;  // [2][kMinStates][4]
  const uint16_t* dmin;     // [8][kMinStates]
  const uint16_t* subsets;  // [kCappedSubsets]
  int qoff[10][10];
  int qdim[10][10];
};

// ---------------------------------------------------------------------------
// Midgame (paper, "Open source and data": serial retrograde below a position).
// ---------------------------------------------------------------------------

struct MidBoard {
  uint32_t root_b[4];    // root black 9-bit pattern per quadrant
  uint32_t root_w[4];    // root white
  uint32_t k;            // empty cells
  uint32_t mover;        // 1 black, 2 white (root)
  uint8_t qstart[8];     // slots of quadrant q are [qstart[q], qstart[q+1])
  uint8_t slot_bit[16];  // local cell (3r+c) of slot i
  uint64_t table;        // first super value of this board's fill table
  uint64_t out;          // index of this board in the output array
  uint64_t masks;        // first 32-byte entry of this board's colour-subset five tables
};

// One (board, level) piece of a level launch.  Entries of the level list
// are (fill index | black slots << 32 | white slots << 48).
struct MidSeg {
  uint32_t block0;         // first thread block of this segment (segments start on block boundaries)
  uint32_t loff;           // this level's first entry in the board's compact fill table
  const uint64_t* list;    // fill list of (board k, root mover, level)
  const uint32_t* ranks;   // child positions in level + 1, (k - level) per fill
  uint32_t count;          // entries
  uint32_t board;          // index into the board array
  uint32_t level;          // stones added
  uint32_t final;          // 1: store to the output array (board's out index) instead of the table
  uint32_t coff;           // level + 1's first entry in the board's compact fill table
  uint32_t pad;
};

// One level of a plan: its segments and thread blocks.
struct MidLevel {
  int32_t seg0, nsegs;
  uint32_t blocks;
  uint32_t seg_blocks;  // blocks of every segment when all are equal, else 0; may carry kSharedSegs
};

// Flag in MidLevel::seg_blocks (and the seg_blocks argument of the midgame
// kernels): the level's segments differ only in board (segment j is board
// segs[0].board + j) and block0, so only segs[0] is stored and the kernel
// derives the rest from the block index.
constexpr uint32_t kSharedSegs = 0x80000000u;

// Blocks of every segment of a level when all are equal (segment j then
// starts at block j * that), else 0.
inline uint32_t uniform_seg_blocks(const MidSeg* segs, int nsegs, uint32_t kblock) {
  if (nsegs <= 0) return 0;
  const uint32_t b = (segs[0].count + kblock - 1) / kblock;
  for (int j = 0; j < nsegs; j++)
    if ((segs[j].count + kblock - 1) / kblock != b || segs[j].block0 != (uint32_t)j * b) return 0;
  return b;
}

// Level lists for one (k, root mover): for level m, fills with m stones,
// ceil(m/2) of the root mover's colour; sorted by fill index.
// Level lists of one (k, root mover), built on the host: level m's fills in
// increasing fill index, flat, level after level (offset[m] = fills of the
// levels below m).  A board's compact fill table uses the same positions:
// the value of fill e of level m sits at offset[m] + e.  For each fill of
// level m < k and each of its empty slots in increasing order, ranks holds
// the child's position in level m + 1 (ranks_at[m] + e (k - m) + j).
struct FillLists {
  std::vector<uint64_t> flat;       // idx | black slots << 32 | white slots << 48
  std::vector<uint64_t> offset;     // per level
  std::vector<uint32_t> count;      // per level
  std::vector<uint32_t> ranks;      // child positions
  std::vector<uint64_t> ranks_at;   // per level
};
void build_fill_lists(int k, int mover, FillLists* out);
uint64_t fills_total(int k);  // fills of every level: sum_m C(k, m) C(m, ceil(m/2))

struct LevelLists {
  int k = -1, mover = 0;
  uint64_t* d_entries = nullptr;
  uint32_t* d_ranks = nullptr;
  std::vector<uint64_t> offset;    // per level
  std::vector<uint32_t> count;     // per level
  std::vector<uint64_t> ranks_at;  // per level
  uint64_t total = 0;              // entries of a board's compact table
};
const LevelLists* level_lists(int k, int mover, std::string* err);
// Host validation of one midgame root (fills everything but table/out).
int validate_midgame_board(uint64_t packed, int max_empty, MidBoard* mb, int i);
int report_error(int code, const char* message);  // sets pp_last_error_string
// Autotuner cache (pp_tune.cpp): the device part of a key, a lookup that
// counts hits and misses, and recording a choice.
std::string tune_device_tag();
bool tune_lookup(const std::string& key, pp_batch_opts* o);
bool tune_peek(const std::string& key, pp_batch_opts* o);  // a lookup that counts neither hit nor miss
void tune_record(const std::string& key, const pp_batch_opts& o);
bool tables_ready();
std::mutex& table_mutex();  // guards level_lists

// ---------------------------------------------------------------------------
// Sections (paper, "Data layout and distribution", Fig. "lines").
// ---------------------------------------------------------------------------

struct SecTask {
  uint32_t block0;          // first thread block of this task (tasks start on block boundaries)
  uint32_t pad0;
  uint64_t size;            // parent boards in the section
  uint64_t out;             // first output super value (index into the out array)
  const pp_super* child[4]; // first value of the child section of quadrant q
  uint64_t cstride[4][4];   // strides of that child section (quadrant 0 fastest)
  uint32_t dim[4];          // parent dims
  uint16_t qoff[4];         // parent quadrant list offsets into qlist
  uint8_t bw[4][2];
  uint8_t n;                // slice
  uint8_t mover;            // 1 black, 2 white
  uint8_t movable;          // bit q: quadrant q has an empty cell
  uint8_t sym[4];           // symmetry carrying child section q onto the stored (D4-minimal) one; 0 = none
  uint8_t prepared;         // 1: child values in prepared form (pp_prepare_children)
  uint16_t cqoff[4];        // qlist offset of quadrant q's counts after the move (before the symmetry)
};

// A slice-35 section processed line by line (paper, Fig. "lines"): every
// board has one empty cell, in quadrant q (the line axis); its child is a
// full board of slice 36 on the child section's line along q.
struct LineTask {
  uint32_t warp0;         // first warp of this task (tasks in warp order; a warp owns 32 lines)
  uint32_t lines;         // parent lines = boards / dim[q]
  uint32_t dim[4];        // parent dims
  uint32_t stride[4];     // parent strides within the section (quadrant 0 fastest)
  uint32_t cstride[4];    // child section strides
  uint32_t cdim;          // child dim along q
  uint16_t qoff[4];       // parent quadrant list offsets
  uint64_t out;           // first output value of the section
  const pp_super* child;  // first transformed value (X2, X3) of the child section (null: on demand)
  uint32_t mover;         // 1 black, 2 white
  uint32_t cqoff;         // qlist offset of quadrant q's counts in the child section
  uint32_t q;             // the line axis (the non-full quadrant); every block holds one q
  uint32_t pad;
};
#ifndef PP_LINE_WARPS
#define PP_LINE_WARPS 4
#endif
// warps per block of the slice-35 line kernel: at its ~96 registers, blocks
// of 4 warps fit 5 to an SM (20 warps) where blocks of 8 fit 2 (16)
constexpr int kLineWarps = PP_LINE_WARPS;

// A section of any slice below 35 processed by lines along one of its
// non-full quadrants Q (paper, Fig. "lines"): a lane owns the boards that
// share the other three quadrants' states and walks Q's states.  Moves in Q
// read the child section S+Q along its Q axis; moves in another non-full
// quadrant R read S+R along its Q axis at the lane's fixed R child state.
struct SecLineTask {
  uint32_t warp0;            // first warp of this task (tasks in warp order; a warp owns 32 lines)
  uint32_t lines;            // boards / dim[Q]
  uint64_t out;              // first output value of the section
  const pp_super* child[4];  // child section of quadrant q (moves in q), null when q is full
  uint64_t cstride[4][4];    // strides of that child section
  uint32_t dim[4];           // parent dims
  uint32_t stride[4];        // parent strides (quadrant 0 fastest)
  uint16_t qoff[4];          // parent quadrant list offsets
  uint8_t mover;             // 1 black, 2 white
  uint8_t movable;           // bit q: quadrant q has an empty cell
  uint8_t prepared;          // 1: child values in prepared form (pp_prepare_children)
  uint8_t pad;
};

// ---------------------------------------------------------------------------
// Kernel launchers (pp_kernels.cu).  All return a cudaError_t value.
// ---------------------------------------------------------------------------
int upload_tables(const HostTables& t, DeviceTables* dt, std::string* err);
constexpr int kBlock = 256;  // threads per block of the midgame and section kernels
// d_masks: the colour-subset five tables written by launch_five_tables
// seg_blocks: uniform_seg_blocks of the launch's segments (0: search)
// parity: -1 full tables (64 B entries); 0 or 1 half tables (32 B entries)
// for a root wanted on that parity class of g only
int launch_midgame_level(const MidBoard* d_boards, const MidSeg* d_segs, int nsegs, uint32_t blocks,
                         pp_super* d_table, pp_super* d_out, int final_level, pp_stream s, const void* d_masks,
                         uint32_t seg_blocks, int parity = -1);
int launch_five_tables(const MidBoard* d_boards, int n, int kmax, void* d_masks, pp_stream s);
// the same for the n boards d_boards[slots[i]] (slots: host array, passed in
// the launches' parameters, kSlotBatch per launch)
constexpr int kSlotBatch = 1024;
int launch_five_tables_slots(const MidBoard* d_boards, const uint16_t* slots, int n, int kmax, void* d_masks,
                             pp_stream s);
int persistent_midgame_blocks(int ctas_per_sm, bool half = false);  // co-resident blocks of the persistent kernel
// d_sync: 3 words (barrier count, generation, status), zero before the launch
int launch_midgame_persistent(const MidBoard* d_boards, const MidSeg* d_segs, const MidLevel* d_levels, int nlevels,
                              pp_super* d_table, pp_super* d_out, uint32_t* d_sync, int grid, pp_stream s,
                              const void* d_masks, int parity = -1);
int launch_barrier_probe(uint32_t* d_sync, uint32_t limit, pp_stream s);
void set_barrier_spins(uint32_t polls);  // 0 = the default limit
int launch_sections(const SecTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out, pp_stream s, bool d4);
int persistent_section_blocks(int ctas_per_sm, bool d4);
int launch_sections_persistent(const SecTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out,
                               uint32_t* d_counter, int grid, pp_stream s, bool d4);
int launch_digest(const pp_super* d_values, uint64_t n, uint64_t* d_acc, pp_stream s);
int launch_child_transform(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream s);
int launch_prepare(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream s);
// on_demand: the children (full boards of slice 36) are evaluated in the
// kernel from the line's own terms instead of read from a slice-36 array
int launch_line35(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s,
                  bool on_demand = false);
// slice 36 by lines (tasks as for slice 35 with no child)
int launch_line36(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s);
// ready child records of sections (child: first input value of the section,
// out: its first output value, mover: the parents' mover)
int launch_ready(const LineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out, pp_stream s);
// A child section that is not D4-minimal, written out in its own layout
// from its stored least image (so line kernels read it like any section).
struct MatTask {
  uint32_t block0;         // first thread block of this task
  uint32_t sym;            // symmetry carrying this section onto the stored one
  uint64_t size;           // boards
  uint64_t dst;            // first value in the output buffer
  const pp_super* src;     // the stored least image
  uint64_t sstride[4];     // its strides, by quadrant position
  uint32_t dim[4];         // this section's dims
  uint16_t qoff[4];        // qlist offsets of this section's quadrant counts
};
int launch_materialise(const MatTask* d_tasks, int ntasks, uint32_t blocks, pp_super* d_out, pp_stream s);

// rm: the one other quadrant with empty cells (0..3, not q), -1 none, 4 any
int launch_section_lines(int q, int rm, const SecLineTask* d_tasks, int ntasks, uint32_t warps, pp_super* d_out,
                         pp_stream s, bool ready = false);
int launch_five_masks(const uint64_t* d_boards, int n, uint64_t* d_out, pp_stream s);
int launch_rmax(const pp_super* d_in, int n, pp_super* d_out, pp_stream s);
int launch_shift(const pp_super* d_in, int n, int q, int u, pp_super* d_out, pp_stream s);
int launch_symmetry(const pp_super* d_in, int n, int sym, uint32_t turns, pp_super* d_out, pp_stream s);
void count_launch();
void set_launch_counting(bool on);
void add_launches(uint64_t n);
uint64_t launch_total();

}  // namespace pp
