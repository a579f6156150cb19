/*
 * pentago_gb300.h -- C ABI of the GB300 (sm_103a) pentago retrograde library.
 *
 * The library computes rotation-abstracted values ("super values") of pentago
 * positions exactly, following Irving, "Pentago is a First Player Win:
 * Strongly Solving a Game Using Parallel In-Core Retrograde Analysis":
 *
 *   - game value v_c(s): Section "Problem definition";
 *   - super value: for each g in L = Z4^4 (independent quarter turns of the
 *     four quadrants) two bits, win = [v_c(g s) = 1] and
 *     notlose = [v_c(g s) >= 0]: Section "Abstracting over rotations";
 *   - slices, sections and rotation-minimal quadrant states: Section
 *     "Data layout and distribution";
 *   - the from-scratch solver for positions with many stones ("midgame"):
 *     Section "Open source and data".
 *
 * Conventions (the paper leaves them open):
 *   - cell (R,C), R,C in 0..5; quadrant q = 2*[R>=3] + [C>=3] (q0 top-left,
 *     q1 top-right, q2 bottom-left, q3 bottom-right); local r = R%3, c = C%3;
 *   - board: uint64, quadrant q's 16-bit field [16q, 16q+16) holds
 *     sum digit * 3^(3r+c), digit 0 empty, 1 black, 2 white;
 *   - g = (g0..g3), g_q = anticlockwise quarter turns of quadrant q, one turn
 *     moving local (r,c) to (2-c, r); beta(g) = g0 + 4g1 + 16g2 + 64g3 and bit
 *     beta of a table is word beta>>6, bit beta&63;
 *   - black moves when the colour counts are equal, white when black has one
 *     more; every value is from the side to move.
 *
 * Memory: every device pointer is allocated and owned by the caller (for
 * example as a PyTorch tensor) and must be 16-byte aligned; midgame
 * workspaces, server arenas and the value arrays of the section and slice
 * calls 32-byte aligned (they are accessed 256 bits at a time).  The library
 * owns
 * only its constant tables (uploaded by pp_init) and the small descriptor
 * buffers of plans and servers.  All entry points return 0 (PP_OK) or an
 * error code; on error pp_last_error_string() describes it.  Inputs are
 * validated on the host before any launch; kernels never trap.
 */
#ifndef PENTAGO_GB300_H
#define PENTAGO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (0 = the legacy default stream). */
typedef struct CUstream_st* pp_stream;

/* Super value: win and not-lose tables, 256 bits each (64 bytes). */
typedef struct pp_super {
  uint64_t win[4];
  uint64_t notlose[4];
} pp_super;

/* One section of a slice: per-quadrant (black, white) counts, the number of
 * rotation-minimal states per quadrant, and the section's first super value
 * within its slice arena.  Values are stored as a dense 4-D array with
 * quadrant 0's index fastest: i0 + d0*(i1 + d1*(i2 + d2*i3)). */
typedef struct pp_section_desc {
  uint8_t bw[4][2];
  uint16_t dim[4];
  uint64_t offset;
} pp_section_desc;

enum {
  PP_OK = 0,
  PP_EINVAL = 1,   /* bad argument, board, count, size or alignment */
  PP_ENOMEM = 2,   /* workspace too small, or admission refused */
  PP_ETIMEOUT = 3, /* a bounded device-side wait expired */
  PP_ECUDA = 4,    /* a CUDA call failed */
  PP_ENOTINIT = 5, /* pp_init has not run */
  PP_EIO = 6       /* a file could not be read or written */
};

/* ---- library ----------------------------------------------------------- */

/* Build the quadrant, standardisation and rotated five-in-a-row tables
 * (Section "Data layout and distribution"; "Abstracting over rotations") and
 * upload them to the current device.  Idempotent.  Must precede every other
 * call and any stream capture. */
int pp_init(void);
void pp_shutdown(void);
const char* pp_last_error_string(void);

/* Number of kernel launches made by this process so far (all entry points). */
uint64_t pp_launch_count(void);

/* ---- layout queries (host only) ----------------------------------------- */

/* Rotation-minimal quadrant states with the given counts (Section "Data
 * layout and distribution": a quadrant is kept when its code is the least of
 * its four rotations; states are listed in increasing code order).  Returns
 * their number; copies up to max codes into codes when it is non-null. */
int pp_quadrant_states(int black, int white, uint16_t* codes, int max);

/* All sections of slice n (0 <= n <= 36), in increasing order of their count
 * tuples, with offsets back to back starting at 0.  Returns the number of
 * sections (negative error code on bad n); writes up to max descriptors and,
 * when total is non-null, the slice's total number of super values. */
int pp_slice_sections(int n, pp_section_desc* out, int max, uint64_t* total);

/* Batch options for plans and pp_slice_step; zero fields mean "choose automatically"
 * (the autotuner's cached choice). */
typedef struct pp_batch_opts {
  int persistent;        /* 1: one persistent launch over all sections */
  int threads_per_block; /* 0 = auto */
  int ctas_per_sm;       /* 0 = auto */
  int stage_children;    /* 0 = auto; 1: by lines, one warp lane per line of
                          * boards (slice 35: child values turned once into
                          * their rmax'd forms; below 35: lines along a non-full
                          * quadrant, the other quadrants' line terms once per
                          * line); 2: one thread per board */
  int largest_first;     /* 1: sections ordered largest first (load balance) */
} pp_batch_opts;

/* ---- midgame solver: Section "Open source and data" --------------------- */
/*
 * For each board, the super value of the position, computed by retrograde
 * analysis over every filling of its empty cells (level by level from the
 * full board back to the board itself; rotations enter only through rmax,
 * no quadrant standardisation).  Each board must have valid colour counts,
 * digits < 3, at most max_empty <= 16 empty cells, and no five in a row as
 * given (g = 0); otherwise PP_EINVAL and nothing is launched.
 *
 * The workspace holds the boards' compact fill tables: one 64-byte super
 * value per fill of every level, F(k) = sum_m C(k, m) C(m, ceil(m/2)) values
 * for k empty cells (143,365 for k = 12, against 3^12 = 531,441 dense),
 * level after level, each level's fills in increasing fill index (sum d_i 3^i
 * over the board's empty cells); a fill finds its children through a shared
 * list of their positions.  Then come the five tables, 2 x 2^max_empty masks
 * of 32 bytes reserved per board (each colour's rotated five-in-a-row mask
 * for every subset of the empty cells a fill can hold: ceil(k/2) cells of
 * the colour that moves first, floor(k/2) of the other; a fill reads its
 * masks instead of evaluating lines), then room for n results used by
 * pp_midgame_solve_host: at most
 * n (F(max_empty) 64 + 2^max_empty 64 + 64) bytes, as
 * pp_midgame_workspace_bytes gives.
 */
int pp_midgame_workspace_bytes(int n, int max_empty, size_t* bytes);

/* A plan: boards validated and described on the host, descriptors uploaded
 * (one allocation per plan; boards sharing their number of empty cells and
 * mover share one descriptor per level).  Running a plan is pure device
 * work on the given stream (no host synchronisation), so a run can be
 * captured in a CUDA graph.  A plan is not safe for concurrent use from
 * several threads; distinct plans are. */
typedef struct pp_midgame_plan pp_midgame_plan;
int pp_midgame_plan_create(const uint64_t* h_boards, int n, int max_empty,
                           pp_midgame_plan** plan);
int pp_midgame_plan_run(pp_midgame_plan* plan, void* d_workspace, size_t ws_bytes,
                        pp_super* d_out, pp_stream stream);
void pp_midgame_plan_destroy(pp_midgame_plan* plan);

/* Execution mode of a plan (batching; pp_batch_opts.persistent).  Every
 * mode first fills the five tables (one launch), then runs the levels:
 *   0 or 2  one launch per level;
 *   1       one persistent cooperative launch running every level, blocks
 *           striding over each level's work and meeting at a grid barrier
 *           between levels (ctas_per_sm limits resident blocks, 0 = all that
 *           fit); the barrier's wait is bounded and reports PP_ETIMEOUT
 *           through pp_midgame_plan_status instead of hanging.  The default
 *           of a new plan (and so of pp_midgame_solve), falling back to 2
 *           where the device cannot co-schedule the grid;
 *   3       a CUDA graph of the level launches, captured on first use for
 *           the given workspace and output pointers and replayed.
 * threads_per_block must be 0 or 256; stage_children is ignored. */
int pp_midgame_plan_configure(pp_midgame_plan* plan, const pp_batch_opts* opts);

/* One parity class of g (Section "Open source and data": rmax flips the
 * parity of g0 + g1 + g2 + g3, so a solve wanted on one class needs one class
 * per level, alternating, and stores 32 bytes per position instead of 64).
 * parity -1 (the default) computes every rotation; 0 or 1 only the rotations
 * with g0 + g1 + g2 + g3 = parity (mod 2).  Class 0 holds g = 0, the position
 * as given.  d_out then holds that class's bits and zeros in the other; the
 * workspace needed is pp_midgame_parity_workspace_bytes (half-size fill
 * tables).  Setting the parity of a plan drops its captured graph. */
int pp_midgame_plan_set_parity(pp_midgame_plan* plan, int parity);
int pp_midgame_parity_workspace_bytes(int n, int max_empty, size_t* bytes);
int pp_midgame_solve_parity(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty, int parity,
                            void* d_workspace, size_t ws_bytes, pp_stream stream);

/* Autotuner: times every mode on this plan (each run overwrites d_out and
 * the workspace with the same values), keeps the fastest, and reports it. */
int pp_midgame_plan_autotune(pp_midgame_plan* plan, void* d_workspace, size_t ws_bytes, pp_super* d_out,
                             pp_stream stream, pp_batch_opts* chosen);

/* Synchronises the stream; PP_ETIMEOUT if a persistent run's grid barrier
 * gave up, else PP_OK. */
int pp_midgame_plan_status(pp_midgame_plan* plan, pp_stream stream);

/* Failure-path self-test of the bounded grid barrier (no paper counterpart):
 * a two-block cooperative launch in which one block never arrives, so the
 * other's wait (about 65 thousand polls, a few milliseconds) runs out.
 * d_sync: 4 device words (caller-owned scratch).  Returns PP_ETIMEOUT when the
 * wait expired and was reported as designed, PP_OK if it did not. */
int pp_selftest_barrier_timeout(uint32_t* d_sync, pp_stream stream);

/* Failure-path testing aid (no paper counterpart): the number of polls a
 * persistent midgame launch's grid barrier waits before it gives up, for
 * launches made after the call (process-wide; 0 restores the default of
 * about 2 s).  With a limit of a few polls the barrier gives up at the first
 * level whose blocks do not all arrive together: the kernel stops early and
 * every entry point that ran it reports PP_ETIMEOUT (pp_midgame_plan_status,
 * pp_midgame_solve, pp_midgame_solve_host, pp_midgame_solve_parity).  Always
 * returns PP_OK. */
int pp_set_barrier_poll_limit(uint32_t polls);

/* Convenience: d_boards on the device (read back once, synchronising the
 * stream), plan, run; d_out[i] receives board i's super value.  The plan
 * runs in the mode the autotuner cache holds for its shape (see the
 * autotuner cache below) when that is mode 1 or 2; a shape never tuned, or
 * tuned to a graph (not worth capturing for one run), runs the plan default
 * (mode 1).  Values never depend on the mode.  pp_midgame_solve_host and
 * pp_midgame_solve_parity choose their mode the same way. */
int pp_midgame_solve(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty,
                     void* d_workspace, size_t ws_bytes, pp_stream stream);

/* End to end from host memory: h_boards and h_out are host arrays (pinned
 * memory is fastest); the boards are copied in, solved, and the values copied
 * out; returns after the stream has finished. */
int pp_midgame_solve_host(const uint64_t* h_boards, int n, pp_super* h_out, int max_empty,
                          void* d_workspace, size_t ws_bytes, pp_stream stream);

/* The same midgame solve without any device allocation (the paper has no
 * counterpart; this is a library convenience).  Some callers may not call
 * cudaMalloc or any allocator once they run: an application whose device
 * memory is entirely owned by another framework's pool, a latency-critical
 * service thread that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree imply, or a plugin host that forbids allocation
 * after start-up.  Such a caller passes only d_boards and d_out (device
 * arrays, 16-byte aligned); descriptors, fill lists, fill and five tables live in
 * one fixed 64 MiB device array inside the library, which every GPU that has
 * used this entry point keeps until the process exits.  A batch that needs
 * more than 64 MiB (for example 8 boards with 12 empty cells need 76 MB)
 * returns PP_ENOMEM before anything is copied or launched.  pp_init must
 * have run.  The first call on each device looks up the array's device
 * address (set-up, with that device current).  All calls share the one
 * array, so calls whose work
 * overlaps on the GPU (different streams, or different host threads without
 * ordering) race; calls on one stream are ordered.  The boards are read back
 * to the host once (the stream is synchronised for that); the solve itself
 * is queued asynchronously on the stream. */
int pp_midgame_solve_noalloc(const uint64_t* d_boards, int n, pp_super* d_out, int max_empty,
                             pp_stream stream);

/* ---- serving: many midgame queries as they arrive -------------------------- */
/*
 * A request server for midgame queries (the paper's backend answers positions
 * beyond its database by a from-scratch solve, Section "Open source and
 * data").  A worker thread keeps the fill and five tables of admitted
 * queries in the caller's device arena (F(k) + 2^k super values, 64 bytes
 * each, for k empty cells; F as for pp_midgame_workspace_bytes) and
 * advances all
 * admitted queries by one level per kernel launch: queries that arrive while
 * others run join at the next level boundary and share launches with them
 * (continuous batching).  Admission is first come, first served, limited by
 * max_slots and by a free arena range of the query's footprint.
 */
typedef struct pp_server pp_server;

typedef struct pp_result {
  uint64_t req_id;
  int32_t status;                  /* PP_OK, or the error of the launch */
  int32_t empty;                   /* empty cells of the query */
  double submit_s, admit_s, done_s; /* host clock, seconds since creation */
  pp_super value;
} pp_result;

typedef struct pp_server_stats {
  uint64_t submitted, admitted, completed, launches, queued, max_active;
  uint64_t arena_free_largest; /* bytes */
} pp_server_stats;

/* d_arena: caller-owned device memory, 32-byte aligned, kept alive until
 * pp_server_destroy; max_slots: queries in flight (1..4096); max_empty: the
 * largest query accepted (<= 16).  Builds the fill lists of every size up to
 * max_empty once (a few seconds for 16). */
int pp_server_create(void* d_arena, size_t arena_bytes, int max_slots, int max_empty, pp_server** server);
/* The same server with an arena the library allocates (mem_budget bytes,
 * rounded down to a multiple of 64; PP_ENOMEM if the device cannot hold it)
 * and frees in pp_server_destroy: for callers that hold no device memory of
 * their own. */
int pp_server_create_budget(size_t mem_budget, int max_slots, int max_empty, pp_server** server);
/* The same server on one parity class of the rotations (-1: every rotation;
 * 0 or 1, as pp_midgame_plan_set_parity): half fill tables, so a query with
 * k empty cells needs (F(k) + 2^(k+1)) x 32 bytes of arena, rounded up to a
 * multiple of 64, and its result holds that class's bits with zeros in the
 * other. */
int pp_server_create_parity(void* d_arena, size_t arena_bytes, int max_slots, int max_empty, int parity,
                            pp_server** server);
/* Validates the board on the host (PP_EINVAL as for pp_midgame_solve;
 * PP_ENOMEM if its footprint exceeds the whole arena) and queues it. */
int pp_server_submit(pp_server* server, uint64_t board, uint64_t req_id);
/* Moves up to max finished results into out (oldest first); returns their
 * number, or a negative error code. */
int pp_server_poll(pp_server* server, pp_result* out, int max);
/* Blocks until at least count results wait to be polled or timeout_s passes;
 * returns the number waiting (negative error code on failure). */
int pp_server_wait(pp_server* server, int count, double timeout_s);
int pp_server_get_stats(pp_server* server, pp_server_stats* stats);
/* Finishes the admitted queries, drops the queued ones, frees the server. */
void pp_server_destroy(pp_server* server);

/* ---- retrograde step over sections: Section "Data layout and
 * distribution" and Fig. "lines" -------------------------------------------- */
/*
 * pp_section_compute: every super value of one section of slice n from the
 * sections of slice n+1 it depends on.  For each quadrant q that is not full,
 * d_child[q] points at the first value of the child section whose counts are
 * the parent's with one more stone of the mover's colour in quadrant q (a
 * section laid out as pp_slice_sections describes it); for full quadrants
 * d_child[q] is ignored.  Slice 36 takes no children (values from five in a
 * row or a tie).  d_out receives the section's dense 4-D array.
 */
int pp_section_compute(int n, const pp_section_desc* parent, const pp_super* const d_child[4],
                       pp_super* d_out, pp_stream stream);
/* The same with a descriptor of each child section beside its values:
 * child_desc[q] must be the section of slice n+1 whose counts are the
 * parent's with one more stone of the mover's colour in quadrant q, with
 * that section's dims (its offset is not read: d_child[q] already points at
 * its values).  A missing or different descriptor for a quadrant that is not
 * full is PP_EINVAL before anything is launched; full quadrants' entries are
 * ignored, and so is child_desc when d_child is null (slice 36, or slice 35
 * with its children evaluated on demand). */
int pp_section_compute_desc(int n, const pp_section_desc* parent, const pp_super* const d_child[4],
                            const pp_section_desc* const child_desc[4], pp_super* d_out, pp_stream stream);



/* pp_slice_step: all sections of slice n.  in_values (slice n+1, laid out as
 * pp_slice_sections(n+1)) is ignored for n = 36.  For n = 35 it may be null:
 * slice 36 is then computed on demand (Section "Data layout and
 * distribution": the last slice is not stored), each child evaluated in the
 * line kernel from its board, with the same values as from a stored slice
 * 36 (by lines only; not with stage_children 2 nor for D4 layouts).
 * out_values receives
 * slice n laid out as pp_slice_sections(n).  When filter is non-null (one byte
 * per section of slice n), only the sections with a non-zero byte are
 * computed, and they are written back to back in out_values in section order
 * (so a slice too large for the device can be produced batch by batch). */
int pp_slice_step(int n, const pp_super* in_values, pp_super* out_values,
                  const uint8_t* filter, const pp_batch_opts* opts, pp_stream stream);

/* A slice plan: the sections of one step laid out once (tasks uploaded), so a
 * run is launches only and can be captured in a CUDA graph (batching of many
 * uneven sections per launch).  Arguments as for pp_slice_step; the input and
 * output pointers are fixed at creation.  Options: persistent = 1 runs a grid
 * sized to the device whose blocks claim work from a counter, 2 (or 0) one
 * block per 256 boards; largest_first orders the sections for load balance;
 * stage_children as above.  pp_slice_plan_autotune times the candidates on
 * the plan (each run rewrites the same output) and keeps the fastest. */
typedef struct pp_slice_plan pp_slice_plan;
int pp_slice_plan_create(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                         const pp_batch_opts* opts, pp_slice_plan** plan);
int pp_slice_plan_configure(pp_slice_plan* plan, const pp_batch_opts* opts);
int pp_slice_plan_run(pp_slice_plan* plan, pp_stream stream);
int pp_slice_plan_autotune(pp_slice_plan* plan, pp_stream stream, pp_batch_opts* chosen);

/* Prepared children (Section "Abstracting over rotations": rmax distributes
 * over OR and commutes with quadrant turns and with the board symmetries).
 * A board below slice 35 ORs ~notlose and ~win of its children, each turned
 * by the child's standardising turn, and applies rmax once to each OR.  The
 * rmax can instead be applied once per child value: pp_prepare_children
 * writes, for each of n values, win slot ~rmax(~win) and not-lose slot
 * ~rmax(~notlose) (d_out may equal d_in; 16-byte aligned device arrays,
 * caller-owned; asynchronous on the stream).  A slice plan whose input holds
 * prepared values of slice n+1 (for every section the plan reads) is told
 * so with pp_slice_plan_set_prepared(plan, 1); its boards then skip their
 * rmax and its output is the same, bit for bit.  Only for plans of slices
 * below 35 (PP_EINVAL otherwise).
 *
 * Ready children (the same, and Section "Problem definition": a move that
 * makes five wins at once).  A board's immediate-win mask is the OR over
 * its moves of the child's five-in-a-row set F_c of the board's mover c,
 * turned as the child value is.  pp_prepare_children_ready writes, for every
 * section of slice n+1 that the input holds, win slot ~(F_c | rmax(~win))
 * and not-lose slot ~(F_c | rmax(~notlose)) with c the mover of slice n
 * (n in 0..34; d4: the D4-reduced layout).  The input is laid out as the
 * slice's sections (pp_slice_sections(n+1)), or, with in_offsets (one entry
 * per section of slice n+1: its first value in d_in, or PP_ABSENT), as
 * pp_slice_step_sparse reads it; in_count is the number of values in d_in
 * (PP_EINVAL for a section past them, or for two sections that overlap);
 * d_out receives the same layout (it may equal d_in;
 * 32-byte aligned device arrays, caller-owned; asynchronous on the stream).
 * The library keeps the uploaded work list of the last 64 argument sets, so
 * a repeated call is a kernel launch only and may be captured in a CUDA
 * graph; a first call with new arguments while its stream is capturing is
 * PP_EINVAL.  A plan told pp_slice_plan_set_prepared(plan, 2) reads such values: its
 * boards skip their rmax and every line with one more stone, and its output
 * is the same, bit for bit.  One-shot pp_slice_step, pp_d4_slice_step and
 * pp_slice_step_sparse below slice 35 make ready records of their input
 * themselves, in a stream-ordered temporary the size of the input, when
 * they write at least as many boards as the input holds (else, or when the
 * temporary cannot be had, they read the input as it is). */
int pp_prepare_children(const pp_super* d_in, uint64_t n, pp_super* d_out, pp_stream stream);
int pp_prepare_children_ready(int n, int d4, const pp_super* d_in, const uint64_t* in_offsets, uint64_t in_count,
                              pp_super* d_out, pp_stream stream);
/* prepared: 0 raw values, 1 prepared (pp_prepare_children), 2 ready
 * (pp_prepare_children_ready) */
int pp_slice_plan_set_prepared(pp_slice_plan* plan, int prepared);

/* Out-of-core steps (Section "Data layout and distribution": slice n reads
 * only slice n+1; the paper keeps the slices in the memory of many nodes).
 * A stager computes sections of slice n < 35 from a slice n+1 held partly
 * in device memory and partly in (pinned) host memory:
 *   d_base, base_count: one device array of super values;
 *   dev_offsets[i]: where section i of slice n+1 (as pp_slice_sections or,
 *     with d4, pp_d4_slice_sections lists them) starts in d_base, or
 *     PP_ABSENT (~0) when it is not on the device;
 *   h_src[i]: host pointer to section i's values, used when dev_offsets[i]
 *     is PP_ABSENT (NULL when held nowhere); pinned memory lets the copies
 *     run asynchronously;
 *   [stage_at, stage_at + stage_values) of d_base: room for the host
 *     sections a step reads, used in two halves by alternate steps (it must
 *     not overlap a device section);
 *   prepared: the form of the values: 0 raw, 1 prepared
 *     (pp_prepare_children), 2 ready (pp_prepare_children_ready).
 * The arrays are copied at creation; the caller keeps d_base and the host
 * sections alive and unchanged while steps run.  pp_stager_step computes
 * the sections of slice n kept by filter (one byte per section; NULL =
 * all) into d_out, back to back in section order (as pp_slice_step with a
 * filter).  It copies the host sections they read into the next staging
 * half on copy_stream (after the step that last read that half, so one
 * step's copies overlap the previous step's work), and runs the step on
 * stream once they have arrived.  *staged_values (may be NULL) receives the
 * values copied.  PP_EINVAL when a section read is held nowhere, PP_ENOMEM
 * when a step's host sections exceed half the staging room (nothing is
 * launched then). */
typedef struct pp_stager pp_stager;
int pp_stager_create(int n, int d4, pp_super* d_base, uint64_t base_count, const uint64_t* dev_offsets,
                     const pp_super* const* h_src, uint64_t stage_at, uint64_t stage_values, int prepared,
                     pp_stager** stager);
int pp_stager_step(pp_stager* stager, pp_super* d_out, const uint8_t* filter, pp_stream stream,
                   pp_stream copy_stream, uint64_t* staged_values);
void pp_stager_destroy(pp_stager* stager);

/* Autotuner cache (batching: how uneven boards and sections are assigned to
 * the device; no paper counterpart beyond the balancing of uneven lines in
 * Section "Data layout and distribution").  pp_midgame_plan_autotune and
 * pp_slice_plan_autotune first look the plan's shape up in a process-wide
 * cache: on a hit they configure the plan with the cached choice and time
 * nothing; on a miss they time the candidates and record the fastest.  The
 * shape is the device (compute capability and SM count) and, for a midgame
 * plan, its parity class, max_empty and the number of boards with each
 * number of empty cells; for a slice plan, the slice, the layout (full or
 * D4) and the sections the filter keeps.  If the environment variable
 * PP_AUTOTUNE_CACHE names a file, the first lookup merges it into the cache
 * (a missing or malformed file is then skipped) and every new entry rewrites
 * it, so later processes reuse the choices.  Processes sharing one file
 * may drop each other's new entries (the last rename wins): the file is a
 * cache, and a dropped entry only means that shape is timed again.
 *
 * File format: text, one entry per line, "<key>TAB<persistent>
 * <threads_per_block> <ctas_per_sm> <stage_children> <largest_first>" (the
 * pp_batch_opts fields); lines starting with '#' and empty lines are skipped.
 * pp_autotune_cache_load merges a file (entries replace those of the same
 * key; *entries = entries read, may be null): PP_EIO if it cannot be read,
 * PP_EINVAL if any line is malformed or out of range, and then nothing is
 * merged.  pp_autotune_cache_save writes every entry (through a temporary
 * file renamed over path): PP_EIO on failure.  pp_autotune_cache_clear
 * empties the cache and its counters (the environment's file is not read
 * again).  pp_autotune_cache_stats reports the entries and the lookups that
 * hit and missed (each pointer may be null).  These four need neither
 * pp_init nor a GPU and are thread-safe. */
int pp_autotune_cache_load(const char* path, int* entries);
int pp_autotune_cache_save(const char* path);
int pp_autotune_cache_clear(void);
int pp_autotune_cache_stats(int* entries, int* hits, int* misses);
void pp_slice_plan_destroy(pp_slice_plan* plan);

/* ---- D4-reduced slices: Section "Data layout and distribution" (only
 * sections whose counts are least under D4 are computed) and Fig. "lines"
 * (input lines are turned before use) ------------------------------------ */
/*
 * pp_d4_slice_sections: the D4-minimal sections of slice n -- those whose
 * count tuple ((b0,w0),...,(b3,w3)) is lexicographically least among its
 * eight images under the board symmetries (see pp_symmetry_info) -- in
 * increasing order, offsets back to back.  Within a section every
 * rotation-minimal board is stored, as for pp_slice_sections, so a section
 * that is its own image holds symmetric boards twice (the paper's accepted
 * overcount).  Returns the number of sections or a negative error code.
 *
 * pp_d4_slice_step / pp_d4_slice_plan_create: as pp_slice_step and
 * pp_slice_plan_create, with in_values laid out as pp_d4_slice_sections(n+1)
 * and out_values as pp_d4_slice_sections(n) (compact in section order when a
 * filter is given; one byte per D4-minimal section).  A move whose child
 * section is not minimal reads the child's least image: the child board is
 * mapped by the symmetry s that carries its section there (the first in
 * symmetry order when several do), each quadrant is standardised, and the
 * stored value is read back as f_c(g) = f_{c*}(phi_s(g) + t).  Below slice
 * 35, by lines (stage_children 1 or 0), such child sections are first written
 * out in their own layout in a temporary buffer (one pass; the plan keeps
 * the buffer), then every section runs by lines; stage_children 2 runs one
 * thread per board reading through the symmetries directly.  The plan is
 * run, configured, autotuned and destroyed with the pp_slice_plan_* calls.
 * Values equal those of the full layout on every stored board.
 */
int pp_d4_slice_sections(int n, pp_section_desc* out, int max, uint64_t* total);
int pp_d4_slice_step(int n, const pp_super* in_values, pp_super* out_values,
                     const uint8_t* filter, const pp_batch_opts* opts, pp_stream stream);
int pp_d4_slice_plan_create(int n, const pp_super* in_values, pp_super* out_values, const uint8_t* filter,
                            const pp_batch_opts* opts, pp_slice_plan** plan);

/* ---- sparse inputs: a slice computed from part of the next slice --------
 * Section "Data layout and distribution": slice n needs only slice n+1, and
 * a section reads at most one child section per quadrant that can take a
 * stone.  A set of sections of slice n can therefore be computed from just
 * the child sections it reads, and those from theirs: a dependency cone that
 * fits in HBM where a whole slice (1.4 TB for D4 slice 32) does not.
 *
 * pp_slice_children marks in child_filter (one byte per section of slice
 * n+1, zeroed first) every section that the sections of slice n kept by
 * filter (null = all) read: for each quadrant q with fewer than 9 stones,
 * the counts with the mover's count in q raised by one, taken to their
 * least image under D4 when d4 != 0 (the layout of pp_d4_slice_sections).
 * Host only; 0 <= n <= 35.
 *
 * pp_slice_step_sparse / pp_slice_plan_create_sparse: as pp_slice_step /
 * pp_slice_plan_create (d4 = 0) or the pp_d4_ forms (d4 != 0), for
 * 0 <= n <= 34, with the sections of slice n+1 held anywhere in in_values:
 * in_offsets[i] (host array, one entry per section of slice n+1 in the
 * layout's order) is the first value of section i in in_values, or
 * PP_ABSENT.  in_count is the number of values in in_values.  A section
 * read but absent, or one that would run past in_count, is PP_EINVAL before
 * any launch.  The compact output of a filtered step (sections back to back
 * in section order) is a valid sparse input for the step below it, so cones
 * are computed slice by slice from the top. */
#define PP_ABSENT (~(uint64_t)0)
int pp_slice_children(int n, int d4, const uint8_t* filter, uint8_t* child_filter);
int pp_slice_step_sparse(int n, int d4, const pp_super* in_values, const uint64_t* in_offsets, uint64_t in_count,
                         pp_super* out_values, const uint8_t* filter, const pp_batch_opts* opts, pp_stream stream);
int pp_slice_plan_create_sparse(int n, int d4, const pp_super* in_values, const uint64_t* in_offsets,
                                uint64_t in_count, pp_super* out_values, const uint8_t* filter,
                                const pp_batch_opts* opts, pp_slice_plan** plan);

/* Board symmetries (Section "Abstracting over rotations": D4 and
 * G = L x| D4).  Symmetry s = k + 4m (0 <= s < 8) is a left-right mirror
 * (column C -> 5 - C) when m = 1, followed by k anticlockwise quarter turns of
 * the whole board ((R, C) -> (5 - C, R)).  It carries quadrant q to position
 * qmap[q] and acts on the pattern inside by the same map, so a quadrant turn
 * g_q becomes a turn eps * g_q of quadrant qmap[q] (eps = -1 when the
 * symmetry reflects): s (g b) = phi_s(g) (s b) with
 * phi_s(g)[qmap[q]] = eps * g[q].  Host only, no GPU needed. */
int pp_symmetry_info(int sym, int qmap[4], int* reflects);
/* The packed board s b (each quadrant code must be < 3^9). */
int pp_symmetry_board(uint64_t board, int sym, uint64_t* out);

/* Digest of n super values (no paper counterpart; a verification and
 * streaming aid): adds to d_acc[0] the win bits, to d_acc[1] the not-lose
 * bits, XORs into d_acc[2] an order-independent 64-bit hash of (index,
 * value), adds n to d_acc[3].  d_acc: 4 device uint64, caller-initialised. */
int pp_super_digest(const pp_super* d_values, uint64_t n, uint64_t* d_acc, pp_stream stream);

/* ---- building blocks (exposed for unit tests) ------------------------------ */

/* Rotated five-in-a-row masks (Section "Abstracting over rotations": the set
 * of g in L for which a colour has five in a row in g s).  d_out holds 8
 * uint64 per board: words 0-3 black's mask, 4-7 white's mask, bit beta(g). */
int pp_five_masks(const uint64_t* d_boards, int n, uint64_t* d_out, pp_stream stream);

/* rmax (Section "Abstracting over rotations"): out(g) = OR over the eight
 * single-quadrant quarter turns r of in(g + r), for both tables of each of
 * n super values. */
int pp_rmax(const pp_super* d_in, int n, pp_super* d_out, pp_stream stream);

/* Translation along one quadrant axis: out(g) = in(g + u e_q), both tables,
 * 0 <= q, u <= 3 (the re-indexing of a child whose quadrant q is u turns away
 * from its rotation-minimal representative; Section "Data layout and
 * distribution"). */
int pp_shift(const pp_super* d_in, int n, int q, int u, pp_super* d_out, pp_stream stream);

/* The f_b -> f_{gb} transform for g in G (Section "Abstracting over
 * rotations": cyclic shifts, dimension transpositions and reflections of the
 * 4x4x4x4 tables): out(g) = in(phi_sym(g) + t) for both tables of n super
 * values, t = turns[0..3] (each 0..3).  When in holds f_{c*} for
 * c* = t^{-1} (sym c), out holds f_c. */
int pp_symmetry_transform(const pp_super* d_in, int n, int sym, const int turns[4], pp_super* d_out,
                          pp_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* PENTAGO_GB300_H */
