/*
 * pentago_oracle.c -- a plain, slow CPU statement of the pentago game value.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product library never links or calls it,
 * and it shares no code, table or constant generator with the product.
 *
 * Everything here works on explicit 6x6 boards, one quadrant rotation at a
 * time.  There are no 256-bit tables, no rmax, no precomputed win tables and
 * no standardisation of quadrants: the point is that a reader can check every
 * step against the paper by eye.
 *
 * Game rules (paper, Introduction): a 6x6 board of four 3x3 quadrants; a turn
 * places a stone on an empty cell and then turns one quadrant 90 degrees
 * either way; five in a row by placement wins at once; simultaneous fives, or
 * a full board with no five, is a tie.
 *
 * Value function (paper, Section "Problem definition"):
 *   terminal (f_b(s) or f_w(s) or 36 stones):   v_c(s) = f_c(s) - f_cbar(s)
 *   otherwise  v_c(s) = max over placements a of  1 if f_c(a),
 *                                                 else max over rotations b of a of h_c(b)
 *   h_c(b) = f_c(b) - f_cbar(b) if both colours have five, else -v_cbar(b).
 *
 * Rotation-abstracted value (paper, Section "Abstracting over rotations"):
 * for every g in L = Z4^4 the value of the quadrant-rotated board g s is kept
 * as two bits, "win" (v = 1) and "not lose" (v >= 0).
 *
 * Conventions (the paper leaves them open; the product uses the same ones,
 * written down independently):
 *   - cell (R,C), R,C in 0..5, is index 6R+C; quadrant q = 2*[R>=3] + [C>=3];
 *     local coordinates r = R mod 3, c = C mod 3;
 *   - a board is a uint64: quadrant q occupies bits [16q, 16q+16) and holds
 *     sum over local cells of digit * 3^(3r+c), digit 0 empty, 1 black, 2 white;
 *   - g = (g0,g1,g2,g3), g_q = number of anticlockwise quarter turns of
 *     quadrant q, one turn moving local (r,c) to (2-c, r);
 *   - beta(g) = g0 + 4 g1 + 16 g2 + 64 g3; bit beta of a 256-bit table is
 *     word beta>>6, bit beta&63;
 *   - black moves when the colour counts are equal, white when black has one
 *     more (paper, "Problem definition"); values are from the mover's side.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { EMPTY = 0, BLACK = 1, WHITE = 2 };

enum {
  ORACLE_OK = 0,
  ORACLE_EBOARD = -1,   /* bad digit or impossible colour counts */
  ORACLE_ESIZE = -2,    /* too many empty cells for this routine */
  ORACLE_ENOMEM = -3,
  ORACLE_ECHECK = -4,   /* internal consistency check failed */
};

typedef struct {
  int8_t c[36];
} board_t;

static int pow3(int e) {
  int p = 1;
  while (e-- > 0) p *= 3;
  return p;
}

static int decode(uint64_t packed, board_t* b) {
  for (int q = 0; q < 4; q++) {
    int code = (int)((packed >> (16 * q)) & 0xffff);
    if (code >= 19683) return ORACLE_EBOARD;
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) {
        int digit = (code / pow3(3 * r + c)) % 3;
        int R = 3 * (q >> 1) + r, C = 3 * (q & 1) + c;
        b->c[6 * R + C] = (int8_t)digit;
      }
  }
  return ORACLE_OK;
}

static uint64_t encode(const board_t* b) {
  uint64_t packed = 0;
  for (int q = 0; q < 4; q++) {
    int code = 0;
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) {
        int R = 3 * (q >> 1) + r, C = 3 * (q & 1) + c;
        code += b->c[6 * R + C] * pow3(3 * r + c);
      }
    packed |= (uint64_t)code << (16 * q);
  }
  return packed;
}

/* One anticlockwise quarter turn of quadrant q: local (r,c) -> (2-c, r). */
static void turn_quadrant(board_t* b, int q) {
  int8_t old[3][3];
  int R0 = 3 * (q >> 1), C0 = 3 * (q & 1);
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) old[r][c] = b->c[6 * (R0 + r) + C0 + c];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) b->c[6 * (R0 + 2 - c) + C0 + r] = old[r][c];
}

/* Rotate quadrant q by d quarter turns, d in {+1, -1} (or any integer). */
static void rotate_quadrant(board_t* b, int q, int d) {
  int turns = ((d % 4) + 4) % 4;
  for (int t = 0; t < turns; t++) turn_quadrant(b, q);
}

/* The quadrant-rotated board g s, g given by beta(g). */
static void apply_g(board_t* b, int beta) {
  for (int q = 0; q < 4; q++) rotate_quadrant(b, q, (beta >> (2 * q)) & 3);
}

/* f_c: does colour have five in a row?  Scan every run of five cells along
 * rows, columns and both diagonals. */
static int has_five(const board_t* b, int colour) {
  static const int dir[4][2] = {{0, 1}, {1, 0}, {1, 1}, {1, -1}};
  for (int R = 0; R < 6; R++)
    for (int C = 0; C < 6; C++)
      for (int d = 0; d < 4; d++) {
        int R4 = R + 4 * dir[d][0], C4 = C + 4 * dir[d][1];
        if (R4 < 0 || R4 > 5 || C4 < 0 || C4 > 5) continue;
        int all = 1;
        for (int i = 0; i < 5 && all; i++)
          all = b->c[6 * (R + i * dir[d][0]) + C + i * dir[d][1]] == colour;
        if (all) return 1;
      }
  return 0;
}

static int count_colour(const board_t* b, int colour) {
  int n = 0;
  for (int i = 0; i < 36; i++) n += b->c[i] == colour;
  return n;
}

/* Colour to move, or 0 when the counts are not those of a game position. */
static int mover(const board_t* b) {
  int nb = count_colour(b, BLACK), nw = count_colour(b, WHITE);
  if (nb == nw) return BLACK;
  if (nb == nw + 1) return WHITE;
  return 0;
}

static int other(int colour) { return colour == BLACK ? WHITE : BLACK; }

/* ------------------------------------------------------------------------ */
/* O1: memoised brute-force negamax on explicit boards.                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t* keys; /* packed explicit board + 1; 0 marks an empty slot */
  int8_t* vals;
  size_t cap, used;
} memo_t;

static uint64_t board_key(const board_t* b) {
  uint64_t k = 0;
  for (int i = 35; i >= 0; i--) k = 3 * k + (uint64_t)b->c[i];
  return k + 1;
}

static size_t memo_slot(const memo_t* m, uint64_t key) {
  uint64_t h = key * 0x9E3779B97F4A7C15ull;
  return (size_t)(h >> 20) & (m->cap - 1);
}

static int memo_grow(memo_t* m) {
  memo_t n;
  n.cap = m->cap ? 2 * m->cap : (1u << 16);
  n.used = 0;
  n.keys = (uint64_t*)calloc(n.cap, sizeof(uint64_t));
  n.vals = (int8_t*)calloc(n.cap, 1);
  if (!n.keys || !n.vals) {
    free(n.keys);
    free(n.vals);
    return ORACLE_ENOMEM;
  }
  for (size_t i = 0; i < m->cap; i++)
    if (m->keys[i]) {
      size_t s = memo_slot(&n, m->keys[i]);
      while (n.keys[s]) s = (s + 1) & (n.cap - 1);
      n.keys[s] = m->keys[i];
      n.vals[s] = m->vals[i];
      n.used++;
    }
  free(m->keys);
  free(m->vals);
  *m = n;
  return ORACLE_OK;
}

static int memo_find(const memo_t* m, uint64_t key, int* val) {
  if (!m->cap) return 0;
  size_t s = memo_slot(m, key);
  while (m->keys[s]) {
    if (m->keys[s] == key) {
      *val = m->vals[s];
      return 1;
    }
    s = (s + 1) & (m->cap - 1);
  }
  return 0;
}

static int memo_put(memo_t* m, uint64_t key, int val) {
  if (2 * (m->used + 1) > m->cap && memo_grow(m)) return ORACLE_ENOMEM;
  size_t s = memo_slot(m, key);
  while (m->keys[s] && m->keys[s] != key) s = (s + 1) & (m->cap - 1);
  if (!m->keys[s]) m->used++;
  m->keys[s] = key;
  m->vals[s] = (int8_t)val;
  return ORACLE_OK;
}

/* v_c(s) with c the colour to move in s, following "Problem definition". */
static int negamax(memo_t* memo, const board_t* s, int* err) {
  int c = mover(s), cb = other(c);
  int fc = has_five(s, c), fcb = has_five(s, cb);
  int full = count_colour(s, EMPTY) == 0;
  if (fc || fcb || full) return fc - fcb;
  uint64_t key = board_key(s);
  int cached;
  if (memo_find(memo, key, &cached)) return cached;

  int best = -1;
  for (int p = 0; p < 36 && best < 1; p++) {
    if (s->c[p] != EMPTY) continue;
    board_t a = *s;
    a.c[p] = (int8_t)c;
    if (has_five(&a, c)) { /* placement five: immediate win, no rotation */
      best = 1;
      break;
    }
    for (int q = 0; q < 4 && best < 1; q++)
      for (int d = -1; d <= 1 && best < 1; d += 2) {
        board_t b = a;
        rotate_quadrant(&b, q, d);
        int bc = has_five(&b, c), bcb = has_five(&b, cb);
        int h = (bc && bcb) ? bc - bcb : -negamax(memo, &b, err);
        if (h > best) best = h;
      }
  }
  if (memo_put(memo, key, best)) *err = ORACLE_ENOMEM;
  return best;
}

static void set_bits(uint64_t out[8], int beta, int value) {
  if (value == 1) out[beta >> 6] |= 1ull << (beta & 63);
  if (value >= 0) out[4 + (beta >> 6)] |= 1ull << (beta & 63);
}

/* Super value of one board by brute force, one rotated root at a time.
 * out[0..3] = win table, out[4..7] = not-lose table.  At most max_empty
 * empty cells are accepted (the search is exponential). */
int oracle_brute_force(uint64_t packed, int max_empty, uint64_t out[8]) {
  board_t s;
  memset(out, 0, 8 * sizeof(uint64_t));
  if (decode(packed, &s) || !mover(&s)) return ORACLE_EBOARD;
  if (count_colour(&s, EMPTY) > max_empty) return ORACLE_ESIZE;
  memo_t memo = {0};
  int err = ORACLE_OK;
  for (int beta = 0; beta < 256 && !err; beta++) {
    board_t gs = s;
    apply_g(&gs, beta);
    set_bits(out, beta, negamax(&memo, &gs, &err));
  }
  free(memo.keys);
  free(memo.vals);
  return err;
}

/* ------------------------------------------------------------------------ */
/* O2: rotation-separate retrograde over all fillings of the empty cells.    */
/* ------------------------------------------------------------------------ */
/*
 * This is the serial "midgame" solver of the paper's Section "Open source and
 * data", written without any of its optimisations: every fill of the root's
 * k empty cells and every one of the 256 rotations is a separate explicit
 * board with an int8 value.  Levels are visited from k stones added (full
 * board) down to 0 (the root), so every child value exists when needed.
 *
 * Fill index: the root's empty cells in increasing cell index are slots
 * 0..k-1; slot i holds digit d_i (0 empty, 1 black, 2 white) and the fill
 * index is sum d_i 3^i.  The table is dense, 3^k x 256 int8 (11 GB for the
 * largest accepted k = 16).
 *
 * With check != 0 every child lookup also rebuilds the child board
 * explicitly and verifies that rotating the placed board by (q, d) equals
 * the child fill under rotation g + d e_q.
 *
 * The fills of one level depend only on the level below, so a level's fills
 * may be shared among host threads (each fill is still evaluated by exactly
 * the steps below, by one thread); levels stay in order.
 */
typedef struct {
  board_t root;
  int slot_cell[36], k, first, second, check;
  int8_t* V;
} midgame_t;

/* V[idx][*] for one fill with m stones added; fills of other levels and
 * invalid digit strings are left alone (zero: the table starts cleared). */
static int midgame_fill(const midgame_t* G, int m, int idx) {
  const int k = G->k, first = G->first, second = G->second;
  int8_t* V = G->V;
  int err = ORACLE_OK;
  int digit[36], placed = 0, n_first = 0, n_second = 0;
  for (int i = 0, x = idx; i < k; i++, x /= 3) {
    digit[i] = x % 3;
    placed += digit[i] != EMPTY;
    n_first += digit[i] == first;
    n_second += digit[i] == second;
  }
  /* stones alternate starting with the root's mover */
  if (placed != m || n_first != (m + 1) / 2 || n_second != m / 2) return ORACLE_OK;

  board_t s = G->root;
  for (int i = 0; i < k; i++) s.c[G->slot_cell[i]] = (int8_t)digit[i];
  int c = mover(&s), cb = other(c);

  for (int beta = 0; beta < 256; beta++) {
    board_t B = s;
    apply_g(&B, beta);
    int fc = has_five(&B, c), fcb = has_five(&B, cb);
    int value;
    if (fc || fcb || m == k) {
      value = fc - fcb; /* terminal: a five, or 36 stones */
    } else {
      value = -1;
      for (int i = 0; i < k && value < 1; i++) {
        if (digit[i] != EMPTY) continue;
        /* the move: colour c on root cell slot_cell[i], seen under g */
        board_t child = s;
        child.c[G->slot_cell[i]] = (int8_t)c;
        board_t A = child;
        apply_g(&A, beta);
        if (has_five(&A, c)) {
          value = 1;
          break;
        }
        int child_idx = idx + c * pow3(i);
        for (int q = 0; q < 4; q++)
          for (int d = -1; d <= 1; d += 2) {
            int gq = (beta >> (2 * q)) & 3;
            int beta2 = (beta & ~(3 << (2 * q))) | (((gq + d + 4) & 3) << (2 * q));
            if (G->check) {
              board_t lhs = A, rhs = child;
              rotate_quadrant(&lhs, q, d);
              apply_g(&rhs, beta2);
              if (memcmp(lhs.c, rhs.c, 36)) err = ORACLE_ECHECK;
            }
            int h = -V[(size_t)child_idx * 256 + beta2];
            if (h > value) value = h;
          }
      }
    }
    V[(size_t)idx * 256 + beta] = (int8_t)value;
  }
  return err;
}

/* One level's fills, shared among threads: thread t of n takes the chunks
 * of 4096 consecutive fill indices whose number is t mod n. */
typedef struct {
  const midgame_t* G;
  int m, t, n, err;
} level_part_t;

static void* midgame_level_part(void* arg) {
  level_part_t* P = (level_part_t*)arg;
  const int nfill = pow3(P->G->k), chunk = 4096;
  for (int lo = P->t * chunk; lo < nfill && !P->err; lo += P->n * chunk)
    for (int idx = lo; idx < lo + chunk && idx < nfill && !P->err; idx++)
      P->err = midgame_fill(P->G, P->m, idx);
  return NULL;
}

int oracle_midgame_threads(uint64_t packed, int max_empty, int check, uint64_t out[8],
                           int8_t* all_values, int nthreads) {
  midgame_t G;
  memset(out, 0, 8 * sizeof(uint64_t));
  if (decode(packed, &G.root) || !mover(&G.root)) return ORACLE_EBOARD;
  int k = 0;
  for (int p = 0; p < 36; p++)
    if (G.root.c[p] == EMPTY) G.slot_cell[k++] = p;
  if (k > max_empty || k > 16) return ORACLE_ESIZE;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  G.k = k;
  G.first = mover(&G.root);
  G.second = other(G.first);
  G.check = check;

  size_t nfill = (size_t)pow3(k);
  G.V = (int8_t*)calloc(nfill, 256); /* fills that are no valid position stay 0 */
  if (!G.V) return ORACLE_ENOMEM;
  int err = ORACLE_OK;

  for (int m = k; m >= 0 && !err; m--) {
    level_part_t part[256];
    pthread_t tid[256];
    int running[256] = {0};
    for (int t = 0; t < nthreads; t++) part[t] = (level_part_t){&G, m, t, nthreads, ORACLE_OK};
    for (int t = 1; t < nthreads; t++)
      running[t] = pthread_create(&tid[t], NULL, midgame_level_part, &part[t]) == 0;
    midgame_level_part(&part[0]);
    for (int t = 1; t < nthreads; t++) {
      if (running[t])
        pthread_join(tid[t], NULL);
      else
        midgame_level_part(&part[t]); /* no thread could be started: do it here */
    }
    for (int t = 0; t < nthreads; t++)
      if (part[t].err) err = part[t].err;
  }
  if (!err) {
    for (int beta = 0; beta < 256; beta++) set_bits(out, beta, G.V[beta]);
    if (all_values) memcpy(all_values, G.V, nfill * 256);
  }
  free(G.V);
  return err;
}

int oracle_midgame(uint64_t packed, int max_empty, int check, uint64_t out[8],
                   int8_t* all_values) {
  return oracle_midgame_threads(packed, max_empty, check, out, all_values, 1);
}

/* Many boards, each by oracle_midgame on one thread; thread t of n takes the
 * boards whose number is t mod n.  out holds 8 words per board; the first
 * error met is returned (the other boards are still computed). */
typedef struct {
  const uint64_t* boards;
  int64_t count;
  uint64_t* out;
  int max_empty, t, n, err;
} batch_part_t;

static void* midgame_batch_part(void* arg) {
  batch_part_t* P = (batch_part_t*)arg;
  for (int64_t i = P->t; i < P->count; i += P->n) {
    int rc = oracle_midgame(P->boards[i], P->max_empty, 0, P->out + 8 * i, NULL);
    if (rc && !P->err) P->err = rc;
  }
  return NULL;
}

int oracle_midgame_batch(const uint64_t* boards, int64_t count, int max_empty, uint64_t* out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  batch_part_t part[256];
  pthread_t tid[256];
  int running[256] = {0};
  for (int t = 0; t < nthreads; t++) part[t] = (batch_part_t){boards, count, out, max_empty, t, nthreads, ORACLE_OK};
  for (int t = 1; t < nthreads; t++)
    running[t] = pthread_create(&tid[t], NULL, midgame_batch_part, &part[t]) == 0;
  midgame_batch_part(&part[0]);
  int err = ORACLE_OK;
  for (int t = 1; t < nthreads; t++) {
    if (running[t])
      pthread_join(tid[t], NULL);
    else
      midgame_batch_part(&part[t]);
  }
  for (int t = 0; t < nthreads; t++)
    if (part[t].err && !err) err = part[t].err;
  return err;
}

/* ------------------------------------------------------------------------ */
/* Small explicit helpers exposed for tests.                                 */
/* ------------------------------------------------------------------------ */

/* f_c of the board rotated by beta(g). */
int oracle_has_five(uint64_t packed, int beta, int colour) {
  board_t b;
  if (decode(packed, &b)) return ORACLE_EBOARD;
  apply_g(&b, beta);
  return has_five(&b, colour);
}

/* The board g s, re-encoded. */
uint64_t oracle_rotate(uint64_t packed, int beta) {
  board_t b;
  if (decode(packed, &b)) return ~0ull;
  apply_g(&b, beta);
  return encode(&b);
}

/* Cells of a packed board, 36 digits in cell order 6R+C. */
int oracle_cells(uint64_t packed, int8_t cells[36]) {
  board_t b;
  if (decode(packed, &b)) return ORACLE_EBOARD;
  memcpy(cells, b.c, 36);
  return ORACLE_OK;
}

uint64_t oracle_pack(const int8_t cells[36]) {
  board_t b;
  memcpy(b.c, cells, 36);
  return encode(&b);
}
